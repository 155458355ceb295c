"""The C-ABI library builds, loads without a GPU and exports what include/inpaint.h declares."""
import ctypes
import os
import re

import pytest

from oracle import inpaint_oracle as O
from paper_2509_10466_gb300 import binding, build as B, synthetic as S
from paper_2509_10466_gb300.config import ModelConfig, WORKLOADS


@pytest.fixture(scope="module")
def lib():
    B.build()
    return binding.load()


def header_functions(root):
    text = open(os.path.join(root, "include", "inpaint.h")).read()
    return sorted(set(re.findall(r"INPAINT_API\s+[\w\s\*]+?\b(inpaint_\w+)\s*\(", text)))


def test_header_declares_the_entry_points(repo_root):
    names = header_functions(repo_root)
    for must in ("inpaint_init", "inpaint_frame", "inpaint_batch", "inpaint_backward", "inpaint_l1_hole_loss",
                 "inpaint_num_params", "inpaint_token_masks", "inpaint_sync", "inpaint_destroy", "inpaint_strerror"):
        assert must in names


def test_library_exports_every_declared_symbol(lib, repo_root):
    for name in header_functions(repo_root):
        assert hasattr(lib, name), name
    assert sorted(binding.declared_symbols()) == header_functions(repo_root)


def test_library_has_no_driver_link_dependency():
    # loads on a machine without libcuda: the driver API is resolved at run time
    ctypes.CDLL(binding.lib_path())


@pytest.mark.parametrize("name", sorted(WORKLOADS))
def test_num_params_matches_blob_format(lib, name):
    cfg = WORKLOADS[name].model
    assert binding.inpaint_num_params(cfg) == S.num_params(cfg) == O.num_params(cfg)


@pytest.mark.parametrize("bad", [dict(window=4), dict(patch=2), dict(dim=96, heads=2), dict(heads=3),
                                 dict(precision=3), dict(dim=96, heads=3, precision=1),
                                 dict(dim=96, heads=3, precision=2), dict(mlp_ratio=0)])
def test_invalid_configs_are_rejected(lib, bad):
    cfg = ModelConfig(**{**dict(dim=128, heads=4, window=8, blocks=2, mlp_ratio=2), **bad})
    with pytest.raises(binding.InpaintError) as e:
        binding.inpaint_num_params(cfg)
    assert e.value.code == binding.E_INVAL


def test_strerror_covers_codes(lib):
    for code in range(7):
        assert binding.strerror(code) and "unknown" not in binding.strerror(code)
    assert "unknown" in binding.strerror(99)


@pytest.mark.parametrize("name,seed", [("plain_fp32_256", 0), ("fd_64", 7), ("precision_512", 123456789)])
def test_default_weights_match_the_documented_generator(lib, name, seed):
    # the C library's host generator against the numpy restatement of the documented
    # counter-based stream (SplitMix64 output function, Box-Muller in FP64); libm and
    # numpy may differ in the last bit of log / cos, so one float32 ulp is allowed
    import numpy as np
    cfg = WORKLOADS[name].model
    c_blob = binding.inpaint_default_weights(cfg, seed)
    py_blob = S.default_weights(cfg, seed)
    assert c_blob.shape == py_blob.shape
    ulp = np.spacing(np.abs(py_blob).astype(np.float32))
    assert np.all(np.abs(c_blob - py_blob) <= ulp)


def test_default_weights_layout_and_distribution(lib):
    import numpy as np
    from scipy import stats
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=2, mlp_ratio=2, pos_bias=1)
    w = binding.inpaint_default_weights(cfg, 3)
    at = 0
    for nm, shape in S.param_shapes(cfg):
        n = int(np.prod(shape))
        a = w[at:at + n]
        leaf = nm.rsplit(".", 1)[1]
        if leaf in ("w", "relpos"):
            assert a.std() > 0
        elif (".ln" in nm or nm.startswith("ln")) and leaf == "g":
            assert np.all(a == 1.0)
        else:
            assert np.all(a == 0.0)
        at += n
    assert at == w.size
    # the matrices together are N(0, 0.02): Kolmogorov-Smirnov against the normal law
    mats = np.concatenate([w[o:o + int(np.prod(s))] for o, (nm, s) in
                           zip(np.cumsum([0] + [int(np.prod(s)) for _, s in S.param_shapes(cfg)])[:-1],
                               S.param_shapes(cfg)) if nm.endswith(".w")])
    assert stats.kstest(mats / 0.02, "norm").pvalue > 1e-3
    # different seeds give different blobs, the same seed the same one
    assert not np.array_equal(w, binding.inpaint_default_weights(cfg, 4))
    assert np.array_equal(w, binding.inpaint_default_weights(cfg, 3))
