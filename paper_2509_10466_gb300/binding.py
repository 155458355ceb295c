"""ctypes binding of ``libinpaint.so`` (the C ABI declared in ``include/inpaint.h``).

Argument marshalling only: every step of the inpainting pass runs in the library's
CUDA kernels.  Functions keep the C names; tensors are passed as raw pointers
(``tensor.data_ptr()``) and the current torch CUDA stream is used unless one is given.
Loading fails loudly if the library has not been built: there is no fallback path.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from .config import ModelConfig

_LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libinpaint.so")
_lib = None

INPAINT_OK, E_INVAL, E_NOMEM, E_CUDA, E_TIMEOUT, E_STATE, E_DEVICE = range(7)
PROFILE_CLASSES = 15
PROFILE_NAMES = ("embed", "layernorm", "qkv_gemm", "attention", "proj_gemm", "fc1_gemm", "fc2_gemm",
                 "decoder1", "decoder2", "head_composite", "other", "proj_mlp_fused", "point_cloud", "splat",
                 "qkv_attention")


class InpaintError(RuntimeError):
    def __init__(self, code: int, what: str):
        self.code = code
        detail = ""
        if code == E_CUDA:
            ce = load().inpaint_last_cuda_error()
            detail = f", {load().inpaint_cuda_error_name(ce).decode()}"
        super().__init__(f"{what}: {strerror(code)} (code {code}{detail})")


class InpaintConfig(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("heads", ctypes.c_int32), ("window", ctypes.c_int32),
                ("blocks", ctypes.c_int32), ("mlp_ratio", ctypes.c_int32), ("patch", ctypes.c_int32),
                ("dec_c1", ctypes.c_int32), ("dec_c2", ctypes.c_int32), ("precision", ctypes.c_int32),
                ("shift", ctypes.c_int32), ("seed", ctypes.c_uint64), ("hbm_budget_bytes", ctypes.c_size_t),
                ("mem_slots", ctypes.c_int32), ("pos_bias", ctypes.c_int32)]

    @classmethod
    def from_model(cls, cfg: ModelConfig, seed: int = 0, hbm_budget_bytes: int = 0) -> "InpaintConfig":
        return cls(cfg.dim, cfg.heads, cfg.window, cfg.blocks, cfg.mlp_ratio, cfg.patch, cfg.dec_c1, cfg.dec_c2,
                   cfg.precision, cfg.shift, seed, hbm_budget_bytes, cfg.mem_slots, cfg.pos_bias)


_P = ctypes.c_void_p
_I = ctypes.c_int
_SIGS = {
    "inpaint_strerror": (ctypes.c_char_p, [_I]),
    "inpaint_memory_bytes": (_I, [_P, _I, _I, _P]),
    "inpaint_point_cloud": (_I, [_P, _P, _P, _I, _I, _P, _P, _P, _P]),
    "inpaint_point_splat": (_I, [_P, _P, ctypes.c_int64, _P, _P, _I, _I, _P, _P, _P, _P]),
    "inpaint_batch_mem": (_I, [_P, _P, ctypes.c_size_t, _P, _P, _I, _I, _I, _P, _P, _P, _P, _P]),
    "inpaint_last_cuda_error": (_I, []),
    "inpaint_cuda_error_name": (ctypes.c_char_p, [_I]),
    "inpaint_num_params": (_I, [ctypes.POINTER(InpaintConfig), ctypes.POINTER(ctypes.c_size_t)]),
    "inpaint_init": (_I, [ctypes.POINTER(InpaintConfig), _P, ctypes.c_size_t, ctypes.POINTER(_P)]),
    "inpaint_set_weights": (_I, [_P, _P, _I, _P]),
    "inpaint_get_weights": (_I, [_P, _P]),
    "inpaint_workspace_bytes": (_I, [_P, _I, _I, _I, ctypes.POINTER(ctypes.c_size_t)]),
    "inpaint_frame": (_I, [_P, _P, _P, _I, _I, _P, _P]),
    "inpaint_batch": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P]),
    "inpaint_batch_ws": (_I, [_P, _P, ctypes.c_size_t, _P, _P, _I, _I, _I, _P, _P, _P]),
    "inpaint_batch_host": (_I, [_P, _P, _P, _I, _I, _I, _P, _P]),
    "inpaint_token_masks": (_I, [_P, _P, ctypes.c_size_t]),
    "inpaint_fullres": (_I, [_P, _P, _P, _P, _I, _I, _I, _I, _P, _P, _P]),
    "inpaint_l1_hole_loss": (_I, [_P, _P, _P, _P, _I, _I, _I, _P, _P, _P]),
    "inpaint_l1_hole_loss_noalloc": (_I, [_P, _P, _P, _I, _I, _I, _P, _P, _P]),
    "inpaint_backward": (_I, [_P, _P, _P, _P, _I, _I, _I, _P, _P]),
    "inpaint_sync": (_I, [_P, _P, _I]),
    "inpaint_profile_enable": (_I, [_P, _I]),
    "inpaint_profile_read": (_I, [_P, _P, _P]),
    "inpaint_launch_count": (_I, [_P, ctypes.POINTER(ctypes.c_int64)]),
    "inpaint_destroy": (None, [_P]),
    "inpaint_test_gemm_bf16": (_I, [_P, _P, _P, _I, _I, _I, _P]),
    "inpaint_test_gelu": (_I, [_P, _P, _P, _I, _P]),
    "inpaint_test_gelu_h16": (_I, [_P, _P, _I, _P]),
    "inpaint_train_step": (_I, [_P, _P, _P, _P, _I, _I, _I, _P, _P, _P, _P]),
    "inpaint_test_wait_expiry": (_I, [_P, _I, _P]),
    "inpaint_default_weights": (_I, [ctypes.POINTER(InpaintConfig), ctypes.c_uint64, _P, ctypes.c_size_t]),
}


def lib_path() -> str:
    return _LIB_PATH


def load():
    """Load libinpaint.so and declare its signatures (raises if it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(_LIB_PATH):
            raise RuntimeError(f"{_LIB_PATH} is missing: build it with paper_2509_10466_gb300.build.build()")
        lib = ctypes.CDLL(_LIB_PATH)
        for name, (res, args) in _SIGS.items():
            fn = getattr(lib, name)
            fn.restype = res
            fn.argtypes = args
        _lib = lib
    return _lib


def declared_symbols():
    return list(_SIGS)


def strerror(code: int) -> str:
    return load().inpaint_strerror(code).decode()


def _check(code: int, what: str):
    if code != INPAINT_OK:
        raise InpaintError(code, what)


def _stream(stream):
    if stream is None:
        import torch
        return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    if hasattr(stream, "cuda_stream"):
        return ctypes.c_void_p(stream.cuda_stream)
    return ctypes.c_void_p(int(stream))


def _ptr(t):
    """Raw pointer of a tensor; the C ABI reads dense row-major memory, so strided views are refused."""
    if t is None:
        return None
    if not t.is_contiguous():
        raise ValueError("tensors passed to libinpaint must be contiguous (call .contiguous() first)")
    return ctypes.c_void_p(t.data_ptr())


# ----------------------------------------------------------------------------- same-name wrappers

def inpaint_num_params(cfg: ModelConfig) -> int:
    n = ctypes.c_size_t()
    c = InpaintConfig.from_model(cfg)
    _check(load().inpaint_num_params(ctypes.byref(c), ctypes.byref(n)), "inpaint_num_params")
    return n.value


def inpaint_init(cfg: ModelConfig, weights, seed: int = 0, hbm_budget_bytes: int = 0):
    """weights: a float32 blob, or None for the library's default blob of `seed`."""
    c = InpaintConfig.from_model(cfg, seed, hbm_budget_bytes)
    ctx = ctypes.c_void_p()
    if weights is None:
        _check(load().inpaint_init(ctypes.byref(c), None, 0, ctypes.byref(ctx)), "inpaint_init")
        return ctx
    w = np.ascontiguousarray(weights, dtype=np.float32)
    _check(load().inpaint_init(ctypes.byref(c), w.ctypes.data_as(ctypes.c_void_p), w.size, ctypes.byref(ctx)),
           "inpaint_init")
    return ctx


def inpaint_default_weights(cfg: ModelConfig, seed: int = 0) -> np.ndarray:
    """The library's default weight blob of `seed` (host code; no GPU needed)."""
    n = inpaint_num_params(cfg)
    out = np.empty(n, np.float32)
    c = InpaintConfig.from_model(cfg, seed)
    _check(load().inpaint_default_weights(ctypes.byref(c), seed, out.ctypes.data_as(ctypes.c_void_p), n),
           "inpaint_default_weights")
    return out


def inpaint_destroy(ctx):
    load().inpaint_destroy(ctx)


def inpaint_set_weights(ctx, weights, stream=None):
    """weights: a CUDA float32 tensor (device update on the stream) or a numpy array (host)."""
    if isinstance(weights, np.ndarray):
        w = np.ascontiguousarray(weights, dtype=np.float32)
        _check(load().inpaint_set_weights(ctx, w.ctypes.data_as(ctypes.c_void_p), 0, _stream(stream)),
               "inpaint_set_weights")
    else:
        _check(load().inpaint_set_weights(ctx, _ptr(weights), 1, _stream(stream)), "inpaint_set_weights")


def inpaint_get_weights(ctx, n: int) -> np.ndarray:
    out = np.empty(n, np.float32)
    _check(load().inpaint_get_weights(ctx, out.ctypes.data_as(ctypes.c_void_p)), "inpaint_get_weights")
    return out


def inpaint_workspace_bytes(ctx, B: int, H: int, W: int) -> int:
    n = ctypes.c_size_t()
    _check(load().inpaint_workspace_bytes(ctx, B, H, W, ctypes.byref(n)), "inpaint_workspace_bytes")
    return n.value


def inpaint_frame(ctx, x, hole, out, stream=None):
    _, H, W = hole.shape
    _check(load().inpaint_frame(ctx, _ptr(x), _ptr(hole), H, W, _ptr(out), _stream(stream)), "inpaint_frame")


def inpaint_batch(ctx, x, hole, out, pred=None, stream=None):
    B, H, W = hole.shape
    _check(load().inpaint_batch(ctx, _ptr(x), _ptr(hole), B, H, W, _ptr(out), _ptr(pred), _stream(stream)),
           "inpaint_batch")


def inpaint_memory_bytes(ctx, H: int, W: int) -> int:
    n = ctypes.c_size_t(0)
    _check(load().inpaint_memory_bytes(ctx, H, W, ctypes.byref(n)), "inpaint_memory_bytes")
    return n.value


def inpaint_batch_mem(ctx, x, hole, out, mem_in, mem_out, pred=None, stream=None, workspace=None):
    """mem_in: list over frames of lists of m device buffers (uint8 CUDA tensors) or None;
    mem_out: list over frames of a device buffer or None; workspace: None (the context's)
    or a uint8 CUDA tensor of at least inpaint_workspace_bytes."""
    B, H, W = hole.shape
    nbytes = 0 if workspace is None else workspace.numel() * workspace.element_size()
    tab_in = None
    if mem_in is not None:
        flat = [None if t is None else _ptr(t).value for slots in mem_in for t in slots]
        tab_in = (ctypes.c_void_p * len(flat))(*flat)
    tab_out = None
    if mem_out is not None:
        tab_out = (ctypes.c_void_p * B)(*[None if t is None else _ptr(t).value for t in mem_out])
    _check(load().inpaint_batch_mem(ctx, _ptr(workspace), nbytes, _ptr(x), _ptr(hole), B, H, W, _ptr(out), _ptr(pred),
                                    tab_in, tab_out, _stream(stream)), "inpaint_batch_mem")


def _host_f32(vals, n):
    a = (ctypes.c_float * n)(*[float(v) for v in np.asarray(vals, dtype=np.float64).reshape(-1)])
    return a


def inpaint_point_cloud(ctx, depth, rgb, cam, R, t, points, stream=None):
    """depth [H, W], rgb [3, H, W] and points [H*W, 6] are float32 CUDA tensors; cam =
    (fx, fy, cx, cy); R [3, 3] and t [3] map camera points to the world."""
    H, W = depth.shape
    rt = np.concatenate([np.asarray(R, np.float64).reshape(9), np.asarray(t, np.float64).reshape(3)])
    _check(load().inpaint_point_cloud(ctx, _ptr(depth), _ptr(rgb), H, W, _host_f32(cam, 4), _host_f32(rt, 12),
                                      _ptr(points), _stream(stream)), "inpaint_point_cloud")


def inpaint_point_splat(ctx, points, view, R, t, img, depth_out=None, index_out=None, stream=None):
    """points [N, 6]; img [3, Ho, Wo]; depth_out [Ho, Wo] float32; index_out [Ho, Wo] int32."""
    _, Ho, Wo = img.shape
    rt = np.concatenate([np.asarray(R, np.float64).reshape(9), np.asarray(t, np.float64).reshape(3)])
    _check(load().inpaint_point_splat(ctx, _ptr(points), points.shape[0], _host_f32(view, 4), _host_f32(rt, 12), Ho,
                                      Wo, _ptr(img), _ptr(depth_out), _ptr(index_out), _stream(stream)),
           "inpaint_point_splat")


def inpaint_batch_ws(ctx, workspace, x, hole, out, pred=None, stream=None):
    B, H, W = hole.shape
    nbytes = workspace.numel() * workspace.element_size()
    _check(load().inpaint_batch_ws(ctx, _ptr(workspace), nbytes, _ptr(x), _ptr(hole), B, H, W, _ptr(out),
                                   _ptr(pred), _stream(stream)), "inpaint_batch_ws")


def inpaint_batch_host(ctx, x: np.ndarray | object, hole, out, stream=None):
    """Host buffers (pinned torch CPU tensors or numpy arrays); blocks until `out` is filled."""
    B, H, W = hole.shape

    def hp(a):
        return ctypes.c_void_p(a.ctypes.data) if isinstance(a, np.ndarray) else ctypes.c_void_p(a.data_ptr())

    _check(load().inpaint_batch_host(ctx, hp(x), hp(hole), B, H, W, hp(out), _stream(stream)), "inpaint_batch_host")


def inpaint_fullres(ctx, x, obj_masks, selected, out, hole_half=None, stream=None):
    """Full-resolution frames -> half-resolution inpainting -> x2 upscaled composite (see inpaint.h)."""
    B, _, H, W = x.shape
    K = obj_masks.shape[1]
    _check(load().inpaint_fullres(ctx, _ptr(x), _ptr(obj_masks), _ptr(selected), B, K, H, W, _ptr(out),
                                  _ptr(hole_half), _stream(stream)), "inpaint_fullres")


def inpaint_token_masks(ctx, blocks: int, B: int, Ntok: int) -> np.ndarray:
    out = np.empty(((blocks + 1), B, Ntok), np.uint8)
    _check(load().inpaint_token_masks(ctx, out.ctypes.data_as(ctypes.c_void_p), out.size), "inpaint_token_masks")
    return out


def inpaint_l1_hole_loss(ctx, out, target, hole, loss, grad_out=None, stream=None):
    B, H, W = hole.shape
    _check(load().inpaint_l1_hole_loss(ctx, _ptr(out), _ptr(target), _ptr(hole), B, H, W, _ptr(loss),
                                       _ptr(grad_out), _stream(stream)), "inpaint_l1_hole_loss")


def inpaint_l1_hole_loss_noalloc(out, target, hole, loss, grad_out=None, stream=None):
    """Hole-L1 loss that allocates no device memory (fixed library scratch; see inpaint.h)."""
    B, H, W = hole.shape
    _check(load().inpaint_l1_hole_loss_noalloc(_ptr(out), _ptr(target), _ptr(hole), B, H, W, _ptr(loss),
                                               _ptr(grad_out), _stream(stream)), "inpaint_l1_hole_loss_noalloc")


def inpaint_backward(ctx, x, hole, grad_out, grad_weights, stream=None):
    B, H, W = hole.shape
    _check(load().inpaint_backward(ctx, _ptr(x), _ptr(hole), _ptr(grad_out), B, H, W, _ptr(grad_weights),
                                   _stream(stream)), "inpaint_backward")


def inpaint_sync(ctx, stream=None, timeout_ms: int = -1) -> int:
    """Returns the status code (0, E_TIMEOUT or E_DEVICE) instead of raising for those two."""
    code = load().inpaint_sync(ctx, _stream(stream), timeout_ms)
    if code not in (INPAINT_OK, E_TIMEOUT, E_DEVICE):
        _check(code, "inpaint_sync")
    return code


def inpaint_profile_enable(ctx, on: bool):
    _check(load().inpaint_profile_enable(ctx, 1 if on else 0), "inpaint_profile_enable")


def inpaint_profile_read(ctx):
    ms = (ctypes.c_float * PROFILE_CLASSES)()
    n = (ctypes.c_int64 * PROFILE_CLASSES)()
    _check(load().inpaint_profile_read(ctx, ms, n), "inpaint_profile_read")
    return {PROFILE_NAMES[i]: (float(ms[i]), int(n[i])) for i in range(PROFILE_CLASSES)}


def inpaint_launch_count(ctx) -> int:
    n = ctypes.c_int64()
    _check(load().inpaint_launch_count(ctx, ctypes.byref(n)), "inpaint_launch_count")
    return n.value


def inpaint_test_gemm_bf16(A, Bt, C, stream=None):
    M, K = A.shape
    N = Bt.shape[0]
    _check(load().inpaint_test_gemm_bf16(_ptr(A), _ptr(Bt), _ptr(C), M, N, K, _stream(stream)),
           "inpaint_test_gemm_bf16")


def inpaint_test_wait_expiry(ctx, limit_us: int, stream=None):
    _check(load().inpaint_test_wait_expiry(ctx, limit_us, _stream(stream)), "inpaint_test_wait_expiry")


def inpaint_train_step(ctx, x, hole, target, loss, grad_weights, out=None, stream=None):
    """Forward + hole-L1 loss + weight gradient in one call (device tensors)."""
    B, H, W = hole.shape
    _check(load().inpaint_train_step(ctx, _ptr(x), _ptr(hole), _ptr(target), B, H, W, _ptr(loss),
                                     _ptr(grad_weights), _ptr(out) if out is not None else None, _stream(stream)),
           "inpaint_train_step")


def inpaint_test_gelu_h16(x, y, stream=None):
    _check(load().inpaint_test_gelu_h16(_ptr(x), _ptr(y), x.numel(), _stream(stream)), "inpaint_test_gelu_h16")


def inpaint_test_gelu(x, y_bf16_form, y_fp32_form, stream=None):
    _check(load().inpaint_test_gelu(_ptr(x), _ptr(y_bf16_form), _ptr(y_fp32_form), x.numel(), _stream(stream)),
           "inpaint_test_gelu")


# ----------------------------------------------------------------------------- convenience object

class Inpainter:
    """Owns one library context; methods take torch CUDA tensors."""

    def __init__(self, cfg: ModelConfig, weights, hbm_budget_bytes: int = 0, seed: int = 0):
        """weights: a float32 blob, or None for the library's default blob of `seed`."""
        self.cfg = cfg
        self.n_params = inpaint_num_params(cfg)
        self.ctx = inpaint_init(cfg, weights, seed=seed, hbm_budget_bytes=hbm_budget_bytes)

    def close(self):
        if self.ctx is not None:
            inpaint_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __call__(self, x, hole, want_pred: bool = False, stream=None):
        import torch
        out = torch.empty_like(x)
        pred = torch.empty_like(x) if want_pred else None
        inpaint_batch(self.ctx, x, hole, out, pred, stream)
        return (out, pred) if want_pred else out

    def memory_buffer(self, H: int, W: int):
        """A fresh device buffer for one frame's memory tensor (256-byte aligned)."""
        import torch
        n = inpaint_memory_bytes(self.ctx, H, W)
        return torch.empty(max(n, 1), dtype=torch.uint8, device="cuda")

    def with_memory(self, x, hole, mem_in, mem_out, want_pred: bool = False, stream=None):
        import torch
        out = torch.empty_like(x)
        pred = torch.empty_like(x) if want_pred else None
        inpaint_batch_mem(self.ctx, x, hole, out, mem_in, mem_out, pred, stream)
        return (out, pred) if want_pred else out

    def token_masks(self, B: int, H: int, W: int) -> np.ndarray:
        mult = self.cfg.patch * self.cfg.window
        Ht = -(-H // mult) * mult // self.cfg.patch
        Wt = -(-W // mult) * mult // self.cfg.patch
        return inpaint_token_masks(self.ctx, self.cfg.blocks, B, Ht * Wt)
