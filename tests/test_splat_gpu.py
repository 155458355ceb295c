"""Point cloud and z-buffered splat on the GPU against the CPU oracle: bit-exact point
buffers, images, depths and winning indices (the projection decides integers, and both
sides evaluate it in float32 with the same rounding order)."""
import numpy as np
import pytest
import torch

from oracle import splat_oracle as P
from paper_2509_10466_gb300 import binding, synthetic as S
from paper_2509_10466_gb300.config import BF16, ModelConfig

from helpers import lib
from test_oracle_splat import rot, scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    lib()
    cfg = ModelConfig(dim=64, heads=2, window=8, blocks=1, mlp_ratio=2, precision=BF16)
    inp = binding.Inpainter(cfg, S.make_weights(cfg, seed=0))
    yield inp.ctx
    inp.close()


def gpu_cloud_and_splat(ctx, depth, rgb, cam, R, t, view, Rv, tv, Ho, Wo):
    H, W = depth.shape
    d = torch.from_numpy(depth).cuda()
    c = torch.from_numpy(rgb).cuda()
    pts = torch.empty(H * W, 6, device="cuda")
    binding.inpaint_point_cloud(ctx, d, c, cam, R, t, pts)
    img = torch.full((3, Ho, Wo), 7.0, device="cuda")
    dep = torch.empty(Ho, Wo, device="cuda")
    ind = torch.empty(Ho, Wo, dtype=torch.int32, device="cuda")
    binding.inpaint_point_splat(ctx, pts, view, Rv, tv, img, dep, ind)
    torch.cuda.synchronize()
    return pts.cpu().numpy(), img.cpu().numpy(), dep.cpu().numpy(), ind.cpu().numpy()


def check(ctx, depth, rgb, cam, R, t, view, Rv, tv, Ho, Wo):
    g = gpu_cloud_and_splat(ctx, depth, rgb, cam, R, t, view, Rv, tv, Ho, Wo)
    pts = P.point_cloud(depth, rgb, cam, R, t)
    r = (pts,) + P.splat(pts, view, Rv, tv, Ho, Wo)
    np.testing.assert_array_equal(g[0], r[0])          # NaN positions compare equal too
    for a, b in zip(g[1:], r[1:]):
        np.testing.assert_array_equal(a, b)
    return g


@pytest.mark.parametrize("H,W,Ho,Wo,seed", [(48, 64, 48, 64, 1), (37, 53, 61, 29, 2), (120, 200, 90, 160, 3)])
def test_cloud_and_splat_match_the_oracle_bit_for_bit(ctx, H, W, Ho, Wo, seed):
    depth, rgb = scene(H, W, seed)
    cam = (0.8 * W, 0.8 * W, W / 2 - 0.3, H / 2 + 0.2)
    view = (0.7 * Wo, 0.7 * Wo, Wo / 2, Ho / 2)
    R, t = rot(0.05, -0.1, 0.02), np.array([0.1, -0.05, 0.2])
    Rv, tv = rot(-0.02, 0.15, 0.0), np.array([-0.2, 0.0, 0.3])
    g = check(ctx, depth, rgb, cam, R, t, view, Rv, tv, Ho, Wo)
    assert (g[3] >= 0).sum() > 0.2 * Ho * Wo           # the view is substantially covered


def test_identity_round_trip_on_the_gpu(ctx):
    depth, rgb = scene(72, 128, 4)
    cam = (100.0, 100.0, 64.0, 36.0)
    _, img, dep, ind = check(ctx, depth, rgb, cam, np.eye(3), np.zeros(3), cam, np.eye(3), np.zeros(3), 72, 128)
    valid = np.isfinite(depth) & (depth > 0)
    assert np.array_equal(img[:, valid], rgb[:, valid])


def test_720p_frame_sampled_against_the_oracle(ctx):
    """A 1280x720 frame splatted to a rotated 1280x720 view; the whole output is compared."""
    depth, rgb = scene(720, 1280, 5)
    cam = (900.0, 900.0, 640.0, 360.0)
    check(ctx, depth, rgb, cam, rot(0.01, 0.02, 0.0), np.array([0.0, 0.0, 0.0]), cam, rot(0.0, -0.08, 0.01),
          np.array([0.15, 0.02, 0.1]), 720, 1280)


def test_edge_cases(ctx):
    # no usable depth at all: an empty image
    depth = np.zeros((16, 16), np.float32)
    rgb = np.ones((3, 16, 16), np.float32)
    cam = (10.0, 10.0, 8.0, 8.0)
    _, img, dep, ind = check(ctx, depth, rgb, cam, np.eye(3), np.zeros(3), cam, np.eye(3), np.zeros(3), 16, 16)
    assert np.all(ind == -1) and np.all(img == 0) and np.all(np.isinf(dep))
    # everything behind the viewer
    depth = np.full((16, 16), 2.0, np.float32)
    _, img, dep, ind = check(ctx, depth, rgb, cam, np.eye(3), np.zeros(3), cam, np.eye(3), np.array([0, 0, -5.0]),
                             16, 16)
    assert np.all(ind == -1)
    # zero points and invalid arguments
    img = torch.zeros(3, 8, 8, device="cuda")
    binding.inpaint_point_splat(ctx, torch.empty(0, 6, device="cuda"), cam, np.eye(3), np.zeros(3), img)
    torch.cuda.synchronize()
    assert float(img.abs().sum()) == 0
    with pytest.raises(binding.InpaintError):
        binding.inpaint_point_cloud(ctx, torch.zeros(4, 4, device="cuda"), torch.zeros(3, 4, 4, device="cuda"),
                                    (0.0, 1.0, 0.0, 0.0), np.eye(3), np.zeros(3), torch.empty(16, 6, device="cuda"))
