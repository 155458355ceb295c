"""CPU oracle of the point-cloud recolouring and headless point splat.

TEST INFRASTRUCTURE ONLY.  Only the test suite and bench.py's CPU legs may import or call
this module; the product path never does, and this module imports nothing from it.

What it computes, in the paper's terms: the inpainted frame's RGB values are
transplanted onto the depth measurements to form a coloured point cloud (Section
"Point Cloud Visualisation"); points are mapped from the camera's space into the
viewer's world by the rigid transform p' = R p + t (Section "Perspective Alignment",
with the calibration chain that produces R and t); the paper then renders the cloud with
OpenGL, which this path replaces by a z-buffered point splat into an image buffer at a
remote viewpoint.  Readings used here (the paper gives no camera model or raster rule):

* pinhole camera with intrinsics (fx, fy, cx, cy); pixel (row v, column u) has its
  centre at (u + 0.5, v + 0.5); depth d > 0 and finite is valid, anything else is not;
* back-projection: x = d (u + 0.5 - cx) / fx, y = d (v + 0.5 - cy) / fy, z = d;
* world point = R p + t, each component summed as ((r0 x + r1 y) + r2 z) + t;
* viewer: q = Rv w + tv (same order); visible if q_z > 1e-3; projected column
  u' = fx' (q_x / q_z) + cx' and row v' = fy' (q_y / q_z) + cy'; the point covers pixel
  (floor(v'), floor(u')) if that lies inside the Ho x Wo image;
* z-buffer: per pixel the point with the smallest q_z wins, ties to the smaller source
  index (row-major pixel index of the frame); empty pixels are colour 0, depth +inf,
  index -1.

The projection decides integers (the pixel and the winner), so it is evaluated in
float32 with every product, sum and quotient rounded separately, in the order above -
the same arithmetic the CUDA path uses - while the rest is plain numpy.
"""
from __future__ import annotations

import numpy as np

F32 = np.float32
NEAR = F32(1e-3)


def _rigid(R, t, x, y, z):
    """Rows of R applied to (x, y, z) plus t, float32, ((r0 x + r1 y) + r2 z) + t."""
    R = np.asarray(R, F32).reshape(3, 3)
    t = np.asarray(t, F32).reshape(3)
    out = []
    for k in range(3):
        a = R[k, 0] * x
        b = R[k, 1] * y
        c = R[k, 2] * z
        out.append(((a + b) + c) + t[k])
    return out


def point_cloud(depth, rgb, cam, R, t):
    """depth [H, W], rgb [3, H, W], cam (fx, fy, cx, cy) -> points [H*W, 6] (x, y, z, r, g, b)
    in world space; invalid pixels have NaN coordinates."""
    depth = np.asarray(depth, F32)
    H, W = depth.shape
    fx, fy, cx, cy = (F32(c) for c in cam)
    v, u = np.meshgrid(np.arange(H, dtype=F32), np.arange(W, dtype=F32), indexing="ij")
    su = (u + F32(0.5)) - cx
    sv = (v + F32(0.5)) - cy
    x = (depth * su) / fx
    y = (depth * sv) / fy
    z = depth
    wx, wy, wz = _rigid(R, t, x, y, z)
    valid = np.isfinite(depth) & (depth > 0)
    pts = np.empty((H * W, 6), F32)
    for k, a in enumerate((wx, wy, wz)):
        pts[:, k] = np.where(valid, a, F32(np.nan)).reshape(-1)
    for c in range(3):
        pts[:, 3 + c] = np.asarray(rgb, F32)[c].reshape(-1)
    return pts


def splat(points, view, Rv, tv, Ho, Wo):
    """points [N, 6] -> image [3, Ho, Wo], depth [Ho, Wo] (+inf empty), index [Ho, Wo] (-1 empty)."""
    pts = np.asarray(points, F32)
    fx, fy, cx, cy = (F32(c) for c in view)
    ok = np.isfinite(pts[:, 0]) & np.isfinite(pts[:, 1]) & np.isfinite(pts[:, 2])
    qx, qy, qz = _rigid(Rv, tv, pts[:, 0], pts[:, 1], pts[:, 2])
    with np.errstate(invalid="ignore", divide="ignore", over="ignore"):
        ok &= qz > NEAR
        up = fx * (qx / qz) + cx
        vp = fy * (qy / qz) + cy
        ok &= np.isfinite(up) & np.isfinite(vp)
        ok &= (up >= 0) & (up < F32(Wo)) & (vp >= 0) & (vp < F32(Ho))
    idx = np.nonzero(ok)[0]
    col = np.floor(up[idx]).astype(np.int64)
    row = np.floor(vp[idx]).astype(np.int64)
    pix = row * Wo + col
    order = np.lexsort((idx, qz[idx], pix))         # by pixel, then depth, then index
    pix_o, idx_o = pix[order], idx[order]
    first = np.ones(len(pix_o), bool)
    first[1:] = pix_o[1:] != pix_o[:-1]
    win_pix, win_idx = pix_o[first], idx_o[first]
    img = np.zeros((3, Ho * Wo), F32)
    dep = np.full(Ho * Wo, np.inf, F32)
    ind = np.full(Ho * Wo, -1, np.int32)
    img[:, win_pix] = pts[win_idx, 3:6].T
    dep[win_pix] = qz[win_idx]
    ind[win_pix] = win_idx.astype(np.int32)
    return img.reshape(3, Ho, Wo), dep.reshape(Ho, Wo), ind.reshape(Ho, Wo)


def zed_pose(R_head, t_head, R_zedbox, p_zedbox, R_head_now, t_head_now):
    """The paper's calibration chain: the virtual ZED box's pose relative to the headset at
    calibration, then the ZED camera's pose in the world for the headset's current pose.
    Returns (R_zed, t_zed) with p_world = R_zed p_zed + t_zed."""
    R_head, R_zedbox, R_head_now = (np.asarray(a, np.float64).reshape(3, 3) for a in (R_head, R_zedbox, R_head_now))
    t_head, p_zedbox, t_head_now = (np.asarray(a, np.float64).reshape(3) for a in (t_head, p_zedbox, t_head_now))
    R_inv = np.linalg.inv(R_head)
    p_zed_in_head = R_inv @ (p_zedbox - t_head)
    R_zed_in_head = R_inv @ R_zedbox
    t_zed = R_head_now @ p_zed_in_head + t_head_now
    R_zed = R_head_now @ R_zed_in_head
    return R_zed, t_zed
