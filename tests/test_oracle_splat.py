"""Pins of the point-cloud / splat oracle (CPU only): a closed-form round trip, a hand-made
z-test, a closed-form projection under an axial translation, and the paper's pose chain."""
import numpy as np

from oracle import splat_oracle as P

F32 = np.float32


def rot(ax, ay, az):
    cx, sx, cy, sy, cz, sz = np.cos(ax), np.sin(ax), np.cos(ay), np.sin(ay), np.cos(az), np.sin(az)
    Rx = np.array([[1, 0, 0], [0, cx, -sx], [0, sx, cx]])
    Ry = np.array([[cy, 0, sy], [0, 1, 0], [-sy, 0, cy]])
    Rz = np.array([[cz, -sz, 0], [sz, cz, 0], [0, 0, 1]])
    return Rz @ Ry @ Rx


def scene(H, W, seed):
    rng = np.random.default_rng(seed)
    depth = rng.uniform(0.5, 5.0, (H, W)).astype(F32)
    depth[rng.random((H, W)) < 0.1] = 0
    depth[rng.random((H, W)) < 0.05] = np.nan
    rgb = rng.random((3, H, W)).astype(F32)
    return depth, rgb


def test_identity_views_reproduce_the_frame():
    """Same camera, identity transforms: every point lands on its own pixel."""
    H, W = 24, 40
    depth, rgb = scene(H, W, 1)
    cam = (30.0, 28.0, 19.5, 11.0)
    pts = P.point_cloud(depth, rgb, cam, np.eye(3), np.zeros(3))
    img, dep, ind = P.splat(pts, cam, np.eye(3), np.zeros(3), H, W)
    valid = np.isfinite(depth) & (depth > 0)
    assert np.array_equal(ind[valid], np.nonzero(valid.reshape(-1))[0].astype(np.int32))
    assert np.all(ind[~valid] == -1)
    assert np.array_equal(img[:, valid], rgb[:, valid]) and np.all(img[:, ~valid] == 0)
    assert np.array_equal(dep[valid], depth[valid]) and np.all(np.isinf(dep[~valid]))


def test_nearer_point_wins_and_equal_depths_go_to_the_lower_index():
    view = (10.0, 10.0, 2.0, 2.0)
    # four points on the optical axis of pixel (2, 2) and one elsewhere
    pts = np.array([[0, 0, 3.0, 1, 0, 0],
                    [0, 0, 2.0, 0, 1, 0],      # nearest -> wins pixel (2, 2)
                    [0, 0, 2.0, 0, 0, 1],      # same depth, higher index
                    [0, 0, 0.0005, 1, 1, 1],   # in front of the near plane: culled
                    [0.5, 0, 5.0, 0.5, 0.5, 0.5]], F32)
    img, dep, ind = P.splat(pts, view, np.eye(3), np.zeros(3), 4, 4)
    assert ind[2, 2] == 1 and dep[2, 2] == F32(2.0) and np.array_equal(img[:, 2, 2], [0, 1, 0])
    assert ind[2, 3] == 4                      # u' = 10 * 0.1 + 2 = 3
    assert (ind >= 0).sum() == 2


def test_axial_translation_scales_about_the_principal_point():
    """Moving the viewer back by s along the axis maps a point at depth d and image offset
    a from the principal point to offset a * d / (d + s) (closed form, float64)."""
    H, W = 32, 48
    rng = np.random.default_rng(3)
    depth = rng.uniform(1.0, 3.0, (H, W)).astype(F32)
    rgb = rng.random((3, H, W)).astype(F32)
    cam = (40.0, 40.0, 24.0, 16.0)
    s = 1.5
    pts = P.point_cloud(depth, rgb, cam, np.eye(3), np.zeros(3))
    img, dep, ind = P.splat(pts, cam, np.eye(3), np.array([0, 0, s]), H, W)
    v, u = np.mgrid[0:H, 0:W]
    a_u = (u + 0.5 - 24.0) * depth / (depth + s) + 24.0
    a_v = (v + 0.5 - 16.0) * depth / (depth + s) + 16.0
    # pixels whose closed-form position is not near a pixel border
    safe = (np.abs(a_u - np.round(a_u)) > 1e-3) & (np.abs(a_v - np.round(a_v)) > 1e-3)
    idx = (v * W + u)[safe]
    hit = np.isin(idx, ind)
    rows, cols = np.floor(a_v[safe]).astype(int), np.floor(a_u[safe]).astype(int)
    # every surviving winner sits where the closed form puts it
    won = ind[rows[hit], cols[hit]] == idx[hit]
    assert won.mean() > 0.5 and hit.mean() > 0.3
    for k in np.nonzero(hit)[0][:200]:
        r, c = rows[k], cols[k]
        if ind[r, c] == idx[k]:
            assert abs(dep[r, c] - (depth.reshape(-1)[idx[k]] + s)) < 1e-5


def test_pose_chain_is_rigid_with_the_headset():
    """The calibration chain: with the headset where it was at calibration the camera pose
    is the virtual box's pose; moving the headset by (Rm, tm) moves the camera likewise."""
    R_head, t_head = rot(0.1, -0.3, 0.2), np.array([0.2, 1.5, -0.4])
    R_box, p_box = rot(-0.2, 0.5, 0.1), np.array([0.7, 1.1, 0.3])
    R0, t0 = P.zed_pose(R_head, t_head, R_box, p_box, R_head, t_head)
    assert np.allclose(R0, R_box, atol=1e-12) and np.allclose(t0, p_box, atol=1e-12)
    Rm, tm = rot(0.4, 0.1, -0.7), np.array([-1.0, 0.2, 2.0])
    R1, t1 = P.zed_pose(R_head, t_head, R_box, p_box, Rm @ R_head, Rm @ t_head + tm)
    assert np.allclose(R1, Rm @ R_box, atol=1e-12) and np.allclose(t1, Rm @ p_box + tm, atol=1e-12)


def test_back_projection_closed_form():
    H, W = 5, 7
    depth = np.full((H, W), 2.0, F32)
    rgb = np.zeros((3, H, W), F32)
    cam = (10.0, 20.0, 3.5, 2.5)               # the centre of pixel (2, 3) is the principal point
    R, t = rot(0.3, 0.2, 0.1), np.array([1.0, -2.0, 0.5])
    pts = P.point_cloud(depth, rgb, cam, R, t)
    centre = pts[2 * W + 3, :3]
    assert np.allclose(centre, R @ np.array([0, 0, 2.0]) + t, atol=1e-6)
    corner = pts[0, :3]
    assert np.allclose(corner, R @ np.array([2.0 * (0.5 - 3.5) / 10, 2.0 * (0.5 - 2.5) / 20, 2.0]) + t, atol=1e-6)
