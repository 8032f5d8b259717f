"""Pins of the oracle's Patch-Grid sampling (Sec. II-B; no GPU): counts and positions by
construction, back-projection checked by re-projecting, nearest-keypoint depth against
a brute-force numpy search, depth-image holes, ragged borders."""
import numpy as np

from paper_2509_13536_gb300 import scenegen as sg


def _cam(W=200, H=130):
    c = sg.room_poses(1, 5, W, H)[0]
    return c


def _reproject(cam, xw):
    """Project world points with the camera as the library receives it (float32 values)."""
    f = lambda a: np.asarray(a, np.float32).astype(np.float64)
    R = f(cam.R).reshape(3, 3)
    pc = xw @ R.T + f(cam.t)
    fx, fy, cx, cy = (float(np.float32(x)) for x in (cam.fx, cam.fy, cam.cx, cam.cy))
    return np.stack([fx * pc[:, 0] / pc[:, 2] + cx, fy * pc[:, 1] / pc[:, 2] + cy, pc[:, 2]], 1)


def test_full_patches_give_no_samples(orc):
    cam = _cam(64, 64)
    g = np.stack(np.meshgrid(np.arange(4, 64, 8), np.arange(4, 64, 8)), -1).reshape(-1, 2).astype(np.float32)
    out = orc.patch_grid(cam, g, np.ones(len(g), np.float32), patch=32, min_keypoints=4, grid=2)
    assert len(out["samples"]) == 0


def test_empty_keypoints_depth_image_grid_and_reprojection(orc):
    cam = _cam(200, 130)  # ragged: 7 x 5 patches of 32, the last ones clipped
    depth = np.full((130, 200), 2.5, np.float32)
    out = orc.patch_grid(cam, np.zeros((0, 2), np.float32), None, depth, patch=32, min_keypoints=1, grid=3)
    s = out["samples"]
    assert len(s) == 7 * 5 * 9 and np.all(out["source"] == 0)
    assert np.all(s[:, 0] < 200) and np.all(s[:, 1] < 130) and np.all(s[:, 2] == 2.5)
    # first patch: centres of a 3 x 3 split of [0, 32)^2; last column patch is 200 - 192 = 8 wide
    np.testing.assert_allclose(s[:3, 0], np.float32([32 / 6, 16, 32 - 32 / 6]), rtol=1e-7)
    last = s[6 * 9:7 * 9]
    np.testing.assert_allclose(sorted(set(last[:, 0])), np.float32([192 + 8 / 6, 196, 200 - 8 / 6]), rtol=1e-7)
    np.testing.assert_allclose(_reproject(cam, s[:, 3:]), s[:, :3], rtol=1e-6, atol=1e-6)  # R in float32 is orthonormal to ~1e-7


def test_depth_hole_falls_back_to_nearest_keypoint(orc):
    cam = _cam(64, 32)
    depth = np.full((32, 64), 3.0, np.float32)
    depth[8, 8] = 0  # the first sample of the first patch (grid 2 on 32 px: centres 8, 24)
    kp = np.float32([[40, 20], [10, 10], [11, 9]])
    kd = np.float32([1.0, 2.0, -1.0])  # the third has no depth
    out = orc.patch_grid(cam, kp, kd, depth, patch=32, min_keypoints=3, grid=2)
    s, src = out["samples"], out["source"]
    assert len(s) == 8
    assert src[0] == 1 and s[0, 2] == 2.0 and np.all(src[1:] == 0) and np.all(s[1:, 2] == 3.0)


def test_nearest_keypoint_matches_brute_force(orc):
    rng = np.random.default_rng(3)
    cam = _cam(320, 240)
    # clustered keypoints (texture-rich spots) plus a few scattered ones, some without depth
    centres = rng.uniform([0, 0], [320, 240], (6, 2))
    kp = np.concatenate([c + rng.normal(0, 12, (40, 2)) for c in centres] + [rng.uniform(0, 320, (10, 2))])
    kp = kp.astype(np.float32)
    kd = rng.uniform(0.5, 4, len(kp)).astype(np.float32)
    kd[rng.random(len(kp)) < 0.2] = 0
    out = orc.patch_grid(cam, kp, kd, None, patch=32, min_keypoints=5, grid=2)
    s, src = out["samples"], out["source"]
    assert len(s) > 20 and np.all(src == 1)
    inside = (kp[:, 0] >= 0) & (kp[:, 0] < 320) & (kp[:, 1] >= 0) & (kp[:, 1] < 240)
    cnt = np.zeros((8, 10), int)
    for u, v in kp[inside]:
        cnt[int(v) // 32, int(u) // 32] += 1
    assert len(s) == int((cnt < 5).sum()) * 4
    valid = np.nonzero(kd > 0)[0]
    for u, v, d in s[:, :3]:
        du = kp[valid, 0] - np.float32(u)
        dv = kp[valid, 1] - np.float32(v)
        d2 = du * du + dv * dv  # float32, same expression
        assert d == kd[valid[np.argmin(d2)]]
    np.testing.assert_allclose(_reproject(cam, s[:, 3:]), s[:, :3], rtol=1e-6, atol=1e-6)  # R in float32 is orthonormal to ~1e-7


def test_keypoints_outside_the_image_are_ignored(orc):
    cam = _cam(64, 64)
    kp = np.float32([[-5, 10], [70, 10], [10, 64.5]] * 3)
    out = orc.patch_grid(cam, kp, np.ones(len(kp), np.float32), None, patch=32, min_keypoints=1, grid=1)
    assert len(out["samples"]) == 4
