"""GPU parity of Patch-Grid sampling (Sec. II-B) against the oracle: sample positions,
depths and their source bit for bit (the decisions are float32 on both sides), world
points to float32 rounding."""
import numpy as np
import pytest
import torch

from paper_2509_13536_gb300 import api, scenegen as sg

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_13536_gb300 import build
    build.build()


def _compare(orc, cam, kp, kd, depth, **prm):
    ref = orc.patch_grid(cam, kp, kd, depth, **prm)
    t = lambda a: None if a is None else torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()
    out, src = api.patch_grid_sample(cam, t(kp.reshape(-1, 2)), t(kd), t(depth), **prm)
    torch.cuda.synchronize()
    out = out.cpu().numpy().astype(np.float64)
    assert out.shape[0] == ref["samples"].shape[0]
    np.testing.assert_array_equal(out[:, :3], ref["samples"][:, :3])
    np.testing.assert_array_equal(src.cpu().numpy(), ref["source"])
    np.testing.assert_allclose(out[:, 3:], ref["samples"][:, 3:], rtol=2e-6, atol=2e-6)
    return out.shape[0]


def _clustered(rng, W, H, n_clusters=8, per=60, scattered=20):
    centres = rng.uniform([0, 0], [W, H], (n_clusters, 2))
    kp = np.concatenate([c + rng.normal(0, 0.03 * W, (per, 2)) for c in centres] +
                        [rng.uniform([0, 0], [W, H], (scattered, 2))]).astype(np.float32)
    kd = rng.uniform(0.5, 4.0, len(kp)).astype(np.float32)
    kd[rng.random(len(kp)) < 0.25] = 0  # inactive keypoints: no depth
    return kp, kd


@pytest.mark.parametrize("W,H,patch,grid,kmin", [(1200, 680, 32, 2, 5), (640, 480, 40, 3, 3), (321, 203, 16, 1, 2)])
def test_patch_grid_keypoint_depth(orc, W, H, patch, grid, kmin):
    rng = np.random.default_rng(W + H)
    cam = sg.room_poses(1, 3, W, H)[0]
    kp, kd = _clustered(rng, W, H)
    n = _compare(orc, cam, kp, kd, None, patch=patch, min_keypoints=kmin, grid=grid)
    assert n > 0


def test_patch_grid_depth_image_with_holes(orc):
    rng = np.random.default_rng(5)
    cam = sg.room_poses(1, 4, 640, 480)[0]
    kp, kd = _clustered(rng, 640, 480)
    depth = rng.uniform(1, 3, (480, 640)).astype(np.float32)
    depth[rng.random(depth.shape) < 0.3] = 0  # missing depth
    n = _compare(orc, cam, kp, kd, depth, patch=32, min_keypoints=4, grid=2)
    assert n > 100


def test_patch_grid_no_depth_anywhere_drops_samples(orc):
    cam = sg.room_poses(1, 4, 128, 96)[0]
    kp = np.float32([[10, 10], [50, 50]])
    assert _compare(orc, cam, kp, None, None, patch=32, min_keypoints=1, grid=2) == 0


def test_patch_grid_capacity_error():
    cam = sg.room_poses(1, 4, 64, 64)[0]
    L = api.load()
    p = api._abi.mgs_pg_params(32, 1, 2, 0)
    c = api.camera_struct(cam)
    ws = torch.empty(L.mgs_patch_grid_workspace_size(64, 64, api.C.byref(p)), dtype=torch.uint8, device="cuda")
    out = torch.empty(3, 6, device="cuda")
    depth = torch.ones(64, 64, device="cuda")
    n = api.C.c_int64(0)
    st = L.mgs_patch_grid_sample(api.C.byref(c), 0, None, None, api._ptr(depth), api.C.byref(p), api._ptr(out),
                                 None, 3, api.C.byref(n), api._ptr(ws), ws.numel(), None)
    assert st == api._abi.MGS_ERR_WORKSPACE and n.value == 16
