"""GPU parity of the Eq. 12 mapping loss (L1 + SSIM + depth residual) and the isotropic
term against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import torch

from paper_2509_13536_gb300 import api, scenegen as sg
from tests import _gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_13536_gb300 import build
    build.build()


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a, np.float32)).cuda()


def _case(rng, V, H, W, depth=True):
    x = rng.uniform(0, 1, (V, 3, H, W)).astype(np.float32)
    y = np.clip(x + rng.normal(0, 0.15, x.shape), 0, 1).astype(np.float32)
    y[:, :, ::7, ::5] = x[:, :, ::7, ::5]  # exact ties: sign 0
    d = rng.uniform(1, 3, (V, H, W)).astype(np.float32)
    dt = (d + rng.normal(0, 0.05, d.shape)).astype(np.float32)
    dt[:, ::4, ::3] = 0  # no ground truth there
    return x, y, (d if depth else None), (dt if depth else None)


def _run(x, y, d, dt, lam, wd):
    V = x.shape[0]
    xr, yr = _dev(x), _dev(y)
    dr = _dev(d) if d is not None else torch.zeros(x.shape[0], *x.shape[2:], device="cuda")
    dtr = _dev(dt) if dt is not None else None
    g_rgb = torch.full_like(xr, 7.0)
    g_d = torch.full_like(dr, 7.0)
    rendered = [api.Image(xr[v], dr[v], None) for v in range(V)]
    target = [api.Image(yr[v], None if dtr is None else dtr[v], None) for v in range(V)]
    grad = [api.Image(g_rgb[v], g_d[v], None) for v in range(V)]
    loss = api.mapping_loss(rendered, target, grad, lam, wd)
    torch.cuda.synchronize()
    return loss.cpu().numpy().astype(np.float64), _gpu.to_np(g_rgb), _gpu.to_np(g_d)


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)


@pytest.mark.parametrize("V,H,W", [(2, 45, 67), (1, 16, 32), (3, 7, 5)])
def test_mapping_loss_matches_oracle(orc, V, H, W):
    rng = np.random.default_rng(V * 100 + H)
    x, y, d, dt = _case(rng, V, H, W)
    loss, g_rgb, g_d = _run(x, y, d, dt, 0.2, 0.7)
    ref = orc.mapping_loss(x, y, d, dt, lam=0.2, w_depth=0.7)
    np.testing.assert_allclose(loss, ref["loss"], rtol=2e-5, atol=1e-7)
    assert _rel(g_rgb, ref["g_rgb"]) < 1e-4, _rel(g_rgb, ref["g_rgb"])
    assert np.abs(g_rgb - ref["g_rgb"]).max() < 1e-3 * np.abs(ref["g_rgb"]).max()
    np.testing.assert_array_equal(np.sign(g_d), np.sign(ref["g_depth"]))
    np.testing.assert_allclose(g_d, ref["g_depth"], rtol=1e-6, atol=0)


@pytest.mark.parametrize("V,H,W", [(2, 45, 67), (3, 7, 5)])
def test_mapping_loss_l1_form_matches_oracle(orc, V, H, W):
    """lambda = 0 (the L1 form of Eq. 12, no SSIM windows): loss parts and cotangents
    as the oracle's, with exact ties giving a zero cotangent."""
    rng = np.random.default_rng(V * 31 + W)
    x, y, d, dt = _case(rng, V, H, W)
    loss, g_rgb, g_d = _run(x, y, d, dt, 0.0, 0.1)
    ref = orc.mapping_loss(x, y, d, dt, lam=0.0, w_depth=0.1)
    np.testing.assert_allclose(loss, ref["loss"], rtol=2e-5, atol=1e-7)
    assert np.all(loss[:, 1] == 0)
    np.testing.assert_array_equal(np.sign(g_rgb), np.sign(ref["g_rgb"]))
    np.testing.assert_allclose(g_rgb, ref["g_rgb"], rtol=1e-6, atol=0)
    np.testing.assert_allclose(g_d, ref["g_depth"], rtol=1e-6, atol=0)


def test_mapping_loss_without_depth_and_identical_images(orc):
    rng = np.random.default_rng(7)
    x, _, _, _ = _case(rng, 2, 33, 40)
    loss, g_rgb, g_d = _run(x, x, None, None, 0.2, 1.0)
    np.testing.assert_allclose(loss, 0, atol=2e-6)
    assert np.abs(g_rgb).max() < 1e-6 * 0.2
    assert np.all(g_d == 0)


def test_mapping_loss_full_keyframe(orc):
    """One 1200x680 keyframe of the benchmark workload, rendered, against a perturbed
    map's rendering: the benchmark's image size and value statistics."""
    scene, cams = sg.workload("room1m_sh3")
    cam = cams[0]
    g = api.Gaussians.from_scene(scene, "cuda")
    imgs, _ = api.render(g, [cam])
    pert = scene.copy()
    pert.means = (pert.means + np.random.default_rng(1).normal(0, 0.003, pert.means.shape)).astype(np.float32)
    gp = api.Gaussians.from_scene(pert, "cuda")
    tgt, _ = api.render(gp, [cam])
    torch.cuda.synchronize()
    x, y = _gpu.to_np(imgs[0].rgb)[None], _gpu.to_np(tgt[0].rgb)[None]
    d, dt = _gpu.to_np(imgs[0].depth)[None], _gpu.to_np(tgt[0].depth)[None]
    loss, g_rgb, g_d = _run(x, y, d, dt, 0.2, 0.1)
    ref = orc.mapping_loss(x, y, d, dt, lam=0.2, w_depth=0.1)
    np.testing.assert_allclose(loss, ref["loss"], rtol=5e-5, atol=1e-7)
    assert _rel(g_rgb, ref["g_rgb"]) < 1e-4
    np.testing.assert_allclose(g_d, ref["g_depth"], rtol=1e-6, atol=0)


@pytest.mark.parametrize("dt", [torch.float32, torch.float16])
def test_iso_loss_matches_oracle(orc, dt):
    sc = sg.box_scene(5000, 3)
    g = api.Gaussians.from_scene(sc, "cuda", geom_dtype=dt)
    grads = api.Grads.zeros_like(g, stats=False)
    loss = api.iso_loss(g, 2.0, grads)
    torch.cuda.synchronize()
    ls = _gpu.to_np(g.log_scales)
    val, gref = orc.iso_loss(ls, w_iso=2.0)
    np.testing.assert_allclose(float(loss.item()), val, rtol=1e-5)
    first = _gpu.to_np(grads.log_scales)
    np.testing.assert_allclose(first, gref, rtol=1e-4, atol=1e-12)
    api.iso_loss(g, 2.0, grads)  # the gradient is added, not written
    torch.cuda.synchronize()
    np.testing.assert_allclose(_gpu.to_np(grads.log_scales), 2 * first, rtol=1e-6, atol=0)
