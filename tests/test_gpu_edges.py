"""GPU edge cases against the oracle: the hand-built scenes at the alpha cutoff, the 0.99
clamp, the transmittance stop and the depth tie-break; the maximum number of views in
one launch; degenerate merge inputs."""
import math

import numpy as np
import pytest
import torch

from paper_2509_13536_gb300 import api, scenegen as sg
from tests import _gpu
from tests._scenes import camera, make_scene, random_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_13536_gb300 import build
    build.build()


def _render(sc, cams):
    g = api.Gaussians.from_scene(sc, "cuda")
    imgs, ws = api.render(g, cams)
    torch.cuda.synchronize()
    return g, imgs, ws


def _same_as_oracle(orc, sc, cam, tol=_gpu.IMG_TOL):
    _, imgs, _ = _render(sc, [cam])
    ref = orc.render(sc, cam)
    assert not ref["flags"].any()
    for name in ("rgb", "depth", "alpha"):
        np.testing.assert_allclose(_gpu.to_np(getattr(imgs[0], name)), ref[name], atol=tol, rtol=0)
    return imgs[0], ref


@pytest.mark.parametrize("sign", [+1, -1])
def test_alpha_cutoff_scene(orc, sign):
    """alpha = 1/255 (1 +- 1e-3) at pixel (19, 16): blended above, skipped below, as in the oracle."""
    f, z, s = 100.0, 2.0, 0.04
    sig2 = (f * math.exp(float(np.float32(math.log(s)))) / z) ** 2 + 0.3
    o = (1 / 255) * (1 + sign * 1e-3) * math.exp(0.5 * 9.0 / sig2)
    sc = make_scene([[0, 0, z]], [[s, s, s]], [[1, 0, 0, 0]], [o], [[1, 1, 1]])
    img, ref = _same_as_oracle(orc, sc, camera(32, 32, f, f, 16, 16))
    a = float(_gpu.to_np(img.alpha)[16, 19])
    assert (a > 0) == (sign > 0) and (ref["alpha"][16, 19] > 0) == (sign > 0)


def test_opacity_clamp_scene(orc):
    sc = make_scene([[0, 0, 2.0]], [[0.1, 0.1, 0.1]], [[1, 0, 0, 0]], [0.9999], [[1, 1, 1]])
    img, _ = _same_as_oracle(orc, sc, camera(32, 32, 100, 100, 16, 16))
    assert abs(float(_gpu.to_np(img.alpha)[16, 16]) - 0.99) < 1e-6


def test_transmittance_stop_scene_and_its_gradient(orc):
    """Six alpha-0.95 layers: at the centre pixel the 4th takes T below 1e-4 and is
    blended, the 5th and 6th are not (off-centre pixels, with smaller alpha, reach them).
    Image and gradients as in the oracle."""
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1], [1, 0, 1]]
    z = [2.0, 2.5, 3.0, 3.5, 4.0, 4.5]
    n = len(z)
    sc = make_scene([[0, 0, zz] for zz in z], [[0.5, 0.5, 0.5]] * n, [[1, 0, 0, 0]] * n, [0.95] * n, cols)
    cam = camera(32, 32, 100, 100, 16, 16)
    g, imgs, ws = _render(sc, [cam])
    ref = orc.render(sc, cam)
    np.testing.assert_allclose(_gpu.to_np(imgs[0].rgb), ref["rgb"], atol=_gpu.IMG_TOL)
    cot_np, dL = _gpu.masked_cotangents([cam], [ref], 3)
    grads = api.render_backward(g, [cam], dL, ws)
    torch.cuda.synchronize()
    refg = _gpu.oracle_backward(orc, sc, [cam], cot_np)
    o = 1 / (1 + math.exp(-float(sc.opacity_logit[0])))
    assert abs(float(_gpu.to_np(imgs[0].alpha)[16, 16]) - (1 - (1 - o) ** 4)) < 1e-6
    _gpu.check_grads(grads, refg)


def test_clamp_entries_mixed_with_plain_ones(orc):
    """Entries whose opacity exceeds 0.98 can reach the 0.99 clamp and take the clamped
    path of both blends (the 8-entry groups of the forward, the 16-entry batches of the
    backward); they share tiles and batches with entries that skip it.  Two views at a
    ragged 150x110: images against the oracle's outcomes and every gradient element
    within the element-wise bound."""
    rng = np.random.default_rng(11)
    n = 400
    means = rng.uniform(-1.0, 1.0, size=(n, 3)) + np.array([0.0, 0.0, 3.0])
    scales = np.exp(rng.uniform(math.log(0.02), math.log(0.15), size=(n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    op = rng.uniform(0.1, 0.9, size=n)
    op[::3] = rng.uniform(0.985, 0.9999, size=op[::3].shape)  # a third can reach the clamp
    sh = rng.normal(0, 0.3, size=(n, 4, 3))
    sh[:, 0, :] = (rng.random((n, 3)) - 0.5) / (0.5 / math.sqrt(math.pi))
    sc = make_scene(means, scales, q, op, None, 1, sh)
    th = 0.2
    Ry = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    cams = [camera(150, 110, 100, 100, 74.5, 54.5),
            camera(150, 110, 110, 105, 70.0, 58.0, R=Ry, t=-Ry @ np.array([0.3, 0.0, -0.2]))]
    # the scene does what it is for (oracle projection of view 0): entries reach the
    # clamp at a pixel centre
    p = orc.project(sc, cams[0])
    u = np.rint(p["mean2d"])
    d = u - p["mean2d"]
    A, B, C = p["conic"][:, 0], p["conic"][:, 1], p["conic"][:, 2]
    a_peak = p["opacity"] * np.exp(-0.5 * (A * d[:, 0] ** 2 + 2 * B * d[:, 0] * d[:, 1] + C * d[:, 1] ** 2))
    inside = (u[:, 0] >= 0) & (u[:, 0] < 150) & (u[:, 1] >= 0) & (u[:, 1] < 110)
    assert ((p["visible"] > 0) & inside & (a_peak > 0.99)).sum() >= 5
    g, imgs, ws = _render(sc, cams)
    refs = [orc.render_outcomes(sc, c) for c in cams]
    for v in range(2):
        _gpu.check_image(imgs[v], refs[v], what=f"clamp mix view {v}")
    cot_np, dL = _gpu.masked_cotangents(cams, refs, 12)
    grads = api.render_backward(g, cams, dL, ws)
    torch.cuda.synchronize()
    _gpu.check_grads(grads, _gpu.oracle_backward(orc, sc, cams, cot_np), what="clamp mix")


def test_gaussians_around_the_image_border(orc):
    """Centres projected up to 60 px outside a 120x90 image, depths from just behind the
    near plane (0.2) to 3, in two views: the projection's cheap per-view test skips
    about half of the (Gaussian, view) items here, and may skip only those the full test
    rejects, so both views' images match the oracle's outcomes."""
    rng = np.random.default_rng(41)
    n = 2000
    W, H, f = 120, 90, 100.0
    z = np.where(rng.random(n) < 0.08, rng.uniform(0.19, 0.23, n), rng.uniform(0.23, 3.0, n))
    u = rng.uniform(-60, W + 60, n)
    v = rng.uniform(-60, H + 60, n)
    means = np.stack([(u - (W - 1) / 2) * z / f, (v - (H - 1) / 2) * z / f, z], 1)
    smax = np.where(z < 0.23, 0.004, 0.05)
    scales = np.exp(rng.uniform(math.log(0.002), np.log(smax)[:, None], size=(n, 3)))
    q = rng.normal(size=(n, 4))
    q /= np.linalg.norm(q, axis=1, keepdims=True)
    op = rng.uniform(0.05, 0.9, n)
    sh = rng.normal(0, 0.3, size=(n, 4, 3))
    sh[:, 0, :] = (rng.random((n, 3)) - 0.5) / (0.5 / math.sqrt(math.pi))
    sc = make_scene(means, scales, q, op, None, 1, sh)
    th = 0.2
    Ry = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    cams = [camera(W, H, f, f, (W - 1) / 2, (H - 1) / 2),
            camera(W, H, f, 0.9 * f, W / 2 + 7, H / 2 - 5, R=Ry, t=np.array([0.05, -0.03, 0.02]))]
    _, imgs, _ = _render(sc, cams)
    for k, c in enumerate(cams):
        _gpu.check_image(imgs[k], orc.render_outcomes(sc, c), what=f"border view {k}")


def test_depth_tie_keeps_index_order(orc):
    cols = [[1, 0, 0], [0, 1, 0]]
    sc = make_scene([[0, 0, 2.0], [0, 0, 2.0]], [[0.3] * 3] * 2, [[1, 0, 0, 0]] * 2, [0.6, 0.5], cols)
    img, ref = _same_as_oracle(orc, sc, camera(32, 32, 100, 100, 16, 16))
    assert abs(float(_gpu.to_np(img.rgb)[0, 16, 16]) - ref["rgb"][0, 16, 16]) < 1e-6


def test_maximum_views_in_one_launch(orc):
    """MGS_MAX_VIEWS = 32 keyframes of mixed sizes in one call; each matches the oracle."""
    rng = np.random.default_rng(32)
    sc = random_scene(rng, 3000, sh_degree=1)
    cams = []
    for v in range(32):
        W, H = [(48, 40), (64, 48), (37, 29)][v % 3]
        t = np.float32([rng.uniform(-0.2, 0.2), rng.uniform(-0.2, 0.2), rng.uniform(-0.5, 0.5)])
        cams.append(camera(W, H, 60.0, 60.0, W / 2, H / 2, t=t))
    _, imgs, _ = _render(sc, cams)
    for v, c in enumerate(cams):
        _gpu.check_image(imgs[v], orc.render_outcomes(sc, c), what=f"view {v}")
    with pytest.raises(Exception):
        api.render(api.Gaussians.from_scene(sc, "cuda"), cams + cams[:1])  # 33 views: rejected


def test_gradients_over_many_views(orc):
    """24 views of one map in one call, placed around it so that Gaussians take their
    gradients from anywhere between 0 and 24 views: the reverse projection's work plan
    (Gaussians bucketed by gradient-view count, most first) covers every bucket, and every
    gradient element matches the oracle's sum over the views within the element-wise
    bound."""
    rng = np.random.default_rng(24)
    sc = random_scene(rng, 600, sh_degree=1, spread=1.5, depth=0.0)
    cams = []
    for v in range(24):
        th = 2 * math.pi * v / 24
        W, H = [(40, 32), (48, 36), (33, 29)][v % 3]
        d = rng.uniform(2.4, 3.0)
        centre = np.array([d * math.sin(th), rng.uniform(-0.4, 0.4), -d * math.cos(th)])
        fwd = -centre / np.linalg.norm(centre)
        right = np.cross([0.0, 1.0, 0.0], fwd)
        right /= np.linalg.norm(right)
        down = np.cross(fwd, right)
        R = np.stack([right, down, fwd])
        cams.append(camera(W, H, rng.uniform(60, 90), rng.uniform(60, 90), W / 2, H / 2, R=R, t=-R @ centre))
    g, imgs, ws = _render(sc, cams)
    refs = [orc.render_outcomes(sc, c) for c in cams]
    for v in range(len(cams)):
        _gpu.check_image(imgs[v], refs[v], what=f"view {v}")
    cot_np, dL = _gpu.masked_cotangents(cams, refs, 25)
    grads = api.render_backward(g, cams, dL, ws)
    torch.cuda.synchronize()
    vis = grads.vis_count.cpu().numpy()
    assert len(np.unique(vis)) >= 20  # drawing-view counts spread over the buckets
    _gpu.check_grads(grads, _gpu.oracle_backward(orc, sc, cams, cot_np), what="24 views")


def test_merge_degenerate_inputs(orc):
    from tests.test_oracle_merge import _voxel_scene
    rng = np.random.default_rng(8)
    sc = _voxel_scene(rng, 20, 4)
    for sub in (sc.subset(np.arange(0)), sc.subset(np.arange(1))):
        g = api.Gaussians.from_scene(sub, "cuda")
        out, partner, _ = api.mgs_voxel_merge(g, 0.02)
        torch.cuda.synchronize()
        assert out.n == sub.n and np.all(partner.cpu().numpy() == -1)
    g = api.Gaussians.from_scene(sc, "cuda")
    high = torch.full((sc.n,), 1.0, device="cuda")  # nothing passes the Eq. 3 mask
    out, partner, vox = api.mgs_voxel_merge(g, 0.02, grad_stat=high)
    torch.cuda.synchronize()
    assert out.n == sc.n and np.all(partner.cpu().numpy() == -1)
    assert np.all(vox.cpu().numpy() == np.iinfo(np.int32).min)
