"""The oracle's hand-written reverse pass against central finite differences of its own
forward, parameter by parameter (no GPU).  Decisions (who contributes where, where each
pixel stops) are checked identical at theta +- h through the decision hash."""
import math

import numpy as np
import pytest

from tests._scenes import camera, make_scene, random_scene

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")


def _loss(orc, sc, cam, w, **over):
    out = orc.render(sc, cam, margin=None, hash_decisions=True, n_threads=1, **over)
    L = (w[0] * out["rgb"]).sum() + (w[1] * out["depth"]).sum() + (w[2] * out["alpha"]).sum()
    return L, out["hash"]


def _fd_check(orc, sc, cam, seed, max_skipped_frac=0.05):
    rng = np.random.default_rng(seed)
    H, W = cam.height, cam.width
    w = (rng.uniform(-1, 1, (3, H, W)), rng.uniform(-1, 1, (H, W)), rng.uniform(-1, 1, (H, W)))
    g = orc.render_backward(sc, cam, *w, margin=None, n_threads=1)
    base = {k: getattr(sc, k).astype(np.float64) for k in FIELDS}
    _, h0 = _loss(orc, sc, cam, w, **base)
    checked = skipped = 0
    worst = 0.0
    for k in FIELDS:
        arr = base[k]
        for idx in np.ndindex(arr.shape):
            th = arr[idx]
            h = 1e-6 * max(1.0, abs(th))
            p = {kk: vv.copy() for kk, vv in base.items()}
            p[k][idx] = th + h
            Lp, hp = _loss(orc, sc, cam, w, **p)
            p[k][idx] = th - h
            Lm, hm = _loss(orc, sc, cam, w, **p)
            if hp != h0 or hm != h0:
                skipped += 1
                continue
            fd = (Lp - Lm) / (2 * h)
            an = g[k][idx]
            err = abs(fd - an) / max(1e-3, abs(an), abs(fd))
            worst = max(worst, err)
            assert err < 2e-5, (k, idx, fd, an)
            checked += 1
    assert checked > 0 and skipped <= max_skipped_frac * (checked + skipped)
    return worst, checked, g


@pytest.mark.parametrize("deg", [0, 1, 3])
def test_backward_matches_finite_differences(orc, deg):
    rng = np.random.default_rng(10 + deg)
    sc = random_scene(rng, 10, sh_degree=deg, spread=0.8, depth=2.5)
    cam = camera(40, 32, 30, 30, 19.6, 15.3)
    worst, checked, g = _fd_check(orc, sc, cam, seed=deg)
    assert checked > 10 * (3 + 3 + 4 + 1 + 3 * (deg + 1) ** 2) * 0.9


def test_backward_fov_clamp_and_colour_clamp(orc):
    """A Gaussian beyond the 1.3 FOV clamp but still overlapping the image, and one whose
    raw colour is negative in one channel (max(0, .) active)."""
    fx = 30.0
    W, H = 40, 32
    lim = 1.3 * (0.5 * W / fx)
    z = 2.0
    means = [[lim * z * 1.1, 0.1, z], [0.0, 0.05, 2.3], [-0.2, -0.1, 2.6]]
    scales = [[0.8, 0.3, 0.4], [0.2, 0.3, 0.1], [0.3, 0.2, 0.25]]
    quats = [[0.9, 0.1, 0.2, 0.3], [0.7, -0.2, 0.1, 0.5], [1.0, 0.0, 0.3, -0.1]]
    sh = np.zeros((3, 4, 3))
    sh[:, 0, :] = [[0.5, 0.2, -2.5], [0.3, -0.4, 0.6], [0.1, 0.1, 0.1]]
    sh[:, 1:, :] = np.random.default_rng(4).normal(0, 0.2, (3, 3, 3))
    sc = make_scene(means, scales, quats, [0.7, 0.6, 0.5], None, 1, sh)
    cam = camera(W, H, fx, fx, 19.5, 15.5)
    proj = orc.project(sc, cam)
    assert proj["visible"][0] == 1
    assert (proj["rgb"][0] == 0).any()  # colour clamp active
    _fd_check(orc, sc, cam, seed=9)


def test_grad_stat_is_mean_gradient_norm(orc):
    rng = np.random.default_rng(5)
    sc = random_scene(rng, 30, sh_degree=1)
    cam = camera(48, 32, 30, 30, 24, 16)
    H, W = 32, 48
    w = (rng.uniform(-1, 1, (3, H, W)), rng.uniform(-1, 1, (H, W)), rng.uniform(-1, 1, (H, W)))
    g = orc.render_backward(sc, cam, *w)
    vis = orc.project(sc, cam)["visible"] > 0
    np.testing.assert_allclose(g["grad_stat"], np.linalg.norm(g["means"], axis=1), rtol=1e-12)
    np.testing.assert_array_equal(g["vis_count"], vis.astype(np.float64))


def test_tile_subset_backward_equals_masked_cotangent(orc):
    from paper_2509_13536_gb300 import scenegen as sg
    sc, cams = sg.workload("box10k")
    sc = sc.subset(np.arange(2000))
    cam = cams[0]
    gr, gd, ga = (x[0] for x in sg.image_cotangents(1, 320, 240, 0))
    tiles = np.array([3, 40, 41, 120, 250])
    mask = np.zeros((240, 320), bool)
    for t in tiles:
        ty, tx = divmod(int(t), 20)
        mask[ty * 16:ty * 16 + 16, tx * 16:tx * 16 + 16] = True
    a = orc.render_backward(sc, cam, gr, gd, ga, tiles=tiles)
    b = orc.render_backward(sc, cam, gr * mask, gd * mask, ga * mask)
    for k in FIELDS:
        np.testing.assert_allclose(a[k], b[k], rtol=1e-12, atol=1e-14)


def test_gradient_scale_bounds_and_single_term_equality(orc):
    """The per-element error scale (sum over paths of |term| x the term's relative error
    budget, u = 32 x 2^-24 with zero margins) is never below u |gradient| (triangle
    inequality), equals it (plus the evaluation budget of Y00) for the DC coefficient
    when one pixel carries the only cotangent (a single term, no cancellation), stays large where two mirror
    pixels' terms cancel, and grows with the alpha and T margins."""
    u = 32 * 2.0 ** -24
    zero = orc.margins(alpha_rel=0, T_rel=0, cond_rel=0)
    rng = np.random.default_rng(5)
    sc = random_scene(rng, 40, sh_degree=2, spread=1.0, depth=2.5)
    cam = camera(48, 32, 30, 30, 23.7, 15.2)
    w = (rng.uniform(-1, 1, (3, 32, 48)), rng.uniform(-1, 1, (32, 48)), rng.uniform(-1, 1, (32, 48)))
    g = orc.render_backward(sc, cam, *w, margin=zero, grads=orc.new_grads(sc.n, 2, scale=True))
    gm = orc.render_backward(sc, cam, *w, margin=orc.margins(), grads=orc.new_grads(sc.n, 2, scale=True))
    for k in FIELDS:
        assert (g["scale_" + k] >= u * np.abs(g[k]) * (1 - 1e-12)).all(), k
        assert (g["scale_" + k] > 0).any()
        assert (gm["scale_" + k] >= g["scale_" + k] * (1 - 1e-12)).all(), k
        assert (gm["scale_" + k] > 1.5 * g["scale_" + k]).any(), k
    # one Gaussian on the axis, one pixel of cotangent on the red channel
    one = make_scene([[0, 0, 2.0]], [[0.05] * 3], [[1, 0, 0, 0]], [0.7], [[0.3, 0.6, 0.9]], sh_degree=1,
                     sh=np.full((1, 4, 3), 0.1))
    cam1 = camera(32, 32, 100, 100, 16, 16)
    gr = np.zeros((3, 32, 32)); gr[0, 18, 19] = 0.7
    g1 = orc.render_backward(one, cam1, gr, None, None, margin=zero, grads=orc.new_grads(1, 1, scale=True))
    assert np.abs(g1["sh"]).max() > 0
    # the DC basis function does not depend on the direction: only the 16 x 2^-24 of its
    # evaluation is added to the single term's budget (d colour = g_sh0 / Y00)
    Y00 = 0.28209479177387814
    want = (u + 16 * 2.0 ** -24 / Y00) * abs(g1["sh"][0, 0, 0])
    np.testing.assert_allclose(g1["scale_sh"][0, 0, 0], want, rtol=1e-12)
    assert (g1["scale_sh"] >= u * np.abs(g1["sh"])).all()
    # two mirror pixels with equal cotangent: their du terms cancel (screen-space du ~ 0);
    # what is left of the mean's x-gradient comes through the Jacobian, far below its scale
    gr = np.zeros((3, 32, 32)); gr[0, 16, 13] = 1.0; gr[0, 16, 19] = 1.0
    g2 = orc.render_backward(one, cam1, gr, None, None, margin=zero, grads=orc.new_grads(1, 1, scale=True))
    assert abs(g2["grad2d"][0, 0]) < 1e-9 * np.abs(g2["grad2d"][0]).max()
    assert g2["scale_means"][0, 0] > 100 * u * abs(g2["means"][0, 0])
