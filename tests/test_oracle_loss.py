"""Pins of the oracle's mapping loss (Sec. II-E, Eq. 12) and isotropic term (no GPU).

SSIM is pinned by its identity (SSIM(x, x) = 1 with zero gradient), its symmetry, an
evaluation whose window sums come from scipy's Gaussian filter (same 11-tap window,
zero padding), and central differences of the loss for the gradient; the L1, depth and
isotropic parts by closed forms and finite differences."""
import numpy as np
import pytest

LAM = 0.2


def _imgs(rng, V=1, H=20, W=23):
    x = rng.uniform(0, 1, (V, 3, H, W))
    y = np.clip(x + rng.normal(0, 0.2, x.shape), 0, 1)
    return x, y


def test_ssim_identity_and_zero_gradient(orc):
    rng = np.random.default_rng(0)
    x, _ = _imgs(rng, 2)
    out = orc.mapping_loss(x, x, lam=LAM)
    np.testing.assert_allclose(out["loss"], 0, atol=1e-14)
    assert np.abs(out["g_rgb"]).max() < 1e-14


def test_ssim_symmetric(orc):
    rng = np.random.default_rng(1)
    x, y = _imgs(rng)
    a = orc.mapping_loss(x, y, lam=LAM, grads=False)["loss"]
    b = orc.mapping_loss(y, x, lam=LAM, grads=False)["loss"]
    np.testing.assert_allclose(a, b, rtol=1e-13)


def test_ssim_against_scipy_window(orc):
    ndimage = pytest.importorskip("scipy.ndimage")
    rng = np.random.default_rng(2)
    x, y = _imgs(rng, 1, 31, 17)
    f = lambda a: ndimage.gaussian_filter(a, 1.5, mode="constant", cval=0.0, truncate=5 / 1.5)
    vals = []
    for c in range(3):
        X, Y = x[0, c], y[0, c]
        mx, my = f(X), f(Y)
        sx, sy, sxy = f(X * X) - mx ** 2, f(Y * Y) - my ** 2, f(X * Y) - mx * my
        C1, C2 = 0.01 ** 2, 0.03 ** 2
        vals.append(((2 * mx * my + C1) * (2 * sxy + C2)) / ((mx ** 2 + my ** 2 + C1) * (sx + sy + C2)))
    ssim = np.mean(vals)
    out = orc.mapping_loss(x, y, lam=1.0, grads=False)
    np.testing.assert_allclose(out["loss"][0, 1], 1 - ssim, rtol=1e-11)
    np.testing.assert_allclose(out["loss"][0, 0], 0.0, atol=0)


def test_l1_and_depth_closed_forms(orc):
    rng = np.random.default_rng(3)
    x, y = _imgs(rng, 2, 9, 11)
    d = rng.uniform(1, 3, (2, 9, 11))
    dt = d + rng.normal(0, 0.1, d.shape)
    dt[:, ::3, ::2] = 0  # no ground truth there
    out = orc.mapping_loss(x, y, d, dt, lam=0.0, w_depth=0.5)
    np.testing.assert_allclose(out["loss"][:, 0], np.abs(x - y).mean(axis=(1, 2, 3)), rtol=1e-13)
    np.testing.assert_allclose(out["loss"][:, 1], 0.0, atol=0)
    valid = dt > 0
    np.testing.assert_allclose(out["loss"][:, 2], 0.5 * (np.abs(d - dt) * valid).mean(axis=(1, 2)), rtol=1e-13)
    np.testing.assert_allclose(out["g_rgb"], np.sign(x - y) / x[0].size, rtol=1e-13)
    np.testing.assert_allclose(out["g_depth"], 0.5 * np.sign(d - dt) * valid / d[0].size, rtol=1e-13)


def test_loss_gradient_finite_differences(orc):
    rng = np.random.default_rng(4)
    x, y = _imgs(rng, 1, 14, 13)
    d = rng.uniform(1, 3, (1, 14, 13))
    dt = d + rng.normal(0, 0.1, d.shape)
    out = orc.mapping_loss(x, y, d, dt, lam=LAM, w_depth=0.3)
    total = lambda xx, dd: orc.mapping_loss(xx, y, dd, dt, lam=LAM, w_depth=0.3, grads=False)["loss"].sum()
    h = 1e-6
    for _ in range(40):
        c, py, px = rng.integers(3), rng.integers(14), rng.integers(13)
        if abs(x[0, c, py, px] - y[0, c, py, px]) < 1e-4:
            continue
        xp, xm = x.copy(), x.copy()
        xp[0, c, py, px] += h
        xm[0, c, py, px] -= h
        fd = (total(xp, d) - total(xm, d)) / (2 * h)
        assert abs(fd - out["g_rgb"][0, c, py, px]) < 1e-7 * max(1.0, abs(fd) * 1e3), (c, py, px)
    for _ in range(10):
        py, px = rng.integers(14), rng.integers(13)
        dp, dm = d.copy(), d.copy()
        dp[0, py, px] += h
        dm[0, py, px] -= h
        fd = (total(x, dp) - total(x, dm)) / (2 * h)
        np.testing.assert_allclose(out["g_depth"][0, py, px], fd, rtol=1e-6, atol=1e-12)


def test_iso_closed_form_and_gradient(orc):
    v, g = orc.iso_loss(np.log([[1.0, 2.0, 3.0]]), w_iso=1.5)
    np.testing.assert_allclose(v, 1.5 * 2.0 / 3.0, rtol=1e-14)
    v0, g0 = orc.iso_loss(np.log(np.full((5, 3), 0.02)))
    assert v0 == 0 and np.all(g0 == 0)
    rng = np.random.default_rng(5)
    ls = rng.uniform(-5, -2, (7, 3))
    v, g = orc.iso_loss(ls, w_iso=2.0)
    h = 1e-7
    for i in range(7):
        for k in range(3):
            lp, lm = ls.copy(), ls.copy()
            lp[i, k] += h
            lm[i, k] -= h
            fd = (orc.iso_loss(lp, 2.0)[0] - orc.iso_loss(lm, 2.0)[0]) / (2 * h)
            np.testing.assert_allclose(g[i, k], fd, rtol=1e-5, atol=1e-12)
