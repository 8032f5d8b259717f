"""Pins of the FP64 oracle's projection and blending against closed forms, invariants
and a brute-force evaluation (no GPU).  Sec. II-C Eq. 1-2, Sec. II-E Eq. 11."""
import math

import numpy as np
import pytest

from tests._scenes import Y00, camera, make_scene, random_scene

pytestmark = pytest.mark.filterwarnings("ignore")


def _rot_z(th):
    c, s = math.cos(th), math.sin(th)
    return np.array([[c, -s], [s, c]])


def test_single_gaussian_on_axis_closed_form(orc):
    """On the optical axis J's third column vanishes: Sigma_I = D R2 diag(sx^2, sy^2) R2^T D + 0.3 I,
    D = diag(fx/z, fy/z), R2 the in-plane rotation; alpha = o exp(-1/2 d^T Sigma_I^-1 d)."""
    z, th, sx, sy, sz, o = 2.5, 0.7, 0.05, 0.02, 0.03, 0.8
    fx, fy, cx, cy, W, H = 400.0, 300.0, 60.0, 40.0, 128, 96
    q = [math.cos(th / 2), 0, 0, math.sin(th / 2)]
    col = [0.2, 0.5, 0.9]
    sc = make_scene([[0, 0, z]], [[sx, sy, sz]], [q], [o], [col])
    cam = camera(W, H, fx, fy, cx, cy)
    p = orc.project(sc, cam)
    s32 = np.exp(sc.log_scales.astype(np.float64))[0]
    R2 = _rot_z(th)
    D = np.diag([fx / z, fy / z])
    cov = D @ R2 @ np.diag(s32[:2] ** 2) @ R2.T @ D + 0.3 * np.eye(2)
    np.testing.assert_allclose(p["mean2d"][0], [cx, cy], atol=1e-12)
    np.testing.assert_allclose(p["depth"][0], z, rtol=1e-12)
    np.testing.assert_allclose(p["cov2d"][0], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-5)
    conic = np.linalg.inv(cov)
    np.testing.assert_allclose(p["conic"][0], [conic[0, 0], conic[0, 1], conic[1, 1]], rtol=1e-5)
    lam = np.linalg.eigvalsh(cov).max()
    r = math.ceil(3 * math.sqrt(lam))
    assert p["radius"][0] == r
    rect = [max(0, math.floor((cx - r) / 16)), max(0, math.floor((cy - r) / 16)),
            min((W + 15) // 16 - 1, math.floor((cx + r) / 16)), min((H + 15) // 16 - 1, math.floor((cy + r) / 16))]
    assert list(p["rect"][0]) == rect
    out = orc.render(sc, cam)
    yy, xx = np.mgrid[0:H, 0:W]
    d = np.stack([cx - xx, cy - yy], -1)
    power = -0.5 * np.einsum("...i,ij,...j->...", d, conic, d)
    a = np.minimum(0.99, o * np.exp(power))
    a[a < 1 / 255] = 0
    in_rect = ((xx // 16 >= rect[0]) & (xx // 16 <= rect[2]) & (yy // 16 >= rect[1]) & (yy // 16 <= rect[3]))
    a[~in_rect] = 0
    o32 = 1 / (1 + math.exp(-float(sc.opacity_logit[0])))
    a = a * (o32 / o)
    np.testing.assert_allclose(out["alpha"], a, atol=2e-6)
    c32 = sc.sh[0, 0].astype(np.float64) * Y00 + 0.5
    for ch in range(3):
        np.testing.assert_allclose(out["rgb"][ch], c32[ch] * out["alpha"], atol=1e-12)
    np.testing.assert_allclose(out["depth"], z * out["alpha"], rtol=1e-9, atol=1e-12)


def _project_points(R, t, fx, fy, cx, cy, X):
    P = X @ R.T + t
    return np.stack([fx * P[:, 0] / P[:, 2] + cx, fy * P[:, 1] / P[:, 2] + cy], 1)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_projection_matches_sigma_point_covariance(orc, seed):
    """For a tiny Gaussian the linearised projection (Eq. 1) equals the covariance of the
    projected symmetric sigma points mu +- sqrt(3) L e_k (exact for linear maps)."""
    from paper_2509_13536_gb300 import scenegen as sg
    rng = np.random.default_rng(seed)
    cam = sg.look_at(rng.uniform(-1, 1, 3), rng.uniform(-1, 1, 3) + [0, 0, 5], 320, 240)
    R, t = cam.R.astype(np.float64), cam.t.astype(np.float64)
    centre = -R.T @ t
    fwd = R[2]
    mu = centre + 3.0 * fwd + 0.6 * R[0] - 0.4 * R[1]
    q = rng.normal(size=4)
    s = np.array([2e-4, 1e-4, 3e-4])
    sc = make_scene([mu], [s], [q], [0.5], [[0.5, 0.5, 0.5]])
    p = orc.project(sc, cam)
    mu64 = sc.means[0].astype(np.float64)
    S = orc.covariance(sc.quats[0], np.exp(sc.log_scales[0].astype(np.float64)))
    L = np.linalg.cholesky(S)
    pts = np.concatenate([mu64 + math.sqrt(3) * L[:, k] * sg_ for k in range(3) for sg_ in (1, -1)]).reshape(6, 3)
    uv = _project_points(R, t, cam.fx, cam.fy, cam.cx, cam.cy, pts)
    uv0 = _project_points(R, t, cam.fx, cam.fy, cam.cx, cam.cy, mu64[None])[0]
    dev = uv - uv0
    cov_sp = dev.T @ dev / 6
    np.testing.assert_allclose(p["mean2d"][0], uv0, rtol=1e-12)
    got = np.array([[p["cov2d"][0, 0] - 0.3, p["cov2d"][0, 1]], [p["cov2d"][0, 1], p["cov2d"][0, 2] - 0.3]])
    np.testing.assert_allclose(got, cov_sp, rtol=2e-3, atol=1e-9 * np.abs(cov_sp).max())


def test_fov_clamp_uses_clamped_ray(orc):
    """Beyond 1.3x the half field of view the Jacobian is taken at the clamped ray."""
    fx = fy = 100.0
    W, H = 64, 64
    lim = 1.3 * (0.5 * W / fx)
    z, x = 2.0, 2.0 * (lim * 1.5)
    sc = make_scene([[x, 0.0, z]], [[0.05, 0.05, 0.05]], [[1, 0, 0, 0]], [0.5], [[0.5, 0.5, 0.5]])
    p = orc.project(sc, camera(W, H, fx, fy, 32, 32))
    s = float(np.exp(np.float64(sc.log_scales[0, 0])))
    xc = lim * z
    J = np.array([[fx / z, 0, -fx * xc / (z * z)], [0, fy / z, 0]])
    cov = J @ (s * s * np.eye(3)) @ J.T + 0.3 * np.eye(2)
    np.testing.assert_allclose(p["cov2d"][0], [cov[0, 0], cov[0, 1], cov[1, 1]], rtol=1e-6)


def test_sh_basis_orthonormal_by_quadrature(orc):
    """Real spherical harmonics up to degree 3 are orthonormal on the sphere (product
    Gauss-Legendre in cos(theta) x trapezoid in phi, exact for these degrees)."""
    zs, wz = np.polynomial.legendre.leggauss(12)
    phis = np.linspace(0, 2 * np.pi, 24, endpoint=False)
    G = np.zeros((16, 16))
    for z, w in zip(zs, wz):
        for ph in phis:
            r = math.sqrt(1 - z * z)
            Y, _ = orc.sh_basis(3, [r * math.cos(ph), r * math.sin(ph), z])
            G += np.outer(Y, Y) * w * (2 * np.pi / len(phis))
    np.testing.assert_allclose(G, np.eye(16), atol=1e-12)
    Y, _ = orc.sh_basis(0, [0, 0, 1])
    assert abs(Y[0] - Y00) < 1e-15


def test_sh_gradient_tangential_matches_finite_difference(orc):
    rng = np.random.default_rng(3)
    for _ in range(5):
        d = rng.normal(size=3); d /= np.linalg.norm(d)
        Y, dY = orc.sh_basis(3, d)
        tng = np.cross(d, rng.normal(size=3)); tng /= np.linalg.norm(tng)
        h = 1e-6
        dp = (d + h * tng) / np.linalg.norm(d + h * tng)
        dm = (d - h * tng) / np.linalg.norm(d - h * tng)
        fd = (orc.sh_basis(3, dp)[0] - orc.sh_basis(3, dm)[0]) / (2 * h)
        np.testing.assert_allclose(dY @ tng, fd, atol=1e-8)


def test_sh0_colour_recipe(orc):
    from paper_2509_13536_gb300 import scenegen as sg
    sc = sg.box_scene(50, 5, 0)
    p = orc.project(sc, sg.box_camera())
    want = sc.sh[:, 0, :].astype(np.float64) * Y00 + 0.5
    vis = p["visible"] > 0
    np.testing.assert_allclose(p["rgb"][vis], np.maximum(0, want[vis]), atol=1e-12)


def test_blend_invariants(orc):
    """White Gaussians: rgb = sum_i w_i must equal 1 - prod(1 - alpha_i) (telescoping);
    one colour c: rgb = c * alpha; one depth plane z: depth = z * alpha."""
    rng = np.random.default_rng(7)
    n = 300
    means = np.c_[rng.uniform(-1, 1, (n, 2)), np.full(n, 3.0)]
    scales = np.exp(rng.uniform(math.log(0.02), math.log(0.2), (n, 3)))
    q = rng.normal(size=(n, 4))
    op = rng.uniform(0.1, 0.9, n)
    col = np.tile([0.3, 0.6, 0.9], (n, 1))
    sc = make_scene(means, scales, q, op, col)
    cam = camera(96, 64, 60, 60, 48, 32)
    out = orc.render(sc, cam)
    c32 = sc.sh[0, 0].astype(np.float64) * Y00 + 0.5
    for ch in range(3):
        np.testing.assert_allclose(out["rgb"][ch], c32[ch] * out["alpha"], atol=1e-12)
    np.testing.assert_allclose(out["depth"], 3.0 * out["alpha"], atol=1e-11)
    white = make_scene(means, scales, q, op, np.ones((n, 3)))
    ow = orc.render(white, cam)
    np.testing.assert_allclose(ow["rgb"][0] + ow["T_final"], 1.0, atol=1e-12)
    assert (ow["alpha"] > 0.5).mean() > 0.2  # the scene really overlaps


@pytest.mark.parametrize("seed", range(6))
def test_binned_equals_bruteforce(orc, seed):
    """Tile binning + per-tile sort == per-pixel scan over all Gaussians with explicit products."""
    rng = np.random.default_rng(100 + seed)
    sc = random_scene(rng, 64, sh_degree=seed % 4, spread=1.2, depth=2.5)
    if seed % 2:
        sc.means[:5, 2] = rng.uniform(-1.0, 0.25, 5)  # some behind or at the near plane
    cam = camera(48, 32, 30, 30, 23.7, 15.2)
    a = orc.render(sc, cam, margin=None)
    b = orc.render_bruteforce(sc, cam)
    for k in ("rgb", "depth", "alpha"):
        np.testing.assert_allclose(a[k], b[k], atol=1e-12)


def _iso_sigma2(f, s, z):
    return (f * s / z) ** 2 + 0.3


def test_alpha_cutoff_hand_built(orc):
    """A pixel whose alpha is 1/255*(1 + 1e-3) is blended; at 1/255*(1 - 1e-3) it is not."""
    f, z, s, W, H = 100.0, 2.0, 0.04, 32, 32
    for sign in (+1, -1):
        sig2 = _iso_sigma2(f, math.exp(float(np.float32(math.log(s)))), z)
        d = 3.0  # pixel (16+3, 16)
        o = (1 / 255) * (1 + sign * 1e-3) * math.exp(0.5 * d * d / sig2)
        sc = make_scene([[0, 0, z]], [[s, s, s]], [[1, 0, 0, 0]], [o], [[1, 1, 1]])
        out = orc.render(sc, camera(W, H, f, f, 16, 16))
        o32 = 1 / (1 + math.exp(-float(sc.opacity_logit[0])))
        expect = o32 * math.exp(-0.5 * d * d / sig2)
        got = out["alpha"][16, 19]
        if expect >= 1 / 255:
            assert abs(got - expect) < 1e-12 and sign > 0
        else:
            assert got == 0.0 and sign < 0


def test_opacity_clamp_hand_built(orc):
    sc = make_scene([[0, 0, 2.0]], [[0.1, 0.1, 0.1]], [[1, 0, 0, 0]], [0.9999], [[1, 1, 1]])
    out = orc.render(sc, camera(32, 32, 100, 100, 16, 16))
    assert abs(out["alpha"][16, 16] - 0.99) < 1e-15


def test_transmittance_stop_hand_built(orc):
    """Layers with alpha 0.95 at the centre pixel: T = 0.05^k; the 4th layer takes T below
    1e-4 and is still blended, the 5th and 6th are not."""
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1], [1, 0, 1]]
    z = [2.0, 2.5, 3.0, 3.5, 4.0, 4.5]
    n = len(z)
    sc = make_scene([[0, 0, zz] for zz in z], [[0.5, 0.5, 0.5]] * n, [[1, 0, 0, 0]] * n, [0.95] * n, cols)
    out = orc.render(sc, camera(32, 32, 100, 100, 16, 16))
    o = 1 / (1 + math.exp(-float(sc.opacity_logit[0])))
    c32 = np.maximum(0, sc.sh[:, 0, :].astype(np.float64) * Y00 + 0.5)
    expect = sum(c32[k] * o * (1 - o) ** k for k in range(4))
    np.testing.assert_allclose(out["rgb"][:, 16, 16], expect, atol=1e-14)
    assert out["n_contrib"][16, 16] == 4 and out["n_eval"][16, 16] == 4
    assert abs(out["T_final"][16, 16] - (1 - o) ** 4) < 1e-18


def test_depth_order_and_index_tiebreak(orc):
    cols = [[1, 0, 0], [0, 1, 0]]
    sc = make_scene([[0, 0, 3.0], [0, 0, 2.0]], [[0.3] * 3] * 2, [[1, 0, 0, 0]] * 2, [0.6, 0.5], cols)
    out = orc.render(sc, camera(32, 32, 100, 100, 16, 16))
    o = 1 / (1 + np.exp(-sc.opacity_logit.astype(np.float64)))
    c = np.maximum(0, sc.sh[:, 0, :].astype(np.float64) * Y00 + 0.5)
    np.testing.assert_allclose(out["rgb"][:, 16, 16], c[1] * o[1] + c[0] * o[0] * (1 - o[1]), atol=1e-14)
    sc2 = make_scene([[0, 0, 2.0], [0, 0, 2.0]], [[0.3] * 3] * 2, [[1, 0, 0, 0]] * 2, [0.6, 0.5], cols)
    out2 = orc.render(sc2, camera(32, 32, 100, 100, 16, 16))
    o2 = 1 / (1 + np.exp(-sc2.opacity_logit.astype(np.float64)))
    np.testing.assert_allclose(out2["rgb"][:, 16, 16], c[0] * o2[0] + c[1] * o2[1] * (1 - o2[0]), atol=1e-14)


def test_tile_subset_matches_full_render(orc):
    from paper_2509_13536_gb300 import scenegen as sg
    sc, cams = sg.workload("box10k")
    full = orc.render(sc, cams[0])
    tiles = np.array([0, 7, 33, 150, 299])
    part = orc.render(sc, cams[0], tiles=tiles)
    for t in tiles:
        ty, tx = divmod(int(t), 20)
        sl = (slice(ty * 16, ty * 16 + 16), slice(tx * 16, tx * 16 + 16))
        np.testing.assert_array_equal(part["alpha"][sl], full["alpha"][sl])
        np.testing.assert_array_equal(part["rgb"][(slice(None),) + sl], full["rgb"][(slice(None),) + sl])


def test_sh_basis_matches_cartesian_forms(orc):
    """The basis at fixed directions equals the textbook Cartesian forms of the real
    orthonormal harmonics, index l^2 + l + m, without the Condon-Shortley phase
    (Y_1,-1 ~ y, Y_1,0 ~ z, Y_1,1 ~ x, ...).  A swapped index or a flipped sign keeps
    the basis orthonormal, so the quadrature pin alone would not see it."""
    pi = math.pi
    forms = {
        0: lambda x, y, z: 0.5 * math.sqrt(1 / pi),
        1: lambda x, y, z: math.sqrt(3 / (4 * pi)) * y,
        2: lambda x, y, z: math.sqrt(3 / (4 * pi)) * z,
        3: lambda x, y, z: math.sqrt(3 / (4 * pi)) * x,
        4: lambda x, y, z: 0.5 * math.sqrt(15 / pi) * x * y,
        5: lambda x, y, z: 0.5 * math.sqrt(15 / pi) * y * z,
        6: lambda x, y, z: 0.25 * math.sqrt(5 / pi) * (3 * z * z - 1),
        7: lambda x, y, z: 0.5 * math.sqrt(15 / pi) * x * z,
        8: lambda x, y, z: 0.25 * math.sqrt(15 / pi) * (x * x - y * y),
        9: lambda x, y, z: 0.25 * math.sqrt(35 / (2 * pi)) * y * (3 * x * x - y * y),
        10: lambda x, y, z: 0.5 * math.sqrt(105 / pi) * x * y * z,
        11: lambda x, y, z: 0.25 * math.sqrt(21 / (2 * pi)) * y * (5 * z * z - 1),
        12: lambda x, y, z: 0.25 * math.sqrt(7 / pi) * z * (5 * z * z - 3),
        13: lambda x, y, z: 0.25 * math.sqrt(21 / (2 * pi)) * x * (5 * z * z - 1),
        14: lambda x, y, z: 0.25 * math.sqrt(105 / pi) * z * (x * x - y * y),
        15: lambda x, y, z: 0.25 * math.sqrt(35 / (2 * pi)) * x * (x * x - 3 * y * y),
    }
    dirs = [(1, 0, 0), (0, 1, 0), (0, 0, 1), (0.48, -0.6, 0.64), (-0.36, 0.48, -0.8)]
    for d in dirs:
        d = np.asarray(d, float) / np.linalg.norm(d)
        Y, _ = orc.sh_basis(3, d)
        want = np.array([forms[k](*d) for k in range(16)])
        np.testing.assert_allclose(Y, want, atol=1e-14)
    # on the axes: Y_1,-1 = Y_1,0 = 0 at +x and only Y_1,1 carries the sign of x
    Yx, _ = orc.sh_basis(1, [1, 0, 0])
    assert Yx[1] == 0 and Yx[2] == 0 and Yx[3] > 0


# ---------------------------------------------------------------- near-tie outcomes
def _o32(sc, i=0):
    return 1 / (1 + math.exp(-float(sc.opacity_logit[i])))


def _c32(sc):
    return np.maximum(0, sc.sh[:, 0, :].astype(np.float64) * Y00 + 0.5)


@pytest.mark.parametrize("sign", [+1, -1])
def test_outcomes_alpha_cutoff_tie(orc, sign):
    """alpha = 1/255 (1 +- 1e-7) at pixel (19, 16), inside the alpha margin: one tie; the
    image takes the FP64 decision and the other outcome the opposite one."""
    f, z, s, W, H = 100.0, 2.0, 0.04, 32, 32
    sig2 = _iso_sigma2(f, math.exp(float(np.float32(math.log(s)))), z)
    o = (1 / 255) * (1 + sign * 1e-7) * math.exp(0.5 * 9.0 / sig2)
    sc = make_scene([[0, 0, z]], [[s, s, s]], [[1, 0, 0, 0]], [o], [[0.2, 0.5, 0.9]])
    out = orc.render_outcomes(sc, camera(W, H, f, f, 16, 16))
    expect = _o32(sc) * math.exp(-0.5 * 9.0 / sig2)
    assert abs(expect * 255 - 1) < 1e-6
    assert out["n_ties"][16, 19] == 1 and out["flags"][16, 19] & 1
    blended, other = (out["alpha"], out["alt_alpha"]) if expect >= 1 / 255 else (out["alt_alpha"], out["alpha"])
    assert abs(blended[16, 19] - expect) < 1e-15 and other[16, 19] == 0.0
    c = _c32(sc)[0]
    alt_rgb = out["alt_rgb"][:, 16, 19]
    np.testing.assert_allclose(alt_rgb, c * out["alt_alpha"][16, 19], atol=1e-15)
    np.testing.assert_allclose(out["alt_depth"][16, 19], z * out["alt_alpha"][16, 19], atol=1e-15)
    # pixels with no tie: the other outcome is the image itself
    free = out["n_ties"] == 0
    np.testing.assert_array_equal(out["alt_alpha"][free], out["alpha"][free])


def test_outcomes_transmittance_stop_tie(orc):
    """Centre-pixel alpha o with (1 - o)^4 = 1e-4 (1 + 1e-7): the FP64 pass does not stop
    after the 4th layer and blends the 5th; the other outcome stops after the 4th."""
    cols = [[1, 0, 0], [0, 1, 0], [0, 0, 1], [1, 1, 0], [0, 1, 1], [1, 0, 1]]
    z = [2.0, 2.5, 3.0, 3.5, 4.0, 4.5]
    n = len(z)
    o = 1 - (1e-4 * (1 + 1e-7)) ** 0.25
    sc = make_scene([[0, 0, zz] for zz in z], [[0.5] * 3] * n, [[1, 0, 0, 0]] * n, [o] * n, cols)
    out = orc.render_outcomes(sc, camera(32, 32, 100, 100, 16, 16))
    o32 = _o32(sc)
    assert abs((1 - o32) ** 4 / 1e-4 - 1) < 5e-6
    c = _c32(sc)
    four = sum(c[k] * o32 * (1 - o32) ** k for k in range(4))
    five = four + c[4] * o32 * (1 - o32) ** 4
    assert out["n_ties"][16, 16] == 1 and out["flags"][16, 16] & 2
    got, alt = out["rgb"][:, 16, 16], out["alt_rgb"][:, 16, 16]
    if (1 - o32) ** 4 >= 1e-4:
        np.testing.assert_allclose(got, five, atol=1e-14)
        np.testing.assert_allclose(alt, four, atol=1e-14)
        assert abs(out["alt_alpha"][16, 16] - (1 - (1 - o32) ** 4)) < 1e-15
    else:
        np.testing.assert_allclose(got, four, atol=1e-14)
        np.testing.assert_allclose(alt, five, atol=1e-14)


def test_outcomes_depth_order_tie(orc):
    """Two Gaussians whose camera depth 2 + 2^-23 is a float32 rounding midpoint: equal
    keys, index order in the image, the swapped order as the other outcome."""
    cols = [[1, 0, 0], [0, 1, 0]]
    sc = make_scene([[0, 0, 2.0], [0, 0, 2.0]], [[0.3] * 3] * 2, [[1, 0, 0, 0]] * 2, [0.6, 0.5], cols)
    cam = camera(32, 32, 100, 100, 16, 16, t=[0, 0, 2.0 ** -23])
    out = orc.render_outcomes(sc, cam)
    o = [_o32(sc, 0), _o32(sc, 1)]
    c = _c32(sc)
    assert out["n_ties"][16, 16] == 1 and out["flags"][16, 16] & 4
    np.testing.assert_allclose(out["rgb"][:, 16, 16], c[0] * o[0] + c[1] * o[1] * (1 - o[0]), atol=1e-14)
    np.testing.assert_allclose(out["alt_rgb"][:, 16, 16], c[1] * o[1] + c[0] * o[0] * (1 - o[1]), atol=1e-14)
    np.testing.assert_allclose(out["alt_alpha"][16, 16], out["alpha"][16, 16], atol=1e-15)


def test_outcomes_extent_tie(orc):
    """A Gaussian whose rect edge u + r sits 1e-3 px short of the tile boundary x = 32:
    pixel (32, 16) is outside its rect in the image and inside it in the other outcome,
    where it takes the Gaussian's alpha o exp(-d^2 / (2 lambda))."""
    f, z, s = 100.0, 2.0, 0.1
    s32 = math.exp(float(np.float32(math.log(s))))
    lam = (f * s32 / z) ** 2 + 0.3
    r = math.ceil(3 * math.sqrt(lam))
    u = 32.0 - r - 1e-3  # on the optical axis: principal point at u
    sc = make_scene([[0, 0, z]], [[s, s, s]], [[1, 0, 0, 0]], [0.9], [[1, 1, 1]])
    cam = camera(64, 32, f, f, u, 16.0)
    p = orc.project(sc, cam)
    edge = p["mean2d"][0, 0] + p["radius"][0]
    assert abs(edge - (32 - 1e-3)) < 1e-5 and p["rect"][0, 2] == 1
    out = orc.render_outcomes(sc, cam)
    assert out["n_ties"][16, 32] == 1 and out["flags"][16, 32] & 8
    assert out["alpha"][16, 32] == 0.0
    d = 32.0 - p["mean2d"][0, 0]
    want = _o32(sc) * math.exp(-0.5 * d * d / lam)
    assert abs(out["alt_alpha"][16, 32] - want) < 1e-12 and want > 1 / 255
    assert out["n_ties"][16, 31] == 0 and out["alpha"][16, 31] > 0


def test_outcomes_agree_with_render_on_a_random_scene(orc):
    """The image of render_outcomes is orc_render's; two or more ties leave NaN."""
    rng = np.random.default_rng(11)
    sc = random_scene(rng, 200, sh_degree=2, spread=1.2, depth=2.5)
    cam = camera(80, 48, 40, 40, 40.3, 23.9)
    wide = orc.margins(alpha_rel=0.05, T_rel=0.05)  # wide margins: many ties, some pixels with two
    a = orc.render(sc, cam, margin=wide)
    b = orc.render_outcomes(sc, cam, margin=wide)
    for k in ("rgb", "depth", "alpha", "flags", "n_contrib"):
        np.testing.assert_array_equal(a[k], b[k])
    many = b["n_ties"] >= 2
    assert np.isnan(b["alt_alpha"][many]).all() and not np.isnan(b["alt_alpha"][~many]).any()
    # every flag but the opacity clamp's marks a tie, and every tie sets a flag
    np.testing.assert_array_equal((b["flags"] & 15) != 0, b["n_ties"] > 0)
    one = b["n_ties"] == 1
    assert one.any() and many.any()
    assert (np.abs(b["alt_alpha"] - b["alpha"])[one] > 0).mean() > 0.5
