"""Pins of the oracle's voxel merge (Sec. II-D, Eq. 3-10) and Adam (no GPU)."""
import itertools
import math

import numpy as np
import pytest

from tests._scenes import make_scene


def _spd(rng, scale=0.05):
    q = rng.normal(size=4)
    s = np.exp(rng.uniform(math.log(scale / 5), math.log(scale), 3))
    return q, s


def test_voxel_keys_float32_quotient(orc):
    rng = np.random.default_rng(0)
    m = rng.uniform(-3, 5, (5000, 3)).astype(np.float32)
    m[:10] = np.float32(0.02) * np.arange(10, dtype=np.float32)[:, None]  # exact multiples
    v = np.float32(0.02)
    want = np.floor(m / v).astype(np.int32)  # IEEE float32 division, correctly rounded
    np.testing.assert_array_equal(orc.voxel_keys(m, v), want)


def test_merge_mean_closed_form(orc):
    """Eq. 6 is the stationary point of Eq. 5: Si^-1 (mk - mi) + Sj^-1 (mk - mj) = 0; special cases."""
    rng = np.random.default_rng(1)
    for _ in range(20):
        Si = orc.covariance(*_spd(rng))
        Sj = orc.covariance(*_spd(rng))
        mi, mj = rng.normal(size=3) * 0.01, rng.normal(size=3) * 0.01
        mk = orc.merge_mean(Si, mi, Sj, mj)
        r = np.linalg.solve(Si, mk - mi) + np.linalg.solve(Sj, mk - mj)
        assert np.abs(r).max() < 1e-9 * np.abs(np.linalg.solve(Si, mi - mj)).max()
        np.testing.assert_allclose(orc.merge_mean(Si, mi, Si, mj), 0.5 * (mi + mj), atol=1e-15)
        np.testing.assert_allclose(orc.merge_mean(Si, mi, Sj, mi), mi, atol=1e-15)


def _sqrtm(S):
    w, V = np.linalg.eigh(S)
    return V @ np.diag(np.sqrt(w)) @ V.T


def test_w2_closed_form_eq8(orc):
    rng = np.random.default_rng(2)
    for _ in range(10):
        A = orc.covariance(*_spd(rng))
        B = orc.covariance(*_spd(rng))
        Ah = _sqrtm(A)
        want = np.trace(A + B - 2 * _sqrtm(Ah @ B @ Ah))
        assert abs(orc.w2_sq(A, B) - want) < 1e-12 * np.trace(A + B)
        # commuting case: ||A^1/2 - D^1/2||_F^2
        w, V = np.linalg.eigh(A)
        D = V @ np.diag(rng.uniform(1e-4, 1e-2, 3)) @ V.T
        want = np.linalg.norm(_sqrtm(A) - _sqrtm(D)) ** 2
        assert abs(orc.w2_sq(A, D) - want) < 1e-12 * np.trace(A + D)


def test_barycentre_properties(orc):
    """Eq. 9 closed form: equal inputs, commuting inputs, fixed-point equation, optimality."""
    rng = np.random.default_rng(3)
    for _ in range(20):
        Si = orc.covariance(*_spd(rng))
        Sj = orc.covariance(*_spd(rng))
        np.testing.assert_allclose(orc.w2_barycentre(Si, Si), Si, rtol=1e-11, atol=1e-17)
        w, V = np.linalg.eigh(Si)
        Sc = V @ np.diag(rng.uniform(1e-4, 1e-2, 3)) @ V.T
        half = 0.5 * (_sqrtm(Si) + _sqrtm(Sc))
        np.testing.assert_allclose(orc.w2_barycentre(Si, Sc), half @ half, rtol=1e-9, atol=1e-16)
        Sk = orc.w2_barycentre(Si, Sj)
        Kh = _sqrtm(Sk)
        fp = 0.5 * (_sqrtm(Kh @ Si @ Kh) + _sqrtm(Kh @ Sj @ Kh))
        np.testing.assert_allclose(fp, Sk, rtol=1e-9, atol=1e-12 * np.abs(Sk).max())
        f0 = orc.w2_sq(Sk, Si) + orc.w2_sq(Sk, Sj)
        for _ in range(5):
            E = rng.normal(size=(3, 3)); E = 0.5 * (E + E.T) * 1e-3 * np.abs(Sk).max()
            P = Sk + E
            if np.linalg.eigvalsh(P).min() <= 0:
                continue
            assert orc.w2_sq(P, Si) + orc.w2_sq(P, Sj) >= f0 - 1e-18


def test_lbfgs_from_eq10_init_reaches_closed_form(orc):
    """The paper's solver (L-BFGS over q, s from the slerp / mean-scale + delta start of
    Eq. 10) converges to the closed-form barycentre."""
    rng = np.random.default_rng(4)
    for _ in range(10):
        qi, si = _spd(rng)
        qj = qi + rng.normal(size=4) * 0.3
        sj = si * np.exp(rng.normal(size=3) * 0.2)
        res = orc.w2_lbfgs(qi, si, qj, sj)
        want = orc.w2_barycentre(orc.covariance(qi, si), orc.covariance(qj, sj))
        rel = np.linalg.norm(res["S"] - want) / np.linalg.norm(want)
        assert rel < 1e-7, (rel, res["iters"])


def _voxel_scene(rng, n_vox, per_vox, v=0.02, sh_degree=0):
    means, scales, quats = [], [], []
    for k in range(n_vox):
        base = (np.array([k % 7, (k // 7) % 5, k // 35]) + 0.5) * v
        for _ in range(per_vox):
            means.append(base + rng.uniform(-0.3, 0.3, 3) * v)
            scales.append(np.exp(rng.uniform(math.log(0.004), math.log(0.02), 3)))
            quats.append(rng.normal(size=4))
    n = len(means)
    op = rng.uniform(0.1, 0.9, n)
    cols = rng.random((n, 3))
    birth = rng.permutation(n)
    return make_scene(means, scales, quats, op, cols, sh_degree, birth=birth)


def _reference_pairs(sc, v, chi2=7.815, greedy=True):
    """Independent restatement: keys by numpy float32 division, Eq. 4 with np.linalg.inv."""
    keys = np.floor(sc.means / np.float32(v)).astype(np.int64)
    n = sc.n
    mu = sc.means.astype(np.float64)
    s = np.exp(sc.log_scales.astype(np.float64))
    covs = []
    for i in range(n):
        q = sc.quats[i].astype(np.float64); q /= np.linalg.norm(q)
        w, x, y, z = q
        R = np.array([[1 - 2 * (y * y + z * z), 2 * (x * y - w * z), 2 * (x * z + w * y)],
                      [2 * (x * y + w * z), 1 - 2 * (x * x + z * z), 2 * (y * z - w * x)],
                      [2 * (x * z - w * y), 2 * (y * z + w * x), 1 - 2 * (x * x + y * y)]])
        covs.append(R @ np.diag(s[i] ** 2) @ R.T)
    groups = {}
    for i in range(n):
        groups.setdefault(tuple(keys[i]), []).append(i)
    partner = -np.ones(n, np.int64)
    n_pairs_evaluated = 0
    for mem in groups.values():
        mem = sorted(mem, key=lambda i: (int(sc.birth[i]), i))
        cands = []
        for a, b in itertools.combinations(range(len(mem)), 2):
            i, j = mem[a], mem[b]
            d = mu[j] - mu[i]
            d2 = d @ np.linalg.inv(covs[i]) @ d
            n_pairs_evaluated += 1
            if d2 < chi2:
                cands.append((d2, int(sc.birth[i]), int(sc.birth[j]), i, j))
        cands.sort()
        for c in cands:
            if partner[c[3]] < 0 and partner[c[4]] < 0:
                partner[c[3]], partner[c[4]] = c[4], c[3]
                if not greedy:
                    break
    return partner, n_pairs_evaluated, groups


@pytest.mark.parametrize("greedy", [True, False])
def test_merge_pairs_match_independent_restatement(orc, greedy):
    rng = np.random.default_rng(6)
    sc = _voxel_scene(rng, 60, 5)
    out = orc.voxel_merge(sc, 0.02, greedy=greedy)
    want, n_pairs, groups = _reference_pairs(sc, 0.02, greedy=greedy)
    np.testing.assert_array_equal(out["partner"], want)
    assert n_pairs == sum(len(g) * (len(g) - 1) // 2 for g in groups.values())
    assert (want >= 0).sum() > 10
    assert out["n_out"] == sc.n - (want >= 0).sum() // 2
    if not greedy:
        for mem in groups.values():
            assert (want[mem] >= 0).sum() <= 2


def test_merge_outputs_follow_eq6_eq9_and_inherit_from_older(orc):
    rng = np.random.default_rng(7)
    sc = _voxel_scene(rng, 40, 4, sh_degree=1)
    out = orc.voxel_merge(sc, 0.02)
    part = out["partner"]
    keep = [i for i in range(sc.n) if not (part[i] >= 0 and (int(sc.birth[part[i]]), part[i]) < (int(sc.birth[i]), i))]
    assert len(keep) == out["n_out"]
    for w, i in enumerate(keep):
        assert out["birth"][w] == sc.birth[i]
        np.testing.assert_array_equal(out["sh"][w], sc.sh[i].astype(np.float64))
        assert out["opacity_logit"][w] == np.float64(sc.opacity_logit[i])
        Si = orc.covariance(sc.quats[i], np.exp(sc.log_scales[i].astype(np.float64)))
        j = part[i]
        if j < 0:
            np.testing.assert_allclose(out["cov"][w], Si[[0, 0, 0, 1, 1, 2], [0, 1, 2, 1, 2, 2]], rtol=1e-12)
            continue
        Sj = orc.covariance(sc.quats[j], np.exp(sc.log_scales[j].astype(np.float64)))
        Sk = orc.w2_barycentre(Si, Sj)
        np.testing.assert_allclose(out["means"][w], orc.merge_mean(Si, sc.means[i], Sj, sc.means[j]), rtol=1e-12)
        S_out = orc.covariance(out["quats"][w], np.exp(out["log_scales"][w]))
        np.testing.assert_allclose(S_out, Sk, rtol=1e-9, atol=1e-15)
        assert out["quats"][w][0] >= 0
        assert np.all(np.diff(out["log_scales"][w]) <= 0)  # scales descending


def test_merge_permutation_invariant(orc):
    rng = np.random.default_rng(8)
    sc = _voxel_scene(rng, 50, 4)
    a = orc.voxel_merge(sc, 0.02)
    perm = rng.permutation(sc.n)
    b = orc.voxel_merge(sc.subset(perm), 0.02)
    oa, ob = np.argsort(a["birth"]), np.argsort(b["birth"])
    for k in ("means", "log_scales", "opacity_logit", "cov", "birth"):
        np.testing.assert_allclose(a[k][oa], b[k][ob], rtol=1e-12, atol=0)


def test_merge_mask_eq3(orc):
    rng = np.random.default_rng(9)
    sc = _voxel_scene(rng, 40, 4)
    gs = rng.uniform(0, 2e-3, sc.n)
    kf = rng.integers(0, 10, sc.n)
    out = orc.voxel_merge(sc, 0.02, grad_stat=gs, grad_tau=1e-3, kf_id=kf, kf_min=2, kf_max=7)
    elig = (gs.astype(np.float64) < np.float32(1e-3)) & (kf >= 2) & (kf <= 7)
    assert np.all(out["partner"][~elig] == -1)
    assert (out["partner"][elig] >= 0).any()


def test_merge_mask_eq3_from_sums(orc):
    """Eq. 3 with the statistic given as sums over the drawing views: the mask tests the
    mean (float32 quotient); a Gaussian drawn in no view has mean 0.  Same mask as the
    precomputed mean."""
    rng = np.random.default_rng(19)
    sc = _voxel_scene(rng, 40, 4)
    cnt = rng.integers(0, 6, sc.n).astype(np.float32)
    mean = rng.uniform(0, 2e-3, sc.n).astype(np.float32)
    sums = (mean * cnt).astype(np.float32)
    ref_mean = np.where(cnt > 0, (sums.astype(np.float64) / np.maximum(cnt, 1)).astype(np.float32), 0)
    a = orc.voxel_merge(sc, 0.02, grad_stat=sums, vis_count=cnt, grad_tau=1e-3)
    b = orc.voxel_merge(sc, 0.02, grad_stat=ref_mean, grad_tau=1e-3)
    np.testing.assert_array_equal(a["partner"], b["partner"])
    elig = ref_mean < np.float32(1e-3)
    assert np.all(a["partner"][~elig] == -1) and (a["partner"][elig] >= 0).any()
    assert (cnt == 0).any() and np.all(a["partner"][(cnt == 0)] >= -1)


def test_adam_step_one_closed_form(orc):
    rng = np.random.default_rng(10)
    p0 = rng.normal(size=100)
    g = rng.normal(size=100)
    p, m, v = p0.copy(), np.zeros(100), np.zeros(100)
    orc.adam(p, g, m, v, 1e-3, 0.9, 0.999, 1e-8, 1)
    np.testing.assert_allclose(p, p0 - 1e-3 * g / (np.abs(g) + 1e-8), rtol=0, atol=1e-15)


def test_adam_matches_torch(orc):
    torch = pytest.importorskip("torch")
    rng = np.random.default_rng(11)
    p0 = rng.normal(size=50)
    p, m, v = p0.copy(), np.zeros(50), np.zeros(50)
    tp = torch.tensor(p0, dtype=torch.float64, requires_grad=True)
    opt = torch.optim.Adam([tp], lr=1e-3, betas=(0.9, 0.999), eps=1e-8)
    for step in range(1, 8):
        g = rng.normal(size=50)
        orc.adam(p, g, m, v, 1e-3, 0.9, 0.999, 1e-8, step)
        tp.grad = torch.tensor(g, dtype=torch.float64)
        opt.step()
    np.testing.assert_allclose(p, tp.detach().numpy(), rtol=1e-12, atol=1e-15)
