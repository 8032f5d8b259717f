"""The oracle's voxel merge against the values Sec. II-D prints (tests/golden/
sec2d_merge_values.txt): the chi-square critical value as a decision boundary and as the
distribution's quantile, the Eq. 3 gradient threshold as a decision boundary, the worked
count of pairs per voxel (every pair of a voxel is examined), and the Eq. 10 defaults."""
import inspect
import os

import numpy as np
import pytest

from paper_2509_13536_gb300 import api
from tests._scenes import make_scene

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sec2d_merge_values.txt")
SIGMA = 0.001   # isotropic scale of the hand-built Gaussians (m)
VOXEL = 0.02


def golden():
    vals = {}
    with open(GOLDEN) as f:
        for line in f:
            line = line.strip()
            if line and not line.startswith("#"):
                name, *rest = line.split()
                vals[name] = rest
    return vals


def _voxel(positions):
    n = len(positions)
    return make_scene(np.asarray(positions), [[SIGMA] * 3] * n, [[1.0, 0.0, 0.0, 0.0]] * n, [0.5] * n,
                      [[0.5, 0.5, 0.5]] * n)


def test_chi2_critical_is_the_chi_square_quantile():
    st = pytest.importorskip("scipy.stats")
    chi2 = float(golden()["chi2_critical"][0])
    assert round(float(st.chi2.ppf(0.95, 3)), 3) == chi2


def test_oracle_merges_below_the_critical_value_only(orc):
    """Two Gaussians at Mahalanobis distance^2 just below / above 7.815 (default chi2)."""
    chi2 = float(golden()["chi2_critical"][0])
    for d2, merged in ((chi2 - 0.015, True), (chi2 + 0.015, False)):
        dist = SIGMA * np.sqrt(d2)
        sc = _voxel([[0.005, 0.01, 0.01], [0.005 + dist, 0.01, 0.01]])
        ref = orc.voxel_merge(sc, VOXEL)
        assert not ref["tie"].any()
        assert (ref["partner"][0] == 1) == merged, (d2, ref["partner"])
        assert ref["n_out"] == (1 if merged else 2)


def test_oracle_gradient_threshold_of_eq3(orc):
    """Identical Gaussians merge only if both mean gradients are below 0.001 (default)."""
    tau = float(golden()["grad_tau"][0])
    sc = _voxel([[0.005, 0.01, 0.01], [0.005, 0.01, 0.01]])
    for g, merged in ((0.9 * tau, True), (1.1 * tau, False)):
        ref = orc.voxel_merge(sc, VOXEL, grad_stat=np.array([g, g]))
        assert (ref["partner"][0] == 1) == merged, g


@pytest.mark.parametrize("n", [2, 3, 4])
def test_every_pair_of_a_voxel_is_examined(orc, n):
    """Members 5 sigma apart (distance^2 25 > chi2) except one pair moved together
    (distance^2 0.25): whichever of the voxel's pairs it is, the oracle finds it, so the
    number of distinct pairs it can find equals the worked count."""
    want = dict(tuple(map(int, p.split(":"))) for p in golden()["pairs_per_voxel"])[n]
    found = set()
    for a in range(n):
        for b in range(a + 1, n):
            pos = [[0.002 + 5 * SIGMA * k, 0.01, 0.01] for k in range(n)]
            pos[b] = [pos[a][0] + 0.5 * SIGMA, 0.01, 0.01]
            ref = orc.voxel_merge(_voxel(pos), VOXEL, greedy=False)
            part = ref["partner"]
            assert not ref["tie"].any()
            assert part[a] == b and part[b] == a, (a, b, part)
            assert (part >= 0).sum() == 2
            found.add((a, b))
    assert len(found) == want == n * (n - 1) // 2


def test_eq10_defaults(orc):
    g = golden()
    sig = inspect.signature(orc.w2_lbfgs).parameters
    assert sig["t"].default == float(g["slerp_t"][0])
    assert tuple(sig["delta"].default) == tuple(float(x) for x in g["delta"])
    for fn in (orc.voxel_merge, api.mgs_voxel_merge):  # the oracle's and the library's defaults
        sig = inspect.signature(fn).parameters
        assert sig["chi2"].default == float(g["chi2_critical"][0])
        assert sig["grad_tau"].default == float(g["grad_tau"][0])
