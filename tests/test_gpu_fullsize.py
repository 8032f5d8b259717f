"""Parity at the workloads' full sizes, in the launch configuration the benchmark times.

* room300k (300k Gaussians, 640x480, SH0): the whole image and every gradient.
* room1m_sh3 (1M Gaussians, SH3, 8 keyframes at 1200x680, one multi-view launch): all
  eight keyframes, every pixel, against the oracle's two outcomes of any near-tie
  decision; every gradient element of all 1M Gaussians with the cotangent U[-1, 1] on
  the pixels the oracle does not flag.  Finite differences of the oracle on 64 random
  (Gaussian, component) parameters pin the GPU gradient at this size too.
"""
import warnings

import numpy as np
import pytest
import torch

from paper_2509_13536_gb300 import api, scenegen as sg
from tests import _gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


class ParityReport(UserWarning):
    """Counts of a full-size parity test, shown in the run's warnings summary."""


def _report(what, **kv):
    msg = what + ": " + ", ".join(f"{k} {v:.3g}" if isinstance(v, float) else f"{k} {v}" for k, v in kv.items())
    print(msg)
    warnings.warn(ParityReport(msg))


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_13536_gb300 import build
    build.build()


def _grad_summary(e):
    f = _gpu.FIELDS
    return dict(grad_rel_max=max(e[k] for k in f), grad_elem_ratio_max=max(e[k + "_elem"] for k in f),
                beyond_literal=sum(e.get(k + "_beyond_literal", 0) for k in f),
                max_of_error_model=max(e.get(k + "_of_model", 0.0) for k in f))


def _sum_reports(reps):
    out = {}
    for r in reps:
        for k, v in r.items():
            out[k] = max(out.get(k, 0.0), v) if k in ("rgb", "depth", "alpha") else out.get(k, 0) + v
    return out


def test_room300k_full_image_and_gradients(orc):
    scene, cams = sg.workload("room300k")
    g, imgs, ws = _gpu.render_gpu(scene, cams)
    ref = orc.render_outcomes(scene, cams[0])
    rep = _gpu.check_image(imgs[0], ref, what="room300k")
    cot_np, dL = _gpu.masked_cotangents(cams, [ref], 5)
    grads = api.render_backward(g, cams, dL, ws)
    torch.cuda.synchronize()
    ref_g = _gpu.oracle_backward(orc, scene, cams, cot_np)
    e = _gpu.check_grads(grads, ref_g, what="room300k")
    _report("room300k", **rep, **_grad_summary(e))


def _sampled_tiles(cam, n, rng):
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    return np.sort(rng.choice(tx * ty, n, replace=False)).astype(np.int32)


def _tile_mask(cam, tiles):
    tx = (cam.width + 15) // 16
    m = np.zeros((cam.height, cam.width), bool)
    for t in tiles:
        y, x = divmod(int(t), tx)
        m[y * 16:y * 16 + 16, x * 16:x * 16 + 16] = True
    return m


@pytest.fixture(scope="module")
def big(orc):
    scene, cams = sg.workload("room1m_sh3")
    g = api.Gaussians.from_scene(scene, "cuda")
    imgs, ws = api.render(g, cams)  # all 8 keyframes in one launch, as in the benchmark
    torch.cuda.synchronize()
    refs = [orc.render_outcomes(scene, c) for c in cams]
    cot_np, dL = _gpu.masked_cotangents(cams, refs, 3)
    grads = api.render_backward(g, cams, dL, ws)
    torch.cuda.synchronize()
    return dict(scene=scene, cams=cams, g=g, ws=ws, imgs=imgs, refs=refs, grads=grads, cot=cot_np)


def test_room1m_whole_keyframes_forward(big):
    """All 8 keyframes, every pixel: no-tie pixels within 1e-4 of the oracle's image,
    one-tie pixels within 1e-4 of one of its two outcomes, the rest counted."""
    reps = [_gpu.check_image(big["imgs"][v], big["refs"][v], what=f"room1m view {v}") for v in range(len(big["cams"]))]
    tot = _sum_reports(reps)
    flagged = sum(int((r["flags"] != 0).sum()) for r in big["refs"])
    _report("room1m 8 whole keyframes", **tot, flagged_pixels=flagged)


def test_room1m_whole_keyframes_backward(orc, big):
    """Every gradient element of all 1M Gaussians (no Gaussian excluded), summed over
    the 8 keyframes: relative L2 <= 1e-3 per group and |d| <= 1e-3 (|ref| + 1e-3 rms)."""
    ref = _gpu.oracle_backward(orc, big["scene"], big["cams"], big["cot"])
    e = _gpu.check_grads(big["grads"], ref, what="room1m 8 keyframes")
    np.testing.assert_allclose(_gpu.to_np(big["grads"].vis_count), ref["vis_count"])
    drawn = int((ref["vis_count"] > 0).sum())
    _report("room1m 8 keyframes gradients", gaussians_drawn=drawn, **_grad_summary(e))


def _richardson(f, th, h):
    """Central difference with one Richardson step: O(h^4) truncation."""
    d1 = (f(th + h) - f(th - h)) / (2 * h)
    d2 = (f(th + h / 2) - f(th - h / 2)) / h
    return (4 * d2 - d1) / 3


def test_room1m_finite_differences_64_parameters(orc, big):
    """Central differences (one Richardson step) of the oracle loss on a seeded sample of
    48 tiles per keyframe, for 64 random parameters of Gaussians that reach those
    tiles, against the GPU gradient of the same sparse cotangent: |gpu - fd| within the
    element-wise gradient bound plus the differences' own float64 rounding noise.  The oracle runs on every Gaussian whose tile rect meets
    a sampled tile: the others cannot change those tiles, and dropping them keeps the
    relative order of the rest.  A pick whose decisions move within +-h (decision hash)
    is not differentiable there and is skipped; at most 8 may be."""
    scene, cams = big["scene"], big["cams"]
    rng = np.random.default_rng(2)
    tiles = [_sampled_tiles(c, 48, rng) for c in cams]
    masks = [_tile_mask(c, t) for c, t in zip(cams, tiles)]
    crng = np.random.default_rng(3)
    cot, dL = [], []
    for c, m in zip(cams, masks):
        gr = (crng.uniform(-1, 1, (3, c.height, c.width)) * m).astype(np.float32)
        gd = (crng.uniform(-1, 1, (c.height, c.width)) * m).astype(np.float32)
        ga = (crng.uniform(-1, 1, (c.height, c.width)) * m).astype(np.float32)
        cot.append((gr, gd, ga))
        dL.append(api.Image(*(torch.from_numpy(x).cuda() for x in (gr, gd, ga))))
    grads = api.render_backward(big["g"], cams, dL, big["ws"])  # same saved forward state
    torch.cuda.synchronize()
    ref = orc.new_grads(scene.n, 3, scale=True)
    for c, t, (gr, gd, ga) in zip(cams, tiles, cot):
        orc.render_backward(scene, c, gr, gd, ga, tiles=t, grads=ref)
    # the GPU gradient of this sparse cotangent against the oracle's, on the Gaussians
    # that reach no flagged pixel of the sampled tiles
    _gpu.check_grads(grads, ref, ref["taint"], what="room1m sampled tiles")
    reach = np.zeros(scene.n, bool)
    for c, t in zip(cams, tiles):
        p = orc.project(scene, c)
        tx = (c.width + 15) // 16
        ty_s, tx_s = np.divmod(t, tx)
        r = p["rect"]
        for yy, xx in zip(ty_s, tx_s):
            reach |= (p["visible"] > 0) & (r[:, 0] <= xx) & (xx <= r[:, 2]) & (r[:, 1] <= yy) & (yy <= r[:, 3])
    idx = np.nonzero(reach)[0]  # every Gaussian binned into a sampled tile stays
    sub = scene.subset(idx)
    eligible = np.nonzero((ref["taint"][idx] == 0) & (np.abs(ref["means"][idx]).sum(1) > 0))[0]
    prng = np.random.default_rng(64)
    fields = ["means", "log_scales", "quats", "opacity_logit", "sh"]
    picks = []
    while len(picks) < 64:
        f = fields[prng.integers(len(fields))]
        gi = int(eligible[prng.integers(len(eligible))])
        shape = getattr(sub, f).shape[1:]
        comp = tuple(int(prng.integers(s)) for s in shape)
        picks.append((f, gi, comp))

    def loss(s, with_abs=False):
        L = A = 0.0
        hashes = []
        for c, t, (gr, gd, ga) in zip(cams, tiles, cot):
            out = orc.render(s, c, tiles=t, margin=None, hash_decisions=True)
            L += float((gr * out["rgb"]).sum() + (gd * out["depth"]).sum() + (ga * out["alpha"]).sum())
            if with_abs:
                A += float(np.abs(gr * out["rgb"]).sum() + np.abs(gd * out["depth"]).sum() +
                           np.abs(ga * out["alpha"]).sum())
            hashes.append(out["hash"])
        return (L, hashes, A) if with_abs else (L, hashes)

    base64 = {f: getattr(sub, f).astype(np.float64) for f in fields}
    _, h0, L_abs = loss(sub, with_abs=True)
    # rounding noise of the float64 loss (a few units of 2^-53 of the sum of |terms|)
    # divided by the steps: what the differences cannot resolve
    err_L = 8 * 2.0 ** -53 * L_abs
    checked, skipped, worst = 0, 0, 0.0
    for f, gi, comp in picks:
        th0 = base64[f][(gi,) + comp]
        h = 1e-5 * max(1.0, abs(th0))
        moved = [False]

        def at(th):
            p = {k: v.copy() for k, v in base64.items()}
            p[f][(gi,) + comp] = th
            L, hs = loss(sub.__class__(p["means"], p["log_scales"], p["quats"], p["opacity_logit"], p["sh"],
                                       sub.birth, sub.sh_degree))
            moved[0] |= hs != h0
            return L

        fd = _richardson(at, th0, h)
        if moved[0]:
            skipped += 1
            continue
        gpu = float(_gpu.to_np(getattr(grads, f))[(idx[gi],) + comp])
        lit = 1e-3 * max(abs(fd), 1e-3 * np.sqrt(np.mean(ref[f][idx] ** 2)))
        bound = max(lit, _gpu.ERR_SAFETY * float(ref["scale_" + f][(idx[gi],) + comp])) + 12 * err_L / h
        worst = max(worst, abs(gpu - fd) / bound)
        assert abs(gpu - fd) <= bound, (f, int(idx[gi]), comp, gpu, fd, lit, bound)
        checked += 1
    _report("room1m finite differences", checked=checked, skipped=skipped, worst_rel=worst)
    assert skipped <= 8
