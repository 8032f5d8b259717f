"""Parity at the workloads' full sizes, in the launch configuration the benchmark times.

* room300k (300k Gaussians, 640x480, SH0): the whole image and every gradient.
* room1m_sh3 (1M Gaussians, SH3, 8 keyframes at 1200x680, one multi-view launch): the
  GPU renders all views; the oracle renders a seeded sample of tiles per view; the
  cotangent is non-zero only on those tiles, so the oracle's backward over just those
  tiles gives the exact gradient to compare.  Finite differences of the oracle on 64
  random (Gaussian, component) parameters pin the GPU gradient at this size too.
"""
import numpy as np
import pytest
import torch

from paper_2509_13536_gb300 import api, scenegen as sg
from tests import _gpu

pytestmark = [pytest.mark.gpu, pytest.mark.slow]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_13536_gb300 import build
    build.build()


def test_room300k_full_image_and_gradients(orc):
    scene, cams = sg.workload("room300k")
    g, imgs, ws = _gpu.render_gpu(scene, cams)
    ref = orc.render(scene, cams[0])
    errs, frac = _gpu.check_image(imgs[0], ref, what="room300k")
    cot_np, dL = _gpu.cotangents(cams, 5)
    grads = api.render_backward(g, cams, dL, ws)
    torch.cuda.synchronize()
    ref_g = _gpu.oracle_backward(orc, scene, cams, cot_np)
    e = _gpu.check_grads(grads, ref_g, ref_g["taint"], what="room300k")
    print("room300k", errs, "flagged", frac, "grad rel", e)


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
def big():
    scene, cams = sg.workload("room1m_sh3")
    rng = np.random.default_rng(2)
    tiles = [_sampled_tiles(c, 48, rng) for c in cams]
    masks = [_tile_mask(c, t) for c, t in zip(cams, tiles)]
    g = api.Gaussians.from_scene(scene, "cuda")
    imgs, ws = api.render(g, cams)  # all 8 keyframes in one launch, as in the benchmark
    cot_np, dL = [], []
    crng = np.random.default_rng(3)
    for c, m in zip(cams, masks):
        gr = (crng.uniform(-1, 1, (3, c.height, c.width)) * m).astype(np.float32)
        gd = (crng.uniform(-1, 1, (c.height, c.width)) * m).astype(np.float32)
        ga = (crng.uniform(-1, 1, (c.height, c.width)) * m).astype(np.float32)
        cot_np.append((gr, gd, ga))
        dL.append(api.Image(*(torch.from_numpy(x).cuda() for x in (gr, gd, ga))))
    grads = api.render_backward(g, cams, dL, ws)
    torch.cuda.synchronize()
    return dict(scene=scene, cams=cams, tiles=tiles, masks=masks, imgs=imgs, grads=grads, cot=cot_np)


def test_room1m_sampled_tiles_forward(orc, big):
    worst = 0.0
    flagged = total = 0
    bits = {}
    for v, (c, t, m) in enumerate(zip(big["cams"], big["tiles"], big["masks"])):
        ref = orc.render(big["scene"], c, tiles=t)
        ok = (ref["flags"] == 0) & m
        flagged += int(((ref["flags"] != 0) & m).sum())
        for b, nm in enumerate(("alpha", "T", "order", "extent", "clamp")):
            bits[nm] = bits.get(nm, 0) + int(((ref["flags"] >> b) & 1)[m].sum())
        total += int(m.sum())
        im = big["imgs"][v]
        for name, a, b in (("rgb", _gpu.to_np(im.rgb), ref["rgb"]), ("depth", _gpu.to_np(im.depth), ref["depth"]),
                           ("alpha", _gpu.to_np(im.alpha), ref["alpha"])):
            e = float(np.abs(a - b)[..., ok].max())
            worst = max(worst, e)
            assert e <= _gpu.IMG_TOL, f"view {v} {name} max-abs {e:.3e}"
    print("room1m sampled tiles: max-abs", worst, "flagged", flagged, "of", total, "by decision", bits)
    assert flagged <= _gpu.MAX_FLAGGED * total


def test_room1m_sampled_tiles_backward(orc, big):
    ref = orc.new_grads(big["scene"].n, 3)
    for c, t, (gr, gd, ga) in zip(big["cams"], big["tiles"], big["cot"]):
        orc.render_backward(big["scene"], c, gr, gd, ga, tiles=t, grads=ref)
    e = _gpu.check_grads(big["grads"], ref, ref["taint"], what="room1m sampled")
    print("room1m sampled-tile gradients rel", e, "tainted", int(ref["taint"].sum()))


def test_room1m_finite_differences_64_parameters(orc, big):
    """Central differences of the oracle loss (same sparse cotangent) for 64 random
    parameters of Gaussians that reach the sampled tiles, against the GPU gradient.
    The oracle runs on every Gaussian whose tile rect meets a sampled tile: the others
    cannot change those tiles, and dropping them keeps the relative order of the rest.
    The parameters are picked among the untainted Gaussians with a non-zero gradient."""
    scene, cams = big["scene"], big["cams"]
    ref = orc.new_grads(scene.n, 3)
    for c, t, (gr, gd, ga) in zip(cams, big["tiles"], big["cot"]):
        orc.render_backward(scene, c, gr, gd, ga, tiles=t, grads=ref)
    reach = np.zeros(scene.n, bool)
    for c, t in zip(cams, big["tiles"]):
        p = orc.project(scene, c)
        tx = (c.width + 15) // 16
        ty_s, tx_s = np.divmod(t, tx)
        r = p["rect"]
        for yy, xx in zip(ty_s, tx_s):
            reach |= (p["visible"] > 0) & (r[:, 0] <= xx) & (xx <= r[:, 2]) & (r[:, 1] <= yy) & (yy <= r[:, 3])
    idx = np.nonzero(reach)[0]  # every Gaussian binned into a sampled tile stays
    sub = scene.subset(idx)
    eligible = np.nonzero((ref["taint"][idx] == 0) & (np.abs(ref["means"][idx]).sum(1) > 0))[0]
    rng = np.random.default_rng(64)
    fields = ["means", "log_scales", "quats", "opacity_logit", "sh"]
    picks = []
    while len(picks) < 64:
        f = fields[rng.integers(len(fields))]
        gi = int(eligible[rng.integers(len(eligible))])
        shape = getattr(sub, f).shape[1:]
        comp = tuple(int(rng.integers(s)) for s in shape)
        picks.append((f, gi, comp))

    def loss(s):
        L = 0.0
        hashes = []
        for c, t, (gr, gd, ga) in zip(cams, big["tiles"], big["cot"]):
            out = orc.render(s, c, tiles=t, margin=None, hash_decisions=True)
            L += float((gr * out["rgb"]).sum() + (gd * out["depth"]).sum() + (ga * out["alpha"]).sum())
            hashes.append(out["hash"])
        return L, hashes

    base64 = {f: getattr(sub, f).astype(np.float64) for f in fields}
    _, h0 = loss(sub)
    checked = 0
    for f, gi, comp in picks:
        th = base64[f][(gi,) + comp]
        h = 1e-5 * max(1.0, abs(th))
        vals = []
        for sgn in (1, -1):
            p = {k: v.copy() for k, v in base64.items()}
            p[f][(gi,) + comp] = th + sgn * h
            L, hs = loss(sub.__class__(p["means"], p["log_scales"], p["quats"], p["opacity_logit"], p["sh"],
                                       sub.birth, sub.sh_degree))
            vals.append((L, hs))
        if vals[0][1] != h0 or vals[1][1] != h0:
            continue  # a decision moved within +-h: not differentiable here
        fd = (vals[0][0] - vals[1][0]) / (2 * h)
        gpu = float(_gpu.to_np(getattr(big["grads"], f))[(idx[gi],) + comp])
        scale = max(abs(fd), 1e-3 * np.sqrt(np.mean(ref[f][idx] ** 2)))
        assert abs(gpu - fd) <= 2e-3 * scale + 1e-6, (f, int(idx[gi]), comp, gpu, fd)
        checked += 1
    assert checked >= 56
