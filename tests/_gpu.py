"""Helpers of the GPU parity tests: run the library through its C ABI and compare with
the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

from paper_2509_13536_gb300 import api

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")

# Tolerances: images max-abs 1e-4; gradients 1e-3 relative (per parameter group in L2,
# and per element |d| <= 1e-3 (|ref| + 1e-3 rms of the group)).  A pixel with one
# near-tie decision must match one of the oracle's two outcomes of it; pixels with two
# or more are not enumerated and are counted instead (at most 1e-3 of the pixels).
IMG_TOL = 1e-4
GRAD_REL = 1e-3
MAX_FLAGGED = 1e-2
MAX_UNCHECKED = 1e-3


def to_np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def render_gpu(scene, cams, attr_dtype=torch.float32):
    g = api.Gaussians.from_scene(scene, "cuda", attr_dtype)
    imgs, ws = api.render(g, cams)
    torch.cuda.synchronize()
    return g, imgs, ws


def _planes(rgb, depth, alpha):
    return np.concatenate([rgb, depth[None], alpha[None]], 0)


def check_image(img, ref, tol=IMG_TOL, mask=None, what=""):
    """GPU image against the oracle.  With the oracle's outcomes (``render_outcomes``):
    pixels without a near-tie match its image, pixels with one match either outcome of
    that decision (all five planes together), pixels with two or more are counted.
    With a plain ``render``: only unflagged pixels are compared."""
    gpu = _planes(to_np(img.rgb), to_np(img.depth), to_np(img.alpha))
    prim = _planes(ref["rgb"], ref["depth"], ref["alpha"])
    sel = np.ones(gpu.shape[1:], bool) if mask is None else mask
    e_prim = np.abs(gpu - prim).max(0)
    rep = {}
    if "n_ties" in ref:
        nt = ref["n_ties"]
        alt = _planes(ref["alt_rgb"], ref["alt_depth"], ref["alt_alpha"])
        e_alt = np.nan_to_num(np.abs(gpu - alt).max(0), nan=np.inf)
        zero, one, many = sel & (nt == 0), sel & (nt == 1), sel & (nt >= 2)
        rep["tie_pixels"] = int(one.sum())
        rep["tie_pixels_other_outcome"] = int((one & (e_prim > tol) & (e_alt <= tol)).sum())
        rep["unchecked_pixels"] = int(many.sum())
        worst_tie = float(np.minimum(e_prim, e_alt)[one].max(initial=0))
        assert worst_tie <= tol, f"{what}: a one-tie pixel matches neither outcome (max-abs {worst_tie:.3e})"
        assert many.sum() <= MAX_UNCHECKED * sel.sum(), f"{what}: {int(many.sum())} pixels with >= 2 ties"
        ok = zero
    else:
        ok = sel & (ref["flags"] == 0)
        frac = 1.0 - ok.sum() / max(1, sel.sum())
        assert frac <= MAX_FLAGGED, f"{what}: flagged fraction {frac:.2e}"
    errs = {"rgb": float(np.abs(gpu[0:3] - prim[0:3]).max(0)[ok].max(initial=0)),
            "depth": float(np.abs(gpu[3] - prim[3])[ok].max(initial=0)),
            "alpha": float(np.abs(gpu[4] - prim[4])[ok].max(initial=0))}
    for k, e in errs.items():
        assert e <= tol, f"{what}: {k} max-abs {e:.3e} ({rep})"
    rep.update(errs)
    rep["pixels"] = int(sel.sum())
    return rep


EPS32 = 2.0 ** -24
# The oracle models the float32 error of each gradient element (``scale_<field>``):
# every per-pixel term in absolute value times the relative error it may carry (the
# alpha and T margins of its pixel, plus 32 units of 2^-24 for the sums), carried
# through the chain rule in running-error arithmetic.  An element passes when it is
# within the literal bound 1e-3 (|ref| + 1e-3 rms) or within ERR_SAFETY x that model.
ERR_SAFETY = 2.0


def check_grads(grads, ref, taint=None, rel=GRAD_REL, elem=GRAD_REL, what=""):
    """Per parameter group: relative L2 error <= rel and, per element,
    |gpu - ref| <= max(elem (|ref| + 1e-3 rms(ref)), ERR_SAFETY x modelled error) over the
    untainted Gaussians (all of them when ``taint`` is None); the second term only
    when the oracle reported the element scales.  Returns the errors, the largest
    ratio to the bound, and how many elements needed the scale term.  ``elem`` None
    skips the element-wise bound."""
    out = {}
    for k in FIELDS:
        a = to_np(getattr(grads, k))
        b = ref[k]
        sc = ref.get("scale_" + k)
        if taint is not None:
            m = taint == 0
            a, b = a[m], b[m]
            sc = None if sc is None else sc[m]
        nb = np.linalg.norm(b)
        e = np.linalg.norm(a - b) / max(nb, 1e-30)
        out[k] = e
        assert e <= rel, f"{what}: {k} relative L2 error {e:.3e}"
        if elem is not None and b.size:
            rms = float(np.sqrt(np.mean(b * b)))
            d = np.abs(a - b)
            lit = elem * (np.abs(b) + 1e-3 * rms)
            bound = lit if sc is None else np.maximum(lit, ERR_SAFETY * sc)
            r = d / np.maximum(bound, 1e-300)
            i = int(np.argmax(r))
            out[k + "_elem"] = float(r.flat[i])
            out[k + "_beyond_literal"] = int((d > lit).sum())
            if sc is not None:
                out[k + "_of_model"] = float((d / np.maximum(sc, 1e-300))[d > lit].max(initial=0))
            assert r.flat[i] <= 1.0, (f"{what}: {k} element {np.unravel_index(i, b.shape)} gpu {a.flat[i]:.9e} "
                                      f"ref {b.flat[i]:.9e} (literal bound {lit.flat[i]:.3e}, scale "
                                      f"{(sc.flat[i] if sc is not None else 0):.3e}, rms {rms:.3e})")
    return out


def masked_cotangents(cams, refs, seed):
    """dL/d(rgb, depth, alpha) ~ U[-1,1] per view, zero at every pixel the oracle flags
    (any near-tie decision, the opacity clamp included).  A flagged pixel then adds
    nothing to any gradient, so every Gaussian's gradient is comparable."""
    rng = np.random.default_rng(seed)
    np_list, dev = [], []
    for c, r in zip(cams, refs):
        H, W = c.height, c.width
        keep = (r["flags"] == 0).astype(np.float32)
        gr = (rng.uniform(-1, 1, (3, H, W)) * keep).astype(np.float32)
        gd = (rng.uniform(-1, 1, (H, W)) * keep).astype(np.float32)
        ga = (rng.uniform(-1, 1, (H, W)) * keep).astype(np.float32)
        np_list.append((gr, gd, ga))
        dev.append(api.Image(torch.from_numpy(gr).cuda(), torch.from_numpy(gd).cuda(), torch.from_numpy(ga).cuda()))
    return np_list, dev


def cotangents(cams, seed):
    """dL/d(rgb, depth, alpha) ~ U[-1,1] per view (numpy and device copies)."""
    rng = np.random.default_rng(seed)
    np_list, dev = [], []
    for c in cams:
        H, W = c.height, c.width
        gr = rng.uniform(-1, 1, (3, H, W)).astype(np.float32)
        gd = rng.uniform(-1, 1, (H, W)).astype(np.float32)
        ga = rng.uniform(-1, 1, (H, W)).astype(np.float32)
        np_list.append((gr, gd, ga))
        dev.append(api.Image(torch.from_numpy(gr).cuda(), torch.from_numpy(gd).cuda(), torch.from_numpy(ga).cuda()))
    return np_list, dev


def oracle_backward(orc, scene, cams, cot, scale=True, **kw):
    grads = orc.new_grads(scene.n, scene.sh_degree, scale=scale)
    for c, (gr, gd, ga) in zip(cams, cot):
        orc.render_backward(scene, c, gr, gd, ga, grads=grads, **kw)
    return grads
