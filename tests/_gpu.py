"""Helpers of the GPU parity tests: run the library through its C ABI and compare with
the FP64 oracle on the same seeded inputs."""
import numpy as np
import torch

from paper_2509_13536_gb300 import api

FIELDS = ("means", "log_scales", "quats", "opacity_logit", "sh")

# Tolerances: images max-abs 1e-4 on unflagged pixels; gradients 1e-3 relative.  At most
# 1% of the pixels may hold a near-tie decision: the share grows with the number of
# Gaussians a pixel walks (thousands in the 1M-Gaussian room).
IMG_TOL = 1e-4
GRAD_REL = 1e-3
MAX_FLAGGED = 1e-2


def to_np(t):
    return t.detach().float().cpu().numpy().astype(np.float64)


def render_gpu(scene, cams, attr_dtype=torch.float32):
    g = api.Gaussians.from_scene(scene, "cuda", attr_dtype)
    imgs, ws = api.render(g, cams)
    torch.cuda.synchronize()
    return g, imgs, ws


def check_image(img, ref, tol=IMG_TOL, max_flagged=MAX_FLAGGED, what=""):
    ok = ref["flags"] == 0
    frac = 1.0 - ok.mean()
    assert frac <= max_flagged, f"{what}: flagged fraction {frac:.2e}"
    errs = {}
    errs["rgb"] = float(np.abs(to_np(img.rgb) - ref["rgb"])[:, ok].max(initial=0))
    errs["depth"] = float(np.abs(to_np(img.depth) - ref["depth"])[ok].max(initial=0))
    errs["alpha"] = float(np.abs(to_np(img.alpha) - ref["alpha"])[ok].max(initial=0))
    for k, e in errs.items():
        assert e <= tol, f"{what}: {k} max-abs {e:.3e} (flagged {frac:.2e})"
    return errs, frac


def check_grads(grads, ref, taint=None, rel=GRAD_REL, what=""):
    """Per parameter group: relative L2 error over untainted Gaussians <= rel."""
    out = {}
    for k in FIELDS:
        a = to_np(getattr(grads, k))
        b = ref[k]
        if taint is not None:
            m = taint == 0
            a, b = a[m], b[m]
        nb = np.linalg.norm(b)
        e = np.linalg.norm(a - b) / max(nb, 1e-30)
        out[k] = e
        assert e <= rel, f"{what}: {k} relative L2 error {e:.3e}"
    return out


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


def oracle_backward(orc, scene, cams, cot, **kw):
    grads = orc.new_grads(scene.n, scene.sh_degree)
    for c, (gr, gd, ga) in zip(cams, cot):
        orc.render_backward(scene, c, gr, gd, ga, grads=grads, **kw)
    return grads
