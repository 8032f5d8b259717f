"""ctypes front of the FP64 oracle (``oracle.cpp``).

TEST INFRASTRUCTURE ONLY: imported by the tests, the smoke check and the
benchmark's CPU-baseline leg.  The product path never imports this module.

Inputs are the float32 arrays of a ``scenegen.Scene`` / ``scenegen.Camera``;
they are widened exactly to float64 and every computation runs in float64.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

# Margins below which a discrete decision counts as a near-tie; see orc_margins.  The
# float32 kernels' exponent is off by up to ~(sqrt(gamma kappa) + kappa) units of 2^-24
# relative, in the worst direction (measured for the projection: median 0.6, 99.9th
# percentile 6.9, largest 10.6 x sqrt(gamma kappa)), so cond_rel is 8 x 2^-24; ex2
# and the opacity add ~1e-6 (alpha_rel); T is a product of float32 factors (T_rel
# plus the accumulated alpha margins); the extent margins exceed the error of the
# float32 centre (~1e-4 px) and of 3 sqrt(lambda_max).
DEFAULT_MARGINS = dict(alpha_rel=2e-6, T_rel=5e-6, depth_rel=1e-12, extent_px=2e-3,
                       radius_abs=2e-4, near_rel=1e-5, clamp_rel=1e-5, cond_rel=8 * 2.0 ** -24)


def build(force: bool = False) -> str:
    """Compile liboracle.so with the host compiler (plain C++17, no CUDA)."""
    src = os.path.join(HERE, "oracle.cpp")
    hdr = os.path.join(HERE, "oracle.h")
    os.makedirs(BUILD, exist_ok=True)
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(src), os.path.getmtime(hdr))):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call(["g++", "-O2", "-std=c++17", "-ffp-contract=off", "-shared", "-fPIC", "-pthread",
                           src, "-o", tmp])
    os.replace(tmp, LIB)
    return LIB


class Camera(C.Structure):
    _fields_ = [("R", C.c_double * 9), ("t", C.c_double * 3), ("fx", C.c_double),
                ("fy", C.c_double), ("cx", C.c_double), ("cy", C.c_double),
                ("near_z", C.c_double), ("width", C.c_int32), ("height", C.c_int32)]


class Gaussians(C.Structure):
    _fields_ = [("n", C.c_int64), ("sh_degree", C.c_int32), ("means", C.c_void_p),
                ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("opacity_logit", C.c_void_p), ("sh", C.c_void_p)]


class Margins(C.Structure):
    _fields_ = [(k, C.c_double) for k in ("alpha_rel", "T_rel", "depth_rel", "extent_px",
                                          "radius_abs", "near_rel", "clamp_rel", "cond_rel")]


class Projection(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in ("mean2d", "conic", "cov2d", "rgb", "depth", "opacity",
                                          "radius", "rect", "visible")]


GRAD_KEYS = ("means", "log_scales", "quats", "opacity_logit", "sh", "grad2d", "taint", "grad_stat", "vis_count",
             "scale_means", "scale_log_scales", "scale_quats", "scale_opacity_logit", "scale_sh")


class Grads(C.Structure):
    _fields_ = [(k, C.c_void_p) for k in GRAD_KEYS]


class MergeParams(C.Structure):
    _fields_ = [("chi2", C.c_double), ("grad_tau", C.c_double), ("kf_min", C.c_int32),
                ("kf_max", C.c_int32), ("grad_stat", C.c_void_p), ("kf_id", C.c_void_p),
                ("vis_count", C.c_void_p), ("greedy", C.c_int32)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            _lib = C.CDLL(build())
            _lib.orc_w2_sq.restype = C.c_double
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _f64(a):
    return np.ascontiguousarray(a, dtype=np.float64)


class _Params:
    """float64 copies of a scene's parameters, kept alive with their ctypes struct."""

    def __init__(self, scene=None, *, means=None, log_scales=None, quats=None,
                 opacity_logit=None, sh=None, sh_degree=None):
        src = scene
        self.means = _f64(means if means is not None else src.means)
        self.log_scales = _f64(log_scales if log_scales is not None else src.log_scales)
        self.quats = _f64(quats if quats is not None else src.quats)
        self.opacity_logit = _f64(opacity_logit if opacity_logit is not None else src.opacity_logit)
        self.sh = _f64(sh if sh is not None else src.sh)
        self.deg = int(sh_degree if sh_degree is not None else src.sh_degree)
        self.n = self.means.shape[0]
        self.struct = Gaussians(self.n, self.deg, _p(self.means), _p(self.log_scales),
                                _p(self.quats), _p(self.opacity_logit), _p(self.sh))


def camera_struct(cam) -> Camera:
    c = Camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).reshape(-1)]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32).reshape(-1)]
    c.fx, c.fy, c.cx, c.cy = (float(np.float32(v)) for v in (cam.fx, cam.fy, cam.cx, cam.cy))
    c.near_z = float(np.float32(cam.near))
    c.width, c.height = int(cam.width), int(cam.height)
    return c


def margins(**kw) -> Margins:
    d = dict(DEFAULT_MARGINS)
    d.update(kw)
    return Margins(**d)


def _threads(n_threads):
    return int(n_threads) if n_threads else (os.cpu_count() or 1)


def project(scene, cam, **over):
    P = _Params(scene, **over)
    n = P.n
    out = dict(mean2d=np.zeros((n, 2)), conic=np.zeros((n, 3)), cov2d=np.zeros((n, 3)),
               rgb=np.zeros((n, 3)), depth=np.zeros(n), opacity=np.zeros(n),
               radius=np.zeros(n, np.int32), rect=np.zeros((n, 4), np.int32),
               visible=np.zeros(n, np.int32))
    pr = Projection(**{k: _p(v) for k, v in out.items()})
    rc = lib().orc_project(C.byref(P.struct), C.byref(camera_struct(cam)), C.byref(pr))
    assert rc == 0
    return out


def sh_basis(degree, d):
    Y = np.zeros(16)
    dY = np.zeros((16, 3))
    rc = lib().orc_sh_basis(C.c_int32(degree), _p(_f64(d)), _p(Y), _p(dY))
    assert rc == 0
    k = (degree + 1) ** 2
    return Y[:k], dY[:k]


def render(scene, cam, *, tiles=None, margin=None, n_threads=None, hash_decisions=False, **over):
    """Forward render of one view; returns a dict of float64 / int arrays."""
    P = _Params(scene, **over)
    W, H = cam.width, cam.height
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), alpha=np.zeros((H, W)),
               T_final=np.ones((H, W)), n_contrib=np.zeros((H, W), np.int32),
               n_eval=np.zeros((H, W), np.int32), flags=np.zeros((H, W), np.uint8))
    t = None if tiles is None else np.ascontiguousarray(tiles, np.int32)
    h = C.c_uint64(0)
    m = margin if margin is not None else margins()
    rc = lib().orc_render(C.byref(P.struct), C.byref(camera_struct(cam)), C.byref(m), _p(t),
                          C.c_int32(-1 if t is None else t.size), _p(out["rgb"]), _p(out["depth"]),
                          _p(out["alpha"]), _p(out["T_final"]), _p(out["n_contrib"]),
                          _p(out["n_eval"]), _p(out["flags"]),
                          C.byref(h) if hash_decisions else None, C.c_int32(_threads(n_threads)))
    assert rc == 0
    if hash_decisions:
        out["hash"] = h.value
    return out


def render_outcomes(scene, cam, *, tiles=None, margin=None, n_threads=None, **over):
    """Forward render of one view plus, per pixel, the number of near-tie decisions that
    can change the image (``n_ties``) and the image with a single such decision taken
    the other way (``alt_rgb``, ``alt_depth``, ``alt_alpha``; NaN where n_ties >= 2)."""
    P = _Params(scene, **over)
    W, H = cam.width, cam.height
    out = dict(rgb=np.zeros((3, H, W)), depth=np.zeros((H, W)), alpha=np.zeros((H, W)),
               T_final=np.ones((H, W)), n_contrib=np.zeros((H, W), np.int32),
               flags=np.zeros((H, W), np.uint8), alt_rgb=np.zeros((3, H, W)),
               alt_depth=np.zeros((H, W)), alt_alpha=np.zeros((H, W)), n_ties=np.zeros((H, W), np.int32))
    t = None if tiles is None else np.ascontiguousarray(tiles, np.int32)
    m = margin if margin is not None else margins()
    rc = lib().orc_render_outcomes(C.byref(P.struct), C.byref(camera_struct(cam)), C.byref(m), _p(t),
                                   C.c_int32(-1 if t is None else t.size), _p(out["rgb"]), _p(out["depth"]),
                                   _p(out["alpha"]), _p(out["T_final"]), _p(out["n_contrib"]),
                                   _p(out["flags"]), _p(out["alt_rgb"]), _p(out["alt_depth"]),
                                   _p(out["alt_alpha"]), _p(out["n_ties"]), C.c_int32(_threads(n_threads)))
    assert rc == 0
    return out


def render_bruteforce(scene, cam, **over):
    P = _Params(scene, **over)
    W, H = cam.width, cam.height
    rgb, depth, alpha = np.zeros((3, H, W)), np.zeros((H, W)), np.zeros((H, W))
    rc = lib().orc_render_bruteforce(C.byref(P.struct), C.byref(camera_struct(cam)), _p(rgb),
                                     _p(depth), _p(alpha))
    assert rc == 0
    return dict(rgb=rgb, depth=depth, alpha=alpha)


def render_backward(scene, cam, g_rgb=None, g_depth=None, g_alpha=None, *, tiles=None,
                    margin=None, n_threads=None, grads=None, **over):
    """Gradient of sum(g_rgb*rgb + g_depth*depth + g_alpha*alpha) for one view.

    ``grads`` (optional) is a dict of float64 accumulators, updated in place."""
    P = _Params(scene, **over)
    n, K = P.n, (P.deg + 1) ** 2
    if grads is None:
        grads = new_grads(n, P.deg)
    gs = Grads(**{k: _p(grads.get(k)) for k in GRAD_KEYS})
    t = None if tiles is None else np.ascontiguousarray(tiles, np.int32)
    m = margin if margin is not None else margins()
    gr = None if g_rgb is None else _f64(g_rgb)
    gd = None if g_depth is None else _f64(g_depth)
    ga = None if g_alpha is None else _f64(g_alpha)
    rc = lib().orc_render_backward(C.byref(P.struct), C.byref(camera_struct(cam)), C.byref(m),
                                   _p(t), C.c_int32(-1 if t is None else t.size), _p(gr), _p(gd),
                                   _p(ga), C.byref(gs), C.c_int32(_threads(n_threads)))
    assert rc == 0
    return grads


def new_grads(n, deg, scale=False):
    """float64 gradient accumulators; ``scale`` adds the per-element scale arrays
    (``scale_<field>``, see orc_grads)."""
    K = (deg + 1) ** 2
    d = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
             opacity_logit=np.zeros(n), sh=np.zeros((n, K, 3)), grad2d=np.zeros((n, 10)),
             taint=np.zeros(n, np.uint8), grad_stat=np.zeros(n), vis_count=np.zeros(n))
    if scale:
        for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
            d["scale_" + k] = np.zeros_like(d[k])
    return d


def voxel_keys(means, voxel):
    m = _f64(means)
    keys = np.zeros((m.shape[0], 3), np.int32)
    rc = lib().orc_voxel_keys(C.c_int64(m.shape[0]), _p(m), C.c_double(float(np.float32(voxel))),
                              _p(keys))
    assert rc == 0
    return keys


def voxel_merge(scene, voxel, *, chi2=7.815, greedy=True, grad_stat=None, grad_tau=1e-3,
                kf_id=None, kf_min=0, kf_max=0, vis_count=None, tie_rel=1e-4, **over):
    P = _Params(scene, **over)
    n, K = P.n, (P.deg + 1) ** 2
    birth = np.ascontiguousarray(scene.birth, np.uint64)
    gs = None if grad_stat is None else _f64(grad_stat)
    kf = None if kf_id is None else np.ascontiguousarray(kf_id, np.int32)
    vc = None if vis_count is None else _f64(vis_count)
    prm = MergeParams(float(np.float32(chi2)), float(np.float32(grad_tau)), kf_min, kf_max,
                      _p(gs), _p(kf), _p(vc), 1 if greedy else 0)
    out = dict(means=np.zeros((n, 3)), log_scales=np.zeros((n, 3)), quats=np.zeros((n, 4)),
               opacity_logit=np.zeros(n), sh=np.zeros((n, K, 3)), birth=np.zeros(n, np.uint64),
               cov=np.zeros((n, 6)), partner=np.zeros(n, np.int32), tie=np.zeros(n, np.uint8))
    n_out = C.c_int64(0)
    rc = lib().orc_voxel_merge(C.byref(P.struct), _p(birth), C.c_double(float(np.float32(voxel))),
                               C.byref(prm), _p(out["means"]), _p(out["log_scales"]),
                               _p(out["quats"]), _p(out["opacity_logit"]), _p(out["sh"]),
                               _p(out["birth"]), _p(out["cov"]), _p(out["partner"]),
                               C.byref(n_out), C.c_double(tie_rel), _p(out["tie"]))
    assert rc == 0
    k = n_out.value
    for key in ("means", "log_scales", "quats", "opacity_logit", "sh", "birth", "cov"):
        out[key] = out[key][:k]
    out["n_out"] = k
    return out


def w2_barycentre(Si, Sj):
    Sk = np.zeros(9)
    lib().orc_w2_barycentre(_p(_f64(Si).reshape(-1)), _p(_f64(Sj).reshape(-1)), _p(Sk))
    return Sk.reshape(3, 3)


def w2_sq(A, B):
    return lib().orc_w2_sq(_p(_f64(A).reshape(-1)), _p(_f64(B).reshape(-1)))


def w2_lbfgs(qi, si, qj, sj, t=0.5, delta=(0.001, 0.002, 0.003)):
    qk, sk, Sk, f = np.zeros(4), np.zeros(3), np.zeros(9), C.c_double(0)
    it = lib().orc_w2_lbfgs(_p(_f64(qi)), _p(_f64(si)), _p(_f64(qj)), _p(_f64(sj)),
                            C.c_double(t), _p(_f64(delta)), _p(qk), _p(sk), _p(Sk), C.byref(f))
    return dict(q=qk, s=sk, S=Sk.reshape(3, 3), iters=it, objective=f.value)


def merge_mean(Si, mi, Sj, mj):
    mk = np.zeros(3)
    lib().orc_merge_mean(_p(_f64(Si).reshape(-1)), _p(_f64(mi)), _p(_f64(Sj).reshape(-1)),
                         _p(_f64(mj)), _p(mk))
    return mk


def covariance(q, s):
    S = np.zeros(9)
    lib().orc_covariance(_p(_f64(q)), _p(_f64(s)), _p(S))
    return S.reshape(3, 3)


def adam(param, grad, m, v, lr, b1, b2, eps, step):
    """In-place FP64 Adam step on float64 arrays."""
    for a in (param, m, v):
        assert a.dtype == np.float64 and a.flags.c_contiguous
    g = _f64(grad)
    rc = lib().orc_adam(C.c_int64(param.size), _p(param), _p(g), _p(m), _p(v), C.c_double(lr),
                        C.c_double(b1), C.c_double(b2), C.c_double(eps), C.c_int32(step))
    assert rc == 0


def mapping_loss(x, y, d=None, dt=None, lam=0.2, w_depth=1.0, grads=True):
    """Eq. 12 per view: x, y [V,3,H,W]; d, dt [V,H,W] (optional).  Returns dict with
    loss [V,3] (weighted L1, SSIM and depth parts) and g_rgb / g_depth."""
    x64, y64 = _f64(x), _f64(y)
    V, _, H, W = x64.shape
    loss = np.zeros((V, 3))
    g_rgb = np.zeros_like(x64) if grads else None
    d64 = None if d is None else _f64(d)
    dt64 = None if dt is None else _f64(dt)
    g_depth = np.zeros((V, H, W)) if grads else None
    rc = lib().orc_mapping_loss(C.c_int32(V), C.c_int32(H), C.c_int32(W), _p(x64), _p(y64), _p(d64),
                                _p(dt64), C.c_double(lam), C.c_double(w_depth), _p(loss), _p(g_rgb),
                                _p(g_depth))
    assert rc == 0
    return dict(loss=loss, g_rgb=g_rgb, g_depth=g_depth)


def iso_loss(log_scales, w_iso=1.0):
    ls = _f64(log_scales)
    grad = np.zeros_like(ls)
    val = C.c_double(0)
    rc = lib().orc_iso_loss(C.c_int64(ls.shape[0]), _p(ls), C.c_double(w_iso), C.byref(val), _p(grad))
    assert rc == 0
    return val.value, grad


def patch_grid(cam, kp_uv, kp_depth=None, depth_image=None, patch=32, min_keypoints=4, grid=2):
    """Patch-Grid sampling (Sec. II-B) for one keyframe.  Returns dict with samples
    [n, 6] = (u, v, depth, x, y, z world) and source [n] (0 depth image, 1 keypoint)."""
    kp = np.ascontiguousarray(kp_uv, np.float32).reshape(-1, 2)
    K = kp.shape[0]
    kd = None if kp_depth is None else np.ascontiguousarray(kp_depth, np.float32)
    di = None if depth_image is None else np.ascontiguousarray(depth_image, np.float32)
    W, H = int(cam.width), int(cam.height)
    cap = ((W + patch - 1) // patch) * ((H + patch - 1) // patch) * grid * grid
    out = np.zeros((max(cap, 1), 6))
    src = np.zeros(max(cap, 1), np.int32)
    n = C.c_int64(0)
    rc = lib().orc_patch_grid(C.byref(camera_struct(cam)), C.c_int32(K), kp.ctypes.data_as(C.c_void_p),
                              None if kd is None else kd.ctypes.data_as(C.c_void_p),
                              None if di is None else di.ctypes.data_as(C.c_void_p),
                              C.c_int32(patch), C.c_int32(min_keypoints), C.c_int32(grid),
                              _p(out), src.ctypes.data_as(C.c_void_p), C.byref(n))
    assert rc == 0
    return dict(samples=out[:n.value], source=src[:n.value])
