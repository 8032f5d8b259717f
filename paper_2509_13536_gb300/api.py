"""Torch-facing wrappers of the libmemgs C ABI.

Everything here marshals arguments: tensors become device pointers, the current
torch CUDA stream becomes the ``stream`` argument, and every computation happens in
the library's kernels.  Tensors must live on a CUDA device; there is no CPU path.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
from typing import List, Optional, Sequence

import numpy as np
import torch

from . import _abi
from ._abi import MemgsError, check, load

_DTYPES = {torch.float32: _abi.MGS_F32, torch.float16: _abi.MGS_F16, torch.bfloat16: _abi.MGS_BF16}


def _ptr(t: Optional[torch.Tensor]):
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("libmemgs takes CUDA tensors only")
    if not t.is_contiguous():
        raise ValueError("libmemgs takes contiguous tensors only")
    return C.c_void_p(t.data_ptr())


def _stream(stream=None):
    s = stream if stream is not None else torch.cuda.current_stream()
    return C.c_void_p(s.cuda_stream)


@dataclasses.dataclass
class Gaussians:
    """Device-resident Gaussian map in the library's structure-of-arrays layout."""
    means: torch.Tensor          # f32 [n,3]
    log_scales: torch.Tensor     # attr [n,3]
    quats: torch.Tensor          # attr [n,4]
    opacity_logit: torch.Tensor  # attr [n]
    sh: torch.Tensor             # attr [n,K,3]
    birth: Optional[torch.Tensor] = None  # int64 [n] (stored as uint64 bit patterns)

    @property
    def n(self) -> int:
        return int(self.means.shape[0])

    @property
    def sh_degree(self) -> int:
        return int(round(self.sh.shape[1] ** 0.5)) - 1

    @property
    def attr_dtype(self) -> torch.dtype:
        """Storage type of the appearance group (opacity logit, SH)."""
        return self.sh.dtype

    @property
    def geom_dtype(self) -> torch.dtype:
        """Storage type of the geometry group (log-scales, quaternions)."""
        return self.log_scales.dtype

    @staticmethod
    def from_scene(scene, device="cuda", attr_dtype=torch.float32, geom_dtype=torch.float32,
                   quat_dtype=None) -> "Gaussians":
        """Upload a scene; opacity/SH stored as attr_dtype, log-scales as geom_dtype,
        quaternions as quat_dtype (default: geom_dtype); means are always f32."""
        d = torch.device(device)
        f = lambda a, dt: torch.from_numpy(np.ascontiguousarray(a)).to(d).to(dt).contiguous()
        return Gaussians(f(scene.means, torch.float32), f(scene.log_scales, geom_dtype),
                         f(scene.quats, geom_dtype if quat_dtype is None else quat_dtype),
                         f(scene.opacity_logit, attr_dtype),
                         f(scene.sh, attr_dtype), torch.from_numpy(scene.birth.astype(np.int64)).to(d))

    def params(self):
        return [self.means, self.log_scales, self.quats, self.opacity_logit, self.sh]

    def struct(self) -> _abi.mgs_gaussians:
        if self.means.dtype != torch.float32:
            raise ValueError("means must be float32")
        if self.opacity_logit.dtype != self.sh.dtype:
            raise ValueError("opacity_logit and sh must share one dtype")
        return _abi.mgs_gaussians(self.n, self.sh_degree, _DTYPES[self.sh.dtype], _DTYPES[self.log_scales.dtype],
                                  _DTYPES[self.quats.dtype], _ptr(self.means),
                                  _ptr(self.log_scales), _ptr(self.quats), _ptr(self.opacity_logit),
                                  _ptr(self.sh), _ptr(self.birth))

    def empty_like(self) -> "Gaussians":
        return Gaussians(*(torch.empty_like(t) for t in self.params()),
                         None if self.birth is None else torch.empty_like(self.birth))


def camera_struct(cam) -> _abi.mgs_camera:
    c = _abi.mgs_camera()
    c.R[:] = [float(x) for x in np.asarray(cam.R, np.float32).reshape(-1)]
    c.t[:] = [float(x) for x in np.asarray(cam.t, np.float32).reshape(-1)]
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.width, c.height = int(cam.width), int(cam.height)
    c.near_z = float(getattr(cam, "near", 0.2))
    return c


def _cam_array(cams):
    arr = (_abi.mgs_camera * len(cams))()
    for i, c in enumerate(cams):
        arr[i] = camera_struct(c)
    return arr


@dataclasses.dataclass
class Image:
    rgb: torch.Tensor    # [3,H,W]
    depth: torch.Tensor  # [H,W]
    alpha: torch.Tensor  # [H,W]


def _image_array(images: Sequence[Optional[Image]]):
    arr = (_abi.mgs_image * len(images))()
    for i, im in enumerate(images):
        if im is None:
            arr[i] = _abi.mgs_image(None, None, None)
        else:
            arr[i] = _abi.mgs_image(_ptr(im.rgb), _ptr(im.depth), _ptr(im.alpha))
    return arr


def new_images(cams, device="cuda") -> List[Image]:
    out = []
    for c in cams:
        H, W = int(c.height), int(c.width)
        out.append(Image(torch.empty(3, H, W, device=device), torch.empty(H, W, device=device),
                         torch.empty(H, W, device=device)))
    return out


@dataclasses.dataclass
class Grads:
    means: torch.Tensor
    log_scales: torch.Tensor
    quats: torch.Tensor
    opacity_logit: torch.Tensor
    sh: torch.Tensor
    grad_stat: Optional[torch.Tensor] = None
    vis_count: Optional[torch.Tensor] = None
    overwrite: bool = False  # mgs_render_backward stores (instead of adds) the call's gradients

    @staticmethod
    def zeros_like(g: Gaussians, stats: bool = True) -> "Grads":
        z = lambda t: torch.zeros(t.shape, dtype=torch.float32, device=t.device)
        n = g.n
        return Grads(z(g.means), z(g.log_scales), z(g.quats), z(g.opacity_logit), z(g.sh),
                     torch.zeros(n, device=g.means.device) if stats else None,
                     torch.zeros(n, device=g.means.device) if stats else None)

    def tensors(self):
        return [self.means, self.log_scales, self.quats, self.opacity_logit, self.sh]

    def struct(self) -> _abi.mgs_grads:
        return _abi.mgs_grads(_ptr(self.means), _ptr(self.log_scales), _ptr(self.quats),
                              _ptr(self.opacity_logit), _ptr(self.sh), _ptr(self.grad_stat),
                              _ptr(self.vis_count), int(self.overwrite), 0)


class RenderWorkspace:
    """Caller-owned scratch of mgs_render / mgs_render_backward, grown on demand.

    It holds the saved state of the last render (projected records, sorted lists,
    per-pixel T and contributor counts) that the backward pass reads.  ``generation``
    counts renders into it and regrowths of it, so that a backward pass can tell that
    the state it needs was overwritten."""

    def __init__(self, device="cuda", key_headroom: float = 1.25):
        self.device = torch.device(device)
        self.buf: Optional[torch.Tensor] = None
        self.headroom = key_headroom
        self.n_keys = 0
        self.generation = 0
        self.status: Optional[torch.Tensor] = None  # pinned {keys, overflow} of an asynchronous render
        self.pending = False

    def status_buffer(self) -> torch.Tensor:
        if self.status is None:
            self.status = torch.zeros(2, dtype=torch.int64, pin_memory=True)
        return self.status

    def check(self, stream=None) -> int:
        """After asynchronous renders: wait for the stream, then the key count of the
        last one.  If its keys exceeded the capacity (its images are empty), grow the
        workspace for them and raise: that render has to be repeated."""
        if not self.pending:
            return self.n_keys
        (stream or torch.cuda.current_stream()).synchronize()
        self.pending = False
        keys, over = int(self.status[0]), int(self.status[1])
        self.n_keys = keys
        if over:
            self.buf = None
            self.generation += 1
            raise MemgsError(_abi.MGS_ERR_WORKSPACE, "mgs_render_async",
                             f"{keys} keys exceeded the workspace; it is released, the next render regrows it")
        return keys

    def ensure(self, n, cams, key_capacity) -> torch.Tensor:
        arr = _cam_array(cams)
        need = load().mgs_render_workspace_size(n, arr, len(cams), int(key_capacity))
        if need == 0:
            raise ValueError("invalid render arguments")
        if self.buf is None or self.buf.numel() < need:
            self.buf = None
            self.buf = torch.empty(need, dtype=torch.uint8, device=self.device)
            self.generation += 1
        return self.buf


def mgs_render(g: Gaussians, cams, out: List[Image], ws: RenderWorkspace, stream=None, sync=True) -> int:
    """One call of mgs_render; grows the workspace and retries when it is too small.
    sync=False (with a workspace sized by an earlier render): mgs_render_async, no host
    synchronisation; the key count and an overflow are checked by ws.check()."""
    L = load()
    gs = g.struct()
    arr = _cam_array(cams)
    imgs = _image_array(out)
    if not sync and ws.buf is not None:
        check(L.mgs_render_async(C.byref(gs), arr, len(cams), imgs, _ptr(ws.buf), ws.buf.numel(),
                                 C.c_void_p(ws.status_buffer().data_ptr()), _stream(stream)), "mgs_render_async")
        ws.pending = True
        ws.generation += 1
        return -1
    if ws.buf is None:
        ws.ensure(g.n, cams, max(1024, 8 * g.n * len(cams)))
    for _ in range(3):
        nk = C.c_int64(0)
        st = L.mgs_render(C.byref(gs), arr, len(cams), imgs, _ptr(ws.buf), ws.buf.numel(), C.byref(nk),
                          _stream(stream))
        if st == _abi.MGS_ERR_WORKSPACE and nk.value > 0:
            ws.ensure(g.n, cams, int(nk.value * ws.headroom) + 1024)
            continue
        check(st, "mgs_render")
        ws.n_keys = nk.value
        ws.generation += 1
        return nk.value
    check(st, "mgs_render")
    return 0


def mgs_render_multi(maps: Sequence[Gaussians], map_of_view: Sequence[int], cams, out: List[Image],
                     ws: RenderWorkspace, stream=None) -> int:
    """One call of mgs_render_multi (view v from maps[map_of_view[v]]); grows the
    workspace and retries when it is too small.  Returns the key count."""
    L = load()
    ms = (_abi.mgs_gaussians * len(maps))()
    for i, g in enumerate(maps):
        ms[i] = g.struct()
    mov = (C.c_int32 * len(cams))(*[int(m) for m in map_of_view])
    arr = _cam_array(cams)
    imgs = _image_array(out)

    def grow(keys):
        need = L.mgs_render_multi_workspace_size(ms, len(maps), mov, arr, len(cams), int(keys))
        if need == 0:
            raise ValueError("invalid render arguments")
        if ws.buf is None or ws.buf.numel() < need:
            ws.buf = None
            ws.buf = torch.empty(need, dtype=torch.uint8, device=ws.device)
            ws.generation += 1

    if ws.buf is None:
        grow(max(1024, 8 * sum(maps[m].n for m in map_of_view)))
    for _ in range(3):
        nk = C.c_int64(0)
        st = L.mgs_render_multi(ms, len(maps), mov, arr, len(cams), imgs, _ptr(ws.buf), ws.buf.numel(),
                                C.byref(nk), _stream(stream))
        if st == _abi.MGS_ERR_WORKSPACE:
            # nk = 0: not even the layout without keys fitted; else the keys did not
            grow(int(nk.value * ws.headroom) + 1024 if nk.value > 0 else 8 * sum(maps[m].n for m in map_of_view))
            continue
        check(st, "mgs_render_multi")
        ws.n_keys = nk.value
        ws.generation += 1
        return nk.value
    check(st, "mgs_render_multi")
    return 0


def mgs_render_backward(g: Gaussians, cams, dL: Sequence[Optional[Image]], ws: RenderWorkspace,
                        grads: Grads, stream=None):
    L = load()
    gs = g.struct()
    check(L.mgs_render_backward(C.byref(gs), _cam_array(cams), len(cams), _image_array(dL),
                                _ptr(ws.buf), ws.buf.numel(), C.byref(grads.struct()), _stream(stream)),
          "mgs_render_backward")


def render(g: Gaussians, cams, ws: Optional[RenderWorkspace] = None, stream=None):
    """render(gaussians, cameras) -> list of Image (rgb [3,H,W], depth, alpha) per view."""
    ws = ws or RenderWorkspace(g.means.device)
    out = new_images(cams, g.means.device)
    mgs_render(g, cams, out, ws, stream)
    return out, ws


def render_backward(g: Gaussians, cams, dL: Sequence[Optional[Image]], ws: RenderWorkspace,
                    grads: Optional[Grads] = None, stream=None) -> Grads:
    """render_backward(dL/dimage) -> dL/dgaussians (accumulated into ``grads``)."""
    grads = grads or Grads.zeros_like(g)
    mgs_render_backward(g, cams, dL, ws, grads, stream)
    return grads


def mgs_project(g: Gaussians, cam, stream=None):
    n, dev = g.n, g.means.device
    out = dict(mean2d=torch.zeros(n, 2, device=dev), conic=torch.zeros(n, 3, device=dev),
               rgb=torch.zeros(n, 3, device=dev), depth=torch.zeros(n, device=dev),
               radius=torch.zeros(n, dtype=torch.int32, device=dev),
               rect=torch.zeros(n, 4, dtype=torch.int32, device=dev))
    c = camera_struct(cam)
    check(load().mgs_project(C.byref(g.struct()), C.byref(c), _ptr(out["mean2d"]), _ptr(out["conic"]),
                             _ptr(out["rgb"]), _ptr(out["depth"]), _ptr(out["radius"]),
                             _ptr(out["rect"]), _stream(stream)), "mgs_project")
    return out


project = mgs_project


def mgs_voxel_merge(g: Gaussians, voxel_size: float, chi2: float = 7.815, greedy: bool = True,
                    grad_stat: Optional[torch.Tensor] = None, grad_tau: float = 1e-3,
                    kf_id: Optional[torch.Tensor] = None, kf_min: int = 0, kf_max: int = 0,
                    workspace: Optional[torch.Tensor] = None, out: Optional[Gaussians] = None,
                    partner: Optional[torch.Tensor] = None, vox: Optional[torch.Tensor] = None,
                    vis_count: Optional[torch.Tensor] = None, solver: str = "closed_form", stream=None,
                    status: Optional[torch.Tensor] = None):
    """voxel_merge(gaussians, voxel_size, thresholds) -> (gaussians, partner, voxel coords).

    ``grad_stat`` with ``vis_count``: the sums the backward pass accumulates (Grads.grad_stat,
    Grads.vis_count); the Eq. 3 mask then tests their quotient.  ``workspace``, ``out``,
    ``partner`` and ``vox`` may be passed preallocated.  ``status`` (a pinned int32 [2]
    tensor): mgs_voxel_merge_async, no host synchronisation; the returned map then has
    the input's capacity and status receives {survivors, flags} with the stream."""
    if g.birth is None:
        raise ValueError("voxel merge needs birth stamps")
    L = load()
    n, dev = g.n, g.means.device
    need = L.mgs_voxel_merge_workspace_size(n)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(need, dtype=torch.uint8, device=dev)
    out = out if out is not None else g.empty_like()
    partner = partner if partner is not None else torch.empty(n, dtype=torch.int32, device=dev)
    vox = vox if vox is not None else torch.empty(n, 3, dtype=torch.int32, device=dev)
    if solver not in ("closed_form", "lbfgs"):
        raise ValueError("solver is 'closed_form' or 'lbfgs'")
    p = _abi.mgs_merge_params(chi2, grad_tau, kf_min, kf_max, _ptr(grad_stat), _ptr(kf_id),
                              _ptr(vis_count), 1 if greedy else 0, 1 if solver == "lbfgs" else 0)
    if status is not None:
        check(L.mgs_voxel_merge_async(C.byref(g.struct()), float(voxel_size), C.byref(p), C.byref(out.struct()),
                                      _ptr(partner), _ptr(vox), C.c_void_p(status.data_ptr()), _ptr(workspace),
                                      workspace.numel(), _stream(stream)), "mgs_voxel_merge_async")
        return out, partner, vox
    n_out = C.c_int64(0)
    check(L.mgs_voxel_merge(C.byref(g.struct()), float(voxel_size), C.byref(p), C.byref(out.struct()),
                            _ptr(partner), _ptr(vox), C.byref(n_out), _ptr(workspace),
                            workspace.numel(), _stream(stream)), "mgs_voxel_merge")
    k = n_out.value
    res = Gaussians(out.means[:k], out.log_scales[:k], out.quats[:k], out.opacity_logit[:k], out.sh[:k],
                    out.birth[:k])
    return res, partner, vox


voxel_merge = mgs_voxel_merge


def merge_stats():
    """(merged pairs, L-BFGS iterations) of this thread's last mgs_voxel_merge."""
    out = (C.c_int64 * 2)()
    load().mgs_merge_stats(out)
    return int(out[0]), int(out[1])


def mgs_adam_step(g: Gaussians, grads: Grads, m: Grads, v: Grads, lr: float, beta1=0.9,
                  beta2=0.999, eps=1e-8, step: int = 1, zero_grads: bool = False, stream=None):
    check(load().mgs_adam_step(C.byref(g.struct()), C.byref(grads.struct()), C.byref(m.struct()),
                               C.byref(v.struct()), lr, beta1, beta2, eps, step, 1 if zero_grads else 0,
                               _stream(stream)), "mgs_adam_step")


adam_step = mgs_adam_step


def mgs_mapping_loss(rendered: Sequence[Image], target: Sequence[Image], grad: Sequence[Image],
                     lambda_ssim: float = 0.2, w_depth: float = 1.0, loss: Optional[torch.Tensor] = None,
                     workspace: Optional[torch.Tensor] = None, stream=None) -> torch.Tensor:
    """Eq. 12 per view: (1-lambda) L1 + lambda (1 - SSIM) + w_depth depth L1.  ``target[v].depth``
    None = no depth term.  Writes the cotangents into ``grad`` and returns loss [V, 3]
    (L1, SSIM, depth parts, weighted)."""
    V = len(rendered)
    H, W = int(rendered[0].rgb.shape[-2]), int(rendered[0].rgb.shape[-1])
    dev = rendered[0].rgb.device
    L = load()
    need = L.mgs_mapping_loss_workspace_size(V, W, H)
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    loss = loss if loss is not None else torch.empty(V, 3, device=dev)
    check(L.mgs_mapping_loss(V, W, H, _image_array(rendered), _image_array(target), _image_array(grad),
                             float(lambda_ssim), float(w_depth), _ptr(loss), _ptr(workspace), workspace.numel(),
                             _stream(stream)), "mgs_mapping_loss")
    return loss


mapping_loss = mgs_mapping_loss


def mgs_iso_loss(g: Gaussians, w_iso: float = 1.0, grads: Optional[Grads] = None,
                 loss: Optional[torch.Tensor] = None, workspace: Optional[torch.Tensor] = None,
                 stream=None) -> torch.Tensor:
    """Isotropic term of Eq. 12; adds its gradient to ``grads.log_scales`` when given."""
    L = load()
    need = L.mgs_iso_loss_workspace_size(g.n)
    dev = g.means.device
    if workspace is None or workspace.numel() < need:
        workspace = torch.empty(max(need, 1), dtype=torch.uint8, device=dev)
    loss = loss if loss is not None else torch.empty(1, device=dev)
    gs = None if grads is None else C.byref(grads.struct())
    check(L.mgs_iso_loss(C.byref(g.struct()), float(w_iso), gs, _ptr(loss), _ptr(workspace), workspace.numel(),
                         _stream(stream)), "mgs_iso_loss")
    return loss


iso_loss = mgs_iso_loss


def mgs_patch_grid_sample(cam, kp_uv: torch.Tensor, kp_depth: Optional[torch.Tensor] = None,
                          depth_image: Optional[torch.Tensor] = None, patch: int = 32,
                          min_keypoints: int = 4, grid: int = 2, stream=None):
    """Patch-Grid sampling (Sec. II-B) for one keyframe -> (samples [n, 6] = u, v, depth,
    world xyz; source [n]: 0 depth image, 1 nearest keypoint)."""
    L = load()
    dev = kp_uv.device
    p = _abi.mgs_pg_params(int(patch), int(min_keypoints), int(grid), 0)
    c = camera_struct(cam)
    W, H = int(cam.width), int(cam.height)
    cap = L.mgs_patch_grid_capacity(W, H, C.byref(p))
    need = L.mgs_patch_grid_workspace_size(W, H, C.byref(p))
    if need == 0:
        raise ValueError("invalid patch-grid parameters")
    ws = torch.empty(need, dtype=torch.uint8, device=dev)
    out = torch.empty(max(cap, 1), 6, device=dev)
    src = torch.empty(max(cap, 1), dtype=torch.int32, device=dev)
    n = C.c_int64(0)
    kp = kp_uv.contiguous()
    check(L.mgs_patch_grid_sample(C.byref(c), int(kp.shape[0]), _ptr(kp) if kp.numel() else None, _ptr(kp_depth),
                                  _ptr(depth_image), C.byref(p), _ptr(out), _ptr(src), cap, C.byref(n),
                                  _ptr(ws), ws.numel(), _stream(stream)), "mgs_patch_grid_sample")
    return out[:n.value], src[:n.value]


patch_grid_sample = mgs_patch_grid_sample


def mgs_l1_loss_grad(pred: torch.Tensor, target: torch.Tensor, scale: float, grad: torch.Tensor,
                     loss: Optional[torch.Tensor] = None, stream=None):
    check(load().mgs_l1_loss_grad(_ptr(pred), _ptr(target), pred.numel(), scale, _ptr(grad), _ptr(loss),
                                  _stream(stream)), "mgs_l1_loss_grad")


def mgs_sort_pairs(keys: torch.Tensor, vals: Optional[torch.Tensor] = None, begin_bit=0, end_bit=32,
                   stream=None):
    """Stable sort of int32-stored u32 keys (in place); returns the values / permutation."""
    L = load()
    n = keys.numel()
    ws = torch.empty(L.mgs_sort_workspace_size(n), dtype=torch.uint8, device=keys.device)
    out = None if vals is not None else torch.empty(n, dtype=torch.int32, device=keys.device)
    check(L.mgs_sort_pairs(_ptr(keys), _ptr(vals), _ptr(out), n, begin_bit, end_bit, _ptr(ws), ws.numel(),
                           _stream(stream)), "mgs_sort_pairs")
    return vals if vals is not None else out


def version() -> str:
    return load().mgs_version().decode()


def launch_count() -> int:
    return int(load().mgs_launch_count())


def profile_enable(on: bool):
    load().mgs_profile_enable(1 if on else 0)


def profile_read():
    """{kernel group: (total ms, launches)} recorded since profile_enable(True)."""
    L = load()
    k = 32
    names = C.create_string_buffer(32 * k)
    ms = (C.c_double * k)()
    cnt = (C.c_int64 * k)()
    n = L.mgs_profile_read(k, names, ms, cnt)
    raw = names.raw
    out = {}
    for i in range(min(n, k)):
        nm = raw[32 * i:32 * i + 32].split(b"\0", 1)[0].decode()
        out[nm] = (float(ms[i]), int(cnt[i]))
    return out


def render_stats(g: Gaussians, cams, ws: RenderWorkspace, stream=None):
    """Fragment counts of the last render on ``ws``: evaluated, contributing, walked by the
    backward pass, (Gaussian, tile) keys, padded counts, and drawn (view, Gaussian) items."""
    st = (C.c_uint64 * 9)()
    check(load().mgs_render_stats(C.byref(g.struct()), _cam_array(cams), len(cams), _ptr(ws.buf),
                                  ws.buf.numel(), st, _stream(stream)), "mgs_render_stats")
    return dict(evaluated=int(st[0]), contributing=int(st[1]), backward_walked=int(st[2]), keys=int(st[3]),
                fwd_padded_tile=int(st[4]), bwd_padded_tile=int(st[5]), fwd_padded_warp=int(st[6]),
                bwd_padded_warp=int(st[7]), drawn_items=int(st[8]))


# ---------------------------------------------------------------------------------
class RenderFn(torch.autograd.Function):
    """Differentiable multi-view render through libmemgs.

    apply(means, log_scales, quats, opacity_logit, sh, cams, ws, grads=None, sync=True) ->
    (rgb [V,3,H,W], depth [V,H,W], alpha [V,H,W]) for views of one resolution.  The
    backward pass is mgs_render_backward on the saved state in ``ws``; it refuses to run
    if ``ws`` was rendered into or regrown after this forward pass.  sync=False renders
    with mgs_render_async (no host synchronisation; ws.check() reports an overflow).

    ``grads`` None: the backward pass returns new f32 gradient tensors (plain autograd).
    ``grads`` a Grads: the library accumulates the gradients into those buffers in place
    (with the Eq. 3 statistics when the Grads has them) and the backward pass returns
    None for the parameters: no allocation and no copy in the step; whoever owns the
    buffers (MappingStep's Adam) consumes and clears them.
    """

    @staticmethod
    def forward(ctx, means, log_scales, quats, opacity_logit, sh, cams, ws, grads=None, sync=True):
        g = Gaussians(means.detach(), log_scales.detach(), quats.detach(), opacity_logit.detach(),
                      sh.detach())
        V = len(cams)
        H, W = int(cams[0].height), int(cams[0].width)
        if any(int(c.height) != H or int(c.width) != W for c in cams):
            raise ValueError("RenderFn renders views of one resolution")
        rgb = torch.empty(V, 3, H, W, device=means.device)
        depth = torch.empty(V, H, W, device=means.device)
        alpha = torch.empty(V, H, W, device=means.device)
        out = [Image(rgb[v], depth[v], alpha[v]) for v in range(V)]
        mgs_render(g, cams, out, ws, sync=sync)
        ctx.set_materialize_grads(False)  # an unused output's cotangent stays None: no zero-filled tensor
        ctx.cams, ctx.ws, ctx.grads = cams, ws, grads
        ctx.generation, ctx.buf = ws.generation, ws.buf
        ctx.save_for_backward(means, log_scales, quats, opacity_logit, sh)
        return rgb, depth, alpha

    @staticmethod
    def backward(ctx, g_rgb, g_depth, g_alpha):
        ws = ctx.ws
        if ws.generation != ctx.generation or ws.buf is not ctx.buf:
            raise RuntimeError("RenderFn.backward: the render workspace was reused or regrown after this "
                               "forward pass; give each pending render its own RenderWorkspace")
        means, log_scales, quats, opacity_logit, sh = ctx.saved_tensors
        g = Gaussians(means, log_scales, quats, opacity_logit, sh)
        V = len(ctx.cams)
        c = lambda t: None if t is None else t.contiguous()
        g_rgb, g_depth, g_alpha = c(g_rgb), c(g_depth), c(g_alpha)
        arr = (_abi.mgs_image * V)()
        for v in range(V):
            arr[v] = _abi.mgs_image(None if g_rgb is None else _ptr(g_rgb[v]),
                                    None if g_depth is None else _ptr(g_depth[v]),
                                    None if g_alpha is None else _ptr(g_alpha[v]))
        if ctx.grads is not None:
            grads = ctx.grads
        else:  # fresh tensors the library stores into (no zero fill needed)
            e = lambda t: torch.empty(t.shape, dtype=torch.float32, device=t.device)
            grads = Grads(e(means), e(log_scales), e(quats), e(opacity_logit), e(sh), overwrite=True)
        check(load().mgs_render_backward(C.byref(g.struct()), _cam_array(ctx.cams), V, arr,
                                         _ptr(ws.buf), ws.buf.numel(), C.byref(grads.struct()),
                                         _stream()), "mgs_render_backward")
        if ctx.grads is not None:
            return None, None, None, None, None, None, None, None, None
        cast = lambda gr, p: gr if p.dtype == torch.float32 else gr.to(p.dtype)
        return (grads.means, cast(grads.log_scales, log_scales), cast(grads.quats, quats),
                cast(grads.opacity_logit, opacity_logit), cast(grads.sh, sh), None, None, None, None)


def render_views(g: Gaussians, cams, ws: Optional[RenderWorkspace] = None):
    """Differentiable render of same-resolution views: returns (rgb, depth, alpha) tensors."""
    ws = ws or RenderWorkspace(g.means.device)
    return RenderFn.apply(g.means, g.log_scales, g.quats, g.opacity_logit, g.sh, cams, ws)


class MappingStep:
    """The batched mapping step of Sec. II-E driven through torch.autograd.

    Each call: render every keyframe of the batch in one multi-view launch through
    RenderFn (forward A1-A4), the mapping loss against the keyframe images
    (mgs_mapping_loss: Eq. 12, lambda = 0 gives its plain L1 form, plus the
    isotropic term when w_iso > 0), torch.autograd.backward from the rendered images
    with the loss kernel's cotangents (RenderFn.backward: A5-A6 store the gradients
    into the step's buffers, which therefore need no clearing), the isotropic term's
    gradient added when w_iso > 0, then the in-kernel Adam step.  The Eq. 3 sums keep
    accumulating over steps.  Every kernel of the step is the library's; the parameter tensors are
    updated in place.  Returns the device loss tensor [V, 3] (weighted L1, SSIM and
    depth parts per view); ``loss_iso`` holds the isotropic term.

    The first call renders synchronously (it sizes the render workspace from the key
    count, with headroom); later calls render with mgs_render_async, so a step makes no
    host round trip.  check() waits for the stream and raises if a render's keys
    outgrew the workspace (that step's images were empty; the next step regrows it).
    """

    def __init__(self, g: Gaussians, cams, lr=1e-3, lambda_ssim=0.0, w_depth=0.1, w_iso=0.0,
                 betas=(0.9, 0.999), eps=1e-8, stats=True):
        self.g = g
        self.cams = list(cams)
        self.lr, self.betas, self.eps = float(lr), betas, float(eps)
        self.lambda_ssim, self.w_depth, self.w_iso = float(lambda_ssim), float(w_depth), float(w_iso)
        self.params = [p.requires_grad_(True) for p in g.params()]
        self.grads = Grads.zeros_like(g, stats=stats)
        self.grads.overwrite = True  # the render backward stores each step's gradients
        self.m = Grads.zeros_like(g, stats=False)
        self.v = Grads.zeros_like(g, stats=False)
        self.ws = RenderWorkspace(g.means.device)
        V = len(self.cams)
        H, W = int(self.cams[0].height), int(self.cams[0].width)
        dev = g.means.device
        self.g_rgb = torch.empty(V, 3, H, W, device=dev)
        self.g_depth = torch.empty(V, H, W, device=dev)
        self.loss = torch.zeros(V, 3, device=dev)
        self.loss_iso = torch.zeros(1, device=dev)
        L = load()
        self.loss_ws = torch.empty(max(1, L.mgs_mapping_loss_workspace_size(V, W, H)), dtype=torch.uint8,
                                   device=dev)
        self.iso_ws = torch.empty(max(1, L.mgs_iso_loss_workspace_size(g.n)), dtype=torch.uint8, device=dev)
        self.step_count = 0
        self._dL = [Image(self.g_rgb[v], self.g_depth[v], None) for v in range(V)]
        self.ws.headroom = 1.1

    def __call__(self, target_rgb: torch.Tensor, target_depth: Optional[torch.Tensor] = None,
                 before_update: Optional[torch.cuda.Event] = None):
        """One step against keyframe images target_rgb [V,3,H,W] (and target_depth [V,H,W]).
        ``before_update``: an event the parameter update waits for on the step's stream
        (a reader of the parameters on another stream, e.g. the previous step's merge)."""
        self.step_count += 1
        rgb, depth, alpha = RenderFn.apply(*self.params, self.cams, self.ws, self.grads, self.ws.buf is None)
        V = len(self.cams)
        rendered = [Image(rgb[v].detach(), depth[v].detach(), alpha[v].detach()) for v in range(V)]
        targets = [Image(target_rgb[v], None if target_depth is None else target_depth[v], None)
                   for v in range(V)]
        mgs_mapping_loss(rendered, targets, self._dL, self.lambda_ssim, self.w_depth, loss=self.loss,
                         workspace=self.loss_ws)
        torch.autograd.backward((rgb, depth), (self.g_rgb, self.g_depth))
        g = self.g
        if self.w_iso > 0:
            mgs_iso_loss(g, self.w_iso, self.grads, loss=self.loss_iso, workspace=self.iso_ws)
        if before_update is not None:
            torch.cuda.current_stream().wait_event(before_update)
        with torch.no_grad():
            mgs_adam_step(g, self.grads, self.m, self.v, self.lr, self.betas[0], self.betas[1], self.eps,
                          self.step_count, zero_grads=False)
        return self.loss

    def check(self) -> int:
        """Key count of the last render (waits for the stream); raises on an overflow."""
        return self.ws.check()


class Server:
    """Continuous-batching render server (mgs_server_*): resident scenes, asynchronous
    requests, admission by free memory of a device arena owned by this object."""

    def __init__(self, arena_bytes: int, n_slots: int = 8, max_batch_views: int = 8, device=None):
        self.device = torch.device(device or "cuda")
        self.arena = torch.empty(int(arena_bytes), dtype=torch.uint8, device=self.device)
        cfg = _abi.mgs_server_config(n_slots, max_batch_views, self.device.index or 0, 0,
                                     _ptr(self.arena), int(arena_bytes))
        self.h = C.c_void_p()
        check(load().mgs_server_create(C.byref(cfg), C.byref(self.h)), "mgs_server_create")
        self.scenes = []
        self.keep = {}

    def add_scene(self, g: Gaussians) -> int:
        sid = C.c_int32(0)
        check(load().mgs_server_add_scene(self.h, C.byref(g.struct()), C.byref(sid)), "mgs_server_add_scene")
        self.scenes.append(g)
        return sid.value

    def submit(self, scene_id: int, cam, out: Image, tag: int, t_submit: float = 0.0):
        c = camera_struct(cam)
        im = _abi.mgs_image(_ptr(out.rgb), _ptr(out.depth), _ptr(out.alpha))
        self.keep[tag] = out
        check(load().mgs_server_submit(self.h, scene_id, C.byref(c), C.byref(im), tag, t_submit),
              "mgs_server_submit")

    def poll(self, max_n: int = 256, wait_s: float = 0.0):
        """[(tag, t_submit, t_start, t_done, status)] of completed requests."""
        tags = (C.c_int64 * max_n)()
        ts, t0, t1 = (C.c_double * max_n)(), (C.c_double * max_n)(), (C.c_double * max_n)()
        st = (C.c_int32 * max_n)()
        n = load().mgs_server_poll(self.h, max_n, tags, ts, t0, t1, st, wait_s)
        res = []
        for i in range(n):
            self.keep.pop(tags[i], None)
            res.append((tags[i], ts[i], t0[i], t1[i], st[i]))
        return res

    @staticmethod
    def clock() -> float:
        return float(load().mgs_server_clock())

    def stats(self):
        """{launches, requests, max_views, mixed_scene_launches} since creation."""
        out = (C.c_int64 * 4)()
        check(load().mgs_server_stats(self.h, out), "mgs_server_stats")
        return dict(launches=int(out[0]), requests=int(out[1]), max_views=int(out[2]),
                    mixed_scene_launches=int(out[3]))

    def close(self):
        if self.h:
            load().mgs_server_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
