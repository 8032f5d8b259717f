"""The mapping step driven through torch.autograd (RenderFn + MappingStep) against the
FP64 oracle's own steps: render (Eq. 11), the Eq. 12 loss with its isotropic term,
the reverse pass, Adam.  Sec. II-E."""
import numpy as np
import pytest
import torch

from paper_2509_13536_gb300 import api, scenegen as sg
from tests import _gpu

pytestmark = pytest.mark.gpu

FIELDS = _gpu.FIELDS
LR, B1, B2, EPS = 1e-3, 0.9, 0.999, 1e-8
LAM, W_DEPTH, W_ISO = 0.2, 0.5, 0.1


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_13536_gb300 import build
    build.build()


def _scene_with(scene, params):
    s = scene.copy()
    for k in FIELDS:
        setattr(s, k, params[k])
    return s


def _oracle_grad(orc, scene, cams, y, dt, P):
    """Loss and summed gradient of the oracle at parameters P (float64)."""
    sc = _scene_with(scene, P)
    outs = [orc.render_outcomes(sc, c) for c in cams]
    x = np.stack([o["rgb"] for o in outs])
    d = np.stack([o["depth"] for o in outs])
    lo = orc.mapping_loss(x, y, d, dt, lam=LAM, w_depth=W_DEPTH)
    grads = orc.new_grads(scene.n, scene.sh_degree, scale=True)
    for v, c in enumerate(cams):
        orc.render_backward(sc, c, lo["g_rgb"][v], lo["g_depth"][v], None, grads=grads)
    iso, g_ls = orc.iso_loss(P["log_scales"], W_ISO)
    grads["log_scales"] += g_ls
    grads["scale_log_scales"] += np.abs(g_ls)
    return dict(x=x, d=d, flags=np.stack([o["flags"] for o in outs]), loss=lo["loss"], iso=iso,
                grads={k: grads[k].copy() for k in FIELDS},
                scale={k: grads["scale_" + k].copy() for k in FIELDS}, taint=grads["taint"].copy())


def _grad_bound(gt, scale):
    """The element-wise gradient bound of the other parity tests."""
    return np.maximum(1e-3 * (np.abs(gt) + 1e-3 * np.sqrt(np.mean(gt ** 2))), _gpu.ERR_SAFETY * scale)


def _oracle_steps(orc, scene, cams, y, dt, n_steps=2):
    """The oracle's own steps from the FP64 copy of the map: per step the per-view images,
    flags and loss, the summed gradient and the parameters after Adam."""
    P = {k: getattr(scene, k).astype(np.float64).copy() for k in FIELDS}
    M = {k: np.zeros_like(v) for k, v in P.items()}
    Vs = {k: np.zeros_like(v) for k, v in P.items()}
    hist = []
    for t in range(1, n_steps + 1):
        h = _oracle_grad(orc, scene, cams, y, dt, P)
        hist.append(h)
        for k in FIELDS:
            orc.adam(P[k], h["grads"][k], M[k], Vs[k], LR, B1, B2, EPS, t)
        h["P_after"] = {k: v.copy() for k, v in P.items()}
    return hist, P


def _second_step_gradient_spread(orc, scene, cams, y, dt, hist):
    """How far the step-2 gradient moves when the step-1 parameters move within what the
    step-1 gradient bound allows (the Adam step over g1 +- e1, plus float32 rounding):
    the oracle's step-2 gradient at P1 + s B1 for four sign patterns s (all-plus,
    all-minus, two seeded random ones), largest change per element."""
    P1 = hist[0]["P_after"]
    B = {}
    for k in FIELDS:
        g1 = hist[0]["grads"][k]
        e1 = _grad_bound(g1, hist[0]["scale"][k])
        d0 = _adam_np([g1])
        B[k] = np.maximum(np.abs(_adam_np([g1 + e1]) - d0), np.abs(_adam_np([g1 - e1]) - d0)) + \
            np.spacing(np.abs(P1[k]).astype(np.float32)).astype(np.float64)
    rng = np.random.default_rng(23)
    spread = {k: np.zeros_like(v) for k, v in P1.items()}
    for pattern in range(4):
        Pp = {}
        for k in FIELDS:
            sgn = 1.0 if pattern == 0 else -1.0 if pattern == 1 else rng.choice([-1.0, 1.0], P1[k].shape)
            Pp[k] = P1[k] + sgn * B[k]
        hp = _oracle_grad(orc, scene, cams, y, dt, Pp)
        for k in FIELDS:
            spread[k] = np.maximum(spread[k], np.abs(hp["grads"][k] - hist[1]["grads"][k]))
    return spread


def _adam_np(g_list):
    """Parameter change after len(g_list) Adam steps (bias-corrected), in float64."""
    m = v = 0.0
    delta = 0.0
    for t, g in enumerate(g_list, 1):
        m = B1 * m + (1 - B1) * g
        v = B2 * v + (1 - B2) * g * g
        delta = delta - LR * (m / (1 - B1 ** t)) / (np.sqrt(v / (1 - B2 ** t)) + EPS)
    return delta


@pytest.fixture(scope="module")
def mapping_case(orc):
    """A small room map, 2 keyframes, random keyframe images; Gaussians that reach a pixel
    with a near-tie decision in either step are dropped, and target values within 1e-4
    of the oracle's rendered value are moved, until the oracle's two steps take no
    near-tie decision and no L1 sign is in doubt (all on the CPU, oracle only)."""
    scene = sg.room_scene(6000, 17, sh_degree=1)
    cams = sg.room_poses(2, 18, 96, 72)
    rng = np.random.default_rng(19)
    V, H, W = len(cams), cams[0].height, cams[0].width
    y = rng.uniform(0, 1, (V, 3, H, W))
    dt = rng.uniform(0.5, 4.0, (V, H, W))
    dt[:, ::5, ::3] = 0
    for _ in range(8):
        hist, P = _oracle_steps(orc, scene, cams, y, dt)
        flagged = any(h["flags"].any() for h in hist)
        taint = np.zeros(scene.n, bool)
        for h in hist:
            taint |= h["taint"] > 0
        moved = False
        for h in hist:
            close = np.abs(h["x"] - y) < 1e-4
            if close.any():
                y = np.where(close, np.where(y > 0.5, y - 0.01, y + 0.01), y)
                moved = True
            dclose = (np.abs(h["d"] - dt) < 1e-4) & (dt > 0)
            if dclose.any():
                dt = np.where(dclose, dt + 0.01, dt)
                moved = True
        if not flagged and not moved:
            dg2 = _second_step_gradient_spread(orc, scene, cams, y, dt, hist)
            break
        if flagged:
            scene = scene.subset(np.nonzero(~taint)[0])
    else:
        pytest.fail("could not scrub the mapping case")
    return dict(scene=scene, cams=cams, y=y.astype(np.float32), dt=dt.astype(np.float32), hist=hist, P=P,
                dg2=dg2)


def test_two_mapping_steps_match_the_oracle(mapping_case):
    """Two MappingStep calls (RenderFn forward, Eq. 12 loss with lambda 0.2 and the depth
    and isotropic terms, autograd backward, in-kernel Adam) against the oracle's own two
    steps from the same map: per-view loss parts, and every parameter element within
    the gradient tolerance propagated through Adam (the largest change of the Adam
    update over g_t +- e_t, t = 1, 2, with e_t the element-wise gradient bound of the
    other parity tests, e_2 widened by how far the step-2 gradient moves when the
    step-1 parameters move within their own bound) plus float32 rounding."""
    c = mapping_case
    scene, cams, hist = c["scene"], c["cams"], c["hist"]
    g = api.Gaussians.from_scene(scene, "cuda")
    step = api.MappingStep(g, cams, lr=LR, lambda_ssim=LAM, w_depth=W_DEPTH, w_iso=W_ISO)
    y, dt = torch.from_numpy(c["y"]).cuda(), torch.from_numpy(c["dt"]).cuda()
    for t in range(2):
        loss = step(y, dt)
        torch.cuda.synchronize()
        np.testing.assert_allclose(loss.cpu().numpy(), hist[t]["loss"], rtol=1e-4, atol=1e-7)
        np.testing.assert_allclose(float(step.loss_iso.item()), hist[t]["iso"], rtol=1e-5)
    worst = 0.0
    for k in FIELDS:
        ref = c["P"][k]
        gpu = _gpu.to_np(getattr(g, k))
        g1, g2 = hist[0]["grads"][k], hist[1]["grads"][k]
        e1 = _grad_bound(g1, hist[0]["scale"][k])
        e2 = _grad_bound(g2, hist[1]["scale"][k]) + c["dg2"][k]
        nominal = _adam_np([g1, g2])
        spread = np.zeros_like(ref)
        for s1 in (-1, 1):
            for s2 in (-1, 1):
                spread = np.maximum(spread, np.abs(_adam_np([g1 + s1 * e1, g2 + s2 * e2]) - nominal))
        bound = spread + 4 * np.spacing(np.abs(ref).astype(np.float32)).astype(np.float64) + 1e-12
        r = np.abs(gpu - ref) / bound
        i = int(np.argmax(r))
        worst = max(worst, float(r.flat[i]))
        assert r.flat[i] <= 1.0, (k, np.unravel_index(i, ref.shape), gpu.flat[i], ref.flat[i], bound.flat[i])
        assert np.abs(gpu - getattr(scene, k)).max() > 0  # the step really moved the map
    print("two mapping steps: worst |gpu - oracle| / bound", worst, "Gaussians", scene.n)


def test_render_fn_gradients_match_the_oracle(orc):
    """RenderFn's backward (plain autograd, new gradient tensors) and its in-place form
    (gradients accumulated into a Grads) against the oracle's gradient, element-wise,
    with the cotangent on unflagged pixels."""
    scene, cams = sg.workload("box10k")
    refs = [orc.render_outcomes(scene, cams[0])]
    cot_np, dL = _gpu.masked_cotangents(cams, refs, 11)
    ref = _gpu.oracle_backward(orc, scene, cams, cot_np)
    g = api.Gaussians.from_scene(scene, "cuda")
    params = [p.clone().requires_grad_(True) for p in g.params()]
    ws = api.RenderWorkspace("cuda")
    rgb, depth, alpha = api.RenderFn.apply(*params, cams, ws)
    torch.autograd.backward((rgb, depth, alpha), (dL[0].rgb[None], dL[0].depth[None], dL[0].alpha[None]))
    torch.cuda.synchronize()
    got = api.Grads(*(p.grad for p in params))
    _gpu.check_grads(got, ref, what="RenderFn")
    into = api.Grads.zeros_like(g, stats=False)
    ws2 = api.RenderWorkspace("cuda")
    params2 = [p.detach().clone().requires_grad_(True) for p in g.params()]
    rgb, depth, alpha = api.RenderFn.apply(*params2, cams, ws2, into)
    torch.autograd.backward((rgb, depth, alpha), (dL[0].rgb[None], dL[0].depth[None], dL[0].alpha[None]))
    torch.cuda.synchronize()
    assert all(p.grad is None for p in params2)
    _gpu.check_grads(into, ref, what="RenderFn in place")


def test_render_fn_refuses_a_reused_workspace():
    """A second render into the same workspace before the first one's backward pass
    overwrites the saved state that backward pass needs: it raises instead of returning
    wrong gradients."""
    scene, cams = sg.workload("box10k")
    g = api.Gaussians.from_scene(scene, "cuda")
    params = [p.clone().requires_grad_(True) for p in g.params()]
    ws = api.RenderWorkspace("cuda")
    rgb1, _, _ = api.RenderFn.apply(*params, cams, ws)
    rgb2, _, _ = api.RenderFn.apply(*params, cams, ws)
    with pytest.raises(RuntimeError, match="reused or regrown"):
        rgb1.backward(torch.ones_like(rgb1))
    rgb2.backward(torch.ones_like(rgb2))  # the latest render's state is intact
    torch.cuda.synchronize()
    assert params[0].grad is not None and torch.isfinite(params[0].grad).all()


def test_merge_on_a_side_stream_sees_its_own_step():
    """The mapping step with the voxel merge of step k on a stream of its own, running
    beside step k+1 (which renders meanwhile, its Adam update waiting for the merge
    through ``before_update``): the merge equals a merge of the map as step k left it,
    taken afterwards on the main stream."""
    scene, cams = sg.workload("box10k")
    g = api.Gaussians.from_scene(scene, "cuda")
    step = api.MappingStep(g, cams, lr=1e-2, lambda_ssim=0.0, w_depth=0.1)
    rng = np.random.default_rng(5)
    y = torch.from_numpy(rng.random((1, 3, cams[0].height, cams[0].width)).astype(np.float32)).cuda()
    dt = torch.from_numpy(rng.uniform(1, 3, (1, cams[0].height, cams[0].width)).astype(np.float32)).cuda()
    side = torch.cuda.Stream()
    ev_updated, ev_merged = torch.cuda.Event(), torch.cuda.Event()
    out = g.empty_like()
    partner = torch.empty(g.n, dtype=torch.int32, device="cuda")
    vox = torch.empty(g.n, 3, dtype=torch.int32, device="cuda")
    status = torch.zeros(2, dtype=torch.int32, pin_memory=True)
    step(y, dt)
    snap = api.Gaussians(*(p.detach().clone() for p in g.params()), g.birth.clone())  # the map after step 1
    ev_updated.record(torch.cuda.current_stream())
    side.wait_event(ev_updated)
    api.mgs_voxel_merge(g, 0.05, out=out, partner=partner, vox=vox, status=status, stream=side)
    ev_merged.record(side)
    for _ in range(2):  # steps 2 and 3 render while the merge runs; step 2's update waits for it
        step(y, dt, before_update=ev_merged)
    torch.cuda.synchronize()
    ref, ref_partner, ref_vox = api.mgs_voxel_merge(snap, 0.05)
    torch.cuda.synchronize()
    k = int(status[0])
    assert k == ref.n and k < g.n  # something merged
    assert torch.equal(partner, ref_partner) and torch.equal(vox, ref_vox)
    for a, b in zip(ref.params(), out.params()):
        assert torch.equal(a, b[:k])
