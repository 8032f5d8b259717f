"""GPU parity of the rasteriser (projection, sort, forward, backward) against the FP64
oracle, through the C ABI.  Sec. II-C Eq. 1-2, Sec. II-E Eq. 11."""
import math

import numpy as np
import pytest
import torch

from paper_2509_13536_gb300 import api, scenegen as sg
from tests import _gpu
from tests._scenes import camera, make_scene, random_scene

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_13536_gb300 import build
    build.build()
    torch.cuda.init()


# ------------------------------------------------------------------ sort
@pytest.mark.parametrize("n", [0, 1, 7, 4095, 4096, 4097, 100_003, (1 << 20) + 123])
@pytest.mark.parametrize("bits", [(0, 32), (0, 15), (3, 20)])
def test_radix_sort_matches_stable_argsort(n, bits):
    rng = np.random.default_rng(n + bits[1])
    keys = rng.integers(0, 2 ** 32, n, dtype=np.uint64).astype(np.uint32)
    if n > 10:
        keys[: n // 3] = keys[0]  # many equal keys: stability matters
    k = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    perm = api.mgs_sort_pairs(k, None, *bits)
    torch.cuda.synchronize()
    b0, b1 = bits
    sub = (keys.astype(np.uint64) >> np.uint64(b0)) & np.uint64((1 << (b1 - b0)) - 1)
    want = np.argsort(sub, kind="stable")
    np.testing.assert_array_equal(perm.cpu().numpy(), want.astype(np.int32))
    np.testing.assert_array_equal(k.cpu().numpy().view(np.uint32), keys[want])


def test_radix_sort_with_values():
    rng = np.random.default_rng(1)
    n = 50_000
    keys = rng.integers(0, 1000, n).astype(np.uint32)
    vals = rng.integers(0, 2 ** 31, n).astype(np.int32)
    k = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    v = torch.from_numpy(vals.copy()).cuda()
    api.mgs_sort_pairs(k, v, 0, 10)
    want = np.argsort(keys, kind="stable")
    np.testing.assert_array_equal(v.cpu().numpy(), vals[want])


def test_radix_sort_of_an_offset_view():
    """keys[1:] (4-byte aligned, not 16) sorts like an aligned copy of the same keys."""
    rng = np.random.default_rng(9)
    n = 70_001
    keys = rng.integers(0, 2 ** 32, n + 1, dtype=np.uint64).astype(np.uint32)
    base = torch.from_numpy(keys.view(np.int32).copy()).cuda()
    view = base[1:]
    assert view.data_ptr() % 16 != 0
    perm = api.mgs_sort_pairs(view, None, 0, 32)
    torch.cuda.synchronize()
    want = np.argsort(keys[1:], kind="stable")
    np.testing.assert_array_equal(perm.cpu().numpy(), want.astype(np.int32))
    np.testing.assert_array_equal(view.cpu().numpy().view(np.uint32), keys[1:][want])


def test_adam_rejects_misaligned_arrays():
    """The optimiser's 16-byte vector accesses need aligned f32 arrays: an offset view is
    refused on the host with an error, before anything is launched."""
    scene, _ = sg.workload("box10k")
    g = api.Gaussians.from_scene(scene, "cuda")
    grads, m, v = (api.Grads.zeros_like(g, stats=False) for _ in range(3))
    m.opacity_logit = torch.zeros(g.n + 1, device="cuda")[1:]
    with pytest.raises(Exception, match="16-byte aligned"):
        api.mgs_adam_step(g, grads, m, v, 1e-3)


# ------------------------------------------------------------------ projection
def test_projection_matches_oracle(orc):
    scene, cams = sg.workload("box10k")
    g = api.Gaussians.from_scene(scene, "cuda")
    out = api.mgs_project(g, cams[0])
    torch.cuda.synchronize()
    ref = orc.project(scene, cams[0])
    drawn = ref["radius"] > 0
    np.testing.assert_allclose(_gpu.to_np(out["mean2d"])[drawn], ref["mean2d"][drawn], atol=2e-5, rtol=0)
    np.testing.assert_allclose(_gpu.to_np(out["depth"]), ref["depth"], rtol=1e-7)
    c = ref["conic"][drawn]
    np.testing.assert_allclose(_gpu.to_np(out["conic"])[drawn], c, rtol=2e-4, atol=2e-6 * np.abs(c).max())
    np.testing.assert_allclose(_gpu.to_np(out["rgb"])[drawn], ref["rgb"][drawn], atol=2e-6)
    # integer extent decisions agree except at near-ties
    cov = ref["cov2d"][drawn]
    mid = 0.5 * (cov[:, 0] + cov[:, 2])
    lam = mid + np.sqrt(np.maximum(0.1, mid ** 2 - (cov[:, 0] * cov[:, 2] - cov[:, 1] ** 2)))
    r3 = 3 * np.sqrt(lam)
    tie = np.abs(r3 - np.round(r3)) < 2e-4
    rad = out["radius"].cpu().numpy()[drawn]
    assert (rad[~tie] == ref["radius"][drawn][~tie]).all()
    rect = out["rect"].cpu().numpy()[drawn]
    rect_ok = (rect == ref["rect"][drawn]).all(1)
    assert rect_ok[~tie].mean() > 0.999


# ------------------------------------------------------------------ forward / backward
def test_render_box10k_matches_oracle(orc):
    scene, cams = sg.workload("box10k")
    g, imgs, ws = _gpu.render_gpu(scene, cams)
    ref = orc.render_outcomes(scene, cams[0])
    rep = _gpu.check_image(imgs[0], ref, what="box10k")
    print("box10k", rep, "keys", ws.n_keys)


def test_backward_box10k_matches_oracle(orc):
    """Every Gaussian's gradient, element by element, with the cotangent U[-1, 1] on the
    pixels the oracle does not flag (zero on the flagged ones, which then add nothing)."""
    scene, cams = sg.workload("box10k")
    g, imgs, ws = _gpu.render_gpu(scene, cams)
    refs = [orc.render_outcomes(scene, cams[0])]
    cot_np, dL = _gpu.masked_cotangents(cams, refs, 0)
    grads = api.render_backward(g, cams, dL, ws)
    torch.cuda.synchronize()
    ref = _gpu.oracle_backward(orc, scene, cams, cot_np)
    errs = _gpu.check_grads(grads, ref, what="box10k")
    print("box10k grads", errs)
    np.testing.assert_allclose(_gpu.to_np(grads.vis_count), ref["vis_count"])
    gs, rs = _gpu.to_np(grads.grad_stat), ref["grad_stat"]
    assert np.linalg.norm(gs - rs) / np.linalg.norm(rs) < 1e-3
    assert (np.abs(gs - rs) <= 1e-3 * (rs + 1e-3 * np.sqrt(np.mean(rs ** 2)))).all()


@pytest.mark.parametrize("deg", [1, 3])
def test_multiview_mixed_resolution_sh(orc, deg):
    rng = np.random.default_rng(20 + deg)
    scene = sg.room_scene(20_000, 5 + deg, sh_degree=deg)
    cams = sg.room_poses(2, 7, 160, 120) + sg.room_poses(1, 8, 97, 61)
    g, imgs, ws = _gpu.render_gpu(scene, cams)
    refs = [orc.render_outcomes(scene, c) for c in cams]
    for v, c in enumerate(cams):
        _gpu.check_image(imgs[v], refs[v], what=f"view {v}")
    cot_np, dL = _gpu.masked_cotangents(cams, refs, 3)
    grads = api.render_backward(g, cams, dL, ws)
    torch.cuda.synchronize()
    ref = _gpu.oracle_backward(orc, scene, cams, cot_np)
    _gpu.check_grads(grads, ref, what=f"multiview deg {deg}")


def test_empty_and_culled_scenes(orc):
    cam = camera(37, 29, 30, 30, 18, 14)
    for n in (0, 5):
        sc = make_scene([[0, 0, -1.0]] * n, [[0.1] * 3] * n, [[1, 0, 0, 0]] * n, [0.5] * n, [[1, 0, 0]] * n)
        g, imgs, ws = _gpu.render_gpu(sc, [cam])
        assert float(imgs[0].alpha.abs().max()) == 0.0 and float(imgs[0].rgb.abs().max()) == 0.0
        dL = [api.Image(torch.ones(3, 29, 37, device="cuda"), torch.ones(29, 37, device="cuda"),
                        torch.ones(29, 37, device="cuda"))]
        grads = api.render_backward(g, [cam], dL, ws)
        torch.cuda.synchronize()
        for t in grads.tensors():
            assert float(t.abs().sum()) == 0.0


@pytest.mark.parametrize("seed", range(4))
def test_ragged_tiny_scenes(orc, seed):
    """Image sizes that are not tile multiples, Gaussians straddling borders, SH 0..3,
    some behind the camera, one covering everything."""
    rng = np.random.default_rng(200 + seed)
    sc = random_scene(rng, 64, sh_degree=seed, spread=1.2, depth=2.5)
    sc.means[:4, 2] = rng.uniform(-1.0, 0.25, 4)
    sc.log_scales[4] = np.log(np.float32(2.0))
    cam = camera(53, 37, 30, 31, 26.1, 17.7)
    g, imgs, ws = _gpu.render_gpu(sc, [cam])
    ref = orc.render_outcomes(sc, cam)
    _gpu.check_image(imgs[0], ref, what=f"ragged {seed}")
    cot_np, dL = _gpu.masked_cotangents([cam], [ref], seed)
    grads = api.render_backward(g, [cam], dL, ws)
    torch.cuda.synchronize()
    ref_g = _gpu.oracle_backward(orc, sc, [cam], cot_np)
    _gpu.check_grads(grads, ref_g, what=f"ragged {seed}")


def test_workspace_regrowth_and_determinism(orc):
    scene, cams = sg.workload("box10k")
    g = api.Gaussians.from_scene(scene, "cuda")
    ws = api.RenderWorkspace("cuda")
    ws.ensure(g.n, cams, 10)  # far too small: the binding must grow it and retry
    a = api.new_images(cams)
    api.mgs_render(g, cams, a, ws)
    b = api.new_images(cams)
    api.mgs_render(g, cams, b, ws)
    torch.cuda.synchronize()
    assert torch.equal(a[0].rgb, b[0].rgb) and torch.equal(a[0].alpha, b[0].alpha)


def test_async_render_matches_and_reports_overflow():
    """mgs_render_async (no host round trip) gives the images and the backward state of
    mgs_render bit for bit; with a workspace too small for its keys it blends nothing,
    reports the overflow through its status, and the binding's check() raises."""
    scene, cams = sg.workload("box10k")
    g = api.Gaussians.from_scene(scene, "cuda")
    ref, ws0 = api.render(g, cams)
    ws = api.RenderWorkspace("cuda")
    api.mgs_render(g, cams, api.new_images(cams), ws)  # sizes the workspace
    out = api.new_images(cams)
    assert api.mgs_render(g, cams, out, ws, sync=False) == -1
    assert ws.check() == ws0.n_keys
    for plane in ("rgb", "depth", "alpha"):
        assert torch.equal(getattr(out[0], plane), getattr(ref[0], plane)), plane
    cot_np, dL = _gpu.cotangents(cams, 4)
    a = api.render_backward(g, cams, dL, ws)
    b = api.render_backward(g, cams, dL, ws0)
    torch.cuda.synchronize()
    for x, y in zip(a.tensors(), b.tensors()):  # same kernels; float atomics land in any order
        assert float((x - y).norm()) <= 1e-5 * float(y.norm())
    small = api.RenderWorkspace("cuda")
    small.ensure(g.n, cams, ws0.n_keys // 2)
    out = api.new_images(cams)
    api.mgs_render(g, cams, out, small, sync=False)
    with pytest.raises(Exception, match="exceeded"):
        small.check()
    assert int(small.status[1]) == 1 and int(small.status[0]) == ws0.n_keys
    assert float(out[0].alpha.abs().max()) == 0.0  # nothing blended


def test_backward_store_mode_equals_accumulating_into_zeros():
    """grads.overwrite: the backward stores the call's gradients -- what adding them to
    zeroed arrays gives, up to the rounding order of the float atomics that sum the
    per-tile moments (relative L2 <= 1e-5) -- with exact zeros for Gaussians no view
    draws (here a quarter behind the camera), whatever the arrays held; the Eq. 3 sums
    still accumulate."""
    rng = np.random.default_rng(21)
    sc = random_scene(rng, 800, sh_degree=1)
    sc.means[::4, 2] = -2.0  # behind the camera in both views
    cams = [camera(96, 80, 90, 90, 47.5, 39.5), camera(96, 80, 100, 95, 45.0, 41.0)]
    g, imgs, ws = _gpu.render_gpu(sc, cams)
    grng = np.random.default_rng(22)
    dL = [api.Image(*(torch.from_numpy(grng.uniform(-1, 1, s).astype(np.float32)).cuda()
                      for s in ((3, 80, 96), (80, 96), (80, 96)))) for _ in cams]
    acc = api.Grads.zeros_like(g)
    api.mgs_render_backward(g, cams, dL, ws, acc)
    junk = lambda t: torch.full(t.shape, float("nan"), dtype=torch.float32, device=t.device)
    st = api.Grads(junk(g.means), junk(g.log_scales), junk(g.quats), junk(g.opacity_logit), junk(g.sh),
                   torch.ones(g.n, device="cuda"), torch.ones(g.n, device="cuda"), overwrite=True)
    for _ in range(2):  # a second call stores again (the sums keep accumulating)
        api.mgs_render_backward(g, cams, dL, ws, st)
    torch.cuda.synchronize()
    for a, b in zip(acc.tensors(), st.tensors()):
        assert torch.isfinite(b).all()
        assert float(torch.linalg.vector_norm(a - b) / torch.linalg.vector_norm(a)) <= 1e-5
    assert (acc.vis_count[::4] == 0).all()
    for t in st.tensors():
        assert (t[::4] == 0).all()
    torch.testing.assert_close(st.grad_stat, 1 + 2 * acc.grad_stat, rtol=1e-6, atol=0)
    assert torch.equal(st.vis_count, 1 + 2 * acc.vis_count)


def test_reused_workspace_backward_equals_a_fresh_one():
    """The projection clears only the drawn items' moment accumulators and the reverse
    pass leaves them dirty: render views A and take the reverse pass, then render other
    views B (other drawn items) on the same workspace and take theirs.  The gradients
    equal those of B on a fresh workspace (up to the rounding order of the float atomics
    that sum the per-tile moments: relative L2 <= 1e-5), and so do those of a second
    reverse pass of B (the dirty buffer is cleared first)."""
    rng = np.random.default_rng(23)
    sc = random_scene(rng, 1500, sh_degree=1, spread=1.3)
    th = 0.5
    Ry = np.array([[math.cos(th), 0, math.sin(th)], [0, 1, 0], [-math.sin(th), 0, math.cos(th)]])
    cams_a = [camera(96, 80, 90, 90, 47.5, 39.5), camera(64, 48, 70, 70, 31.5, 23.5, R=Ry)]
    cams_b = [camera(80, 96, 100, 95, 41.0, 45.0, R=Ry.T, t=np.array([0.2, 0.0, 0.3]))]
    grng = np.random.default_rng(24)

    def cot(cams):
        return [api.Image(*(torch.from_numpy(grng.uniform(-1, 1, s).astype(np.float32)).cuda()
                            for s in ((3, c.height, c.width), (c.height, c.width), (c.height, c.width))))
                for c in cams]

    dL_a, dL_b = cot(cams_a), cot(cams_b)
    g, _, ws = _gpu.render_gpu(sc, cams_a)
    api.render_backward(g, cams_a, dL_a, ws)
    api.render(g, cams_b, ws)
    reused = api.render_backward(g, cams_b, dL_b, ws)
    again = api.render_backward(g, cams_b, dL_b, ws)
    _, _, ws2 = _gpu.render_gpu(sc, cams_b)
    fresh = api.render_backward(g, cams_b, dL_b, ws2)
    torch.cuda.synchronize()
    for a, b, c in zip(fresh.tensors(), reused.tensors(), again.tensors()):
        n = float(torch.linalg.vector_norm(a))
        assert n > 0
        assert float(torch.linalg.vector_norm(a - b)) <= 1e-5 * n
        assert float(torch.linalg.vector_norm(a - c)) <= 1e-5 * n


def test_three_pass_tile_sort_matches_single_views():
    """32 full-HD views in one launch hold 261,120 tiles: the tile sort takes three 8-bit
    passes and writes the tile ranges in the third.  Every image (and its backward
    state) must equal the same view rendered alone, where one or two passes suffice."""
    rng = np.random.default_rng(33)
    sc = random_scene(rng, 20000, sh_degree=1, spread=1.5, depth=3.5)
    cams = []
    for v in range(32):
        t = np.float32([rng.uniform(-0.3, 0.3), rng.uniform(-0.3, 0.3), rng.uniform(-0.5, 0.5)])
        cams.append(camera(1920, 1080, 900.0, 900.0, 959.5, 539.5, t=t))
    g = api.Gaussians.from_scene(sc, "cuda")
    imgs, _ = api.render(g, cams)
    torch.cuda.synchronize()
    for v in (0, 7, 19, 31):
        alone, _ = api.render(g, [cams[v]])
        torch.cuda.synchronize()
        for plane in ("rgb", "depth", "alpha"):
            assert torch.equal(getattr(imgs[v], plane), getattr(alone[0], plane)), (v, plane)
    assert float(imgs[5].alpha.max()) > 0.5  # the views do see the scene
