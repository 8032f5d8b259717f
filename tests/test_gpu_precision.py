"""Reduced-precision attribute storage, all arithmetic FP32.  The default reduced mode
stores the appearance group (opacity logit, SH: 49 of 59 scalars) in FP16 / BF16 and
keeps the geometry (means, log-scales, quaternions) FP32: 138 bytes per SH3 Gaussian
instead of 236.  Checked two ways against the FP64 oracle: (i) fed the dequantised
attributes, at the FP32 path's tolerances; (ii) fed the original FP32 attributes:
PSNR >= 50 dB and gradient relative error <= 1e-2.  Storing the geometry reduced too
(124 bytes) is checked against (i) only: it moves gradients by ~1e-2 (FP16) to ~3e-2
(BF16) relative to the FP32 map."""
import numpy as np
import pytest
import torch

from paper_2509_13536_gb300 import api, scenegen as sg
from tests import _gpu

pytestmark = pytest.mark.gpu

DTYPES = {"f16": torch.float16, "bf16": torch.bfloat16}


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_13536_gb300 import build
    build.build()


def dequantised(scene, dt, geom_dt=torch.float32):
    q = scene.copy()
    for k, d in (("log_scales", geom_dt), ("quats", geom_dt), ("opacity_logit", dt), ("sh", dt)):
        v = torch.from_numpy(getattr(scene, k)).to(d).to(torch.float32).numpy()
        setattr(q, k, v)
    return q


def psnr(a, b):
    mse = float(np.mean((a - b) ** 2))
    return 10 * np.log10(1.0 / max(mse, 1e-30))


def bytes_per_gaussian(g: api.Gaussians):
    return sum(t[0].numel() * t.element_size() for t in g.params())


@pytest.fixture(scope="module")
def workload():
    scene = sg.room_scene(60_000, 11, sh_degree=3)
    cams = sg.room_poses(2, 12, 320, 240)
    return scene, cams


@pytest.mark.parametrize("name", ["f16", "bf16"])
def test_reduced_precision_storage(orc, workload, name):
    scene, cams = workload
    dt = DTYPES[name]
    g = api.Gaussians.from_scene(scene, "cuda", dt)
    assert bytes_per_gaussian(g) == 138
    assert bytes_per_gaussian(api.Gaussians.from_scene(scene, "cuda")) == 236
    imgs, ws = api.render(g, cams)
    deq = dequantised(scene, dt)
    refs = [orc.render_outcomes(deq, c) for c in cams]
    cot_np, dL = _gpu.masked_cotangents(cams, refs, 21)
    grads = api.render_backward(g, cams, dL, ws)
    torch.cuda.synchronize()
    # (i) same inputs as the kernels see: FP32-path tolerances
    for v, c in enumerate(cams):
        _gpu.check_image(imgs[v], refs[v], what=f"{name} view {v} vs dequantised")
    ref_q = _gpu.oracle_backward(orc, deq, cams, cot_np)
    _gpu.check_grads(grads, ref_q, what=f"{name} vs dequantised")
    # (ii) against the original FP32 map
    worst = 1e9
    for v, c in enumerate(cams):
        ref = orc.render(scene, c)
        worst = min(worst, psnr(_gpu.to_np(imgs[v].rgb), ref["rgb"]))
    assert worst >= 50.0, f"{name}: PSNR {worst:.1f} dB"
    ref_f = _gpu.oracle_backward(orc, scene, cams, cot_np)
    errs = _gpu.check_grads(grads, ref_f, ref_f["taint"], rel=1e-2, elem=None, what=f"{name} vs FP32 map")
    print(name, "PSNR", round(worst, 2), "grad rel", {k: f"{e:.2e}" for k, e in errs.items()})


@pytest.mark.parametrize("name", ["f16", "bf16"])
def test_fully_reduced_storage_matches_dequantised_oracle(orc, workload, name):
    """Geometry stored reduced as well (124 B / Gaussian): exact to the FP32-path
    tolerances against the oracle fed the same dequantised values."""
    scene, cams = workload
    dt = DTYPES[name]
    g = api.Gaussians.from_scene(scene, "cuda", dt, dt)
    assert bytes_per_gaussian(g) == 124
    imgs, ws = api.render(g, cams)
    deq = dequantised(scene, dt, dt)
    refs = [orc.render_outcomes(deq, c) for c in cams]
    cot_np, dL = _gpu.masked_cotangents(cams, refs, 22)
    grads = api.render_backward(g, cams, dL, ws)
    torch.cuda.synchronize()
    for v, c in enumerate(cams):
        _gpu.check_image(imgs[v], refs[v], what=f"{name} full view {v}")
    ref = _gpu.oracle_backward(orc, deq, cams, cot_np)
    _gpu.check_grads(grads, ref, what=f"{name} full")


@pytest.mark.parametrize("name", ["f16", "bf16"])
def test_reduced_precision_merge_and_adam_run(orc, name):
    """Merge and Adam accept reduced-precision maps: merge clusters match the FP32 merge of
    the dequantised map; Adam updates stay in the storage type."""
    from tests.test_gpu_merge import scrub
    from tests.test_oracle_merge import _voxel_scene
    dt = DTYPES[name]
    rng = np.random.default_rng(31)
    sc = dequantised(_voxel_scene(rng, 80, 5), dt, dt)
    sc, ref = scrub(orc, sc, 0.02)
    g = api.Gaussians.from_scene(sc, "cuda", dt, dt)
    out, partner, _ = api.mgs_voxel_merge(g, 0.02)
    torch.cuda.synchronize()
    np.testing.assert_array_equal(partner.cpu().numpy(), ref["partner"])
    assert out.log_scales.dtype == dt and out.sh.dtype == dt and out.n == ref["n_out"]
    grads = api.Grads.zeros_like(g, stats=False)
    for t in grads.tensors():
        t.normal_()
    m = api.Grads.zeros_like(g, stats=False)
    v = api.Grads.zeros_like(g, stats=False)
    before = g.sh.clone()
    api.mgs_adam_step(g, grads, m, v, 1e-2, step=1)
    torch.cuda.synchronize()
    assert g.sh.dtype == dt and not torch.equal(before, g.sh)
