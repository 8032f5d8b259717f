#!/usr/bin/env python
"""Benchmark of the batched mapping step: fwd+bwd frames/s at 1M Gaussians, 1200x680.

One step = one pass of the whole hot path over one batch of 8 keyframes: projection
of the 1M-Gaussian SH3 map into all 8 views, depth sort, tile sort, forward blend, L1
loss gradient against the keyframe images, backward blend, per-Gaussian chain rule,
Adam (lr 1e-3) and the voxel merge (v = 0.02 m) of the updated map.  ``value`` =
views rendered and back-propagated per second over all ranks, inputs resident in HBM;
``e2e`` = the same through host buffers (keyframe images copied in from pinned host
memory each step, the loss read back each step).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

``--impl reference`` times the FP64 CPU oracle on a bounded sample of the same
workload (there is no runnable reference implementation of the paper).
"""
from __future__ import annotations

import argparse
import gc
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "fwd+bwd frames/s @1M Gaussians 1200x680"
WORKLOAD = "room1m_sh3"
WORKLOAD_DESC = ("1M Gaussians on the walls of a 4x3x3 m room (20% near-duplicates), SH degree 3, "
                 "8 keyframes at 1200x680 (fx=fy=600); step = render 8 views + L1 grad + backward + "
                 "Adam lr 1e-3 + voxel_merge v=0.02 m")
FWD_FLOP_EVAL, FWD_FLOP_CONTRIB = 10, 10      # per evaluated / per contributing (pixel, entry)
BWD_FLOP_EVAL, BWD_FLOP_CONTRIB = 10, 47
# DRAM bytes per launch (dram__bytes_read.sum + dram__bytes_write.sum) from one ncu capture
# of the full workload (8 views, one launch per step; profiles/ has the command).  A value
# is reported only while the kernel sources still hash to the captured version.
NCU_TRAFFIC_SOURCES = ["paper_2509_13536_gb300/csrc/raster.cu", "paper_2509_13536_gb300/csrc/common.cuh"]
NCU_TRAFFIC = {"sha256_16": "caa7bf7cd63bea3f", "blend_bwd": 670.48e6 + 91.39e6, "blend_fwd": 357.48e6 + 143.22e6}


def algorithmic_bytes(n, views, stats, pb, pixels):
    """HBM bytes per step each kernel group must move at least (model, per the kernels'
    data layout): n Gaussians of pb parameter bytes, views x n (view, Gaussian) items of
    which `drawn_items` are drawn, `keys` (Gaussian, tile) keys, `pixels` output pixels.
    Gradients and Adam state are f32 (236 B per SH3 Gaussian)."""
    d, k, vn = stats["drawn_items"], stats["keys"], views * n
    g32 = 4 * 59  # f32 gradient bytes of an SH3 Gaussian
    return {
        "preprocess": (n * pb + 16 * vn + 48 * d,
                       "parameters once + 16 B per item (rect, count, depth key) + 48 B record per drawn item"),
        "depth_sort": (8 * vn + 80 * d, "first pass over all items (4 B histogram + 4 B key read; the values are "
                                        "the item index), 8 B written per drawn item, three more passes of 20 B "
                                        "per drawn item, the scan of the key counts (12 B per drawn item)"),
        "emit": (52 * d + 8 * k, "52 B read per drawn item (order, offset, count, rect, conic), 8 B per key written"),
        "tile_sort": (40 * k, "two passes of 20 B per key (histogram read, key and value read and written); "
                              "the last pass also writes the tile ranges"),
        "preprocess_bwd": (n * (pb + g32 + 16) + 12 * vn + 48 * d,
                           "parameters read, f32 gradients written (the step's backward stores them), "
                           "Eq. 3 sums read and written, 12 B per item, 48 B moments per drawn item"),
        "adam": (n * 59 * 28, "per f32 parameter: parameter, gradient, m, v read; parameter, m, v written"),
        "l1_loss": (48 * pixels, "per pixel: rgb and depth read, targets read, cotangents written (4 B each)"),
    }


def recorded_traffic(kernel):
    import hashlib
    h = hashlib.sha256()
    for f in NCU_TRAFFIC_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return NCU_TRAFFIC.get(kernel) if h.hexdigest()[:16] == NCU_TRAFFIC["sha256_16"] else None


def parse():
    p = argparse.ArgumentParser()
    p.add_argument("--gpus", type=int, default=1)
    p.add_argument("--steps", type=int, default=200)
    p.add_argument("--warmup", type=int, default=3)
    p.add_argument("--impl", choices=["ours", "reference"], default="ours")
    p.add_argument("--no-cpu-baseline", action="store_true")
    p.add_argument("--cpu-reps", type=int, default=3, help="times the oracle baseline renders keyframe 0")
    p.add_argument("--no-configs", action="store_true", help="skip the box10k and room300k legs")
    p.add_argument("--views", type=int, default=8, help="keyframes per step (8 = the benchmark workload)")
    p.add_argument("--no-e2e", action="store_true")
    p.add_argument("--no-precision", action="store_true")
    p.add_argument("--precision-modes", nargs="*", default=None, help="subset of the storage layouts to measure")
    p.add_argument("--no-eq12", action="store_true")
    p.add_argument("--no-serving", action="store_true")
    p.add_argument("--serve-requests", type=int, default=2000)
    p.add_argument("--serve-rate", type=float, default=200.0)
    p.add_argument("--serve-sweep", type=float, nargs="*", default=[1000.0, 3000.0],
                   help="offered rates (req/s) of the saturation sweep")
    p.add_argument("--serve-sweep-requests", type=int, default=1000)
    return p.parse_args()


def dist_env():
    return int(os.environ.get("RANK", 0)), int(os.environ.get("WORLD_SIZE", 1)), int(os.environ.get("LOCAL_RANK", 0))


def replica_seed(rank):
    """Seed of the perturbed map each rank optimises: replicas are independent maps."""
    return 1234 + rank


def max_over_ranks(ms, world, device):
    """Slowest rank's time (all ranks take part when world > 1): the whole job is as
    fast as its slowest replica."""
    if world <= 1:
        return float(ms)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(ms)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_rate(units_per_rank, world, ms):
    """Units processed by all ranks per second (weak scaling: each rank has its own)."""
    return world * units_per_rank / (ms / 1e3)


class ClockSampler:
    """nvidia-smi clocks and throttle reasons sampled every 100 ms while running."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-i", str(self.index), "-lms", "100"], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except (OSError, FileNotFoundError):
            self.proc = None
        return self

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def __exit__(self, *a):
        if self.proc:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()

    def summary(self):
        if not self.lines:
            return {"unavailable": "nvidia-smi gave no samples"}
        sm, mx, pw, reasons = [], 0.0, [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = max(mx, float(f[2]))
                pw.append(float(f[3]))
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return {"unavailable": "unparsable nvidia-smi output"}
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "power_w_median": statistics.median(pw),
                "samples": len(sm), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------- oracle leg
def oracle_sample(views=1, reps=1):
    """The FP64 oracle's render + backward of the first ``views`` keyframes of the
    workload, whole keyframes (projection and binning of all 1M Gaussians included),
    ``reps`` times; returns (seconds per keyframe, threads used).  The GPU arm's
    cpu_baseline and the reference arm time this same sample."""
    from oracle import oracle
    from paper_2509_13536_gb300 import scenegen as sg
    scene, cams = sg.workload(WORKLOAD)
    threads = os.cpu_count() or 1
    oracle.build()
    jobs = []
    for v, cam in enumerate(cams[:views]):
        gr, gd, ga = (x[0] for x in sg.image_cotangents(1, cam.width, cam.height, v))
        jobs.append((cam, gr, gd, ga))
    t0 = time.perf_counter()
    for _ in range(reps):
        for cam, gr, gd, ga in jobs:
            oracle.render(scene, cam, n_threads=threads)
            oracle.render_backward(scene, cam, gr, gd, ga, n_threads=threads)
    dt = time.perf_counter() - t0
    return dt / (reps * len(jobs)), threads


ORACLE_SAMPLE = "FP64 oracle render + backward of keyframe 0, whole 1200x680 frame (projection and binning of all 1M Gaussians included)"


def run_reference(args):
    rank, world, _ = dist_env()
    if rank != 0:
        return
    times = []
    threads = 1
    for i in range(args.warmup + args.steps):
        dt, threads = oracle_sample(1, 1)
        if i >= args.warmup:
            times.append(dt)
    per_step = sum(times) / len(times)
    value = 1.0 / per_step
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": per_step * 1e3,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC},
            "cpu_baseline": {"value": value, "unit": "frames/s", "cores": threads, "kind": "oracle",
                             "sample": ORACLE_SAMPLE + ", one keyframe per step"},
            "e2e": {"value": value, "unit": "frames/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# ----------------------------------------------------------------------------- our leg
def precision_leg(args, api, torch, scene, cams, make_step, dev):
    """The mapping step with FP16 / BF16 attribute storage beside FP32: frames/s, bytes
    per Gaussian, and accuracy against the FP64 oracle fed the FP32 attributes on a
    seeded tile sample of keyframe 0 (PSNR, max-abs on unflagged pixels, gradient
    relative error per parameter group with the cotangent confined to those tiles)."""
    from oracle import oracle
    cam = cams[0]
    tx, ty = (cam.width + 15) // 16, (cam.height + 15) // 16
    rng = np.random.default_rng(7)
    tiles = np.sort(rng.choice(tx * ty, 48, replace=False)).astype(np.int32)
    mask = np.zeros((cam.height, cam.width), bool)
    for t in tiles:
        y, x = divmod(int(t), tx)
        mask[y * 16:y * 16 + 16, x * 16:x * 16 + 16] = True
    crng = np.random.default_rng(8)
    cot = [(crng.uniform(-1, 1, (3, cam.height, cam.width)) * mask).astype(np.float32),
           (crng.uniform(-1, 1, (cam.height, cam.width)) * mask).astype(np.float32),
           (crng.uniform(-1, 1, (cam.height, cam.width)) * mask).astype(np.float32)]
    ref = oracle.render(scene, cam, tiles=tiles)
    ref_g = oracle.render_backward(scene, cam, *cot, tiles=tiles)
    ok = mask & (ref["flags"] == 0)
    out = {}
    f32, f16, bf16 = torch.float32, torch.float16, torch.bfloat16
    # (name, opacity + SH, log-scales, quaternions)
    modes = (("f32", f32, f32, f32), ("f16", f16, f32, f32), ("f16_quat16", f16, f32, f16),
             ("f16_logscale16", f16, f16, f32), ("f16_all", f16, f16, f16),
             ("bf16", bf16, f32, f32), ("bf16_quat16", bf16, f32, bf16), ("bf16_quatf16", bf16, f32, f16),
             ("bf16_all", bf16, bf16, bf16))
    if args.precision_modes:
        modes = tuple(m for m in modes if m[0] in args.precision_modes)
    for name, dt, gdt, qdt in modes:
        g = api.Gaussians.from_scene(scene, dev, dt, gdt, qdt)
        imgs, wsp = api.render(g, [cam])
        dL = [api.Image(*(torch.from_numpy(x).to(dev) for x in cot))]
        grads = api.render_backward(g, [cam], dL, wsp)
        torch.cuda.synchronize()
        rgb = imgs[0].rgb.cpu().numpy().astype(np.float64)
        mse = float(np.mean((rgb - ref["rgb"])[:, mask] ** 2))
        maxabs = float(np.abs(rgb - ref["rgb"])[:, ok].max())
        rel = {}
        keep = ref_g["taint"] == 0
        for k in ("means", "log_scales", "quats", "opacity_logit", "sh"):
            a = getattr(grads, k).cpu().numpy().astype(np.float64)[keep]
            b = ref_g[k][keep]
            rel[k] = float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30))
        del imgs, wsp, grads
        step, st = make_step(g)
        for _ in range(2):
            step()
        st["join"]()
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        k_steps = max(2, args.steps // 2)
        for _ in range(k_steps):
            step()
        st["join"]()
        e1.record()
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k_steps
        out[name] = {"frames_per_s": len(cams) / (ms / 1e3), "ms_per_step": ms,
                     "bytes_per_gaussian": sum(t[0].numel() * t.element_size() for t in g.params()),
                     "psnr_db_vs_fp64_oracle": 10 * np.log10(1.0 / max(mse, 1e-30)),
                     "max_abs_unflagged": maxabs, "grad_rel_err_max": max(rel.values()), "grad_rel_err": rel}
        del g, step, st
        torch.cuda.empty_cache()
    out["sample"] = f"keyframe 0, {len(tiles)} seeded tiles ({int(mask.sum())} px); oracle fed the FP32 attributes"
    out["modes"] = ("f16/bf16: opacity and SH stored reduced, means, log-scales and quaternions f32; "
                    "*_quat16: quaternions reduced too (bf16_quatf16: quaternions f16); *_logscale16: log-scales "
                    "reduced too; *_all: log-scales and quaternions reduced")
    return out


def merge_solver_leg(api, torch, scene, dev):
    """The voxel merge of the 1M-Gaussian map with each Eq. 9 solver: the closed form and
    the paper's L-BFGS (merged pairs, mean iterations per pair, ms per call)."""
    g = api.Gaussians.from_scene(scene, dev)
    ws = torch.empty(api.load().mgs_voxel_merge_workspace_size(g.n), dtype=torch.uint8, device=dev)
    out, partner = g.empty_like(), torch.empty(g.n, dtype=torch.int32, device=dev)
    vox = torch.empty(g.n, 3, dtype=torch.int32, device=dev)
    res = {}
    for solver in ("closed_form", "lbfgs"):
        call = lambda: api.mgs_voxel_merge(g, 0.02, workspace=ws, out=out, partner=partner, vox=vox, solver=solver)
        call()
        torch.cuda.synchronize()
        t = []
        for _ in range(3):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            call()
            e1.record()
            torch.cuda.synchronize()
            t.append(e0.elapsed_time(e1))
        pairs, iters = api.merge_stats()
        res[solver] = {"ms_per_call": float(np.median(t)), "pairs": pairs,
                       "iterations_per_pair": (iters / pairs) if pairs and solver == "lbfgs" else None}
    del g, ws, out
    torch.cuda.empty_cache()
    return res


def patch_grid_leg(api, torch, cams, dev, target_depth):
    """Patch-Grid sampling of each benchmark keyframe: 600 clustered keypoints (8 spots of
    60 plus 120 scattered, a quarter without depth) and the keyframe's rendered depth
    as the depth image; 32 px patches, fewer than 5 keypoints -> 2 x 2 samples."""
    rng = np.random.default_rng(55)
    jobs = []
    for v, cam in enumerate(cams):
        W, H = cam.width, cam.height
        centres = rng.uniform([0, 0], [W, H], (8, 2))
        kp = np.concatenate([c + rng.normal(0, 0.03 * W, (60, 2)) for c in centres] +
                            [rng.uniform([0, 0], [W, H], (120, 2))]).astype(np.float32)
        kd = rng.uniform(0.5, 4.0, len(kp)).astype(np.float32)
        kd[rng.random(len(kp)) < 0.25] = 0
        jobs.append((cam, torch.from_numpy(kp).to(dev), torch.from_numpy(kd).to(dev), target_depth[v]))
    run = lambda: [api.patch_grid_sample(c, k, d, di, 32, 5, 2)[0].shape[0] for c, k, d, di in jobs]
    run()
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    reps = 5
    for _ in range(reps):
        counts = run()
    dt = (time.perf_counter() - t0) / (reps * len(jobs))
    return {"ms_per_keyframe": dt * 1e3, "samples_per_keyframe": float(np.mean(counts)),
            "note": "host-timed, includes the call's two synchronisations"}


def eq12_leg(args, api, torch, scene, make_step, dev, V):
    """The mapping step with the paper's loss (Eq. 12: 0.8 L1 + 0.2 (1 - SSIM) on rgb,
    0.1 x depth L1, isotropic term) instead of the L1 stand-in: frames/s and the loss
    kernels' share."""
    g = api.Gaussians.from_scene(scene, dev)
    step, st = make_step(g, "eq12")
    for _ in range(3):
        step()
    st["join"]()
    torch.cuda.synchronize()
    k_steps = max(3, args.steps // 2)
    api.profile_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record()
    for _ in range(k_steps):
        step()
    st["join"]()
    e1.record()
    torch.cuda.synchronize()
    prof = api.profile_read()
    api.profile_enable(False)
    ms = e0.elapsed_time(e1) / k_steps
    lv = st["loss_views"].sum(0).cpu().tolist()
    res = {"frames_per_s": V / (ms / 1e3), "ms_per_step": ms, "steps": k_steps,
           "loss_kernels_ms_per_step": prof.get("l1_loss", (0.0, 0))[0] / k_steps,
           "last_loss": {"l1": lv[0], "ssim": lv[1], "depth": lv[2], "iso": float(st["loss_iso"].item())},
           "weights": "lambda_ssim 0.2, w_depth 0.1, w_iso 1"}
    del g, step, st
    torch.cuda.empty_cache()
    return res


SERVE_RES = [(320, 240), (640, 480), (1200, 680), (1920, 1080)]


def serving_leg(args, api, torch, sg, dev):
    """Render serving: 4 resident maps (0.5M, 1M, 2M, 3M Gaussians, SH3), Poisson arrivals,
    each request a random map, pose and resolution.  The continuous-batching server (FP16
    maps, requests of any scene and resolution batched into one launch) against the same
    trace served one request at a time from plain FP32 maps.  Latency = arrival -> image
    ready.  The workload's trace (200 req/s) and a sweep of offered rates up to
    saturation, where the completed frames/s show what batching buys."""
    import threading
    sizes = [500_000, 1_000_000, 2_000_000, 3_000_000]
    scenes = [sg.room_scene(n, 40 + i, sh_degree=3) for i, n in enumerate(sizes)]
    ring = {r: [api.new_images([sg.box_camera(*r)], dev)[0] for _ in range(16)] for r in SERVE_RES}

    def trace(rate, n_req, seed):
        rng = np.random.default_rng(seed)
        arrivals = np.cumsum(rng.exponential(1.0 / rate, n_req))
        reqs = []
        for i in range(n_req):
            w, h = SERVE_RES[rng.integers(len(SERVE_RES))]
            reqs.append((int(rng.integers(len(sizes))), sg.room_poses(1, int(rng.integers(1 << 30)), w, h)[0]))
        return arrivals, reqs

    def run(maps, slots, batch, arena_gb, arrivals, reqs):
        n_req = len(reqs)
        warm = min(200, n_req // 10)
        server = api.Server(int(arena_gb * (1 << 30)), n_slots=slots, max_batch_views=batch, device=dev)
        ids = [server.add_scene(g) for g in maps]
        got = {}
        stop = [False]

        def collect():
            while not stop[0] or len(got) < n_req:
                for tag, ts, ta, td, st in server.poll(256, wait_s=0.05):
                    got[tag] = (ts, ta, td, st)
                if stop[0] and len(got) >= n_req:
                    break

        th = threading.Thread(target=collect, daemon=True)
        # no cyclic garbage collection while requests are timed: a full pass over this
        # process's objects stalls the submitting thread for ~0.1 s
        gc.collect()
        gc.disable()
        th.start()
        t0 = server.clock() + 0.2
        late = np.zeros(n_req)
        for i, (sid, cam) in enumerate(reqs):
            target = t0 + float(arrivals[i])
            d = target - server.clock()
            if d > 0:
                time.sleep(d)
            key = (cam.width, cam.height)
            server.submit(ids[sid], cam, ring[key][i % 16], i, target)
            late[i] = server.clock() - target  # the client's own delay in submitting
        stop[0] = True
        th.join(timeout=600)
        gc.enable()
        st = server.stats()
        server.close()
        ok = [i for i in range(warm, n_req) if i in got and got[i][3] == 0]
        lat = np.array([got[i][2] - got[i][0] for i in ok])
        t_first = t0 + float(arrivals[warm])
        t_last = max(got[i][2] for i in ok)
        queue = np.array([got[i][1] - got[i][0] for i in ok])
        service = np.array([got[i][2] - got[i][1] for i in ok])
        pct = lambda a, q: float(np.percentile(a, q) * 1e3) if len(a) else None
        return {"p50_ms": pct(lat, 50), "p99_ms": pct(lat, 99), "max_ms": float(lat.max() * 1e3),
                "p50_queue_ms": pct(queue, 50), "p99_queue_ms": pct(queue, 99),
                "p50_service_ms": pct(service, 50), "p99_service_ms": pct(service, 99),
                "p99_client_late_ms": pct(late[warm:], 99), "max_client_late_ms": float(late[warm:].max() * 1e3),
                "frames_per_s": len(lat) / (t_last - t_first), "completed": int(len(lat)),
                "failed": int(sum(1 for i in range(warm, n_req) if i in got and got[i][3] != 0)),
                "launches": st["launches"], "requests_per_launch": st["requests"] / max(1, st["launches"]),
                "mixed_scene_launches": st["mixed_scene_launches"]}

    res = {"maps": "0.5M/1M/2M/3M Gaussians, SH3", "resolutions": [f"{w}x{h}" for w, h in SERVE_RES],
           "batching": "FP16 maps, 8 slots, up to 8 requests of any scene and resolution per launch",
           "one_at_a_time": "FP32 maps, 1 slot, 1 request per launch"}
    for label, dtype, slots, batch, arena in (("continuous_batching_fp16", torch.float16, 8, 8, 24),
                                              ("one_at_a_time_fp32", torch.float32, 1, 1, 8)):
        maps = [api.Gaussians.from_scene(sc, dev, dtype) for sc in scenes]
        arrivals, reqs = trace(args.serve_rate, args.serve_requests, 4)
        res[label] = run(maps, slots, batch, arena, arrivals, reqs)
        sweep = {}
        for rate in args.serve_sweep:
            arrivals, reqs = trace(rate, args.serve_sweep_requests, 5)
            sweep[f"{rate:g}_req_per_s"] = run(maps, slots, batch, arena, arrivals, reqs)
        res[label + "_sweep"] = sweep
        del maps
        torch.cuda.empty_cache()
    res.update({"requests": args.serve_requests, "rate_per_s": args.serve_rate,
                "sweep_requests": args.serve_sweep_requests})
    return res


def configs_leg(args, api, torch, sg, dev):
    """The two smaller workloads.  box10k: 10k Gaussians, 320x240, SH0, render + backward
    with U[-1, 1] image cotangents.  room300k: 300k Gaussians, 640x480, SH0, render +
    backward + voxel merge (v = 0.02 m).  GPU frames/s over the steps (CUDA events,
    inputs resident), the merge's ms, the FP64 oracle's frames/s on the same whole
    frames on the host cores, and on room300k the merge partners against the oracle's
    (Gaussians the oracle marks as near a tie left out)."""
    from oracle import oracle
    oracle.build()
    threads = os.cpu_count() or 1
    out = {}
    for name in ("box10k", "room300k"):
        scene, cams = sg.workload(name)
        cam = cams[0]
        g = api.Gaussians.from_scene(scene, dev)
        cot = [x[0] for x in sg.image_cotangents(1, cam.width, cam.height, 0)]
        dL = [api.Image(*(torch.from_numpy(c).to(dev) for c in cot))]
        ws = api.RenderWorkspace(dev)
        imgs = api.new_images(cams, dev)
        grads = api.Grads.zeros_like(g)
        merge = name == "room300k"
        if merge:
            mws = torch.empty(api.load().mgs_voxel_merge_workspace_size(g.n), dtype=torch.uint8, device=dev)
            merged, partner = g.empty_like(), torch.empty(g.n, dtype=torch.int32, device=dev)
            vox = torch.empty(g.n, 3, dtype=torch.int32, device=dev)
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)]
        merge_ms = []

        def step(timed=False):
            api.mgs_render(g, cams, imgs, ws)
            api.mgs_render_backward(g, cams, dL, ws, grads)
            if merge:
                if timed:
                    ev[2].record()
                api.mgs_voxel_merge(g, 0.02, workspace=mws, out=merged, partner=partner, vox=vox)
                if timed:
                    ev[3].record()
                    ev[3].synchronize()
                    merge_ms.append(ev[2].elapsed_time(ev[3]))

        for _ in range(3):
            step()
        torch.cuda.synchronize()
        k = max(20, args.steps)
        ev[0].record()
        for _ in range(k):
            step()
        ev[1].record()
        torch.cuda.synchronize()
        ms = ev[0].elapsed_time(ev[1]) / k
        for _ in range(5):
            step(timed=True)
        res = {"frames_per_s": 1e3 / ms, "ms_per_step": ms, "steps": k, "gaussians": g.n,
               "resolution": f"{cam.width}x{cam.height}",
               "step": "render + backward" + (" + voxel_merge v=0.02 m" if merge else "")}
        if merge:
            res["merge_ms"] = float(np.median(merge_ms))
        t0 = time.perf_counter()
        oracle.render(scene, cam, n_threads=threads)
        oracle.render_backward(scene, cam, *cot, n_threads=threads)
        t_orc = time.perf_counter() - t0
        res["oracle"] = {"frames_per_s": 1.0 / t_orc, "cores": threads, "kind": "FP64 oracle, whole frame"}
        if merge:
            t0 = time.perf_counter()
            ref = oracle.voxel_merge(scene, 0.02)
            res["oracle"]["merge_s"] = time.perf_counter() - t0
            got = partner.cpu().numpy()
            clear = ref["tie"] == 0
            res["clusters"] = {"gaussians_compared": int(clear.sum()), "near_tie_left_out": int((~clear).sum()),
                               "partner_mismatches": int((got != ref["partner"])[clear].sum()),
                               "merged_pairs": int((ref["partner"] >= 0).sum() // 2)}
        out[name] = res
        del g, ws, imgs, grads
        torch.cuda.empty_cache()
    return out


def run_ours(args):
    import torch
    import torch.distributed as dist

    from paper_2509_13536_gb300 import api, build, scenegen as sg

    rank, world, local = dist_env()
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    if world > 1:
        dist.init_process_group("nccl", device_id=dev)
    build.build()
    scene, cams = sg.workload(WORKLOAD)
    cams = cams[:args.views]
    V = len(cams)
    H, W = cams[0].height, cams[0].width
    # targets: keyframes rendered from the unperturbed map
    g_true = api.Gaussians.from_scene(scene, dev)
    tgt = api.new_images(cams, dev)
    ws = api.RenderWorkspace(dev)
    api.mgs_render(g_true, cams, tgt, ws)
    target_rgb = torch.stack([t.rgb for t in tgt]).contiguous()
    target_depth = torch.stack([t.depth for t in tgt]).contiguous()
    del g_true, tgt
    # the keyframe images the step reads (the end-to-end run swaps in double buffers)
    tref = {"rgb": target_rgb, "depth": target_depth}
    # the map being optimised: perturbed copy
    rng = np.random.default_rng(replica_seed(rank))
    pert = scene.copy()
    pert.means += rng.normal(0, 0.005, pert.means.shape).astype(np.float32)
    pert.sh += rng.normal(0, 0.02, pert.sh.shape).astype(np.float32)
    def make_step(g, loss_kind="l1", autograd=True):
        """One mapping step on map g (all buffers allocated here, none inside the step).
        loss_kind "l1": Eq. 12 with lambda = 0 (L1 on rgb plus 0.1 x the depth residual),
        the workload's stand-in; "eq12": Eq. 12 with lambda 0.2, the 0.1 depth residual
        and the isotropic term.  autograd: the step runs through api.MappingStep
        (RenderFn forward, loss kernel, torch.autograd.backward into the gradient
        buffers, in-kernel Adam); otherwise the same kernels are called directly through
        the C ABI.  Both end with the voxel merge of the updated map into a buffer."""
        lam, w_iso = (0.2, 1.0) if loss_kind == "eq12" else (0.0, 0.0)
        merged = g.empty_like()
        partner = torch.empty(g.n, dtype=torch.int32, device=dev)
        vox = torch.empty(g.n, 3, dtype=torch.int32, device=dev)
        mws = torch.empty(api.load().mgs_voxel_merge_workspace_size(g.n), dtype=torch.uint8, device=dev)
        mstatus = torch.zeros(2, dtype=torch.int32, pin_memory=True)  # {survivors, flags}, written by the stream
        # The merge of step k runs on its own stream, alongside the start of step k+1 (the
        # projection and the sorts, which leave the GPU room): it starts once step k's Adam
        # update is done, and step k+1's update waits for it (the merge reads the
        # parameters).  join() makes the calling stream wait for the last merge; every
        # timed region ends with it.  (Released after step k+1's render instead, beside the
        # backward pass, it measured slower.)
        mstream = torch.cuda.Stream(dev)
        ev_updated, ev_merged = torch.cuda.Event(), torch.cuda.Event()

        def merge():
            ev_updated.record(torch.cuda.current_stream())
            mstream.wait_event(ev_updated)
            api.mgs_voxel_merge(g, 0.02, workspace=mws, out=merged, partner=partner, vox=vox, status=mstatus,
                                stream=mstream)
            ev_merged.record(mstream)

        state = {"step": 0, "merge_status": mstatus,
                 "join": lambda: torch.cuda.current_stream().wait_event(ev_merged)}
        if autograd:
            ms = api.MappingStep(g, cams, lr=1e-3, lambda_ssim=lam, w_depth=0.1, w_iso=w_iso)
            state.update(ws=ms.ws, loss=ms.loss, loss_views=ms.loss, loss_iso=ms.loss_iso, mapping=ms)

            def step():
                ms(tref["rgb"], tref["depth"], before_update=ev_merged)
                merge()

            return step, state
        grads = api.Grads.zeros_like(g)
        grads.overwrite = True  # the backward stores each step's gradients: no clearing
        m = api.Grads.zeros_like(g, stats=False)
        v = api.Grads.zeros_like(g, stats=False)
        rgb = torch.empty(V, 3, H, W, device=dev)
        depth = torch.empty(V, H, W, device=dev)
        alpha = torch.empty(V, H, W, device=dev)
        out = [api.Image(rgb[i], depth[i], alpha[i]) for i in range(V)]
        g_rgb = torch.empty_like(rgb)
        g_depth = torch.empty_like(depth)
        dL = [api.Image(g_rgb[i], g_depth[i], None) for i in range(V)]
        ws = api.RenderWorkspace(dev)
        lws = torch.empty(api.load().mgs_mapping_loss_workspace_size(V, W, H), dtype=torch.uint8, device=dev)
        iws = torch.empty(api.load().mgs_iso_loss_workspace_size(g.n), dtype=torch.uint8, device=dev)
        loss_v = torch.zeros(V, 3, device=dev)
        loss_iso = torch.zeros(1, device=dev)
        state.update(ws=ws, loss=loss_v, loss_views=loss_v, loss_iso=loss_iso)

        ws.headroom = 1.1

        def step():
            state["step"] += 1
            api.mgs_render(g, cams, out, ws, sync=ws.buf is None)
            targets = [api.Image(tref["rgb"][i], tref["depth"][i], None) for i in range(V)]
            api.mapping_loss(out, targets, dL, lam, 0.1, loss=loss_v, workspace=lws)
            api.mgs_render_backward(g, cams, dL, ws, grads)
            if w_iso > 0:
                api.iso_loss(g, w_iso, grads, loss=loss_iso, workspace=iws)
            torch.cuda.current_stream().wait_event(ev_merged)  # the previous merge has read the map
            api.mgs_adam_step(g, grads, m, v, 1e-3, 0.9, 0.999, 1e-8, state["step"], zero_grads=False)
            merge()

        return step, state

    g = api.Gaussians.from_scene(pert, dev)
    step, state = make_step(g)
    ws, loss = state["ws"], state["loss"]

    def barrier():
        if world > 1:
            dist.barrier()

    stream = torch.cuda.current_stream()
    for _ in range(max(3, args.warmup)):
        step()
    state["join"]()
    torch.cuda.synchronize()
    barrier()
    with ClockSampler(local) as clocks:
        api.profile_enable(True)
        launches0 = api.launch_count()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        torch.cuda.synchronize()
        e0.record(stream)
        for _ in range(args.steps):
            step()
        state["join"]()
        e1.record(stream)
        torch.cuda.synchronize()
        launches = api.launch_count() - launches0
        prof = api.profile_read()
        api.profile_enable(False)
    ws.check()  # no render of the timed steps outgrew its workspace (raises otherwise)
    barrier()
    ms = max_over_ranks(e0.elapsed_time(e1) / args.steps, world, dev)
    value = whole_job_rate(V, world, ms)

    # end to end: keyframe images arrive from pinned host memory, the loss goes back
    if args.no_e2e:
        args.steps_e2e = 0
    host_rgb = target_rgb.cpu().pin_memory()
    host_depth = target_depth.cpu().pin_memory()
    host_loss = torch.empty(2, V, 3, pin_memory=True)
    # double-buffered keyframe images: a copy stream brings step k+1's images from
    # pinned host memory while step k computes; every step's loss goes back to the host
    dev_rgb = [target_rgb, torch.empty_like(target_rgb)]
    dev_depth = [target_depth, torch.empty_like(target_depth)]
    copy_stream = torch.cuda.Stream(dev)
    ready = [torch.cuda.Event(), torch.cuda.Event()]
    used = [torch.cuda.Event(), torch.cuda.Event()]
    n_e2e = getattr(args, "steps_e2e", args.steps)

    def fetch(slot, after=None):
        with torch.cuda.stream(copy_stream):
            if after is not None:
                copy_stream.wait_event(after)
            dev_rgb[slot].copy_(host_rgb, non_blocking=True)
            dev_depth[slot].copy_(host_depth, non_blocking=True)
            ready[slot].record(copy_stream)

    barrier()
    torch.cuda.synchronize()
    e2, e3 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e2.record(stream)
    if n_e2e > 0:
        fetch(0, e2)  # the first copy is inside the timed region too
    for k in range(n_e2e):
        cur, nxt = k % 2, (k + 1) % 2
        if k + 1 < n_e2e:
            fetch(nxt, used[nxt] if k >= 1 else e2)  # buffer nxt is free once step k-1 finished
        stream.wait_event(ready[cur])
        tref["rgb"], tref["depth"] = dev_rgb[cur], dev_depth[cur]
        step()
        used[cur].record(stream)
        host_loss[cur].copy_(loss, non_blocking=True)
    state["join"]()
    e3.record(stream)
    torch.cuda.synchronize()
    tref["rgb"], tref["depth"] = target_rgb, target_depth
    ms_e2e = max_over_ranks(e2.elapsed_time(e3) / max(1, getattr(args, "steps_e2e", args.steps)), world, dev)
    e2e_value = whole_job_rate(V, world, ms_e2e)
    h2d = host_rgb.numel() * 4 + host_depth.numel() * 4

    # roofline of the dominant kernel group, from a counting pass over the saved state
    stats = api.render_stats(g, cams, ws)
    kern = {k: {"ms_per_step": v[0] / args.steps, "launch_groups": v[1]} for k, v in prof.items() if v[1]}
    props = torch.cuda.get_device_properties(dev)
    csum = clocks.summary()
    f_mhz = csum.get("sm_mhz") or 2070.0
    fp32_peak = props.multi_processor_count * 128 * 2 * f_mhz * 1e6 / 1e12  # TFLOP/s (FMA = 2)
    flops = {"blend_fwd": FWD_FLOP_EVAL * stats["evaluated"] + FWD_FLOP_CONTRIB * stats["contributing"],
             "blend_bwd": BWD_FLOP_EVAL * stats["backward_walked"] + BWD_FLOP_CONTRIB * stats["contributing"]}
    peaks = {}
    try:
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json")))
    except OSError:
        pass
    hbm = peaks.get("hbm_gbs", 6800.0)
    hbm_source = ("measured copy bandwidth (MEASURED_PEAKS.json)" if "hbm_gbs" in peaks
                  else "fallback 6.8 TB/s (no MEASURED_PEAKS.json on this machine)")
    pb = sum(t[0].numel() * t.element_size() for t in g.params())  # parameter bytes per Gaussian
    hbm_bytes = algorithmic_bytes(g.n, V, stats, pb, V * W * H)
    for k, e in kern.items():
        dur = e["ms_per_step"] / 1e3
        if k in flops:
            e.update(flops_per_step=flops[k], achieved_tflops=flops[k] / dur / 1e12,
                     frac_of_fp32=flops[k] / dur / 1e12 / fp32_peak)
        elif k in hbm_bytes:
            e.update(bytes_per_step=hbm_bytes[k][0], achieved_gbs=hbm_bytes[k][0] / dur / 1e9,
                     frac_of_hbm=hbm_bytes[k][0] / dur / 1e9 / hbm, hbm_peak_gbs=hbm, hbm_peak_source=hbm_source,
                     bytes_basis=hbm_bytes[k][1])

    def alu_roofline(name):
        e = kern[name]
        return {"kernel": name, "bound": "alu", "achieved": e["achieved_tflops"], "peak": fp32_peak,
                "unit": "TFLOP/s", "frac": e["frac_of_fp32"], "traffic": recorded_traffic(name),
                "peak_basis": f"{props.multi_processor_count} SMs x 128 FP32 lanes x 2 flop x {f_mhz:.0f} MHz "
                              "(median sampled SM clock)",
                "flops_per_launch": flops[name]}

    dom = max(kern, key=lambda k: kern[k]["ms_per_step"])
    if dom in flops:
        roofline = alu_roofline(dom)
    else:
        e = kern[dom]
        roofline = {"kernel": dom, "bound": "hbm", "achieved": e.get("achieved_gbs"), "peak": hbm, "unit": "GB/s",
                    "frac": e.get("frac_of_hbm"), "traffic": None, "peak_basis": hbm_source}
    roofline_fwd = alu_roofline("blend_fwd") if "blend_fwd" in kern and dom != "blend_fwd" else None

    # the same step with the kernels called directly through the C ABI (no autograd)
    direct = None
    if world == 1:
        gd_ = api.Gaussians.from_scene(pert, dev)
        step_d, st_d = make_step(gd_, autograd=False)
        for _ in range(3):
            step_d()
        st_d["join"]()
        torch.cuda.synchronize()
        d0, d1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        d0.record(stream)
        for _ in range(args.steps):
            step_d()
        st_d["join"]()
        d1.record(stream)
        torch.cuda.synchronize()
        ms_d = d0.elapsed_time(d1) / args.steps
        direct = {"ms_per_step_direct_cabi": ms_d, "ms_per_step_autograd": ms, "autograd_overhead_ms": ms - ms_d,
                  "note": "same kernels and loss; the autograd step adds RenderFn, graph construction and "
                          "torch.autograd.backward on the host"}
        del gd_, step_d
        torch.cuda.empty_cache()
    configs = None
    if world == 1 and not args.no_configs:
        configs = configs_leg(args, api, torch, sg, dev)
    eq12 = None
    if world == 1 and not args.no_eq12:
        eq12 = eq12_leg(args, api, torch, pert, make_step, dev, V)
        eq12["merge_solvers"] = merge_solver_leg(api, torch, pert, dev)
        eq12["patch_grid"] = patch_grid_leg(api, torch, cams, dev, target_depth)
    precision = None
    if world == 1 and not args.no_precision:
        precision = precision_leg(args, api, torch, pert, cams, make_step, dev)
    serving = None
    if world == 1 and not args.no_serving:
        serving = serving_leg(args, api, torch, sg, dev)

    line = {"metric": METRIC, "value": value, "unit": "frames/s", "n_gpus": world, "steps": args.steps,
            "warmup": max(3, args.warmup), "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "desc": WORKLOAD_DESC, "n_gaussians": g.n, "views": V,
                       "resolution": f"{W}x{H}", "parallelism": f"replicas x{world}",
                       "l2": "inputs larger than L2 (236 MB parameters, 384 MB projected records, "
                             f"{stats['keys']} tile keys per step)"},
            "roofline": roofline,
            "roofline_blend_fwd": roofline_fwd,
            "e2e": ({"value": e2e_value, "unit": "frames/s", "h2d_bytes_per_step": h2d,
                     "d2h_bytes_per_step": host_loss[0].numel() * 4} if n_e2e > 0 else None),
            "gpu_launches": launches, "clocks": csum, "kernels": kern, "fragments": stats,
            "merge_survivors": int(state["merge_status"][0]),
            "host_syncs_per_step": "none inside the step (asynchronous render and merge; e2e reads the loss back)"}
    if direct:
        line["autograd"] = direct
    if configs:
        line["configs"] = configs
    if eq12:
        line["eq12_step"] = eq12
    if precision:
        line["precision"] = precision
    if serving:
        line["serving"] = serving
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        dt, threads = oracle_sample(1, args.cpu_reps)
        line["cpu_baseline"] = {"value": 1.0 / dt, "unit": "frames/s", "cores": threads, "kind": "oracle",
                                "sample": ORACLE_SAMPLE + f", {args.cpu_reps} times ({dt:.1f} s each)"}
    if rank == 0:
        print(json.dumps(line), flush=True)
    if world > 1:
        dist.destroy_process_group()


def main():
    args = parse()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
