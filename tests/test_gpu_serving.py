"""Render serving with continuous batching: every request's image is bit-identical to
rendering it alone, whether it was batched with requests of other scenes and
resolutions into one launch, overlapped with other batches, or delayed by a small
arena (admission by free memory)."""
import numpy as np
import pytest
import torch

from paper_2509_13536_gb300 import api, scenegen as sg

pytestmark = pytest.mark.gpu

RES = [(320, 240), (640, 480), (1200, 680)]


@pytest.fixture(scope="module", autouse=True)
def _built():
    from paper_2509_13536_gb300 import build
    build.build()


@pytest.fixture(scope="module")
def scenes():
    out = []
    for k, (n, dt) in enumerate([(40_000, torch.float16), (90_000, torch.float32), (60_000, torch.bfloat16)]):
        out.append(api.Gaussians.from_scene(sg.room_scene(n, 40 + k, sh_degree=3), "cuda", dt))
    return out


def _requests(n, seed):
    rng = np.random.default_rng(seed)
    reqs = []
    for i in range(n):
        w, h = RES[rng.integers(len(RES))]
        cam = sg.room_poses(1, int(rng.integers(1 << 30)), w, h)[0]
        reqs.append((int(rng.integers(3)), cam))
    return reqs


def _run(server, scenes, reqs, burst=True):
    outs = {}
    t0 = server.clock()
    for tag, (sid, cam) in enumerate(reqs):
        out = api.new_images([cam])[0]
        outs[tag] = out
        server.submit(sid, cam, out, tag, t0 if burst else 0.0)
    done = {}
    while len(done) < len(reqs):
        for tag, ts, ta, td, st in server.poll(64, wait_s=1.0):
            assert st == 0, st
            done[tag] = (ts, ta, td)
    return outs, done


def test_multi_map_render_matches_each_view_alone(scenes):
    """Views of three maps (f16, f32 and bf16 storage), interleaved and at mixed
    resolutions, in one mgs_render_multi call: every image is bit-identical to the same
    view rendered alone from its own map."""
    rng = np.random.default_rng(77)
    mov = [0, 2, 2, 1, 0, 1, 2]
    cams = [sg.room_poses(1, int(rng.integers(1 << 30)), *RES[k % 3])[0] for k in range(len(mov))]
    out = [api.new_images([c])[0] for c in cams]
    ws = api.RenderWorkspace("cuda")
    ws.ensure(10, cams[:1], 10)  # far too small: the binding grows it and retries
    api.mgs_render_multi(scenes, mov, cams, out, ws)
    torch.cuda.synchronize()
    for v, (m, cam) in enumerate(zip(mov, cams)):
        alone, _ = api.render(scenes[m], [cam])
        torch.cuda.synchronize()
        for plane in ("rgb", "depth", "alpha"):
            assert torch.equal(getattr(out[v], plane), getattr(alone[0], plane)), (v, plane)


@pytest.mark.parametrize("arena_mb,slots,batch", [(6000, 6, 8), (700, 2, 4)])
def test_each_request_matches_rendering_it_alone(scenes, arena_mb, slots, batch):
    reqs = _requests(40, arena_mb)
    server = api.Server(arena_mb << 20, n_slots=slots, max_batch_views=batch)
    sids = [server.add_scene(g) for g in scenes]
    assert sids == [0, 1, 2]
    outs, done = _run(server, scenes, reqs)
    st = server.stats()
    server.close()
    assert st["requests"] == len(reqs)
    if batch > 1:
        assert st["mixed_scene_launches"] > 0, st  # a burst of 40 requests over 3 scenes mixes them
    for tag, (sid, cam) in enumerate(reqs):
        alone, _ = api.render(scenes[sid], [cam])
        torch.cuda.synchronize()
        assert torch.equal(outs[tag].rgb, alone[0].rgb), tag
        assert torch.equal(outs[tag].depth, alone[0].depth), tag
        assert torch.equal(outs[tag].alpha, alone[0].alpha), tag
    lat = [d[2] - d[0] for d in done.values()]
    assert min(lat) > 0


def test_request_too_big_for_the_arena_fails_cleanly(scenes):
    server = api.Server(2 << 20, n_slots=1, max_batch_views=1)
    server.add_scene(scenes[1])
    cam = sg.room_poses(1, 5, 1200, 680)[0]
    out = api.new_images([cam])[0]
    server.submit(0, cam, out, 7)
    res = server.poll(4, wait_s=10.0)
    server.close()
    assert len(res) == 1 and res[0][0] == 7 and res[0][4] == 2  # MGS_ERR_WORKSPACE
