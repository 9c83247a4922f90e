"""Continuous-batching server through the C ABI: every request's output is
the same alone and in a mixed stream, admission respects the sort-buffer
budget, cancellation and not-ready polls work, and a host-injected failure
ends only its own request. No test faults or hangs the GPU: failures are
injected on the host (GSR_FAULT) and every wait has a deadline."""
import os
import time

import numpy as np
import pytest

from paper_2605_11489_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g

    g.build()
    from paper_2605_11489_gb300 import api

    torch.cuda.set_device(0)
    return api, api.Context(0)


def _wait(srv, rid, deadline_s=60.0):
    from paper_2605_11489_gb300 import abi

    t0 = time.time()
    while True:
        st, lat = srv.poll(rid)
        if st != abi.GS_NOT_READY:
            return st, lat
        assert time.time() - t0 < deadline_s, "request %d not done after %.0f s" % (rid, deadline_s)
        time.sleep(0.001)


def _mixed_requests(n, seed):
    rng = np.random.default_rng(seed)
    res = [(64, 48), (256, 144), (203, 117), (480, 270)]
    cams = []
    for _ in range(n):
        w, h = res[rng.integers(len(res))]
        eye = np.array([0.0, 0.0, 4.0]) + rng.normal(0, 0.5, 3)
        cams.append((int(rng.integers(2)), synth.make_camera(eye, (0, 0, 0), (0, 1, 0), w, h)))
    return cams


def test_requests_same_alone_and_in_the_mix(env):
    api, ctx = env
    import torch

    import oracle
    from gpu_util import GRAD_FRAC, GRAD_FRAC_STRESS, check_render

    arrays = [synth.tiny_scene(4096, 0), synth.clustered_scene(20_000, 5, (2.0, 2.0, 2.0), 8, 3)]
    scenes = [api.Scene.from_arrays(a) for a in arrays]
    srv = api.Server(sort_budget_bytes=256 << 20, max_inflight=6)
    ids = [srv.load_scene(s) for s in scenes]
    reqs = _mixed_requests(40, 1)
    bg = (0.1, 0.2, 0.3)
    outs, rids = [], []
    for sid, cam in reqs:
        o = api.alloc_outputs(cam.width, cam.height)
        outs.append(o)
        rids.append(srv.submit(ids[sid], cam, o, bg=bg))
    lats = []
    for rid in rids:
        st, lat = _wait(srv, rid)
        assert st == 0
        lats.append(lat)
    assert min(lats) > 0
    # The server composites at tile 8 with long lists (over 4 x 512 records) split into
    # chunks and merged exactly, as the plain forward does at chunk 512: bit for bit the
    # same. Other chunkings reassociate fp32 sums: equal up to rounding (well inside the
    # oracle tolerances).
    for (sid, cam), o in zip(reqs, outs):
        same = ctx.forward(scenes[sid], cam, tile=8, bg=bg, chunk=512)
        whole = ctx.forward(scenes[sid], cam, tile=8, bg=bg, chunk=1 << 24)
        for k in same:
            assert torch.equal(o[k], same[k]), k
            assert (o[k] - whole[k]).abs().max().item() < 2e-5, k
    # and served requests of every resolution against the FP64 oracle, every pixel
    seen = set()
    for (sid, cam), o in zip(reqs, outs):
        if (sid, cam.width) in seen:
            continue
        seen.add((sid, cam.width))
        # scene 1 is a close-range stress scene (see gpu_util)
        check_render(o, oracle.render(arrays[sid], cam, bg=bg), grad_frac=GRAD_FRAC_STRESS if sid else GRAD_FRAC)
    assert len(seen) >= 6
    srv.close()


def test_poll_before_ready_and_drain(env):
    api, ctx = env
    from paper_2605_11489_gb300 import abi

    scene = api.Scene.from_arrays(synth.clustered_scene(200_000, 6, (2.0, 2.0, 2.0), 8, 3))
    srv = api.Server(sort_budget_bytes=4 << 30, max_inflight=4)  # ~0.2 GB of sort memory per request at tile 8
    sid = srv.load_scene(scene)
    cam = synth.make_camera((0.5, 0.3, 4.0), (1, 1, 1), (0, 1, 0), 480, 270)
    rids = [srv.submit(sid, cam, api.alloc_outputs(480, 270)) for _ in range(16)]
    st0, _ = srv.poll(rids[-1])
    assert st0 == abi.GS_NOT_READY
    srv.drain()
    for rid in rids:
        st, lat = srv.poll(rid)
        assert st == 0 and lat > 0
    with pytest.raises(Exception):
        abi.check(abi.lib().gs_server_poll(srv.h, 10_000_000, None))
    srv.close()


def test_cancel_queued_request(env):
    api, ctx = env
    from paper_2605_11489_gb300 import abi

    scene = api.Scene.from_arrays(synth.clustered_scene(200_000, 7, (2.0, 2.0, 2.0), 8, 3))
    srv = api.Server(sort_budget_bytes=4 << 30, max_inflight=1)
    sid = srv.load_scene(scene)
    cam = synth.make_camera((0.0, 0.0, 4.0), (1, 1, 1), (0, 1, 0), 480, 270)
    rids = [srv.submit(sid, cam, api.alloc_outputs(480, 270)) for _ in range(12)]
    srv.cancel(rids[-1])
    st, _ = _wait(srv, rids[-1])
    assert st in (abi.GS_ERR_CANCELLED, 0)
    srv.drain()
    srv.close()


def test_admission_waits_for_budget_and_rejects_oversized(env):
    api, ctx = env
    import torch

    from paper_2605_11489_gb300 import abi

    scene = api.Scene.from_arrays(synth.tiny_scene(4096, 8))
    cam = synth.tiny_camera()
    # about 6,700 instances * ~18 B plus alignment: one request's sort memory is ~0.15 MB
    srv = api.Server(sort_budget_bytes=1 << 20, max_inflight=8)
    sid = srv.load_scene(scene)
    outs = [api.alloc_outputs(cam.width, cam.height) for _ in range(10)]
    rids = [srv.submit(sid, cam, o) for o in outs]
    for rid in rids:
        assert _wait(srv, rid)[0] == 0
    ref = ctx.forward(scene, cam, tile=8, chunk=512)  # the server's tile and chunking
    for o in outs:
        assert torch.equal(o["rgb"], ref["rgb"])
    srv.close()
    tiny = api.Server(sort_budget_bytes=4096, max_inflight=2)
    sid = tiny.load_scene(scene)
    rid = tiny.submit(sid, cam, api.alloc_outputs(cam.width, cam.height))
    assert _wait(tiny, rid)[0] == abi.GS_ERR_OOM
    tiny.close()


@pytest.mark.parametrize("fault", ["alloc:1", "enqueue:2"])
def test_injected_host_failure_ends_only_its_request(env, fault):
    api, ctx = env
    scene = api.Scene.from_arrays(synth.tiny_scene(4096, 9))
    cam = synth.tiny_camera()
    old = os.environ.get("GSR_FAULT")
    os.environ["GSR_FAULT"] = fault
    try:
        srv = api.Server(sort_budget_bytes=64 << 20, max_inflight=1)
    finally:
        if old is None:
            del os.environ["GSR_FAULT"]
        else:
            os.environ["GSR_FAULT"] = old
    sid = srv.load_scene(scene)
    rids = [srv.submit(sid, cam, api.alloc_outputs(cam.width, cam.height)) for _ in range(5)]
    sts = [_wait(srv, r)[0] for r in rids]
    assert sum(1 for s in sts if s != 0) == 1, sts
    assert sts[int(fault.split(":")[1])] != 0
    srv.close()


def test_scheduler_thread_failure_fails_pending_requests_and_later_submits(env):
    """GSR_FAULT=thread:2: the scheduler thread throws before its third admission. With one
    in-flight slot, requests 0 and 1 complete first (and equal the plain forward); every
    other request finishes with GS_ERR_INTERNAL once the thread has waited for its GPU
    work; later submits and drain report GS_ERR_INTERNAL; destroy still returns."""
    api, ctx = env
    import torch

    from paper_2605_11489_gb300 import abi

    scene = api.Scene.from_arrays(synth.tiny_scene(4096, 10))
    cam = synth.tiny_camera()
    old = os.environ.get("GSR_FAULT")
    os.environ["GSR_FAULT"] = "thread:2"
    try:
        srv = api.Server(sort_budget_bytes=64 << 20, max_inflight=1)
    finally:
        if old is None:
            del os.environ["GSR_FAULT"]
        else:
            os.environ["GSR_FAULT"] = old
    try:
        sid = srv.load_scene(scene)
        outs = [api.alloc_outputs(cam.width, cam.height) for _ in range(6)]
        rids = [srv.submit(sid, cam, o) for o in outs]
        sts = [_wait(srv, r)[0] for r in rids]
        assert sts == [abi.GS_OK, abi.GS_OK] + [abi.GS_ERR_INTERNAL] * 4, sts
        ref = ctx.forward(scene, cam, tile=8, chunk=512)
        torch.cuda.synchronize()
        for o in outs[:2]:
            for k in ref:
                assert torch.equal(o[k], ref[k]), k
        with pytest.raises(abi.GsError) as e:
            srv.submit(sid, cam, outs[0])
        assert e.value.status == abi.GS_ERR_INTERNAL
        with pytest.raises(abi.GsError) as e:
            srv.drain()
        assert e.value.status == abi.GS_ERR_INTERNAL
    finally:
        srv.close()
