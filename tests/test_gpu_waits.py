"""Bounded device waits and device errors, through the C ABI, without a stuck GPU.

Every wait in the kernels (the radix sort's and the duplication's decoupled
lookbacks, the compositing warps' staged-batch waits) gives up after a bounded
number of polls and raises an error bit instead of spinning. A diagnostic setting (gs_context_debug_waits,
or GSR_FAULT=wait:<k> in the server) makes them give up at once, so that the
failure path runs deterministically on a healthy GPU: the frame must report
GS_ERR_TIMEOUT, nothing may be read or written out of bounds, and the context
(or the server's other requests) must go on rendering correctly.
"""
import os
import time

import numpy as np
import pytest

from paper_2605_11489_gb300 import synth

from gpu_util import GRAD_FRAC_STRESS, check_render

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g

    g.build()
    import oracle
    from paper_2605_11489_gb300 import abi, api

    torch.cuda.set_device(0)
    return abi, api, oracle


def _scene():
    # > 4,096 visible Gaussians, so that the sorts have several partitions that look back
    return synth.clustered_scene(40_000, 21, (2.0, 2.0, 2.0), 8, 0)


def _camera():
    return synth.make_camera((0.6, -0.4, 4.2), (1.0, 1.0, 1.0), (0, 1, 0), 320, 180)


def test_forward_wait_gives_up_reports_timeout_and_context_recovers(env):
    abi, api, O = env
    import torch

    sc, cam = _scene(), _camera()
    scene = api.Scene.from_arrays(sc)
    ref_ctx = api.Context(0)
    ref = ref_ctx.forward(scene, cam)
    ctx = api.Context(0)
    try:
        ctx.debug_waits(True)
        ctx.forward(scene, cam)  # returns before the sort and compositing run
        assert ctx.check() == abi.GS_ERR_TIMEOUT
        assert ctx.check() == abi.GS_OK  # reported once, then cleared
        # a frame whose waits gave up is reported by the next forward, which renders nothing
        ctx.forward(scene, cam)
        ctx.debug_waits(False)
        with pytest.raises(abi.GsError) as ei:
            ctx.forward(scene, cam)
        assert ei.value.status == abi.GS_ERR_TIMEOUT
        # the context renders correctly again
        out = ctx.forward(scene, cam)
        assert ctx.check() == abi.GS_OK
        for k in out:
            assert torch.equal(out[k], ref[k]), k
        check_render(out, O.render(sc, cam), grad_frac=GRAD_FRAC_STRESS)  # a close-range stress scene
    finally:
        torch.cuda.synchronize()
        ctx.close()
        ref_ctx.close()


def test_compositing_batch_wait_gives_up_and_context_recovers(env):
    """Level 2 of the diagnostic makes only compositing's batch waits give up, so the
    sorts finish and the plan is made. Frames with the normal channels stage their batches
    by TMA bulk copies into each warp's mbarrier ring: every warp's first wait gives up,
    waits (bounded) for the copies it has in flight, and the frame reports
    GS_ERR_TIMEOUT. The same frame then renders exactly as on a fresh context."""
    abi, api, O = env
    import torch

    sc, cam = _scene(), _camera()
    scene = api.Scene.from_arrays(sc)
    keys = api.OUTPUT_KEYS + api.NORMAL_KEYS
    ref_ctx = api.Context(0)
    ref = ref_ctx.forward(scene, cam, keys=keys)
    ctx = api.Context(0)
    try:
        with pytest.raises(abi.GsError) as ei:
            ctx.debug_waits(3)
        assert ei.value.status == abi.GS_ERR_INVALID_ARG
        ctx.debug_waits(2)
        ctx.forward(scene, cam, keys=keys)
        assert ctx.check() == abi.GS_ERR_TIMEOUT
        ctx.debug_waits(0)
        out = ctx.forward(scene, cam, keys=keys)
        assert ctx.check() == abi.GS_OK
        for k in out:
            assert torch.equal(out[k], ref[k]), k
    finally:
        torch.cuda.synchronize()
        ctx.close()
        ref_ctx.close()


def test_backward_after_a_frame_that_gave_up_stays_in_bounds(env):
    """A state kept from a frame whose sort gave up holds an unsorted instance list;
    the backward must skip indices it does not own rather than read or write past
    its buffers (the gradients are then meaningless, and the frame was reported)."""
    abi, api, O = env
    import torch

    sc, cam = _scene(), _camera()
    scene = api.Scene.from_arrays(sc)
    ctx = api.Context(0)
    try:
        ctx.debug_waits(True)
        out, st = ctx.forward(scene, cam, state=True)
        g = {k: torch.ones_like(out[k]) for k in ("rgb", "dcdx", "dcdy")}
        ctx.backward(st, scene, g)
        torch.cuda.synchronize()
        st.free()
        assert ctx.check() == abi.GS_ERR_TIMEOUT
        ctx.debug_waits(False)
        out2, st2 = ctx.forward(scene, cam, state=True)
        grads2 = ctx.backward(st2, scene, g)
        torch.cuda.synchronize()
        st2.free()
        assert ctx.check() == abi.GS_OK
        assert all(torch.isfinite(t).all().item() for t in grads2)
    finally:
        torch.cuda.synchronize()
        ctx.close()


def _wait(srv, rid, deadline_s=60.0):
    from paper_2605_11489_gb300 import abi

    t0 = time.time()
    while True:
        st, lat = srv.poll(rid)
        if st != abi.GS_NOT_READY:
            return st
        assert time.time() - t0 < deadline_s
        time.sleep(0.001)


def test_server_request_whose_waits_give_up_fails_alone(env):
    abi, api, O = env
    import torch

    sc, cam = _scene(), _camera()
    scene = api.Scene.from_arrays(sc)
    ref = api.Context(0).forward(scene, cam, tile=8, chunk=512)  # the server's tile and chunking
    old = os.environ.get("GSR_FAULT")
    os.environ["GSR_FAULT"] = "wait:2"
    try:
        srv = api.Server(sort_budget_bytes=256 << 20, max_inflight=1)
    finally:
        if old is None:
            del os.environ["GSR_FAULT"]
        else:
            os.environ["GSR_FAULT"] = old
    try:
        sid = srv.load_scene(scene)
        outs = [api.alloc_outputs(cam.width, cam.height) for _ in range(5)]
        rids = [srv.submit(sid, cam, o) for o in outs]
        sts = [_wait(srv, r) for r in rids]
        assert sts[2] == abi.GS_ERR_TIMEOUT, sts
        assert all(s == abi.GS_OK for i, s in enumerate(sts) if i != 2), sts
        for i, o in enumerate(outs):
            if i != 2:
                for k in o:
                    assert torch.equal(o[k], ref[k]), (i, k)
    finally:
        srv.drain()
        srv.close()


def test_server_destroy_returns_its_device_memory(env):
    abi, api, O = env
    import torch

    sc = synth.clustered_scene(300_000, 22, (2.0, 2.0, 2.0), 8, 3)
    scene = api.Scene.from_arrays(sc)
    cam = _camera()
    outs = [api.alloc_outputs(cam.width, cam.height) for _ in range(8)]
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    srv = api.Server(sort_budget_bytes=1 << 30, max_inflight=4)
    try:
        sid = srv.load_scene(scene)
        rids = [srv.submit(sid, cam, o) for o in outs]
        sts = [_wait(srv, r) for r in rids]
        assert all(s == abi.GS_OK for s in sts), sts
        during = torch.cuda.mem_get_info()[0]
    finally:
        srv.drain()
        srv.close()
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    # the sort budget (1 GiB) and the slots' per-Gaussian buffers; all of it must come back
    assert free0 - during > 1 << 30
    assert abs(free1 - free0) < 8 << 20, (free0, free1)
