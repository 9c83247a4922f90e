"""The two-stream post-rendering pipeline (api.FramePipeline): the low-resolution render of
the next frame overlaps the x S interpolation (Sec. 4.1) and the two warps (Sec. 4.2) of
the current one.

Overlapping must change nothing:
- every output of every step on two streams equals the same step on one stream, bit for bit;
- the last frame's outputs equal direct calls on a plain forward render of that frame.
"""
import numpy as np
import pytest

from paper_2605_11489_gb300 import synth

pytestmark = pytest.mark.gpu


def _orbit(n, W=128, H=72, radius=4.0):
    cams = []
    for k in range(n):
        a = 0.05 * k
        eye = (radius * np.sin(a), 0.4, radius * np.cos(a))
        cams.append(synth.make_camera(eye, (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), W, H))
    return cams


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g

    g.build()
    from paper_2605_11489_gb300 import api

    torch.cuda.set_device(0)
    return api


def _run(api, ctx, scene, cams, weights, overlap, slots=2):
    import torch

    dense = cams
    frames, mids = dense[0::2], dense[1::2]
    pipe = api.FramePipeline(ctx, scene, frames[0], weights, capacity=200000, tile=16, overlap=overlap, slots=slots)
    got = []
    for t, cam in enumerate(frames):
        mid = mids[t - 1] if t > 0 else cam
        k = pipe.step(cam, mid)
        with torch.cuda.stream(pipe.ps):
            got.append({"hr_rgb": pipe.hr_rgb[k].clone(), "hr_da": pipe.hr_da[k].clone(),
                        "bwd": {n: v.clone() for n, v in pipe.bwd.items()},
                        "fwd": {n: v.clone() for n, v in pipe.fwd.items()} if t > 0 else None})
    pipe.synchronize()
    out = [{n: (v.cpu().numpy() if not isinstance(v, dict) else {m: w.cpu().numpy() for m, w in v.items()})
            for n, v in g.items() if v is not None} for g in got]
    pipe.close()
    return out, frames, mids


def _same(a, b):
    return np.array_equal(a, b, equal_nan=True)


@pytest.mark.parametrize("slots", [2, 4])
def test_overlapped_equals_serial_and_direct_calls(env, slots):
    import torch

    api = env
    ctx = api.Context(0)
    scene = api.Scene.from_arrays(synth.tiny_scene(4096, 0))
    weights = synth.gai_weights(4, 32)
    cams = _orbit(13)
    over, frames, mids = _run(api, ctx, scene, cams, weights, True, slots)
    serial, _, _ = _run(api, ctx, scene, cams, weights, False)
    assert len(over) == len(serial) == 7
    for t, (a, b) in enumerate(zip(over, serial)):
        for n in a:
            if isinstance(a[n], dict):
                for m in a[n]:
                    assert _same(a[n][m], b[n][m]), (t, n, m)
            else:
                assert _same(a[n], b[n]), (t, n)
    # the last frame against direct calls on a plain forward render
    t = len(frames) - 1
    lr = ctx.forward(scene, frames[t], tile=16)
    prev = ctx.forward(scene, frames[t - 1], tile=16)
    hr = api.gai_upsample(weights, lr["rgb"], lr["dcdx"], lr["dcdy"])
    da = torch.stack([lr["depth"], lr["alpha"]]).contiguous()
    z = torch.zeros_like(da)
    hr_da = api.gai_upsample(weights, da, z, z)
    bwd = ctx.warp(frames[t], mids[t - 1], lr["depth"], lr["alpha"], 0.0, lr["rgb"], lr["dcdx"], lr["dcdy"])
    pda = torch.stack([prev["depth"], prev["alpha"]]).contiguous()
    phr = api.gai_upsample(weights, prev["rgb"], prev["dcdx"], prev["dcdy"])
    phr_da = api.gai_upsample(weights, pda, torch.zeros_like(pda), torch.zeros_like(pda))
    fwd = ctx.warp(frames[t - 1].scaled(4), mids[t - 1].scaled(4), phr_da[0].contiguous(), phr_da[1].contiguous(),
                   api.FramePipeline.HR_ALPHA_MIN, phr, keys=("motion", "index", "z", "planes"))
    torch.cuda.synchronize()
    assert _same(over[t]["hr_rgb"], hr.cpu().numpy())
    assert _same(over[t]["hr_da"], hr_da.cpu().numpy())
    for m in bwd:
        assert _same(over[t]["bwd"][m], bwd[m].cpu().numpy()), m
    for m in fwd:
        assert _same(over[t]["fwd"][m], fwd[m].cpu().numpy()), m
    assert (over[t]["fwd"]["index"] >= 0).mean() > 0.05  # the 4x frame really lands somewhere
    ctx.close()
