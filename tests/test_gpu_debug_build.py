"""The GSR_DEBUG build on the GPU: every render path the tests exercise, run through
libgsr_debug.so (whose device index guards raise kErrBounds, reported as GS_ERR_INTERNAL),
fires no guard. Runs in a subprocess, because a process loads one of the two libraries."""
import os
import subprocess
import sys

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

SCRIPT = r"""
import numpy as np, torch
from paper_2605_11489_gb300 import build as b
b.build(debug=True)
from paper_2605_11489_gb300 import abi, api, synth
assert abi.LIB_PATH.endswith("libgsr_debug.so")
torch.cuda.set_device(0)
ctx = api.Context(0)

def dense(n, seed):
    rng = np.random.default_rng(seed)
    s = synth.empty_scene(n, 1)
    s.means[:, :n] = rng.normal(0, 0.25, (3, n))
    s.log_scales[:, :n] = rng.normal(-2.6, 0.4, (3, n))
    s.quats[:, :n] = rng.normal(size=(4, n))
    s.logits[:n] = rng.normal(3.0, 1.0, n)
    s.sh[:, :, :n] = rng.normal(0, 0.4, (4, 3, n))
    return s

tiny = api.Scene.from_arrays(synth.tiny_scene(4096, 0))
clus = api.Scene.from_arrays(synth.clustered_scene(200_000, 5, (2.0, 2.0, 2.0), 8, 3))
dsc = api.Scene.from_arrays(dense(3000, 21))
cam = synth.tiny_camera(203, 117)
for scene in (tiny, clus, dsc):
    for tile in (8, 16, 32):
        for chunk in (16, 512, 1 << 24):  # long tiles (one CTA per tile), and none
            out, st = ctx.forward(scene, cam, tile=tile, chunk=chunk, state=True)
            g = {k: torch.ones_like(out[k]) for k in ("rgb", "dcdx", "dcdy")}
            ctx.backward(st, scene, g)
            st.free()
            torch.cuda.synchronize()
            assert ctx.check() == abi.GS_OK, (tile, chunk)
    ctx.forward(scene, cam, keys=api.OUTPUT_KEYS + api.NORMAL_KEYS)
    assert ctx.check() == abi.GS_OK
cams = synth.jittered_tiny_cameras(6, 3)
ctx.stats(reset=True)
for c in cams:
    ctx.forward(clus, c, tile=8, batch=128, chunk=64)
cap = int(ctx.stats(reset=True)["instances_max"] * 1.25) + 4096
fs = api.FrameStream(ctx, clus, cams[0], cap, 8, 128, 64, slots=3)
for c in cams:
    fs.render(c)
fs.synchronize()
fs.close()
srv = api.Server(sort_budget_bytes=256 << 20, max_inflight=4)
sid = srv.load_scene(clus)
rids = [srv.submit(sid, cams[i % 6], api.alloc_outputs(256, 144)) for i in range(8)]
srv.drain()
assert all(srv.poll(r)[0] == abi.GS_OK for r in rids)
srv.close()
print("DEBUG-BUILD-OK")
"""


def test_debug_build_fires_no_index_guard():
    env = dict(os.environ, GSR_DEBUG="1")
    r = subprocess.run([sys.executable, "-c", SCRIPT], cwd=ROOT, env=env, capture_output=True, text=True,
                       timeout=900)
    assert r.returncode == 0 and "DEBUG-BUILD-OK" in r.stdout, (r.stdout[-2000:], r.stderr[-4000:])
