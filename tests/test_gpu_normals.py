"""GPU parity of the RaDe-GS channels against the oracle, through the C ABI
(gs_render_forward with gs_outputs.normal / .nv / .depth_isect).

- The normal and the ray-Gaussian intersection depth are the ones RaDe-GS renders (the
  paper's depth and normal maps, Sec. 5.1).
- The normal-view map Nv is the one the super-sampling takes (Sec. 4.1).
- The intersection depth is held to the depth channel's bar (gpu_util.check_depth): 2e-4
  relative to max(1, |depth|) on >= 99.99 % of the pixels, 5e-3 of the alpha-cut flip
  scale on all.

Bar: the colour's.
- The normal is the same alpha-weighted sum with unit vectors in place of colours, so its
  error per pixel is the colour's: 2e-4 on >= 99.99 % of values, 5e-3 on all.
- That holds on pixels where no blended Gaussian's orientation is open (oracle nrm_amb) and
  no discrete decision sits at its threshold (oracle amb).
- Rendering the normal channel changes no other output: rgb, gradients, depth and alpha equal
  the unsplit forward's bit for bit.
"""
import numpy as np
import pytest

from paper_2605_11489_gb300 import synth

from gpu_util import check_colour, check_depth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g

    g.build()
    import oracle
    from paper_2605_11489_gb300 import api

    torch.cuda.set_device(0)
    return api, oracle, api.Context(0)


def _render(api, ctx, scene, cam, **kw):
    import torch

    keys = api.OUTPUT_KEYS + api.NORMAL_KEYS
    out = ctx.forward(scene, cam, keys=keys, **kw)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy().astype(np.float64) for k, v in out.items()}


def _check(got, ref):
    ok = (ref["nrm_amb"] == 0) & (ref["amb"] == 0)
    assert ok.mean() > 0.99
    check_colour(got["normal"][:, ok], ref["normal"][:, ok], "normal")
    check_colour(got["nv"][ok], ref["nv"][ok], "nv")
    check_depth(got["depth_isect"][ok], ref["depth_isect"][ok], ref["alpha"][ok])
    # the intersection depth really leaves the centre depth: slopes are in play
    assert np.abs(got["depth_isect"] - got["depth"]).max() > 1e-3


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_tiny_scene_normals(env, tile):
    api, oracle, ctx = env
    sc = synth.tiny_scene(4096, 0)
    cam = synth.tiny_camera(256, 144)
    scene = api.Scene.from_arrays(sc)
    got = _render(api, ctx, scene, cam, tile=tile)
    _check(got, oracle.render_normals(sc, cam))
    # the other outputs are the unsplit forward's, bit for bit
    plain = _render(api, ctx, scene, cam, tile=tile, chunk=1 << 24)
    for k in api.OUTPUT_KEYS:
        assert np.array_equal(got[k], plain[k]), k


def test_jittered_cameras_and_a_ragged_image(env):
    api, oracle, ctx = env
    sc = synth.tiny_scene(4096, 0)
    scene = api.Scene.from_arrays(sc)
    for cam in synth.jittered_tiny_cameras(3, 5, width=203, height=117):
        _check(_render(api, ctx, scene, cam, tile=16), oracle.render_normals(sc, cam))


def test_large_scene_full_frame(env):
    """The 1M workload's frame 0 at 960x540, every pixel against the oracle."""
    api, oracle, ctx = env
    sc = synth.large_scene(1_000_000, 1)
    cam = synth.orbit_cameras(60, 960, 540)[0]
    got = _render(api, ctx, api.Scene.from_arrays(sc), cam, tile=8)
    _check(got, oracle.render_normals(sc, cam))


def test_normal_channel_is_rejected_where_it_is_not_rendered(env):
    import torch

    from paper_2605_11489_gb300 import abi

    api, oracle, ctx = env
    sc = synth.tiny_scene(256, 0)
    cam = synth.tiny_camera(64, 36)
    scene = api.Scene.from_arrays(sc)
    out = api.alloc_outputs(64, 36, api.OUTPUT_KEYS + api.NORMAL_KEYS)
    with pytest.raises(abi.GsError) as e:  # with a backward state
        ctx.forward(scene, cam, out=out, state=True)
    assert e.value.status == abi.GS_ERR_INVALID_ARG
    with pytest.raises(abi.GsError) as e:  # in a graph
        ctx.graph(scene, cam, out, capacity=10000)
    assert e.value.status == abi.GS_ERR_INVALID_ARG
    host = {k: torch.empty(v.shape).pin_memory() for k, v in out.items()}
    with pytest.raises(abi.GsError) as e:  # into host memory
        ctx.forward_to_host(scene, cam, host)
    assert e.value.status == abi.GS_ERR_INVALID_ARG
    # the context still renders afterwards
    _check(_render(api, ctx, scene, cam), oracle.render_normals(sc, cam))
