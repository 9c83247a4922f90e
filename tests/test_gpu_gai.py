"""GPU parity of the gradient-aware interpolation (Sec. 4.1, Eq. 5-8) against the oracle,
through the C ABI (gs_gai_upsample).

Bar: |gpu - oracle| <= 64 u T per output, with u = 2^-24 and T the sum of the absolute terms
of the output's evaluation as M x + b (oracle.gai.gai_term_scale). The derivation:
- the GPU folds the two layers of Eq. 8 into M and b in double and rounds each entry once
  to fp32 (<= u relative);
- it then evaluates 27 fused multiply-adds onto the bias, each adding <= u of the running
  |sum|;
- in all, <= ~30 u T. The bar takes 64 u T, about a factor 2 over that.
Inputs are synthetic or the oracle's own render, the same fp32 numbers on both sides.
"""
import numpy as np
import pytest

from paper_2605_11489_gb300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g

    g.build()
    import oracle
    from oracle import gai as og
    from paper_2605_11489_gb300 import api

    torch.cuda.set_device(0)
    return api, oracle, og


def _dev(a):
    import torch

    return torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _check(api, og, weights, I, Ix, Iy):
    import torch

    out = api.gai_upsample(weights, _dev(I), _dev(Ix), _dev(Iy))
    torch.cuda.synchronize()
    got = out.cpu().numpy().astype(np.float64)
    S, wc, bc, wt, bt = weights
    planes = [np.asarray(a, np.float32).astype(np.float64) for a in (I, Ix, Iy)]
    for c in range(planes[0].shape[0]):  # one channel at a time keeps the FP64 oracle's memory small
        sl = [p[c:c + 1] for p in planes]
        ref = og.gai(*sl, wc, bc, wt, bt, S)[0]
        scale = og.gai_term_scale(*sl, wc, bc, wt, bt, S)[0]
        err = np.abs(got[c] - ref)
        bound = 64 * U32 * scale
        assert np.all(err <= bound), "channel %d: %d outputs out of bound, worst ratio %.3g" % (
            c, (err > bound).sum(), (err / np.maximum(bound, 1e-300)).max())
    return got


@pytest.mark.parametrize("S", [2, 3, 4])
def test_random_weights_ragged_image(env, S):
    api, oracle, og = env
    rng = np.random.default_rng(S)
    I, Ix, Iy = (rng.standard_normal((3, 23, 37)).astype(np.float32) for _ in range(3))
    _check(api, og, synth.gai_weights(S, 32, seed=S), I, Ix, Iy)


@pytest.mark.parametrize("S", [2, 4])
def test_hermite_weights_on_the_oracle_render(env, S):
    """The analytic Hermite weights of the oracle applied to the oracle's render of the tiny
    scene (colour and its Eq. 3 gradients): the interpolation the paper feeds to GASS."""
    api, oracle, og = env
    sc = synth.tiny_scene(4096, 0)
    cam = synth.tiny_camera(256, 144)
    r = oracle.render(sc, cam)
    Wc, bc, Wt, bt = og.hermite_weights(S, 4, channels=32)
    _check(api, og, (S, Wc, bc, Wt, bt), r["rgb"], r["dcdx"], r["dcdy"])


def test_single_pixel_and_single_channel(env):
    api, oracle, og = env
    one = lambda v: np.full((1, 1, 1), v, np.float32)
    got = _check(api, og, synth.gai_weights(4, 20, seed=5), one(0.7), one(-1.5), one(2.25))
    assert got.shape == (1, 4, 4)


def test_many_channels_and_features(env):
    api, oracle, og = env
    rng = np.random.default_rng(9)
    I, Ix, Iy = (rng.standard_normal((7, 17, 9)).astype(np.float32) for _ in range(3))
    _check(api, og, synth.gai_weights(3, 100, seed=2), I, Ix, Iy)


def test_invalid_arguments_are_rejected(env):
    import ctypes as C

    import torch

    from paper_2605_11489_gb300 import abi

    api, oracle, og = env
    p = _dev(np.zeros((3, 8, 8)))
    S, wc, bc, wt, bt = synth.gai_weights(4, 32)
    with pytest.raises(abi.GsError) as e:  # scale 5
        api.gai_upsample((5, wc, bc, np.zeros((25, 32), np.float32), None), p, p, p)
    assert e.value.status == abi.GS_ERR_INVALID_ARG
    raw = torch.empty(3 * 32 * 32 + 4, dtype=torch.float32, device="cuda")
    w = abi.GsGaiWeights(4, 32, wc.ctypes.data, bc.ctypes.data, wt.ctypes.data, bt.ctypes.data)
    st = abi.lib().gs_gai_upsample(C.byref(w), p.data_ptr(), p.data_ptr(), p.data_ptr(), 3, 8, 8,
                                   raw.data_ptr() + 4, None)
    assert st == abi.GS_ERR_INVALID_ARG  # output not 16-byte aligned
    w0 = abi.GsGaiWeights(4, 0, wc.ctypes.data, None, wt.ctypes.data, None)
    assert abi.lib().gs_gai_upsample(C.byref(w0), p.data_ptr(), p.data_ptr(), p.data_ptr(), 3, 8, 8,
                                     raw.data_ptr(), None) == abi.GS_ERR_INVALID_ARG


def test_full_size_960x540_to_3840x2160(env):
    """The benchmark's size and call: three 960x540 planes (smooth colour, N(0, 1)
    gradients) at S = 4 with the seeded weights, every output against the oracle."""
    api, oracle, og = env
    f = synth.warp_frame(960, 540, seed=13, channels=3, grad_channels=3)
    _check(api, og, synth.gai_weights(4, 32), f["planes"], f["dcdx"], f["dcdy"])
