"""gs_sort_pairs_static: the radix sort for callers that cannot allocate.

Some callers may not call cudaMalloc: under a framework whose caching
allocator owns the device's memory, or in a real-time loop that must not
allocate after start-up. This entry point sorts with scratch from a static
device array instead. The test calls it through the C ABI on the render's own
(tile, depth) instance list, twice in a row on different frames, and checks
each result bit for bit against the sorted keys and values that
gs_render_forward produced for the same frame (integer work: the tolerance is
exact equality); then at exactly its capacity, in place, against NumPy's
stable argsort. The file is named to be collected last.
"""
import ctypes as C

import numpy as np
import pytest

from paper_2605_11489_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g

    g.build()
    from paper_2605_11489_gb300 import abi, api

    torch.cuda.set_device(0)
    return abi, api, api.Context(0)


def _render_keys(api, ctx, sc, cam, tile=16):
    out, st = ctx.forward(api.Scene.from_arrays(sc), cam, tile=tile, state=True)
    v = st.view()
    st.free()
    return v


def _emission_order(keys, vals):
    """The duplication pass's output order (Gaussian index, then tile row-major),
    recovered from the sorted list: the input the render's sort received."""
    tiles = (keys >> np.uint64(32)).astype(np.int64)
    order = np.lexsort((tiles, vals))
    return keys[order], vals[order]


def _sort_static(abi, keys, vals, bits, in_place=False):
    import torch

    kin = torch.from_numpy(keys.view(np.int64)).cuda()
    vin = torch.from_numpy(vals.view(np.int32)).cuda()
    kout = kin if in_place else torch.empty_like(kin)
    vout = vin if in_place else torch.empty_like(vin)
    status = torch.full((1,), -1, dtype=torch.int32, device="cuda")
    s = torch.cuda.current_stream()
    abi.check(abi.lib().gs_sort_pairs_static(kin.data_ptr(), vin.data_ptr(), kout.data_ptr(), vout.data_ptr(),
                                             len(keys), bits, status.data_ptr(), s.cuda_stream))
    s.synchronize()
    assert status.item() == 0  # no lookback gave up
    return kout.cpu().numpy().view(np.uint64), vout.cpu().numpy().view(np.uint32)


def test_static_sort_matches_render_sort_two_calls(env):
    abi, api, ctx = env
    frames = [(synth.tiny_scene(4096, 0), synth.tiny_camera()),
              (synth.clustered_scene(60_000, 3, (2.0, 2.0, 2.0), 8, 3), synth.tiny_camera(480, 270))]
    for sc, cam in frames:  # two calls in a row, different sizes: the shared scratch is re-cleared
        v = _render_keys(api, ctx, sc, cam)
        ref_k, ref_v = v["keys"], v["vals"]
        assert len(ref_k) > 1000
        in_k, in_v = _emission_order(ref_k, ref_v)
        tile_bits = max(1, int(np.ceil(np.log2(max(v["n_tiles"], 2)))))
        got_k, got_v = _sort_static(abi, in_k, in_v, 32 + tile_bits)
        assert np.array_equal(got_k, ref_k)
        assert np.array_equal(got_v, ref_v)


@pytest.mark.parametrize("bits", [40, 64])
def test_static_sort_at_capacity_in_place(env, bits):
    """Exactly 1,048,576 pairs (the capacity), keys_in == keys_out and vals_in ==
    vals_out, against NumPy's stable sort of the same keys on their low `bits` bits."""
    abi, api, ctx = env
    rng = np.random.default_rng(bits)
    n = 1 << 20
    keys = rng.integers(0, 1 << 63, n, dtype=np.int64).view(np.uint64)
    keys[::7] = keys[3]  # many equal keys: stability matters
    vals = np.arange(n, dtype=np.uint32)
    mask = np.uint64((1 << bits) - 1) if bits < 64 else np.uint64(0xFFFFFFFFFFFFFFFF)
    order = np.argsort(keys & mask, kind="stable")
    got_k, got_v = _sort_static(abi, keys, vals, bits, in_place=True)
    assert np.array_equal(got_v, vals[order])
    assert np.array_equal(got_k, keys[order])


def test_static_sort_rejects_more_than_its_capacity(env):
    abi, api, ctx = env
    import torch

    k = torch.zeros(8, dtype=torch.int64, device="cuda")
    v = torch.zeros(8, dtype=torch.int32, device="cuda")
    st = abi.lib().gs_sort_pairs_static(k.data_ptr(), v.data_ptr(), k.data_ptr(), v.data_ptr(), (1 << 20) + 1, 40,
                                        None, None)
    assert st == abi.GS_ERR_INVALID_ARG
    assert b"1048576" in abi.lib().gs_last_error()
    # n = 0 is a no-op
    assert abi.lib().gs_sort_pairs_static(k.data_ptr(), v.data_ptr(), k.data_ptr(), v.data_ptr(), 0, 40, None,
                                          None) == 0
