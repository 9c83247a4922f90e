"""GPU parity of the frame-interpolation warp (Sec. 4.2, "Forward-Backward Warping")
against the oracle, through the C ABI (gs_warp).

Bars:
  - motion map, winning source index, winner's target z, warped planes: bit for bit
    (one fixed fp32 round-to-nearest sequence decides the landing position and the
    depth test on both sides; the planes are copies);
  - warped gradient: within the rounding bound of its fp32 evaluation. The GPU takes
    the Jacobian entries as fp32 differences of the same fp32 positions the oracle
    subtracts in FP64 (relative error <= u = 2^-24 each), the determinant and the two
    numerators as compensated 2x2 differences of products (<= 2u relative) and one
    rounded division. First-order propagation gives
        |dg_x| <= c u [(|g0 J11| + |g1 J10|) + |g_x| (|J00 J11| + |J01 J10|)] / |det| + c u |g_x|
    (and the same for g_y with (|g1 J00| + |g0 J01|)), with c = 16 as a safety factor
    over the c = 4 the derivation gives. Pixels whose determinant lies within
    16 u (|J00 J11| + |J01 J10|) of 0 can take the fold decision either way and are
    left out (they must be rare).
"""
import numpy as np
import pytest

from paper_2605_11489_gb300 import synth

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24
C_SAFE = 16.0


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g

    g.build()
    import oracle
    from paper_2605_11489_gb300 import api

    torch.cuda.set_device(0)
    return api, oracle, api.Context(0)


def _dev(a):
    import torch

    return None if a is None else torch.from_numpy(np.ascontiguousarray(a, dtype=np.float32)).cuda()


def _gpu_warp(api, ctx, src, dst, f, amin=0.0, use_alpha=True, grads=True, planes=True):
    import torch

    out = ctx.warp(src, dst, _dev(f["depth"]), _dev(f["alpha"]) if use_alpha else None, amin,
                   _dev(f["planes"]) if planes else None, _dev(f["dcdx"]) if grads else None,
                   _dev(f["dcdy"]) if grads else None)
    torch.cuda.synchronize()
    return {k: v.cpu().numpy() for k, v in out.items()}


def _oracle_warp(oracle, src, dst, f, amin=0.0, use_alpha=True, grads=True, planes=True):
    return oracle.warp(src, dst, f["depth"], f["alpha"] if use_alpha else None, amin,
                       f["planes"] if planes else None, f["dcdx"] if grads else None, f["dcdy"] if grads else None)


def check_warp(g, r, f, grads=True, planes=True):
    """Compare one gs_warp result with the oracle's; returns (hits, ambiguous folds)."""
    # motion: the same fp32 numbers, NaN exactly where a pixel does not move
    assert np.array_equal(g["motion"], r["motion"], equal_nan=True)
    assert np.array_equal(g["index"], r["index"])
    assert np.array_equal(g["z"].view(np.uint32), r["z"].view(np.uint32))
    hit = r["index"] >= 0
    if planes:
        assert np.array_equal(g["planes"], r["out"].astype(np.float32))
    if not grads:
        return int(hit.sum()), 0
    assert np.all(g["dcdx"][:, ~hit] == 0) and np.all(g["dcdy"][:, ~hit] == 0)
    J00, J01, J10, J11 = r["jac"]
    det = J00 * J11 - J01 * J10
    cross = np.abs(J00 * J11) + np.abs(J01 * J10)
    amb = hit & (np.abs(det) <= C_SAFE * U32 * cross)
    ok = hit & ~amb
    p = r["index"][ok]
    dd = np.abs(det[ok])
    a, b, c_, d = J00[ok], J01[ok], J10[ok], J11[ok]
    for ch in range(r["out_dcdx"].shape[0]):
        g0 = f["dcdx"][ch].reshape(-1)[p].astype(np.float64)
        g1 = f["dcdy"][ch].reshape(-1)[p].astype(np.float64)
        rx, ry = r["out_dcdx"][ch][ok], r["out_dcdy"][ch][ok]
        tx = C_SAFE * U32 * ((np.abs(g0 * d) + np.abs(g1 * c_)) + np.abs(rx) * cross[ok]) / dd + C_SAFE * U32 * np.abs(rx)
        ty = C_SAFE * U32 * ((np.abs(g1 * a) + np.abs(g0 * b)) + np.abs(ry) * cross[ok]) / dd + C_SAFE * U32 * np.abs(ry)
        ex = np.abs(g["dcdx"][ch][ok] - rx)
        ey = np.abs(g["dcdy"][ch][ok] - ry)
        assert np.all(ex <= tx), "dcdx[%d]: %d pixels out of bound, worst excess %.3g" % (
            ch, (ex > tx).sum(), (ex - tx).max())
        assert np.all(ey <= ty), "dcdy[%d]: %d pixels out of bound, worst excess %.3g" % (
            ch, (ey > ty).sum(), (ey - ty).max())
    assert amb.sum() <= max(2, 1e-3 * hit.sum()), "too many near-zero determinants: %d" % amb.sum()
    return int(hit.sum()), int(amb.sum())


@pytest.mark.parametrize("seed,amin", [(0, 0.0), (1, 0.3), (2, 0.0)])
def test_low_resolution_frame_toward_the_intermediate_pose(env, seed, amin):
    """Frame 1 (colour, depth, normals + image gradients) warped from P1 to P0.5."""
    api, oracle, ctx = env
    P0, P05, P1 = synth.interpolation_cameras(240, 135, k=seed)
    f = synth.warp_frame(240, 135, seed=seed, channels=7, grad_channels=3)
    g = _gpu_warp(api, ctx, P1, P05, f, amin)
    r = _oracle_warp(oracle, P1, P05, f, amin)
    hits, _ = check_warp(g, r, f)
    assert hits > 0.5 * 240 * 135 and (r["index"] < 0).any()


def test_high_resolution_frame_without_gradients(env):
    """Frame 0 at 4x (colour, depth, normals) warped from P0 to P0.5, no gradient planes."""
    api, oracle, ctx = env
    P0, P05, _ = synth.interpolation_cameras(160, 90)
    src, dst = P0.scaled(4), P05.scaled(4)
    f = synth.warp_frame(640, 360, seed=5, channels=7, grad_channels=0)
    g = _gpu_warp(api, ctx, src, dst, f, grads=False)
    r = _oracle_warp(oracle, src, dst, f, grads=False)
    check_warp(g, r, f, grads=False)


def test_ragged_sizes_and_another_target_resolution(env):
    """Source 203x117 toward a 150x91 target with other intrinsics and a rolled pose."""
    api, oracle, ctx = env
    _, P05, P1 = synth.interpolation_cameras(203, 117, k=3)
    vm = P05.viewmat.reshape(3, 4).astype(np.float64)
    c, s = np.cos(0.07), np.sin(0.07)
    Rz = np.array([[c, -s, 0.0], [s, c, 0.0], [0.0, 0.0, 1.0]])
    dst = synth.Camera((Rz @ vm).astype(np.float32).reshape(12), P05.fx * 0.8, P05.fy * 0.75, 74.3, 46.1, 150, 91,
                       0.2)
    f = synth.warp_frame(203, 117, seed=8, channels=3, grad_channels=2)
    g = _gpu_warp(api, ctx, P1, dst, f, 0.1)
    r = _oracle_warp(oracle, P1, dst, f, 0.1)
    check_warp(g, r, f)


def test_point_depth_without_alpha(env):
    api, oracle, ctx = env
    _, P05, P1 = synth.interpolation_cameras(128, 72, k=7)
    f = synth.warp_frame(128, 72, seed=9, channels=2, grad_channels=1)
    f["depth"] = np.where(f["alpha"] > 0, f["depth"] / np.maximum(f["alpha"], 1e-6), 0.0).astype(np.float32)
    g = _gpu_warp(api, ctx, P1, P05, f, use_alpha=False)
    r = _oracle_warp(oracle, P1, P05, f, use_alpha=False)
    check_warp(g, r, f)


def test_equal_depths_go_to_the_smaller_source_index(env):
    """A camera backing away from a constant-depth plane: every target z is the same
    fp32 number, so the depth test falls to the source index on both sides."""
    api, oracle, ctx = env
    eye = np.eye(3, 4, dtype=np.float32).reshape(12)
    src = synth.Camera(eye.copy(), 30.0, 30.0, 16.0, 12.0, 32, 24, 0.2)
    back = eye.copy()
    back[11] = 3.0
    dst = synth.Camera(back, 30.0, 30.0, 16.0, 12.0, 32, 24, 0.2)
    rng = np.random.default_rng(3)
    f = dict(depth=np.full((24, 32), 4.0, np.float32), alpha=None, planes=rng.random((2, 24, 32)).astype(np.float32),
             dcdx=rng.standard_normal((1, 24, 32)).astype(np.float32),
             dcdy=rng.standard_normal((1, 24, 32)).astype(np.float32))
    g = _gpu_warp(api, ctx, src, dst, f, use_alpha=False)
    r = _oracle_warp(oracle, src, dst, f, use_alpha=False)
    check_warp(g, r, f)
    assert len(np.unique(r["z"][r["index"] >= 0])) == 1


def test_empty_and_degenerate_frames(env):
    api, oracle, ctx = env
    P0, P05, P1 = synth.interpolation_cameras(64, 36)
    f = synth.warp_frame(64, 36, seed=1, channels=2, grad_channels=1)
    # nothing moves: alpha 0 everywhere
    f0 = dict(f, alpha=np.zeros_like(f["alpha"]))
    g = _gpu_warp(api, ctx, P1, P05, f0)
    assert np.isnan(g["motion"]).all() and (g["index"] == -1).all() and (g["planes"] == 0).all()
    check_warp(g, _oracle_warp(oracle, P1, P05, f0), f0)
    # the target camera looks the other way: every point is behind its near plane
    vm = P05.viewmat.reshape(3, 4).copy()
    vm[0] *= -1.0
    vm[2] *= -1.0
    away = synth.Camera(vm.reshape(12), P05.fx, P05.fy, P05.cx, P05.cy, 64, 36, 0.2)
    g = _gpu_warp(api, ctx, P1, away, f)
    assert (g["index"] == -1).all() and np.isnan(g["motion"]).all()
    check_warp(g, _oracle_warp(oracle, P1, away, f), f)
    # 1 x 1 images (no neighbours: the identity Jacobian)
    one = dict(depth=np.full((1, 1), 50.0, np.float32), alpha=np.ones((1, 1), np.float32),
               planes=np.full((1, 1, 1), 0.25, np.float32), dcdx=np.full((1, 1, 1), 2.0, np.float32),
               dcdy=np.full((1, 1, 1), -1.0, np.float32))
    c1 = synth.Camera(P1.viewmat, 1.0, 1.0, 0.5, 0.5, 1, 1, 0.2)
    g = _gpu_warp(api, ctx, c1, c1, one)
    r = _oracle_warp(oracle, c1, c1, one)
    check_warp(g, r, one)
    assert g["index"][0, 0] == 0 and g["dcdx"][0, 0, 0] == 2.0 and g["dcdy"][0, 0, 0] == -1.0


def test_calls_in_a_row_leave_the_depth_test_slots_empty(env):
    """The depth-test slots are reset by each call's gather: a sequence of calls of
    different sizes gives the same results as each call alone."""
    api, oracle, ctx = env
    P0, P05, P1 = synth.interpolation_cameras(96, 54)
    fa = synth.warp_frame(96, 54, seed=2, channels=1, grad_channels=1)
    P0s, P05s = P0.scaled(2), P05.scaled(2)
    fb = synth.warp_frame(192, 108, seed=3, channels=1, grad_channels=1)
    first = _gpu_warp(api, ctx, P1, P05, fa)
    big = _gpu_warp(api, ctx, P0s, P05s, fb)
    again = _gpu_warp(api, ctx, P1, P05, fa)
    big2 = _gpu_warp(api, ctx, P0s, P05s, fb)
    for k in first:
        assert np.array_equal(first[k], again[k], equal_nan=True), k
        assert np.array_equal(big[k], big2[k], equal_nan=True), k
    check_warp(big, _oracle_warp(oracle, P0s, P05s, fb), fb)


def test_invalid_arguments_are_rejected(env):
    import torch

    from paper_2605_11489_gb300 import abi

    api, oracle, ctx = env
    _, P05, P1 = synth.interpolation_cameras(32, 18)
    f = synth.warp_frame(32, 18, seed=4, channels=1, grad_channels=1)
    d = _dev(f["depth"])
    with pytest.raises(abi.GsError) as e:  # NULL depth
        ctx.warp(P1, P05, None)
    assert e.value.status == abi.GS_ERR_INVALID_ARG
    bad = synth.Camera(P05.viewmat, P05.fx, P05.fy, P05.cx, P05.cy, 32, 18, -1.0)
    with pytest.raises(abi.GsError) as e:  # negative near plane on the target
        ctx.warp(P1, bad, d)
    assert e.value.status == abi.GS_ERR_INVALID_ARG
    with pytest.raises(abi.GsError) as e:  # gradients asked for without the dcdy input
        ctx.warp(P1, P05, d, dcdx=_dev(f["dcdx"]))
    assert e.value.status == abi.GS_ERR_INVALID_ARG
    raw = torch.empty(32 * 18 + 1, dtype=torch.float32, device="cuda")
    gi = abi.GsWarpInput(raw.data_ptr() + 2, None, 0.0, 0, None, 0, None, None)
    go = abi.GsWarpOutput(None, None, None, None, None, None)
    sc, dc = api.camera_struct(P1), api.camera_struct(P05)
    import ctypes as C

    st = abi.lib().gs_warp(ctx.h, C.byref(sc), C.byref(dc), C.byref(gi), C.byref(go), None)
    assert st == abi.GS_ERR_INVALID_ARG  # misaligned plane
    # the context still works afterwards
    g = _gpu_warp(api, ctx, P1, P05, f)
    check_warp(g, _oracle_warp(oracle, P1, P05, f), f)


def test_full_size_forward_backward_pair(env):
    """The interpolation workload's sizes, in the calls the benchmark times: the 4x
    frame 0 (3840x2160, 7 planes) toward P0.5 and the 960x540 frame 1 (7 planes + 3
    gradient planes) toward P0.5, against the oracle on every pixel."""
    api, oracle, ctx = env
    w = synth.interp_inputs()
    g = _gpu_warp(api, ctx, w["P0_hr"], w["P05_hr"], w["hr"], grads=False)
    r = _oracle_warp(oracle, w["P0_hr"], w["P05_hr"], w["hr"], grads=False)
    hits, _ = check_warp(g, r, w["hr"], grads=False)
    assert hits > 0.5 * 3840 * 2160
    g = _gpu_warp(api, ctx, w["P1"], w["P05"], w["lr"])
    r = _oracle_warp(oracle, w["P1"], w["P05"], w["lr"])
    check_warp(g, r, w["lr"])
