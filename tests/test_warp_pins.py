"""Pins of the oracle's frame-interpolation geometry (Sec. 4.2, "Forward-Backward Warping").

The oracle computes V[x] = Proj(UnProj(x, D, P_src), P_dst) - x, the depth-tested
forward warp w(., V) and the warped gradient w(G, V) . dx/dy. These tests hold it to
what the geometry fixes independently of its code: closed forms of V for a camera
that translates, zooms or rolls in front of a fronto-parallel plane, the analytic
Jacobian of those maps (which the oracle only sees through central differences),
and a brute-force per-target-pixel search for the depth test on tiny frames.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_11489_gb300 import synth


def _cam(width=64, height=48, fx=70.0, fy=55.0, eye=(0.3, -0.2, -5.0), viewmat=None):
    base = synth.make_camera(eye, (0.0, 0.0, 0.0), (0.0, -1.0, 0.0), width, height)
    vm = base.viewmat if viewmat is None else np.asarray(viewmat, np.float32)
    return synth.Camera(vm.copy(), fx, fy, width / 2.0 + 0.37, height / 2.0 - 0.21, width, height, 0.2)


def _with_viewmat(cam, vm):
    return synth.Camera(np.asarray(vm, np.float32).reshape(12), cam.fx, cam.fy, cam.cx, cam.cy, cam.width,
                        cam.height, cam.near)


def _grid(cam):
    j, i = np.mgrid[0:cam.height, 0:cam.width].astype(np.float64)
    return i + 0.5, j + 0.5


def _rt(cam):
    vm = cam.viewmat.astype(np.float64).reshape(3, 4)
    return vm[:, :3], vm[:, 3]


def _plane_frame(cam, d, seed=0, G=2):
    """Constant point depth d in front of ``cam`` (no alpha), random planes and gradients."""
    rng = np.random.default_rng(seed)
    H, W = cam.height, cam.width
    return dict(depth=np.full((H, W), d, np.float32), planes=rng.random((3, H, W)).astype(np.float32),
                dcdx=rng.standard_normal((G, H, W)).astype(np.float32),
                dcdy=rng.standard_normal((G, H, W)).astype(np.float32))


def _interior(cam, margin=2):
    m = np.zeros((cam.height, cam.width), bool)
    m[margin:-margin, margin:-margin] = True
    return m


def test_identity_camera_leaves_every_pixel_in_place():
    cam = _cam()
    f = synth.warp_frame(cam.width, cam.height, seed=3)
    r = oracle.warp(cam, cam, f["depth"], f["alpha"], 0.0, f["planes"], f["dcdx"], f["dcdy"])
    moves = f["alpha"] > 0
    assert np.all(np.isnan(r["motion64"][0][~moves]))
    # FP64 map; the fp32 viewmat's rotation is orthonormal only to ~1e-7, and UnProj uses R^T.
    assert np.max(np.abs(r["motion64"][:, moves])) < 1e-5
    assert np.max(np.abs(r["motion"][:, moves])) < 1e-4  # fp32 sequence: a few ulps of the pixel position
    idx = np.arange(cam.width * cam.height).reshape(cam.height, cam.width)
    assert np.array_equal(r["index"], np.where(moves, idx, -1))
    assert np.array_equal(r["out"], np.where(moves, f["planes"], 0.0))
    inner = moves & _interior(cam)
    np.testing.assert_allclose(r["out_dcdx"][:, inner], f["dcdx"][:, inner], rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(r["out_dcdy"][:, inner], f["dcdy"][:, inner], rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("k", [(3, 0), (-2, 5), (0, -4)])
def test_sideways_translation_shifts_the_image_by_whole_pixels(k):
    """Camera moved by (kx d/fx, ky d/fy) along its own x and y axes in front of a
    plane at camera depth d: every pixel moves by (-kx, -ky) exactly (V = -f delta/d)."""
    cam = _cam()
    d = 6.0
    R, t = _rt(cam)
    delta = np.array([k[0] * d / np.float32(cam.fx), k[1] * d / np.float32(cam.fy), 0.0])
    dst = _with_viewmat(cam, np.concatenate([R, (t - delta)[:, None]], axis=1))
    f = _plane_frame(cam, d)
    r = oracle.warp(cam, dst, f["depth"], None, 0.0, f["planes"], f["dcdx"], f["dcdy"])
    # Closed form (FP64 map; the fp32 viewmat rounds delta, hence the tolerance).
    np.testing.assert_allclose(r["motion64"][0], -k[0], atol=2e-5)
    np.testing.assert_allclose(r["motion64"][1], -k[1], atol=2e-5)
    H, W = cam.height, cam.width
    j, i = np.mgrid[0:H, 0:W]
    si, sj = i + k[0], j + k[1]  # the source pixel that lands on target (i, j)
    inside = (si >= 0) & (si < W) & (sj >= 0) & (sj < H)
    assert np.array_equal(r["index"][inside], (sj * W + si)[inside])
    assert np.all(r["index"][~inside] == -1)
    np.testing.assert_allclose(r["z"][inside], d, rtol=1e-6)
    # A pure translation has dy/dx = I: gradients are carried unchanged.
    inner = inside & (si > 1) & (si < W - 2) & (sj > 1) & (sj < H - 2)
    src = (sj * W + si)[inner]
    np.testing.assert_allclose(r["out_dcdx"][:, inner], f["dcdx"].reshape(2, -1)[:, src], rtol=1e-4, atol=1e-5)
    np.testing.assert_allclose(r["out_dcdy"][:, inner], f["dcdy"].reshape(2, -1)[:, src], rtol=1e-4, atol=1e-5)


@pytest.mark.parametrize("dz", [1.5, -2.0])
def test_dolly_scales_about_the_principal_point(dz):
    """Camera moved by dz along its optical axis toward a plane at depth d: positions
    scale by s = d / (d - dz) about the principal point, V = (s - 1)(x - c), the
    Jacobian is s I and the warped gradient is G / s."""
    cam = _cam(width=80, height=60)
    d = 7.0
    s = d / (d - dz)
    R, t = _rt(cam)
    dst = _with_viewmat(cam, np.concatenate([R, (t - np.array([0.0, 0.0, dz]))[:, None]], axis=1))
    f = _plane_frame(cam, d, seed=1)
    r = oracle.warp(cam, dst, f["depth"], None, 0.0, f["planes"], f["dcdx"], f["dcdy"])
    x, y = _grid(cam)
    cx, cy = np.float32(cam.cx), np.float32(cam.cy)
    np.testing.assert_allclose(r["motion64"][0], (s - 1.0) * (x - cx), atol=1e-5)
    np.testing.assert_allclose(r["motion64"][1], (s - 1.0) * (y - cy), atol=1e-5)
    np.testing.assert_allclose(r["z"][r["index"] >= 0], d - dz, rtol=1e-6)
    hit = r["index"] >= 0
    p = r["index"][hit]
    si, sj = p % cam.width, p // cam.width
    # Winners whose source pixel has both neighbours in each direction moving see J = s I.
    inner = (si > 0) & (si < cam.width - 1) & (sj > 0) & (sj < cam.height - 1)
    for key, gkey in (("out_dcdx", "dcdx"), ("out_dcdy", "dcdy")):
        want = f[gkey].reshape(2, -1)[:, p[inner]] / s
        np.testing.assert_allclose(r[key][:, hit][:, inner], want, rtol=2e-4, atol=1e-5)
    # The Jacobian the oracle reports is s I there, and the identity at holes.
    jac = r["jac"][:, hit][:, inner]
    np.testing.assert_allclose(jac, np.array([s, 0.0, 0.0, s])[:, None] * np.ones_like(jac), atol=2e-4 * s)
    assert np.array_equal(r["jac"][:, ~hit], np.array([1.0, 0.0, 0.0, 1.0])[:, None] * np.ones((4, (~hit).sum())))
    if s > 1:
        assert (~hit).sum() > 0  # magnification opens holes between the source pixels
    else:
        assert hit.sum() < (r["motion64"][0] == r["motion64"][0]).sum()  # several sources per target


@pytest.mark.parametrize("theta", [0.05, -0.2])
def test_roll_about_the_optical_axis_rotates_the_gradient(theta):
    """Camera rolled by theta about its optical axis (fx != fy): positions follow
    u' - cx = cos(t)(u - cx) - (fx/fy) sin(t)(v - cy), v' - cy = (fy/fx) sin(t)(u - cx)
    + cos(t)(v - cy), for any depth. The warped gradient is G J^-1 with that
    (non-symmetric) J: a transposed or mis-signed inverse fails here."""
    cam = _cam(width=72, height=56)
    R, t = _rt(cam)
    c, s_ = math.cos(theta), math.sin(theta)
    Rz = np.array([[c, -s_, 0.0], [s_, c, 0.0], [0.0, 0.0, 1.0]])
    dst = _with_viewmat(cam, np.concatenate([Rz @ R, (Rz @ t)[:, None]], axis=1))
    rng = np.random.default_rng(5)
    d = (4.0 + rng.random((cam.height, cam.width))).astype(np.float32)  # depth does not matter for a roll
    f = _plane_frame(cam, 1.0, seed=2)
    r = oracle.warp(cam, dst, d, None, 0.0, f["planes"], f["dcdx"], f["dcdy"])
    x, y = _grid(cam)
    fx, fy = np.float32(cam.fx), np.float32(cam.fy)
    cx, cy = np.float32(cam.cx), np.float32(cam.cy)
    J = np.array([[c, -(fx / fy) * s_], [(fy / fx) * s_, c]])
    up = cx + J[0, 0] * (x - cx) + J[0, 1] * (y - cy)
    vp = cy + J[1, 0] * (x - cx) + J[1, 1] * (y - cy)
    np.testing.assert_allclose(r["motion64"][0], up - x, atol=2e-5)
    np.testing.assert_allclose(r["motion64"][1], vp - y, atol=2e-5)
    hit = r["index"] >= 0
    p = r["index"][hit]
    si, sj = p % cam.width, p // cam.width
    inner = (si > 0) & (si < cam.width - 1) & (sj > 0) & (sj < cam.height - 1)
    g = np.stack([f["dcdx"].reshape(2, -1)[:, p[inner]], f["dcdy"].reshape(2, -1)[:, p[inner]]], axis=-1)
    np.testing.assert_allclose(r["jac"][:, hit][:, inner], J.reshape(4, 1) * np.ones((4, inner.sum())), atol=2e-4)
    want = g @ np.linalg.inv(J)  # row vector times dx/dy
    np.testing.assert_allclose(r["out_dcdx"][:, hit][:, inner], want[..., 0], rtol=2e-4, atol=2e-5)
    np.testing.assert_allclose(r["out_dcdy"][:, hit][:, inner], want[..., 1], rtol=2e-4, atol=2e-5)


def _spec_positions(src, dst, depth, alpha, amin):
    """The fp32 sequence the oracle documents, evaluated with numpy float32 scalars
    (IEEE round-to-nearest, no fused operations)."""
    f = np.float32
    H, W = src.height, src.width
    R = src.viewmat.astype(np.float32)
    Q = dst.viewmat.astype(np.float32)
    out = {}
    for j in range(H):
        for i in range(W):
            a = f(alpha[j, i])
            if not a > f(amin):
                continue
            d = f(depth[j, i]) / a
            xn = ((f(i) + f(0.5)) - f(src.cx)) / f(src.fx)
            yn = ((f(j) + f(0.5)) - f(src.cy)) / f(src.fy)
            a0, a1, a2 = xn * d - R[3], yn * d - R[7], d - R[11]
            w = [(R[0 + c] * a0 + R[4 + c] * a1) + R[8 + c] * a2 for c in range(3)]
            X, Y, Z = [((Q[4 * r] * w[0] + Q[4 * r + 1] * w[1]) + Q[4 * r + 2] * w[2]) + Q[4 * r + 3]
                       for r in range(3)]
            if not Z > f(dst.near):
                continue
            out[j * W + i] = ((f(dst.fx) * X) / Z + f(dst.cx), (f(dst.fy) * Y) / Z + f(dst.cy), Z)
    return out


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_depth_test_equals_a_brute_force_search_per_target_pixel(seed):
    """Tiny frames with heavy overlap (the target camera backs off and turns): for every
    target pixel, the winner is the (z, index)-smallest of all source pixels whose
    position falls inside it; a pixel nobody reaches is a hole."""
    src = _cam(width=19, height=13, fx=20.0, fy=18.0)
    P0, P05, _ = synth.interpolation_cameras(23, 11)
    vm = synth.look_at((0.9, -0.6, -6.5), (0.2, 0.1, 0.0), (0.0, -1.0, 0.0))
    dst = synth.Camera(vm, 16.0, 15.0, 11.7, 5.4, 23, 11, 0.2)
    f = synth.warp_frame(19, 13, seed=seed, depth_range=(3.0, 6.0), occluders=6, holes=2, channels=2)
    r = oracle.warp(src, dst, f["depth"], f["alpha"], 0.05, f["planes"])
    pos = _spec_positions(src, dst, f["depth"], f["alpha"], 0.05)
    # The motion output is exactly the documented fp32 sequence.
    W = src.width
    for p, (u, v, z) in pos.items():
        i, j = p % W, p // W
        assert r["motion"][0, j, i] == np.float32(u - (np.float32(i) + np.float32(0.5)))
        assert r["motion"][1, j, i] == np.float32(v - (np.float32(j) + np.float32(0.5)))
    moving = np.zeros((src.height, W), bool)
    moving.flat[list(pos)] = True
    assert np.array_equal(~np.isnan(r["motion"][0]), moving)
    n_win = 0
    for tj in range(dst.height):
        for ti in range(dst.width):
            cands = [(np.float32(z).view(np.uint32), p) for p, (u, v, z) in pos.items()
                     if 0 <= u < dst.width and 0 <= v < dst.height and math.floor(u) == ti and math.floor(v) == tj]
            if not cands:
                assert r["index"][tj, ti] == -1 and r["z"][tj, ti] == 0
                assert np.all(r["out"][:, tj, ti] == 0)
                continue
            zb, p = min(cands)
            n_win += 1
            assert r["index"][tj, ti] == p
            assert r["z"][tj, ti] == pos[p][2]
            assert np.array_equal(r["out"][:, tj, ti], f["planes"].reshape(2, -1)[:, p])
    assert n_win > 0 and (r["index"] < 0).any()
    # Overlap happened: fewer winners than in-bounds moving sources.
    landed = sum(1 for u, v, z in pos.values() if 0 <= u < dst.width and 0 <= v < dst.height)
    assert n_win < landed


def test_pixels_at_or_below_alpha_min_do_not_move():
    cam = _cam()
    P = _with_viewmat(cam, cam.viewmat)
    f = synth.warp_frame(cam.width, cam.height, seed=9)
    amin = 0.5
    r = oracle.warp(cam, P, f["depth"], f["alpha"], amin, f["planes"])
    still = ~(f["alpha"] > np.float32(amin))
    assert still.any() and (~still).any()
    assert np.all(np.isnan(r["motion"][:, still]))
    assert not np.isin(np.flatnonzero(still), r["index"]).any()


def test_fp32_motion_is_the_fp64_map_up_to_rounding():
    P0, P05, P1 = synth.interpolation_cameras(240, 135)
    f = synth.warp_frame(240, 135, seed=4)
    r = oracle.warp(P1, P05, f["depth"], f["alpha"], 0.0)
    m32, m64 = r["motion"].astype(np.float64), r["motion64"]
    assert np.array_equal(np.isnan(m32), np.isnan(m64))
    ok = ~np.isnan(m64)
    assert ok.mean() > 0.5
    # |u| <= ~ 2 W; a handful of fp32 roundings of that size.
    assert np.max(np.abs(m32[ok] - m64[ok])) < 64 * np.finfo(np.float32).eps * 2 * 240
    assert np.max(np.abs(m64[ok])) > 1.0  # the half-step orbit really moves the pixels


def test_equal_depths_go_to_the_smaller_source_index():
    """Axis-aligned cameras backing away from a plane of constant depth: every target z
    is the same fp32 number, several source pixels share each target pixel, and the
    first of them in row-major order wins."""
    eye = np.eye(3, 4, dtype=np.float32).reshape(12)
    src = synth.Camera(eye.copy(), 30.0, 30.0, 16.0, 12.0, 32, 24, 0.2)
    back = eye.copy()
    back[11] = 3.0  # camera moved back by 3 along its optical axis
    dst = synth.Camera(back, 30.0, 30.0, 16.0, 12.0, 32, 24, 0.2)
    d = np.full((24, 32), 4.0, np.float32)
    f = _plane_frame(src, 4.0, seed=7)
    r = oracle.warp(src, dst, d, None, 0.0, f["planes"])
    pos = _spec_positions(src, dst, d, np.ones_like(d), -1.0)
    assert len({z for _, _, z in pos.values()}) == 1
    for tj in range(dst.height):
        for ti in range(dst.width):
            cands = [p for p, (u, v, z) in pos.items() if math.floor(u) == ti and math.floor(v) == tj]
            assert r["index"][tj, ti] == (min(cands) if cands else -1)
    assert np.bincount(np.floor(np.array([u for u, _, _ in pos.values()])).astype(int)).max() > 24
