"""Pins of the oracle's EWA projection away from the optical axis (Sec. 3: "EWA
splatting", Sigma = R S S^T R^T; Sigma2D = J W Sigma W^T J^T + 0.3 I).

Nothing here repeats the oracle's own formula. The expected screen-space
covariance comes from the camera's pinhole map itself, (fx x/z + cx, fy y/z + cy)
after the world->camera transform:
  - its Jacobian by central differences at the mean (the local affine
    approximation that defines EWA splatting), with Sigma built by SciPy's
    quaternion rotation;
  - propagation of a covariance through the exact map by symmetric sigma points,
    and by Monte-Carlo samples, as the covariance shrinks to 0;
  - beyond 1.3x the half field of view (the 3DGS guard), the Jacobian of the same
    map taken at the point whose x/z (y/z) is clamped to the guard.
A camera rotated about every axis, fx != fy and an off-centre principal point
make a transposed W, a swapped fx/fy or a sign flip of the off-diagonal Jacobian
terms change the result by far more than the tolerances.
"""
import math

import numpy as np
import pytest
from scipy.spatial.transform import Rotation

from paper_2605_11489_gb300 import synth

pytestmark = pytest.mark.usefixtures("oracle_lib")

LOWPASS = 0.3


def _camera():
    vm = synth.look_at((1.3, -0.7, 4.2), (0.2, 0.1, 0.0), (0.15, 1.0, 0.25))
    return synth.Camera(vm, 210.0, 170.0, 101.3, 77.9, 200, 150, 0.2)


def _rot_t(cam):
    m = cam.viewmat.astype(np.float64).reshape(3, 4)
    return m[:, :3], m[:, 3]


def _pinhole_cam(cam, p):
    """Camera-space point(s) [..., 3] -> pixel coordinates [..., 2]."""
    p = np.asarray(p, dtype=np.float64)
    return np.stack([cam.fx * p[..., 0] / p[..., 2] + cam.cx, cam.fy * p[..., 1] / p[..., 2] + cam.cy], axis=-1)


def _pinhole_world(cam, x):
    R, t = _rot_t(cam)
    return _pinhole_cam(cam, np.asarray(x, dtype=np.float64) @ R.T + t)


def _fd_jacobian(f, x, h):
    x = np.asarray(x, dtype=np.float64)
    cols = []
    for k in range(3):
        e = np.zeros(3)
        e[k] = h
        cols.append((f(x + e) - f(x - e)) / (2 * h))
    return np.stack(cols, axis=1)  # [2, 3]


def _sigma(log_s, q_wxyz):
    """Sigma = R diag(s^2) R^T with R from SciPy (scalar-last quaternion order)."""
    s = np.exp(np.asarray(log_s, dtype=np.float64))
    w, x, y, z = (float(v) for v in q_wxyz)
    R = Rotation.from_quat([x, y, z, w]).as_matrix()
    return R @ np.diag(s * s) @ R.T


def _scene(cam, cam_points, log_scales, quats, logits):
    """Gaussians whose means sit at the given camera-space points (fp32 inputs)."""
    R, t = _rot_t(cam)
    n = len(cam_points)
    sc = synth.empty_scene(n, 0)
    for i, p in enumerate(cam_points):
        sc.means[:, i] = R.T @ (np.asarray(p, dtype=np.float64) - t)
        sc.log_scales[:, i] = log_scales[i]
        sc.quats[:, i] = quats[i]
        sc.logits[i] = logits[i]
        sc.sh[0, :, i] = 0.5
    return sc


def _inputs(sc, i):
    f64 = lambda a: a.astype(np.float64)
    return f64(sc.means[:, i]), f64(sc.log_scales[:, i]), f64(sc.quats[:, i])


def _off_axis_gaussians(cam, seed, n=24, lim_frac=0.93):
    """Rotated anisotropic Gaussians at off-axis camera-space positions inside the guard."""
    rng = np.random.default_rng(seed)
    limx = 1.3 * (0.5 * cam.width) / cam.fx
    limy = 1.3 * (0.5 * cam.height) / cam.fy
    pts, ls, qs, lg = [], [], [], []
    for _ in range(n):
        z = rng.uniform(2.0, 6.0)
        pts.append((rng.uniform(-lim_frac, lim_frac) * limx * z, rng.uniform(-lim_frac, lim_frac) * limy * z, z))
        ls.append(rng.uniform(-3.5, -1.0, 3) + np.array([0.0, -0.8, -1.6]))
        qs.append(rng.normal(size=4))
        lg.append(rng.normal(1.0, 1.0))
    return _scene(cam, pts, ls, qs, lg)


def _cov2d(p, i):
    A, B, C = p["cov2d"][i]
    return np.array([[A, B], [B, C]])


def test_cov2d_equals_fd_jacobian_of_the_pinhole_map_off_axis(oracle_lib):
    """Sigma2D = Jw Sigma Jw^T + 0.3 I, Jw the central-difference Jacobian of
    world -> pixel at the mean; the conic is its inverse, (u, v) the map at the mean."""
    O = oracle_lib
    cam = _camera()
    sc = _off_axis_gaussians(cam, seed=5)
    p = O.project(sc, cam)
    worst = 0.0
    for i in range(sc.n):
        mu, ls, q = _inputs(sc, i)
        Jw = _fd_jacobian(lambda x: _pinhole_world(cam, x), mu, 1e-5)
        ref = Jw @ _sigma(ls, q) @ Jw.T + LOWPASS * np.eye(2)
        got = _cov2d(p, i)
        err = np.abs(got - ref).max() / np.abs(ref).max()
        worst = max(worst, err)
        assert err < 1e-7, (i, got, ref)
        assert np.allclose(p["uv"][i], _pinhole_world(cam, mu), rtol=0, atol=1e-9)
        conic = np.linalg.inv(ref)
        assert np.allclose(p["conic"][i], (conic[0, 0], conic[0, 1], conic[1, 1]), rtol=1e-6, atol=0)
    # the off-axis terms matter here: the on-axis Jacobian (J02 = J12 = 0) would be far off
    mu, ls, q = _inputs(sc, 0)
    R, t = _rot_t(cam)
    tz = (R @ mu + t)[2]
    J_on = np.array([[cam.fx / tz, 0, 0], [0, cam.fy / tz, 0]]) @ R
    on = J_on @ _sigma(ls, q) @ J_on.T + LOWPASS * np.eye(2)
    assert np.abs(on - _cov2d(p, 0)).max() > 1e-2 * np.abs(on).max()


def test_cov2d_equals_sigma_point_propagation(oracle_lib):
    """Covariance propagated through the exact pinhole map by symmetric sigma points
    mu +- eps sqrt(3) L e_k (L L^T = Sigma), divided by eps^2, tends to
    Sigma2D - 0.3 I as eps -> 0 (the local affine approximation of EWA)."""
    O = oracle_lib
    cam = _camera()
    sc = _off_axis_gaussians(cam, seed=6)
    p = O.project(sc, cam)
    eps = 1e-4
    for i in range(sc.n):
        mu, ls, q = _inputs(sc, i)
        L = np.linalg.cholesky(_sigma(ls, q))
        pts = [mu + sgn * eps * math.sqrt(3.0) * L[:, k] for k in range(3) for sgn in (1.0, -1.0)]
        y = _pinhole_world(cam, np.array(pts))
        d = y - y.mean(axis=0)
        cov = d.T @ d / len(pts) / eps ** 2
        ref = _cov2d(p, i) - LOWPASS * np.eye(2)
        assert np.abs(cov - ref).max() < 1e-6 * np.abs(ref).max(), (i, cov, ref)


def test_cov2d_equals_monte_carlo_covariance_of_projected_samples(oracle_lib):
    """Empirical covariance of the pinhole images of samples of N(mu, eps^2 Sigma),
    divided by eps^2, against Sigma2D - 0.3 I (sampling error ~ 3e-3 at 4e5 samples)."""
    O = oracle_lib
    cam = _camera()
    sc = _off_axis_gaussians(cam, seed=7, n=6)
    p = O.project(sc, cam)
    rng = np.random.default_rng(11)
    eps = 1e-3
    for i in range(sc.n):
        mu, ls, q = _inputs(sc, i)
        Sig = _sigma(ls, q)
        x = rng.multivariate_normal(mu, eps ** 2 * Sig, size=400_000)
        y = _pinhole_world(cam, x)
        cov = np.cov(y.T) / eps ** 2
        ref = _cov2d(p, i) - LOWPASS * np.eye(2)
        ev = np.linalg.eigvalsh(ref).max()
        assert np.abs(cov - ref).max() < 2e-2 * ev, (i, cov, ref)


@pytest.mark.parametrize("kx,ky", [(1.6, 0.3), (-1.9, -0.2), (0.1, 1.7), (2.2, -1.5)])
def test_guard_clamp_uses_the_jacobian_at_the_clamped_point(oracle_lib, kx, ky):
    """Beyond 1.3x the half field of view, the Jacobian is that of the pinhole map
    at the camera-space point whose x/z (y/z) is clamped to the guard; the
    projected centre (u, v) itself is not clamped."""
    O = oracle_lib
    cam = _camera()
    limx = 1.3 * (0.5 * cam.width) / cam.fx
    limy = 1.3 * (0.5 * cam.height) / cam.fy
    z = 3.7
    pc = np.array([kx * limx * z, ky * limy * z, z])
    sc = _scene(cam, [pc], [np.array([-0.6, -1.4, -2.3])], [np.array([0.8, 0.3, -0.4, 0.5])], [2.0])
    p = O.project(sc, cam)
    mu, ls, q = _inputs(sc, 0)
    R, t = _rot_t(cam)
    pt = R @ mu + t
    clamped = np.array([np.clip(pt[0] / pt[2], -limx, limx) * pt[2], np.clip(pt[1] / pt[2], -limy, limy) * pt[2],
                        pt[2]])
    Jc = _fd_jacobian(lambda v: _pinhole_cam(cam, v), clamped, 1e-6) @ R
    Sig = _sigma(ls, q)
    ref = Jc @ Sig @ Jc.T + LOWPASS * np.eye(2)
    got = _cov2d(p, 0)
    assert np.abs(got - ref).max() < 1e-7 * np.abs(ref).max(), (got, ref)
    assert np.allclose(p["uv"][0], _pinhole_cam(cam, pt), rtol=0, atol=1e-9)
    # without the clamp the Jacobian is a different one
    Ju = _fd_jacobian(lambda v: _pinhole_cam(cam, v), pt, 1e-6) @ R
    unclamped = Ju @ Sig @ Ju.T + LOWPASS * np.eye(2)
    assert np.abs(unclamped - got).max() > 1e-2 * np.abs(got).max()


def test_discrete_rect_and_depth_follow_the_continuous_projection(oracle_lib):
    """The fp32 discrete spec's depth key and support rectangle against the FP64
    projection pinned above: z32 is the camera-space z within 2 fp32 ulp, and the
    rectangle is the box of pixel centres inside the ellipse o G >= 1/255, i.e.
    half-extents sqrt(k Sigma2D_xx), sqrt(k Sigma2D_yy) with k = 2 ln(255 o)
    (the exact bounding box of the ellipse), except where an edge lies within
    1e-3 px of a pixel centre (fp32 rounding may decide it either way)."""
    O = oracle_lib
    tiny = synth.tiny_scene(2048, seed=3)
    checked = guarded = 0
    for ci, cam in enumerate([_camera()] + synth.jittered_tiny_cameras(3, 9, 200, 150)):
        # plus large Gaussians centred beyond the guard whose support still reaches the image
        rng = np.random.default_rng(40 + ci)
        limx = 1.3 * (0.5 * cam.width) / cam.fx
        limy = 1.3 * (0.5 * cam.height) / cam.fy
        pts, ls, qs, lg = [], [], [], []
        for j in range(64):
            z = rng.uniform(3.0, 8.0)
            a, b = rng.uniform(1.15, 2.5) * rng.choice([-1, 1]), rng.uniform(-0.9, 0.9)
            if j % 2:
                a, b = b, a
            pts.append((a * limx * z, b * limy * z, z))
            ls.append(rng.uniform(-0.5, 1.2, 3))
            qs.append(rng.normal(size=4))
            lg.append(rng.normal(2.0, 1.0))
        far = _scene(cam, pts, ls, qs, lg)
        sc = synth.empty_scene(tiny.n + far.n, 0)
        for name in ("means", "log_scales", "quats"):
            getattr(sc, name)[:, : tiny.n] = getattr(tiny, name)[:, : tiny.n]
            getattr(sc, name)[:, tiny.n: sc.n] = getattr(far, name)[:, : far.n]
        sc.logits[: tiny.n] = tiny.logits[: tiny.n]
        sc.logits[tiny.n: sc.n] = far.logits[: far.n]
        p = O.project(sc, cam)
        R, t = _rot_t(cam)
        mu = sc.means[:, : sc.n].astype(np.float64)
        tz = (R @ mu + t[:, None])[2]
        vis = p["visible"] == 1
        z32 = p["z32"].astype(np.float64)
        assert (np.abs(z32[vis] - tz[vis]) <= 2 * np.spacing(np.abs(tz[vis]).astype(np.float32))).all()
        o = 1.0 / (1.0 + np.exp(-sc.logits[: sc.n].astype(np.float64)))
        k = 2.0 * np.log(255.0 * o)
        ex = np.sqrt(k * p["cov2d"][:, 0])
        ey = np.sqrt(k * p["cov2d"][:, 2])
        u, v = p["uv"][:, 0], p["uv"][:, 1]
        lo_x, hi_x = u - ex - 0.5, u + ex - 0.5
        lo_y, hi_y = v - ey - 0.5, v + ey - 0.5
        for i in np.nonzero(vis)[0]:
            edges = np.array([lo_x[i], hi_x[i], lo_y[i], hi_y[i]])
            if (np.abs(edges - np.round(edges)) < 1e-3).any():
                continue
            ref = (max(0, math.ceil(lo_x[i])), max(0, math.ceil(lo_y[i])), min(cam.width - 1, math.floor(hi_x[i])),
                   min(cam.height - 1, math.floor(hi_y[i])))
            assert tuple(p["rect"][i]) == ref, (i, tuple(p["rect"][i]), ref)
            checked += 1
            guarded += i >= tiny.n
        # a Gaussian not visible is culled for a reason the continuous projection shows
        for i in np.nonzero(~vis)[0][:200]:
            if tz[i] <= cam.near + 1e-4 or o[i] * 255.0 < 1.0 + 1e-6:
                continue
            edges = np.array([lo_x[i], hi_x[i], lo_y[i], hi_y[i]])
            if (np.abs(edges - np.round(edges)) < 1e-3).any():
                continue
            empty = (math.floor(hi_x[i]) < max(0, math.ceil(lo_x[i])) or math.ceil(lo_x[i]) > cam.width - 1
                     or math.floor(hi_y[i]) < max(0, math.ceil(lo_y[i])) or math.ceil(lo_y[i]) > cam.height - 1
                     or math.floor(hi_x[i]) < 0 or math.floor(hi_y[i]) < 0)
            assert empty, i
    assert checked > 2000 and guarded > 40
