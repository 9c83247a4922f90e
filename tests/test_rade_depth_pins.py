"""Pins of the oracle's RaDe-GS intersection depth (oracle.render_normals' depth_isect,
the depth the paper renders with RaDe-GS, Sec. 5.1), against definitions that share
nothing with the oracle's arithmetic:

  - the exact densest point of a 3-D Gaussian along the camera ray through image point
    p, t*(p) = (d^T Sigma_c^-1 mu_c) / (d^T Sigma_c^-1 d), d = ((u - cx)/fx, (v - cy)/fy, 1),
    with Sigma_c and mu_c built here from scipy's quaternion rotation;
  - the ray-plane depth (n . mu_c) / (n . d) of a flat disc (one scale ~0).

The oracle's depth is affine in the pixel (the mean of z given (u, v) in the EWA ray space),
so it must equal t* at the projected centre and share its first derivatives there; with
footprints tens of pixels wide the 0.3 px^2 low-pass moves the slope by < 1e-3 of itself.
With one Gaussian, depth_isect / alpha is that affine depth at each pixel centre.
"""
import numpy as np
import pytest

from paper_2605_11489_gb300 import synth

Rotation = pytest.importorskip("scipy.spatial.transform").Rotation


def _one(mean, log_scales, quat, logit=2.0):
    s = synth.empty_scene(1, 0)
    s.means[:, 0] = mean
    s.log_scales[:, 0] = log_scales
    s.quats[:, 0] = quat
    s.logits[0] = logit
    s.sh[0, :, 0] = 1.0
    return s


def _camera_frame(cam, s):
    """mu_c, Sigma_c of Gaussian 0 in camera coordinates (float64, from the fp32 inputs)."""
    V = np.asarray(cam.viewmat, np.float64).reshape(3, 4)
    Rw, t = V[:, :3], V[:, 3]
    w, x, y, z = (float(v) for v in s.quats[:, 0])
    R = Rotation.from_quat([x, y, z, w]).as_matrix()  # scalar-last
    S = np.diag(np.exp(s.log_scales[:, 0].astype(np.float64)))
    Sig = R @ S @ S @ R.T
    mu = Rw @ s.means[:, 0].astype(np.float64) + t
    return mu, Rw @ Sig @ Rw.T


def _ray(cam, u, v):
    return np.array([(u - cam.cx) / cam.fx, (v - cam.cy) / cam.fy, 1.0])


def _t_star(cam, mu, Sig, u, v):
    d = _ray(cam, u, v)
    Si = np.linalg.inv(Sig)
    return (d @ Si @ mu) / (d @ Si @ d)


def _oracle_depth(O, s, cam):
    """The oracle's per-pixel intersection depth z(p) = depth_isect / alpha, and alpha."""
    r = O.render_normals(s, cam)
    a = r["alpha"]
    with np.errstate(invalid="ignore", divide="ignore"):
        z = np.where(a > 0, r["depth_isect"] / np.where(a > 0, a, 1.0), np.nan)
    return z, a


def _centre(cam, mu):
    return cam.fx * mu[0] / mu[2] + cam.cx, cam.fy * mu[1] / mu[2] + cam.cy


CASES = [  # (mean, log-scales, quaternion w x y z): off the optical axis, rotated, anisotropic
    ((0.35, -0.2, 0.3), (0.1, -0.25, -0.6), (0.9, 0.3, -0.2, 0.25)),
    ((-0.4, 0.25, -0.5), (-0.1, 0.15, -0.4), (0.6, -0.5, 0.4, 0.45)),
    ((0.3, 0.3, 0.6), (0.2, -0.5, -0.2), (0.2, 0.8, 0.5, -0.3)),
]


@pytest.mark.parametrize("case", range(len(CASES)))
def test_intersection_depth_matches_the_exact_ray_maximum_to_first_order(case):
    import oracle as O

    mean, ls, q = CASES[case]
    s = _one(mean, ls, q)
    cam = synth.tiny_camera(256, 144)
    mu, Sig = _camera_frame(cam, s)
    u0, v0 = _centre(cam, mu)
    assert abs(mu[0] / mu[2]) > 0.05 and abs(mu[1] / mu[2]) > 0.03  # off the axis: J02, J12 matter
    z, a = _oracle_depth(O, s, cam)
    px, py = int(np.floor(u0)), int(np.floor(v0))
    assert a[py, px] > 0 and a[py, px + 1] > 0 and a[py + 1, px] > 0
    # the oracle's slope (exact differences of an affine function) against the derivative
    # of the exact ray maximum at the projected centre
    gx, gy = z[py, px + 1] - z[py, px], z[py + 1, px] - z[py, px]
    h = 0.25
    ex = (_t_star(cam, mu, Sig, u0 + h, v0) - _t_star(cam, mu, Sig, u0 - h, v0)) / (2 * h)
    ey = (_t_star(cam, mu, Sig, u0, v0 + h) - _t_star(cam, mu, Sig, u0, v0 - h)) / (2 * h)
    assert max(abs(ex), abs(ey)) > 1e-3  # a real slope
    scale = np.hypot(ex, ey)
    assert abs(gx - ex) <= 2e-3 * scale and abs(gy - ey) <= 2e-3 * scale, (gx, ex, gy, ey)
    # and its value: the camera z of the mean at the projected centre
    zc = z[py, px] + gx * (u0 - (px + 0.5)) + gy * (v0 - (py + 0.5))
    assert abs(zc - mu[2]) <= 1e-9 * mu[2]
    assert abs(_t_star(cam, mu, Sig, u0, v0) - mu[2]) <= 1e-12 * mu[2]
    # near the centre the affine depth leaves the exact maximum by no more than the latter's
    # second-order term (its Hessian at the centre, by central differences), plus the
    # slope tolerance times the distance
    t = lambda du, dv: _t_star(cam, mu, Sig, u0 + du, v0 + dv)
    k = 1.0
    H = np.array([[t(k, 0) - 2 * t(0, 0) + t(-k, 0), (t(k, k) - t(k, -k) - t(-k, k) + t(-k, -k)) / 4],
                  [0.0, t(0, k) - 2 * t(0, 0) + t(0, -k)]]) / k ** 2
    H[1, 0] = H[0, 1]
    hn = np.abs(np.linalg.eigvalsh(H)).max()
    for dx, dy in ((3, 0), (0, -3), (2, 2), (-4, 1)):
        p, r = px + dx, py + dy
        D = np.hypot(p + 0.5 - u0, r + 0.5 - v0)
        e = _t_star(cam, mu, Sig, p + 0.5, r + 0.5)
        assert abs(z[r, p] - e) <= 0.5 * hn * D * D * 1.25 + 2e-3 * scale * D, (dx, dy, z[r, p], e)


def test_intersection_depth_of_a_flat_disc_is_the_ray_plane_depth_to_first_order():
    """A disc (third scale 1e-4 of the others) tilted towards the camera: its densest point
    along a ray is where the ray meets its plane, depth (n . mu_c) / (n . d)."""
    import oracle as O

    q = np.array([0.92, 0.25, -0.3, 0.05])
    s = _one((0.3, -0.15, 0.2), (0.0, -0.1, np.log(1e-4)), q)
    cam = synth.tiny_camera(256, 144)
    mu, _ = _camera_frame(cam, s)
    V = np.asarray(cam.viewmat, np.float64).reshape(3, 4)
    w, x, y, z_ = (float(v) for v in s.quats[:, 0])
    n = V[:, :3] @ Rotation.from_quat([x, y, z_, w]).as_matrix()[:, 2]  # the thin axis, camera frame

    def plane_depth(u, v):
        d = _ray(cam, u, v)
        return (n @ mu) / (n @ d)

    assert abs(n[2]) < 0.95  # tilted: the plane depth varies across the image
    u0, v0 = _centre(cam, mu)
    z, a = _oracle_depth(O, s, cam)
    px, py = int(np.floor(u0)), int(np.floor(v0))
    gx, gy = z[py, px + 1] - z[py, px], z[py + 1, px] - z[py, px]
    h = 0.25
    ex = (plane_depth(u0 + h, v0) - plane_depth(u0 - h, v0)) / (2 * h)
    ey = (plane_depth(u0, v0 + h) - plane_depth(u0, v0 - h)) / (2 * h)
    scale = np.hypot(ex, ey)
    assert scale > 1e-3
    assert abs(gx - ex) <= 2e-3 * scale and abs(gy - ey) <= 2e-3 * scale, (gx, ex, gy, ey)


def test_isotropic_gaussian_on_the_axis_has_a_flat_intersection_depth():
    """On the optical axis an isotropic Gaussian's densest point along every nearby ray is
    at the depth of its centre to first order: the affine depth is the constant z."""
    import oracle as O

    s = _one((0.0, 0.0, 0.0), (-0.5, -0.5, -0.5), (1.0, 0.0, 0.0, 0.0))
    cam = synth.tiny_camera(96, 64)
    z, a = _oracle_depth(O, s, cam)
    m = a > 0
    assert m.sum() > 200
    assert np.all(np.abs(z[m] - 4.0) <= 1e-12 * 4.0)


def test_intersection_depth_blends_like_the_colour():
    """Two Gaussians: depth_isect = z_1(p) a_1 + z_2(p) a_2 (1 - a_1), each z_k(p) the
    single-Gaussian affine depth, at every pixel where neither decision is open."""
    import oracle as O

    cam = synth.tiny_camera(128, 72)
    a_ = _one((0.2, 0.1, 0.5), (-0.6, -0.9, -0.7), (0.8, 0.2, 0.4, -0.1), logit=0.5)
    b_ = _one((0.0, 0.05, -0.4), (-0.4, -0.8, -0.5), (0.3, -0.6, 0.2, 0.5), logit=0.0)
    both = synth.empty_scene(2, 0)
    for f in ("means", "log_scales", "quats"):
        getattr(both, f)[:, 0] = getattr(a_, f)[:, 0]
        getattr(both, f)[:, 1] = getattr(b_, f)[:, 0]
    both.logits[0], both.logits[1] = a_.logits[0], b_.logits[0]
    both.sh[0, :, :2] = 1.0
    za, aa = _oracle_depth(O, a_, cam)
    zb, ab = _oracle_depth(O, b_, cam)
    r = O.render_normals(both, cam)
    ok = r["amb"] == 0
    za, zb = np.nan_to_num(za), np.nan_to_num(zb)
    # a_ is in front (camera at z = 4 looks down -z): it blends first
    want = za * aa + zb * ab * (1.0 - aa)
    assert (ok & (aa > 0) & (ab > 0)).sum() > 50
    assert np.allclose(r["depth_isect"][ok], want[ok], rtol=1e-12, atol=1e-12)
