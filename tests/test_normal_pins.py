"""Pins of the oracle's normal channel and normal-view map.

- The normal is RaDe-GS's, which the paper renders with (Sec. 5.1): a Gaussian's shortest
  axis, facing the camera, blended with the colour's weights.
- The normal-view inner product map Nv is the one GASS takes (Sec. 4.1).

The pins use geometry the code does not state:
- a disc tilted by theta about the camera's x axis has the normal (0, sin theta, -cos theta),
  so N = that normal times alpha, and Nv at the principal point is cos theta times alpha;
- the quaternion's sign and a half turn of the disc leave the normal unchanged;
- equal scales pick the first axis;
- a convex combination of unit normals has |N| <= alpha.
"""
import math

import numpy as np
import pytest

import oracle
from paper_2605_11489_gb300 import synth


def _one(scales, quat, z=5.0, logit=2.0, W=41, H=31):
    sc = synth.empty_scene(1, 0)
    sc.means[:, 0] = (0.0, 0.0, z)
    sc.log_scales[:, 0] = np.log(np.asarray(scales, np.float64))
    sc.quats[:, 0] = quat
    sc.logits[0] = logit
    sc.sh[0, :, 0] = 0.5
    cam = synth.Camera(np.eye(3, 4, dtype=np.float32).reshape(12), 30.0, 30.0, W / 2.0, H / 2.0, W, H, 0.2)
    return sc, cam


def _quat_x(theta):
    return (math.cos(theta / 2), math.sin(theta / 2), 0.0, 0.0)


@pytest.mark.parametrize("theta", [0.0, 0.3, -0.7, 1.2])
def test_tilted_disc_normal_and_nv(theta):
    """Scales (0.3, 0.2, 0.01): the disc's normal is its local z axis, rotated by theta about x:
    (0, -sin, cos) in the camera frame, which faces away from a camera looking down +z, so the
    rendered normal is its opposite (0, sin theta, -cos theta)."""
    sc, cam = _one((0.3, 0.2, 0.01), _quat_x(theta))
    r = oracle.render_normals(sc, cam)
    want = np.array([0.0, math.sin(theta), -math.cos(theta)])
    assert r["alpha"].max() > 0.5
    # the quaternion is stored in fp32, so the geometry holds to ~1e-8 relative
    np.testing.assert_allclose(r["normal"], want[:, None, None] * r["alpha"][None], rtol=1e-6, atol=1e-12)
    # Nv = -N . ray: at the principal point the ray is (0, 0, 1) -> cos(theta) alpha; the
    # principal point (W/2, H/2) is a pixel corner here, so check the 2x2 pixels around it
    # against the exact rays of their centres
    H, W = cam.height, cam.width
    for py in (H // 2 - 1, H // 2):
        for px in (W // 2 - 1, W // 2):
            ray = np.array([(px + 0.5 - cam.cx) / cam.fx, (py + 0.5 - cam.cy) / cam.fy, 1.0])
            ray /= np.linalg.norm(ray)
            assert r["nv"][py, px] == pytest.approx(-(want @ ray) * r["alpha"][py, px], rel=1e-6, abs=1e-12)
    if theta == 0.0:
        assert np.abs(r["nv"][H // 2, W // 2] - r["alpha"][H // 2, W // 2]) < 1e-3


def test_quaternion_sign_and_half_turn_leave_the_normal_unchanged():
    base = oracle.render_normals(*_one((0.3, 0.2, 0.01), _quat_x(0.4)))
    neg = oracle.render_normals(*_one((0.3, 0.2, 0.01), tuple(-c for c in _quat_x(0.4))))
    flipped = oracle.render_normals(*_one((0.3, 0.2, 0.01), _quat_x(0.4 + math.pi)))
    np.testing.assert_allclose(neg["normal"], base["normal"], atol=1e-12)
    np.testing.assert_allclose(flipped["normal"], base["normal"], atol=1e-9)
    np.testing.assert_allclose(flipped["nv"], base["nv"], atol=1e-9)


def test_the_smallest_scale_picks_the_axis_and_ties_take_the_first():
    # smallest scale on local x: the normal is the rotated x axis (1, 0, 0) rotated by 0.3
    # about x, i.e. (1, 0, 0) itself (perpendicular to the view ray: Nv = 0 at the centre)
    r = oracle.render_normals(*_one((0.01, 0.2, 0.3), _quat_x(0.3)))
    n = r["normal"] / np.maximum(r["alpha"], 1e-300)[None]
    hit = r["alpha"] > 1e-3
    np.testing.assert_allclose(np.abs(n[0][hit]), 1.0, atol=1e-12)
    np.testing.assert_allclose(n[1:, hit], 0.0, atol=1e-12)
    assert r["nrm_amb"].max() == 1  # exactly perpendicular to the view direction: open
    # equal smallest scales on y and z: y (the first) wins
    r = oracle.render_normals(*_one((0.3, 0.01, 0.01), _quat_x(0.0)))
    n = r["normal"] / np.maximum(r["alpha"], 1e-300)[None]
    np.testing.assert_allclose(np.abs(n[1][r["alpha"] > 1e-3]), 1.0, atol=1e-12)


def test_normal_is_a_convex_combination():
    sc = synth.tiny_scene(4096, 0)
    cam = synth.tiny_camera(128, 72)
    r = oracle.render_normals(sc, cam)
    n = np.linalg.norm(r["normal"], axis=0)
    assert np.all(n <= r["alpha"] + 1e-12)
    assert np.all(np.abs(r["nv"]) <= r["alpha"] + 1e-12)
    # every normal faces the camera along its own view ray, so they mostly reinforce: the
    # blended normal points toward the camera (Nv > 0) almost everywhere it is covered
    covered = r["alpha"] > 0.5
    assert covered.mean() > 0.05 and (r["nv"][covered] > 0.0).mean() > 0.99
    assert np.median(n[covered] / r["alpha"][covered]) > 0.5
    # the same alpha as the colour render
    np.testing.assert_array_equal(r["alpha"], oracle.render(sc, cam)["alpha"])
