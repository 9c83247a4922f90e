"""Seeded synthetic inputs: Gaussian scenes, cameras and request streams.

This module is the single source of inputs for both the CUDA render path and the
CPU oracle. It holds none of the render arithmetic (no projection, no SH
evaluation, no compositing): it only draws parameters and builds camera poses.

Scene layout (attribute-planar SoA, fp32, every plane padded to ``n_pad``, a
multiple of 4, so that each plane starts on a 16-byte boundary):

    means       [3, n_pad]          x, y, z (world units)
    log_scales  [3, n_pad]          log of the per-axis scale
    quats       [4, n_pad]          w, x, y, z (not normalised: the renderer does it)
    logits      [n_pad]             opacity logit (opacity = sigmoid(logit))
    sh          [(deg+1)^2, 3, n_pad]  SH coefficients, l-major, m = -l..l

The Gaussian model (mean, covariance from rotation and scale, opacity, SH colour)
is the one of the paper's preliminaries (Sec. 3, Eq. 1 and the text after it).
Camera: OpenCV axes (x right, y down, z forward), world->camera ``viewmat`` as a
row-major 3x4 [R | t]; pixel (i, j) is sampled at (i + 0.5, j + 0.5).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

# The DC colour is drawn uniformly in [0, 1] and stored as the SH DC coefficient
# k00 with colour = k00 * Y00 + 0.5, Y00 = 1 / (2 sqrt(pi)). So k00 is uniform on
# [-0.5 / Y00, 0.5 / Y00] = [-sqrt(pi), sqrt(pi)].
_DC_HALF_RANGE = math.sqrt(math.pi)


@dataclass
class SceneArrays:
    n: int
    deg: int
    means: np.ndarray
    log_scales: np.ndarray
    quats: np.ndarray
    logits: np.ndarray
    sh: np.ndarray

    @property
    def n_pad(self) -> int:
        return self.means.shape[1]

    @property
    def n_coeffs(self) -> int:
        return (self.deg + 1) ** 2

    def subset(self, idx: np.ndarray) -> "SceneArrays":
        """Scene made of the Gaussians ``idx`` (in that order), re-padded."""
        idx = np.asarray(idx, dtype=np.int64)
        out = empty_scene(len(idx), self.deg)
        out.means[:, : len(idx)] = self.means[:, idx]
        out.log_scales[:, : len(idx)] = self.log_scales[:, idx]
        out.quats[:, : len(idx)] = self.quats[:, idx]
        out.logits[: len(idx)] = self.logits[idx]
        out.sh[:, :, : len(idx)] = self.sh[:, :, idx]
        return out

    def nbytes(self) -> int:
        return sum(a.nbytes for a in (self.means, self.log_scales, self.quats, self.logits, self.sh))


def pad4(n: int) -> int:
    return max(4, (n + 3) // 4 * 4)


def empty_scene(n: int, deg: int) -> SceneArrays:
    if deg not in (0, 1, 2, 3):
        raise ValueError("sh degree must be 0..3")
    n_pad = pad4(n)
    k = (deg + 1) ** 2
    z = lambda *s: np.zeros(s, dtype=np.float32)
    return SceneArrays(n, deg, z(3, n_pad), z(3, n_pad), z(4, n_pad), z(n_pad), z(k, 3, n_pad))


@dataclass
class Camera:
    viewmat: np.ndarray  # (12,) float32, row-major [R | t]
    fx: float
    fy: float
    cx: float
    cy: float
    width: int
    height: int
    near: float = 0.2
    eye: np.ndarray = field(default=None, repr=False)

    def shifted(self, dcx: float = 0.0, dcy: float = 0.0) -> "Camera":
        return Camera(self.viewmat.copy(), self.fx, self.fy, self.cx + dcx, self.cy + dcy,
                      self.width, self.height, self.near, self.eye)

    def scaled(self, factor: int) -> "Camera":
        """Same pose at ``factor`` times the resolution (the high-resolution frame of a
        super-sampling factor S = factor)."""
        return Camera(self.viewmat.copy(), _fp32(self.fx * factor), _fp32(self.fy * factor),
                      _fp32(self.cx * factor), _fp32(self.cy * factor), self.width * factor,
                      self.height * factor, self.near, self.eye)


# ----------------------------------------------------------------------------- scenes

def tiny_scene(n: int = 4096, seed: int = 0) -> SceneArrays:
    """4,096-Gaussian unit-cube scene: means U[-1,1]^3, log-scales N(-4, 0.5),
    quaternions N(0,1)^4 (uniform direction on S^3), logits N(0,1), SH degree 0 with
    DC colour U[0,1]."""
    rng = np.random.default_rng(seed)
    s = empty_scene(n, 0)
    s.means[:, :n] = rng.uniform(-1.0, 1.0, (3, n))
    s.log_scales[:, :n] = rng.normal(-4.0, 0.5, (3, n))
    s.quats[:, :n] = rng.normal(0.0, 1.0, (4, n))
    s.logits[:n] = rng.normal(0.0, 1.0, n)
    s.sh[0, :, :n] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (3, n))
    return s


def _random_rotation(rng: np.random.Generator) -> np.ndarray:
    q, r = np.linalg.qr(rng.normal(size=(3, 3)))
    q = q * np.sign(np.diag(r))
    if np.linalg.det(q) < 0:
        q[:, 0] = -q[:, 0]
    return q


def clustered_scene(n: int, seed: int, block=(100.0, 100.0, 20.0), n_clusters: int = 64,
                    deg: int = 3, chunk: int = 1 << 20) -> SceneArrays:
    """Large-scale clustered scene: ``n_clusters`` anisotropic Gaussian blobs with
    centres uniform over the block, random orientation and per-axis std
    log-uniform in [0.5, 8] (world units); points clipped to the block.
    log-scales N(-3, 1) clipped to [-7, 0]; logits N(0, 1.5); SH degree ``deg``
    with non-DC coefficients N(0, 0.2) and DC colour U[0, 1]."""
    rng = np.random.default_rng(seed)
    s = empty_scene(n, deg)
    bx, by, bz = block
    lo = np.zeros(3)
    hi = np.array([bx, by, bz])
    counts = np.full(n_clusters, n // n_clusters, dtype=np.int64)
    counts[: n % n_clusters] += 1
    start = 0
    for c in range(n_clusters):
        m = int(counts[c])
        centre = rng.uniform(lo, hi)
        rot = _random_rotation(rng)
        std = np.exp(rng.uniform(math.log(0.5), math.log(8.0), 3))
        pts = rng.normal(size=(m, 3)) * std
        pts = pts @ rot.T + centre
        np.clip(pts, lo, hi, out=pts)
        s.means[:, start:start + m] = pts.T
        start += m
    s.log_scales[:, :n] = np.clip(rng.normal(-3.0, 1.0, (3, n)), -7.0, 0.0)
    s.quats[:, :n] = rng.normal(0.0, 1.0, (4, n))
    s.logits[:n] = rng.normal(0.0, 1.5, n)
    s.sh[0, :, :n] = rng.uniform(-_DC_HALF_RANGE, _DC_HALF_RANGE, (3, n))
    k = (deg + 1) ** 2
    for j in range(1, k):
        for c3 in range(3):
            for a in range(0, n, chunk):
                b = min(n, a + chunk)
                s.sh[j, c3, a:b] = rng.standard_normal(b - a, dtype=np.float32) * np.float32(0.2)
    return s


def large_scene(n: int = 1_000_000, seed: int = 1) -> SceneArrays:
    """1M Gaussians over a 100 x 100 x 20 m block, SH degree 3."""
    return clustered_scene(n, seed, (100.0, 100.0, 20.0))


def ultra_scene(n: int = 6_000_000, seed: int = 2) -> SceneArrays:
    """6M Gaussians over a 300 x 300 x 40 m aerial layout, SH degree 3."""
    return clustered_scene(n, seed, (300.0, 300.0, 40.0))


def serving_scene(n: int, seed: int) -> SceneArrays:
    """Serving scenes: the clustered generator with block side scaled by
    sqrt(n / 1M) * 100 m (height 20 m)."""
    side = math.sqrt(n / 1.0e6) * 100.0
    return clustered_scene(n, seed, (side, side, 20.0))


# ----------------------------------------------------------------------------- cameras

def look_at(eye, target, up) -> np.ndarray:
    """World->camera [R | t] (row-major 3x4) for OpenCV axes: rows of R are the
    camera's right, down and forward directions in world coordinates."""
    eye = np.asarray(eye, dtype=np.float64)
    f = np.asarray(target, dtype=np.float64) - eye
    f /= np.linalg.norm(f)
    r = np.cross(f, np.asarray(up, dtype=np.float64))
    r /= np.linalg.norm(r)
    d = np.cross(f, r)
    rot = np.stack([r, d, f])
    t = -rot @ eye
    return np.concatenate([rot, t[:, None]], axis=1).reshape(12).astype(np.float32)


def _fp32(v: float) -> float:
    """The nearest fp32 value: the render's camera carries fp32 intrinsics, so the
    generated cameras hold exactly the numbers every consumer receives."""
    return float(np.float32(v))


def make_camera(eye, target, up, width: int, height: int, vfov_deg: float = 60.0,
                near: float = 0.2) -> Camera:
    """Pinhole camera; the field of view is vertical: fy = fx = (H/2) / tan(vfov/2)
    (rounded to fp32), principal point at the image centre."""
    f = _fp32((height / 2.0) / math.tan(math.radians(vfov_deg) / 2.0))
    return Camera(look_at(eye, target, up), f, f, width / 2.0, height / 2.0, int(width),
                  int(height), _fp32(near), np.asarray(eye, dtype=np.float64))


def tiny_camera(width: int = 256, height: int = 144) -> Camera:
    return make_camera((0.0, 0.0, 4.0), (0.0, 0.0, 0.0), (0.0, 1.0, 0.0), width, height)


def jittered_tiny_cameras(count: int = 64, seed: int = 7, width: int = 256,
                          height: int = 144) -> list[Camera]:
    rng = np.random.default_rng(seed)
    cams = []
    for _ in range(count):
        eye = np.array([0.0, 0.0, 4.0]) + rng.normal(0.0, 0.6, 3)
        tgt = rng.normal(0.0, 0.15, 3)
        cams.append(make_camera(eye, tgt, (0.0, 1.0, 0.0), width, height))
    return cams


def orbit_cameras(frames: int = 60, width: int = 960, height: int = 540,
                  centre=(50.0, 50.0, 10.0), radius: float = 80.0,
                  altitude: float = 40.0) -> list[Camera]:
    """Orbit around ``centre`` at ``radius`` and height ``altitude``, world up +z."""
    cams = []
    for k in range(frames):
        th = 2.0 * math.pi * k / frames
        eye = (centre[0] + radius * math.cos(th), centre[1] + radius * math.sin(th), altitude)
        cams.append(make_camera(eye, centre, (0.0, 0.0, 1.0), width, height))
    return cams


def flythrough_cameras(frames: int = 60, width: int = 1920, height: int = 1080,
                       side: float = 300.0, altitude: float = 60.0,
                       pitch_deg: float = 30.0) -> list[Camera]:
    """Straight fly-through along +x across the block at ``altitude``, pitched down."""
    cams = []
    p = math.radians(pitch_deg)
    for k in range(frames):
        x = side * (0.05 + 0.9 * k / max(1, frames - 1))
        eye = np.array([x, side / 2.0, altitude])
        tgt = eye + np.array([math.cos(p), 0.0, -math.sin(p)])
        cams.append(make_camera(eye, tgt, (0.0, 0.0, 1.0), width, height))
    return cams


SERVING_RESOLUTIONS = ((480, 270), (960, 540), (1280, 720), (1920, 1080))
SERVING_SCENE_SIZES = (500_000, 1_000_000, 3_000_000, 6_000_000)


@dataclass
class Request:
    scene: int
    camera: Camera
    arrival_s: float


def serving_requests(count: int = 2000, seed: int = 5, rate_hz: float = 100.0,
                     scene_sizes=SERVING_SCENE_SIZES,
                     resolutions=SERVING_RESOLUTIONS) -> list[Request]:
    """Poisson arrivals at ``rate_hz``; scene uniform; random orbit camera (azimuth
    U[0, 2pi), radius U[0.6, 1] * 0.8 * side, altitude U[0.3, 0.6] * side); resolution
    uniform over ``resolutions``."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for _ in range(count):
        t += rng.exponential(1.0 / rate_hz)
        sc = int(rng.integers(len(scene_sizes)))
        side = math.sqrt(scene_sizes[sc] / 1.0e6) * 100.0
        az = rng.uniform(0.0, 2.0 * math.pi)
        rad = rng.uniform(0.6, 1.0) * 0.8 * side
        alt = rng.uniform(0.3, 0.6) * side
        w, h = resolutions[int(rng.integers(len(resolutions)))]
        c = (side / 2.0, side / 2.0, 10.0)
        eye = (c[0] + rad * math.cos(az), c[1] + rad * math.sin(az), alt)
        out.append(Request(sc, make_camera(eye, c, (0.0, 0.0, 1.0), w, h), t))
    return out


def upstream_grads(width: int, height: int, seed: int = 3) -> dict:
    """N(0,1) upstream gradients on RGB, dC/dx and dC/dy (planar [3, H, W])."""
    rng = np.random.default_rng(seed)
    return {k: rng.standard_normal((3, height, width), dtype=np.float32)
            for k in ("rgb", "dcdx", "dcdy")}


# ----------------------------------------------------------------------------- frame interpolation inputs

def interpolation_cameras(width: int = 960, height: int = 540, frames: int = 60, k: int = 0):
    """(P0, P0.5, P1): frames k and k + 1 of the ``frames``-frame orbit of the large
    scene and the pose half-way between them (the same orbit sampled twice as densely)."""
    dense = orbit_cameras(2 * frames, width, height)
    return dense[2 * k], dense[2 * k + 1], dense[2 * k + 2]


def warp_frame(width: int, height: int, seed: int, depth_range=(40.0, 130.0), occluders: int = 24,
               holes: int = 6, channels: int = 3, grad_channels: int = 3) -> dict:
    """A synthetic rendered frame as the frame-interpolation warp sees it: a smooth
    tilted-surface depth with nearer rectangular occluders (depth discontinuities),
    empty regions (alpha 0) and soft alpha at their edges, smooth colour planes and
    N(0, 1) gradient planes. ``depth`` is unnormalised like the render's depth channel
    (point depth x alpha). All planes fp32, [H, W] or [C, H, W]."""
    rng = np.random.default_rng(seed)
    ys, xs = np.mgrid[0:height, 0:width].astype(np.float64)
    u, v = (xs + 0.5) / width, (ys + 0.5) / height
    d0, d1 = depth_range
    base = d0 + (d1 - d0) * (0.35 + 0.4 * v + 0.15 * u + 0.05 * np.sin(7.0 * u + 3.0 * v))
    point = base.copy()
    for _ in range(occluders):
        w, h = rng.uniform(0.03, 0.2) * width, rng.uniform(0.03, 0.2) * height
        x0, y0 = rng.uniform(-0.1, 1.0) * width, rng.uniform(-0.1, 1.0) * height
        m = (xs >= x0) & (xs < x0 + w) & (ys >= y0) & (ys < y0 + h)
        point[m] = np.minimum(point[m], rng.uniform(0.4, 0.9) * base[m])
    alpha = np.ones((height, width))
    for _ in range(holes):
        cx, cy = rng.uniform(0, width), rng.uniform(0, height)
        r = rng.uniform(0.02, 0.1) * max(width, height)
        dist = np.hypot(xs - cx, ys - cy)
        alpha = np.minimum(alpha, np.clip((dist - r) / (0.25 * r + 1.0), 0.0, 1.0))
    planes = np.stack([0.5 + 0.5 * np.sin(rng.uniform(2, 12) * u + rng.uniform(2, 12) * v + rng.uniform(0, 6))
                       for _ in range(channels)]) if channels else np.zeros((0, height, width))
    return dict(depth=(point * alpha).astype(np.float32), alpha=alpha.astype(np.float32),
                planes=planes.astype(np.float32),
                dcdx=rng.standard_normal((grad_channels, height, width)).astype(np.float32),
                dcdy=rng.standard_normal((grad_channels, height, width)).astype(np.float32))


def interp_inputs(width: int = 960, height: int = 540, scale: int = 4, k: int = 0, seed: int = 11,
                  channels: int = 7, grad_channels: int = 3) -> dict:
    """The frame-interpolation warp workload of Sec. 4.2 for frames k, k + 1 of the large
    scene's orbit: P0, P0.5, P1 at the low resolution; the high-resolution frame 0
    (``scale`` x the size: colour, depth and normal planes, ``channels`` in all) that is
    warped toward P0.5 at high resolution, and the low-resolution frame 1 (the same
    planes plus ``grad_channels`` image-gradient planes) warped toward P0.5 at low
    resolution."""
    P0, P05, P1 = interpolation_cameras(width, height, k=k)
    hr = warp_frame(width * scale, height * scale, seed, channels=channels, grad_channels=0)
    lr = warp_frame(width, height, seed + 1, channels=channels, grad_channels=grad_channels)
    return dict(P0=P0, P05=P05, P1=P1, P0_hr=P0.scaled(scale), P05_hr=P05.scaled(scale), hr=hr, lr=lr)


# ----------------------------------------------------------------------------- super-sampling weights

def gai_weights(scale: int = 4, features: int = 32, seed: int = 21):
    """Seeded stand-in weights of the gradient-aware interpolation's two layers (Sec. 4.1,
    Eq. 8; the trained ones are not available): (scale, wc [C, 27], bc [C], wt [S*S, C],
    bt [S*S]), fp32, N(0, 1/27) and N(0, 1/C) entries, small biases."""
    rng = np.random.default_rng(seed)
    S, Cf = scale, features
    wc = (rng.standard_normal((Cf, 27)) / np.sqrt(27.0)).astype(np.float32)
    bc = (0.01 * rng.standard_normal(Cf)).astype(np.float32)
    wt = (rng.standard_normal((S * S, Cf)) / np.sqrt(Cf)).astype(np.float32)
    bt = (0.01 * rng.standard_normal(S * S)).astype(np.float32)
    return S, wc, bc, wt, bt
