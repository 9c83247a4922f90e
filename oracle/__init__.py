"""CPU FP64 oracle of the 3DGS^3 low-resolution render (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may
import this package. The product path (``paper_2605_11489_gb300``) never does,
and the two share no code: the only common module is the seeded input generator
``paper_2605_11489_gb300.synth``, which holds none of the render arithmetic.

The C source (``oracle.c``) is a plain, per-pixel, untiled reference renderer:
FP64 continuous math, plus an fp32 round-to-nearest sequence for the discrete
decisions (depth key, support rectangle). It also holds the frame-interpolation
geometry of Sec. 4.2 (camera motion vectors, the depth-tested forward warp and the
warped gradient), with the target pixel and the depth test decided by an fp32
sequence in the same way. Every function here is a thin ctypes wrapper around it.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "oracle.c")
_LIB_PATH = os.path.join(_HERE, "liboracle.so")
_lock = threading.Lock()
_lib = None

CFLAGS = ["-O2", "-std=c11", "-fopenmp", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared"]


def build(force: bool = False) -> str:
    """Compile oracle.c into liboracle.so next to it (gcc, OpenMP, no FP contraction)."""
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + ".tmp%d" % os.getpid()
        subprocess.run(["gcc", *CFLAGS, _SRC, "-o", tmp, "-lm"], check=True)
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


class _Scene(C.Structure):
    _fields_ = [("n", C.c_int64), ("stride", C.c_int64), ("deg", C.c_int32), ("_pad", C.c_int32),
                ("means", C.c_void_p), ("log_scales", C.c_void_p), ("quats", C.c_void_p),
                ("logits", C.c_void_p), ("sh", C.c_void_p)]


class _Camera(C.Structure):
    _fields_ = [("viewmat", C.c_double * 12), ("fx", C.c_double), ("fy", C.c_double),
                ("cx", C.c_double), ("cy", C.c_double), ("near_plane", C.c_double),
                ("width", C.c_int32), ("height", C.c_int32), ("bg", C.c_double * 3)]


def lib():
    global _lib
    with _lock:
        if _lib is None:
            build()
            L = C.CDLL(_LIB_PATH)
            P = C.c_void_p
            L.or_spec_exp.restype = C.c_float
            L.or_spec_exp.argtypes = [C.c_float]
            L.or_spec_log.restype = C.c_float
            L.or_spec_log.argtypes = [C.c_float]
            L.or_sh_basis.argtypes = [C.c_int, P, P, P]
            L.or_cov3d.argtypes = [P, P, P, P]
            L.or_project.argtypes = [P, P, C.c_int32] + [P] * 10
            L.or_render.argtypes = [P, P, C.c_int] + [P] * 10
            L.or_render_pixels.argtypes = [P, P, C.c_int64, P, P, P, P, P, P]
            L.or_render_band.argtypes = [P, P, C.c_int, C.c_int, P, P, P, P, P]
            L.or_render_normals.argtypes = [P, P, P, P, P, P, P, P]
            L.or_count_instances.restype = C.c_int64
            L.or_count_instances.argtypes = [P, P, C.c_int32]
            L.or_keys.argtypes = [P, P, C.c_int32, C.c_int64, P, P, P]
            L.or_backward.argtypes = [P, P] + [P] * 11
            L.or_warp.argtypes = [P, P, P, P, C.c_double, C.c_int32, P, C.c_int32] + [P] * 10
            L.or_warp.restype = C.c_int
            L.or_max_threads.restype = C.c_int
            L.or_set_threads.argtypes = [C.c_int]
            _lib = L
    return _lib


def _ptr(a):
    return None if a is None else a.ctypes.data


class OScene:
    """FP64 copy of a ``synth.SceneArrays`` (the fp32 values promoted exactly)."""

    def __init__(self, s):
        self.n, self.deg = s.n, s.deg
        self.stride = s.n_pad
        self.means = np.ascontiguousarray(s.means, dtype=np.float64)
        self.log_scales = np.ascontiguousarray(s.log_scales, dtype=np.float64)
        self.quats = np.ascontiguousarray(s.quats, dtype=np.float64)
        self.logits = np.ascontiguousarray(s.logits, dtype=np.float64)
        self.sh = np.ascontiguousarray(s.sh, dtype=np.float64)

    def struct(self):
        return _Scene(self.n, self.stride, self.deg, 0, _ptr(self.means), _ptr(self.log_scales),
                      _ptr(self.quats), _ptr(self.logits), _ptr(self.sh))


def _as_oscene(s):
    return s if isinstance(s, OScene) else OScene(s)


def _cam(cam, bg=(0.0, 0.0, 0.0)):
    c = _Camera()
    for k in range(12):
        c.viewmat[k] = float(cam.viewmat[k])
    c.fx, c.fy, c.cx, c.cy = float(cam.fx), float(cam.fy), float(cam.cx), float(cam.cy)
    c.near_plane = float(cam.near)
    c.width, c.height = int(cam.width), int(cam.height)
    for k in range(3):
        c.bg[k] = float(bg[k])
    return c


def spec_exp(x: float) -> float:
    return lib().or_spec_exp(float(x))


def spec_log(x: float) -> float:
    return lib().or_spec_log(float(x))


def sh_basis(deg: int, d) -> tuple[np.ndarray, np.ndarray]:
    d = np.ascontiguousarray(d, dtype=np.float64)
    k = (deg + 1) ** 2
    y = np.zeros(k)
    dy = np.zeros((k, 3))
    lib().or_sh_basis(deg, _ptr(d), _ptr(y), _ptr(dy))
    return y, dy


def cov3d(s, q):
    s = np.ascontiguousarray(s, dtype=np.float64)
    q = np.ascontiguousarray(q, dtype=np.float64)
    sig = np.zeros(9)
    R = np.zeros(9)
    lib().or_cov3d(_ptr(s), _ptr(q), _ptr(sig), _ptr(R))
    return sig.reshape(3, 3), R.reshape(3, 3)


def project(scene, cam, tile: int = 16) -> dict:
    """Per-Gaussian projection: discrete fields (visible, z32, rect, ntiles) and
    FP64 continuous fields (uv, conic, opacity, rgb, depth, cov2d)."""
    s = _as_oscene(scene)
    n = s.n
    out = dict(visible=np.zeros(n, np.int32), z32=np.zeros(n, np.float32), rect=np.zeros((n, 4), np.int32),
               ntiles=np.zeros(n, np.int32), uv=np.zeros((n, 2)), conic=np.zeros((n, 3)),
               opacity=np.zeros(n), rgb=np.zeros((n, 3)), depth=np.zeros(n), cov2d=np.zeros((n, 3)))
    st, cm = s.struct(), _cam(cam)
    lib().or_project(C.byref(st), C.byref(cm), tile, *[_ptr(out[k]) for k in
                     ("visible", "z32", "rect", "ntiles", "uv", "conic", "opacity", "rgb", "depth", "cov2d")])
    return out


def render(scene, cam, bg=(0.0, 0.0, 0.0), mode: str = "binned") -> dict:
    """Full-frame FP64 render. Returns planar rgb/dcdx/dcdy [3,H,W], depth,
    alpha, final_T [H,W], n_blended [H,W], the per-pixel decision signature, and
    `amb`: 1 where a discrete decision (alpha cap 0.99, cut 1/255, stop at
    T < 1e-4) lies within 1e-5 relative of its threshold, so that fp32
    rounding elsewhere may decide it the other way."""
    s = _as_oscene(scene)
    H, W = cam.height, cam.width
    out = dict(rgb=np.zeros((3, H, W)), dcdx=np.zeros((3, H, W)), dcdy=np.zeros((3, H, W)),
               depth=np.zeros((H, W)), alpha=np.zeros((H, W)), final_T=np.zeros((H, W)),
               n_blended=np.zeros((H, W), np.int32), sig=np.zeros((H, W), np.uint32),
               amb=np.zeros((H, W), np.int32), gabs=np.zeros((2, 3, H, W)))
    st, cm = s.struct(), _cam(cam, bg)
    rc = lib().or_render(C.byref(st), C.byref(cm), 1 if mode == "binned" else 0,
                         *[_ptr(out[k]) for k in ("rgb", "dcdx", "dcdy", "depth", "alpha", "final_T",
                                                  "n_blended", "sig", "amb", "gabs")])
    if rc != 0:
        raise RuntimeError("or_render failed: %d" % rc)
    return out


def render_normals(scene, cam) -> dict:
    """The normal channel and the normal-view map (binned FP64 render).
    - normal [3, H, W]: the camera-space normals of the blended Gaussians, weighted like the
      colour (sum n_i a_i T_i). n_i is the axis of the Gaussian's smallest scale, turned to face
      the camera: the normal RaDe-GS renders, which the paper uses for its depth and normal
      maps (Sec. 5.1).
    - nv [H, W]: -normal . (unit ray of the pixel centre), the normal-view inner product map
      of Sec. 4.1.
    - alpha [H, W].
    - nrm_amb [H, W]: 1 where a blended Gaussian's axis is within 1e-5 of perpendicular to its
      view direction, so that rounding may turn its normal either way.
    - amb [H, W]: the render's decision flag.
    - depth_isect [H, W]: RaDe-GS's ray-Gaussian intersection depth, sum z_i(p) a_i T_i. z_i(p)
      is the densest point of Gaussian i along the ray of pixel p in the EWA ray space (u, v,
      camera z) of the projection: the mean of z given (u, v) = p, affine in p,
      z_i(p) = z_i + Sigma_{z,uv} (Sigma2D + 0.3 I)^-1 (p - mu2D_i)."""
    s = _as_oscene(scene)
    H, W = cam.height, cam.width
    out = dict(normal=np.zeros((3, H, W)), nv=np.zeros((H, W)), alpha=np.zeros((H, W)),
               nrm_amb=np.zeros((H, W), np.int32), amb=np.zeros((H, W), np.int32), depth_isect=np.zeros((H, W)))
    st, cm = s.struct(), _cam(cam, (0.0, 0.0, 0.0))
    rc = lib().or_render_normals(C.byref(st), C.byref(cm),
                                 *[_ptr(out[k]) for k in ("normal", "nv", "alpha", "nrm_amb", "amb", "depth_isect")])
    if rc != 0:
        raise RuntimeError("or_render_normals failed: %d" % rc)
    return out


def render_band(scene, cam, y0: int, y1: int, bg=(0.0, 0.0, 0.0)) -> dict:
    """Binned FP64 render of rows [y0, y1) (rest of the planes left at zero)."""
    s = _as_oscene(scene)
    H, W = cam.height, cam.width
    out = dict(rgb=np.zeros((3, H, W)), dcdx=np.zeros((3, H, W)), dcdy=np.zeros((3, H, W)),
               depth=np.zeros((H, W)), alpha=np.zeros((H, W)))
    st, cm = s.struct(), _cam(cam, bg)
    rc = lib().or_render_band(C.byref(st), C.byref(cm), int(y0), int(y1),
                              *[_ptr(out[k]) for k in ("rgb", "dcdx", "dcdy", "depth", "alpha")])
    if rc != 0:
        raise RuntimeError("or_render_band failed: %d" % rc)
    return out


def render_pixels(scene, cam, px, py, bg=(0.0, 0.0, 0.0)) -> dict:
    """Brute-force render of sampled pixels (each pixel scans every visible
    Gaussian). Returns per sample: rgb/dcdx/dcdy [n, 3], depth/alpha [n],
    n_blended, amb and gabs [n, 2, 3] (as in render())."""
    s = _as_oscene(scene)
    px = np.ascontiguousarray(px, dtype=np.int32)
    py = np.ascontiguousarray(py, dtype=np.int32)
    n = len(px)
    out = np.zeros((n, 11))
    nb = np.zeros(n, np.int32)
    amb = np.zeros(n, np.int32)
    gabs = np.zeros((n, 2, 3))
    st, cm = s.struct(), _cam(cam, bg)
    rc = lib().or_render_pixels(C.byref(st), C.byref(cm), n, _ptr(px), _ptr(py), _ptr(out), _ptr(nb), _ptr(amb),
                                _ptr(gabs))
    if rc != 0:
        raise RuntimeError("or_render_pixels failed: %d" % rc)
    return dict(rgb=out[:, 0:3], dcdx=out[:, 3:6], dcdy=out[:, 6:9], depth=out[:, 9], alpha=out[:, 10],
                n_blended=nb, amb=amb, gabs=gabs)


def keys(scene, cam, tile: int = 16) -> dict:
    """Sorted (tile, depth) instance list: keys u64, vals u32, ranges [n_tiles, 2]."""
    s = _as_oscene(scene)
    st, cm = s.struct(), _cam(cam)
    L = lib()
    K = L.or_count_instances(C.byref(st), C.byref(cm), tile)
    tw = (cam.width + tile - 1) // tile
    th = (cam.height + tile - 1) // tile
    k = np.zeros(max(K, 1), np.uint64)
    v = np.zeros(max(K, 1), np.uint32)
    r = np.zeros((tw * th, 2), np.uint32)
    rc = L.or_keys(C.byref(st), C.byref(cm), tile, K, _ptr(k), _ptr(v), _ptr(r))
    if rc != 0:
        raise RuntimeError("or_keys failed: %d" % rc)
    return dict(keys=k[:K], vals=v[:K], ranges=r, n_tiles=tw * th)


def backward(scene, cam, g_rgb=None, g_dcdx=None, g_dcdy=None, g_depth=None, g_alpha=None,
             bg=(0.0, 0.0, 0.0)) -> dict:
    """FP64 adjoint of L = sum <g_*, output_*>. Returns planar grads shaped like the
    scene's planes (means [3,n_pad], log_scales, quats, logits, sh) and the 2D
    adjoints g2d [n, 10] = (u, v, conic a, b, c, opacity, depth, r, g, b)."""
    s = _as_oscene(scene)
    S = s.stride
    f64 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    ups = [f64(g_rgb), f64(g_dcdx), f64(g_dcdy), f64(g_depth), f64(g_alpha)]
    out = dict(means=np.zeros((3, S)), log_scales=np.zeros((3, S)), quats=np.zeros((4, S)),
               logits=np.zeros(S), sh=np.zeros(((s.deg + 1) ** 2, 3, S)), g2d=np.zeros((s.n, 10)))
    st, cm = s.struct(), _cam(cam, bg)
    rc = lib().or_backward(C.byref(st), C.byref(cm), *[_ptr(a) for a in ups],
                           *[_ptr(out[k]) for k in ("means", "log_scales", "quats", "logits", "sh", "g2d")])
    if rc != 0:
        raise RuntimeError("or_backward failed: %d" % rc)
    return out


def warp(src_cam, dst_cam, depth, alpha=None, alpha_min=0.0, planes=None, dcdx=None, dcdy=None) -> dict:
    """Frame-interpolation geometry of Sec. 4.2 for one source frame (oracle.c, or_warp).

    depth, alpha: [H, W] of the source frame (alpha None: depth is a point depth).
    planes: [C, H, W] carried by the forward warp; dcdx, dcdy: [G, H, W] source image
    gradients. Returns motion [2, H, W] (fp32 spec, NaN where a pixel does not move),
    motion64 (the same map in FP64), index [Ht, Wt] (winning source pixel, -1 = hole),
    z [Ht, Wt] (winner's target-camera z, fp32 spec), out [C, Ht, Wt], out_dcdx/out_dcdy
    [G, Ht, Wt] (the warped gradient w(G, V) . dx/dy), jac [4, Ht, Wt] (the Jacobian
    J = [[du/dx, du/dy], [dv/dx, dv/dy]] of the landing map used at each target pixel,
    row-major entries; the identity at holes)."""
    W, H, Wt, Ht = src_cam.width, src_cam.height, dst_cam.width, dst_cam.height
    f64 = lambda a: None if a is None else np.ascontiguousarray(a, dtype=np.float64)
    depth, alpha = f64(depth), f64(alpha)
    assert depth.shape == (H, W) and (alpha is None or alpha.shape == (H, W))
    planes = f64(planes) if planes is not None else np.zeros((0, H, W))
    C_ = planes.shape[0]
    G = 0 if dcdx is None else int(np.shape(dcdx)[0])
    dcdx = f64(dcdx) if G else None
    dcdy = f64(dcdy) if G else None
    res = dict(motion=np.zeros((2, H, W), np.float32), motion64=np.zeros((2, H, W)),
               index=np.zeros((Ht, Wt), np.int32), z=np.zeros((Ht, Wt), np.float32),
               out=np.zeros((C_, Ht, Wt)), out_dcdx=np.zeros((G, Ht, Wt)), out_dcdy=np.zeros((G, Ht, Wt)),
               jac=np.zeros((4, Ht, Wt)))
    sc, dc = _cam(src_cam), _cam(dst_cam)
    rc = lib().or_warp(C.byref(sc), C.byref(dc), _ptr(depth), _ptr(alpha), float(alpha_min), C_, _ptr(planes), G,
                       _ptr(dcdx), _ptr(dcdy), *[_ptr(res[k]) for k in
                       ("motion", "motion64", "index", "z", "out", "out_dcdx", "out_dcdy", "jac")])
    if rc != 0:
        raise MemoryError("or_warp: allocation failed")
    return res


def max_threads() -> int:
    return lib().or_max_threads()


def set_threads(n: int) -> None:
    lib().or_set_threads(int(n))
