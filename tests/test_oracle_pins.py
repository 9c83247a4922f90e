"""Pins of the CPU oracle against what the paper and mathematics fix.

Each test checks the oracle against something other than itself: a closed
form, a library routine on the same mathematical object, finite differences of
the continuous image (the gradient channels are exact derivatives of the
continuous signal, Sec. 3 "3DGS Image Gradients"), or an invariant of Eq. 2.
"""
import math

import numpy as np
import pytest

from paper_2605_11489_gb300 import synth

pytestmark = pytest.mark.usefixtures("oracle_lib")

OUT_KEYS = ("rgb", "dcdx", "dcdy", "depth", "alpha")


# ----------------------------------------------------------------------------- spec exp/log

def test_spec_exp_error_bound(oracle_lib):
    O = oracle_lib
    xs = np.concatenate([np.linspace(-87, 88, 20001), np.linspace(-1, 1, 4001)]).astype(np.float32)
    got = np.array([O.spec_exp(x) for x in xs], dtype=np.float64)
    ref = np.exp(xs.astype(np.float64))
    rel = np.abs(got - ref) / ref
    # a few ULP of fp32 (2^-23 = 1.19e-7) away from the subnormal range
    assert rel[ref > 1e-37].max() < 4e-7


def test_spec_log_error_bound(oracle_lib):
    O = oracle_lib
    xs = np.concatenate([np.linspace(1.0, 255.0, 20001), np.geomspace(1e-30, 1e30, 4001)]).astype(np.float32)
    got = np.array([O.spec_log(x) for x in xs], dtype=np.float64)
    ref = np.log(xs.astype(np.float64))
    err = np.abs(got - ref) / np.maximum(np.abs(ref), 1.0)
    assert err.max() < 4e-7
    assert O.spec_log(1.0) == 0.0


# ----------------------------------------------------------------------------- SH

def _real_sh_scipy(l, m, theta, phi):
    """Real SH with the Condon-Shortley phase from scipy's complex Y_l^m."""
    import scipy.special as sp

    if hasattr(sp, "sph_harm_y"):
        Y = lambda mm: sp.sph_harm_y(l, mm, theta, phi)
    else:  # older scipy: sph_harm(m, n, azimuth, polar)
        Y = lambda mm: sp.sph_harm(mm, l, phi, theta)
    if m > 0:
        return math.sqrt(2.0) * np.real(Y(m))
    if m < 0:
        return math.sqrt(2.0) * np.imag(Y(-m))
    return np.real(Y(0))


def _sphere_quadrature(nt=24, nphi=48):
    x, w = np.polynomial.legendre.leggauss(nt)  # cos(theta) nodes
    phi = (np.arange(nphi) + 0.5) * 2 * math.pi / nphi
    ct, ph = np.meshgrid(x, phi, indexing="ij")
    wt = np.repeat(w[:, None], nphi, axis=1) * (2 * math.pi / nphi)
    st = np.sqrt(1 - ct ** 2)
    dirs = np.stack([st * np.cos(ph), st * np.sin(ph), ct], axis=-1).reshape(-1, 3)
    return dirs, wt.reshape(-1), np.arccos(ct).reshape(-1), ph.reshape(-1)


def test_sh_orthonormal_by_quadrature(oracle_lib):
    O = oracle_lib
    dirs, w, _, _ = _sphere_quadrature()
    Y = np.stack([O.sh_basis(3, d)[0] for d in dirs])  # [P, 16]
    G = (Y * w[:, None]).T @ Y
    assert np.abs(G - np.eye(16)).max() < 1e-12


def test_sh_matches_scipy_complex_harmonics(oracle_lib):
    O = oracle_lib
    dirs, _, th, ph = _sphere_quadrature(7, 11)
    Y = np.stack([O.sh_basis(3, d)[0] for d in dirs])
    k = 0
    for l in range(4):
        for m in range(-l, l + 1):
            ref = _real_sh_scipy(l, m, th, ph)
            assert np.abs(Y[:, k] - ref).max() < 1e-12, (l, m)
            k += 1


def test_sh_degree0_constant_and_gradient_fd(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(11)
    for _ in range(20):
        d = rng.normal(size=3)
        y0, _ = O.sh_basis(0, d / np.linalg.norm(d))
        assert y0[0] == pytest.approx(0.5 / math.sqrt(math.pi), abs=1e-15)
        y, dy = O.sh_basis(3, d)
        h = 1e-6
        for a in range(3):
            e = np.zeros(3)
            e[a] = h
            fd = (O.sh_basis(3, d + e)[0] - O.sh_basis(3, d - e)[0]) / (2 * h)
            assert np.abs(fd - dy[:, a]).max() < 1e-7


# ----------------------------------------------------------------------------- covariance

def test_cov3d_eigen_structure(oracle_lib):
    O = oracle_lib
    rng = np.random.default_rng(3)
    for _ in range(50):
        s = np.exp(rng.normal(-1, 1, 3))
        q = rng.normal(size=4) * rng.uniform(0.1, 5.0)
        Sig, R = O.cov3d(s, q)
        assert np.abs(Sig - Sig.T).max() < 1e-14 * Sig.max()
        assert np.abs(R @ R.T - np.eye(3)).max() < 1e-13
        assert np.linalg.det(R) == pytest.approx(1.0, abs=1e-12)
        # columns of R are eigenvectors with eigenvalues s^2
        for k in range(3):
            v = R[:, k]
            assert np.abs(Sig @ v - s[k] ** 2 * v).max() < 1e-12 * max(1.0, s.max() ** 2)
        ev = np.sort(np.linalg.eigvalsh(Sig))
        assert np.allclose(ev, np.sort(s ** 2), rtol=1e-10, atol=1e-14)


# ----------------------------------------------------------------------------- closed forms

def _single_scene(log_s, logit, dc, z_world=0.0, deg=0):
    s = synth.empty_scene(1, deg)
    s.means[:, 0] = (0.0, 0.0, z_world)
    s.log_scales[:, 0] = log_s
    s.quats[:, 0] = (0.3, -0.5, 0.7, 0.2)  # any rotation: the Gaussian is isotropic
    s.logits[0] = logit
    s.sh[0, :, 0] = dc
    return s


@pytest.mark.parametrize("log_s,logit", [(-3.0, 0.5), (-2.0, 3.0), (-4.5, -1.0), (-1.5, 6.0)])
def test_single_isotropic_gaussian_closed_form(oracle_lib, log_s, logit):
    """One isotropic Gaussian on the optical axis: Sigma2D = ((f s / z)^2 + 0.3) I,
    alpha(p) = min(0.99, o exp(-|p - c|^2 / (2 sigma^2))), rgb = col alpha,
    dC/dx = -col alpha (x - cx) / sigma^2 (0 where capped), depth = z alpha."""
    O = oracle_lib
    cam = synth.tiny_camera(96, 64)
    dc = np.array([1.2, -0.4, 0.1])
    sc = _single_scene(np.float32(log_s), np.float32(logit), dc.astype(np.float32))
    out = O.render(sc, cam, mode="brute")
    s = math.exp(float(np.float32(log_s)))
    o = 1.0 / (1.0 + math.exp(-float(np.float32(logit))))
    z = 4.0
    sig2 = (cam.fx * s / z) ** 2 + 0.3
    col = np.maximum(dc.astype(np.float32).astype(np.float64) * (0.5 / math.sqrt(math.pi)) + 0.5, 0.0)
    X, Y = np.meshgrid(np.arange(cam.width) + 0.5, np.arange(cam.height) + 0.5)
    dx, dy = X - cam.cx, Y - cam.cy
    raw = o * np.exp(-(dx ** 2 + dy ** 2) / (2 * sig2))
    capped = raw > 0.99
    a = np.where(capped, 0.99, raw)
    live = a >= 1.0 / 255.0
    # an opaque single Gaussian would stop compositing only if T(1-a) < 1e-4: not reachable with a <= 0.99
    ax = np.where(capped, 0.0, -a * dx / sig2)
    ay = np.where(capped, 0.0, -a * dy / sig2)
    exp = dict(rgb=col[:, None, None] * a * live, dcdx=col[:, None, None] * ax * live,
               dcdy=col[:, None, None] * ay * live, depth=z * a * live, alpha=a * live)
    amb = np.abs(raw - 1.0 / 255.0) < 1e-6  # the alpha cut itself
    for k in OUT_KEYS:
        got, ref = out[k], exp[k]
        m = ~amb if got.ndim == 2 else np.broadcast_to(~amb, got.shape)
        assert np.abs(got - ref)[m].max() < 1e-12, k
    assert (out["n_blended"][~amb] == live[~amb]).all()


def test_two_gaussians_on_axis_closed_form(oracle_lib):
    """Two isotropic Gaussians on the axis at z = 3.5 (front) and 4.5 (back):
    I = c1 a1 + c2 a2 (1 - a1); its x-derivative by the product rule,
    I' = c1 a1' + c2 (a2' (1 - a1) - a2 a1'), independently of the Eq. 4 recursion."""
    O = oracle_lib
    cam = synth.tiny_camera(80, 48)
    s = synth.empty_scene(2, 0)
    s.means[:, 0] = (0.0, 0.0, -0.5)   # back (camera at z = 4 looking at -z)
    s.means[:, 1] = (0.0, 0.0, 0.5)    # front
    s.log_scales[:, 0] = np.float32(-2.6)
    s.log_scales[:, 1] = np.float32(-3.1)
    s.quats[0, :2] = 1.0
    s.logits[0] = np.float32(1.5)
    s.logits[1] = np.float32(0.3)
    s.sh[0, :, 0] = np.float32([0.9, 0.1, -0.7])
    s.sh[0, :, 1] = np.float32([-0.2, 1.1, 0.4])
    bg = (0.25, 0.5, 0.75)
    out = O.render(s, cam, bg=bg, mode="brute")
    X, Y = np.meshgrid(np.arange(cam.width) + 0.5, np.arange(cam.height) + 0.5)
    dx, dy = X - cam.cx, Y - cam.cy

    def gauss(i, z):
        sc = math.exp(float(s.log_scales[0, i]))
        o = 1.0 / (1.0 + math.exp(-float(s.logits[i])))
        sig2 = (cam.fx * sc / z) ** 2 + 0.3
        a = o * np.exp(-(dx ** 2 + dy ** 2) / (2 * sig2))
        assert a.max() < 0.99
        keep = a >= 1 / 255
        a = a * keep
        return a, -a * dx / sig2, -a * dy / sig2, keep, np.abs(a - 1 / 255) < 1e-6
    a1, a1x, a1y, k1, m1 = gauss(1, 3.5)
    a2, a2x, a2y, k2, m2 = gauss(0, 4.5)
    col = lambda i: s.sh[0, :, i].astype(np.float64) * (0.5 / math.sqrt(math.pi)) + 0.5
    c1, c2 = col(1)[:, None, None], col(0)[:, None, None]
    bgv = np.array(bg)[:, None, None]
    T = (1 - a1) * (1 - a2)
    Tx = -a1x * (1 - a2) - (1 - a1) * a2x
    Ty = -a1y * (1 - a2) - (1 - a1) * a2y
    ref = dict(rgb=c1 * a1 + c2 * a2 * (1 - a1) + bgv * T,
               dcdx=c1 * a1x + c2 * (a2x * (1 - a1) - a2 * a1x) + bgv * Tx,
               dcdy=c1 * a1y + c2 * (a2y * (1 - a1) - a2 * a1y) + bgv * Ty,
               depth=3.5 * a1 + 4.5 * a2 * (1 - a1), alpha=1 - T)
    ok = ~(m1 | m2)
    for k in OUT_KEYS:
        m = ok if out[k].ndim == 2 else np.broadcast_to(ok, out[k].shape)
        assert np.abs(out[k] - ref[k])[m].max() < 1e-12, k


# ----------------------------------------------------------------------------- FD of the continuous image

def _fd_grad_check(O, scene, cam, bg, h=1e-4):
    base = O.render(scene, cam, bg=bg)
    res = {}
    for axis, key in ((0, "dcdx"), (1, "dcdy")):
        dcx, dcy = (h, 0.0) if axis == 0 else (0.0, h)
        p = O.render(scene, cam.shifted(dcx, dcy), bg=bg)
        m = O.render(scene, cam.shifted(-dcx, -dcy), bg=bg)
        # shifting the principal point by +h moves the image content by +h, so
        # dI/dx = -(I(c + h) - I(c - h)) / (2h)
        fd = -(p["rgb"] - m["rgb"]) / (2 * h)
        same = (p["sig"] == base["sig"]) & (m["sig"] == base["sig"])
        err = np.abs(fd - base[key])[:, same]
        scale = np.abs(base[key]).max()
        res[key] = (err.max() / scale, same.mean())
    return res


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.2, 0.5, 0.9)])
def test_gradient_channels_match_fd_of_image(oracle_lib, bg):
    O = oracle_lib
    sc = synth.tiny_scene()
    cam = synth.tiny_camera()
    res = _fd_grad_check(O, sc, cam, bg)
    for key, (rel, frac) in res.items():
        assert frac > 0.99, key
        assert rel < 1e-6, (key, rel)


def test_gradient_channels_fd_deg3_scene(oracle_lib):
    O = oracle_lib
    sc = _deg3_scene(300, seed=21)
    cam = synth.tiny_camera(128, 72)
    for key, (rel, frac) in _fd_grad_check(O, sc, cam, (0.1, 0.0, 0.3)).items():
        assert frac > 0.98 and rel < 1e-6, (key, rel, frac)


# ----------------------------------------------------------------------------- invariants

def test_brute_equals_binned_bitwise(oracle_lib):
    O = oracle_lib
    for n, seed in ((512, 5), (4096, 0)):
        sc = synth.tiny_scene(n, seed)
        cam = synth.jittered_tiny_cameras(2, seed)[1]
        a = O.render(sc, cam, mode="brute")
        b = O.render(sc, cam, mode="binned")
        for k in a:
            assert np.array_equal(a[k], b[k]), k


def test_sampled_pixels_and_bands_equal_the_brute_force_image(oracle_lib):
    """render_pixels (each sample scans every visible Gaussian, used for the
    full-size samples) and render_band (the timed CPU baseline's unit) give the
    brute-force image's values at those pixels / rows, bit for bit."""
    O = oracle_lib
    sc = synth.tiny_scene(2048, 7)
    cam = synth.jittered_tiny_cameras(3, 7)[2]
    bg = (0.1, 0.3, 0.2)
    full = O.render(sc, cam, bg=bg, mode="brute")
    rng = np.random.default_rng(1)
    px = rng.integers(0, cam.width, 300)
    py = rng.integers(0, cam.height, 300)
    s = O.render_pixels(sc, cam, px, py, bg=bg)
    for k in OUT_KEYS:
        ref = full[k][:, py, px].T if full[k].ndim == 3 else full[k][py, px]
        assert np.array_equal(s[k], ref), k
    assert np.array_equal(s["amb"], full["amb"][py, px])
    y0, y1 = 37, 61
    band = O.render_band(sc, cam, y0, y1, bg=bg)
    for k in OUT_KEYS:
        assert np.array_equal(band[k][..., y0:y1, :], full[k][..., y0:y1, :]), k
        assert not band[k][..., :y0, :].any() and not band[k][..., y1:, :].any(), k


def test_blend_weights_sum_to_alpha(oracle_lib):
    """With every colour 1 and bg 0, Eq. 2 gives I = sum a_i T_i = 1 - T_final."""
    O = oracle_lib
    sc = synth.tiny_scene()
    sc.sh[0, :, :] = np.float32(math.sqrt(math.pi))  # colour 1 up to the fp32 rounding of sqrt(pi)
    col = float(np.float32(math.sqrt(math.pi))) * (0.5 / math.sqrt(math.pi)) + 0.5
    out = O.render(sc, synth.tiny_camera())
    for c in range(3):
        assert np.abs(out["rgb"][c] - col * out["alpha"]).max() < 1e-12
    assert (out["alpha"] >= 0).all() and (out["alpha"] < 1).all()
    assert np.allclose(out["alpha"], 1 - out["final_T"], atol=1e-15)
    # transmittance never drops below the termination threshold times (1 - 0.99)
    assert out["final_T"].min() >= 1e-4 * 0.01 - 1e-18


def test_permutation_invariance(oracle_lib):
    O = oracle_lib
    cam = synth.tiny_camera()
    full = synth.tiny_scene()
    z = O.project(full, cam)["z32"]
    # drop every Gaussian that shares its fp32 depth with another: with exact
    # ties the (depth, index) order depends on the input order by definition
    _, inv, cnt = np.unique(z, return_inverse=True, return_counts=True)
    sc = full.subset(np.nonzero(cnt[inv] == 1)[0])
    assert sc.n >= full.n - 8
    perm = np.random.default_rng(9).permutation(sc.n)
    a = O.render(sc, cam)
    b = O.render(sc.subset(perm), cam)
    for k in OUT_KEYS:
        assert np.array_equal(a[k], b[k]), k


def test_integer_principal_point_shift_translates_image(oracle_lib):
    O = oracle_lib
    sc = synth.tiny_scene()
    cam = synth.tiny_camera()
    k = 7
    a = O.render(sc, cam)
    b = O.render(sc, cam.shifted(float(k), 0.0))
    same = a["sig"][:, : -k] == b["sig"][:, k:]
    assert same.mean() > 0.999
    for key in OUT_KEYS:
        x, y = a[key][..., : -k], b[key][..., k:]
        m = same if x.ndim == 2 else np.broadcast_to(same, x.shape)
        assert np.abs(x - y)[m].max() < 1e-9, key


def test_alpha_bounds_of_contributors_and_cut(oracle_lib):
    """Every blended alpha is in [1/255, 0.99]: a pixel with exactly one contributor
    has alpha in that range, and pixels with none are exactly background."""
    O = oracle_lib
    sc = synth.tiny_scene()
    out = O.render(sc, synth.tiny_camera(), bg=(0.3, 0.3, 0.3))
    one = out["n_blended"] == 1
    assert one.any()
    assert (out["alpha"][one] >= 1 / 255 - 1e-15).all() and (out["alpha"][one] <= 0.99 + 1e-15).all()
    none = out["n_blended"] == 0
    assert (out["alpha"][none] == 0).all()
    assert (out["rgb"][:, none] == 0.3).all()


# ----------------------------------------------------------------------------- keys

def test_keys_match_library_stable_sort(oracle_lib):
    """The sorted (tile, depth) instance list equals numpy's stable lexsort of the
    index-ordered instances built from the projection's rectangles."""
    O = oracle_lib
    sc = synth.tiny_scene()
    for tile in (8, 16, 32):
        for cam in synth.jittered_tiny_cameras(3, 4):
            p = O.project(sc, cam, tile)
            tw = (cam.width + tile - 1) // tile
            ks, vs = [], []
            for i in np.nonzero(p["visible"])[0]:
                x0, y0, x1, y1 = p["rect"][i]
                zb = np.uint64(p["z32"][i:i + 1].view(np.uint32)[0])
                for ty in range(y0 // tile, y1 // tile + 1):
                    for tx in range(x0 // tile, x1 // tile + 1):
                        ks.append((np.uint64(ty * tw + tx) << np.uint64(32)) | zb)
                        vs.append(i)
            ks = np.array(ks, dtype=np.uint64)
            vs = np.array(vs, dtype=np.uint32)
            order = np.argsort(ks, kind="stable")
            got = O.keys(sc, cam, tile)
            assert np.array_equal(got["keys"], ks[order])
            assert np.array_equal(got["vals"], vs[order])
            assert p["ntiles"].sum() == len(ks)
            t = (got["keys"] >> np.uint64(32)).astype(np.int64)
            for tid in range(got["n_tiles"]):
                s0, s1 = got["ranges"][tid]
                assert (t[s0:s1] == tid).all() and (s1 - s0) == (t == tid).sum()


# ----------------------------------------------------------------------------- backward

def _deg3_scene(n, seed, extra_offscreen=True):
    rng = np.random.default_rng(seed)
    s = synth.empty_scene(n, 3)
    s.means[:, :n] = rng.uniform(-1, 1, (3, n))
    s.log_scales[:, :n] = rng.normal(-3.2, 0.5, (3, n))
    s.quats[:, :n] = rng.normal(size=(4, n))
    s.logits[:n] = rng.normal(0.5, 1.5, n)
    s.sh[0, :, :n] = rng.uniform(-1.7, 1.7, (3, n))
    s.sh[1:, :, :n] = rng.normal(0, 0.2, (15, 3, n))
    if extra_offscreen:
        # two large Gaussians whose centres are beyond the Jacobian guard limit
        for j, sx in ((0, 1.0), (1, -1.0)):
            s.means[:, j] = (sx * 9.0, 0.2, 0.0)
            s.log_scales[:, j] = (1.2, 0.9, 1.0)
            s.logits[j] = 2.0
    return s


def _loss(O, sc, cam, ups, bg):
    out = O.render(sc, cam, bg=bg)
    L = sum(float((ups[k] * out[k]).sum()) for k in ups)
    return L, out["sig"]


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.3, 0.6, 0.1)])
def test_backward_matches_central_fd(oracle_lib, bg):
    O = oracle_lib
    cam = synth.tiny_camera(64, 40)
    sc = _deg3_scene(160, seed=31)
    osc = O.OScene(sc)
    rng = np.random.default_rng(2)
    ups = {k: rng.standard_normal((3, cam.height, cam.width)) for k in ("rgb", "dcdx", "dcdy")}
    ups["depth"] = rng.standard_normal((cam.height, cam.width))
    ups["alpha"] = rng.standard_normal((cam.height, cam.width))
    g = O.backward(osc, cam, ups["rgb"], ups["dcdx"], ups["dcdy"], ups["depth"], ups["alpha"], bg=bg)
    _, sig0 = _loss(O, osc, cam, ups, bg)
    vis = np.nonzero(O.project(osc, cam)["visible"])[0]
    assert 0 in vis  # the off-screen guard-clamped Gaussian is in view
    checked = 0
    worst = 0.0
    planes = [("means", 3), ("log_scales", 3), ("quats", 4), ("logits", 1), ("sh", 48)]
    picks = list(vis[:2]) + list(rng.choice(vis, 14, replace=False))
    for i in picks:
        for name, rows in planes:
            arr = getattr(osc, name)
            for r in range(rows):
                if name == "sh" and r % 3 != 0 and r > 3:
                    continue
                idx = (i,) if name == "logits" else ((r // 3, r % 3, i) if name == "sh" else (r, i))
                x0 = arr[idx]
                h = 1e-6 * max(1.0, abs(x0))
                arr[idx] = x0 + h
                Lp, sp = _loss(O, osc, cam, ups, bg)
                arr[idx] = x0 - h
                Lm, sm = _loss(O, osc, cam, ups, bg)
                arr[idx] = x0
                if not (np.array_equal(sp, sig0) and np.array_equal(sm, sig0)):
                    continue  # a discrete decision flipped
                fd = (Lp - Lm) / (2 * h)
                ad = g[name][idx]
                err = abs(fd - ad) / max(abs(fd), 1e-3)
                worst = max(worst, err)
                assert err < 2e-4, (name, r, i, fd, ad)
                checked += 1
    assert checked > 200
