"""GPU backward (K7 reverse walk + K8 chain rule) against the FP64 oracle's
adjoint, which is itself pinned to central finite differences, plus direct
fp32 finite differences of the GPU forward and the torch.autograd.Function.

Tolerance for a gradient plane g against the oracle adjoint r:
    |g - r| <= 2e-3 * |r| + 2e-4 * max|r| (over the plane)
fp32 accumulation of per-pixel adjoints (float atomics in any order) and the
fp32 state recovery T_i = T_{i+1} / (1 - a_i) give relative errors of ~1e-5
per term; terms of both signs from thousands of pixels cancel, so the
plane's largest magnitude sets the absolute floor. Upstream gradients are
zeroed at pixels where a discrete decision is within 1e-5 of its threshold
(the oracle's `amb`), where forward and reference may legitimately differ.
"""
import numpy as np
import pytest

from paper_2605_11489_gb300 import synth

pytestmark = pytest.mark.gpu

PLANES = ("means", "log_scales", "quats", "logits", "sh")


@pytest.fixture(scope="module")
def env():
    import torch

    import __graft_entry__ as g

    g.build()
    import oracle
    from paper_2605_11489_gb300 import api

    torch.cuda.set_device(0)
    return api, oracle, api.Context(0)


def _deg3_scene(n, seed, deg=3):
    rng = np.random.default_rng(seed)
    s = synth.empty_scene(n, deg)
    nk = (deg + 1) ** 2
    s.means[:, :n] = rng.uniform(-1, 1, (3, n))
    s.log_scales[:, :n] = rng.normal(-3.3, 0.5, (3, n))
    s.quats[:, :n] = rng.normal(size=(4, n))
    s.logits[:n] = rng.normal(0.3, 1.5, n)
    s.sh[0, :, :n] = rng.uniform(-1.7, 1.7, (3, n))
    s.sh[1:, :, :n] = rng.normal(0, 0.2, (nk - 1, 3, n))
    return s


def _upstream(oracle, sc, cam, bg, seed=3, with_depth_alpha=False):
    ref = oracle.render(sc, cam, bg=bg)
    ups = synth.upstream_grads(cam.width, cam.height, seed)
    ok = (ref["amb"] == 0).astype(np.float32)
    out = {k: (v * ok).astype(np.float32) for k, v in ups.items()}
    if with_depth_alpha:
        rng = np.random.default_rng(seed + 1)
        out["depth"] = (rng.standard_normal((cam.height, cam.width)) * ok).astype(np.float32)
        out["alpha"] = (rng.standard_normal((cam.height, cam.width)) * ok).astype(np.float32)
    return out


def _gpu_grads(api, ctx, sc, cam, ups, bg, tile=16):
    import torch

    scene = api.Scene.from_arrays(sc)
    out, st = ctx.forward(scene, cam, bg=bg, state=True, tile=tile)
    gi = {k: torch.from_numpy(v).cuda() for k, v in ups.items()}
    grads = ctx.backward(st, scene, gi)
    torch.cuda.synchronize()
    st.free()
    return {k: g.cpu().numpy().astype(np.float64) for k, g in zip(PLANES, grads)}


def _compare(got, ref, n, name_extra=""):
    for k in PLANES:
        g = got[k][..., :n]
        r = ref[k][..., :n]
        scale = np.abs(r).max()
        bound = 2e-3 * np.abs(r) + 2e-4 * scale + 1e-9
        bad = np.abs(g - r) > bound
        assert not bad.any(), "%s%s: %d/%d out of tolerance, worst |d| %.3g (scale %.3g)" % (
            k, name_extra, bad.sum(), bad.size, np.abs(g - r).max(), scale)


@pytest.mark.parametrize("bg", [(0.0, 0.0, 0.0), (0.3, 0.6, 0.1)])
def test_backward_matches_oracle_adjoint_subset(env, bg):
    """The 2,048-Gaussian, 128x72 parity subset (first 2,048 Gaussians of the
    tiny-scene generator, seed 4), upstream N(0,1) on rgb, dC/dx, dC/dy."""
    api, O, ctx = env
    sc = synth.tiny_scene(4096, 4).subset(np.arange(2048))
    cam = synth.tiny_camera(128, 72)
    ups = _upstream(O, sc, cam, bg)
    got = _gpu_grads(api, ctx, sc, cam, ups, bg)
    ref = O.backward(sc, cam, ups.get("rgb"), ups.get("dcdx"), ups.get("dcdy"), bg=bg)
    _compare(got, ref, sc.n)


@pytest.mark.parametrize("tile", [8, 16, 32])
def test_backward_deg3_with_depth_and_alpha(env, tile):
    api, O, ctx = env
    sc = _deg3_scene(600, 8)
    cam = synth.jittered_tiny_cameras(2, 6, 160, 96)[1]
    bg = (0.2, 0.1, 0.4)
    ups = _upstream(O, sc, cam, bg, with_depth_alpha=True)
    got = _gpu_grads(api, ctx, sc, cam, ups, bg, tile=tile)
    ref = O.backward(sc, cam, ups["rgb"], ups["dcdx"], ups["dcdy"], ups["depth"], ups["alpha"], bg=bg)
    _compare(got, ref, sc.n, " tile %d" % tile)


@pytest.mark.parametrize("deg", [1, 2])
def test_backward_sh_degrees_1_and_2(env, deg):
    """The chain through SH is compiled per degree: degrees 1 and 2 against the oracle."""
    api, O, ctx = env
    sc = _deg3_scene(500, 20 + deg, deg)
    cam = synth.jittered_tiny_cameras(2, 9, 144, 80)[0]
    bg = (0.1, 0.2, 0.3)
    ups = _upstream(O, sc, cam, bg)
    got = _gpu_grads(api, ctx, sc, cam, ups, bg, tile=8)
    ref = O.backward(sc, cam, ups["rgb"], ups["dcdx"], ups["dcdy"], bg=bg)
    _compare(got, ref, sc.n, " deg %d" % deg)


def test_backward_against_fp32_finite_differences(env):
    """Central differences of the GPU's own forward for a handful of parameters
    (h = 1e-3 relative; fp32 loss noise ~1e-6 relative makes 3e-2 the bound)."""
    api, O, ctx = env
    import torch

    sc = _deg3_scene(200, 12)
    cam = synth.tiny_camera(96, 64)
    bg = (0.0, 0.0, 0.0)
    ups = _upstream(O, sc, cam, bg)
    got = _gpu_grads(api, ctx, sc, cam, ups, bg)
    gi = {k: torch.from_numpy(v).cuda() for k, v in ups.items()}

    def loss(s):
        out = ctx.forward(api.Scene.from_arrays(s), cam, bg=bg)
        return sum(float((out[k].double() * gi[k].double()).sum()) for k in gi)

    vis = np.nonzero(O.project(sc, cam)["visible"])[0]
    rng = np.random.default_rng(0)
    checked = 0
    for i in rng.choice(vis, 6, replace=False):
        for plane, idx in (("means", (0, i)), ("means", (2, i)), ("log_scales", (1, i)), ("quats", (0, i)),
                           ("logits", (i,)), ("sh", (0, 1, i)), ("sh", (5, 2, i))):
            arr = getattr(sc, plane)
            x0 = float(arr[idx])
            h = 1e-3 * max(1.0, abs(x0))
            arr[idx] = np.float32(x0 + h)
            hp = float(arr[idx]) - x0
            lp = loss(sc)
            arr[idx] = np.float32(x0 - h)
            hm = x0 - float(arr[idx])
            lm = loss(sc)
            arr[idx] = np.float32(x0)
            fd = (lp - lm) / (hp + hm)
            ad = got[plane][idx]
            if abs(fd) < 1e-3 and abs(ad) < 1e-3:
                continue
            assert abs(fd - ad) <= 3e-2 * max(abs(fd), abs(ad)) + 1e-3, (plane, idx, fd, ad)
            checked += 1
    assert checked >= 10


def test_autograd_function_matches_direct_backward(env):
    api, O, ctx = env
    import torch

    sc = _deg3_scene(300, 3)
    cam = synth.tiny_camera(96, 64)
    scene = api.Scene.from_arrays(sc)
    params = [t.clone().requires_grad_(True) for t in scene.params()]
    rgb, dcdx, dcdy, depth, alpha = api.render(ctx, params, cam, n=sc.n, deg=3)
    rng = np.random.default_rng(1)
    w = {k: torch.from_numpy(rng.standard_normal(t.shape).astype(np.float32)).cuda()
         for k, t in zip(api.OUTPUT_KEYS, (rgb, dcdx, dcdy, depth, alpha))}
    L = (rgb * w["rgb"]).sum() + (dcdx * w["dcdx"]).sum() + (dcdy * w["dcdy"]).sum() + \
        (depth * w["depth"]).sum() + (alpha * w["alpha"]).sum()
    L.backward()
    out, st = ctx.forward(scene, cam, state=True)
    direct = ctx.backward(st, scene, w)
    st.free()
    for p, d in zip(params, direct):
        torch.testing.assert_close(p.grad, d, rtol=1e-5, atol=1e-6)


def test_backward_accumulates(env):
    api, O, ctx = env
    import torch

    sc = synth.tiny_scene(512, 2)
    cam = synth.tiny_camera(96, 64)
    scene = api.Scene.from_arrays(sc)
    out, st = ctx.forward(scene, cam, state=True)
    gi = {"rgb": torch.ones_like(out["rgb"])}
    g1 = ctx.backward(st, scene, gi)
    g1 = [t.clone() for t in g1]
    g2 = ctx.backward(st, scene, gi, grads=[t.clone() for t in g1])
    st.free()
    for a, b in zip(g1, g2):
        torch.testing.assert_close(b, 2 * a, rtol=1e-5, atol=1e-7)


def test_backward_rejects_a_different_scene(env):
    api, O, ctx = env
    import torch

    from paper_2605_11489_gb300 import abi

    scene = api.Scene.from_arrays(synth.tiny_scene(64, 0))
    other = api.Scene.from_arrays(synth.tiny_scene(32, 0))
    out, st = ctx.forward(scene, synth.tiny_camera(32, 32), state=True)
    with pytest.raises(abi.GsError) as e:
        ctx.backward(st, other, {"rgb": torch.ones_like(out["rgb"])})
    assert e.value.status == abi.GS_ERR_INVALID_ARG
    st.free()
