"""Helpers shared by the GPU parity tests: tolerance checks between the CUDA
render (fp32) and the FP64 oracle.

Tolerances (stated for the render's outputs):
  colour (rgb, and alpha, which is 1 - T on the same scale): |gpu - ref| <= 2e-4
      on >= 99.99 % of values and <= 5e-3 on all; the excess is the alpha = 1/255
      cut flipping under fp32 rounding (a flip moves a pixel by at most about
      c * 1/255).
  depth: 2e-4 relative to max(1, |ref depth|) on >= 99.99 % of the pixels; on all,
      5e-3 relative to max(1, |ref depth|, ref depth / ref alpha): an alpha-cut
      flip moves depth by about z / 255, z the flipping Gaussian's depth, which
      the alpha-weighted mean depth depth / alpha stands for.
  gradient channels ("1e-3 relative"): per channel,
      |g - g_ref| <= 1e-3 * max(|g_ref|, 1e-2 * rms(g_ref over the image))
      on >= 99.99 % of the pixels whose colour is within 2e-4 and where no
      discrete decision lies within 1e-5 of its threshold (the oracle's `amb`:
      the alpha cut, cap and stop, where the derivative jumps). On all of those
      pixels the error must also stay within that bound plus 2e-4 * S, S the
      oracle's error scale of the channel: the magnitudes of the operands of every
      Eq. 3 term (c |T_x| a and c T a (|conic_a dx| + |conic_b dy|), the products
      inside conic d included, plus |bg T_x|), each weighted by the conditioning of
      that Gaussian's alpha at the pixel. The pixels outside the relative bar are
      those whose terms cancel (S / |g| in the hundreds) and, among their
      Gaussians, one whose fp32 evaluation is ill-conditioned: a footprint tens
      of pixels long and under a pixel wide, seen at a pixel far along its long
      axis, where the alpha of any fp32 evaluation from these fp32 inputs moves
      by up to ~2e-4 of itself (a rotation of the footprint by one ulp moves its
      thin axis by 1e-5 px at 200 px). On the paper-shaped workloads (the 1M and
      6M scenes at their resolutions) and the tiny scene they are a few in a
      million; tests on close-range stress scenes full of such footprints state
      their own fraction. Both counts are returned so that tests can report them.
"""
import numpy as np

COLOUR_TOL = 2e-4
COLOUR_TOL_ALL = 5e-3
COLOUR_FRAC = 0.9999
GRAD_REL = 1e-3
GRAD_RMS_FLOOR = 1e-2
GRAD_FRAC = 0.9999
GRAD_EVAL_FLOOR = 2e-4
# close-range stress scenes: dense 2 m clusters of up-to-metre Gaussians seen from 4 m
GRAD_FRAC_STRESS = 0.99


def check_colour(got, ref, name, scale=None, frac=COLOUR_FRAC, tol_all=COLOUR_TOL_ALL):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    if scale is not None:
        err = err / scale
    ok = err <= COLOUR_TOL
    assert ok.mean() >= frac, "%s: %.5f%% within %.0e (max err %.3g)" % (name, 100 * ok.mean(), COLOUR_TOL, err.max())
    assert err.max() <= tol_all, "%s: max err %.3g > %.0e" % (name, err.max(), tol_all)
    return ok


def depth_scale(ref_depth):
    return np.maximum(1.0, np.abs(ref_depth))


def check_depth(got, ref_depth, ref_alpha, frac=COLOUR_FRAC):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref_depth)
    ok = err <= COLOUR_TOL * depth_scale(ref_depth)
    assert ok.mean() >= frac, "depth: %.5f%% within 2e-4 of max(1, |depth|) (max rel err %.3g)" % (
        100 * ok.mean(), (err / depth_scale(ref_depth)).max())
    flip = np.maximum(depth_scale(ref_depth), np.abs(ref_depth) / np.maximum(ref_alpha, 1e-12))
    assert (err <= COLOUR_TOL_ALL * flip).all(), "depth: max err %.3g of the flip scale" % (err / flip).max()
    return ok


def grad_bound(ref, rms, rel=GRAD_REL):
    """A 1e-3 relative bar on a gradient value, with a floor of 1e-2 of the channel's rms so
    that values near zero are not held to an absolute bar finer than fp32 rounding:
    1e-3 * max(|g|, 1e-2 * rms)."""
    return rel * np.maximum(np.abs(ref), GRAD_RMS_FLOOR * rms)


def check_grad_channel(got, ref, mask, name, scale, rms=None, frac=GRAD_FRAC):
    """One gradient channel against the oracle on the pixels of `mask`: the relative bar
    on >= `frac` of them, the bar plus 2e-4 * S on all. Returns (fraction within the
    relative bar, pixels outside it)."""
    got = np.asarray(got, dtype=np.float64)
    if rms is None:
        rms = np.sqrt(np.mean(ref ** 2))
    err = np.abs(got - ref)
    b = grad_bound(ref, rms)
    m = mask
    n = max(int(m.sum()), 1)
    out16 = (err > b) & m
    frac_ok = 1.0 - out16.sum() / n
    assert frac_ok >= frac, "%s: %.5f%% within 1e-3 relative (%d pixels out, worst %.3g x the bound)" % (
        name, 100 * frac_ok, int(out16.sum()), (err / b)[m].max())
    bad = (err > b + GRAD_EVAL_FLOOR * scale) & m
    assert not bad.any(), "%s: %d pixels beyond the bound + 2e-4 S, worst %.3g vs %.3g" % (
        name, int(bad.sum()), err[bad].max(), (b + GRAD_EVAL_FLOOR * scale)[bad].min())
    return frac_ok, int(out16.sum())


def check_render(out, ref, frac=COLOUR_FRAC, grad_frac=GRAD_FRAC):
    """out: dict of torch tensors (or arrays) from the GPU; ref: oracle.render dict.
    Returns (mask of the pixels the gradient bar applies to, per-channel gradient counts)."""
    g = {k: (v.detach().cpu().numpy() if hasattr(v, "detach") else v) for k, v in out.items()}
    ok_rgb = check_colour(g["rgb"], ref["rgb"], "rgb", frac=frac)
    check_colour(g["alpha"], ref["alpha"], "alpha", frac=frac)
    check_depth(g["depth"], ref["depth"], ref["alpha"], frac=frac)
    mask = ok_rgb.all(axis=0)
    if "amb" in ref:
        mask &= ref["amb"] == 0
    counts = {}
    for i, key in enumerate(("dcdx", "dcdy")):
        for c in range(3):
            counts["%s[%d]" % (key, c)] = check_grad_channel(g[key][c], ref[key][c], mask, "%s[%d]" % (key, c),
                                                             ref["gabs"][i][c], frac=grad_frac)
    return mask, counts
