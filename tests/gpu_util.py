"""Helpers shared by the GPU parity tests: tolerance checks between the CUDA
render (fp32) and the FP64 oracle.

Tolerances (stated for the render's outputs):
  colour (rgb, and alpha, which is 1 - T on the same scale): |gpu - ref| <= 2e-4
      on >= 99.99 % of values and <= 5e-3 on all; the excess is the alpha = 1/255
      cut flipping under fp32 rounding (a flip moves a pixel by at most about
      c * 1/255).
  depth: the same, scaled by max(1, ref depth / ref alpha): depth = sum z a T is
      the alpha terms weighted by the contributors' depth, so the same per-term
      error shows up multiplied by their (alpha-weighted mean) depth.
  gradient channels: |g - g_ref| <= 1e-3 * (|g_ref| + S) + 1e-5 per channel,
      where S is the oracle's per-pixel sum of |terms| of Eq. 3 (incl. the bg
      term), on pixels whose colour is within 2e-4 and with no discrete decision
      within 1e-5 of its threshold (oracle `amb`): "1e-3 relative", measured
      against the magnitude of the terms the gradient is made of. The projected
      centre u is an fp32 number (ulp up to 1.2e-4 px below 2048 px); a term
      c T a (conic d)_x moves by c T a (|e|^2 + |conic|) ulp(u), up to ~5e-4
      of itself for the Gaussians here (sigma >= 0.55 px after the low-pass),
      and terms that nearly cancel keep that absolute error. A 1e-5 absolute floor covers pixels where conic * d
      itself nearly cancels, so its relative error is unbounded while its
      absolute error stays ~ c T a |conic| ulp(u) (about 1e-5 for |u| near
      1000 px; 1e-5 is 1/400 of one 8-bit level).
"""
import numpy as np

COLOUR_TOL = 2e-4
COLOUR_TOL_ALL = 5e-3
COLOUR_FRAC = 0.9999
GRAD_REL = 1e-3


def check_colour(got, ref, name, scale=None, frac=COLOUR_FRAC, tol_all=COLOUR_TOL_ALL):
    got = np.asarray(got, dtype=np.float64)
    err = np.abs(got - ref)
    if scale is not None:
        err = err / scale
    ok = err <= COLOUR_TOL
    assert ok.mean() >= frac, "%s: %.5f%% within %.0e (max err %.3g)" % (name, 100 * ok.mean(), COLOUR_TOL, err.max())
    assert err.max() <= tol_all, "%s: max err %.3g > %.0e" % (name, err.max(), tol_all)
    return ok


def grad_bound(ref, scale, rel=GRAD_REL):
    return rel * (np.abs(ref) + scale) + 1e-5


def depth_scale(ref_depth, ref_alpha):
    return np.maximum(1.0, np.abs(ref_depth) / np.maximum(ref_alpha, 1e-12))


def check_grad(got, ref, mask, name, scale, rel=GRAD_REL):
    got = np.asarray(got, dtype=np.float64)
    for c in range(ref.shape[0]):
        r = ref[c]
        bound = grad_bound(r, scale[c], rel)
        bad = (np.abs(got[c] - r) > bound) & mask
        assert not bad.any(), "%s[%d]: %d pixels out of tolerance, worst %.3g vs bound %.3g" % (
            name, c, bad.sum(), np.abs(got[c] - r)[bad].max(), bound[bad].min())


def check_render(out, ref, frac=COLOUR_FRAC):
    """out: dict of torch tensors from the GPU; ref: oracle.render dict."""
    g = {k: v.detach().cpu().numpy() for k, v in out.items()}
    ok_rgb = check_colour(g["rgb"], ref["rgb"], "rgb", frac=frac)
    check_colour(g["alpha"], ref["alpha"], "alpha", frac=frac)
    check_colour(g["depth"], ref["depth"], "depth", scale=depth_scale(ref["depth"], ref["alpha"]), frac=frac,
                 tol_all=COLOUR_TOL_ALL)
    mask = ok_rgb.all(axis=0)
    if "amb" in ref:
        mask &= ref["amb"] == 0
    check_grad(g["dcdx"], ref["dcdx"], mask, "dcdx", ref["gabs"][0])
    check_grad(g["dcdy"], ref["dcdy"], mask, "dcdy", ref["gabs"][1])
    return mask
