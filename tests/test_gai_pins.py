"""Pins of the oracle's gradient-aware interpolation (Sec. 4.1, Eq. 5-8).

They hold it to what the definition fixes independently of its code:
- The least-squares Hermite weights reproduce every polynomial of their degree at the
  high-resolution pixel centres: values and gradients of the polynomial in, the polynomial
  out (Eq. 5 with an exact fit).
- One-hot weights route exactly one input (plane q, node offset (i, j)) to exactly one output
  sub-pixel (u, v). This pins the column-wise Vec order, the zero padding and the
  high-resolution block layout.
- A per-pixel Python loop applies the matrix form of Eq. 7, M = Wt Wc with bias Wt bc + bt,
  and must equal the Conv -> TConv evaluation (Eq. 8).
"""
import numpy as np
import pytest

from oracle import gai as G


def _poly(coef, X, Y):
    return sum(c * X ** a * Y ** b for (a, b), c in coef.items())


def _poly_dx(coef, X, Y):
    return sum(c * a * X ** (a - 1) * Y ** b for (a, b), c in coef.items() if a)


def _poly_dy(coef, X, Y):
    return sum(c * b * X ** a * Y ** (b - 1) for (a, b), c in coef.items() if b)


@pytest.mark.parametrize("S", [2, 3, 4])
def test_hermite_weights_reproduce_quartic_images(S):
    """A random degree-4 polynomial image in pixel units (pixel (x, y) sampled at its
    centre (x + 0.5, y + 0.5)), its exact gradients per low-resolution pixel: the
    interpolation equals the polynomial at every high-resolution centre away from the
    zero-padded border."""
    rng = np.random.default_rng(S)
    H, W = 9, 11
    coef = {(a, b): rng.standard_normal() * 0.3 ** (a + b) for a in range(5) for b in range(5 - a)}
    ys, xs = np.mgrid[0:H, 0:W].astype(np.float64)
    X, Y = xs + 0.5 - W / 2, ys + 0.5 - H / 2
    I = _poly(coef, X, Y)[None]
    Ix, Iy = _poly_dx(coef, X, Y)[None], _poly_dy(coef, X, Y)[None]
    out = G.gai(I, Ix, Iy, *G.hermite_weights(S, 4, channels=32), S)
    hy, hx = np.mgrid[0:S * H, 0:S * W].astype(np.float64)
    want = _poly(coef, (hx + 0.5) / S - W / 2, (hy + 0.5) / S - H / 2)
    inner = np.zeros((S * H, S * W), bool)
    inner[S:-S, S:-S] = True
    np.testing.assert_allclose(out[0][inner], want[inner], rtol=1e-9, atol=1e-9 * np.abs(want).max())
    # Not every image is reproduced: a degree-6 term is outside the fitted space.
    I6 = (X ** 6)[None]
    out6 = G.gai(I6, (6 * X ** 5)[None], np.zeros_like(I6), *G.hermite_weights(S, 4), S)
    assert np.abs(out6[0][inner] - ((hx + 0.5) / S - W / 2)[inner] ** 6).max() > 1e-3


def test_hermite_weights_of_a_constant_and_a_ramp():
    """Degree 0 and 1 by hand: a constant image stays constant; I = x with dI/dx = 1
    gives the sub-pixel x coordinate."""
    S = 4
    one = np.ones((1, 5, 6))
    zero = np.zeros_like(one)
    out = G.gai(one, zero, zero, *G.hermite_weights(S), S)
    np.testing.assert_allclose(out[0, S:-S, S:-S], 1.0, atol=1e-12)
    x = np.broadcast_to(np.arange(6, dtype=np.float64) + 0.5, (1, 5, 6))
    out = G.gai(x, one, zero, *G.hermite_weights(S), S)
    hx = (np.arange(6 * S) + 0.5) / S
    np.testing.assert_allclose(out[0, S:-S, S:-S], np.broadcast_to(hx, (5 * S, 6 * S))[S:-S, S:-S], atol=1e-12)


@pytest.mark.parametrize("q,i,j,u,v", [(0, 0, 0, 0, 0), (0, 1, 0, 2, 1), (1, -1, 1, 3, 3), (2, 0, -1, 1, 2),
                                       (2, 1, 1, 0, 3)])
def test_one_hot_weights_route_one_node_to_one_subpixel(q, i, j, u, v):
    S, H, W = 4, 6, 7
    rng = np.random.default_rng(7)
    planes = [rng.standard_normal((2, H, W)) for _ in range(3)]
    Wc = np.zeros((1, 27))
    Wc[0, 9 * q + 3 * (i + 1) + (j + 1)] = 1.0
    Wt = np.zeros((S * S, 1))
    Wt[u * S + v, 0] = 1.0
    out = G.gai(*planes, Wc, None, Wt, None, S)
    src = np.zeros((2, H + 2, W + 2))
    src[:, 1:-1, 1:-1] = planes[q]
    want = src[:, 1 + j:1 + j + H, 1 + i:1 + i + W]  # node (x0 + i, y0 + j), zero outside
    np.testing.assert_array_equal(out[:, v::S, u::S], want)
    mask = np.ones((S * H, S * W), bool)
    mask[v::S, u::S] = False
    assert np.all(out[:, mask] == 0.0)


def test_conv_tconv_equals_the_matrix_form_per_pixel():
    S, H, W, C = 3, 4, 5, 32
    rng = np.random.default_rng(11)
    planes = [rng.standard_normal((3, H, W)) for _ in range(3)]
    Wc, bc = rng.standard_normal((C, 27)), rng.standard_normal(C)
    Wt, bt = rng.standard_normal((S * S, C)), rng.standard_normal(S * S)
    out = G.gai(*planes, Wc, bc, Wt, bt, S)
    M, b = Wt @ Wc, Wt @ bc + bt
    for c in range(3):
        for y in range(H):
            for x in range(W):
                vec = []
                for P in planes:            # Eq. 7: I, dI/dx, dI/dy blocks
                    for i in (-1, 0, 1):    # column-wise: x offset outer
                        for j in (-1, 0, 1):
                            inside = 0 <= x + i < W and 0 <= y + j < H
                            vec.append(P[c, y + j, x + i] if inside else 0.0)
                blk = M @ np.array(vec) + b
                for u in range(S):
                    for v in range(S):
                        assert out[c, S * y + v, S * x + u] == pytest.approx(blk[u * S + v], rel=1e-12, abs=1e-12)


def test_term_scale_bounds_the_output():
    S = 2
    rng = np.random.default_rng(3)
    planes = [rng.standard_normal((1, 5, 5)) for _ in range(3)]
    w = (rng.standard_normal((8, 27)), rng.standard_normal(8), rng.standard_normal((4, 8)), rng.standard_normal(4))
    out = G.gai(*planes, *w, S)
    scale = G.gai_term_scale(*planes, *w, S)
    assert np.all(np.abs(out) <= scale * (1 + 1e-12)) and np.all(scale > 0)
