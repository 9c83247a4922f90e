"""CPU FP64 oracle of the gradient-aware interpolation of Sec. 4.1 (test infrastructure only).

Only the tests, ``__graft_entry__.smoke()`` and the bench's CPU-baseline leg may import
this module; the product path never does.

What it computes (Eq. 5-8). For every low-resolution pixel (x0, y0) and colour channel, the
input vector is the 27 values of Eq. 7:
    [Vec(I_3x3), Vec(dI/dx_3x3), Vec(dI/dy_3x3)]
over the 3x3 block of nodes (x0 + i, y0 + j), i, j in {-1, 0, 1}.
- Vec is column-wise vectorisation: a column is one x offset i, and its entries run over the
  y offsets j. Input index = 9 q + 3 (i + 1) + (j + 1), with q = 0 (I), 1 (dI/dx), 2 (dI/dy).
- Nodes outside the image read 0 (the zero padding of a 3x3 convolution).

Eq. 8 realises M in Eq. 7 as a 3x3 convolution to C feature channels, followed by an SxS
transposed convolution of stride S:
    F = Wc x + bc                  Wc [C, 27], bc [C]
    B = Wt F + bt                  Wt [S*S, C], bt [S*S]
Output s = u S + v is the high-resolution pixel (S x0 + u, S y0 + v). This is again
column-wise: u is the x sub-index, v the y sub-index. The same weights serve every colour
channel.

`hermite_weights` gives one analytic M, used as a pin:
- the least-squares fit, to the 27 conditions of Eq. 5, of a bivariate polynomial of total
  degree <= `degree` in the offsets from the centre pixel, in low-resolution pixel units;
- evaluated at the high-resolution pixel centres, whose offsets are ((u + 0.5) / S - 0.5,
  (v + 0.5) / S - 0.5).

It reproduces every polynomial of that degree exactly, and the pins check that. The paper
trains M instead (its weights are not available).
"""
from __future__ import annotations

import numpy as np

OFFSETS = (-1, 0, 1)


def gai_inputs(I, Ix, Iy) -> np.ndarray:
    """The Eq. 7 input vectors: [Cc, H, W] planes -> [Cc, H, W, 27] (FP64, zero padded)."""
    planes = [np.asarray(a, np.float64) for a in (I, Ix, Iy)]
    Cc, H, W = planes[0].shape
    X = np.zeros((Cc, H, W, 27))
    for q, P in enumerate(planes):
        pad = np.zeros((Cc, H + 2, W + 2))
        pad[:, 1:-1, 1:-1] = P
        for i in OFFSETS:
            for j in OFFSETS:
                # node (x0 + i, y0 + j) of every pixel
                X[..., 9 * q + 3 * (i + 1) + (j + 1)] = pad[:, 1 + j:1 + j + H, 1 + i:1 + i + W]
    return X


def gai(I, Ix, Iy, Wc, bc, Wt, bt, S: int) -> np.ndarray:
    """Conv3x3 -> TConv SxS (Eq. 8) in FP64: [Cc, H, W] planes -> [Cc, S H, S W]."""
    Wc, Wt = np.asarray(Wc, np.float64), np.asarray(Wt, np.float64)
    bc = np.zeros(Wc.shape[0]) if bc is None else np.asarray(bc, np.float64)
    bt = np.zeros(Wt.shape[0]) if bt is None else np.asarray(bt, np.float64)
    assert Wc.shape[1] == 27 and Wt.shape == (S * S, Wc.shape[0])
    X = gai_inputs(I, Ix, Iy)
    F = X @ Wc.T + bc          # Conv(I): the coefficient vector in the polynomial space
    B = F @ Wt.T + bt          # TConv(F): S*S pixel values per low-resolution pixel
    Cc, H, W, _ = B.shape
    out = np.zeros((Cc, S * H, S * W))
    for u in range(S):
        for v in range(S):
            out[:, v::S, u::S] = B[..., u * S + v]
    return out


def gai_term_scale(I, Ix, Iy, Wc, bc, Wt, bt, S: int) -> np.ndarray:
    """Per output: the sum of |terms| of its evaluation as (Wt Wc) x + (Wt bc + bt), bounding
    any evaluation order's rounding error (sum of |M_sk x_k| + |b_s|), in [Cc, S H, S W]."""
    Wc, Wt = np.asarray(Wc, np.float64), np.asarray(Wt, np.float64)
    bc = np.zeros(Wc.shape[0]) if bc is None else np.asarray(bc, np.float64)
    bt = np.zeros(Wt.shape[0]) if bt is None else np.asarray(bt, np.float64)
    M = Wt @ Wc
    b = Wt @ bc + bt
    A = np.abs(gai_inputs(I, Ix, Iy)) @ np.abs(M).T + np.abs(b)
    Cc, H, W, _ = A.shape
    out = np.zeros((Cc, S * H, S * W))
    for u in range(S):
        for v in range(S):
            out[:, v::S, u::S] = A[..., u * S + v]
    return out


def _monomials(degree: int):
    return [(a, b) for a in range(degree + 1) for b in range(degree + 1 - a)]


def hermite_weights(S: int, degree: int = 4, channels: int | None = None):
    """(Wc, bc, Wt, bt) of the least-squares Hermite fit described in the module docstring.
    `channels` (>= the number of monomials) pads the feature dimension with zeros."""
    mono = _monomials(degree)
    P = len(mono)
    A = np.zeros((27, P))
    for m, (a, b) in enumerate(mono):
        for i in OFFSETS:
            for j in OFFSETS:
                k = 3 * (i + 1) + (j + 1)
                A[k, m] = float(i) ** a * float(j) ** b
                A[9 + k, m] = a * float(i) ** (a - 1) * float(j) ** b if a else 0.0
                A[18 + k, m] = b * float(i) ** a * float(j) ** (b - 1) if b else 0.0
    E = np.zeros((S * S, P))
    for u in range(S):
        for v in range(S):
            dx, dy = (u + 0.5) / S - 0.5, (v + 0.5) / S - 0.5
            E[u * S + v] = [dx ** a * dy ** b for a, b in mono]
    C = P if channels is None else channels
    assert C >= P
    Wc = np.zeros((C, 27))
    Wc[:P] = np.linalg.pinv(A)
    Wt = np.zeros((S * S, C))
    Wt[:, :P] = E
    return Wc, np.zeros(C), Wt, np.zeros(S * S)
