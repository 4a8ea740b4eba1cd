"""Overlap blending of neighbouring tiles' fields within a slide, float64.

TEST INFRASTRUCTURE ONLY: imported by tests/ (and nothing on the product path).

The paper reconstructs a slide patch by patch from overlapping patches
(Sec. 2.3, 3.2) and blends the overlaps of registered fields of view without
giving a rule (Sec. 2.5; the SIFT registration itself is out of scope). Where
neighbouring windows overlap, this checker states the blending the library
performs, in output (upsampled)
pixels; window t (row-major on a rows x cols grid, as apic_slide_windows lists
them) covers [u y0_t, u y0_t + L) x [u x0_t, u x0_t + L), L = u tile:
  1. relative global phase of window t and its left / upper neighbour s:
     c_ts = sum over their common pixels of f_t(p) conj(f_s(p)), so that
     phi_t - phi_s = arg c_ts (each tile keeps the phase gauge of Eq. 5, an
     arbitrary constant per tile);
  2. phases chained along the grid: the first window has phi = 0, the rest of
     the first row follows its left neighbours, every other window its upper
     neighbour (a zero c leaves the neighbour's phase unchanged);
  3. blended field = sum_t w_t(p) exp(-i phi_t) f_t(p) / sum_t w_t(p), with
     w_t(y, x) = r_t(y) r_t(x): on each axis a linear ramp across the overlap
     with the previous window (rising) and with the next (falling), 1 elsewhere
     and at the slide's edges; two ramps across one overlap sum to 1.
"""
from __future__ import annotations

import numpy as np


def grid_shape(windows):
    """(rows, cols) of a row-major window list [n][6] (y0, x0, own y0, own x0, own y1, own x1)."""
    cols = int(np.sum(windows[:, 0] == windows[0, 0]))
    return len(windows) // cols, cols


def _starts(windows, rows, cols):
    return windows[::cols, 0].astype(np.int64), windows[:cols, 1].astype(np.int64)


def ramp(starts, j, p, L):
    """Weight of window j (start starts[j], length L) at position p on one axis."""
    s = starts[j]
    w = 1.0
    if j > 0:
        ov = starts[j - 1] + L - s
        if ov > 0 and p < s + ov:
            w *= (p - s + 0.5) / ov
    if j + 1 < len(starts):
        ov = s + L - starts[j + 1]
        if ov > 0 and p >= starts[j + 1]:
            w *= (s + L - p - 0.5) / ov
    return w


def correlations(fields, windows, u):
    """[n][2] complex: sum over the overlap with the left / upper neighbour of f_t conj(f_s) (0 if none)."""
    rows, cols = grid_shape(windows)
    n, L = len(fields), fields.shape[1]
    c = np.zeros((n, 2), dtype=np.complex128)
    for k in range(n):
        y0, x0 = u * int(windows[k, 0]), u * int(windows[k, 1])
        for d, nb in ((0, k - 1 if k % cols else -1), (1, k - cols if k >= cols else -1)):
            if nb < 0:
                continue
            sy, sx = u * int(windows[nb, 0]), u * int(windows[nb, 1])
            ya, yb = max(y0, sy), min(y0 + L, sy + L)
            xa, xb = max(x0, sx), min(x0 + L, sx + L)
            if ya >= yb or xa >= xb:
                continue
            ft = fields[k][ya - y0:yb - y0, xa - x0:xb - x0]
            fs = fields[nb][ya - sy:yb - sy, xa - sx:xb - sx]
            c[k, d] = np.sum(ft * np.conj(fs))
    return c


def phases(corr, rows, cols):
    """exp(-i phi_t) per window, chained along the grid (first row left to right, then down)."""
    z = np.ones(len(corr), dtype=np.complex128)
    for k in range(1, cols):
        c = corr[k, 0]
        z[k] = z[k - 1] * (np.conj(c) / abs(c) if abs(c) > 0 else 1.0)
    for k in range(cols, rows * cols):
        c = corr[k, 1]
        z[k] = z[k - cols] * (np.conj(c) / abs(c) if abs(c) > 0 else 1.0)
    return z


def blend(fields, windows, z, slide_h, slide_w, u):
    """[u slide_h][u slide_w] complex: the weighted, phase-aligned sum of the windows' fields."""
    rows, cols = grid_shape(windows)
    ys, xs = _starts(windows, rows, cols)
    ys, xs = u * ys, u * xs
    L = fields.shape[1]
    H, W = u * slide_h, u * slide_w
    acc = np.zeros((H, W), dtype=np.complex128)
    wsum = np.zeros((H, W), dtype=np.float64)
    ry = [np.array([ramp(ys, i, p, L) for p in range(ys[i], ys[i] + L)]) for i in range(rows)]
    rx = [np.array([ramp(xs, j, p, L) for p in range(xs[j], xs[j] + L)]) for j in range(cols)]
    for i in range(rows):
        for j in range(cols):
            k = i * cols + j
            w = np.outer(ry[i], rx[j])
            acc[ys[i]:ys[i] + L, xs[j]:xs[j] + L] += w * z[k] * fields[k]
            wsum[ys[i]:ys[i] + L, xs[j]:xs[j] + L] += w
    return acc / wsum
