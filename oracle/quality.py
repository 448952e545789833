"""Error measures of the foreground estimate (Section IV-C), in double precision.

TEST INFRASTRUCTURE, like the rest of ``oracle``: only ``tests/`` and ``bench.py``'s
CPU leg may import it. Each measure is summed over the pixels with 0 < alpha_gt < 1 and
weighted by alpha_gt (Section IV-C):
  SAD  = sum alpha_i |F_est_i - F_gt_i|_1
  MSE  = sum alpha_i |F_est_i - F_gt_i|_2^2
  GRAD = sum alpha_i |grad F_est_i - grad F_gt_i|_2^2
where the norms run over the three colour channels and, for GRAD, over both gradient
components of each channel. The gradient image is taken with first-order Gaussian
derivative filters of standard deviation sigma = 1.4 (Section IV-C).

Readings where the paper is silent: the filters are the sampled Gaussian
g(k) = exp(-k^2 / (2 sigma^2)) normalised to sum 1 and its derivative
g'(k) = -k / sigma^2 g(k), on k = -r..r with r = floor(4 sigma + 0.5) = 6; the x
component convolves rows with g' and columns with g (the y component the other way
round); pixels beyond the border repeat the nearest border pixel.
"""
from __future__ import annotations

import numpy as np

SIGMA = 1.4
TRUNCATE = 4.0


def gaussian_kernels(sigma: float = SIGMA, truncate: float = TRUNCATE):
    """Taps k = -r..r, the normalised Gaussian g and its derivative g' (float64)."""
    r = int(truncate * sigma + 0.5)
    k = np.arange(-r, r + 1, dtype=np.float64)
    g = np.exp(-0.5 * k * k / (sigma * sigma))
    g /= g.sum()
    dg = -k / (sigma * sigma) * g
    return k, g, dg


def convolve1d(a: np.ndarray, kern: np.ndarray, axis: int) -> np.ndarray:
    """out[x] = sum_j kern(j) a[x - j] along `axis`, j = -r..r, borders repeated."""
    r = len(kern) // 2
    a = np.asarray(a, np.float64)
    pad = [(0, 0)] * a.ndim
    pad[axis] = (r, r)
    ap = np.pad(a, pad, mode="edge")
    n = a.shape[axis]
    out = np.zeros_like(a)
    for t, j in enumerate(range(-r, r + 1)):
        sl = [slice(None)] * a.ndim
        sl[axis] = slice(r - j, r - j + n)       # a[x - j] sits at padded index x - j + r
        out += kern[t] * ap[tuple(sl)]
    return out


def gradient(F: np.ndarray, sigma: float = SIGMA):
    """(gx, gy) of an [H][W] or [H][W][C] image: Gaussian derivative along x (axis 1) or
    y (axis 0), Gaussian smoothing along the other axis."""
    _, g, dg = gaussian_kernels(sigma)
    gx = convolve1d(convolve1d(F, dg, axis=1), g, axis=0)
    gy = convolve1d(convolve1d(F, g, axis=1), dg, axis=0)
    return gx, gy


def measures(F_est, F_gt, alpha_gt, sigma: float = SIGMA) -> dict:
    """SAD, MSE and GRAD of Section IV-C for [H][W][3] foregrounds and an [H][W] matte."""
    Fe = np.asarray(F_est, np.float64)
    Fg = np.asarray(F_gt, np.float64)
    a = np.asarray(alpha_gt, np.float64)
    m = (a > 0) & (a < 1)
    wgt = np.where(m, a, 0.0)
    d = Fe - Fg
    sad = float(np.sum(wgt * np.abs(d).sum(axis=-1)))
    mse = float(np.sum(wgt * (d * d).sum(axis=-1)))
    gxe, gye = gradient(Fe, sigma)
    gxg, gyg = gradient(Fg, sigma)
    grad = float(np.sum(wgt * (((gxe - gxg) ** 2) + ((gye - gyg) ** 2)).sum(axis=-1)))
    return {"sad": sad, "mse": mse, "grad": grad, "pixels": int(m.sum())}
