"""Minimiser of the global cost whose per-pixel minimisation the method iterates, in
double precision, by a sparse direct solve.

TEST INFRASTRUCTURE, like the rest of ``oracle``: only ``tests/`` and ``bench.py``'s
CPU leg may import it.

Summing the local cost of Section III-C over the pixels, with each 4-neighbour edge
counted once, gives per channel c
  E(F, B) = sum_i (alpha_i F_i + (1 - alpha_i) B_i - I_i)^2
          + sum_{edges {i,j}} (eps_r + omega |alpha_i - alpha_j|) [(F_i - F_j)^2 + (B_i - B_j)^2],
whose stationarity conditions are exactly those of a fixed point of the unclamped
per-pixel update (a pixel's clamped "neighbour" is itself and drops out). grad E = 0 is
the linear system H x = b with x = (F, B), b = (alpha I, (1 - alpha) I) and
  H = [[diag(alpha^2) + L, diag(alpha (1 - alpha))], [diag(alpha (1 - alpha)), diag((1 - alpha)^2) + L]],
L the weighted graph Laplacian of the 4-neighbour grid. H is positive definite when alpha
is not constant.
"""
from __future__ import annotations

import numpy as np


def system(alpha, eps_r: float = 5e-3, omega: float = 0.1):
    """The sparse matrix H (2n x 2n, pixels in row-major order, F block first)."""
    import scipy.sparse as sp
    a = np.asarray(alpha, np.float64)
    h, w = a.shape
    n = h * w
    idx = np.arange(n).reshape(h, w)
    rows, cols, vals = [], [], []
    # edges to the right and downwards, each once
    for (i, j) in ((idx[:, :-1], idx[:, 1:]), (idx[:-1, :], idx[1:, :])):
        i = i.reshape(-1)
        j = j.reshape(-1)
        d = eps_r + omega * np.abs(a.reshape(-1)[i] - a.reshape(-1)[j])
        rows += [i, j, i, j]
        cols += [i, j, j, i]
        vals += [d, d, -d, -d]
    L = sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(n, n))
    av = a.reshape(-1)
    H = sp.bmat([[sp.diags(av * av) + L, sp.diags(av * (1 - av))],
                 [sp.diags(av * (1 - av)), sp.diags((1 - av) ** 2) + L]], format="csc")
    return H


def minimiser(I, alpha, eps_r: float = 5e-3, omega: float = 0.1):
    """(F, B) [H][W][3] minimising E per channel (no clamp)."""
    from scipy.sparse.linalg import splu
    I = np.asarray(I, np.float64)
    a = np.asarray(alpha, np.float64)
    h, w = a.shape
    n = h * w
    lu = splu(system(a, eps_r, omega))
    av = a.reshape(-1)
    F = np.empty((h, w, 3))
    B = np.empty((h, w, 3))
    for c in range(3):
        Ic = I[..., c].reshape(-1)
        x = lu.solve(np.concatenate([av * Ic, (1 - av) * Ic]))
        F[..., c] = x[:n].reshape(h, w)
        B[..., c] = x[n:].reshape(h, w)
    return F, B


def gradient_norm(I, alpha, F, B, eps_r: float = 5e-3, omega: float = 0.1) -> float:
    """|H x - b|_2 over all channels: how far (F, B) is from stationarity."""
    I = np.asarray(I, np.float64)
    a = np.asarray(alpha, np.float64)
    H = system(a, eps_r, omega)
    av = a.reshape(-1)
    tot = 0.0
    for c in range(3):
        x = np.concatenate([np.asarray(F)[..., c].reshape(-1), np.asarray(B)[..., c].reshape(-1)])
        Ic = I[..., c].reshape(-1)
        r = H @ x - np.concatenate([av * Ic, (1 - av) * Ic])
        tot += float(r @ r)
    return tot ** 0.5
