"""Regularisation sweep (Section IV-F): the error of the estimated foreground over a grid
of (eps_r, omega) on images whose true foreground is known.

Every solve and every error measure runs on the GPU (fg_estimate, fg_quality); this
module only loops over the grid and adds up the per-image measures.
"""
from __future__ import annotations

from . import fgml


def regularisation_sweep(images, eps_values, omega_values, stream=None):
    """images: list of (I, alpha, F_true) device tensors of one dtype. Returns a list of
    {"eps_r", "omega", "sad", "mse", "grad"} with the measures summed over the images."""
    rows = []
    for eps in eps_values:
        for omega in omega_values:
            p = fgml.params(eps_r=eps, omega=omega)
            tot = {"sad": 0.0, "mse": 0.0, "grad": 0.0}
            for I, A, Ft in images:
                F, _ = fgml.estimate(I, A, p, stream=stream)
                q = fgml.quality(F, Ft, A, stream=stream)
                for k in tot:
                    tot[k] += q[k]
            rows.append({"eps_r": float(eps), "omega": float(omega), **tot})
    return rows
