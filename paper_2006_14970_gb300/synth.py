"""Seeded synthetic inputs (image I, alpha matte) shaped like matting photographs.

This module holds input generation only, none of the solver's arithmetic; the oracle and
the GPU library receive the same arrays from it. It stands in for the ground-truth
foreground dataset of Rhemann et al. used in the paper's experiments (Section IV-B),
which is not available here: no item of that dataset is reproduced.

Recipe (numpy PCG64, seed = 2006149700 + workload index, + i for the i-th batch image):
  * smooth field: value noise on a grid of about 8 cells across the longer side,
    N(0, 1) node values, smoothstep interpolation, min-max normalised to [0, 1];
  * F and B: independent smooth fields, 3 channels each;
  * alpha: smoothstep(t0, t1, z) of a smooth field z, t0/t1 its 40th/60th percentiles
    (about 40 % alpha = 0, 40 % alpha = 1, 20 % fractional edge);
  * hair variant: percentile band 37/63, plus thin strands (random cubic Bezier curves,
    Gaussian cross profile, peak alpha U(0.3, 0.9), merged by max) until the fraction
    of pixels with 0 < alpha < 1 reaches the requested target (30 % by default);
  * composite: I = clip(alpha F + (1 - alpha) B + N(0, 0.01^2), 0, 1).
Arrays are float32, I [H][W][3] and alpha [H][W], C-contiguous.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

SEED_BASE = 2006149700


def _smoothstep01(t):
    t = np.clip(t, 0.0, 1.0)
    return t * t * (3.0 - 2.0 * t)


def smooth_field(rng: np.random.Generator, w: int, h: int, cells: float = 8.0) -> np.ndarray:
    """Value noise in [0, 1], float32 [h][w]."""
    longer = max(w, h)
    gw = max(1, int(round(cells * w / longer)))
    gh = max(1, int(round(cells * h / longer)))
    grid = rng.standard_normal((gh + 1, gw + 1))

    def axis(n, g):
        u = (np.arange(n) + 0.5) * (g / n)
        i0 = np.minimum(np.floor(u).astype(np.int64), g - 1)
        s = _smoothstep01(u - i0)
        return i0, s

    ix, sx = axis(w, gw)
    iy, sy = axis(h, gh)
    gx = grid[:, ix] * (1.0 - sx) + grid[:, ix + 1] * sx            # (gh+1, w)
    f = gx[iy, :] * (1.0 - sy)[:, None] + gx[iy + 1, :] * sy[:, None]
    lo, hi = f.min(), f.max()
    f = (f - lo) / (hi - lo) if hi > lo else np.zeros_like(f)
    return f.astype(np.float32)


def _strands(rng, alpha: np.ndarray, target: float, max_strands: int = 100000) -> float:
    """Adds hair-like strands to alpha (in place, merged by max) until the fraction of
    fractional pixels reaches ``target``. Returns the achieved fraction."""
    h, w = alpha.shape
    frac = float(np.mean((alpha > 0) & (alpha < 1)))
    flat = alpha.reshape(-1)
    drawn = 0
    while frac < target and drawn < max_strands:
        batch = max(1, min(64, int((target - frac) * w * h / 400)))
        for _ in range(batch):
            length = rng.uniform(0.05, 0.25) * max(w, h)
            p0 = rng.uniform([0, 0], [w, h])
            ang = rng.uniform(0, 2 * np.pi)
            d = np.array([np.cos(ang), np.sin(ang)]) * length
            ctrl = [p0, p0 + d / 3 + rng.normal(0, length / 4, 2),
                    p0 + 2 * d / 3 + rng.normal(0, length / 4, 2), p0 + d]
            ns = max(8, int(length * 2))
            t = np.linspace(0, 1, ns)[:, None]
            pts = ((1 - t) ** 3 * ctrl[0] + 3 * (1 - t) ** 2 * t * ctrl[1]
                   + 3 * (1 - t) * t ** 2 * ctrl[2] + t ** 3 * ctrl[3])
            sigma = rng.uniform(0.5, 1.5) / 2.0          # 1-3 px wide
            peak = rng.uniform(0.3, 0.9)
            r = int(np.ceil(3 * sigma))
            oy, ox = np.mgrid[-r:r + 1, -r:r + 1]
            cx = np.floor(pts[:, 0]).astype(np.int64)
            cy = np.floor(pts[:, 1]).astype(np.int64)
            px = cx[:, None] + ox.reshape(1, -1)
            py = cy[:, None] + oy.reshape(1, -1)
            dist2 = (px + 0.5 - pts[:, 0:1]) ** 2 + (py + 0.5 - pts[:, 1:2]) ** 2
            val = peak * np.exp(-dist2 / (2 * sigma * sigma))
            ok = (px >= 0) & (px < w) & (py >= 0) & (py < h) & (val >= 0.02)
            idx = (py[ok] * w + px[ok])
            np.maximum.at(flat, idx, val[ok].astype(np.float32))
            drawn += 1
        frac = float(np.mean((alpha > 0) & (alpha < 1)))
    return frac


@dataclass
class Sample:
    I: np.ndarray          # float32 [H][W][3]
    alpha: np.ndarray      # float32 [H][W]
    F: np.ndarray          # generating foreground, float32 [H][W][3]
    B: np.ndarray          # generating background, float32 [H][W][3]
    fractional: float      # fraction of pixels with 0 < alpha < 1


def make_sample(w: int, h: int, seed: int, hair: bool = False,
                hair_target: float = 0.30, noise: float = 0.01) -> Sample:
    """One seeded (I, alpha) pair of size w x h (see the module docstring)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    F = np.stack([smooth_field(rng, w, h) for _ in range(3)], axis=-1)
    B = np.stack([smooth_field(rng, w, h) for _ in range(3)], axis=-1)
    z = smooth_field(rng, w, h, cells=6.0)
    lo_p, hi_p = (37.0, 63.0) if hair else (40.0, 60.0)
    t0, t1 = np.percentile(z, [lo_p, hi_p])
    if t1 > t0:
        alpha = _smoothstep01((z - t0) / (t1 - t0)).astype(np.float32)
    else:
        alpha = (z > t0).astype(np.float32)
    if hair:
        _strands(rng, alpha, hair_target)
    a3 = alpha[..., None]
    I = a3 * F + (1.0 - a3) * B
    I = I + rng.normal(0.0, noise, I.shape).astype(np.float32)
    I = np.clip(I, 0.0, 1.0).astype(np.float32)
    frac = float(np.mean((alpha > 0) & (alpha < 1)))
    return Sample(np.ascontiguousarray(I), np.ascontiguousarray(alpha), F, B, frac)


# Named workloads: (width, height, seed offset, hair)
WORKLOADS = {
    "single_128x128": (128, 128, 0, False),
    "single_2048x1536_hair": (2048, 1536, 1, True),
    "single_7680x4320": (7680, 4320, 3, False),
}


def workload(name: str) -> Sample:
    w, h, k, hair = WORKLOADS[name]
    return make_sample(w, h, SEED_BASE + k, hair=hair)


def batch_sizes(n: int = 64, lo: int = 256, hi: int = 2048, seed: int = SEED_BASE + 2):
    """Image sizes for a batch of uneven images: each side log-uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed))
    ws = np.exp(rng.uniform(np.log(lo), np.log(hi), n)).round().astype(int)
    hs = np.exp(rng.uniform(np.log(lo), np.log(hi), n)).round().astype(int)
    return list(zip(ws.tolist(), hs.tolist()))


def batch(n: int = 64, lo: int = 256, hi: int = 2048, seed: int = SEED_BASE + 2):
    """A batch of uneven images, image i seeded with seed + 1 + i."""
    return [make_sample(w, h, seed + 1 + i) for i, (w, h) in
            enumerate(batch_sizes(n, lo, hi, seed))]
