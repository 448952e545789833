"""FP64 CPU oracle for multi-level foreground estimation.

TEST INFRASTRUCTURE. This package states, plainly and slowly, what the GPU library
computes (Algorithm 1 and the per-pixel closed-form solve of Section III-C of
"Fast Multi-Level Foreground Estimation"). Only ``tests/``, ``__graft_entry__.smoke()``
and the CPU-baseline leg of ``bench.py`` may import it; the library under
``paper_2006_14970_gb300`` never does, and the two share no code.

The arithmetic lives in ``ml_oracle.c`` (plain C, double precision, optional OpenMP over
rows for the orders whose result does not depend on the visiting order). This module
only builds that file with gcc and marshals numpy arrays to it.

Every function here is pinned by ``tests/test_oracle_*.py`` against things other than
itself: exact-integer evaluation of the level schedule, the local cost it minimises,
dense solves of the global quadratic, closed forms and exact invariants.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ml_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")

JACOBI, REDBLACK, RASTER_GS = 0, 1, 2


class _Params(ctypes.Structure):
    _fields_ = [
        ("eps_r", ctypes.c_double),
        ("omega", ctypes.c_double),
        ("small_size", ctypes.c_int),
        ("small_iters", ctypes.c_int),
        ("big_iters", ctypes.c_int),
        ("order", ctypes.c_int),
        ("clamp", ctypes.c_int),
        ("init", ctypes.c_double),
    ]


@dataclass
class Params:
    """Hyper-parameters of Algorithm 1; defaults are the paper's (Section III-D, IV-F)."""

    eps_r: float = 5e-3
    omega: float = 0.1
    small_size: int = 32
    small_iters: int = 10
    big_iters: int = 2
    order: int = JACOBI
    clamp: bool = True
    init: float = 0.0

    def _c(self) -> _Params:
        return _Params(self.eps_r, self.omega, self.small_size, self.small_iters,
                       self.big_iters, self.order, int(bool(self.clamp)), self.init)


def build(force: bool = False) -> str:
    """Compile ml_oracle.c into a shared library with gcc; returns its path.

    ``-ffp-contract=off`` keeps gcc from fusing a*b+c into one rounding, so the oracle
    evaluates exactly the expressions written in the C file on every host.
    """
    if not force and os.path.exists(_LIB_PATH) and \
            os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC):
        return _LIB_PATH
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fPIC", "-shared", _SRC,
            "-o", tmp, "-lm"]
    try:
        subprocess.run(base[:1] + ["-fopenmp"] + base[1:], check=True,
                       capture_output=True)
    except subprocess.CalledProcessError:
        subprocess.run(base, check=True, capture_output=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


_lib = None


def _load():
    global _lib
    if _lib is None:
        lib = ctypes.CDLL(build())
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        pp = ctypes.POINTER(_Params)
        lib.oracle_num_levels.argtypes = [ctypes.c_int, ctypes.c_int]
        lib.oracle_level_side.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.oracle_level_iters.argtypes = [ctypes.c_int, ctypes.c_int, pp]
        lib.oracle_schedule.argtypes = [ctypes.c_int, ctypes.c_int, pp, ip, ip, ip,
                                        ctypes.c_int]
        lib.oracle_resize_nearest.argtypes = [dp, ctypes.c_int, ctypes.c_int, ctypes.c_int,
                                              dp, ctypes.c_int, ctypes.c_int]
        lib.oracle_resize_nearest.restype = None
        lib.oracle_level_iterate.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, dp, dp,
                                             ctypes.c_int, pp]
        lib.oracle_ml.argtypes = [dp, dp, ctypes.c_int, ctypes.c_int, pp, dp, dp]
        lib.oracle_set_threads.argtypes = [ctypes.c_int]
        _lib = lib
    return _lib


def _dptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _f64(a) -> np.ndarray:
    return np.ascontiguousarray(np.asarray(a, dtype=np.float64))


def set_threads(n: int) -> int:
    """Sets the OpenMP thread count (n <= 0 leaves it); returns the count in force."""
    return _load().oracle_set_threads(int(n))


def max_threads() -> int:
    return _load().oracle_max_threads()


def num_levels(w: int, h: int) -> int:
    """n_l = max(1, ceil(log2(max(w, h)))) (Algorithm 1)."""
    return _load().oracle_num_levels(int(w), int(h))


def schedule(w: int, h: int, params: Params | None = None):
    """Level sizes and iteration counts [(w_l, h_l, k_l) for l = 1..n_l] (Algorithm 1)."""
    p = (params or Params())._c()
    cap = 64
    ws = (ctypes.c_int * cap)()
    hs = (ctypes.c_int * cap)()
    ks = (ctypes.c_int * cap)()
    n = _load().oracle_schedule(int(w), int(h), ctypes.byref(p), ws, hs, ks, cap)
    if n < 0:
        raise ValueError("too many levels")
    return [(ws[i], hs[i], ks[i]) for i in range(n)]


def resize_nearest(src: np.ndarray, dw: int, dh: int) -> np.ndarray:
    """Nearest resize of [h][w] or [h][w][c] to (dh, dw): the resize() of Algorithm 1."""
    s = _f64(src)
    ch = 1 if s.ndim == 2 else s.shape[2]
    out = np.empty((dh, dw) if s.ndim == 2 else (dh, dw, ch), np.float64)
    _load().oracle_resize_nearest(_dptr(s), s.shape[1], s.shape[0], ch, _dptr(out),
                                  int(dw), int(dh))
    return out


def level_iterate(I, alpha, F, B, iters: int, params: Params | None = None):
    """``iters`` sweeps of the per-pixel update at one level; returns new (F, B)."""
    I = _f64(I)
    a = _f64(alpha)
    F = _f64(F).copy()
    B = _f64(B).copy()
    h, w = a.shape
    assert I.shape == (h, w, 3) and F.shape == (h, w, 3) and B.shape == (h, w, 3)
    p = (params or Params())._c()
    rc = _load().oracle_level_iterate(_dptr(I), _dptr(a), w, h, _dptr(F), _dptr(B),
                                      int(iters), ctypes.byref(p))
    if rc != 0:
        raise RuntimeError(f"oracle_level_iterate failed ({rc})")
    return F, B


def ml(I, alpha, params: Params | None = None):
    """Algorithm 1, ML(I_hat, alpha_hat) -> (F, B), in double precision.

    I: [H][W][3] in [0, 1]; alpha: [H][W] in [0, 1]. Returns float64 arrays.
    """
    I = _f64(I)
    a = _f64(alpha)
    h, w = a.shape
    if I.shape != (h, w, 3):
        raise ValueError("I must be [H][W][3] matching alpha [H][W]")
    F = np.empty((h, w, 3), np.float64)
    B = np.empty((h, w, 3), np.float64)
    p = (params or Params())._c()
    rc = _load().oracle_ml(_dptr(I), _dptr(a), w, h, ctypes.byref(p), _dptr(F), _dptr(B))
    if rc != 0:
        raise RuntimeError(f"oracle_ml failed ({rc})")
    return F, B


def composite(alpha, F, B_new):
    """I_new = alpha F + (1 - alpha) B_new per pixel and channel: the compositing equation
    (Section I) with a new background, in double precision."""
    a = _f64(alpha)[..., None]
    return a * _f64(F) + (1.0 - a) * _f64(B_new)
