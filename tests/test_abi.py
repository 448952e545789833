"""The C ABI without a GPU: the library builds, loads, exports every declared function,
and its host-side planner and argument checks behave; no kernel is launched here."""
import ctypes
import subprocess

import numpy as np
import pytest

import oracle


def test_library_exports_every_declared_function(fgml):
    names = fgml.declared_functions()
    assert {"fg_estimate", "fg_estimate_host", "fg_level_pass", "fg_schedule",
            "fg_params_default", "fg_sync", "fg_last_error"} <= set(names)
    lib = fgml.load()
    for n in names:
        assert hasattr(lib, n), n
    out = subprocess.run(["nm", "-D", "--defined-only", fgml.library_path()],
                         capture_output=True, text=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    assert set(names) <= exported
    # nothing but the C ABI is exported under the fg_ prefix
    assert {n for n in exported if n.startswith("fg_")} == set(names)


def test_params_default_is_the_papers(fgml):
    p = fgml.params()
    assert abs(p.eps_r - 5e-3) < 1e-9 and abs(p.omega - 0.1) < 1e-8
    assert (p.small_size, p.small_iters, p.big_iters, p.order, p.clamp, p.init) == \
        (32, 10, 2, 0, 1, 0.0)


def test_schedule_matches_oracle_for_all_sizes(fgml):
    # the library's planner is its own implementation of Algorithm 1's level sizes;
    # it must agree with the pinned oracle everywhere
    for s in range(1, 8193):
        assert fgml.schedule(s, 1) == oracle.schedule(s, 1), s
    rng = np.random.default_rng(0)
    for _ in range(3000):
        w, h = (int(v) for v in rng.integers(1, 32768, 2))
        assert fgml.schedule(w, h) == oracle.schedule(w, h), (w, h)
    p = fgml.params(small_size=20, small_iters=3, big_iters=5)
    assert fgml.schedule(2048, 1536, p) == oracle.schedule(
        2048, 1536, oracle.Params(small_size=20, small_iters=3, big_iters=5))


def test_schedule_rejects_bad_sizes(fgml):
    lib = fgml.load()
    assert lib.fg_schedule(0, 5, None, None, None, None, 64) == -1
    assert lib.fg_schedule(5, 40000, None, None, None, None, 64) == -1
    assert lib.fg_schedule(8192, 8192, None, None, None, None, 3) == -1


def test_invalid_arguments_are_reported_without_touching_the_gpu(fgml):
    lib = fgml.load()
    img = fgml.Image(None, 4, 4, 48, 0)
    st = lib.fg_estimate(ctypes.byref(img), ctypes.byref(img), None, ctypes.byref(img),
                         ctypes.byref(img), None)
    assert st == fgml.FG_ERR_INVALID_ARG
    assert b"NULL" in lib.fg_last_error()
    good = fgml.Image(0x1000, 4, 4, 48, 0)
    zero = fgml.Image(0x2000, 0, 4, 48, 0)
    st = lib.fg_estimate(ctypes.byref(zero), ctypes.byref(good), None, ctypes.byref(good),
                         ctypes.byref(good), None)
    assert st == fgml.FG_ERR_INVALID_ARG
    small_pitch = fgml.Image(0x3000, 4, 4, 20, 0)
    st = lib.fg_estimate(ctypes.byref(small_pitch), ctypes.byref(good), None,
                         ctypes.byref(good), ctypes.byref(good), None)
    assert st == fgml.FG_ERR_INVALID_ARG and b"pitch" in lib.fg_last_error()
    # outputs overlapping the inputs
    I = fgml.Image(0x10000, 4, 4, 48, 0)
    A = fgml.Image(0x20000, 4, 4, 16, 0)
    F = fgml.Image(0x10010, 4, 4, 48, 0)
    B = fgml.Image(0x30000, 4, 4, 48, 0)
    st = lib.fg_estimate(ctypes.byref(I), ctypes.byref(A), None, ctypes.byref(F),
                         ctypes.byref(B), None)
    assert st == fgml.FG_ERR_INVALID_ARG and b"overlap" in lib.fg_last_error()
    # bad parameters
    F = fgml.Image(0x40000, 4, 4, 48, 0)
    for kw in ({"eps_r": 0.0}, {"omega": -1.0}, {"big_iters": -1}):
        p = fgml.params(**kw)
        st = lib.fg_estimate(ctypes.byref(I), ctypes.byref(A), ctypes.byref(p),
                             ctypes.byref(F), ctypes.byref(B), None)
        assert st == fgml.FG_ERR_INVALID_ARG, kw
    # the raster Gauss-Seidel order of the oracle is sequential and has no GPU form
    p = fgml.params(order=2)
    st = lib.fg_estimate(ctypes.byref(I), ctypes.byref(A), ctypes.byref(p), ctypes.byref(F),
                         ctypes.byref(B), None)
    assert st == fgml.FG_ERR_UNSUPPORTED


def test_product_package_does_not_use_the_oracle():
    # the library and its binding never import, load or call the oracle
    import os
    import re
    pkg = os.path.join(os.path.dirname(os.path.dirname(__file__)), "paper_2006_14970_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".h", ".cuh", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b|liboracle|ml_oracle", text, re.M), f
