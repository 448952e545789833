"""fg_estimate_noalloc: the entry point for callers that cannot let the library allocate
device memory (a process whose memory is all reserved by its own pool, or a loop that
cannot absorb cudaMalloc's implicit synchronisation). Its intermediate levels use a fixed
array inside the library. This file is collected last on purpose: if it fails, a run that
stops at the first failure has already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

from paper_2006_14970_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4   # the parity tolerance of the other GPU tests


def _dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_noalloc_matches_estimate_on_two_calls_in_a_row(fgml):
    # two different images back to back: the second call reuses the array the first one
    # left behind, and must still match the allocating entry point
    for w, h, seed in [(1024, 768, 31), (2048, 1536, 32)]:
        s = synth.make_sample(w, h, seed)
        I, A = _dev(s.I), _dev(s.alpha)
        F_ref, B_ref = fgml.estimate(I, A)
        F, B = fgml.estimate_noalloc(I, A)
        torch.cuda.synchronize()
        assert float((F - F_ref).abs().max()) <= TOL
        assert float((B - B_ref).abs().max()) <= TOL


def test_noalloc_rejects_images_beyond_its_scratch(fgml):
    lib = fgml.load()
    fn = lib.fg_estimate_noalloc
    fn.argtypes = [ctypes.POINTER(fgml.Image)] * 2 + [ctypes.POINTER(fgml.Params)] + \
        [ctypes.POINTER(fgml.Image)] * 2 + [ctypes.c_void_p]
    fn.restype = ctypes.c_int
    # argument checks run before any device work, so fake aligned addresses suffice
    w, h = 7680, 4320
    I = fgml.Image(0x100000000, w, h, w * 12, 0)
    A = fgml.Image(0x300000000, w, h, w * 4, 0)
    F = fgml.Image(0x500000000, w, h, w * 12, 0)
    B = fgml.Image(0x700000000, w, h, w * 12, 0)
    st = fn(ctypes.byref(I), ctypes.byref(A), None, ctypes.byref(F), ctypes.byref(B), None)
    assert st == fgml.FG_ERR_INVALID_ARG
    msg = lib.fg_last_error().decode()
    assert "no-allocation scratch" in msg and "7680x4320" in msg
