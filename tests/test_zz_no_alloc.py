"""fg_estimate_noalloc: the entry point for callers that cannot let the library allocate
device memory (a process whose memory is all reserved by its own pool, or a loop that
cannot absorb cudaMalloc's implicit synchronisation). Its intermediate levels use a fixed
array inside the library. Each case is compared element by element with the FP64 oracle
and with the allocating entry point fg_estimate, through the C ABI. This file is
collected last on purpose: if it fails, a run that stops at the first failure has
already run every other test."""
import ctypes

import numpy as np
import pytest
import torch

import oracle
from paper_2006_14970_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4   # the FP32 parity tolerance of the other GPU tests
BF16_TOL = 1.2e-2   # the BF16 bound against the oracle on the rounded inputs


def _dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().to(dt)


def _max_abs(x, y):
    return float(np.abs(np.asarray(x, np.float64) - y).max())


def _check(fgml, s, dt=torch.float32):
    I, A = _dev(s.I, dt), _dev(s.alpha, dt)
    F_ref, B_ref = fgml.estimate(I, A)
    F = torch.full_like(I, float("nan"))   # unwritten pixels would stay NaN
    B = torch.full_like(I, float("nan"))
    fgml.estimate_noalloc(I, A, None, F, B)
    fgml.sync()
    Fh, Bh = F.float().cpu().numpy(), B.float().cpu().numpy()
    assert np.isfinite(Fh).all() and np.isfinite(Bh).all()
    if dt == torch.float32:
        Fo, Bo = oracle.ml(s.I, s.alpha)
        tol = TOL
    else:
        Fo, Bo = oracle.ml(I.float().cpu().numpy(), A.float().cpu().numpy())
        tol = BF16_TOL
    assert max(_max_abs(Fh, Fo), _max_abs(Bh, Bo)) <= tol
    assert float((F.float() - F_ref.float()).abs().max()) <= TOL
    assert float((B.float() - B_ref.float()).abs().max()) <= TOL


def test_noalloc_matches_oracle_and_estimate_on_two_calls_in_a_row(fgml):
    # two different images back to back: the second call reuses the array the first one
    # left behind
    for w, h, seed in [(1024, 768, 31), (2048, 1536, 32)]:
        _check(fgml, synth.make_sample(w, h, seed))


@pytest.mark.parametrize("w,h,dt", [
    (1001, 777, torch.float32),    # rows off the 16-byte grid: read in place, no aligned copy
    (30, 20, torch.float32),       # every level in the coarse kernel, which writes F and B
    (128, 128, torch.float32),     # coarse kernel, then small-level passes
    (1024, 768, torch.bfloat16),   # 16-bit storage: other level sizes in the same array
])
def test_noalloc_other_paths(fgml, w, h, dt):
    _check(fgml, synth.make_sample(w, h, 40 + w % 97), dt)
    # and once more straight after, on another image of the same size
    _check(fgml, synth.make_sample(w, h, 41 + w % 97), dt)


def test_noalloc_debug_range_check(fgml, monkeypatch):
    # FGML_DEBUG=1 checks the inputs here too, with the counter inside the fixed array
    s = synth.make_sample(64, 48, 4401)
    I, A = _dev(s.I), _dev(s.alpha)
    bad_I = I.clone()
    bad_I[2, 7, 0] = float("nan")
    bad_A = A.clone()
    bad_A[5, 1] = -0.25
    monkeypatch.setenv("FGML_DEBUG", "1")
    for bi, ba in ((bad_I, A), (I, bad_A)):
        with pytest.raises(fgml.FgmlError) as e:
            fgml.estimate_noalloc(bi, ba)
        assert e.value.status == fgml.FG_ERR_RANGE
    F, B = fgml.estimate_noalloc(I, A)   # clean inputs pass the check and solve
    fgml.sync()
    Fo, Bo = oracle.ml(s.I, s.alpha)
    assert max(_max_abs(F.cpu().numpy(), Fo), _max_abs(B.cpu().numpy(), Bo)) <= TOL


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
