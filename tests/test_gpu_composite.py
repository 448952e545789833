"""Compositing epilogue (fg_estimate_composite): I_new = alpha F + (1 - alpha) B_new formed
by the last level's pass. F and B must equal fg_estimate's bit for bit; I_new must equal
the composite of that F (float32 arithmetic, one rounding) and match the oracle's
composite of the oracle's F within the parity tolerance, on every kernel that can run the
last level: coarse-only images, the small-level and tile kernels, a zero-sweep top level
and the red-black kernel."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14970_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().to(dt)


CASES = [((32, 30), {}), ((128, 128), {}), ((1939, 611), {}), ((2048, 1536), {}),
         ((403, 257), {"big_iters": 0}), ((403, 257), {"order": 1}), ((517, 389), {"clamp": 0})]


@pytest.mark.parametrize("wh,kw", CASES)
def test_composite_matches_estimate_and_oracle(fgml, wh, kw):
    w, h = wh
    s = synth.make_sample(w, h, 2000 + w, hair=w >= 300)
    Bn = np.random.default_rng(w + h).random((h, w, 3), dtype=np.float32)
    I, A, Bnd = _dev(s.I), _dev(s.alpha), _dev(Bn)
    p = fgml.params(**kw)
    F0, B0 = fgml.estimate(I, A, p)
    F, B, In = fgml.estimate_composite(I, A, Bnd, p)
    torch.cuda.synchronize()
    assert torch.equal(F, F0) and torch.equal(B, B0)
    # the composite of the stored F, recomputed on the host
    a64 = s.alpha.astype(np.float64)[..., None]
    want = a64 * F.cpu().numpy() + (1 - a64) * Bn
    assert np.abs(In.cpu().numpy() - want).max() <= 4e-7
    # and against the oracle's estimate
    Fo, _ = oracle.ml(s.I, s.alpha, oracle.Params(**kw))
    tol = TOL if kw.get("clamp", 1) else 5e-4
    assert np.abs(In.cpu().numpy() - oracle.composite(s.alpha, Fo, Bn)).max() <= tol


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_composite_reduced_precision(fgml, dt):
    s = synth.make_sample(640, 480, 2100, hair=True)
    Bn = np.random.default_rng(5).random((480, 640, 3), dtype=np.float32)
    I, A, Bnd = _dev(s.I, dt), _dev(s.alpha, dt), _dev(Bn, dt)
    F, B, In = fgml.estimate_composite(I, A, Bnd)
    torch.cuda.synchronize()
    a = A.double().cpu().numpy()[..., None]
    want = a * F.double().cpu().numpy() + (1 - a) * Bnd.double().cpu().numpy()
    ulp = {torch.bfloat16: 2 ** -8, torch.float16: 2 ** -11}[dt]
    assert np.abs(In.double().cpu().numpy() - want).max() <= ulp


def test_composite_rejects_overlap(fgml):
    s = synth.make_sample(64, 48, 3)
    I, A = _dev(s.I), _dev(s.alpha)
    with pytest.raises(fgml.FgmlError):
        fgml.estimate_composite(I, A, I.clone(), I_new=I)
