"""Red-black order on the GPU: every level's iterations update the pixels with x + y even,
then those with x + y odd, each colour in place. Compared element by element with the
FP64 oracle's red-black mode (same visiting order, so the same iterates up to float32
rounding) at sizes that span several tiles and ragged edges, on single level passes and
on the whole multi-level method."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14970_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4
RB = 1


def _dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().to(dt)


def _max_err(F, B, Fo, Bo):
    return max(np.abs(F.float().cpu().numpy() - Fo).max(), np.abs(B.float().cpu().numpy() - Bo).max())


@pytest.mark.parametrize("wh", [(1, 1), (2, 3), (5, 3), (33, 17), (64, 64), (128, 128), (300, 200),
                                (517, 389), (1939, 611), (77, 1301)])
def test_estimate_redblack_matches_oracle(fgml, wh):
    w, h = wh
    s = synth.make_sample(w, h, 1200 + w + h, hair=w >= 300)
    F, B = fgml.estimate(_dev(s.I), _dev(s.alpha), fgml.params(order=RB))
    torch.cuda.synchronize()
    Fo, Bo = oracle.ml(s.I, s.alpha, oracle.Params(order=oracle.REDBLACK))
    assert _max_err(F, B, Fo, Bo) <= TOL


def test_estimate_redblack_workload_2048x1536(fgml):
    s = synth.workload("single_2048x1536_hair")
    F, B = fgml.estimate(_dev(s.I), _dev(s.alpha), fgml.params(order=RB))
    torch.cuda.synchronize()
    Fo, Bo = oracle.ml(s.I, s.alpha, oracle.Params(order=oracle.REDBLACK))
    assert _max_err(F, B, Fo, Bo) <= TOL


@pytest.mark.parametrize("kw", [dict(clamp=0), dict(small_iters=3, big_iters=5), dict(big_iters=1),
                                dict(big_iters=0), dict(eps_r=0.02, omega=1.0), dict(init=0.5)])
def test_estimate_redblack_parameters(fgml, kw):
    s = synth.make_sample(403, 257, 1300)
    F, B = fgml.estimate(_dev(s.I), _dev(s.alpha), fgml.params(order=RB, **kw))
    torch.cuda.synchronize()
    Fo, Bo = oracle.ml(s.I, s.alpha, oracle.Params(order=oracle.REDBLACK, **kw))
    tol = TOL if kw.get("clamp", 1) else 5e-4
    assert _max_err(F, B, Fo, Bo) <= tol, kw


@pytest.mark.parametrize("case", [(128, 96, 64, 48, 1), (128, 96, 64, 48, 2), (200, 100, 100, 50, 3),
                                  (1000, 37, 497, 19, 2), (33, 700, 33, 700, 4)])
def test_level_pass_redblack(fgml, case):
    # one level from a given start: the oracle resizes I, alpha and the start by the same
    # nearest rule and runs its red-black iterations
    w, h, sw, sh, iters = case
    s = synth.make_sample(w, h, 1400 + iters)
    rng = np.random.default_rng(1400 + w)
    Fs = rng.random((sh, sw, 3), dtype=np.float32)
    Bs = rng.random((sh, sw, 3), dtype=np.float32)
    F, B = fgml.level_pass(_dev(s.I), _dev(s.alpha), _dev(Fs), _dev(Bs), iters, w, h,
                           fgml.params(order=RB))
    torch.cuda.synchronize()
    F0 = oracle.resize_nearest(Fs.astype(np.float64), w, h)
    B0 = oracle.resize_nearest(Bs.astype(np.float64), w, h)
    Fo, Bo = oracle.level_iterate(s.I, s.alpha, F0, B0, iters, oracle.Params(order=oracle.REDBLACK))
    assert _max_err(F, B, Fo, Bo) <= TOL


def test_redblack_is_not_jacobi_and_batch_matches_single(fgml):
    s = synth.make_sample(300, 211, 1500, hair=True)
    I, A = _dev(s.I), _dev(s.alpha)
    Fj, _ = fgml.estimate(I, A)
    Fr, Br = fgml.estimate(I, A, fgml.params(order=RB))
    out = fgml.estimate_batch([(I, A), (I, A)], fgml.params(order=RB))
    torch.cuda.synchronize()
    assert float((Fj - Fr).abs().max()) > 1e-3      # a different iteration
    for F, B in out:
        assert torch.equal(F, Fr) and torch.equal(B, Br)


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_redblack_reduced_precision(fgml, dt):
    bound = {torch.bfloat16: 1.2e-2, torch.float16: 1.5e-3}[dt]
    s = synth.make_sample(640, 480, 1600, hair=True)
    I, A = _dev(s.I, dt), _dev(s.alpha, dt)
    F, B = fgml.estimate(I, A, fgml.params(order=RB))
    torch.cuda.synchronize()
    Fo, Bo = oracle.ml(I.float().cpu().numpy(), A.float().cpu().numpy(),
                       oracle.Params(order=oracle.REDBLACK))
    assert _max_err(F, B, Fo, Bo) <= bound
