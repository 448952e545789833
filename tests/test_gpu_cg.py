"""Converged reference (fg_minimiser_cg): the unclamped minimiser of the global cost by
float64 preconditioned conjugate gradients on the GPU, against the oracle's sparse direct
solve of the same stationarity conditions, and against the GPU's own unclamped
iteration run to convergence."""
import numpy as np
import pytest
import torch

from oracle import minimiser as om
from paper_2006_14970_gb300 import synth

pytestmark = pytest.mark.gpu

# fg_params carries eps_r and omega as float32: the oracle gets the same rounded values
EPS, OMEGA = float(np.float32(5e-3)), float(np.float32(0.1))


def _f32(v):
    return float(np.float32(v))


def _dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().to(dt)


@pytest.mark.parametrize("wh", [(1, 9), (9, 1), (37, 23), (64, 48), (200, 150)])
def test_cg_matches_sparse_direct_solve(fgml, wh):
    w, h = wh
    rng = np.random.default_rng(w * 100 + h)
    a = rng.random((h, w)).astype(np.float32)
    I = rng.random((h, w, 3)).astype(np.float32)
    F, B, it, rel = fgml.minimiser_cg(_dev(I), _dev(a), None, max_iters=50000, rel_tol=1e-13)
    assert rel <= 1e-12, (it, rel)
    # the GPU's x satisfies the oracle's stationarity conditions, and so lies within the
    # conditioning of the system of the direct solve
    Fg, Bg = F.cpu().numpy(), B.cpu().numpy()
    bnorm = np.sqrt(np.sum((a[..., None] * I) ** 2 + ((1 - a[..., None]) * I) ** 2))
    assert om.gradient_norm(I, a, Fg, Bg, EPS, OMEGA) <= 1e-11 * bnorm
    Fo, Bo = om.minimiser(I, a, EPS, OMEGA)
    assert np.abs(Fg - Fo).max() < 1e-9 and np.abs(Bg - Bo).max() < 1e-9


def test_cg_on_the_synthetic_workload_and_parameters(fgml):
    s = synth.make_sample(160, 120, 3000, hair=True)
    for eps, om_ in ((5e-3, 0.1), (0.05, 1.0)):
        p = fgml.params(eps_r=eps, omega=om_)
        F, B, it, rel = fgml.minimiser_cg(_dev(s.I), _dev(s.alpha), p, rel_tol=1e-12)
        Fo, Bo = om.minimiser(s.I, s.alpha, _f32(eps), _f32(om_))
        assert rel <= 1e-11
        assert np.abs(F.cpu().numpy() - Fo).max() < 1e-8 and np.abs(B.cpu().numpy() - Bo).max() < 1e-8


def test_cg_warm_start_and_16_bit_inputs(fgml):
    s = synth.make_sample(96, 80, 3100, hair=True)
    I, A = _dev(s.I, torch.bfloat16), _dev(s.alpha, torch.bfloat16)
    Fm, Bm = fgml.estimate(I, A)
    F, B, it, rel = fgml.minimiser_cg(I, A, None, Fm, Bm, rel_tol=1e-12)
    Fo, Bo = om.minimiser(I.float().cpu().numpy(), A.float().cpu().numpy(), EPS, OMEGA)
    assert rel <= 1e-11
    assert np.abs(F.cpu().numpy() - Fo).max() < 1e-8 and np.abs(B.cpu().numpy() - Bo).max() < 1e-8


def test_unclamped_gpu_iteration_converges_to_the_cg_minimiser(fgml):
    # many red-black iterations of the GPU level pass at full resolution, without the
    # clamp, reach the same stationary point as the float64 CG solve
    rng = np.random.default_rng(12)
    h, w = 24, 40
    a = rng.random((h, w)).astype(np.float32)
    I = rng.random((h, w, 3)).astype(np.float32)
    Id, Ad = _dev(I), _dev(a)
    Fm, Bm, _, _ = fgml.minimiser_cg(Id, Ad, None, rel_tol=1e-13)
    F0 = torch.zeros((h, w, 3), device="cuda")
    F, B = fgml.level_pass(Id, Ad, F0, F0, 3000, w, h, fgml.params(order=1, clamp=0))
    torch.cuda.synchronize()
    assert float((F.double() - Fm).abs().max()) < 2e-5 and float((B.double() - Bm).abs().max()) < 2e-5
