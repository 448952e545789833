"""Error measures on the GPU (fg_quality) against the FP64 oracle's measures (Section
IV-C), on the solver's own output for the seeded workloads with the generator's known
foreground, plus degenerate mattes, tiny and ragged images and 16-bit storage."""
import numpy as np
import pytest
import torch

import oracle
from oracle import quality as oq
from paper_2006_14970_gb300 import synth

pytestmark = pytest.mark.gpu


def _dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().to(dt)


def _check(got, want, rel):
    for k in ("sad", "mse", "grad"):
        assert got[k] == pytest.approx(want[k], rel=rel, abs=1e-9), (k, got, want)


@pytest.mark.parametrize("name", ["single_128x128", "single_2048x1536_hair"])
def test_quality_of_the_estimate_matches_oracle(fgml, name):
    s = synth.workload(name)
    I, A = _dev(s.I), _dev(s.alpha)
    F, _ = fgml.estimate(I, A)
    got = fgml.quality(F, _dev(s.F), A)
    want = oq.measures(F.cpu().numpy(), s.F, s.alpha)
    print(name, got, want["pixels"])
    _check(got, want, 2e-5)


@pytest.mark.parametrize("wh", [(1, 1), (5, 3), (13, 40), (1939, 611)])
def test_quality_ragged_and_tiny(fgml, wh):
    w, h = wh
    rng = np.random.default_rng(w * 7 + h)
    Fe = rng.random((h, w, 3), dtype=np.float32)
    Fg = rng.random((h, w, 3), dtype=np.float32)
    a = rng.choice(np.array([0.0, 1.0, 0.3, 0.75], np.float32), size=(h, w))
    got = fgml.quality(_dev(Fe), _dev(Fg), _dev(a))
    _check(got, oq.measures(Fe, Fg, a), 2e-5)


def test_quality_binary_matte_is_zero(fgml):
    rng = np.random.default_rng(2)
    Fe = rng.random((64, 80, 3), dtype=np.float32)
    a = (rng.random((64, 80)) > 0.5).astype(np.float32)
    got = fgml.quality(_dev(Fe), _dev(np.zeros_like(Fe)), _dev(a))
    assert got == {"sad": 0.0, "mse": 0.0, "grad": 0.0}


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_quality_reduced_precision_inputs(fgml, dt):
    s = synth.make_sample(300, 200, 77, hair=True)
    Fe = _dev(s.F + 0.01 * np.sin(np.arange(300))[None, :, None], dt)
    Fg, A = _dev(s.F, dt), _dev(s.alpha, dt)
    got = fgml.quality(Fe, Fg, A)
    want = oq.measures(Fe.float().cpu().numpy(), Fg.float().cpu().numpy(), A.float().cpu().numpy())
    _check(got, want, 1e-4)


def test_regularisation_sweep_grid(fgml):
    from paper_2006_14970_gb300 import sweep
    ss = [synth.make_sample(256, 192, 900 + i, hair=True) for i in range(2)]
    imgs = [(_dev(s.I), _dev(s.alpha), _dev(s.F)) for s in ss]
    rows = sweep.regularisation_sweep(imgs, [1e-3, 5e-3, 5e-2], [0.0, 0.1, 1.0])
    assert [(r["eps_r"], r["omega"]) for r in rows] == \
        [(e, o) for e in (1e-3, 5e-3, 5e-2) for o in (0.0, 0.1, 1.0)]
    assert all(np.isfinite([r["sad"], r["mse"], r["grad"]]).all() for r in rows)
    # the paper's point of the grid equals one solve plus one measure per image, and the
    # oracle's measures of the GPU's estimates
    r = rows[4]
    want = {"sad": 0.0, "mse": 0.0, "grad": 0.0}
    for (I, A, Ft), s in zip(imgs, ss):
        F, _ = fgml.estimate(I, A, fgml.params(eps_r=5e-3, omega=0.1))
        m = oq.measures(F.cpu().numpy(), s.F, s.alpha)
        for k in want:
            want[k] += m[k]
    _check(r, want, 2e-5)
