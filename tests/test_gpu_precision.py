"""Reduced-precision storage: I, alpha, F and B stored as bfloat16 or float16, every solve in
float32. Errors are measured against the FP64 oracle twice: on the original float32
inputs (end to end) and on the inputs rounded to the storage type (what the storage of
F and B between levels and at the output adds). The bounds are the measured errors of
the seeded workloads with a margin; each test prints what it measured."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14970_gb300 import synth

pytestmark = pytest.mark.gpu

# max-abs bounds per storage type: (vs oracle on rounded inputs, vs oracle on float32 inputs)
BOUNDS = {torch.bfloat16: (1.2e-2, 1.6e-2), torch.float16: (1.5e-3, 2.0e-3)}


def _errors(fgml, s, dt):
    I = torch.from_numpy(s.I).cuda().to(dt)
    A = torch.from_numpy(s.alpha).cuda().to(dt)
    F, B = fgml.estimate(I, A)
    torch.cuda.synchronize()
    F = F.float().cpu().numpy().astype(np.float64)
    B = B.float().cpu().numpy().astype(np.float64)
    Iq = I.float().cpu().numpy()
    Aq = A.float().cpu().numpy()
    Fq, Bq = oracle.ml(Iq, Aq)          # oracle on the rounded inputs
    Fo, Bo = oracle.ml(s.I, s.alpha)    # oracle on the float32 inputs
    out = {}
    for name, (x, y) in {"q": ((F, B), (Fq, Bq)), "e2e": ((F, B), (Fo, Bo))}.items():
        d = np.concatenate([np.abs(x[0] - y[0]), np.abs(x[1] - y[1])], axis=-1)
        out[name] = (float(d.max()), float(d.mean()), d.reshape(-1, 6).max(axis=0).tolist())
    return out


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
@pytest.mark.parametrize("name", ["single_128x128", "single_2048x1536_hair"])
def test_reduced_precision_error_bounds(fgml, dt, name):
    s = synth.workload(name)
    e = _errors(fgml, s, dt)
    print(f"{name} {dt}: max/mean abs vs oracle(rounded inputs) {e['q'][0]:.2e}/{e['q'][1]:.2e}"
          f", vs oracle(float32 inputs) {e['e2e'][0]:.2e}/{e['e2e'][1]:.2e}; per channel "
          f"(F rgb, B rgb) {['%.1e' % v for v in e['e2e'][2]]}")
    bq, be = BOUNDS[dt]
    assert e["q"][0] <= bq and e["e2e"][0] <= be


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_reduced_precision_8k(fgml, dt):
    s = synth.workload("single_7680x4320")
    e = _errors(fgml, s, dt)
    print(f"7680x4320 {dt}: max/mean abs vs oracle(rounded inputs) {e['q'][0]:.2e}/{e['q'][1]:.2e}"
          f", vs oracle(float32 inputs) {e['e2e'][0]:.2e}/{e['e2e'][1]:.2e}")
    bq, be = BOUNDS[dt]
    assert e["q"][0] <= bq and e["e2e"][0] <= be


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_reduced_precision_ragged_and_host_path(fgml, dt):
    s = synth.make_sample(1939, 611, 77)
    e = _errors(fgml, s, dt)
    bq, be = BOUNDS[dt]
    assert e["q"][0] <= bq and e["e2e"][0] <= be
    # the host-buffer entry point gives the same bits as the device one
    I = torch.from_numpy(s.I).to(dt)
    A = torch.from_numpy(s.alpha).to(dt)
    Fd, Bd = fgml.estimate(I.cuda(), A.cuda())
    torch.cuda.synchronize()
    Fh, Bh = fgml.estimate_host(I.pin_memory(), A.pin_memory())
    assert torch.equal(Fh, Fd.cpu()) and torch.equal(Bh, Bd.cpu())
