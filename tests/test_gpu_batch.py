"""Work-list batches: many images of uneven sizes in one coarse launch plus one persistent
launch. Every image must match its single-image result and the FP64 oracle within the
parity tolerance; the bounded dependency wait must give up cleanly when its count is
never reached."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14970_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _dev(a, dt=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda().to(dt)


def _samples(sizes, seed):
    return [synth.make_sample(w, h, seed + i) for i, (w, h) in enumerate(sizes)]


def test_batch_uneven_sizes_matches_single_and_oracle(fgml):
    sizes = [(1, 1), (5, 3), (40, 33), (64, 64), (77, 301), (300, 200), (517, 389), (1000, 97),
             (33, 1024), (1939, 611)]
    ss = _samples(sizes, 500)
    imgs = [(_dev(s.I), _dev(s.alpha)) for s in ss]
    out = fgml.estimate_batch(imgs)
    fgml.sync()
    for (I, A), (F, B), s in zip(imgs, out, ss):
        Fs, Bs = fgml.estimate(I, A)
        torch.cuda.synchronize()
        assert float((F - Fs).abs().max()) <= TOL and float((B - Bs).abs().max()) <= TOL
        Fo, Bo = oracle.ml(s.I, s.alpha)
        assert np.abs(F.cpu().numpy() - Fo).max() <= TOL
        assert np.abs(B.cpu().numpy() - Bo).max() <= TOL


def test_batch_repeated_and_reordered(fgml):
    sizes = [(256, 300), (640, 480), (128, 1024)]
    ss = _samples(sizes, 600)
    imgs = [(_dev(s.I), _dev(s.alpha)) for s in ss]
    a = fgml.estimate_batch(imgs)
    b = fgml.estimate_batch(imgs[::-1])[::-1]
    c = fgml.estimate_batch(imgs)
    fgml.sync()
    for x, y, z in zip(a, b, c):
        assert torch.equal(x[0], z[0]) and torch.equal(x[1], z[1])
        assert float((x[0] - y[0]).abs().max()) <= TOL and float((x[1] - y[1]).abs().max()) <= TOL


def test_batch_replay_reads_new_contents_and_keeps_its_own_work_list(fgml):
    # a repeated batch (same buffers) replays its cached launch graph: it must read what the
    # buffers hold now, and two batches alternating on one stream must not share work lists
    ss1 = _samples([(300, 211), (1939, 611), (64, 64)], 900)
    ss2 = _samples([(517, 389), (128, 1024)], 910)
    new1 = _samples([(300, 211), (1939, 611), (64, 64)], 920)
    imgs1 = [(_dev(s.I), _dev(s.alpha)) for s in ss1]
    imgs2 = [(_dev(s.I), _dev(s.alpha)) for s in ss2]
    out1 = [(torch.empty_like(I), torch.empty_like(I)) for I, _ in imgs1]
    out2 = [(torch.empty_like(I), torch.empty_like(I)) for I, _ in imgs2]
    for rep in range(3):
        fgml.estimate_batch(imgs1, outputs=out1)
        fgml.estimate_batch(imgs2, outputs=out2)
    fgml.sync()
    for (F, B), s in zip(out1 + out2, ss1 + ss2):
        Fo, Bo = oracle.ml(s.I, s.alpha)
        assert np.abs(F.cpu().numpy() - Fo).max() <= TOL
        assert np.abs(B.cpu().numpy() - Bo).max() <= TOL
    # new contents in the same input buffers, outputs poisoned first
    for (I, A), s in zip(imgs1, new1):
        I.copy_(_dev(s.I))
        A.copy_(_dev(s.alpha))
    for F, B in out1:
        F.fill_(float("nan"))
        B.fill_(float("nan"))
    fgml.estimate_batch(imgs1, outputs=out1)
    fgml.sync()
    for (F, B), s in zip(out1, new1):
        Fo, Bo = oracle.ml(s.I, s.alpha)
        assert np.abs(F.cpu().numpy() - Fo).max() <= TOL
        assert np.abs(B.cpu().numpy() - Bo).max() <= TOL


def test_batch_replay_reads_new_contents_and_keeps_its_own_work_list(fgml):
    # a batch seen a second time (same buffers) is captured and then replayed: it must read
    # what the buffers hold now, and two batches alternating on one stream must not share
    # work lists
    ss1 = _samples([(300, 211), (1939, 611), (64, 64)], 900)
    ss2 = _samples([(517, 389), (128, 1024)], 910)
    new1 = _samples([(300, 211), (1939, 611), (64, 64)], 920)
    imgs1 = [(_dev(s.I), _dev(s.alpha)) for s in ss1]
    imgs2 = [(_dev(s.I), _dev(s.alpha)) for s in ss2]
    out1 = [(torch.empty_like(I), torch.empty_like(I)) for I, _ in imgs1]
    out2 = [(torch.empty_like(I), torch.empty_like(I)) for I, _ in imgs2]
    for rep in range(3):
        fgml.estimate_batch(imgs1, outputs=out1)
        fgml.estimate_batch(imgs2, outputs=out2)
    fgml.sync()
    for (F, B), s in zip(out1 + out2, ss1 + ss2):
        Fo, Bo = oracle.ml(s.I, s.alpha)
        assert np.abs(F.cpu().numpy() - Fo).max() <= TOL
        assert np.abs(B.cpu().numpy() - Bo).max() <= TOL
    # new contents in the same input buffers, outputs poisoned first
    for (I, A), s in zip(imgs1, new1):
        I.copy_(_dev(s.I))
        A.copy_(_dev(s.alpha))
    for F, B in out1:
        F.fill_(float("nan"))
        B.fill_(float("nan"))
    fgml.estimate_batch(imgs1, outputs=out1)
    fgml.sync()
    for (F, B), s in zip(out1, new1):
        Fo, Bo = oracle.ml(s.I, s.alpha)
        assert np.abs(F.cpu().numpy() - Fo).max() <= TOL
        assert np.abs(B.cpu().numpy() - Bo).max() <= TOL


@pytest.mark.parametrize("dt", [torch.bfloat16, torch.float16])
def test_batch_reduced_precision_within_bound(fgml, dt):
    # each level's F and B are rounded to the storage type, so the batch and the
    # single-image kernels may differ by a few units of the last place; both must stay
    # within the stated reduced-precision bound of the oracle on the rounded inputs
    bound = {torch.bfloat16: 1.2e-2, torch.float16: 1.5e-3}[dt]
    ss = _samples([(300, 211), (1024, 768), (70, 900)], 700)
    imgs = [(_dev(s.I, dt), _dev(s.alpha, dt)) for s in ss]
    out = fgml.estimate_batch(imgs)
    fgml.sync()
    for (I, A), (F, B) in zip(imgs, out):
        Fo, Bo = oracle.ml(I.float().cpu().numpy(), A.float().cpu().numpy())
        assert np.abs(F.float().cpu().numpy() - Fo).max() <= bound
        assert np.abs(B.float().cpu().numpy() - Bo).max() <= bound


def test_batch_parameters(fgml):
    ss = _samples([(181, 97), (400, 257)], 800)
    imgs = [(_dev(s.I), _dev(s.alpha)) for s in ss]
    for kw in [dict(clamp=0), dict(small_iters=3, big_iters=5), dict(big_iters=0),
               dict(eps_r=0.02, omega=1.0)]:
        p = fgml.params(**kw)
        out = fgml.estimate_batch(imgs, p)
        fgml.sync()
        for (I, A), (F, B) in zip(imgs, out):
            Fs, Bs = fgml.estimate(I, A, p)
            torch.cuda.synchronize()
            tol = TOL if kw.get("clamp", 1) else 5e-4
            assert float((F - Fs).abs().max()) <= tol and float((B - Bs).abs().max()) <= tol, kw


def test_batch_of_64_uneven_images(fgml):
    # the batched workload: 64 images, sides log-uniform in [256, 2048]
    ss = synth.batch(64)
    imgs = [(_dev(s.I), _dev(s.alpha)) for s in ss]
    out = fgml.estimate_batch(imgs)
    fgml.sync()
    for k, ((I, A), (F, B)) in enumerate(zip(imgs, out)):
        Fs, Bs = fgml.estimate(I, A)
        torch.cuda.synchronize()
        assert float((F - Fs).abs().max()) <= TOL and float((B - Bs).abs().max()) <= TOL, k
    for k in (0, 17, 42):
        Fo, Bo = oracle.ml(ss[k].I, ss[k].alpha)
        assert np.abs(out[k][0].cpu().numpy() - Fo).max() <= TOL
        assert np.abs(out[k][1].cpu().numpy() - Bo).max() <= TOL


def test_bounded_wait_gives_up_and_context_survives(fgml):
    st = fgml.selftest_bounded_wait()
    assert st == fgml.FG_ERR_TIMEOUT, fgml.load().fg_last_error()
    # the device is still usable and the error word is clear again
    s = synth.make_sample(200, 150, 900)
    F, B = fgml.estimate(_dev(s.I), _dev(s.alpha))
    fgml.sync()
    Fo, Bo = oracle.ml(s.I, s.alpha)
    assert np.abs(F.cpu().numpy() - Fo).max() <= TOL


def test_autotune_picks_a_strip_shape_and_results_do_not_change(fgml):
    ss = _samples([(300, 211), (1024, 768), (77, 900), (640, 480)], 1000)
    imgs = [(_dev(s.I), _dev(s.alpha)) for s in ss]
    before = fgml.estimate_batch(imgs)
    fgml.sync()
    chosen, ms = fgml.autotune_batch(imgs)
    assert 0 <= chosen < 6 and ms > 0
    after = fgml.estimate_batch(imgs)
    fgml.sync()
    for (F0, B0), (F1, B1) in zip(before, after):
        assert torch.equal(F0, F1) and torch.equal(B0, B1)


def test_autotune_writes_the_tune_cache(fgml, tmp_path, monkeypatch):
    path = tmp_path / "tune.txt"
    path.write_text("Some Other GPU\t1,2,3\n")
    monkeypatch.setenv("FGML_TUNE_CACHE", str(path))
    ss = _samples([(300, 211), (640, 480)], 1100)
    imgs = [(_dev(s.I), _dev(s.alpha)) for s in ss]
    chosen, _ = fgml.autotune_batch(imgs)
    lines = path.read_text().splitlines()
    assert lines[0] == "Some Other GPU\t1,2,3"          # other models' lines are kept
    name = torch.cuda.get_device_name(0)
    mine = [l for l in lines if l.startswith(name + "\t")]
    assert len(mine) == 1
    per_sm, lo, hi = (int(v) for v in mine[0].split("\t")[1].split(","))
    assert per_sm > 0 and 0 < lo <= hi
