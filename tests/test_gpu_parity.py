"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle, element by
element on the same seeded inputs. Bar: max-abs <= 1e-4 per channel in float32."""
import numpy as np
import pytest
import torch

import oracle
from paper_2006_14970_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _dev(a, dtype=torch.float32):
    return torch.from_numpy(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def _random_inputs(w, h, seed):
    rng = np.random.default_rng(seed)
    if w * h >= 64 * 64:
        s = synth.make_sample(w, h, seed)
        return s.I, s.alpha
    a = rng.random((h, w)).astype(np.float32)
    a[rng.random((h, w)) < 0.3] = 0.0
    a[rng.random((h, w)) < 0.3] = 1.0
    return rng.random((h, w, 3)).astype(np.float32), a


def _gpu_ml(fgml, I, a, p=None):
    F, B = fgml.estimate(_dev(I), _dev(a), p)
    torch.cuda.synchronize()
    return F.cpu().numpy().astype(np.float64), B.cpu().numpy().astype(np.float64)


def _maxabs(x, y):
    return [float(np.max(np.abs(x[..., c] - y[..., c]))) for c in range(x.shape[-1])]


def _assert_close(F, B, Fo, Bo, tol=TOL, what=""):
    eF, eB = _maxabs(F, Fo), _maxabs(B, Bo)
    assert max(eF) <= tol and max(eB) <= tol, f"{what} max-abs F {eF} B {eB}"


@pytest.mark.parametrize("name", ["single_128x128", "single_2048x1536_hair"])
def test_workload_parity(fgml, name):
    s = synth.workload(name)
    F, B = _gpu_ml(fgml, s.I, s.alpha)
    Fo, Bo = oracle.ml(s.I, s.alpha)
    _assert_close(F, B, Fo, Bo, what=name)


SIZES = [(1, 1), (2, 1), (1, 2), (3, 1), (1, 37), (5, 7), (33, 31), (64, 64), (65, 64),
         (61, 67), (127, 3), (3, 127), (300, 201), (1000, 17), (17, 1000), (4097, 3),
         (121, 122), (259, 260), (1939, 1192)]


@pytest.mark.parametrize("w,h", SIZES)
def test_ragged_and_degenerate_sizes(fgml, w, h):
    I, a = _random_inputs(w, h, 1000 + w * 7 + h)
    F, B = _gpu_ml(fgml, I, a)
    Fo, Bo = oracle.ml(I, a)
    _assert_close(F, B, Fo, Bo, what=f"{w}x{h}")


@pytest.mark.parametrize("kw", [dict(clamp=0), dict(init=0.5), dict(eps_r=0.02, omega=1.0),
                                dict(small_iters=3, big_iters=5), dict(big_iters=1),
                                dict(big_iters=0), dict(small_size=100, small_iters=4),
                                dict(omega=0.0)])
def test_parameters(fgml, kw):
    I, a = _random_inputs(181, 97, 5)
    p = fgml.params(**kw)
    F, B = _gpu_ml(fgml, I, a, p)
    okw = {k: (bool(v) if k == "clamp" else v) for k, v in kw.items()}
    Fo, Bo = oracle.ml(I, a, oracle.Params(**okw))
    tol = TOL if kw.get("clamp", 1) else 5e-4
    _assert_close(F, B, Fo, Bo, tol=tol, what=str(kw))


@pytest.mark.parametrize("iters", [0, 1, 2, 3, 4, 7])
@pytest.mark.parametrize("w,h,sw,sh,Iw,Ih", [(130, 70, 66, 35, 260, 140), (61, 200, 61, 200, 61, 200),
                                             (500, 9, 251, 5, 1001, 17), (7, 3, 2, 2, 7, 3),
                                             (128, 96, 64, 48, 128, 96),
                                             (200, 100, 200, 100, 200, 100),
                                             (1000, 37, 497, 19, 1000, 37)])
def test_level_pass_against_oracle_sweeps(fgml, iters, w, h, sw, sh, Iw, Ih):
    rng = np.random.default_rng(iters * 100 + w)
    I = rng.random((Ih, Iw, 3)).astype(np.float32)
    a = rng.random((Ih, Iw)).astype(np.float32)
    Fs = rng.random((sh, sw, 3)).astype(np.float32)
    Bs = rng.random((sh, sw, 3)).astype(np.float32)
    F, B = fgml.level_pass(_dev(I), _dev(a), _dev(Fs), _dev(Bs), iters, w, h)
    torch.cuda.synchronize()
    Il, al = oracle.resize_nearest(I, w, h), oracle.resize_nearest(a, w, h)
    Fo, Bo = oracle.level_iterate(Il, al, oracle.resize_nearest(Fs, w, h),
                                  oracle.resize_nearest(Bs, w, h), iters)
    _assert_close(F.cpu().numpy().astype(np.float64), B.cpu().numpy().astype(np.float64),
                  Fo, Bo, what=f"iters={iters}")


def test_pitched_inputs_and_outputs(fgml):
    I, a = _random_inputs(203, 150, 9)
    Ib = torch.zeros((150, 260, 3), device="cuda")
    Ab = torch.zeros((150, 230), device="cuda")
    Ib[:, :203] = _dev(I)
    Ab[:, :203] = _dev(a)
    Fb = torch.full((150, 211, 3), -7.0, device="cuda")
    Bb = torch.full((150, 211, 3), -7.0, device="cuda")
    fgml.estimate(Ib[:, :203], Ab[:, :203], None, Fb[:, :203], Bb[:, :203])
    torch.cuda.synchronize()
    Fo, Bo = oracle.ml(I, a)
    _assert_close(Fb[:, :203].cpu().numpy().astype(np.float64),
                  Bb[:, :203].cpu().numpy().astype(np.float64), Fo, Bo, what="pitched")
    # nothing written outside the images
    assert bool((Fb[:, 203:] == -7.0).all()) and bool((Bb[:, 203:] == -7.0).all())


def test_every_output_pixel_is_written(fgml):
    I, a = _random_inputs(613, 419, 10)
    F = torch.full((419, 613, 3), float("nan"), device="cuda")
    B = torch.full((419, 613, 3), float("nan"), device="cuda")
    fgml.estimate(_dev(I), _dev(a), None, F, B)
    torch.cuda.synchronize()
    assert not bool(torch.isnan(F).any()) and not bool(torch.isnan(B).any())


def test_exact_invariants_on_gpu(fgml):
    h, w = 211, 307
    I = np.full((h, w, 3), 0.37, np.float32)
    F, B = _gpu_ml(fgml, I, np.ones((h, w), np.float32))
    assert np.all(B == 0.0) and np.max(np.abs(F - 0.37)) < 1e-6
    F, B = _gpu_ml(fgml, I, np.zeros((h, w), np.float32))
    assert np.all(F == 0.0) and np.max(np.abs(B - 0.37)) < 1e-6
    Ir, ar = _random_inputs(w, h, 11)
    F, B = _gpu_ml(fgml, Ir, ar)
    assert F.min() >= 0 and F.max() <= 1 and B.min() >= 0 and B.max() <= 1


def test_host_entry_point_matches_device_entry_point(fgml):
    s = synth.make_sample(517, 389, 12)
    Fd, Bd = fgml.estimate(_dev(s.I), _dev(s.alpha))
    torch.cuda.synchronize()
    Fh, Bh = fgml.estimate_host(torch.from_numpy(s.I).pin_memory(),
                                torch.from_numpy(s.alpha).pin_memory())
    assert torch.equal(Fh, Fd.cpu()) and torch.equal(Bh, Bd.cpu())


def test_repeated_calls_and_streams_are_deterministic(fgml):
    s = synth.make_sample(700, 500, 13)
    I, a = _dev(s.I), _dev(s.alpha)
    F1, B1 = fgml.estimate(I, a)
    st = torch.cuda.Stream()
    with torch.cuda.stream(st):
        F2, B2 = fgml.estimate(I, a)
    st.synchronize()
    torch.cuda.synchronize()
    F3, B3 = fgml.estimate(I, a)
    torch.cuda.synchronize()
    assert torch.equal(F1, F2) and torch.equal(B1, B2)
    assert torch.equal(F1, F3) and torch.equal(B1, B3)


def test_full_size_8k_parity(fgml):
    s = synth.workload("single_7680x4320")
    F, B = _gpu_ml(fgml, s.I, s.alpha)
    Fo, Bo = oracle.ml(s.I, s.alpha)
    _assert_close(F, B, Fo, Bo, what="7680x4320")


def test_unaligned_base_pointers(fgml):
    # image rows and bases off the 16-byte grid: the row ring copies such segments by
    # lanes instead of bulk copies, with the same results
    for w, h, off in [(301, 97, 1), (1939, 64, 3), (64, 40, 2)]:
        I, a = _random_inputs(w, h, 40 + off)
        Ib = torch.empty(h * w * 3 + off, device="cuda")
        Ab = torch.empty(h * w + off, device="cuda")
        Iv = Ib[off:].view(h, w, 3)
        Av = Ab[off:].view(h, w)
        Iv.copy_(_dev(I))
        Av.copy_(_dev(a))
        Fb = torch.empty(h * w * 3 + off, device="cuda")
        Bb = torch.empty(h * w * 3 + off, device="cuda")
        F, B = fgml.estimate(Iv, Av, None, Fb[off:].view(h, w, 3), Bb[off:].view(h, w, 3))
        torch.cuda.synchronize()
        Fo, Bo = oracle.ml(I, a)
        _assert_close(F.cpu().numpy().astype(np.float64), B.cpu().numpy().astype(np.float64),
                      Fo, Bo, what=f"unaligned {w}x{h}+{off}")
    fgml.sync()   # no bounded wait gave up


@pytest.mark.parametrize("wh", [(2047, 1535), (1939, 611)])
def test_packed_rows_off_the_grid_equal_padded_rows(fgml, wh):
    # tightly packed rows whose width is not a multiple of 16 bytes go through the
    # library's row-aligned copy; the same image in 16-byte padded rows does not: both
    # must give the same bits, and match the oracle
    w, h = wh
    s = synth.make_sample(w, h, 4100 + w, hair=True)
    I = torch.from_numpy(s.I).cuda()
    A = torch.from_numpy(s.alpha).cuda()
    pitch = (3 * w + 3) // 4 * 4
    Ip = torch.zeros((h, pitch), device="cuda")[:, :3 * w].view(h, w, 3)
    Ap = torch.zeros((h, (w + 3) // 4 * 4), device="cuda")[:, :w]
    Ip.copy_(I)
    Ap.copy_(A)
    F1, B1 = fgml.estimate(I, A)
    F2, B2 = fgml.estimate(Ip, Ap)
    torch.cuda.synchronize()
    assert torch.equal(F1, F2) and torch.equal(B1, B2)
    Fo, Bo = oracle.ml(s.I, s.alpha)
    assert np.abs(F1.cpu().numpy() - Fo).max() <= 1e-4 and np.abs(B1.cpu().numpy() - Bo).max() <= 1e-4


def test_host_entry_points_sync_and_pipelined(fgml):
    # host buffers in and out: the synchronous call, and a pipelined sequence on two streams
    # of the asynchronous one, give the device path's bits for every image
    ss = [synth.make_sample(w, h, 4300 + w) for w, h in ((640, 480), (1023, 767), (333, 1025))]
    want = []
    for s in ss:
        F, B = fgml.estimate(torch.from_numpy(s.I).cuda(), torch.from_numpy(s.alpha).cuda())
        torch.cuda.synchronize()
        want.append((F.cpu(), B.cpu()))
    hs = [(torch.from_numpy(s.I).pin_memory(), torch.from_numpy(s.alpha).pin_memory()) for s in ss]
    for (I, A), (Fw, Bw) in zip(hs, want):
        F, B = fgml.estimate_host(I, A)
        assert torch.equal(F, Fw) and torch.equal(B, Bw)
    streams = [torch.cuda.Stream(), torch.cuda.Stream()]
    outs = []
    for k in range(6):
        I, A = hs[k % 3]
        outs.append(fgml.estimate_host_async(I, A, stream=streams[k % 2]))
    torch.cuda.synchronize()
    for k, (F, B) in enumerate(outs):
        assert torch.equal(F, want[k % 3][0]) and torch.equal(B, want[k % 3][1])


def test_debug_input_range_check(fgml, monkeypatch):
    s = synth.make_sample(64, 48, 4400)
    I = torch.from_numpy(s.I).cuda()
    A = torch.from_numpy(s.alpha).cuda()
    nan_I = I.clone()
    nan_I[3, 5, 1] = float("nan")
    big_A = A.clone()
    big_A[0, 0] = 1.5
    monkeypatch.setenv("FGML_DEBUG", "1")
    for bi, ba in ((nan_I, A), (I, big_A)):
        with pytest.raises(fgml.FgmlError) as e:
            fgml.estimate(bi, ba)
        assert e.value.status == fgml.FG_ERR_RANGE
    F, B = fgml.estimate(I, A)
    torch.cuda.synchronize()
    monkeypatch.delenv("FGML_DEBUG")
    fgml.estimate(nan_I, A)      # unchecked: the call itself succeeds
    torch.cuda.synchronize()


def test_allocation_failure_is_reported_and_recoverable(fgml, monkeypatch):
    # the workspace of a fresh stream cannot grow: the call reports FG_ERR_OOM, launches
    # nothing, and works once allocation is allowed again
    s = synth.make_sample(700, 500, 4500)
    I = torch.from_numpy(s.I).cuda()
    A = torch.from_numpy(s.alpha).cuda()
    st = torch.cuda.Stream()
    monkeypatch.setenv("FGML_FAIL_ALLOC", "1")
    with pytest.raises(fgml.FgmlError) as e:
        fgml.estimate(I, A, stream=st)
    assert e.value.status == fgml.FG_ERR_OOM
    monkeypatch.delenv("FGML_FAIL_ALLOC")
    F, B = fgml.estimate(I, A, stream=st)
    st.synchronize()
    F0, B0 = fgml.estimate(I, A)
    torch.cuda.synchronize()
    assert torch.equal(F, F0) and torch.equal(B, B0)
    fgml.release_workspace(st)


def test_outputs_leave_guard_bands_untouched(fgml):
    # F and B inside larger buffers: rows padded with guard columns and guard rows above and
    # below, all filled with a sentinel that the solve must not touch
    w, h, g = 517, 389, 7
    s = synth.make_sample(w, h, 4600)
    I = torch.from_numpy(s.I).cuda()
    A = torch.from_numpy(s.alpha).cuda()
    sentinel = -12345.0
    bufs = [torch.full((h + 2 * g, 3 * w + 2 * 3 * g), sentinel, device="cuda") for _ in range(2)]
    F, B = (b[g:g + h, 3 * g:3 * g + 3 * w].view(h, w, 3) for b in bufs)
    fgml.estimate(I, A, None, F, B)
    torch.cuda.synchronize()
    for b in bufs:
        inner = torch.zeros_like(b, dtype=torch.bool)
        inner[g:g + h, 3 * g:3 * g + 3 * w] = True
        assert bool((b[~inner] == sentinel).all())
    Fo, Bo = oracle.ml(s.I, s.alpha)
    assert np.abs(F.cpu().numpy() - Fo).max() <= 1e-4


_ONE_SOLVE = """
import sys
import numpy as np, torch
from paper_2006_14970_gb300 import fgml, synth
w, h, dt = int(sys.argv[2]), int(sys.argv[3]), getattr(torch, sys.argv[4])
s = synth.make_sample(w, h, 4242)
F, B = fgml.estimate(torch.from_numpy(s.I).cuda().to(dt), torch.from_numpy(s.alpha).cuda().to(dt))
np.save(sys.argv[1], torch.cat([F, B], 2).float().cpu().numpy())
"""


@pytest.mark.parametrize("w,h,dt", [(1024, 768, "float32"), (2047, 1535, "float32"),
                                    (700, 1100, "bfloat16")])
def test_small_levels_in_one_launch_match_one_launch_per_level(fgml, tmp_path, w, h, dt):
    # the run of small levels above the coarse ones as one launch (each block computing its
    # tile's dependency cone) against one launch per level (FGML_CONE=0, read once per
    # process, hence the separate processes): the same sweeps on the same values, so the
    # results agree to float32 rounding of the sums (16-bit: both round each level to the
    # storage type)
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    outs = []
    for cone in ("1", "0"):
        path = str(tmp_path / f"out_{cone}.npy")
        env = dict(os.environ, FGML_CONE=cone, PYTHONPATH=root)
        subprocess.run([sys.executable, "-c", _ONE_SOLVE, path, str(w), str(h), dt], cwd=root,
                       env=env, check=True, timeout=600)
        outs.append(np.load(path))
    tol = 1e-5 if dt == "float32" else 2 ** -6
    assert np.abs(outs[0] - outs[1]).max() <= tol
