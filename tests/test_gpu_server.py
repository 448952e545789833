"""Serving with continuous batching: jobs submitted while others run are admitted as slots
and memory free up; each job's result is the same alone and in the mix (within the
parity tolerance for float32, and a few units of the last place for 16-bit storage,
where each level's F and B are rounded to the storage type)."""
import random
import threading
import time

import numpy as np
import pytest
import torch

from paper_2006_14970_gb300 import synth

pytestmark = pytest.mark.gpu

TOL = {torch.float32: 1e-4, torch.bfloat16: 2 ** -6, torch.float16: 2 ** -9}


def _alone(fgml, I, A):
    F, B = fgml.estimate(I.cuda(), A.cuda())
    torch.cuda.synchronize()
    return F.cpu(), B.cpu()


def _jobs(n, seed, lo=64, hi=900, dtypes=(torch.float32, torch.bfloat16)):
    rng = random.Random(seed)
    out = []
    for i in range(n):
        w = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        h = int(np.exp(rng.uniform(np.log(lo), np.log(hi))))
        s = synth.make_sample(w, h, 3000 + seed + i)
        dt = dtypes[i % len(dtypes)]
        out.append((torch.from_numpy(s.I).to(dt).pin_memory(),
                    torch.from_numpy(s.alpha).to(dt).pin_memory()))
    return out


def test_server_results_equal_alone_and_in_mix(fgml):
    jobs = _jobs(24, 1)
    with fgml.Server(streams=2, max_batch=8) as srv:
        # submissions from two threads with small random gaps, so that jobs arrive while
        # earlier batches run
        tickets = [None] * len(jobs)

        def feed(idx):
            rng = random.Random(idx[0])
            for i in idx:
                tickets[i] = srv.submit(*jobs[i])
                time.sleep(rng.uniform(0, 0.002))

        th = [threading.Thread(target=feed, args=(list(range(k, len(jobs), 2)),)) for k in (0, 1)]
        for t in th:
            t.start()
        for t in th:
            t.join()
        outs = [srv.wait(t, 60000) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["batches"] >= 2            # the work came in several batches
    for (I, A), (F, B) in zip(jobs, outs):
        Fa, Ba = _alone(fgml, I, A)
        tol = TOL[I.dtype]
        assert float((F.float() - Fa.float()).abs().max()) <= tol
        assert float((B.float() - Ba.float()).abs().max()) <= tol


def test_server_admission_by_memory_budget(fgml):
    jobs = _jobs(10, 2, lo=300, hi=600, dtypes=(torch.float32,))
    need = [I.numel() * 4 * 13 // 3 + (1 << 20) for I, _ in jobs]
    one = max(need)
    # room for about two of the largest jobs at a time: the rest wait in the queue
    # instead of failing (smaller jobs may fit three at a time)
    with fgml.Server(hbm_budget_bytes=int(2.2 * one), streams=2, max_batch=4) as srv:
        tickets = [srv.submit(I, A) for I, A in jobs]
        outs = [srv.wait(t, 60000) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["max_bytes"] <= st["budget_bytes"]
    assert st["max_inflight"] <= int(2.2 * one) // min(need) < len(jobs)
    for (I, A), (F, B) in zip(jobs, outs):
        Fa, Ba = _alone(fgml, I, A)
        assert float((F - Fa).abs().max()) <= TOL[torch.float32]


def test_server_rejects_a_job_above_the_budget(fgml):
    with fgml.Server(hbm_budget_bytes=1 << 20) as srv:
        I = torch.zeros((512, 512, 3)).pin_memory()
        A = torch.zeros((512, 512)).pin_memory()
        with pytest.raises(fgml.FgmlError) as e:
            srv.submit(I, A)
        assert e.value.status == fgml.FG_ERR_INVALID_ARG


def test_server_latency_records(fgml):
    jobs = _jobs(6, 3, dtypes=(torch.float32,))
    with fgml.Server() as srv:
        t = [srv.submit(I, A) for I, A in jobs]
        for x in t:
            srv.wait(x, 60000)
        for x in t:
            a, b = srv.times(x)
            assert 0 <= a <= b
            srv.release(x)


def test_server_device_resident_inputs_and_outputs(fgml):
    # jobs whose I and alpha are already in device memory are read in place; device F and
    # B are written in place; host jobs run in the same mix
    jobs = _jobs(9, 4, dtypes=(torch.float32, torch.bfloat16))
    with fgml.Server(streams=2, max_batch=4) as srv:
        tickets, kinds = [], []
        for i, (I, A) in enumerate(jobs):
            kind = i % 3   # 0: all device, 1: device inputs and host outputs, 2: all host
            if kind == 0:
                t = srv.submit(I.cuda(), A.cuda())
            elif kind == 1:
                t = srv.submit(I.cuda(), A.cuda(), torch.empty(I.shape, dtype=I.dtype).pin_memory(),
                               torch.empty(I.shape, dtype=I.dtype).pin_memory())
            else:
                t = srv.submit(I, A)
            tickets.append(t)
            kinds.append(kind)
        outs = [srv.wait(t, 60000) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    for (I, A), (F, B), kind in zip(jobs, outs, kinds):
        assert F.is_cuda == (kind == 0)
        Fa, Ba = _alone(fgml, I, A)
        tol = TOL[I.dtype]
        assert float((F.cpu().float() - Fa.float()).abs().max()) <= tol
        assert float((B.cpu().float() - Ba.float()).abs().max()) <= tol


def test_server_rejects_unknown_request_flags(fgml):
    import ctypes
    lib = fgml._server_lib()
    with fgml.Server() as srv:
        I = torch.zeros((8, 8, 3)).pin_memory()
        A = torch.zeros((8, 8)).pin_memory()
        r = fgml.Request(I.data_ptr(), A.data_ptr(), 8, 8, fgml.FG_F32, I.data_ptr(), I.data_ptr(),
                         8, None)
        t = ctypes.c_uint64()
        st = lib.fg_server_submit(srv._h, ctypes.byref(r), ctypes.byref(t))
        assert st == fgml.FG_ERR_INVALID_ARG
        assert "flags" in lib.fg_server_last_error().decode()


def test_server_large_job_advances_by_levels_beside_small_jobs(fgml):
    # a 4000x3000 job is split into several launches (its level passes, a few at a time);
    # small jobs submitted right after it are copied up between its pieces, run in launches
    # of their own and complete before it
    big = synth.make_sample(4000, 3000, 3500)
    Ib = torch.from_numpy(big.I).pin_memory()
    Ab = torch.from_numpy(big.alpha).pin_memory()
    Fb, Bb = torch.empty_like(Ib).pin_memory(), torch.empty_like(Ib).pin_memory()
    small = _jobs(12, 5, lo=64, hi=256, dtypes=(torch.float32,))
    outs = [(torch.empty_like(I).pin_memory(), torch.empty_like(I).pin_memory()) for I, _ in small]
    with fgml.Server(streams=2, max_batch=16, step_work=4 << 20) as srv:
        # first use of the server's pool and kernels, outside the timed scenario
        for t in [srv.submit(Ib, Ab, Fb, Bb)] + [srv.submit(I, A, F, B) for (I, A), (F, B) in zip(small, outs)]:
            srv.wait(t, 60000)
        st0 = srv.stats()
        tb = srv.submit(Ib, Ab, Fb, Bb)
        ts = [srv.submit(I, A, F, B) for (I, A), (F, B) in zip(small, outs)]
        for t in ts + [tb]:
            srv.wait(t, 60000)
        done_small = max(srv.times(t)[1] for t in ts)
        done_big = srv.times(tb)[1]
        st = srv.stats()
    assert st["completed"] == 2 * (len(small) + 1) and st["failed"] == 0
    assert st["batches"] - st0["batches"] >= 4
    assert done_small < done_big
    Fa, Ba = _alone(fgml, Ib, Ab)
    assert float((Fb - Fa).abs().max()) <= TOL[torch.float32]
    assert float((Bb - Ba).abs().max()) <= TOL[torch.float32]
    for (I, A), (F, B) in zip(small, outs):
        Fa, Ba = _alone(fgml, I, A)
        assert float((F - Fa).abs().max()) <= TOL[torch.float32]
        assert float((B - Ba).abs().max()) <= TOL[torch.float32]


def test_server_one_pass_per_launch(fgml):
    # a budget below every pass: each launch runs one pass of one job, so every pass
    # after the first of a job starts from a state another launch wrote
    jobs = _jobs(5, 6, lo=200, hi=400, dtypes=(torch.float32, torch.bfloat16))
    with fgml.Server(streams=3, max_batch=8, step_work=1) as srv:
        tickets = [srv.submit(I, A) for I, A in jobs]
        outs = [srv.wait(t, 60000) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    assert st["batches"] >= 3 * len(jobs)   # every job has at least three level passes
    for (I, A), (F, B) in zip(jobs, outs):
        Fa, Ba = _alone(fgml, I, A)
        tol = TOL[I.dtype]
        assert float((F.float() - Fa.float()).abs().max()) <= tol
        assert float((B.float() - Ba.float()).abs().max()) <= tol


def test_server_red_black_runs_whole_jobs(fgml):
    # the work list runs the Jacobi order only: a red-black server launches whole jobs
    p = fgml.params(order=fgml.FG_ORDER_REDBLACK)
    jobs = _jobs(6, 7, lo=100, hi=500, dtypes=(torch.float32,))
    with fgml.Server(streams=2, max_batch=4, p=p) as srv:
        tickets = [srv.submit(I, A) for I, A in jobs]
        outs = [srv.wait(t, 60000) for t in tickets]
        st = srv.stats()
    assert st["completed"] == len(jobs) and st["failed"] == 0
    for (I, A), (F, B) in zip(jobs, outs):
        Fa, Ba = fgml.estimate(I.cuda(), A.cuda(), p)
        torch.cuda.synchronize()
        assert float((F - Fa.cpu()).abs().max()) <= TOL[torch.float32]
        assert float((B - Ba.cpu()).abs().max()) <= TOL[torch.float32]
