"""Benchmark of multi-level foreground estimation on GB300.

One step = one fg_estimate call (all levels of Algorithm 1) on a 2048x1536 RGB image
with FP32 storage and compute, synthetic seeded inputs already resident in HBM; L2 is
flushed (a 256 MiB write) before every timed step, outside the timed events. The line
also reports the 7680x4320 image, the roofline of the dominant kernel (the top-level
pass) against the measured HBM copy bandwidth, an end-to-end figure through the C ABI
with host buffers (copies inside the timed region), and the FP64 CPU oracle timed on
this host's cores as a baseline.

Usage: python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference] [--no-8k]
Multi-GPU (torchrun, one process per GPU): every rank solves its own image (replicas,
weak scaling); the timing is the maximum over ranks.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import re
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("Mpix/s at 2048×1536 and 8K; achieved HBM GB/s vs peak; "
          "serving p50/p99 latency")
WORKLOAD = "single_2048x1536_hair"
BIG = "single_7680x4320"
L2_FLUSH_BYTES = 256 << 20


def _peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


def _dist():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return world, rank, local


def rank_max(v: float, world: int, device) -> float:
    """The largest of every rank's v (the slowest rank's time): one all-reduce when the
    job has several ranks."""
    if world == 1:
        return v
    import torch
    t = torch.tensor([v], device=device, dtype=torch.float64)
    torch.distributed.all_reduce(t, op=torch.distributed.ReduceOp.MAX)
    return float(t.item())


def replica_throughput(world: int, pixels_per_rank: int, ms: float) -> float:
    """Whole-job Mpix/s of `world` replicas that each solved `pixels_per_rank` pixels in
    `ms` milliseconds (the slowest rank's time): weak scaling, no data-path exchange."""
    return world * pixels_per_rank / (ms * 1e-3) / 1e6


class Clocks:
    """Samples SM clocks and throttle reasons with nvidia-smi during the timed region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.path = None

    def __enter__(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "200", "-f", self.path],
                stdout=subprocess.DEVNULL, stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None
        return self

    def __exit__(self, *exc):
        if self.proc is not None:
            self.proc.terminate()
            try:
                self.proc.wait(timeout=5)
            except Exception:
                self.proc.kill()

    def summary(self):
        if not self.path or not os.path.exists(self.path):
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower() == "active":
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "samples": len(sm), "reasons": sorted(reasons)}


def kernel_source_sha256(sources) -> str:
    """sha256 of the kernel's source files, concatenated in the order given."""
    h = hashlib.sha256()
    for src in sources:
        with open(src, "rb") as f:
            h.update(f.read())
    return h.hexdigest()


def _traffic_from_profile(kernel_srcs, profile: str):
    """DRAM bytes per launch recorded by ncu in profiles/, if the kernel source is unchanged
    since the capture (the summary records the sources' sha256)."""
    path = os.path.join(ROOT, "profiles", profile)
    if not os.path.exists(path):
        return None
    text = open(path).read()
    m = re.search(r"traffic_bytes_per_launch:\s*([0-9.]+)", text)
    h = re.search(r"source_sha256:\s*([0-9a-f]{64})", text)
    if not m or not h:
        return None
    return float(m.group(1)) if kernel_source_sha256(kernel_srcs) == h.group(1) else None


def cpu_baseline(sample: str, seconds: float = 10.0):
    """The FP64 oracle, as it stands, on this host's cores: repeated full solves of the
    workload image for about `seconds`."""
    import oracle
    from paper_2006_14970_gb300 import synth
    s = synth.workload(sample)
    h, w = s.alpha.shape
    threads = oracle.set_threads(0)
    n, t0 = 0, time.perf_counter()
    while True:
        oracle.ml(s.I, s.alpha)
        n += 1
        dt = time.perf_counter() - t0
        if dt >= seconds or n >= 50:
            break
    out = {"value": n * w * h / dt / 1e6, "unit": "Mpix/s", "cores": threads, "kind": "oracle",
           "sample": f"{n} full FP64 solves of the {w}x{h} workload image ({dt:.1f} s)"}
    # the paper times its method single-threaded: the oracle on one core, best of 3
    oracle.set_threads(1)
    best = None
    for _ in range(3):
        t1 = time.perf_counter()
        oracle.ml(s.I, s.alpha)
        d1 = time.perf_counter() - t1
        best = d1 if best is None else min(best, d1)
    oracle.set_threads(threads)
    out["single_thread"] = {"value": w * h / best / 1e6, "unit": "Mpix/s", "cores": 1,
                            "sample": f"best of 3 FP64 solves of the {w}x{h} image ({best:.2f} s each)"}
    return out


def batch_section(fgml, synth, torch, dev, timed, world, args):
    """64 images with sides log-uniform in [256, 2048]: one fg_estimate_batch call against
    the same images solved one at a time with float32 storage (the plain form), both on
    device-resident inputs; then the same batch with bfloat16 storage (I, alpha, F, B in
    16 bits, every solve in float32) and its largest difference to the float32 batch."""
    ss = synth.batch(64)
    imgs = [(torch.from_numpy(s.I).to(dev), torch.from_numpy(s.alpha).to(dev)) for s in ss]
    outs = [(torch.empty_like(I), torch.empty_like(I)) for I, _ in imgs]
    npx = sum(s.alpha.size for s in ss)
    steps = max(3, args.steps // 4)
    # the work list's strip shape is chosen by measurement on this batch first
    chosen, tune_ms = fgml.autotune_batch(imgs, None, outs)
    job = fgml.Batch(imgs, outs)   # arguments marshalled once, as a serving loop would
    ms_b = timed(job.run, steps, args.warmup)

    def one_by_one():
        for (I, A), (F, B) in zip(imgs, outs):
            fgml.estimate(I, A, None, F, B)
    ms_1 = timed(one_by_one, steps, args.warmup)
    # bfloat16 storage, same images and work list
    imgs16 = [(I.to(torch.bfloat16), A.to(torch.bfloat16)) for I, A in imgs]
    outs16 = [(torch.empty_like(I), torch.empty_like(I)) for I, _ in imgs16]
    fgml.autotune_batch(imgs16, None, outs16)
    job16 = fgml.Batch(imgs16, outs16)
    ms_16 = timed(job16.run, steps, args.warmup)
    fgml.estimate_batch(imgs, None, outs)
    torch.cuda.synchronize()
    d16 = max(max(float((F16.float() - F).abs().max()), float((B16.float() - B).abs().max()))
              for (F16, B16), (F, B) in zip(outs16, outs))
    del imgs16, outs16
    return {"workload": "batch_64_uneven_256_2048_fp32", "images": len(ss), "pixels": int(npx),
            "value": world * npx / (ms_b * 1e-3) / 1e6, "unit": "Mpix/s", "ms_per_step": ms_b,
            "one_at_a_time": {"value": world * npx / (ms_1 * 1e-3) / 1e6, "unit": "Mpix/s",
                              "ms_per_step": ms_1},
            "bf16": {"value": world * npx / (ms_16 * 1e-3) / 1e6, "unit": "Mpix/s",
                     "ms_per_step": ms_16, "max_abs_vs_f32_batch": d16,
                     "vs_f32_one_at_a_time": ms_1 / ms_16},
            # coarse levels, work list, and the row-aligned copy when some rows are off the
            # 16-byte grid
            "launches_per_step": 2 + int(any((3 * s.alpha.shape[1] * 4) % 16 for s in ss)),
            "strip_shape_candidate": chosen,
            "autotune_ms_per_call": tune_ms}


def serving_section(fgml, synth, torch, args):
    """Poisson arrivals of jobs (sides log-uniform in [256, 4096], random aspect, host
    buffers) into the continuous-batching server, at several multiples of the measured
    one-at-a-time float32 capacity: the mixed workload (half float32, half bfloat16
    requests) and the same jobs with bfloat16 storage only."""
    import threading
    rng = np.random.Generator(np.random.PCG64(synth.SEED_BASE + 4))
    base = []
    for i in range(16):
        w = int(np.exp(rng.uniform(np.log(256), np.log(4096))))
        h = int(np.exp(rng.uniform(np.log(256), np.log(4096))))
        s = synth.make_sample(w, h, synth.SEED_BASE + 400 + i)
        base.append((s, w * h))

    def pinned(x, dt):
        return torch.from_numpy(x).to(dt).pin_memory()

    def outputs(I):   # one pinned output pair per template: the bench never reads them
        return (torch.empty(I.shape, dtype=I.dtype, pin_memory=True),
                torch.empty(I.shape, dtype=I.dtype, pin_memory=True))

    f32 = []
    for s, n in base:
        I, A = pinned(s.I, torch.float32), pinned(s.alpha, torch.float32)
        f32.append((I, A, n, outputs(I)))
    # one-at-a-time float32 capacity through the host-buffer entry point: every template
    # once first (workspace growth, launch-graph capture), then passes over the 16
    # templates for at least a second, pinned outputs
    for I, A, _, (F, B) in f32:
        fgml.estimate_host(I, A, None, F, B)
    calls, px, t0 = 0, 0, time.perf_counter()
    while True:
        for I, A, n, (F, B) in f32:
            fgml.estimate_host(I, A, None, F, B)
            calls += 1
            px += n
        dt1 = time.perf_counter() - t0
        if dt1 >= 1.0:
            break
    cap_req = calls / dt1
    cap_px = px / dt1
    out = {"workload": "serving_poisson_256_4096_mixed_f32_bf16",
           "one_at_a_time_f32": {"req_s": cap_req, "mpix_s": cap_px / 1e6, "calls": calls,
                                 "seconds": dt1},
           "rates": [], "bf16_only": [], "device_rates": []}
    mixed = []
    for i, (s, n) in enumerate(base):
        dt = torch.float32 if i % 2 == 0 else torch.bfloat16
        I, A = pinned(s.I, dt), pinned(s.alpha, dt)
        mixed.append((I, A, n, outputs(I)))
    bf16 = []
    for s, n in base:
        I, A = pinned(s.I, torch.bfloat16), pinned(s.alpha, torch.bfloat16)
        bf16.append((I, A, n, outputs(I)))
    n_req = max(16, args.serving_requests)

    def sweep(templates, rates, key, cap=None):
        for x in rates:
            rate = x * (cap or cap_req)
            gaps = rng.exponential(1.0 / rate, n_req)
            picks = rng.integers(0, len(templates), n_req)
            with fgml.Server(streams=2, max_batch=32) as srv:
                tickets, done, subs, lat = [], [], [], []
                lock = threading.Lock()
                finished = threading.Event()

                def collect():
                    k = 0
                    while k < n_req:
                        with lock:
                            have = len(tickets)
                        if k >= have:
                            time.sleep(0.0002)
                            continue
                        t = tickets[k]
                        srv.wait(t, 120000)
                        a, b = srv.times(t)
                        lat.append(b - a)
                        done.append(b)
                        subs.append(a)
                        srv.release(t)
                        k += 1
                    finished.set()

                th = threading.Thread(target=collect)
                th.start()
                start = time.perf_counter()
                at = 0.0
                for g, k in zip(gaps, picks):
                    at += g
                    while time.perf_counter() - start < at:
                        pass
                    I, A, _, (F, B) = templates[k]
                    t = srv.submit(I, A, F, B)
                    with lock:
                        tickets.append(t)
                finished.wait()
                th.join()
                st = srv.stats()
            span = max(done) - min(subs)   # from the first arrival to the last completion
            lat_ms = np.array(lat) * 1e3
            out[key].append({"x_capacity": x, "offered_req_s": rate, "requests": n_req,
                             "mpix_s": st["pixels"] / span / 1e6,
                             "p50_ms": float(np.percentile(lat_ms, 50)),
                             "p99_ms": float(np.percentile(lat_ms, 99)), "batches": st["batches"],
                             "max_inflight": st["max_inflight"]})

    sweep(mixed, (0.25, 0.5, 0.75, 0.9, 1.0, 1.2), "rates")
    sweep(bf16, (0.5, 1.0, 1.5, 2.0), "bf16_only")
    del mixed, bf16
    # the same mixed jobs with I, alpha, F and B resident in device memory (read and
    # written in place): latency without the host link, at multiples of the device-resident
    # one-at-a-time capacity
    dev_t = []
    for i, (s, n) in enumerate(base):
        dt = torch.float32 if i % 2 == 0 else torch.bfloat16
        I = torch.from_numpy(s.I).to(dt).cuda()
        A = torch.from_numpy(s.alpha).to(dt).cuda()
        dev_t.append((I, A, n, (torch.empty_like(I), torch.empty_like(I))))
    for I, A, _, (F, B) in dev_t:
        fgml.estimate(I, A, None, F, B)
    torch.cuda.synchronize()
    calls, t0 = 0, time.perf_counter()
    while True:
        for I, A, n, (F, B) in dev_t:
            fgml.estimate(I, A, None, F, B)
            torch.cuda.synchronize()
            calls += 1
        dt1 = time.perf_counter() - t0
        if dt1 >= 1.0:
            break
    cap_dev = calls / dt1
    out["device_resident"] = {"one_at_a_time_req_s": cap_dev, "rates": []}
    sweep(dev_t, (0.25, 0.5, 0.75, 1.0, 1.5), "device_rates", cap_dev)
    out["device_resident"]["rates"] = out.pop("device_rates")
    del dev_t
    return out


def quality_section(fgml, synth, torch, dev, timed):
    """Error measures of Section IV-C against the generator's known foreground: the
    2048x1536 workload at the paper's parameters (plus the time of one fg_quality call),
    and the regularisation sweep of Section IV-F over four 512x384 images with hair."""
    from paper_2006_14970_gb300 import sweep
    s = synth.workload(WORKLOAD)
    I = torch.from_numpy(s.I).to(dev)
    A = torch.from_numpy(s.alpha).to(dev)
    Ft = torch.from_numpy(s.F).to(dev)
    F, _ = fgml.estimate(I, A)
    at_default = fgml.quality(F, Ft, A)
    ms = timed(lambda: fgml.quality(F, Ft, A), 5, 3)
    imgs = []
    for i in range(4):
        t = synth.make_sample(512, 384, synth.SEED_BASE + 700 + i, hair=True)
        imgs.append((torch.from_numpy(t.I).to(dev), torch.from_numpy(t.alpha).to(dev),
                     torch.from_numpy(t.F).to(dev)))
    rows = sweep.regularisation_sweep(imgs, [1e-4, 1e-3, 5e-3, 1e-2, 1e-1], [0.0, 0.1, 1.0])
    best = min(rows, key=lambda r: r["mse"])
    return {"workload": "single_2048x1536_hair_fp32", "fractional_pixels": int(
                ((s.alpha > 0) & (s.alpha < 1)).sum()),
            "at_paper_parameters": at_default, "fg_quality_ms": ms,
            "sweep": {"images": "4 x 512x384 with hair", "rows": rows,
                      "min_mse_at": {"eps_r": best["eps_r"], "omega": best["omega"]}}}


def converged_section(fgml, synth, torch, dev):
    """Distance of the method's output from the minimiser of the global cost (float64
    conjugate gradients, warm-started from the method's output, to a relative residual of
    1e-10) on the 2048x1536 workload. The minimiser is unclamped; the method clamps."""
    s = synth.workload(WORKLOAD)
    I = torch.from_numpy(s.I).to(dev)
    A = torch.from_numpy(s.alpha).to(dev)
    F, B = fgml.estimate(I, A)
    t0 = time.perf_counter()
    Fm, Bm, it, rel = fgml.minimiser_cg(I, A, None, F, B, max_iters=20000, rel_tol=1e-10)
    secs = time.perf_counter() - t0
    frac = torch.from_numpy((s.alpha > 0) & (s.alpha < 1)).to(dev)
    dF = (F.double() - Fm).abs()
    dB = (B.double() - Bm).abs()
    inside = ((Fm >= 0) & (Fm <= 1)).all(dim=-1) & frac
    return {"workload": "single_2048x1536_hair_fp32", "cg_iterations": it,
            "cg_relative_residual": rel, "cg_seconds": secs,
            "F_max_abs": float(dF.max()), "F_rms": float(dF.pow(2).mean().sqrt()),
            "B_max_abs": float(dB.max()), "B_rms": float(dB.pow(2).mean().sqrt()),
            "F_rms_fractional": float(dF[frac].pow(2).mean().sqrt()),
            "F_max_abs_fractional_minimiser_in_unit_box": float(dF[inside].max())
            if bool(inside.any()) else None}


def run_reference(args):
    world, rank, _ = _dist()
    if rank != 0:
        return 0
    base = cpu_baseline(WORKLOAD, seconds=max(5.0, 2.0 * args.steps))
    line = {"impl": "reference", "metric": METRIC, "value": base["value"], "unit": "Mpix/s",
            "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 2048 * 1536 / base["value"] / 1e3, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": {"workload": "single_2048x1536_hair_fp32", "w": 2048, "h": 1536},
            "cpu_baseline": base,
            "e2e": {"value": base["value"], "unit": "Mpix/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="fgml", choices=["fgml", "reference"])
    ap.add_argument("--no-8k", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-batch", action="store_true")
    ap.add_argument("--no-serving", action="store_true")
    ap.add_argument("--no-quality", action="store_true")
    ap.add_argument("--no-cg", action="store_true")
    ap.add_argument("--e2e-streams", type=int, default=3)
    ap.add_argument("--serving-requests", type=int, default=1000)
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)
    if args.warmup < 3:
        args.warmup = 3

    import torch
    world, rank, local = _dist()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    else:
        torch.cuda.set_device(0)
    dev = torch.device("cuda", torch.cuda.current_device())

    from paper_2006_14970_gb300 import build as fbuild
    fbuild.build()
    from paper_2006_14970_gb300 import fgml, synth

    stream = torch.cuda.current_stream()
    flush = torch.empty(L2_FLUSH_BYTES // 4, dtype=torch.float32, device=dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize()

    def max_over_ranks(v: float) -> float:
        return rank_max(v, world, dev)

    def timed(fn, steps, warmup):
        for _ in range(warmup):
            fn()
        barrier()
        total = 0.0
        for _ in range(steps):
            flush.fill_(1.0)                       # evict L2, outside the timed events
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            fn()
            e1.record(stream)
            e1.synchronize()
            total += e0.elapsed_time(e1)
        barrier()
        return max_over_ranks(total) / steps       # ms per step

    def image_case(name):
        s = synth.workload(name)
        h, w = s.alpha.shape
        I = torch.from_numpy(s.I).to(dev)
        A = torch.from_numpy(s.alpha).to(dev)
        F = torch.empty_like(I)
        B = torch.empty_like(I)
        return s, w, h, I, A, F, B

    peak, peak_kind = _peaks()
    lv_src = [os.path.join(ROOT, "paper_2006_14970_gb300", "csrc", f)
              for f in ("level_tile.cu", "tile_common.cuh")]

    def top_pass_roofline(w, h, I, A, steps, warmup, profile):
        """The top-level pass alone (fg_level_pass: the same kernel and launch shape as
        inside fg_estimate), from a previous level of random F and B in the storage type
        of I, rows padded to 16 bytes like the library's own intermediate levels."""
        levels = fgml.schedule(w, h)
        (pw, ph, _), (_, _, k) = levels[-2], levels[-1]
        es = I.element_size()
        q = 16 // es
        pitch = (3 * pw + q - 1) // q * q
        Fs = torch.rand((ph, pitch), device=dev).to(I.dtype)[:, :3 * pw].view(ph, pw, 3)
        Bs = torch.rand((ph, pitch), device=dev).to(I.dtype)[:, :3 * pw].view(ph, pw, 3)
        Fd = torch.empty((h, w, 3), device=dev, dtype=I.dtype)
        Bd = torch.empty((h, w, 3), device=dev, dtype=I.dtype)
        ms = timed(lambda: fgml.level_pass(I, A, Fs, Bs, k, w, h, None, Fd, Bd), steps, warmup)
        algo = es * (10 * w * h + 6 * pw * ph)     # read I, alpha, previous F/B; write F, B
        achieved = algo / (ms * 1e-3) / 1e9
        return {"bound": "hbm", "kernel": f"level_tile_kernel<{'float' if es == 4 else 'bf16'},2>",
                "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "peak_kind": f"{peak_kind} copy bandwidth (burst)",
                "algorithmic_bytes": algo, "ms": ms,
                "traffic": _traffic_from_profile(lv_src, profile) if profile else None}

    s, w, h, I, A, F, B = image_case(WORKLOAD)
    levels = fgml.schedule(w, h)
    # one launch for the levels of at most 1024 pixels (the coarse kernel), one for the run
    # of levels of at most 0.3 Mpx after them (the cone kernel), one per level pass above
    n_coarse = sum(1 for (lw, lh, _) in levels if lw * lh <= 1024)
    n_cone = 0
    while (n_coarse + n_cone < len(levels) and n_cone < 8
           and levels[n_coarse + n_cone][0] * levels[n_coarse + n_cone][1] <= 300000):
        n_cone += 1
    launches_per_step = 1 + int(n_cone > 0) + (len(levels) - n_coarse - n_cone)

    with Clocks(local) as clk:
        ms = timed(lambda: fgml.estimate(I, A, None, F, B), args.steps, args.warmup)
        roof = top_pass_roofline(w, h, I, A, args.steps, args.warmup,
                                 "level_tile_2048x1536.md")
    clocks = clk.summary()
    value = replica_throughput(world, w * h, ms)

    # end to end through the C ABI with host buffers (pinned), copies inside the timed
    # region: a sequence of images on several streams (fg_estimate_host_async), so one image's
    # copy back overlaps the next one's copy in and solve; every step still copies its own
    # inputs in and its F and B out. No L2 flush: every step streams 126 MB over the host
    # link and ~200 MB through HBM, more than L2 holds.
    Ih = torch.from_numpy(s.I).pin_memory()
    Ah = torch.from_numpy(s.alpha).pin_memory()
    ns = max(2, args.e2e_streams)
    outs = [(torch.empty_like(Ih).pin_memory(), torch.empty_like(Ih).pin_memory()) for _ in range(ns)]
    sts = [torch.cuda.Stream() for _ in range(ns)]

    def host_steps(k):
        for i in range(k):
            fgml.estimate_host_async(Ih, Ah, None, outs[i % ns][0], outs[i % ns][1], stream=sts[i % ns])

    host_steps(2 * args.warmup)
    barrier()
    n_e2e = max(4, args.steps)
    e_start = torch.cuda.Event(enable_timing=True)
    e_end = torch.cuda.Event(enable_timing=True)
    e_start.record(sts[0])
    for st in sts[1:]:
        st.wait_event(e_start)
    host_steps(n_e2e)
    for st in sts[1:]:
        e_side = torch.cuda.Event()
        e_side.record(st)
        sts[0].wait_event(e_side)
    e_end.record(sts[0])
    e_end.synchronize()
    ms_e2e = max_over_ranks(e_start.elapsed_time(e_end)) / n_e2e
    # the same, one call at a time (each call waits for its result)
    ms_e2e_1 = timed(lambda: fgml.estimate_host(Ih, Ah, None, outs[0][0], outs[0][1]), max(3, args.steps // 2),
                     args.warmup)
    e2e = {"value": replica_throughput(world, w * h, ms_e2e), "unit": "Mpix/s",
           "h2d_bytes_per_step": int(Ih.numel() * 4 + Ah.numel() * 4),
           "d2h_bytes_per_step": int(2 * Ih.numel() * 4), "ms_per_step": ms_e2e,
           "steps": n_e2e, "how": f"fg_estimate_host_async on {ns} streams, pinned host buffers",
           "one_call_at_a_time": {"value": replica_throughput(world, w * h, ms_e2e_1),
                                  "ms_per_step": ms_e2e_1}}

    big = None
    if not args.no_8k:
        del I, A, F, B
        s8, w8, h8, I8, A8, F8, B8 = image_case(BIG)
        ms8 = timed(lambda: fgml.estimate(I8, A8, None, F8, B8), max(3, args.steps // 2),
                    args.warmup)
        roof8 = top_pass_roofline(w8, h8, I8, A8, max(3, args.steps // 2), args.warmup,
                                  "level_tile_7680x4320.md")
        big = {"workload": "single_7680x4320_fp32", "value": world * w8 * h8 / (ms8 * 1e-3) / 1e6,
               "unit": "Mpix/s", "ms_per_step": ms8, "roofline": roof8, "storage": {}}
        # reduced-precision storage (I, alpha, F, B in 16 bits; solves in float32): throughput
        # and the largest difference to the float32 path on the same inputs
        torch.cuda.synchronize()
        for name, dt in (("bf16", torch.bfloat16), ("f16", torch.float16)):
            I16, A16 = I8.to(dt), A8.to(dt)
            F16, B16 = torch.empty_like(I16), torch.empty_like(I16)
            ms16 = timed(lambda: fgml.estimate(I16, A16, None, F16, B16), max(3, args.steps // 2),
                         args.warmup)
            d = max(float((F16.float() - F8).abs().max()), float((B16.float() - B8).abs().max()))
            big["storage"][name] = {"value": world * w8 * h8 / (ms16 * 1e-3) / 1e6,
                                    "unit": "Mpix/s", "ms_per_step": ms16,
                                    "max_abs_vs_f32_path": d,
                                    "vs_f32": ms8 / ms16}
            if name == "bf16":
                big["storage"][name]["roofline"] = top_pass_roofline(
                    w8, h8, I16, A16, max(3, args.steps // 2), args.warmup,
                    "level_tile_7680x4320_bf16.md")
            del I16, A16, F16, B16

    batch = None
    if not args.no_batch:
        batch = batch_section(fgml, synth, torch, dev, timed, world, args)
    serving = None
    if not args.no_serving:
        serving = serving_section(fgml, synth, torch, args)

    quality = None
    if not args.no_quality:
        quality = quality_section(fgml, synth, torch, dev, timed)

    converged = None
    if not args.no_cg:
        converged = converged_section(fgml, synth, torch, dev)

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        cpu = cpu_baseline(WORKLOAD)

    # the other workloads of the metric in the line's config (the 7680x4320 image in float32
    # and bfloat16, the batch and serving forms against float32 one image at a time)
    secondary = {}
    if big:
        secondary["single_7680x4320_fp32"] = {
            "mpix_s": big["value"], "ms_per_step": big["ms_per_step"],
            "top_pass_hbm_frac": big["roofline"]["frac"]}
        b16 = big["storage"].get("bf16")
        if b16:
            secondary["single_7680x4320_bf16"] = {
                "mpix_s": b16["value"], "ms_per_step": b16["ms_per_step"],
                "top_pass_hbm_frac": b16["roofline"]["frac"],
                "max_abs_vs_f32_path": b16["max_abs_vs_f32_path"], "speedup_vs_fp32": b16["vs_f32"]}
    if batch:
        secondary["batch_64_uneven"] = {
            "fp32_one_at_a_time_mpix_s": batch["one_at_a_time"]["value"],
            "fp32_batched_mpix_s": batch["value"], "bf16_batched_mpix_s": batch["bf16"]["value"],
            "bf16_max_abs_vs_f32": batch["bf16"]["max_abs_vs_f32_batch"]}
    if serving:
        best = lambda rows: max((r["mpix_s"] for r in rows), default=None)
        secondary["serving_poisson"] = {
            "fp32_one_at_a_time_mpix_s": serving["one_at_a_time_f32"]["mpix_s"],
            "capacity_req_s": serving["one_at_a_time_f32"]["req_s"],
            "mixed_best_mpix_s": best(serving["rates"]),
            "bf16_best_mpix_s": best(serving["bf16_only"]),
            "p50_p99_ms_at_0.75x": next(([r["p50_ms"], r["p99_ms"]] for r in serving["rates"]
                                          if r["x_capacity"] == 0.75), None),
            "device_resident_p50_p99_ms_at_0.75x": next(
                ([r["p50_ms"], r["p99_ms"]] for r in serving["device_resident"]["rates"]
                 if r["x_capacity"] == 0.75), None),
            "device_resident_best_mpix_s": best(serving["device_resident"]["rates"])}

    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": "Mpix/s", "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f32", "data": "synthetic",
                "config": {"workload": "single_2048x1536_hair_fp32", "w": w, "h": h,
                           "levels": len(levels), "l2": "flushed before every timed step",
                           "parallelism": "replicas" if world > 1 else "single",
                           "secondary": secondary},
                "roofline": roof, "e2e": e2e, "gpu_launches": launches_per_step * args.steps,
                "clocks": clocks, "cpu_baseline": cpu, "big": big, "batch": batch,
                "serving": serving, "quality": quality, "converged_reference": converged,
                "library": fgml.version()}
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


if __name__ == "__main__":
    sys.exit(main())
