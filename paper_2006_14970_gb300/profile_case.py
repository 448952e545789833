"""Runs one kernel case a few times, for profiler captures (ncu -k ... -s <warm-up> -c ...).

    python -m paper_2006_14970_gb300.profile_case level_pass 4096 2304 [--repeat 4]
    python -m paper_2006_14970_gb300.profile_case estimate 2048 1536 [--dtype bf16]
    python -m paper_2006_14970_gb300.profile_case batch 64 0

level_pass: the top-level pass of a W x H image (sweeps of the top level, starting F/B
gathered from the level below it), the dominant launch of a solve.
estimate: complete fg_estimate calls.
batch: fg_estimate_batch of the first W images of the 64-image batched workload (H unused).
Inputs come from the seeded synthetic generator; nothing is checked here.
"""
from __future__ import annotations

import argparse

import torch

from . import build as _build


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("case", choices=["level_pass", "estimate", "batch"])
    ap.add_argument("w", type=int)
    ap.add_argument("h", type=int)
    ap.add_argument("--repeat", type=int, default=4)
    ap.add_argument("--dtype", default="f32", choices=["f32", "bf16", "f16"])
    ap.add_argument("--small-iters", type=int, default=None)
    ap.add_argument("--big-iters", type=int, default=None)
    ap.add_argument("--pad", action="store_true", help="batch: rows of I and alpha padded to 16 bytes")
    a = ap.parse_args()
    _build.build()
    from . import fgml, synth
    kw = {}
    if a.small_iters is not None:
        kw["small_iters"] = a.small_iters
    if a.big_iters is not None:
        kw["big_iters"] = a.big_iters
    prm = fgml.params(**kw) if kw else None
    dt = {"f32": torch.float32, "bf16": torch.bfloat16, "f16": torch.float16}[a.dtype]
    if a.case != "batch":
        s = synth.make_sample(a.w, a.h, synth.SEED_BASE + 50)
        I = torch.from_numpy(s.I).cuda().to(dt)
        A = torch.from_numpy(s.alpha).cuda().to(dt)
    start = torch.cuda.Event(enable_timing=True)
    stop = torch.cuda.Event(enable_timing=True)
    if a.case == "batch":
        ss = synth.batch(64)[:a.w]

        def dev(x, ch):
            t = torch.from_numpy(x).cuda().to(dt)
            if not a.pad:
                return t
            h, w = x.shape[0], x.shape[1]
            q = 16 // t.element_size()
            pitch = (ch * w + q - 1) // q * q
            buf = torch.empty((h, pitch), dtype=dt, device="cuda")
            v = buf[:, :ch * w].view(h, w, ch) if ch > 1 else buf[:, :w]
            v.copy_(t)
            return v
        imgs = [(dev(t.I, 3), dev(t.alpha, 1)) for t in ss]
        outs = [(torch.empty_like(I), torch.empty_like(I)) for I, _ in imgs]

        def run():
            fgml.estimate_batch(imgs, prm, outs)
    elif a.case == "level_pass":
        levels = fgml.schedule(a.w, a.h)
        (pw, ph, _), (_, _, k) = levels[-2], levels[-1]
        g = torch.Generator(device="cuda").manual_seed(1)
        # rows padded to 16 bytes, like the library's own intermediate levels
        q = 16 // torch.empty((), dtype=dt).element_size()
        pitch = (3 * pw + q - 1) // q * q
        Fs = torch.rand((ph, pitch), device="cuda", generator=g).to(dt)[:, :3 * pw].view(ph, pw, 3)
        Bs = torch.rand((ph, pitch), device="cuda", generator=g).to(dt)[:, :3 * pw].view(ph, pw, 3)
        F = torch.empty_like(I)
        B = torch.empty_like(I)
        def run():
            fgml.level_pass(I, A, Fs, Bs, k, a.w, a.h, None, F, B)
    else:
        F = torch.empty_like(I)
        B = torch.empty_like(I)

        def run():
            fgml.estimate(I, A, prm, F, B)
    run()
    start.record()
    for _ in range(max(1, a.repeat - 1)):
        run()
    stop.record()
    torch.cuda.synchronize()
    ms = start.elapsed_time(stop) / max(1, a.repeat - 1)
    extra = f" {kw}" if kw else ""
    print(f"{a.case} {a.w}x{a.h} {a.dtype}{extra} x{a.repeat}: {ms * 1e3:.1f} us per call "
          "(back to back, L2 not flushed)")


if __name__ == "__main__":
    main()
