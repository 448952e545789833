"""The multi-GPU path of bench.py is replicas: one image per rank, no data-path exchange,
the slowest rank's time and the whole-job throughput. Its host logic runs here as two
gloo ranks on the CPU (no GPU involved)."""
import os
import socket
import sys

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world), LOCAL_RANK=str(rank))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        assert bench._dist() == (world, rank, rank)
        # each rank's own time; every rank must see the slowest
        ms = 1.0 + 0.5 * rank
        slow = bench.rank_max(ms, world, torch.device("cpu"))
        value = bench.replica_throughput(world, 2048 * 1536, slow)
        # the reference leg runs on rank 0 only; the others return 0 without work
        ref_rc = bench.run_reference(type("A", (), {"steps": 1, "warmup": 1, "gpus": world})) \
            if rank != 0 else None
        out.put((rank, slow, value, ref_rc))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_time_and_sum_replicas():
    ctx = mp.get_context("spawn")
    out = ctx.Queue()
    world, port = 2, _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(out.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    want_ms = 1.5
    for rank, slow, value, ref_rc in res:
        assert slow == pytest.approx(want_ms)
        assert value == pytest.approx(2 * 2048 * 1536 / (want_ms * 1e-3) / 1e6)
    assert res[1][3] == 0


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.rank_max(3.0, 1, torch.device("cpu")) == 3.0
    assert bench.replica_throughput(1, 1000, 1.0) == pytest.approx(1.0)
