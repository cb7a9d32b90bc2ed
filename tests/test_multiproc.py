"""The multi-rank plumbing of bench.py on CPU: two gloo ranks (the GPU runs
use one independent replica per rank and NCCL; the host logic is the same)."""
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, q):
    import sys

    import torch
    import torch.distributed as dist

    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench

    w, r, loc = bench.dist_setup()
    ms = bench.barrier_max(1.0 + rank, world, torch.device("cpu"))  # ranks time 1 ms and 2 ms
    value = bench.weak_value(1000, w, ms)
    printed = []
    bench.run_reference_guard(r, lambda: printed.append(r))
    q.put((r, w, ms, value, printed))
    dist.destroy_process_group()


def test_two_gloo_ranks():
    import torch.multiprocessing as mp

    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # every rank sees the slowest rank's time; the value counts both replicas
    for r, w, ms, value, printed in out:
        assert w == 2 and ms == 2.0
        assert value == pytest.approx(2 * 1000 / 2e-3)
    # only rank 0 runs (and prints) the reference arm
    assert [p for *_, p in out] == [[0], []]
