"""The multi-GPU host logic on CPU (gloo, world size 2): ranks run
independent replicas; the whole-job number takes the slowest rank's time and
the units all ranks processed, and only rank 0 runs the CPU reference arm."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        t, u = bench.reduce_over_ranks(dist, 1.5 + rank, 1000 * (rank + 1))
        out.put((rank, t, u, bench.reference_runs_here()))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_and_reference_rank():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    # slowest rank's time, sum of units, on every rank; reference on rank 0 only
    assert res == [(0, 2.5, 3000.0, True), (1, 2.5, 3000.0, False)]


def test_single_rank_reduction_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.reduce_over_ranks(None, 0.25, 12345) == (0.25, 12345.0)
