"""Row-band decomposition across ranks on the GPU: two gloo ranks, each a
process driving one context over its band (and halo) on cuda:0, exchange
their edge pedestrians through host memory every tick (no kernel of one
rank waits on the other's).  After 10 ticks they must hold exactly the
pedestrians, positions and headings of one context stepping the whole
lattice, and count the same exits: on a 1024^2 floor shaped like the
benchmark's (walls, obstacles, 4 exits, r = 40) and on the 1000 x 200
counter-flow corridor (periodic in x, r = 20)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import scenegen as SG                                 # noqa: E402

pytestmark = pytest.mark.gpu
TICKS = 10


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _scene(which):
    if which == "floor":
        return SG.floor(side=1024, n=40000, exit_len=64, seed=71)
    return SG.corridor()


def _guidance(sfm, sc):
    with sfm.Sim(sc, place=False) as whole:
        return whole.guidance()


def _band_rank(rank, world, port, which, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch
    import torch.distributed as dist
    import paper_1803_04782_gb300 as sfm
    from paper_1803_04782_gb300 import bands as BD
    from paper_1803_04782_gb300 import build as B
    torch.cuda.set_device(0)
    B.build()
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = _scene(which)
        D = _guidance(sfm, sc)
        L = BD.BandLayout(sc.H, sc.periodic_y, int(sc.params["r"]), world)
        peds = BD.Peds(np.arange(sc.n, dtype=np.int32), sc.xy.copy(), sc.heading.copy(),
                       sc.goal.copy())
        own = BD.own_of(L, rank, peds)
        step, sim = BD.sim_stepper(L, rank, sc.W, sc.periodic_x, sc.cell, D, sc.params)
        comm = BD.TorchComm(dist)
        left = 0
        try:
            for t in range(TICKS):
                own, n_left = BD.band_tick(L, rank, comm, step, own, t)
                left += n_left
        finally:
            sim.close()
        out.put((rank, own.ids.tolist(), own.xy.tolist(), own.heading.tolist(), left))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("which", ["floor", "corridor"])
def test_two_band_ranks_reproduce_one_context(which):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")
    import paper_1803_04782_gb300 as sfm
    from paper_1803_04782_gb300 import build as B
    B.build()
    sc = _scene(which)
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_band_rank, args=(r, 2, port, which, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = [q.get(timeout=600) for _ in procs]
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    with sfm.Sim(sc) as whole:
        whole.step(TICKS)
        xy, hd, alive = whole.peds()
        exited = whole.stats()["exited"]
    ids = np.concatenate([np.array(r[1], np.int64) for r in res])
    bxy = np.concatenate([np.array(r[2], np.int64).reshape(-1, 2) for r in res])
    bhd = np.concatenate([np.array(r[3], np.int64) for r in res])
    live = np.flatnonzero(alive)
    assert len(set(ids.tolist())) == len(ids)
    assert sorted(ids.tolist()) == live.tolist()
    order = np.argsort(ids)
    np.testing.assert_array_equal(bxy[order], xy[live])
    np.testing.assert_array_equal(bhd[order], hd[live])
    assert sum(r[4] for r in res) == exited
