"""Row-band decomposition across ranks (paper_1803_04782_gb300/bands.py), on
CPU: the band layout, the halo bookkeeping against a brute-force selection,
the exchange over two gloo ranks, and two gloo ranks each stepping its band
with the FP64 oracle, which must reproduce the oracle's run of the whole
lattice exactly (positions, headings, exits)."""
import os
import socket
import sys

import numpy as np
import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import oracle as O                                   # noqa: E402
import scenegen as SG                                # noqa: E402
from paper_1803_04782_gb300 import bands as BD       # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


@pytest.mark.parametrize("H,py,r,n", [(320, 0, 20, 2), (320, 1, 20, 2), (256, 1, 5, 4),
                                      (1000, 0, 40, 4), (100, 0, 10, 1)])
def test_layout_covers_the_lattice_and_reaches_r_plus_3(H, py, r, n):
    L = BD.BandLayout(H, py, r, n)
    assert L.y0[0] == 0 and L.y1[-1] == H and (L.y0[1:] == L.y1[:-1]).all()
    assert (L.y0 % BD.BIN == 0).all()
    owners = L.owner(np.arange(H))
    for k in range(n):
        assert (owners[L.y0[k]:L.y1[k]] == k).all()
        a, rows = L.rows(k)
        assert a % BD.BIN == 0 or (not py and a == 0)
        for y in range(int(L.y0[k]), int(L.y1[k])):
            # every row within r + 3 of an own row is in the halo'd rows
            near = np.arange(y - r - 3, y + r + 4)
            near = near % H if py else near[(near >= 0) & (near < H)]
            assert L.in_sub(k, near).all()
        yl = L.local_row(k, np.arange(H))
        inside = L.in_sub(k, np.arange(H))
        assert (L.global_row(k, yl[inside]) == np.arange(H)[inside]).all()


@pytest.mark.parametrize("H,py,r,n", [(320, 0, 20, 2), (320, 1, 12, 3), (512, 1, 9, 4)])
def test_sends_match_a_brute_force_selection(H, py, r, n):
    rng = np.random.default_rng(7)
    W, npeds = 64, 3000
    peds = BD.Peds(np.arange(npeds, dtype=np.int32),
                   np.stack([rng.integers(0, W, npeds), rng.integers(0, H, npeds)], 1).astype(np.int32),
                   rng.integers(0, 9, npeds).astype(np.uint8), rng.integers(0, 9, npeds).astype(np.uint8))
    L = BD.BandLayout(H, py, r, n)
    for k in range(n):
        own = BD.own_of(L, k, peds)
        sends = BD.sends_of(L, k, own)
        for j in range(n):
            a, rows = L.rows(j)
            sub_rows = set(((a + np.arange(rows)) % H).tolist()) if py else set(range(a, a + rows))
            want = sorted(int(i) for i, y in zip(own.ids, own.xy[:, 1]) if int(y) in sub_rows)
            if j in sends:
                assert sorted(sends[j].ids.tolist()) == want
            elif j != k:
                assert want == []       # only neighbours' halo'd rows meet rank k's rows
    # every pedestrian is owned once
    got = np.sort(np.concatenate([BD.own_of(L, k, peds).ids for k in range(n)]))
    assert (got == np.arange(npeds)).all()


def _exchange_rank(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    from paper_1803_04782_gb300 import bands as B
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        comm = B.TorchComm(dist)
        other = 1 - rank
        sends = {other: np.arange(5 * (3 + rank), dtype=np.int32).reshape(-1, 5) + 100 * rank}
        recv = comm.exchange(sends)
        empty = comm.exchange({other: np.zeros((0, 5), np.int32)})
        out.put((rank, recv[other].tolist(), empty[other].shape))
    finally:
        dist.destroy_process_group()


def test_two_rank_exchange_delivers_what_the_neighbour_sent():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_exchange_rank, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = dict((r, (a, s)) for r, a, s in (q.get(timeout=120) for _ in procs))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert res[0][0] == (np.arange(20).reshape(-1, 5) + 100).tolist()
    assert res[1][0] == np.arange(15).reshape(-1, 5).tolist()
    assert res[0][1] == (0, 5) and res[1][1] == (0, 5)


def _scenes():
    # a closed room with exits on the north and south walls (pedestrians
    # leave across band edges' rows) and a corridor periodic in x and y
    a = SG.random_scene(90, 224, 1800, r=6, seed=61, obstacles=3, exits=("north", "south", "east"),
                        goal_mode="mixed", heading_mode="random")
    b = SG.random_scene(70, 192, 2500, r=5, seed=62, periodic_x=1, periodic_y=1, ring=False,
                        exits=(), goal_mode="fixed", heading_mode="random")
    return [a, b]


def oracle_stepper(layout, k, sc, D):
    """One rank's band stepped by the FP64 oracle: decide on the sub-lattice
    (field by direct superposition), numbered election, commit."""
    a, n = layout.rows(k)
    rows = np.arange(a, a + n) % layout.H
    cell = np.ascontiguousarray(sc.cell[rows])
    Dk = np.ascontiguousarray(D[rows])
    sub = SG.Scene("band", sc.W, n, sc.periodic_x, 0, cell, np.zeros((0, 2), np.int32),
                   np.zeros(0, np.uint8), np.zeros(0, np.uint8), sc.params)
    m = O.model(sub)

    def step(xy, heading, goal, ids, t):
        xy = np.ascontiguousarray(xy, np.int32).copy()
        heading = np.ascontiguousarray(heading, np.uint8).copy()
        alive = np.ones(xy.shape[0], np.uint8)
        occ, bad = O.occupancy(m, cell, xy, alive)
        assert bad == 0
        ch, _, _, _ = O.decide(m, cell, occ, xy, heading, goal, alive, Dk)
        won, _ = O.vote(m, t, xy, alive, ch, ids=ids)
        O.commit(m, cell, xy, heading, alive, ch, won)
        return xy, heading, alive

    return step


def _oracle_band_rank(rank, world, port, which, ticks, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        sc = _scenes()[which]
        m = O.model(sc)
        D = O.guidance(m, sc.cell)
        L = BD.BandLayout(sc.H, sc.periodic_y, int(sc.params["r"]), world)
        peds = BD.Peds(np.arange(sc.n, dtype=np.int32), sc.xy.copy(), sc.heading.copy(),
                       sc.goal.copy())
        own = BD.own_of(L, rank, peds)
        step = oracle_stepper(L, rank, sc, D)
        comm = BD.TorchComm(dist)
        left = 0
        for t in range(ticks):
            own, l = BD.band_tick(L, rank, comm, step, own, t)
            left += l
        out.put((rank, own.ids.tolist(), own.xy.tolist(), own.heading.tolist(), left))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("which,world", [(0, 2), (1, 2), (1, 3)])
def test_oracle_bands_reproduce_the_whole_lattice(which, world):
    ticks = 6
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_oracle_band_rank, args=(r, world, port, which, ticks, q))
             for r in range(world)]
    for p in procs:
        p.start()
    res = [q.get(timeout=300) for _ in procs]
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    sc = _scenes()[which]
    m = O.model(sc)
    D = O.guidance(m, sc.cell)
    st = O.State(sc)
    for _ in range(ticks):
        O.step(m, sc.cell, D, st)
    ids = np.concatenate([np.array(r[1], np.int64) for r in res])
    xy = np.concatenate([np.array(r[2], np.int64).reshape(-1, 2) for r in res])
    hd = np.concatenate([np.array(r[3], np.int64) for r in res])
    assert len(set(ids.tolist())) == len(ids)              # nobody owned twice
    alive = np.flatnonzero(st.alive)
    assert sorted(ids.tolist()) == alive.tolist()
    order = np.argsort(ids)
    np.testing.assert_array_equal(xy[order], st.xy[alive])
    np.testing.assert_array_equal(hd[order], st.heading[alive])
    assert sum(r[4] for r in res) == st.exited
    if which == 0:
        assert st.exited > 0
    # pedestrians crossed band edges during the run
    L = BD.BandLayout(sc.H, sc.periodic_y, int(sc.params["r"]), world)
    moved_band = L.owner(st.xy[alive, 1]) != L.owner(sc.xy[alive, 1])
    assert moved_band.sum() > 0
