"""CUDA path vs FP64 oracle at the benchmark's full sizes (GPU).

The workloads and the launch configuration are the ones bench.py times: the
16384 x 16384 floor (10^6 exit-seekers, r = 40) in 4 row bands and the
1000 x 200 corridor (20 000 walkers, r = 20) unbanded, as the bench's band
budget sets them, each with the autotuned footprint and graph-replayed ticks
with stage events on every 9th tick; and the batch of 256 uneven rooms stepped by one persistent launch
per tick.  The oracle cannot redo a whole 16384^2 lattice in seconds, so on
the floor and the batch it checks what it can compute one output at a time:
the field at sampled su (every band-edge row among them), the decisions of
sampled pedestrians (every one next to a band edge among them), teacher-forced
from the GPU's state at the start of the tick, and, exactly and for the whole
crowd, the vote and commit that the GPU's choices lead to.  Guidance is
compared on every su.  The corridor is small enough for the whole field and
every decision.  The learned surrogate is judged on the full floor as the
bench runs it.
"""
import numpy as np
import pytest

import bench
import oracle as O
import paper_1803_04782_gb300 as sfm
import scenegen as SG
from paper_1803_04782_gb300 import build as B
from parity import assert_field, compare_choices

pytestmark = pytest.mark.gpu

WARM_TICKS = 6  # graph-replayed ticks before the checked one


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    sfm.lib()


def _bench_sim(name, warm=WARM_TICKS):
    """A context in the configuration bench.py times for workload `name`."""
    sc, _ = bench.workload(name)
    sim = sfm.Sim(sc, hbm_budget_bytes=bench.band_budget(sc, bench.default_bands(name)))
    sim.autotune()
    sim.set_timing(bench.TIMING_EVERY)
    if warm:
        sim.step(warm)
    sim.sync()
    return sc, sim


def _check_vote_and_commit(m, sc, t, xy, hd, al, ch, won, after):
    """The oracle's vote and commit of the whole crowd, fed the GPU's choices,
    give exactly the GPU's winners and next state."""
    won_o, maxc = O.vote(m, t, xy, al, ch)
    assert maxc <= 8
    np.testing.assert_array_equal(won, won_o)
    xy_o, hd_o, al_o = xy.copy(), hd.copy(), al.copy()
    O.commit(m, sc.cell, xy_o, hd_o, al_o, ch, won_o)
    for got, exp in zip(after, (xy_o, hd_o, al_o)):
        np.testing.assert_array_equal(got, exp)


def _edge_rows(H, rows_per_band):
    e = {0, 1, H - 2, H - 1}
    for y in range(rows_per_band, H, rows_per_band):
        e |= {y - 2, y - 1, y, y + 1}
    return np.array(sorted(v for v in e if 0 <= v < H))


def test_floor_16384_full_size_ticks_against_the_oracle():
    """Checked at ticks 0 (run stage by stage, the first after the
    placement), 6, 60 and 200 (replayed from graphs; by tick 200, the
    workload's run length, the crowd has gathered at the exits)."""
    sc, sim = _bench_sim("floor", warm=0)
    with sim:
        st = sim.stats()
        assert st["bands"] >= 4 and st["n"] == 1_000_000
        band_rows = -(-sc.H // st["bands"])
        band_rows = -(-band_rows // 32) * 32
        m = O.model(sc)
        D = O.guidance(m, sc.cell)
        np.testing.assert_array_equal(sim.guidance(), D)
        rng = np.random.default_rng(31)
        W, H = sc.W, sc.H
        edges = _edge_rows(H, band_rows)
        exits = np.flatnonzero(sc.cell.ravel() == SG.EXIT)
        done = 0
        for tick in (0, WARM_TICKS, 60, 200):
            if tick > done:
                sim.step(tick - done)
            xy, hd, al = sim.peds()
            t = sim.stats()["t"]
            assert t == tick
            F = sim.field_banded()  # the field of this state, band by band
            occ, bad = O.occupancy(m, sc.cell, xy, al)
            assert bad == 0
            # sampled su: uniform, every band-edge row (and the lattice's first
            # and last rows) at random columns, and EXIT su
            req = [rng.integers(0, W * H, 16384),
                   (edges[:, None] * W + rng.integers(0, W, (edges.size, 512))).ravel(),
                   rng.choice(exits, 512, replace=False)]
            req = np.unique(np.concatenate(req)).astype(np.int64)
            Fo, So = O.field(m, sc.cell, occ, hd, 3, req)
            assert_field(F.ravel()[req], Fo, So, f"floor field at tick {tick} (sampled su)")
            # one tick from this state
            sim.step(1)
            done = tick + 1
            ch, won = sim.decisions()
            after = sim.peds()
            live = np.flatnonzero(al)
            near_edge = live[np.isin(xy[live, 1], edges)]
            peds = np.unique(np.concatenate([rng.choice(live, 20000, replace=False), near_edge]))
            peds = peds.astype(np.int32)
            ch_o, E, T, adm = O.decide(m, sc.cell, occ, xy, hd, sc.goal, al, D, peds)
            flips = compare_choices(ch[peds], ch_o, E, T, adm)
            assert flips <= 3, f"tick {tick}: {flips} tie flips in {peds.size} sampled decisions"
            _check_vote_and_commit(m, sc, t, xy, hd, al, ch, won, after)
            s = sim.stats()
            assert s["error_flags"] == 0 and s["max_registrants"] <= 8
            assert s["alive"] + s["exited"] == sc.n


def test_floor_8192_bands_equal_one_launch_over_200_ticks():
    """The 8192^2 floor (250 000 exit-seekers, r = 40) for 200 ticks: in 4
    row bands (the ring band buffer) and in one launch a tick, with the
    row-trimmed gather's dealt rounds and tickets, the crowd's positions,
    headings and decisions stay bit-identical at every 25th tick while the
    crowd gathers at the exits (footprints of ever more uneven cost)."""
    sc, _ = bench.workload("floor-mid")
    with sfm.Sim(sc, hbm_budget_bytes=bench.band_budget(sc, 4)) as a, sfm.Sim(sc) as b:
        assert a.stats()["bands"] == 4 and b.stats()["bands"] == 1
        for s in (a, b):
            s.set_footprint("32x32r")
        for _ in range(8):
            a.step(25)
            b.step(25)
            np.testing.assert_array_equal(a.decisions()[0], b.decisions()[0])
            for x, y in zip(a.peds(), b.peds()):
                np.testing.assert_array_equal(x, y)
        assert a.stats()["exited"] == b.stats()["exited"] > 0
        assert a.stats()["error_flags"] == 0 and b.stats()["error_flags"] == 0


def test_corridor_full_size_ticks_against_the_oracle():
    """Two replayed ticks after the warm-up, then two at tick 500 (the
    configuration's run length, the counter-flow jammed): the whole field,
    every decision, and the exact vote and commit."""
    sc, sim = _bench_sim("corridor")
    with sim:
        st = sim.stats()
        assert st["bands"] == 1 and st["n"] == 20000
        m = O.model(sc)
        D = O.guidance(m, sc.cell)
        flips = 0
        for k in range(4):
            if k == 2:
                sim.step(500 - sim.stats()["t"])
            xy, hd, al = sim.peds()
            t = sim.stats()["t"]
            F = sim.field_banded()
            occ, bad = O.occupancy(m, sc.cell, xy, al)
            assert bad == 0
            Fo, So = O.field(m, sc.cell, occ, hd)
            assert_field(F, Fo, So, "corridor field")
            sim.step(1)
            ch, won = sim.decisions()
            after = sim.peds()
            ch_o, E, T, adm = O.decide(m, sc.cell, occ, xy, hd, sc.goal, al, D,
                                       Ffull=Fo.ravel(), Sfull=So.ravel())
            flips += compare_choices(ch, ch_o, E, T, adm)
            _check_vote_and_commit(m, sc, t, xy, hd, al, ch, won, after)
            assert int(after[2].sum()) == sc.n  # periodic in x, no exits: nobody leaves
        assert flips <= 6, f"{flips} tie flips"


def test_batch_of_256_rooms_full_size_tick_against_the_oracle():
    """Checked after 3 replayed ticks and again at tick 60, when the rooms'
    crowds have moved towards their exits and some have emptied."""
    scenes = SG.batch(nscenes=256)
    side = np.array([sc.W for sc in scenes])
    rad = np.array([sc.params["r"] for sc in scenes])
    rng = np.random.default_rng(32)
    pick = {int(np.argmax(side)), int(np.argmin(side)), int(np.argmax(rad)),
            int(np.argmin(rad)), *map(int, rng.choice(len(scenes), 2, replace=False))}
    models = {i: O.model(scenes[i]) for i in pick}
    with sfm.Batch(scenes) as bt:
        bt.autotune()
        for first, upto in ((True, 3), (False, 60)):
            bt.step(upto - bt.stats()["t"])
            bt.sync()
            xs, hs, als = bt.peds()
            t = bt.stats()["t"]
            bt.step(1)
            Fs = bt.fields()
            chs, wons = bt.decisions()
            after = bt.peds()
            s = bt.stats()
            assert s["error_flags"] == 0 and s["max_registrants"] <= 8
            Ds = bt.guidance() if first else None
            for i in sorted(pick):
                sc, m = scenes[i], models[i]
                D = O.guidance(m, sc.cell)
                if first:
                    np.testing.assert_array_equal(Ds[i], D)
                xy, hd, al = xs[i], hs[i], als[i]
                occ, bad = O.occupancy(m, sc.cell, xy, al)
                assert bad == 0
                req = np.unique(rng.integers(0, sc.W * sc.H, 4096)).astype(np.int64)
                Fo, So = O.field(m, sc.cell, occ, hd, 3, req)
                assert_field(Fs[i].ravel()[req], Fo, So, f"batch scene {i} field at tick {t}")
                live = np.flatnonzero(al)
                if live.size:
                    peds = np.sort(rng.choice(live, min(4096, live.size),
                                              replace=False)).astype(np.int32)
                    ch_o, E, T, adm = O.decide(m, sc.cell, occ, xy, hd, sc.goal, al, D, peds)
                    flips = compare_choices(chs[i][peds], ch_o, E, T, adm)
                    assert flips <= 3, f"scene {i} tick {t}: {flips} tie flips"
                _check_vote_and_commit(m, sc, t, xy, hd, al, chs[i], wons[i],
                                       (after[0][i], after[1][i], after[2][i]))


def test_surrogate_on_the_full_floor_meets_the_flip_target():
    """The learned surrogate as bench.py runs it: trained on the GPU for 150
    steps (bench.SURROGATE_TRAINING: the 4096^2 torus canvas, then two
    4096^2 floors with walls, exits and exit-seekers), its margin bound
    calibrated on the 16384^2
    floor (99.9th percentile), then judged there by the exact path after 3
    more ticks.  With the exact fallback at most 0.1 % of the decisions may
    differ from the exact ones, part of the crowd must be decided on the
    surrogate alone, and the network must leave a smaller field error than
    the near part without it."""
    init = sfm.flatten_params(SG.surrogate_init(0))
    trained, curves = bench.train_surrogate(sfm, None, init)
    assert all(np.isfinite(c).all() for c in curves)
    assert curves[0][-10:].mean() < 0.5 * curves[0][:3].mean()
    sc, _ = bench.workload("floor")
    with sfm.Sim(sc) as fsim:
        fsim.step(5)
        live = int(fsim.stats()["alive"])
        evs = {}
        for name, params in (("net", trained), ("near_only", 0 * init)):
            with sfm.Surrogate(coarsen=8, near_radius=3, target_scale=20.0, params=params) as sur:
                d = sur.calibrate(fsim, 0.999)
                assert 0.0 < d < np.inf
                fsim.step(3)
                evs[name] = sur.eval(fsim)
    ev = evs["net"]
    assert ev["decided"] >= 0.99 * live, ev
    assert ev["flip_rate"] <= 1e-3, ev
    assert ev["fallback_rate"] < 1.0, ev
    assert ev["field_rel_err"] < 0.5 * evs["near_only"]["field_rel_err"], evs
