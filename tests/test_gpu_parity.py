"""CUDA path vs FP64 oracle, element by element (GPU).

Scenes span several 32x32 tiles with ragged edges, periodic and closed
boundaries, radii from 0 (no field) to 40 (halo wider than a tile), dense and
sparse crowds, exit-seekers and fixed-direction walkers.  Each tick the GPU
restarts from the oracle's own state, so no GPU output ever feeds the oracle.
"""
import numpy as np
import pytest

import oracle as O
import paper_1803_04782_gb300 as sfm
import scenegen as SG
from paper_1803_04782_gb300 import build as B
from parity import OracleRun, assert_field, compare_choices, sized_subset

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _built():
    B.build()
    sfm.lib()


def _room_mixed():
    return SG.random_scene(100, 77, 300, r=10, seed=101, obstacles=4, exits=("east", "north"),
                           goal_mode="mixed", heading_mode="random")


def _corridor_periodic():
    return SG.random_scene(150, 40, 800, r=12, seed=102, periodic_x=1, exits=(),
                           goal_mode="fixed", heading_mode="goal")


def _torus():
    return SG.random_scene(64, 64, 1000, r=9, seed=103, periodic_x=1, periodic_y=1, ring=False,
                           exits=(), goal_mode="fixed", heading_mode="random")


def _no_field():
    return SG.random_scene(37, 29, 100, r=0, seed=104, obstacles=2, exits=("west", "south"))


def _tall_r1():
    return SG.random_scene(33, 130, 400, r=1, seed=105, exits=("north",), goal_mode="mixed",
                           heading_mode="random")


def _tiny():
    return SG.random_scene(5, 5, 4, r=2, seed=106, exits=("east",), exit_len=1,
                           goal_mode="mixed")


def _dense():
    sc = SG.random_scene(40, 40, 38 * 38 - 2, r=4, seed=107, exits=("east", "west"),
                         exit_len=6, heading_mode="random")
    return sc


def _wide_radius():
    return SG.random_scene(200, 150, 2000, r=40, seed=108, obstacles=6, exits=("east",),
                           exit_len=20, goal_mode="mixed", heading_mode="random")


def _thin_torus():
    # periodic extent exactly 2r+1: a tile's halo wraps around several times
    return SG.random_scene(11, 50, 120, r=5, seed=109, periodic_x=1, exits=("south",),
                           goal_mode="mixed", heading_mode="random")


def _radius41():
    # largest radius of the wide class-table stride (114: no lane range test)
    return SG.random_scene(150, 140, 1400, r=41, seed=113, periodic_x=1, exits=("north",),
                           goal_mode="mixed", heading_mode="random")


def _radius47():
    # narrow class-table stride (102): out-of-reach lanes are masked
    return SG.random_scene(160, 170, 1500, r=47, seed=110, periodic_y=1, exits=("east",),
                           goal_mode="mixed", heading_mode="random")


def _radius50():
    # largest radius of the class-table gather
    return SG.random_scene(230, 140, 1200, r=50, seed=112, obstacles=3, exits=("west",),
                           goal_mode="mixed", heading_mode="random")


def _radius53():
    # beyond the class-table gather: the three-component gather takes over
    return SG.random_scene(200, 150, 1000, r=53, seed=114, obstacles=2, exits=("south",),
                           goal_mode="mixed", heading_mode="random")


def _radius8():
    # smallest radius of the row-trimmed 32 x 16 footprint (2r + 1 = 17 rows)
    return SG.random_scene(131, 97, 900, r=8, seed=115, obstacles=2, exits=("east", "south"),
                           goal_mode="mixed", heading_mode="random")


def _radius16():
    # smallest radius of the row-trimmed 32 x 32 footprint (2r + 1 = 33 rows)
    return SG.random_scene(150, 113, 1100, r=16, seed=116, periodic_y=1, exits=("west",),
                           goal_mode="mixed", heading_mode="random")


SCENES = {f.__name__[1:]: f for f in (_room_mixed, _corridor_periodic, _torus, _no_field,
                                      _tall_r1, _tiny, _dense, _wide_radius, _thin_torus,
                                      _radius41, _radius47, _radius50, _radius53, _radius8,
                                      _radius16)}


@pytest.mark.parametrize("name", list(SCENES))
def test_static_field_and_guidance(name):
    sc = SCENES[name]()
    orc = OracleRun(sc)
    occ0 = np.full(sc.W * sc.H, -1, np.int32)
    Fs, Ss = O.field(orc.m, sc.cell, occ0, np.zeros(1, np.uint8), parts=1)
    with sfm.Sim(sc) as sim:
        assert_field(sim.static_field(), Fs, Ss, "static field")
        np.testing.assert_array_equal(sim.guidance(), orc.D)


@pytest.mark.parametrize("name", list(SCENES))
def test_oracle_forced_ticks(name):
    sc = SCENES[name]()
    orc = OracleRun(sc)
    flips = decisions = 0
    with sfm.Sim(sc) as sim:
        for _ in range(6):
            st = orc.st
            sim.place(st.xy, st.heading, st.goal, st.alive)
            sim.set_time(st.t)
            sim.step(1)
            Fo, So = orc.field()
            assert_field(sim.field(), Fo, So)
            ch_o, E, T, adm = orc.decide(Ffull=Fo.ravel(), Sfull=So.ravel())
            ch_g, won_g = sim.decisions()
            f = compare_choices(ch_g, ch_o, E, T, adm)
            xy_g, h_g, a_g = sim.peds()
            won_o, maxc = orc.advance(ch_o)
            assert maxc <= 8
            if f == 0:
                np.testing.assert_array_equal(won_g, won_o)
                np.testing.assert_array_equal(xy_g, orc.st.xy)
                np.testing.assert_array_equal(h_g, orc.st.heading)
                np.testing.assert_array_equal(a_g, orc.st.alive)
            flips += f
            decisions += int(st.alive.sum())
            stats = sim.stats()
            assert stats["error_flags"] == 0 and stats["max_registrants"] <= 8
    # every flip was checked to lie inside the tie tolerance; exact ties (equal
    # term multisets, frequent at r = 1) are broken differently by FP32 and
    # FP64 sums, so only their rate is bounded
    assert flips <= max(3, 0.02 * decisions), f"{flips} tie flips in {decisions} decisions"


@pytest.mark.parametrize("which", ["paper_r1", "paper_r3_4dir", "room", "tall_r1"])
def test_near_tie_counter_matches_the_oracle(which):
    """The decision kernel's near-tie counter (sfm_stats: decisions whose two
    best admissible energies lie within 1e-5 of their magnitude |F| + |own|
    + |guidance|) against the oracle's count by the same rule in FP64, on the
    same state.  The GPU's energies differ from the oracle's by at most the
    tie tolerance 1e-5 T (T: sum of term magnitudes), so a pedestrian whose
    oracle gap lies within that of the threshold may be counted either way;
    every other one must be counted exactly as the oracle counts it."""
    sc = {"paper_r1": lambda: SG.paper_scene(side=120, density=0.5, ndir=8, r=1, seed=41),
          "paper_r3_4dir": lambda: SG.paper_scene(side=150, density=0.3, ndir=4, r=3, seed=42),
          "room": SG.room, "tall_r1": _tall_r1}[which]()
    orc = OracleRun(sc)
    with sfm.Sim(sc) as sim:
        for _ in range(3):
            st = orc.st
            sim.place(st.xy, st.heading, st.goal, st.alive)
            sim.set_time(st.t)
            sim.step(1)
            stats = sim.stats()
            Fo, So = orc.field()
            occ, _ = O.occupancy(orc.m, sc.cell, st.xy, st.alive)
            ch_o, E, T, adm, Mag = O.decide(orc.m, sc.cell, occ, st.xy, st.heading, st.goal,
                                            st.alive, orc.D, None, Fo.ravel(), So.ravel(),
                                            magnitudes=True)
            live = st.alive.astype(bool)
            assert stats["decided"] == int(live.sum())
            b, s2 = O.best_two(E, adm)
            i = np.arange(len(b))
            ok = live & (s2 >= 0)
            sj = np.where(s2 >= 0, s2, 0)
            with np.errstate(invalid="ignore"):   # dead pedestrians: inf - inf
                gap = E[i, sj] - E[i, b]
                thr = 1e-5 * (Mag[i, b] + Mag[i, sj])
                band = 1e-5 * (T[i, b] + T[i, sj])
                lo = int((ok & (gap <= thr - band)).sum())
                hi = int((ok & (gap <= thr + band)).sum())
            exact = int((ok & O.near_ties(E, Mag, adm)).sum())
            assert lo <= stats["near_ties"] <= hi, (lo, exact, hi, stats["near_ties"])
            ch_g, _ = sim.decisions()
            compare_choices(ch_g, ch_o, E, T, adm)
            orc.advance(ch_o)
        if which == "paper_r1":
            assert stats["near_ties"] > 0   # equal term multisets make exact ties at r = 1


@pytest.mark.parametrize("r,ndir,density", [(3, 8, 0.5), (38, 4, 0.5), (3, 1, 0.9)])
def test_paper_shaped_scenes_oracle_forced(r, ndir, density):
    """The paper's experiment shape (Sec. 5: periodic lattice, no walls or
    exits, fixed-direction walkers in 1/2/4/8 flows, 1x1 pedestrians, walk
    period 1) at the ends of Table III's field geometries (7x7, r = 3, and
    77x77, r = 38) and the densest cell of the 360-combination sweep: the
    whole field and every decision against the oracle, each tick restarted
    from the oracle's state; votes and commits exact when no tie flipped."""
    side = 96 if r == 3 else 160
    sc = SG.paper_scene(side=side, density=density, ndir=ndir, r=r, seed=40 + r + ndir)
    orc = OracleRun(sc)
    flips = decisions = 0
    with sfm.Sim(sc) as sim:
        for _ in range(3):
            st = orc.st
            sim.place(st.xy, st.heading, st.goal, st.alive)
            sim.set_time(st.t)
            sim.step(1)
            Fo, So = orc.field()
            assert_field(sim.field(), Fo, So)
            ch_o, E, T, adm = orc.decide(Ffull=Fo.ravel(), Sfull=So.ravel())
            ch_g, won_g = sim.decisions()
            f = compare_choices(ch_g, ch_o, E, T, adm)
            xy_g, h_g, a_g = sim.peds()
            won_o, maxc = orc.advance(ch_o)
            assert maxc <= 8
            if f == 0:
                np.testing.assert_array_equal(won_g, won_o)
                np.testing.assert_array_equal(xy_g, orc.st.xy)
                np.testing.assert_array_equal(h_g, orc.st.heading)
            flips += f
            decisions += int(st.alive.sum())
    assert flips <= max(3, 0.02 * decisions), f"{flips} tie flips in {decisions} decisions"


def test_free_running_room_100x100_r10_50_ticks():
    """The 100x100 room with 200 exit-seekers, radius 10, 50 ticks: the GPU
    runs on its own and must stay identical to the oracle's run."""
    sc = SG.room()
    orc = OracleRun(sc)
    with sfm.Sim(sc) as sim:
        for t in range(sc.steps):
            sim.step(1)
            Fo, So = orc.field()
            assert_field(sim.field(), Fo, So, f"field at tick {t}")
            ch_o, E, T, adm = orc.decide(Ffull=Fo.ravel(), Sfull=So.ravel())
            ch_g, won_g = sim.decisions()
            assert compare_choices(ch_g, ch_o, E, T, adm) == 0, f"tie flip at tick {t}"
            orc.advance(ch_o)
            xy_g, h_g, a_g = sim.peds()
            np.testing.assert_array_equal(xy_g, orc.st.xy)
            np.testing.assert_array_equal(a_g, orc.st.alive)
            np.testing.assert_array_equal(h_g, orc.st.heading)
        s = sim.stats()
        assert s["alive"] + s["exited"] == sc.n
        assert s["exited"] == orc.st.exited


@pytest.mark.parametrize("bands", [1, 4])
def test_walk_periods_free_running_against_the_oracle(bands):
    """Walk periods (Sec. 2) drawn in 1..5 with random phases on a room of
    mixed exit-seekers and walkers: the GPU runs 20 ticks on its own, banded
    or not, and stays identical to the oracle, which gates each pedestrian
    to its own ticks; inactive pedestrians stay and register nowhere."""
    sc = SG.random_scene(200, 160, 3000, r=12, seed=131, obstacles=4, exits=("east", "north"),
                         goal_mode="mixed", heading_mode="random")
    rng = np.random.default_rng(7)
    period = rng.integers(1, 6, size=sc.n).astype(np.uint8)
    phase = (rng.integers(0, 255, size=sc.n) % period).astype(np.uint8)
    orc = OracleRun(sc)
    orc.st.period, orc.st.phase = period, phase
    budget = sfm.band_budget(sc.W, sc.H, 32) if bands > 1 else 0
    with sfm.Sim(sc, hbm_budget_bytes=budget) as sim:
        assert (sim.stats()["bands"] > 1) == (bands > 1)
        sim.set_walk_periods(period, phase)
        for t in range(20):
            sim.step(1)
            Fo, So = orc.field()
            ch_o, E, T, adm = orc.decide(Ffull=Fo.ravel(), Sfull=So.ravel())
            active = (t % period.astype(int)) == phase
            ch_o = O.gate_periods(orc.st.t, period, phase, ch_o)
            ch_g, won_g = sim.decisions()
            alive = orc.st.alive.astype(bool)
            assert not np.any(ch_g[alive & ~active]), f"inactive pedestrian moved at tick {t}"
            assert compare_choices(ch_g, ch_o, E, T, adm) == 0, f"tie flip at tick {t}"
            won_o, _ = orc.advance(ch_o)
            np.testing.assert_array_equal(won_g, won_o)
            for x, y in zip(sim.peds(), (orc.st.xy, orc.st.heading, orc.st.alive)):
                np.testing.assert_array_equal(x, y)
        # switching periods off again is the plain model; bad periods are refused
        sim.set_walk_periods(None)
        bad = period.copy()
        bad[0] = 0
        with pytest.raises(sfm.SfmError) as e:
            sim.set_walk_periods(bad, phase)
        assert e.value.status == sfm.SFM_EINVAL
        with pytest.raises(sfm.SfmError):
            sim.set_walk_periods(period, period)  # phase == period


@pytest.mark.parametrize("bands,periodic,r", [(1, 0, 10), (4, 0, 10), (1, 1, 10), (4, 0, 36)])
def test_multi_su_pedestrians_free_running_against_the_oracle(bands, periodic, r):
    """Multi-su pedestrians (Sec. 2, Table V): 1x1, 3x3 and 5x5 rectangles in
    one crowd run 25 ticks on their own, banded or not, closed with exits or
    on a torus, identical to the oracle (admissibility over the entered
    strip, claims in the vote, exits through any su of the rectangle).  At
    r = 36 the row-trimmed footprint gathers the field, banded into the ring
    band buffer.  A decision that differs from the oracle's only inside the
    tie tolerance is counted, and the oracle then takes the GPU's choice (as
    valid as its own), so the two runs stay comparable."""
    sc = SG.random_scene(160, 128, 2600, r=r, seed=141, obstacles=0 if periodic else 3,
                         periodic_x=periodic, periodic_y=periodic, ring=not periodic,
                         exits=() if periodic else ("east", "west"), exit_len=14,
                         goal_mode="mixed" if not periodic else "fixed", heading_mode="random")
    rng = np.random.default_rng(11)
    size = rng.choice(np.array([1, 3, 5], np.uint8), size=sc.n, p=[0.6, 0.3, 0.1])
    sub, size = sized_subset(sc, size)
    assert (size == 5).sum() > 10 and (size == 3).sum() > 50
    orc = OracleRun(sub)
    orc.st.w, orc.st.h = size, size
    budget = sfm.band_budget(sub.W, sub.H, 32) if bands > 1 else 0
    with sfm.Sim(sub, place=False, hbm_budget_bytes=budget) as sim:
        if r > 30:
            sim.set_footprint("32x32r")
        sim.place_sized(sub.xy, sub.heading, sub.goal, np.ones(sub.n, np.uint8), size, size)
        flips = 0
        for t in range(25):
            sim.step(1)
            Fo, So = orc.field()
            ch_o, E, T, adm = orc.decide(Ffull=Fo.ravel(), Sfull=So.ravel())
            ch_g, won_g = sim.decisions()
            f = compare_choices(ch_g, ch_o, E, T, adm)
            flips += f
            won_o, maxc = orc.advance(np.asarray(ch_g, np.uint8) if f else ch_o)
            assert maxc <= 8
            np.testing.assert_array_equal(won_g, won_o, err_msg=f"tick {t}")
            for x, y in zip(sim.peds(), (orc.st.xy, orc.st.heading, orc.st.alive)):
                np.testing.assert_array_equal(x, y)
        st = sim.stats()
        assert st["error_flags"] == 0 and st["exited"] == orc.st.exited
        assert flips <= 3, f"{flips} tie flips in 25 ticks"
        if not periodic:
            assert np.any((orc.st.alive == 0) & (size > 1)), "no multi-su pedestrian left"


def test_multi_su_placement_errors():
    sc = SG.random_scene(60, 50, 40, r=4, seed=142, exits=("east",))
    sub, size = sized_subset(sc, np.full(sc.n, 3, np.uint8))
    one = np.ones(sub.n, np.uint8)
    with sfm.Sim(sub, place=False) as sim:
        bad = size.copy()
        bad[0] = 2
        with pytest.raises(sfm.SfmError) as e:
            sim.place_sized(sub.xy, sub.heading, sub.goal, one, bad, size)
        assert e.value.status == sfm.SFM_EINVAL
        xy = sub.xy.copy()
        xy[1] = xy[0] + np.array([2, 0], np.int32)   # rectangles overlap
        with pytest.raises(sfm.SfmError) as e:
            sim.place_sized(xy, sub.heading, sub.goal, one, size, size)
        assert e.value.status == sfm.SFM_ECONFLICT
        xy = sub.xy.copy()
        xy[0] = (1, 1)                                # rectangle on the wall ring
        with pytest.raises(sfm.SfmError) as e:
            sim.place_sized(xy, sub.heading, sub.goal, one, size, size)
        assert e.value.status == sfm.SFM_ECONFLICT
        sim.place_sized(sub.xy, sub.heading, sub.goal, one, size, size)
        sim.step(3)
        assert sim.stats()["error_flags"] == 0


@pytest.mark.parametrize("periodic,footprint,r,rows", [(0, "32x16", 7, 64), (1, "16x16", 7, 64),
                                                       (0, "32x32r", 20, 64), (1, "32x32r", 16, 64),
                                                       (1, "32x32r", 9, 64), (0, "32x32r", 40, 32),
                                                       ("x", "32x32r", 36, 64)])
def test_banded_field_is_bitwise_the_unbanded_field(periodic, footprint, r, rows):
    """Divide-and-conquer (Eq. 1): row bands under an HBM budget give exactly
    the unbanded field and the same ticks, whatever the footprint (the band
    halo rows fall inside footprints).  With the row-trimmed footprint and y
    not periodic the band buffer is a ring that each band's launch extends
    by the next band's first 32 rows, here also with bands of 32 rows (the
    upper halo row then comes from two bands back) and a last band shorter
    than 32 rows (no launch of its own), and periodic in x only (a
    corridor-like lattice: the ring with wrapped columns)."""
    px, py = (1, 0) if periodic == "x" else (periodic, periodic)
    sc = SG.random_scene(300, 260, 5000, r=r, seed=111, periodic_x=px, periodic_y=py,
                         ring=not (px or py), exits=() if (px or py) else ("east",),
                         goal_mode="mixed", heading_mode="random")
    budget = sfm.band_budget(sc.W, sc.H, rows)
    with sfm.Sim(sc) as a, sfm.Sim(sc, hbm_budget_bytes=budget) as b:
        b.set_footprint(footprint)
        assert b.stats()["bands"] >= 4
        a.compute_field()
        np.testing.assert_array_equal(a.field(), b.field_banded())
        for _ in range(5):
            a.step(1)
            b.step(1)
            np.testing.assert_array_equal(a.decisions()[0], b.decisions()[0])
            for x, y in zip(a.peds(), b.peds()):
                np.testing.assert_array_equal(x, y)
        a.compute_field()
        np.testing.assert_array_equal(a.field(), b.field_banded())


@pytest.mark.parametrize("name", ["room_mixed", "torus", "thin_torus", "wide_radius", "radius41",
                                  "radius47", "radius50", "dense", "tall_r1", "corridor_periodic",
                                  "tiny", "radius8", "radius16"])
def test_all_gather_footprints_give_the_same_field_and_ticks(name):
    """The 16x16 and 32x16 footprints and the row-trimmed 32x32 and 32x16
    ones add each su's terms in the same order: fields and ticks are bitwise
    equal, and equal to the autotuner's choice (where the radius is below
    their range the row-trimmed shapes run as the 32x16 gather)."""
    sc = SCENES[name]()
    sims = [sfm.Sim(sc) for _ in range(len(sfm.FOOTPRINTS) + 1)]
    try:
        for s, fp in zip(sims, sfm.FOOTPRINTS):
            s.set_footprint(fp)
        assert sims[-1].autotune() in sfm.FOOTPRINTS
        for s in sims:
            s.compute_field()
        a = sims[0]
        for s in sims[1:]:
            np.testing.assert_array_equal(a.field(), s.field())
        for _ in range(3):
            for s in sims:
                s.step(1)
            for s in sims[1:]:
                np.testing.assert_array_equal(a.field(), s.field())
                np.testing.assert_array_equal(a.decisions()[0], s.decisions()[0])
                for x, y in zip(a.peds(), s.peds()):
                    np.testing.assert_array_equal(x, y)
        with pytest.raises(sfm.SfmError) as e:
            sfm._check(a.ctx, sfm.lib().sfm_set_field_footprint(a.ctx, len(sfm.FOOTPRINTS)))
        assert e.value.status == sfm.SFM_EINVAL
    finally:
        for s in sims:
            s.close()


@pytest.mark.parametrize("name", ["room_mixed", "torus", "dense", "tall_r1", "thin_torus",
                                  "radius41", "no_field"])
def test_grid_and_pedestrian_list_binning_give_the_same_ticks(name):
    """Binning by scanning the class grid and binning from the pedestrian
    list (atomic counts, in-bin rank) produce the same records: fields and
    ticks are bitwise equal, exits and full bins included."""
    sc = SCENES[name]()
    with sfm.Sim(sc) as a, sfm.Sim(sc) as b:
        a.set_binning("grid")
        b.set_binning("peds")
        a.compute_field()
        b.compute_field()
        np.testing.assert_array_equal(a.field(), b.field())
        for t in range(6):
            a.step(1)
            b.step(1)
            np.testing.assert_array_equal(a.field(), b.field(), err_msg=f"tick {t}")
            np.testing.assert_array_equal(a.decisions()[0], b.decisions()[0])
            np.testing.assert_array_equal(a.decisions()[1], b.decisions()[1])
            for x, y in zip(a.peds(), b.peds()):
                np.testing.assert_array_equal(x, y)
        assert a.stats()["exited"] == b.stats()["exited"]
        with pytest.raises(sfm.SfmError) as e:
            sfm._check(a.ctx, sfm.lib().sfm_set_binning(a.ctx, 3))
        assert e.value.status == sfm.SFM_EINVAL


@pytest.mark.parametrize("variant", ["plain", "periods", "sized"])
def test_many_ticks_in_one_call_equal_single_ticks(variant):
    """step(20) replays graphs of 8 ticks and of 1 tick; the trajectory equals
    20 calls of step(1), with walk periods (gated on the device's tick
    counter) and with multi-su pedestrians."""
    sc = SG.random_scene(200, 160, 3000, r=9, seed=151, obstacles=3, exits=("east",),
                         goal_mode="mixed", heading_mode="random")
    size = None
    if variant == "sized":
        rng = np.random.default_rng(3)
        sc, size = sized_subset(sc, rng.choice(np.array([1, 3], np.uint8), size=sc.n))
    with sfm.Sim(sc, place=size is None) as a, sfm.Sim(sc, place=size is None) as b:
        if size is not None:
            for s in (a, b):
                s.place_sized(sc.xy, sc.heading, sc.goal, np.ones(sc.n, np.uint8), size, size)
        if variant == "periods":
            per, pha = SG.walk_periods(sc.n, 4)
            for s in (a, b):
                s.set_walk_periods(per, pha)
        for _ in range(20):
            a.step(1)
        b.step(20)
        for x, y in zip(a.peds(), b.peds()):
            np.testing.assert_array_equal(x, y)
        assert a.stats()["exited"] == b.stats()["exited"]
        assert b.stats()["error_flags"] == 0


@pytest.mark.parametrize("banded,every", [(False, 1), (True, 1), (False, 4), (True, 9)])
def test_timed_ticks_replay_the_same_ticks(banded, every):
    """With stage timing on, timed ticks after the first replay a one-tick
    graph whose stage events are event record nodes, re-pointed before each
    replay; with every = k > 1 only every k-th tick is timed and the others
    replay the untimed graphs.  The trajectory equals untimed stepping, each
    stage reports time for every timed tick, the stages fit inside the whole
    tick, and a placement drops the timed graph (the next timed ticks follow
    the new crowd)."""
    sc = SG.random_scene(200, 160, 3000, r=9, seed=152, obstacles=3, exits=("east",),
                         goal_mode="mixed", heading_mode="random")
    budget = sfm.band_budget(sc.W, sc.H, 64) if banded else 0
    with sfm.Sim(sc, hbm_budget_bytes=budget) as a, sfm.Sim(sc, hbm_budget_bytes=budget) as b:
        assert (a.stats()["bands"] > 1) == banded
        a.step(12)
        b.set_timing(every)
        b.stage_times()
        b.step(5)
        b.step(7)
        ms, ticks = b.stage_times()
        assert ticks == -(-12 // every)
        for x, y in zip(a.peds(), b.peds()):
            np.testing.assert_array_equal(x, y)
        for k in ("bin", "field", "decide", "vote", "commit", "step"):
            assert ms[k] > 0.0, k
        parts = sum(ms[k] for k in ("bin", "field", "decide", "vote", "commit"))
        assert parts <= ms["step"] * 1.0001
        # a new placement: the timed graph is rebuilt for the new crowd
        for s in (a, b):
            s.place(sc.xy[: sc.n // 2], sc.heading[: sc.n // 2], sc.goal[: sc.n // 2])
        b.set_timing(every)  # the next tick is a timed one
        a.step(4)
        b.step(4)
        for x, y in zip(a.peds(), b.peds()):
            np.testing.assert_array_equal(x, y)
        assert b.stage_times()[1] == -(-4 // every)
        assert b.stats()["error_flags"] == 0
        with pytest.raises(sfm.SfmError) as e:
            b.set_timing(-1)
        assert e.value.status == sfm.SFM_EINVAL


@pytest.mark.parametrize("variant", ["plain", "sized", "periods", "pinned"])
def test_place_step_read_loop_equals_plain_ticks(variant):
    """The end-to-end loop (place the crowd read back, step one tick, read)
    keeps the tick graphs across placements of as many pedestrians into the
    same arrays, and follows the trajectory of plain ticks.  With walk periods
    a placement turns them off, so that loop drops its graphs and is compared
    with ticks whose periods are cleared the same way."""
    sc = SG.random_scene(200, 160, 3000, r=9, seed=153, obstacles=3, exits=("east",),
                         goal_mode="mixed", heading_mode="random")
    size = None
    if variant == "sized":
        rng = np.random.default_rng(5)
        sc, size = sized_subset(sc, rng.choice(np.array([1, 3], np.uint8), size=sc.n))
    with sfm.Sim(sc, place=size is None) as a, sfm.Sim(sc, place=size is None) as b:
        def put(s, xy, h, alive):
            if size is None:
                s.place(xy, h, sc.goal, alive)
            else:
                s.place_sized(xy, h, sc.goal, alive, size, size)
        if size is not None:
            for s in (a, b):
                put(s, sc.xy, sc.heading, np.ones(sc.n, np.uint8))
        a.step(3)
        b.step(3)  # builds b's graphs
        if variant == "pinned":  # placed and read in place through pinned buffers (n = 3000 = 0 mod 4)
            xy0, h0, a0 = b.peds()
            hx, hh, hg, ha = _arrays_as("pinned", xy0, h0, sc.goal, a0)
        for tick in range(8):
            if variant == "periods" and tick == 4:
                per, pha = SG.walk_periods(sc.n, 3)
                for s in (a, b):
                    s.set_walk_periods(per, pha)
            if variant == "pinned":
                sfm.sfm_place(b.ctx, hx, hh, hg, ha)
                a.step(1)
                b.step(1)
                sfm.sfm_read_peds(b.ctx, hx, hh, ha)
                for x, y in zip(a.peds(), (hx, hh, ha)):
                    np.testing.assert_array_equal(x, y.numpy())
                continue
            xy, h, alive = b.peds()
            put(b, xy, h, alive)
            if variant == "periods" and tick >= 4:
                put(a, *a.peds())  # a placement clears the walk periods on both
            a.step(1)
            b.step(1)
            for x, y in zip(a.peds(), b.peds()):
                np.testing.assert_array_equal(x, y)
        assert b.stats()["error_flags"] == 0


def _arrays_as(kind, *arrays):
    """NumPy arrays (pageable host memory), or torch tensors in pinned host
    memory or on the GPU: the placement reads the last two in place.
    "pinned_unaligned": pinned tensors one element into their allocation, so
    that no buffer is aligned for the wide accesses."""
    if kind == "numpy":
        return [np.ascontiguousarray(a) for a in arrays]
    import torch
    ts = [torch.from_numpy(np.ascontiguousarray(a)) for a in arrays]
    if kind == "pinned_unaligned":
        out = []
        for t in ts:
            big = torch.empty((t.shape[0] + 1,) + tuple(t.shape[1:]), dtype=t.dtype).pin_memory()
            big[1:] = t
            out.append(big[1:])
        return out
    return [t.pin_memory() if kind == "pinned" else t.cuda() for t in ts]


@pytest.mark.parametrize("src", ["numpy", "pinned", "pinned_unaligned", "device"])
def test_placement_keeping_the_graphs_equals_a_fresh_placement(src):
    """A placement of as many 1x1 pedestrians keeps the tick graphs and
    rewrites the grid entries of the pedestrians it changes only, whether it
    copies pageable host arrays or reads pinned host or device buffers in
    place.  Moves, swapped positions (a su one changed pedestrian leaves and
    another claims), deaths, revivals and heading changes give the same
    fields, decisions and ticks as a fresh context placed with that state;
    overlapping, walled-in and off-lattice placements are still refused, and a
    valid one then works."""
    sc = SG.random_scene(120, 90, 1501, r=6, seed=161, obstacles=3, exits=("east", "north"),
                         goal_mode="mixed", heading_mode="random")  # n = 1 (mod 4): a ragged quad
    rng = np.random.default_rng(17)
    with sfm.Sim(sc) as a:
        a.step(12)
        xy, h, al = a.peds()
        assert (al == 0).any()  # some have left through the exits
        xy, h, al = xy.copy(), h.copy(), al.copy()
        live = np.flatnonzero(al)
        sw = rng.choice(live, 20, replace=False)
        xy[sw[:10]], xy[sw[10:]] = xy[sw[10:]].copy(), xy[sw[:10]].copy()
        rest = np.setdiff1d(live, sw)
        kill = rng.choice(rest, 30, replace=False)
        al[kill] = 0
        turn = rng.choice(rest, 60, replace=False)
        h[turn] = rng.integers(0, 9, turn.size)
        taken = set(map(tuple, xy[al == 1]))
        free = [(x, y) for y in range(sc.H) for x in range(sc.W)
                if sc.cell[y, x] == SG.FREE and (x, y) not in taken]
        free = [free[i] for i in rng.choice(len(free), 80, replace=False)]
        mov = rng.choice(np.setdiff1d(rest, kill), 40, replace=False)
        xy[mov] = free[:40]
        dead = np.flatnonzero(al == 0)
        rev = rng.choice(dead, min(40, dead.size), replace=False)
        xy[rev] = free[40:40 + rev.size]
        al[rev] = 1
        a.place(*_arrays_as(src, xy, h, sc.goal, al))
        t = a.stats()["t"]
        with sfm.Sim(sc, place=False) as b:
            b.place(xy, h, sc.goal, al)
            b.set_time(t)
            for s in (a, b):
                s.compute_field()
            np.testing.assert_array_equal(a.field(), b.field())
            for _ in range(4):
                a.step(1)
                b.step(1)
                np.testing.assert_array_equal(a.field(), b.field())
                np.testing.assert_array_equal(a.decisions()[0], b.decisions()[0])
                for x, y in zip(a.peds(), b.peds()):
                    np.testing.assert_array_equal(x, y)
        xy, h, al = a.peds()
        live = np.flatnonzero(al)
        for bad, status in ((lambda q: q.__setitem__(live[0], q[live[1]]), sfm.SFM_ECONFLICT),
                            (lambda q: q.__setitem__(live[0], (0, 0)), sfm.SFM_ECONFLICT),
                            (lambda q: q.__setitem__(live[0], (sc.W, 3)), sfm.SFM_EINVAL)):
            q = xy.copy()
            bad(q)
            with pytest.raises(sfm.SfmError) as e:
                a.place(*_arrays_as(src, q, h, sc.goal, al))
            assert e.value.status == status
            a.place(xy, h, sc.goal, al)  # a valid placement after the refused one
            a.place(*_arrays_as(src, xy, h, sc.goal, al))  # keeps the graphs again
        a.step(2)
        assert a.stats()["error_flags"] == 0


@pytest.mark.parametrize("variant", ["plain", "periods", "sized"])
def test_snapshot_restore_continues_bit_for_bit(variant):
    """Checkpoint and resume: a snapshot taken after 7 ticks, restored into a
    fresh context on the same lattice, continues exactly as the original run
    (positions, headings, exits, tick counter); snapshots of other lattices
    or parameters, and damaged buffers, are refused."""
    sc = SG.random_scene(180, 150, 2500, r=8, seed=161, obstacles=3, exits=("west",),
                         goal_mode="mixed", heading_mode="random")
    size = None
    if variant == "sized":
        sc, size = sized_subset(sc, np.random.default_rng(4).choice(np.array([1, 3], np.uint8),
                                                                     size=sc.n))
    with sfm.Sim(sc, place=size is None) as a, sfm.Sim(sc, place=False) as b:
        if size is not None:
            a.place_sized(sc.xy, sc.heading, sc.goal, np.ones(sc.n, np.uint8), size, size)
        if variant == "periods":
            a.set_walk_periods(*SG.walk_periods(sc.n, 5))
        a.step(7)
        snap = a.snapshot()
        a.step(12)
        b.restore(snap)
        assert b.stats()["t"] == 7
        b.step(12)
        for x, y in zip(a.peds(), b.peds()):
            np.testing.assert_array_equal(x, y)
        sa, sb = a.stats(), b.stats()
        assert (sa["t"], sa["exited"], sa["alive"]) == (sb["t"], sb["exited"], sb["alive"])
        for bad in (snap[:-1], b"XXXXXXXX" + snap[8:]):
            with pytest.raises(sfm.SfmError) as e:
                b.restore(bad)
            assert e.value.status == sfm.SFM_EINVAL
    other = SG.random_scene(180, 151, 10, r=8, seed=162)
    with sfm.Sim(other, place=False) as c:
        with pytest.raises(sfm.SfmError) as e:
            c.restore(snap)
        assert e.value.status == sfm.SFM_EINVAL
    with sfm.Sim(sc, place=False, beta=2.0) as d:
        with pytest.raises(sfm.SfmError) as e:
            d.restore(snap)
        assert e.value.status == sfm.SFM_EINVAL


def test_field_respects_heading_linearity_closed_form():
    """A single pedestrian in an open periodic lattice: the GPU field equals
    the closed form k d^a (1 + gamma cos) to FP32 rounding."""
    W = H = 96
    cell = np.zeros((H, W), np.uint8)
    for h in range(9):
        with sfm.Sim(W=W, H=H, cell=cell, periodic_x=1, periodic_y=1, r=30) as sim:
            sim.place(np.array([[50, 40]], np.int32), np.array([h], np.uint8))
            sim.compute_field()
            F = sim.field().astype(np.float64)
            X, Y = np.meshgrid(np.arange(W), np.arange(H))
            dx, dy = X - 50, Y - 40
            d = np.hypot(dx, dy)
            ux, uy = SG.DIRS[h] / (np.hypot(*SG.DIRS[h]) if h else 1.0)
            inside = (np.maximum(abs(dx), abs(dy)) <= 30) & (d > 0)
            ref = np.where(inside, np.where(d > 0, d, 1) ** -0.5 *
                           (1 + 0.5 * (ux * dx + uy * dy) / np.where(d > 0, d, 1)), 0.0)
            np.testing.assert_allclose(F, ref, rtol=3e-7, atol=1e-30)


def test_placement_errors_and_state_errors():
    sc = SG.random_scene(40, 30, 10, r=3, seed=120)
    with sfm.Sim(sc, place=False) as sim:
        with pytest.raises(sfm.SfmError) as e:
            sim.step(1)
        assert e.value.status == sfm.SFM_ESTATE
        xy = sc.xy.copy()
        xy[1] = xy[0]
        with pytest.raises(sfm.SfmError) as e:
            sim.place(xy)
        assert e.value.status == sfm.SFM_ECONFLICT
        xy = sc.xy.copy()
        xy[0] = (0, 0)                       # on the wall ring
        with pytest.raises(sfm.SfmError) as e:
            sim.place(xy)
        assert e.value.status == sfm.SFM_ECONFLICT
        xy = sc.xy.copy()
        xy[0] = (40, 3)                      # off-lattice
        with pytest.raises(sfm.SfmError) as e:
            sim.place(xy)
        assert e.value.status == sfm.SFM_EINVAL
        with pytest.raises(sfm.SfmError) as e:
            sim.place(sc.xy, np.full(sc.n, 9, np.uint8))
        assert e.value.status == sfm.SFM_EINVAL
        # a rejected placement leaves a clean lattice: a valid one then works
        sim.place(sc.xy, sc.heading, sc.goal)
        sim.step(3)
        assert sim.stats()["error_flags"] == 0
        # a dead pedestrian may sit anywhere; it is ignored
        alive = np.ones(sc.n, np.uint8)
        alive[0] = 0
        xy = sc.xy.copy()
        xy[0] = xy[1]
        sim.place(xy, alive=alive)
        sim.step(1)
        ch, won = sim.decisions()
        assert ch[0] == 0 and won[0] == 0


def test_empty_crowd_field_is_static_field():
    sc = SG.random_scene(70, 50, 0, r=6, seed=121, obstacles=3, exits=("east",))
    with sfm.Sim(sc) as sim:
        sim.compute_field()
        np.testing.assert_array_equal(sim.field(), sim.static_field())
        sim.step(2)
        assert sim.stats()["t"] == 2


@pytest.mark.parametrize("variant", ["closed_banded", "closed", "torus", "periods_banded"])
def test_sparse_crowd_ticks_follow_the_oracle(variant):
    """A crowd under one pedestrian per 64 su, like the 16384^2 floor's
    (binned from the pedestrian list, few pedestrians a bin): every tick
    follows the oracle's, with the row-trimmed footprint at r = 33, in 4 row
    bands (the ring band buffer) or one, on a closed room with exits and on
    a torus, with and without walk periods."""
    periodic = variant == "torus"
    sc = SG.random_scene(640, 512, 2000, r=33, seed=171, obstacles=0 if periodic else 5,
                         periodic_x=int(periodic), periodic_y=int(periodic), ring=not periodic,
                         exits=() if periodic else ("east", "north", "south"), exit_len=40,
                         goal_mode="mixed", heading_mode="random")
    assert sc.n * 64 < sc.W * sc.H
    banded = variant.endswith("banded")
    orc = OracleRun(sc)
    period = phase = None
    if variant.startswith("periods"):
        rng = np.random.default_rng(17)
        period = rng.integers(1, 4, size=sc.n).astype(np.uint8)
        phase = (rng.integers(0, 255, size=sc.n) % period).astype(np.uint8)
        orc.st.period, orc.st.phase = period, phase
    budget = sfm.band_budget(sc.W, sc.H, 128) if banded else 0
    with sfm.Sim(sc, hbm_budget_bytes=budget) as sim:
        assert (sim.stats()["bands"] == 4) == banded
        sim.set_footprint("32x32r")
        if period is not None:
            sim.set_walk_periods(period, phase)
        flips = 0
        for t in range(8):
            sim.step(1)
            Fo, So = orc.field()
            ch_o, E, T, adm = orc.decide(Ffull=Fo.ravel(), Sfull=So.ravel())
            if period is not None:
                ch_o = O.gate_periods(orc.st.t, period, phase, ch_o)
            ch_g, won_g = sim.decisions()
            # a decision that differs only inside the tie tolerance is counted
            # and the oracle takes the GPU's choice (as valid as its own)
            f = compare_choices(ch_g, ch_o, E, T, adm)
            flips += f
            won_o, _ = orc.advance(np.asarray(ch_g, np.uint8) if f else ch_o)
            np.testing.assert_array_equal(won_g, won_o)
            for x, y in zip(sim.peds(), (orc.st.xy, orc.st.heading, orc.st.alive)):
                np.testing.assert_array_equal(x, y)
        assert sim.stats()["exited"] == orc.st.exited
        assert sim.stats()["error_flags"] == 0
        assert flips <= 2, f"{flips} tie flips in 8 ticks"


def test_clustered_crowd_under_the_ticket_schedule_keeps_the_field_and_ticks():
    """A sparse crowd with one dense cluster, on a lattice large enough for
    the row-trimmed gather's schedule of dealt rounds and tickets (4608^2 su,
    r = 40, footprints of very uneven cost): the field and the ticks are
    bit-identical to the 16x16 gather's, unbanded and in 4 bands (a
    footprint the schedule missed or took twice would show)."""
    W = H = 4608
    base = SG.random_scene(W, H, 70000, r=40, seed=181, exits=("east", "west"), exit_len=64,
                           goal_mode="mixed", heading_mode="random")
    x0, y0, side = 2200, 2300, 150
    rng = np.random.default_rng(182)
    inside = ((base.xy[:, 0] >= x0) & (base.xy[:, 0] < x0 + side) &
              (base.xy[:, 1] >= y0) & (base.xy[:, 1] < y0 + side))
    ys, xs = np.nonzero(base.cell[y0:y0 + side, x0:x0 + side] == SG.FREE)
    pick = rng.random(ys.size) < 0.6
    cl = np.stack([xs[pick] + x0, ys[pick] + y0], axis=1).astype(np.int32)
    xy = np.concatenate([base.xy[~inside], cl]).astype(np.int32)
    n = xy.shape[0]
    sc = SG.Scene("cluster", W, H, 0, 0, base.cell, xy,
                  rng.integers(0, 9, n).astype(np.uint8),
                  np.where(rng.random(n) < 0.5, 0, rng.integers(1, 9, n)).astype(np.uint8),
                  base.params)
    assert cl.shape[0] > 10000
    budget = sfm.band_budget(W, H, H // 4)
    with sfm.Sim(sc) as a, sfm.Sim(sc) as b, sfm.Sim(sc, hbm_budget_bytes=budget) as c:
        a.set_footprint("16x16")
        b.set_footprint("32x32r")
        c.set_footprint("32x32r")
        assert c.stats()["bands"] == 4
        for _ in range(3):
            for s in (a, b, c):
                s.step(1)
            # the field of the tick just taken
            np.testing.assert_array_equal(a.field(), b.field())
            for s in (b, c):
                np.testing.assert_array_equal(a.decisions()[0], s.decisions()[0])
                for x, y in zip(a.peds(), s.peds()):
                    np.testing.assert_array_equal(x, y)
        for s in (a, b, c):
            assert s.stats()["error_flags"] == 0
