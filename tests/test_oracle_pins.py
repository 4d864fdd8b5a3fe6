"""Pins of the FP64 oracle against things other than itself (CPU only).

Each test fixes a part of the oracle by a closed form, a published test vector,
an independent brute-force enumeration, a symmetry, an invariant or a special
case that reduces to a textbook routine, so that a dropped term, a wrong sign,
a swapped index or a transposed operand in ``oracle/sfm_oracle.c`` fails one of
them.
"""
import math
import os

import numpy as np
import pytest

import brute
import oracle as O
import scenegen as SG

GOLD = os.path.join(os.path.dirname(__file__), "golden")

# heading/goal class maps under the mirror x -> W-1-x, y -> H-1-y and the
# transpose (x, y) -> (y, x)
MIRROR_X = np.array([0, 5, 4, 3, 2, 1, 8, 7, 6], np.uint8)
MIRROR_Y = np.array([0, 1, 8, 7, 6, 5, 4, 3, 2], np.uint8)
TRANSPOSE = np.array([0, 3, 2, 1, 8, 7, 6, 5, 4], np.uint8)


def _read_golden(name):
    rows = []
    with open(os.path.join(GOLD, name)) as f:
        for line in f:
            line = line.split("#", 1)[0].strip()
            if line:
                rows.append(line.split())
    return rows


def _single(W, H, x, y, hcls=0, r=3, px=0, py=0, **kw):
    sc = SG.Scene("one", W, H, px, py, np.zeros((H, W), np.uint8),
                  np.array([[x, y]], np.int32), np.array([hcls], np.uint8),
                  np.zeros(1, np.uint8), SG._params(r=r, **kw))
    m = O.model(sc)
    occ, bad = O.occupancy(m, sc.cell, sc.xy)
    assert bad == 0
    F, S = O.field(m, sc.cell, occ, sc.heading)
    return sc, F, S


# ---------------------------------------------------------------- closed forms
def test_paper_example_field_closed_form():
    """Sec. 3.1 s-1: recurrent field with k = 1, alpha = -0.5, 7x7 geometry."""
    g = {row[0]: row[1:] for row in _read_golden("paper_example_field.txt")}
    k, alpha, r = float(g["k"][0]), float(g["alpha"][0]), int(g["r"][0])
    assert (2 * r + 1) == int(g["geometry"][0]) == int(g["geometry"][1])
    sc, F, _ = _single(15, 15, 7, 7, r=r, kP=k, aP=alpha, gamma=0.5)
    f = lambda dx, dy: F[7 + dy, 7 + dx]
    assert f(0, 0) == 0.0                                   # no self field
    assert f(1, 0) == pytest.approx(1.0, abs=1e-15)
    assert f(1, 1) == pytest.approx(2 ** -0.25, abs=1e-15)  # 0.840896415
    assert f(2, 1) == pytest.approx(5 ** -0.25, abs=1e-15)  # 0.668740305
    assert f(2, 2) == pytest.approx(8 ** -0.25, abs=1e-15)  # 0.594603558
    assert f(3, 0) == pytest.approx(3 ** -0.5, abs=1e-15)   # 0.577350269
    assert f(3, 3) == pytest.approx(18 ** -0.25, abs=1e-15)  # 0.485491772
    assert f(-2, 3) == pytest.approx(13 ** -0.25, abs=1e-15)
    # Chebyshev window: zero just outside, including the corners of the 9x9 ring
    for dx, dy in [(4, 0), (0, -4), (4, 4), (-4, 3), (3, -4)]:
        assert f(dx, dy) == 0.0
    # the whole 7x7 sum, with the 48 non-centre offsets written out
    total = sum((dx * dx + dy * dy) ** -0.25 for dx in range(-3, 4) for dy in range(-3, 4)
                if (dx, dy) != (0, 0))
    assert F.sum() == pytest.approx(total, rel=1e-14)
    assert F.sum() == pytest.approx(30.883571323, abs=1e-8)


def test_heading_term_closed_form():
    """Directional part: 1 + gamma cos(angle between heading and offset)."""
    _, F, _ = _single(15, 15, 7, 7, hcls=1, r=3, gamma=0.5)   # heading east
    f = lambda dx, dy: F[7 + dy, 7 + dx]
    assert f(1, 0) == pytest.approx(1.5, abs=1e-15)
    assert f(-1, 0) == pytest.approx(0.5, abs=1e-15)
    assert f(0, 1) == pytest.approx(1.0, abs=1e-15)         # orthogonal: no change
    assert f(0, -2) == pytest.approx(2 ** -0.5, abs=1e-15)
    assert f(1, 1) == pytest.approx(2 ** -0.25 * (1 + 0.5 / 2 ** 0.5), abs=1e-15)
    assert f(-1, -1) == pytest.approx(2 ** -0.25 * (1 - 0.5 / 2 ** 0.5), abs=1e-15)
    assert f(1, 1) == pytest.approx(1.138198194, abs=1e-9)
    assert f(-1, -1) == pytest.approx(0.543594637, abs=1e-9)
    # heading north-east (class 2): offset (2, 1) gets cos = 3 / (sqrt2 sqrt5)
    _, F2, _ = _single(15, 15, 7, 7, hcls=2, r=3, gamma=0.5)
    assert F2[8, 9] == pytest.approx(5 ** -0.25 * (1 + 0.5 * 3 / math.sqrt(10)), abs=1e-15)
    # heading north (class 3) is the transpose of heading east
    _, F3, _ = _single(15, 15, 7, 7, hcls=3, r=3, gamma=0.5)
    np.testing.assert_allclose(F3, F.T, rtol=0, atol=1e-15)


def test_static_kernels_closed_form():
    """Obstacles repel (kO > 0), openings attract (kE < 0), same window rule."""
    W = H = 11
    cell = np.zeros((H, W), np.uint8)
    cell[5, 5] = SG.WALL
    m = O.model(W=W, H=H, r=3, kO=2.0, aO=-1.0)
    occ = np.full(W * H, -1, np.int32)
    F, S = O.field(m, cell, occ, np.zeros(1, np.uint8), parts=1)
    assert F[5, 7] == pytest.approx(1.0, abs=1e-15)          # 2 * 2^-1
    assert F[8, 8] == pytest.approx(2 / math.sqrt(18), abs=1e-15)
    assert F[5, 9] == 0.0
    cell[5, 5] = SG.EXIT
    m = O.model(W=W, H=H, r=3, kE=-1.0, aE=-0.5)
    F, S = O.field(m, cell, occ, np.zeros(1, np.uint8), parts=1)
    assert F[5, 6] == pytest.approx(-1.0, abs=1e-15)
    assert F[7, 6] == pytest.approx(-(5 ** -0.25), abs=1e-15)
    np.testing.assert_allclose(S, np.abs(F), atol=1e-15)
    # pedestrians are not static sources
    F2, _ = O.field(m, cell, occ, np.zeros(1, np.uint8), parts=2)
    assert not F2.any()


# ------------------------------------------------------------ brute force
@pytest.mark.parametrize("px,py,ring,seed", [(0, 0, True, 11), (1, 0, True, 12),
                                             (1, 1, False, 13), (0, 1, True, 14)])
def test_field_matches_all_pairs_brute_force(px, py, ring, seed):
    sc = SG.random_scene(23, 17, 40, r=4, seed=seed, periodic_x=px, periodic_y=py,
                         ring=ring, exits=("east",) if not px else ("south",) if not py else (),
                         obstacles=3, goal_mode="mixed", heading_mode="random")
    sc.params.update(gamma=0.7, kO=1.3, aO=-0.8, kE=-0.9, aE=-0.3)
    m = O.model(sc)
    occ, bad = O.occupancy(m, sc.cell, sc.xy)
    assert bad == 0
    F, S = O.field(m, sc.cell, occ, sc.heading)
    Fb, Sb = brute.field(sc)
    np.testing.assert_allclose(F, Fb, rtol=1e-12, atol=1e-12)
    np.testing.assert_allclose(S, Sb, rtol=1e-12, atol=1e-12)
    # requested-su evaluation returns the same numbers as the full lattice
    req = np.random.default_rng(seed).choice(sc.W * sc.H, 50, replace=False)
    Fr, Sr = O.field(m, sc.cell, occ, sc.heading, req=req)
    np.testing.assert_array_equal(Fr, F.ravel()[req])
    np.testing.assert_array_equal(Sr, S.ravel()[req])


def test_field_superposition_is_linear():
    sc = SG.random_scene(30, 30, 80, r=5, seed=21, heading_mode="random")
    m = O.model(sc)
    occ, _ = O.occupancy(m, sc.cell, sc.xy)
    F, _ = O.field(m, sc.cell, occ, sc.heading, parts=2)
    alive_a = (np.arange(sc.n) % 3 == 0).astype(np.uint8)
    occ_a, _ = O.occupancy(m, sc.cell, sc.xy, alive_a)
    occ_b, _ = O.occupancy(m, sc.cell, sc.xy, 1 - alive_a)
    Fa, _ = O.field(m, sc.cell, occ_a, sc.heading, parts=2)
    Fb, _ = O.field(m, sc.cell, occ_b, sc.heading, parts=2)
    np.testing.assert_allclose(F, Fa + Fb, rtol=1e-13, atol=1e-13)
    Fs, _ = O.field(m, sc.cell, occ, sc.heading, parts=1)
    Ft, _ = O.field(m, sc.cell, occ, sc.heading, parts=3)
    np.testing.assert_allclose(Ft, F + Fs, rtol=1e-13, atol=1e-13)


# -------------------------------------------------------------- symmetries
def _field_of(sc):
    m = O.model(sc)
    occ, bad = O.occupancy(m, sc.cell, sc.xy)
    assert bad == 0
    return O.field(m, sc.cell, occ, sc.heading)[0]


def test_mirror_and_rotation_symmetry():
    sc = SG.random_scene(26, 26, 60, r=5, seed=31, obstacles=4, exits=("east", "north"),
                         heading_mode="random")
    F = _field_of(sc)
    mx = sc.copy()
    mx.cell = sc.cell[:, ::-1].copy()
    mx.xy[:, 0] = sc.W - 1 - sc.xy[:, 0]
    mx.heading = MIRROR_X[sc.heading]
    np.testing.assert_allclose(_field_of(mx), F[:, ::-1], rtol=0, atol=1e-13)
    my = sc.copy()
    my.cell = sc.cell[::-1, :].copy()
    my.xy[:, 1] = sc.H - 1 - sc.xy[:, 1]
    my.heading = MIRROR_Y[sc.heading]
    np.testing.assert_allclose(_field_of(my), F[::-1, :], rtol=0, atol=1e-13)
    tr = sc.copy()
    tr.cell = sc.cell.T.copy()
    tr.xy = sc.xy[:, ::-1].copy()
    tr.heading = TRANSPOSE[sc.heading]
    np.testing.assert_allclose(_field_of(tr), F.T, rtol=0, atol=1e-13)


def test_translation_invariance_on_torus():
    sc = SG.random_scene(24, 20, 50, r=6, seed=41, periodic_x=1, periodic_y=1, ring=False,
                         exits=(), heading_mode="random")
    F = _field_of(sc)
    sh = sc.copy()
    sh.xy[:, 0] = (sc.xy[:, 0] + 7) % sc.W
    sh.xy[:, 1] = (sc.xy[:, 1] + 13) % sc.H
    np.testing.assert_allclose(_field_of(sh), np.roll(np.roll(F, 7, axis=1), 13, axis=0),
                               rtol=0, atol=1e-13)


# --------------------------------------------------------------- guidance
def test_guidance_closed_form_open_plane():
    """No obstacles: chamfer distance 5 max(|dx|,|dy|) + 2 min(|dx|,|dy|)."""
    W, H = 31, 23
    cell = np.zeros((H, W), np.uint8)
    cell[9, 20] = SG.EXIT
    D = O.guidance(O.model(W=W, H=H), cell)
    X, Y = np.meshgrid(np.arange(W), np.arange(H))
    ax, ay = np.abs(X - 20), np.abs(Y - 9)
    np.testing.assert_array_equal(D, 5 * np.maximum(ax, ay) + 2 * np.minimum(ax, ay))


@pytest.mark.parametrize("px,py,seed", [(0, 0, 51), (1, 0, 52), (1, 1, 53)])
def test_guidance_matches_bellman_ford(px, py, seed):
    sc = SG.random_scene(29, 21, 0, r=1, seed=seed, periodic_x=px, periodic_y=py,
                         ring=not (px and py), exits=("west",) if not px else ("north",),
                         obstacles=6)
    if px and py:
        sc.cell[3, 4] = SG.EXIT
    D = O.guidance(O.model(sc), sc.cell)
    np.testing.assert_array_equal(D, brute.guidance(sc.cell, px, py))
    assert (D[sc.cell == SG.WALL] == O.DINF).all()


# ------------------------------------------------------------- decisions
def test_decision_r0_is_steepest_descent_of_guidance():
    """r = 0 removes every field term: the choice is the steepest admissible
    descent of the guidance distance, ties to the smallest class."""
    sc = SG.random_scene(25, 25, 120, r=0, seed=61, obstacles=5, exits=("east", "south"))
    m = O.model(sc)
    D = O.guidance(m, sc.cell)
    occ, _ = O.occupancy(m, sc.cell, sc.xy)
    alive = np.ones(sc.n, np.uint8)
    choice, E, T, adm = O.decide(m, sc.cell, occ, sc.xy, sc.heading, sc.goal, alive, D)
    occ2 = occ.reshape(sc.H, sc.W)
    for i, (x, y) in enumerate(sc.xy):
        best, bestv = 0, 0.0
        for k in range(1, 9):
            nx, ny = x + SG.DIRS[k][0], y + SG.DIRS[k][1]
            if not (0 <= nx < sc.W and 0 <= ny < sc.H):
                continue
            if sc.cell[ny, nx] == SG.WALL or occ2[ny, nx] >= 0:
                continue
            v = (int(D[ny, nx]) - int(D[y, x])) / 5.0
            if v < bestv:
                best, bestv = k, v
        assert choice[i] == best, (i, x, y)


def test_fixed_direction_tie_goes_to_smallest_class():
    W, H = 9, 9
    cell = np.zeros((H, W), np.uint8)
    cell[4, 5] = SG.WALL                                  # blocks the east move
    sc = SG.Scene("tie", W, H, 0, 0, cell, np.array([[4, 4]], np.int32),
                  np.zeros(1, np.uint8), np.array([1], np.uint8), SG._params(r=0))
    m = O.model(sc)
    occ, _ = O.occupancy(m, cell, sc.xy)
    ch, E, _, adm = O.decide(m, cell, occ, sc.xy, sc.heading, sc.goal, np.ones(1, np.uint8),
                             np.zeros((H, W), np.int32))
    assert adm[0, 1] == 0
    assert E[0, 2] == E[0, 8] == -1.0                      # (1,+-1) . (1,0) = 1
    assert ch[0] == 2


def test_near_tie_count_finds_the_exact_tie_of_the_blocked_east_move():
    """The blocked east move leaves NE and SE with equal energies (-1 each,
    an exact tie): the near-tie rule counts it; best is the smaller class."""
    W, H = 9, 9
    cell = np.zeros((H, W), np.uint8)
    cell[4, 5] = SG.WALL
    sc = SG.Scene("tie", W, H, 0, 0, cell, np.array([[4, 4]], np.int32),
                  np.zeros(1, np.uint8), np.array([1], np.uint8), SG._params(r=0))
    m = O.model(sc)
    occ, _ = O.occupancy(m, cell, sc.xy)
    ch, E, T, adm, Mag = O.decide(m, cell, occ, sc.xy, sc.heading, sc.goal,
                                  np.ones(1, np.uint8), np.zeros((H, W), np.int32),
                                  magnitudes=True)
    b, s2 = O.best_two(E, adm)
    assert (b[0], s2[0]) == (2, 8) and ch[0] == 2
    # r = 0: no field, no own term; the magnitude is the guidance term alone
    assert Mag[0, 2] == Mag[0, 8] == 1.0
    assert O.near_ties(E, Mag, adm).tolist() == [True]


def test_near_tie_count_finds_mirror_ties_and_no_others():
    """A pedestrian on the mirror axis of a symmetric closed room, walking
    north with the north su walled: NE and NW are mirror images, so their
    FP64 energies agree up to summation order (a near tie); the lone walker
    of an empty corridor has a clear best move (no near tie)."""
    W, H = 11, 11
    cell = np.zeros((H, W), np.uint8)
    cell[0, :] = cell[-1, :] = cell[:, 0] = cell[:, -1] = SG.WALL
    cell[6, 5] = SG.WALL                                   # north of (5, 5)
    sc = SG.Scene("mirror", W, H, 0, 0, cell, np.array([[5, 5]], np.int32),
                  np.zeros(1, np.uint8), np.array([3], np.uint8), SG._params(r=3))
    m = O.model(sc)
    occ, _ = O.occupancy(m, cell, sc.xy)
    ch, E, T, adm, Mag = O.decide(m, cell, occ, sc.xy, sc.heading, sc.goal,
                                  np.ones(1, np.uint8), O.guidance(m, cell), magnitudes=True)
    b, s2 = O.best_two(E, adm)
    assert {int(b[0]), int(s2[0])} == {2, 4}               # NE and NW
    assert abs(E[0, 2] - E[0, 4]) <= 1e-12 * Mag[0, 2]
    assert O.near_ties(E, Mag, adm).tolist() == [True]
    # the corridor walker of the next test: east beats NE / SE by the wall
    # field's difference, far above 1e-5 of the energies
    Wc, Hc = 40, 7
    cc = np.zeros((Hc, Wc), np.uint8)
    cc[0, :] = cc[Hc - 1, :] = SG.WALL
    sw = SG.Scene("walker", Wc, Hc, 1, 0, cc, np.array([[3, 3]], np.int32),
                  np.array([1], np.uint8), np.array([1], np.uint8), SG._params(r=5))
    mw = O.model(sw)
    occ, _ = O.occupancy(mw, cc, sw.xy)
    ch, E, T, adm, Mag = O.decide(mw, cc, occ, sw.xy, sw.heading, sw.goal,
                                  np.ones(1, np.uint8), O.guidance(mw, cc), magnitudes=True)
    assert ch[0] == 1
    assert O.near_ties(E, Mag, adm).tolist() == [False]


def test_lone_walker_moves_along_its_direction():
    """Own-field removal: a lone pedestrian heading east in an empty periodic
    corridor steps east every tick (its own field would otherwise block it)."""
    W, H = 40, 7
    cell = np.zeros((H, W), np.uint8)
    cell[0, :] = SG.WALL
    cell[H - 1, :] = SG.WALL
    sc = SG.Scene("walker", W, H, 1, 0, cell, np.array([[3, 3]], np.int32),
                  np.array([1], np.uint8), np.array([1], np.uint8), SG._params(r=5))
    m = O.model(sc)
    st = O.State(sc)
    D = O.guidance(m, cell)
    for t in range(60):
        ch, won = O.step(m, cell, D, st)
        assert ch[0] == 1 and won[0] == 1
        assert tuple(st.xy[0]) == ((3 + t + 1) % W, 3)


def test_walk_period_walker_moves_only_on_its_ticks():
    """Walk period (Sec. 2, reading: moves only on ticks t with t mod P =
    phase): the lone east-walker above with period 3 and phase 1 advances one
    su on ticks 1, 4, 7, ... and stays in between, keeping its heading."""
    W, H = 40, 7
    cell = np.zeros((H, W), np.uint8)
    cell[0, :] = SG.WALL
    cell[H - 1, :] = SG.WALL
    sc = SG.Scene("walker", W, H, 1, 0, cell, np.array([[3, 3]], np.int32),
                  np.array([1], np.uint8), np.array([1], np.uint8), SG._params(r=5))
    m = O.model(sc)
    st = O.State(sc)
    st.period = np.array([3], np.uint8)
    st.phase = np.array([1], np.uint8)
    D = O.guidance(m, cell)
    x = 3
    for t in range(30):
        ch, won = O.step(m, cell, D, st)
        if t % 3 == 1:
            x = (x + 1) % W
            assert ch[0] == 1 and won[0] == 1
        else:
            assert ch[0] == 0 and won[0] == 0
        assert tuple(st.xy[0]) == (x, 3) and st.heading[0] == 1
    assert x == 3 + 10


def test_walk_periods_of_one_are_the_plain_model_and_gating_is_exact():
    """All periods 1: the same run as without periods.  Random periods: a
    pedestrian moves (or wins a vote) only on its own ticks, never registers
    otherwise, and its moves over T ticks are at most its active ticks."""
    sc = SG.random_scene(48, 40, 500, r=5, seed=81, obstacles=3, exits=("east",),
                         goal_mode="mixed", heading_mode="random")
    m = O.model(sc)
    D = O.guidance(m, sc.cell)
    a, b = O.State(sc), O.State(sc)
    b.period = np.ones(sc.n, np.uint8)
    b.phase = np.zeros(sc.n, np.uint8)
    for _ in range(8):
        ca, wa = O.step(m, sc.cell, D, a)
        cb, wb = O.step(m, sc.cell, D, b)
        np.testing.assert_array_equal(ca, cb)
        np.testing.assert_array_equal(a.xy, b.xy)
    rng = np.random.default_rng(5)
    st = O.State(sc)
    st.period = rng.integers(1, 6, size=sc.n).astype(np.uint8)
    st.phase = (rng.integers(0, 255, size=sc.n) % st.period).astype(np.uint8)
    moves = np.zeros(sc.n, int)
    T = 15
    for t in range(T):
        xy0 = st.xy.copy()
        ch, won = O.step(m, sc.cell, D, st)
        active = (t % st.period.astype(int)) == st.phase
        moved = np.any(st.xy != xy0, axis=1)
        assert not np.any(moved & ~active)
        assert not np.any((ch > 0) & ~active) and not np.any((won > 0) & ~active)
        moves += moved
    n_active = np.array([sum(1 for t in range(T) if t % p == f) for p, f in zip(st.period, st.phase)])
    assert np.all(moves <= n_active) and moves.sum() > 0
    gated = O.gate_periods(4, st.period, st.phase, np.full(sc.n, 3, np.uint8))
    np.testing.assert_array_equal(gated > 0, (4 % st.period.astype(int)) == st.phase)


def _rect(W, H, px, py, x, y, w, h):
    """su of the w x h rectangle centred on (x, y), or None if it leaves a
    closed lattice (plain Python sets: an independent restatement)."""
    out = set()
    x, y, w, h = int(x), int(y), int(w), int(h)
    for j in range(-(h // 2), h // 2 + 1):
        for i in range(-(w // 2), w // 2 + 1):
            u, v = x + i, y + j
            if px:
                u %= W
            elif not 0 <= u < W:
                return None
            if py:
                v %= H
            elif not 0 <= v < H:
                return None
            out.add((u, v))
    return out


def test_sized_pedestrians_of_one_su_are_the_plain_model():
    sc = SG.random_scene(48, 40, 500, r=5, seed=82, obstacles=3, exits=("east",),
                         goal_mode="mixed", heading_mode="random")
    m = O.model(sc)
    D = O.guidance(m, sc.cell)
    a, b = O.State(sc), O.State(sc)
    b.w = np.ones(sc.n, np.uint8)
    b.h = np.ones(sc.n, np.uint8)
    for _ in range(8):
        ca, wa = O.step(m, sc.cell, D, a)
        cb, wb = O.step(m, sc.cell, D, b)
        np.testing.assert_array_equal(ca, cb)
        np.testing.assert_array_equal(wa, wb)
        np.testing.assert_array_equal(a.xy, b.xy)


def test_wide_pedestrian_walks_open_space_and_is_stopped_by_a_narrow_gap():
    """Multi-su pedestrians (Sec. 2): a 3x3 east-walker crosses an open
    corridor like a 1x1 one, but a 2-su gap in a wall lets only the 1x1 one
    through."""
    W, H = 40, 9
    cell = np.zeros((H, W), np.uint8)
    cell[0, :] = SG.WALL
    cell[H - 1, :] = SG.WALL
    cell[1:H - 1, 20] = SG.WALL
    cell[4:6, 20] = SG.FREE                       # gap: rows 4 and 5
    for size, passes in ((1, True), (3, False)):
        # strong guidance, so the walls' repulsion does not stop the walkers
        sc = SG.Scene("gap", W, H, 0, 0, cell, np.array([[5, 4]], np.int32),
                      np.array([1], np.uint8), np.array([1], np.uint8), SG._params(r=4, beta=20.0))
        m = O.model(sc)
        st = O.State(sc)
        st.w = np.array([size], np.uint8)
        st.h = np.array([size], np.uint8)
        D = O.guidance(m, cell)
        for t in range(30):
            O.step(m, cell, D, st)
            rect = _rect(W, H, 0, 0, st.xy[0, 0], st.xy[0, 1], size, size)
            assert rect is not None and all(cell[v, u] != SG.WALL for u, v in rect)
        assert (st.xy[0, 0] > 20) == passes, (size, st.xy[0])
        if not passes:
            assert st.xy[0, 0] == 18                # its east edge stops at x = 19


def test_sized_vote_against_a_pairwise_restatement():
    """One tick of a crowd of 1x1 and 3x3 pedestrians: winners claim disjoint
    strips of free su, and every losing mover shares a claimed su with a
    mover of smaller (priority, id) -- checked pair by pair with Python sets."""
    sc = SG.random_scene(40, 36, 120, r=4, seed=83, ring=False, periodic_x=1, exits=(),
                         goal_mode="fixed", heading_mode="random")
    rng = np.random.default_rng(9)
    size = np.where(rng.random(sc.n) < 0.5, 3, 1).astype(np.uint8)
    # drop pedestrians whose rectangles overlap, keep a valid placement
    m = O.model(sc)
    keep, taken = [], set()
    for p in range(sc.n):
        rc = _rect(sc.W, sc.H, 1, 0, sc.xy[p, 0], sc.xy[p, 1], size[p], size[p])
        if rc is None or rc & taken or any(sc.cell[v, u] == SG.WALL for u, v in rc):
            continue
        keep.append(p)
        taken |= rc
    xy, goal, head, size = sc.xy[keep], sc.goal[keep], sc.heading[keep], size[keep]
    n = len(keep)
    alive = np.ones(n, np.uint8)
    cov, bad = O.cover(m, sc.cell, xy, alive, size, size)
    assert bad == 0
    occ, _ = O.occupancy(m, sc.cell, xy, alive)
    D = O.guidance(m, sc.cell)
    ch, E, T, adm = O.decide(m, sc.cell, occ, xy, head, goal, alive, D, cov=cov, w=size, h=size)
    t = 5
    won, _ = O.vote(m, t, xy, alive, ch, size, size)
    strip = {}
    for p in range(n):
        if ch[p] == 0:
            continue
        old = _rect(sc.W, sc.H, 1, 0, xy[p, 0], xy[p, 1], size[p], size[p])
        new = _rect(sc.W, sc.H, 1, 0, xy[p, 0] + SG.DIRS[ch[p]][0], xy[p, 1] + SG.DIRS[ch[p]][1],
                    size[p], size[p])
        strip[p] = new - old
        assert strip[p] and not any(cov[v * sc.W + u] >= 0 for u, v in strip[p])
    key = {p: (O.prio(m.seed, t, p), p) for p in strip}
    for p in strip:
        rivals = [q for q in strip if q != p and strip[q] & strip[p]]
        assert bool(won[p]) == all(key[p] < key[q] for q in rivals), p
    winners = [p for p in strip if won[p]]
    for i, p in enumerate(winners):
        for q in winners[i + 1:]:
            assert not strip[p] & strip[q]
    assert sum(won) > 0 and sum(won) < len(strip)


def test_sized_run_keeps_rectangles_disjoint_and_off_walls():
    sc = SG.random_scene(64, 56, 400, r=5, seed=84, obstacles=3, exits=("east", "west"),
                         exit_len=12, goal_mode="mixed", heading_mode="random")
    rng = np.random.default_rng(10)
    m = O.model(sc)
    size = rng.choice(np.array([1, 3, 5], np.uint8), size=sc.n, p=[0.6, 0.3, 0.1])
    keep, taken = [], set()
    for p in range(sc.n):
        rc = _rect(sc.W, sc.H, 0, 0, sc.xy[p, 0], sc.xy[p, 1], size[p], size[p])
        if rc is None or rc & taken or any(sc.cell[v, u] == SG.WALL for u, v in rc):
            continue
        keep.append(p)
        taken |= rc
    sub = SG.Scene("sized", sc.W, sc.H, 0, 0, sc.cell, sc.xy[keep], sc.heading[keep],
                   sc.goal[keep], sc.params)
    st = O.State(sub)
    st.w = size[keep].copy()
    st.h = size[keep].copy()
    D = O.guidance(m, sc.cell)
    moved = 0
    for _ in range(60):
        xy0 = st.xy.copy()
        O.step(m, sc.cell, D, st)
        cov, bad = O.cover(m, sc.cell, st.xy, st.alive, st.w, st.h)
        assert bad == 0
        assert st.alive.sum() + st.exited == sub.n
        moved += int(np.any(st.xy != xy0, axis=1).sum())
    assert moved > 0 and st.exited > 0
    # wide pedestrians leave too: through an exit they step onto
    gone = (st.alive == 0)
    assert np.any(gone & (st.w > 1)), "no multi-su pedestrian left"


def test_decision_energy_matches_brute_force_field():
    sc = SG.random_scene(21, 19, 45, r=4, seed=71, obstacles=2, goal_mode="mixed",
                         heading_mode="random")
    m = O.model(sc)
    D = O.guidance(m, sc.cell)
    occ, _ = O.occupancy(m, sc.cell, sc.xy)
    alive = np.ones(sc.n, np.uint8)
    choice, E, T, adm = O.decide(m, sc.cell, occ, sc.xy, sc.heading, sc.goal, alive, D)
    Fb, _ = brute.field(sc)
    p = sc.params
    for i, (x, y) in enumerate(sc.xy):
        for k in range(9):
            if not adm[i, k]:
                continue
            nx, ny = x + SG.DIRS[k][0], y + SG.DIRS[k][1]
            own = 0.0
            if k:
                hx, hy = brute.unit(int(sc.heading[i]))
                d = math.hypot(*SG.DIRS[k])
                own = p["kP"] * d ** p["aP"] * (1 + p["gamma"] * (hx * SG.DIRS[k][0] +
                                                                  hy * SG.DIRS[k][1]) / d)
            if sc.goal[i] == 0:
                g = p["beta"] * (int(D[ny, nx]) - int(D[y, x])) / 5.0
            else:
                ux, uy = brute.unit(int(sc.goal[i]))
                g = -p["beta"] * (SG.DIRS[k][0] * ux + SG.DIRS[k][1] * uy)
            assert E[i, k] == pytest.approx(Fb[ny, nx] - own + g, abs=1e-12)
        e = np.where(adm[i] == 1, E[i], np.inf)
        assert choice[i] == int(np.argmin(e))


# ----------------------------------------------------------- vote, commit
def test_splitmix64_published_vectors():
    for row in _read_golden("splitmix64_seed0.txt"):
        assert O.splitmix64_nth(0, int(row[0])) == int(row[1], 16)


def test_vote_eight_contenders_fair_and_unique():
    """Eight pedestrians around one empty su all target it (the enrollment
    container's bound of 8, Sec. 3.1 s-2): exactly one wins, the one with the
    smallest priority, and over many ticks each wins about 1/8 of the time."""
    W = H = 7
    xy = np.array([(3 - dx, 3 - dy) for dx, dy in SG.DIRS[1:]], np.int32)
    choice = np.arange(1, 9, dtype=np.uint8)               # everyone steps onto (3, 3)
    alive = np.ones(8, np.uint8)
    m = O.model(W=W, H=H, seed=1234)
    wins = np.zeros(8, int)
    for t in range(4000):
        won, maxc = O.vote(m, t, xy, alive, choice)
        assert maxc == 8 and won.sum() == 1
        w = int(np.argmax(won))
        pr = [O.prio(1234, t, i) for i in range(8)]
        assert w == int(np.argmin(pr))
        wins[w] += 1
    assert wins.min() > 4000 / 8 * 0.8 and wins.max() < 4000 / 8 * 1.2


def _invariants(sc, m, st, prev_xy, prev_alive, n0):
    occ, bad = O.occupancy(m, sc.cell, st.xy, st.alive)
    assert bad == 0                                         # exclusion, none on WALL/EXIT
    assert int(st.alive.sum()) + st.exited == n0            # conservation
    step = np.abs(st.xy - prev_xy)
    if sc.periodic_x:
        step[:, 0] = np.minimum(step[:, 0], sc.W - step[:, 0])
    if sc.periodic_y:
        step[:, 1] = np.minimum(step[:, 1], sc.H - step[:, 1])
    assert step.max(initial=0) <= 1                         # v_max = 1 su per tick


@pytest.mark.parametrize("maker", ["room", "corridor"])
def test_full_run_invariants(maker):
    if maker == "room":
        sc = SG.room(W=60, H=50, n=600, r=6, exit_len=6, seed=81)
        steps = 40
    else:
        sc = SG.corridor(W=120, H=30, n=900, r=5, seed=82)
        steps = 30
    m = O.model(sc)
    D = O.guidance(m, sc.cell)
    st = O.State(sc)
    moved = 0
    for _ in range(steps):
        prev_xy, prev_alive = st.xy.copy(), st.alive.copy()
        occ_before, _ = O.occupancy(m, sc.cell, st.xy, st.alive)
        ch, won = O.step(m, sc.cell, D, st)
        # winners are registrants, every target had been empty at step start
        assert not (won.astype(bool) & (ch == 0)).any()
        tgt = prev_xy + SG.DIRS[ch]
        if sc.periodic_x:
            tgt[:, 0] %= sc.W
        movers = won.astype(bool)
        assert (occ_before.reshape(sc.H, sc.W)[tgt[movers, 1], tgt[movers, 0]] == -1).all()
        # no swaps: a winner's target is never another winner's origin
        orig = set(map(tuple, prev_xy[movers]))
        assert not any(tuple(t) in orig for t in tgt[movers])
        moved += int(movers.sum())
        _invariants(sc, m, st, prev_xy, prev_alive, sc.n)
        assert (st.heading[movers] == ch[movers]).all()
    assert moved > 0
    if maker == "corridor":
        assert st.alive.sum() == sc.n                       # periodic: nobody leaves
    else:
        assert st.exited > 0                                # someone reached the exit


def test_numbered_vote_follows_the_numbers_not_the_array_order():
    """The election with caller-given numbers (a band's ghosts keep their
    whole-lattice numbers): shuffling the pedestrian arrays and numbering
    each pedestrian by its old index gives the same winners as the plain
    vote on the original order; numbering by the identity is the plain vote."""
    sc = SG.random_scene(60, 50, 900, r=3, seed=77, exits=("east",), heading_mode="random")
    m = O.model(sc)
    st = O.State(sc)
    D = O.guidance(m, sc.cell)
    occ, _ = O.occupancy(m, sc.cell, st.xy, st.alive)
    ch, _, _, _ = O.decide(m, sc.cell, occ, st.xy, st.heading, st.goal, st.alive, D)
    assert (ch > 0).sum() > 100
    won, maxc = O.vote(m, 5, st.xy, st.alive, ch)
    assert maxc >= 2                                   # contested su exist
    won_id, _ = O.vote(m, 5, st.xy, st.alive, ch, ids=np.arange(sc.n))
    np.testing.assert_array_equal(won_id, won)
    perm = np.random.default_rng(3).permutation(sc.n)
    won_p, _ = O.vote(m, 5, st.xy[perm], st.alive[perm], ch[perm], ids=perm)
    np.testing.assert_array_equal(won_p, won[perm])
    # other numbers change the priorities, so some contest changes hands
    won_s, _ = O.vote(m, 5, st.xy, st.alive, ch, ids=np.arange(sc.n) + 1000)
    assert not np.array_equal(won_s, won)
