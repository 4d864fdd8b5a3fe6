"""Comparison helpers shared by the GPU parity tests.

Tolerances (derived from the arithmetic; the FP32 path sums the same terms as
the FP64 oracle in another order, each term rounded once):
  * field: |F_gpu - F_oracle| <= 1e-5 * S(c) per su, where S(c) is the sum of
    the magnitudes of every term superposed at c (oracle, FP64);
  * decision: the energies the two sides compare differ by at most
    1e-5 * T, T the magnitude scale of a candidate's energy (field terms,
    own-field term, guidance term), so two candidates whose oracle energies
    lie within 1e-5 * (T_a + T_b) of each other form a tie that either side
    may break; everything else must agree exactly.
"""
import numpy as np

import oracle as O

FIELD_RTOL = 1e-5
TIE_RTOL = 1e-5


def field_rel_err(F_gpu, Fo, So):
    F_gpu = np.asarray(F_gpu, np.float64)
    return np.abs(F_gpu - Fo) / np.maximum(So, 1e-300)


def assert_field(F_gpu, Fo, So, what="field"):
    err = np.abs(np.asarray(F_gpu, np.float64) - Fo)
    bad = err > FIELD_RTOL * So + 1e-30
    if bad.any():
        i = np.flatnonzero(bad.ravel())[0]
        raise AssertionError(
            f"{what}: {int(bad.sum())} su outside 1e-5*S; first flat index {i}: gpu "
            f"{np.asarray(F_gpu).ravel()[i]!r} oracle {Fo.ravel()[i]!r} S {So.ravel()[i]!r}")
    return float(np.max(err / np.maximum(So, 1e-300), initial=0.0))


def tie_sets(E, T, adm, ch_o):
    """Boolean [n, 9]: candidates tied with the oracle's choice within tolerance."""
    n = E.shape[0]
    Ea = np.where(adm == 1, E, np.inf)
    best = Ea[np.arange(n), ch_o]
    Tb = T[np.arange(n), ch_o]
    with np.errstate(invalid="ignore"):
        return np.abs(Ea - best[:, None]) <= TIE_RTOL * (T + Tb[:, None])


def compare_choices(ch_gpu, ch_o, E, T, adm):
    """Returns the number of tie flips; raises on any non-tie disagreement."""
    ch_gpu = np.asarray(ch_gpu)
    diff = ch_gpu != ch_o
    if not diff.any():
        return 0
    ties = tie_sets(E, T, adm, ch_o)
    ok = ties[np.arange(len(ch_gpu)), ch_gpu]
    bad = diff & ~ok
    if bad.any():
        i = int(np.flatnonzero(bad)[0])
        raise AssertionError(f"{int(bad.sum())} decisions differ outside ties; ped {i}: gpu "
                             f"{ch_gpu[i]} oracle {ch_o[i]} E {E[i]} adm {adm[i]}")
    return int(diff.sum())


class OracleRun:
    """Oracle state for a scene, advanced by the oracle's own steps."""

    def __init__(self, scene):
        self.sc = scene
        self.m = O.model(scene)
        self.D = O.guidance(self.m, scene.cell)
        self.st = O.State(scene)

    def field(self, req=None):
        occ, bad = O.occupancy(self.m, self.sc.cell, self.st.xy, self.st.alive)
        assert bad == 0
        return O.field(self.m, self.sc.cell, occ, self.st.heading, 3, req)

    def decide(self, req=None, Ffull=None, Sfull=None):
        occ, _ = O.occupancy(self.m, self.sc.cell, self.st.xy, self.st.alive)
        cov = None
        if self.st.w is not None:
            cov, _ = O.cover(self.m, self.sc.cell, self.st.xy, self.st.alive, self.st.w, self.st.h)
        return O.decide(self.m, self.sc.cell, occ, self.st.xy, self.st.heading, self.st.goal,
                        self.st.alive, self.D, req, Ffull, Sfull, cov, self.st.w, self.st.h)

    def advance(self, choice):
        won, maxc = O.vote(self.m, self.st.t, self.st.xy, self.st.alive, choice, self.st.w,
                           self.st.h)
        left = O.commit(self.m, self.sc.cell, self.st.xy, self.st.heading, self.st.alive,
                        choice, won, self.st.w, self.st.h)
        self.st.t += 1
        self.st.exited += left
        return won, maxc


def rect_cells(W, H, px, py, x, y, w, h):
    """su of the w x h rectangle centred on (x, y); None if it leaves a closed
    lattice."""
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


def sized_subset(sc, size):
    """The scene's pedestrians whose size x size rectangles fit: inside, off
    walls, centre on a FREE su, no overlap with an earlier one.  Returns a
    scene of those pedestrians and their sizes."""
    import scenegen as SG
    keep, taken = [], set()
    for p in range(sc.n):
        rc = rect_cells(sc.W, sc.H, sc.periodic_x, sc.periodic_y, sc.xy[p, 0], sc.xy[p, 1],
                        size[p], size[p])
        if rc is None or rc & taken or any(sc.cell[v, u] == SG.WALL for u, v in rc):
            continue
        if sc.cell[sc.xy[p, 1], sc.xy[p, 0]] != SG.FREE:
            continue
        keep.append(p)
        taken |= rc
    sub = SG.Scene(sc.name + "-sized", sc.W, sc.H, sc.periodic_x, sc.periodic_y, sc.cell,
                   sc.xy[keep].copy(), sc.heading[keep].copy(), sc.goal[keep].copy(), sc.params)
    return sub, np.ascontiguousarray(size[keep], np.uint8)
