"""Seeded synthetic scenes for the discrete social-field pedestrian model.

This module is the only code shared by the CUDA library's tests/benchmark and
the CPU oracle.  It draws inputs (lattice geometry, obstacles, exits, initial
pedestrian placement and headings) and holds none of the model's arithmetic:
no field law, no guidance distance, no move rule, no vote.

Lattice conventions (used by both sides):
  * ``cell[y, x]`` is a ``uint8`` H x W array: 0 = FREE, 1 = WALL, 2 = EXIT.
    ``x`` is the column, ``y`` the row index.
  * Direction classes 0..8 index the stay move and the 8 neighbour moves
    (the move set of the discrete model with v_max = 1 su/tick, Sec. 2):
        0 (0,0)  1 (1,0)  2 (1,1)  3 (0,1)  4 (-1,1)
        5 (-1,0) 6 (-1,-1) 7 (0,-1) 8 (1,-1)
  * A pedestrian is (x, y, heading class, goal class).  The heading class is
    the direction of the last move (0 = none yet).  The goal class is 0 for an
    exit-seeking pedestrian, or 1..8 for a pedestrian with a fixed desired
    direction (the uni/bi/4/8-directional flows of the experiments, Sec. 5).

Workload recipes follow the experiment descriptions of Sec. 5 (uniform random
placement, periodic corridors, 1x1 pedestrians, walk period 1) at the sizes
of the five evaluation configurations: a 100x100 room, a 1000x200
counter-flow corridor, a 16384x16384 floor with 10 % rectangular obstacles and
10^6 pedestrians, a batch of 256 uneven rooms, and the surrogate's training
tiles.  Placement uses NumPy's PCG64 generator seeded per scene.
"""
from __future__ import annotations

import dataclasses
from typing import Dict, List, Optional

import numpy as np

FREE, WALL, EXIT = 0, 1, 2

# Move offsets of the nine direction classes (class index -> (dx, dy)).
DIRS = np.array([(0, 0), (1, 0), (1, 1), (0, 1), (-1, 1),
                 (-1, 0), (-1, -1), (0, -1), (1, -1)], dtype=np.int32)

DEFAULT_PARAMS = dict(r=3, kP=1.0, aP=-0.5, gamma=0.5, kO=1.0, aO=-0.5,
                      kE=-1.0, aE=-0.5, beta=1.0, seed=0)


@dataclasses.dataclass
class Scene:
    """One scene: lattice, cells, pedestrians and model parameters."""
    name: str
    W: int
    H: int
    periodic_x: int
    periodic_y: int
    cell: np.ndarray            # uint8 [H, W]
    xy: np.ndarray              # int32 [N, 2]  (x, y)
    heading: np.ndarray         # uint8 [N]
    goal: np.ndarray            # uint8 [N]
    params: Dict[str, float]
    steps: int = 1

    @property
    def n(self) -> int:
        return int(self.xy.shape[0])

    def copy(self) -> "Scene":
        return Scene(self.name, self.W, self.H, self.periodic_x, self.periodic_y,
                     self.cell.copy(), self.xy.copy(), self.heading.copy(),
                     self.goal.copy(), dict(self.params), self.steps)


def _params(**kw) -> Dict[str, float]:
    p = dict(DEFAULT_PARAMS)
    p.update(kw)
    return p


def wall_ring(W: int, H: int) -> np.ndarray:
    cell = np.zeros((H, W), dtype=np.uint8)
    cell[0, :] = WALL
    cell[H - 1, :] = WALL
    cell[:, 0] = WALL
    cell[:, W - 1] = WALL
    return cell


def add_exit(cell: np.ndarray, side: str, length: int, centre: Optional[int] = None) -> None:
    """Turn ``length`` wall su of one boundary side into EXIT su (centred)."""
    H, W = cell.shape
    span = H if side in ("east", "west") else W
    c = span // 2 if centre is None else centre
    lo = max(1, c - length // 2)
    hi = min(span - 1, lo + length)
    if side == "east":
        cell[lo:hi, W - 1] = EXIT
    elif side == "west":
        cell[lo:hi, 0] = EXIT
    elif side == "north":
        cell[H - 1, lo:hi] = EXIT
    elif side == "south":
        cell[0, lo:hi] = EXIT
    else:
        raise ValueError(side)


def reachable_mask(cell: np.ndarray, periodic_x: int = 0, periodic_y: int = 0) -> np.ndarray:
    """Non-WALL su 8-connected to some EXIT su (connectivity only, no distances)."""
    from scipy import ndimage
    passable = cell != WALL
    lab, _ = ndimage.label(passable, structure=np.ones((3, 3), dtype=bool))
    if periodic_x or periodic_y:
        # merge labels across the periodic seams with a tiny union-find
        parent = np.arange(lab.max() + 1)

        def find(a):
            while parent[a] != a:
                parent[a] = parent[parent[a]]
                a = parent[a]
            return a

        def seam(a_lab, b_lab):
            for dshift in (-1, 0, 1):
                b = np.roll(b_lab, dshift)
                m = (a_lab > 0) & (b > 0)
                for u, v in set(zip(a_lab[m].tolist(), b[m].tolist())):
                    ru, rv = find(u), find(v)
                    if ru != rv:
                        parent[ru] = rv
        if periodic_x:
            seam(lab[:, 0], lab[:, -1])
        if periodic_y:
            seam(lab[0, :], lab[-1, :])
        roots = np.array([find(i) for i in range(parent.size)])
        lab = roots[lab]
    exit_labels = np.unique(lab[cell == EXIT])
    exit_labels = exit_labels[exit_labels > 0]
    lut = np.zeros(int(lab.max()) + 1, dtype=bool)
    lut[exit_labels] = True
    return lut[lab] & passable


def place_uniform(rng: np.random.Generator, mask: np.ndarray, n: int) -> np.ndarray:
    """n distinct su drawn uniformly from ``mask``; returns int32 [n, 2] (x, y)."""
    H, W = mask.shape
    total = int(mask.sum())
    if n > total:
        raise ValueError(f"cannot place {n} pedestrians on {total} free su")
    if mask.size <= (1 << 24):
        idx = rng.choice(np.flatnonzero(mask.ravel()), size=n, replace=False)
    else:
        # rejection sampling for huge lattices (avoids materialising the index list)
        picked = np.empty(0, dtype=np.int64)
        flat = mask.ravel()
        while picked.size < n:
            need = n - picked.size
            cand = rng.integers(0, mask.size, size=int(need * 1.3) + 1024, dtype=np.int64)
            cand = cand[flat[cand]]
            picked = np.concatenate([picked, cand])
            _, first = np.unique(picked, return_index=True)
            picked = picked[np.sort(first)]
        idx = picked[:n]
    xy = np.stack([idx % W, idx // W], axis=1).astype(np.int32)
    return xy


# --------------------------------------------------------------------------
# Evaluation configurations
# --------------------------------------------------------------------------

def room(W=100, H=100, n=200, r=10, exit_len=10, seed=1, steps=50, name="room") -> Scene:
    """Walled room with one exit segment centred on the east wall; exit-seekers."""
    rng = np.random.default_rng(seed)
    cell = wall_ring(W, H)
    add_exit(cell, "east", exit_len)
    xy = place_uniform(rng, cell == FREE, n)
    return Scene(name, W, H, 0, 0, cell, xy, np.zeros(n, np.uint8),
                 np.zeros(n, np.uint8), _params(r=r, seed=seed), steps)


def corridor(W=1000, H=200, n=20000, r=20, seed=2, steps=500, name="corridor") -> Scene:
    """Counter-flow corridor: walls on the first and last rows, periodic in x.

    Half the crowd starts in the west third and walks east (goal class 1), the
    other half starts in the east third and walks west (goal class 5)."""
    rng = np.random.default_rng(seed)
    cell = np.zeros((H, W), dtype=np.uint8)
    cell[0, :] = WALL
    cell[H - 1, :] = WALL
    free = cell == FREE
    west = free.copy()
    west[:, W // 3:] = False
    east = free.copy()
    east[:, : W - W // 3] = False
    na = n // 2
    xy = np.concatenate([place_uniform(rng, west, na), place_uniform(rng, east, n - na)])
    goal = np.concatenate([np.full(na, 1, np.uint8), np.full(n - na, 5, np.uint8)])
    return Scene(name, W, H, 1, 0, cell, xy, goal.copy(), goal,
                 _params(r=r, seed=seed), steps)


def floor(side=16384, n=1_000_000, r=40, coverage=0.10, exit_len=256, side_min=5,
          side_max=200, seed=3, steps=200, reachable=False, name="floor") -> Scene:
    """Large floor: wall ring, one exit centred on each wall, random axis-aligned
    rectangular obstacles (integer sides uniform in [side_min, side_max],
    positions uniform, overlap allowed) added until WALL su cover ``coverage``
    of the area; pedestrians uniform on free su (``reachable=True`` restricts
    them to su 8-connected to an exit; a pedestrian in a sealed pocket has no
    guidance pull and moves by the field alone)."""
    rng = np.random.default_rng(seed)
    W = H = side
    cell = wall_ring(W, H)
    target = int(coverage * W * H)
    walls = int((cell == WALL).sum())
    while walls < target:
        batch = 64
        ws = rng.integers(side_min, side_max + 1, size=batch)
        hs = rng.integers(side_min, side_max + 1, size=batch)
        xs = rng.integers(1, W - 1, size=batch)
        ys = rng.integers(1, H - 1, size=batch)
        for w, h, x0, y0 in zip(ws, hs, xs, ys):
            sl = cell[y0:min(H - 1, y0 + h), x0:min(W - 1, x0 + w)]
            walls += int((sl != WALL).sum())
            sl[...] = WALL
            if walls >= target:
                break
    for s in ("east", "west", "north", "south"):
        add_exit(cell, s, exit_len)
    mask = cell == FREE
    if reachable:
        mask &= reachable_mask(cell)
    xy = place_uniform(rng, mask, n)
    return Scene(name, W, H, 0, 0, cell, xy, np.zeros(n, np.uint8),
                 np.zeros(n, np.uint8), _params(r=r, seed=seed), steps)


def batch(nscenes=256, side_lo=64, side_hi=2048, rho_lo=0.05, rho_hi=0.4, r_lo=5, r_hi=30,
          seed=4, steps=20, name="batch") -> List[Scene]:
    """Independent rooms of uneven size: side ~ U[side_lo, side_hi], density
    ~ U[rho_lo, rho_hi] of free su, radius ~ U[r_lo, r_hi], 1-4 exits of length
    max(4, side/16) on distinct walls chosen by the seed, wall ring, no
    interior obstacles."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(nscenes):
        s = int(rng.integers(side_lo, side_hi + 1))
        rho = float(rng.uniform(rho_lo, rho_hi))
        r = int(rng.integers(r_lo, r_hi + 1))
        ne = int(rng.integers(1, 5))
        cell = wall_ring(s, s)
        sides = rng.permutation(["east", "west", "north", "south"])[:ne]
        for sd in sides:
            add_exit(cell, str(sd), max(4, s // 16))
        free = cell == FREE
        n = int(rho * free.sum())
        xy = place_uniform(rng, free, n)
        out.append(Scene(f"{name}{i}", s, s, 0, 0, cell, xy, np.zeros(n, np.uint8),
                         np.zeros(n, np.uint8), _params(r=r, seed=seed * 1000 + i), steps))
    return out


def random_scene(W, H, n, r, seed, periodic_x=0, periodic_y=0, ring=True, exits=("east",),
                 exit_len=4, obstacles=0, goal_mode="exit", heading_mode="zero",
                 name="random") -> Scene:
    """Small general-purpose scene for tests.

    goal_mode: "exit" (all exit-seekers), "fixed" (random fixed directions 1..8),
    "mixed" (half each).  heading_mode: "zero", "goal" or "random" (0..8)."""
    rng = np.random.default_rng(seed)
    cell = np.zeros((H, W), dtype=np.uint8)
    if ring:
        if not periodic_y:
            cell[0, :] = WALL
            cell[H - 1, :] = WALL
        if not periodic_x:
            cell[:, 0] = WALL
            cell[:, W - 1] = WALL
    for _ in range(obstacles):
        w = int(rng.integers(1, max(2, W // 4)))
        h = int(rng.integers(1, max(2, H // 4)))
        x0 = int(rng.integers(0, W))
        y0 = int(rng.integers(0, H))
        cell[y0:y0 + h, x0:x0 + w] = WALL
    for sd in exits:
        add_exit(cell, sd, exit_len)
    free = cell == FREE
    xy = place_uniform(rng, free, n)
    if goal_mode == "exit":
        goal = np.zeros(n, np.uint8)
    elif goal_mode == "fixed":
        goal = rng.integers(1, 9, size=n).astype(np.uint8)
    elif goal_mode == "mixed":
        goal = np.where(rng.random(n) < 0.5, 0, rng.integers(1, 9, size=n)).astype(np.uint8)
    else:
        raise ValueError(goal_mode)
    if heading_mode == "zero":
        heading = np.zeros(n, np.uint8)
    elif heading_mode == "goal":
        heading = goal.copy()
    elif heading_mode == "random":
        heading = rng.integers(0, 9, size=n).astype(np.uint8)
    else:
        raise ValueError(heading_mode)
    return Scene(name, W, H, periodic_x, periodic_y, cell, xy, heading, goal,
                 _params(r=r, seed=seed), 1)


def training_scene(seed: int, side=1024, r=40, kind="floor") -> Scene:
    """A config-2/3-style scene used to draw training tiles for the surrogate."""
    rng = np.random.default_rng(seed)
    if kind == "corridor":
        sc = corridor(W=side, H=max(64, side // 4), n=int(side * side // 4 * 0.15),
                      r=r, seed=seed)
        sc.heading = rng.integers(0, 9, size=sc.n).astype(np.uint8)
        return sc
    rho = float(rng.uniform(0.002, 0.2))
    n = int(rho * side * side * 0.85)
    sc = floor(side=side, n=n, r=r, exit_len=max(8, side // 64), side_max=max(10, side // 80),
               seed=seed)
    sc.heading = rng.integers(0, 9, size=sc.n).astype(np.uint8)
    return sc


def training_canvas(side=4096, r=40, tile=128, rho_lo=0.002, rho_hi=0.25, seed=500,
                    name="canvas") -> Scene:
    """Periodic torus without walls for surrogate training: each tile x tile
    block gets its own crowd density, log-uniform in [rho_lo, rho_hi] (from the
    sparse large floor to the dense corridor ends); pedestrians walk in fixed
    random directions (classes 1..8), headed that way."""
    rng = np.random.default_rng(seed)
    nt = side // tile
    rho = np.exp(rng.uniform(np.log(rho_lo), np.log(rho_hi), size=(nt, nt)))
    u = rng.random((side, side))
    dens = np.kron(rho, np.ones((tile, tile)))
    ys, xs = np.nonzero(u < dens)
    xy = np.stack([xs, ys], axis=1).astype(np.int32)
    goal = rng.integers(1, 9, size=len(xy)).astype(np.uint8)
    cell = np.zeros((side, side), np.uint8)
    return Scene(name, side, side, 1, 1, cell, xy, goal.copy(), goal,
                 _params(r=r, seed=seed), 1)


FLOW_GOALS = {1: (1,), 2: (1, 5), 4: (1, 3, 5, 7), 8: tuple(range(1, 9))}


def paper_scene(side=1000, density=0.5, ndir=8, r=3, seed=11, name="paper") -> Scene:
    """The paper's experiment shape (Sec. 5): a periodic side x side lattice
    without walls or exits, round(density * side^2) pedestrians uniform on it,
    fixed-direction walkers split evenly over `ndir` flow directions (1: east;
    2: east and west; 4: the axes; 8: every direction), heading = direction."""
    rng = np.random.default_rng(seed)
    cell = np.zeros((side, side), np.uint8)
    n = int(round(density * side * side))
    xy = place_uniform(rng, np.ones((side, side), bool), n)
    dirs = np.array(FLOW_GOALS[ndir], np.uint8)
    goal = dirs[np.arange(n) % len(dirs)]
    rng.shuffle(goal)
    return Scene(name, side, side, 1, 1, cell, xy, goal.copy(), goal, _params(r=r))


def paper_sized_scene(g=3, side=1000, density=0.5, ndir=8, seed=13, name="paper-sized"):
    """Table V's shape: g x g pedestrians (g odd) on a periodic side x side
    lattice covering `density` of its area, i.e. round(density * side^2 / g^2)
    pedestrians, field window 7g x 7g (r = (7g - 1) / 2).  Centres are the
    centres of randomly chosen cells of a g x g block tiling, so rectangles
    never overlap.  Returns (scene, sizes)."""
    rng = np.random.default_rng(seed)
    nb = side // g
    n = int(round(density * side * side / (g * g)))
    pick = rng.choice(nb * nb, size=n, replace=False)
    xy = np.stack([(pick % nb) * g + g // 2, (pick // nb) * g + g // 2], axis=1).astype(np.int32)
    dirs = np.array(FLOW_GOALS[ndir], np.uint8)
    goal = dirs[np.arange(n) % len(dirs)]
    rng.shuffle(goal)
    cell = np.zeros((side, side), np.uint8)
    sc = Scene(name, side, side, 1, 1, cell, xy, goal.copy(), goal, _params(r=(7 * g - 1) // 2))
    return sc, np.full(n, g, np.uint8)


def walk_periods(n, p_max, seed=12):
    """Walk periods uniform in [1, p_max] and phases uniform in [0, period)."""
    rng = np.random.default_rng(seed)
    period = rng.integers(1, p_max + 1, size=n).astype(np.uint8)
    phase = (rng.integers(0, 1 << 16, size=n) % period).astype(np.uint8)
    return period, phase


def config(i: int, **kw):
    """The five evaluation configurations by number (1-based)."""
    if i == 1:
        return room(**kw)
    if i == 2:
        return corridor(**kw)
    if i == 3:
        return floor(**kw)
    if i == 4:
        return batch(**kw)
    raise ValueError(i)


SURROGATE_LAYERS = ((3, 32, 5), (32, 32, 3), (32, 32, 3), (32, 1, 3))  # (Cin, Cout, k)


def surrogate_init(seed: int = 0):
    """Seeded initial weights of the field surrogate's 4 layers: [(W [out, in,
    k, k], b [out]), ...], W normal with standard deviation sqrt(2 / (in k^2)),
    b zero.  Random inputs only: the network's arithmetic lives elsewhere."""
    rng = np.random.default_rng(seed)
    ps = []
    for cin, cout, k in SURROGATE_LAYERS:
        std = np.sqrt(2.0 / (cin * k * k))
        ps.append((rng.normal(0.0, std, (cout, cin, k, k)), np.zeros(cout)))
    return ps
