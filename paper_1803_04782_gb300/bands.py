"""Row-band decomposition of one lattice over several ranks (one process per
device): the multi-device form of the divide-and-conquer split of Sec. 3.3
(Eq. 1, Alg. 3), where the lattice's rows, not a pedestrian's fan-out, are
what is split.

Rank k owns a contiguous band of rows [y0, y1) and every pedestrian standing
in it.  It steps a context (`stepper`) over its band plus `h` = r + 3 rows
on each side, in which the pedestrians its neighbours own within those rows
appear as ghosts, numbered as in the whole lattice.  Each tick:

1. each rank sends each neighbour the pedestrians it owns inside the
   neighbour's halo'd rows (one exchange per neighbour and tick);
2. each rank places its own pedestrians and the ghosts it received, at the
   whole lattice's tick, and steps one tick;
3. each rank keeps the pedestrians whose new su lies in its own rows: its
   own that stayed, and ghosts that crossed into them.  Pedestrians that
   moved out are kept by the neighbour, which computed the same move for
   its ghost.  An owner counts its pedestrians that left through an exit.

Why this is exact: a pedestrian within 2 rows of an edge decides on the
field of the rows up to 3 beyond it, which sums the pedestrians within r of
those rows -- all inside the halo -- and its competitors for a target
within 1 row of the edge stand within 2 rows of it, so both sides compute
the same decisions, elections and moves for every pedestrian either of them
keeps.  Band origins are multiples of the 32-su bin, so each band's bins,
footprints and summation order are those of the whole lattice, and the
fields agree bit for bit.  The guidance distances, which run through other
bands, are the whole lattice's (sfm_set_guidance); the election numbers are
the whole lattice's pedestrian numbers (sfm_set_ids).

The exchange goes through a `comm` object with exchange(sends) -> receives
(`TorchComm` on torch.distributed point-to-point sends: host tensors with
the gloo backend, device tensors with NCCL).  Walk periods and multi-su pedestrians are not
carried.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Callable, Dict, List, Tuple

import numpy as np

BIN = 32          # band origins are multiples of the library's pedestrian bin
HALO_EXTRA = 3    # rows beyond r that the exactness argument above needs


@dataclass
class Peds:
    """Pedestrians in whole-lattice coordinates: number, position, heading
    class, goal class."""
    ids: np.ndarray      # int32 [n]
    xy: np.ndarray       # int32 [n, 2]
    heading: np.ndarray  # uint8 [n]
    goal: np.ndarray     # uint8 [n]

    @property
    def n(self) -> int:
        return int(self.ids.shape[0])

    def take(self, m) -> "Peds":
        return Peds(self.ids[m], self.xy[m], self.heading[m], self.goal[m])

    @staticmethod
    def cat(parts: List["Peds"]) -> "Peds":
        return Peds(np.concatenate([p.ids for p in parts]).astype(np.int32),
                    np.concatenate([p.xy for p in parts]).reshape(-1, 2).astype(np.int32),
                    np.concatenate([p.heading for p in parts]).astype(np.uint8),
                    np.concatenate([p.goal for p in parts]).astype(np.uint8))

    def pack(self) -> np.ndarray:
        """One int32 row per pedestrian: id, x, y, heading, goal."""
        return np.stack([self.ids, self.xy[:, 0], self.xy[:, 1], self.heading.astype(np.int32),
                         self.goal.astype(np.int32)], axis=1).astype(np.int32).reshape(-1, 5)

    @staticmethod
    def unpack(a: np.ndarray) -> "Peds":
        a = np.asarray(a, np.int32).reshape(-1, 5)
        return Peds(a[:, 0].copy(), a[:, 1:3].copy(), a[:, 3].astype(np.uint8),
                    a[:, 4].astype(np.uint8))


class BandLayout:
    """Own rows and halo'd rows of each rank (see the module docstring)."""

    def __init__(self, H: int, periodic_y: int, r: int, nranks: int):
        if nranks < 1:
            raise ValueError("need at least one rank")
        if periodic_y and H % BIN:
            raise ValueError(f"a periodic lattice is split only when its height is a multiple of {BIN}")
        self.H, self.py, self.r, self.nranks = int(H), int(periodic_y), int(r), int(nranks)
        self.h = self.r + HALO_EXTRA
        units = -(-self.H // BIN)
        if units < nranks:
            raise ValueError(f"{H} rows give fewer than {nranks} bands of {BIN} rows")
        cuts = [min(self.H, (k * units // nranks) * BIN) for k in range(nranks + 1)]
        cuts[-1] = self.H
        self.y0 = np.array(cuts[:-1], np.int64)
        self.y1 = np.array(cuts[1:], np.int64)
        if nranks > 1 and (self.y1 - self.y0).min() < self.h + BIN:
            raise ValueError(f"bands of at least r + {HALO_EXTRA} + {BIN} rows needed "
                             f"(ghosts come from the next bands only)")
        s0, s1 = [], []
        for k in range(nranks):
            a = (int(self.y0[k]) - self.h) // BIN * BIN
            b = int(self.y1[k]) + self.h
            if not self.py or nranks == 1:
                a, b = max(a, 0), min(b, self.H)
            if b - a > self.H:
                raise ValueError("a band's halo wraps onto itself")
            s0.append(a)
            s1.append(b)
        self.s0 = np.array(s0, np.int64)
        self.s1 = np.array(s1, np.int64)

    def rows(self, k: int) -> Tuple[int, int]:
        """Whole-lattice origin row (may be negative: wrapped) and height of
        rank k's halo'd sub-lattice."""
        return int(self.s0[k]), int(self.s1[k] - self.s0[k])

    def local_row(self, k: int, y) -> np.ndarray:
        """Row of whole-lattice row y in rank k's sub-lattice (>= height: outside)."""
        y = np.asarray(y, np.int64)
        d = y - self.s0[k]
        return d % self.H if self.py else d

    def in_sub(self, k: int, y) -> np.ndarray:
        d = self.local_row(k, y)
        return (d >= 0) & (d < self.s1[k] - self.s0[k])

    def global_row(self, k: int, yl) -> np.ndarray:
        y = self.s0[k] + np.asarray(yl, np.int64)
        return y % self.H if self.py else y

    def owner(self, y) -> np.ndarray:
        return np.searchsorted(self.y1, np.asarray(y, np.int64), side="right")

    def neighbours(self, k: int) -> List[int]:
        """Ranks whose halo'd rows meet rank k's own rows (and the other way)."""
        out = []
        for j in (k - 1, k + 1):
            if self.py:
                j %= self.nranks
            if 0 <= j < self.nranks and j != k and j not in out:
                out.append(j)
        return out

    def sub_cells(self, k: int, cell: np.ndarray) -> np.ndarray:
        a, n = self.rows(k)
        return np.ascontiguousarray(cell[np.arange(a, a + n) % self.H])


def own_of(layout: BandLayout, k: int, peds: Peds) -> Peds:
    """The pedestrians of a whole-lattice set that rank k owns."""
    return peds.take(layout.owner(peds.xy[:, 1]) == k)


def sends_of(layout: BandLayout, k: int, own: Peds) -> Dict[int, Peds]:
    """What rank k sends each neighbour: its own pedestrians inside the
    neighbour's halo'd rows."""
    return {j: own.take(layout.in_sub(j, own.xy[:, 1])) for j in layout.neighbours(k)}


class TorchComm:
    """Neighbour exchange over torch.distributed point-to-point messages: a
    count, then the packed pedestrians.  The messages are tensors on
    `device`: host tensors for the gloo backend (the default), CUDA tensors
    of the rank's device for NCCL."""

    def __init__(self, dist, device="cpu"):
        self.dist = dist
        self.device = device

    def exchange(self, sends: Dict[int, np.ndarray]) -> Dict[int, np.ndarray]:
        import torch
        d, dev = self.dist, self.device
        counts = {j: torch.tensor([a.shape[0]], dtype=torch.int64, device=dev)
                  for j, a in sends.items()}
        rcounts = {j: torch.zeros(1, dtype=torch.int64, device=dev) for j in sends}
        reqs = [d.irecv(rcounts[j], src=j) for j in sends]
        reqs += [d.isend(counts[j], dst=j) for j in sends]
        for q in reqs:
            q.wait()
        bufs = {j: torch.zeros((int(rcounts[j].item()), 5), dtype=torch.int32, device=dev)
                for j in sends}
        data = {j: torch.from_numpy(np.ascontiguousarray(a, np.int32).reshape(-1, 5)).to(dev)
                for j, a in sends.items()}
        reqs = [d.irecv(bufs[j], src=j) for j in sends if bufs[j].numel()]
        reqs += [d.isend(data[j], dst=j) for j in sends if data[j].numel()]
        for q in reqs:
            q.wait()
        return {j: bufs[j].cpu().numpy() for j in sends}


# a stepper advances the placed pedestrians of a sub-lattice by one tick:
# stepper(xy_local, heading, goal, ids, t) -> (xy_local, heading, alive)
Stepper = Callable[[np.ndarray, np.ndarray, np.ndarray, np.ndarray, int],
                   Tuple[np.ndarray, np.ndarray, np.ndarray]]


def band_tick(layout: BandLayout, k: int, comm, stepper: Stepper, own: Peds,
              t: int) -> Tuple[Peds, int]:
    """One tick of rank k: exchange, place own + ghosts, step, keep what lands
    in the own rows.  Returns (new own pedestrians, own pedestrians that left
    through an exit)."""
    recv = comm.exchange({j: p.pack() for j, p in sends_of(layout, k, own).items()})
    ghosts = [Peds.unpack(a) for a in recv.values()]
    allp = Peds.cat([own] + ghosts)
    xy = allp.xy.copy()
    xy[:, 1] = layout.local_row(k, xy[:, 1])
    nxy, nh, alive = stepper(np.ascontiguousarray(xy, np.int32), allp.heading, allp.goal,
                             allp.ids, t)
    gy = layout.global_row(k, nxy[:, 1])
    keep = (alive != 0) & (layout.owner(gy) == k)
    left = int(np.count_nonzero(alive[:own.n] == 0))
    new = Peds(allp.ids[keep], np.stack([nxy[keep, 0], gy[keep]], axis=1).astype(np.int32),
               np.asarray(nh)[keep].astype(np.uint8), allp.goal[keep])
    return new, left


def sim_stepper(layout: BandLayout, k: int, W: int, periodic_x: int, cell: np.ndarray,
                D: np.ndarray, params: dict, stream=None) -> Tuple[Stepper, object]:
    """A stepper on this library: one context over rank k's halo'd rows (its
    cells, the whole lattice's guidance distances for them), re-placed every
    tick with the whole lattice's pedestrian numbers and tick.  Returns
    (stepper, the Sim, to be closed by the caller)."""
    from . import Sim
    a, n = layout.rows(k)
    rows = np.arange(a, a + n) % layout.H
    sim = Sim(W=W, H=n, cell=np.ascontiguousarray(cell[rows]), periodic_x=periodic_x,
              periodic_y=0, stream=stream, **params)
    sim.set_guidance(np.ascontiguousarray(D[rows], np.int32))

    def step(xy, heading, goal, ids, t):
        sim.place(xy, heading, goal)
        sim.set_ids(ids)
        sim.set_time(t)
        sim.step(1)
        return sim.peds()

    return step, sim
