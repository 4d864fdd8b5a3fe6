"""FP64 CPU oracle of the discrete social-field pedestrian step (test infrastructure).

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
use this package.  It wraps ``sfm_oracle.c`` (plain C, FP64, OpenMP over
independent outputs) with ctypes and NumPy marshalling, and shares no code with
the CUDA library.  The model it computes is stated in the header of
``sfm_oracle.c``: field superposition (Sec. 2, sub-job k-5 of Sec. 3.1), the
decision over 9 candidate su (k-2, v_max = 1), the vote of the enrollment
container (k-3, Sec. 3.1 s-2) and the commit (k-4), i.e. one tick of Alg. 1.
"""
from __future__ import annotations

import ctypes as C
import os
import subprocess
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sfm_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lib = None

FREE, WALL, EXIT = 0, 1, 2
DINF = 1 << 23
DIRS = np.array([(0, 0), (1, 0), (1, 1), (0, 1), (-1, 1),
                 (-1, 0), (-1, -1), (0, -1), (1, -1)], dtype=np.int32)


class Model(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("periodic_x", C.c_int32),
                ("periodic_y", C.c_int32), ("r", C.c_int32), ("pad_", C.c_int32),
                ("kP", C.c_double), ("aP", C.c_double), ("gamma", C.c_double),
                ("kO", C.c_double), ("aO", C.c_double), ("kE", C.c_double),
                ("aE", C.c_double), ("beta", C.c_double), ("seed", C.c_uint64)]


def build(force: bool = False) -> str:
    """Compile sfm_oracle.c into oracle/_build/liboracle.so (gcc, OpenMP if available)."""
    os.makedirs(_BUILD, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    base = ["gcc", "-O2", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"]
    try:
        subprocess.check_call(base[:1] + ["-fopenmp"] + base[1:])
    except subprocess.CalledProcessError:
        subprocess.check_call(base)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def lib():
    global _lib
    if _lib is None:
        build()
        L = C.CDLL(_LIB_PATH)
        P = C.c_void_p
        M = C.POINTER(Model)
        L.orc_num_threads.restype = C.c_int
        L.orc_set_threads.argtypes = [C.c_int]
        L.orc_kernel.restype = C.c_double
        L.orc_kernel.argtypes = [M, C.c_int, C.c_int, C.c_int, C.c_int]
        L.orc_occupancy.restype = C.c_int64
        L.orc_occupancy.argtypes = [M, P, C.c_int32, P, P, P]
        L.orc_field.restype = None
        L.orc_field.argtypes = [M, P, P, P, C.c_int32, C.c_int64, P, P, P]
        L.orc_guidance.restype = C.c_int
        L.orc_guidance.argtypes = [M, P, P]
        L.orc_mix64.restype = C.c_uint64
        L.orc_mix64.argtypes = [C.c_uint64]
        L.orc_splitmix64_nth.restype = C.c_uint64
        L.orc_splitmix64_nth.argtypes = [C.c_uint64, C.c_uint64]
        L.orc_prio.restype = C.c_uint64
        L.orc_prio.argtypes = [C.c_uint64, C.c_int64, C.c_int64]
        L.orc_decide.restype = None
        L.orc_decide.argtypes = [M, P, P, P, P, P, P, P, P, P, C.c_int64, P, P, P, P, P, P, P, P, P]
        L.orc_cover.restype = C.c_int64
        L.orc_cover.argtypes = [M, P, C.c_int32, P, P, P, P, P]
        L.orc_vote_sized.restype = C.c_int32
        L.orc_vote_sized.argtypes = [M, C.c_int64, C.c_int32, P, P, P, P, P, P]
        L.orc_vote.restype = C.c_int32
        L.orc_vote.argtypes = [M, C.c_int64, C.c_int32, P, P, P, P]
        L.orc_vote_numbered.restype = C.c_int32
        L.orc_vote_numbered.argtypes = [M, C.c_int64, C.c_int32, P, P, P, P, P]
        L.orc_commit.restype = C.c_int32
        L.orc_commit.argtypes = [M, P, C.c_int32, P, P, P, P, P, P, P]
        L.orc_step.restype = C.c_int32
        L.orc_step.argtypes = [M, P, P, C.c_int64, C.c_int32, P, P, P, P, P, P, P, P, P, P, P]
        L.orc_gate_periods.restype = None
        L.orc_gate_periods.argtypes = [C.c_int64, C.c_int32, P, P, P]
        _lib = L
    return _lib


def _p(a: Optional[np.ndarray]):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def model(scene=None, **kw) -> Model:
    """Model parameters from a scene (scenegen.Scene) and/or keyword overrides."""
    d = dict(W=1, H=1, periodic_x=0, periodic_y=0, r=3, kP=1.0, aP=-0.5, gamma=0.5,
             kO=1.0, aO=-0.5, kE=-1.0, aE=-0.5, beta=1.0, seed=0)
    if scene is not None:
        d.update(W=scene.W, H=scene.H, periodic_x=scene.periodic_x, periodic_y=scene.periodic_y)
        d.update({k: v for k, v in scene.params.items() if k in d})
    d.update(kw)
    m = Model()
    for k, v in d.items():
        setattr(m, k, v)
    return m


def threads() -> int:
    return lib().orc_num_threads()


def set_threads(n: int) -> None:
    lib().orc_set_threads(int(n))


def kernel(m: Model, kind: int, dx: int, dy: int, hcls: int = 0) -> float:
    """Kernel value of one source (kind 0 pedestrian, 1 WALL, 2 EXIT) at c - source = (dx, dy)."""
    return lib().orc_kernel(C.byref(m), kind, dx, dy, hcls)


def occupancy(m: Model, cell: np.ndarray, xy: np.ndarray, alive=None):
    cell = np.ascontiguousarray(cell, np.uint8)
    xy = np.ascontiguousarray(xy, np.int32)
    alive = None if alive is None else np.ascontiguousarray(alive, np.uint8)
    occ = np.empty(m.W * m.H, np.int32)
    bad = lib().orc_occupancy(C.byref(m), _p(cell), xy.shape[0], _p(xy), _p(alive), _p(occ))
    return occ, int(bad)


def field(m: Model, cell, occ, heading, parts: int = 3, req=None):
    """(F, S) at requested su indices (row-major y*W+x), or the whole lattice [H, W]."""
    cell = np.ascontiguousarray(cell, np.uint8)
    occ = np.ascontiguousarray(occ, np.int32)
    heading = np.ascontiguousarray(heading, np.uint8)
    if heading.size == 0:
        heading = np.zeros(1, np.uint8)
    if req is None:
        n = m.W * m.H
        F = np.empty(n, np.float64)
        S = np.empty(n, np.float64)
        lib().orc_field(C.byref(m), _p(cell), _p(occ), _p(heading), parts, n, None, _p(F), _p(S))
        return F.reshape(m.H, m.W), S.reshape(m.H, m.W)
    req = np.ascontiguousarray(req, np.int64)
    F = np.empty(req.size, np.float64)
    S = np.empty(req.size, np.float64)
    lib().orc_field(C.byref(m), _p(cell), _p(occ), _p(heading), parts, req.size, _p(req),
                    _p(F), _p(S))
    return F, S


def guidance(m: Model, cell) -> np.ndarray:
    """Chamfer (5, 7) geodesic distance to the nearest EXIT, int32 [H, W]; DINF if unreachable."""
    cell = np.ascontiguousarray(cell, np.uint8)
    D = np.empty(m.W * m.H, np.int32)
    lib().orc_guidance(C.byref(m), _p(cell), _p(D))
    return D.reshape(m.H, m.W)


def mix64(z: int) -> int:
    return int(lib().orc_mix64(z & (2**64 - 1)))


def splitmix64_nth(s: int, i: int) -> int:
    return int(lib().orc_splitmix64_nth(s & (2**64 - 1), i))


def prio(seed: int, t: int, pid: int) -> int:
    return int(lib().orc_prio(seed & (2**64 - 1), t, pid))


def cover(m: Model, cell, xy, alive, w, h):
    """Multi-su occupancy: [H, W] int32 holding p on every su of p's w x h
    rectangle (-1 elsewhere), and the number of placement violations."""
    cell = np.ascontiguousarray(cell, np.uint8)
    xy = np.ascontiguousarray(xy, np.int32)
    alive = None if alive is None else np.ascontiguousarray(alive, np.uint8)
    w = np.ascontiguousarray(w, np.uint8)
    h = np.ascontiguousarray(h, np.uint8)
    cov = np.empty(m.W * m.H, np.int32)
    bad = lib().orc_cover(C.byref(m), _p(cell), xy.shape[0], _p(xy), _p(alive), _p(w), _p(h),
                          _p(cov))
    return cov, int(bad)


def decide(m: Model, cell, occ, xy, heading, goal, alive, D, req=None, Ffull=None, Sfull=None,
           cov=None, w=None, h=None, magnitudes=False):
    """Decision of the requested pedestrians: (choice, E[.,9], T[.,9], admissible[.,9]),
    and with magnitudes=True also Mag[.,9] = |F| + |own| + |guidance| per
    candidate (the scale of a near tie, see near_ties).
    cov/w/h: multi-su pedestrians (admissibility over the su a move enters)."""
    cell = np.ascontiguousarray(cell, np.uint8)
    occ = np.ascontiguousarray(occ, np.int32)
    xy = np.ascontiguousarray(xy, np.int32)
    heading = np.ascontiguousarray(heading, np.uint8)
    goal = np.ascontiguousarray(goal, np.uint8)
    alive = np.ascontiguousarray(alive, np.uint8)
    D = np.ascontiguousarray(D, np.int32)
    if Ffull is not None:
        Ffull = np.ascontiguousarray(Ffull, np.float64)
        Sfull = np.ascontiguousarray(Sfull, np.float64)
    n = xy.shape[0] if req is None else len(req)
    reqa = None if req is None else np.ascontiguousarray(req, np.int32)
    choice = np.zeros(max(n, 1), np.uint8)
    E = np.zeros((max(n, 1), 9), np.float64)
    T = np.zeros((max(n, 1), 9), np.float64)
    adm = np.zeros((max(n, 1), 9), np.uint8)
    Mag = np.zeros((max(n, 1), 9), np.float64) if magnitudes else None
    if cov is not None:
        cov = np.ascontiguousarray(cov, np.int32)
        w = np.ascontiguousarray(w, np.uint8)
        h = np.ascontiguousarray(h, np.uint8)
    lib().orc_decide(C.byref(m), _p(cell), _p(occ), _p(xy), _p(heading), _p(goal), _p(alive),
                     _p(D), _p(Ffull), _p(Sfull), n, _p(reqa), _p(choice), _p(E), _p(T), _p(adm),
                     _p(cov), _p(w), _p(h), _p(Mag))
    if magnitudes:
        return choice[:n], E[:n], T[:n], adm[:n], Mag[:n]
    return choice[:n], E[:n], T[:n], adm[:n]


def best_two(E, adm):
    """Per pedestrian: the smallest admissible energy (ties to the smallest
    class), the candidate index holding it, and the next one in that order
    (index -1 when only one candidate is admissible)."""
    n = E.shape[0]
    Ea = np.where(adm == 1, E, np.inf)
    # stable sort by energy: equal energies keep the class order
    order = np.argsort(Ea, axis=1, kind="stable")
    b = order[:, 0]
    s = order[:, 1]
    has2 = np.isfinite(Ea[np.arange(n), s])
    return b, np.where(has2, s, -1)


def near_ties(E, Mag, adm, rtol=1e-5):
    """Boolean per pedestrian: its best and second-best admissible energies
    E_a <= E_b satisfy E_b - E_a <= rtol (Mag_a + Mag_b), the near-tie rule
    the library counts (a field rounded otherwise may break such a choice
    either way).  A pedestrian with one admissible candidate has none."""
    n = E.shape[0]
    b, s = best_two(E, adm)
    ok = s >= 0
    i = np.arange(n)
    sj = np.where(ok, s, 0)
    with np.errstate(invalid="ignore"):   # dead pedestrians: inf - inf
        gap = E[i, sj] - E[i, b]
        return ok & (gap <= rtol * (Mag[i, b] + Mag[i, sj]))


def vote(m: Model, t: int, xy, alive, choice, w=None, h=None, ids=None):
    """Winners of the tick's moves (w/h: multi-su pedestrians, claims; ids:
    the pedestrians' numbers for their priorities, default their indices)."""
    xy = np.ascontiguousarray(xy, np.int32)
    alive = np.ascontiguousarray(alive, np.uint8)
    choice = np.ascontiguousarray(choice, np.uint8)
    won = np.zeros(max(xy.shape[0], 1), np.uint8)
    if w is not None:
        w = np.ascontiguousarray(w, np.uint8)
        h = np.ascontiguousarray(h, np.uint8)
        maxc = lib().orc_vote_sized(C.byref(m), t, xy.shape[0], _p(xy), _p(alive), _p(choice),
                                    _p(w), _p(h), _p(won))
    elif ids is not None:
        ids = np.ascontiguousarray(ids, np.int32)
        maxc = lib().orc_vote_numbered(C.byref(m), t, xy.shape[0], _p(xy), _p(alive),
                                       _p(choice), _p(ids), _p(won))
    else:
        maxc = lib().orc_vote(C.byref(m), t, xy.shape[0], _p(xy), _p(alive), _p(choice),
                              _p(won))
    return won[:xy.shape[0]], int(maxc)


def commit(m: Model, cell, xy, heading, alive, choice, won, w=None, h=None):
    """Apply the moves in place; returns the number of pedestrians that left
    (w/h: multi-su pedestrians leave when their new rectangle meets an EXIT)."""
    cell = np.ascontiguousarray(cell, np.uint8)
    if w is not None:
        w = np.ascontiguousarray(w, np.uint8)
        h = np.ascontiguousarray(h, np.uint8)
    return int(lib().orc_commit(C.byref(m), _p(cell), xy.shape[0], _p(xy), _p(heading),
                                _p(alive), _p(np.ascontiguousarray(choice, np.uint8)),
                                _p(np.ascontiguousarray(won, np.uint8)), _p(w), _p(h)))


class State:
    """Pedestrian state carried between oracle steps."""

    def __init__(self, scene):
        self.xy = np.ascontiguousarray(scene.xy, np.int32).copy()
        self.heading = np.ascontiguousarray(scene.heading, np.uint8).copy()
        self.goal = np.ascontiguousarray(scene.goal, np.uint8).copy()
        self.alive = np.ones(scene.n, np.uint8)
        self.t = 0
        self.exited = 0
        # walk periods (None: every pedestrian active every tick)
        self.period = None
        self.phase = None
        # multi-su pedestrians: odd widths and heights (None: 1 x 1)
        self.w = None
        self.h = None

    def copy(self):
        s = State.__new__(State)
        s.xy, s.heading, s.goal = self.xy.copy(), self.heading.copy(), self.goal.copy()
        s.alive, s.t, s.exited = self.alive.copy(), self.t, self.exited
        s.period = None if self.period is None else self.period.copy()
        s.phase = None if self.phase is None else self.phase.copy()
        s.w = None if self.w is None else self.w.copy()
        s.h = None if self.h is None else self.h.copy()
        return s


def gate_periods(t: int, period, phase, choice):
    """Walk periods: pedestrians with t mod period != phase stay (choice 0).
    Returns the gated copy of choice."""
    choice = np.ascontiguousarray(choice, np.uint8).copy()
    if period is None:
        return choice
    period = np.ascontiguousarray(period, np.uint8)
    phase = np.ascontiguousarray(phase, np.uint8)
    lib().orc_gate_periods(int(t), choice.shape[0], _p(period), _p(phase), _p(choice))
    return choice


def step(m: Model, cell, D, st: State):
    """One tick of Alg. 1 on ``st`` in place; returns (choice, won)."""
    cell = np.ascontiguousarray(cell, np.uint8)
    D = np.ascontiguousarray(D, np.int32)
    n = st.xy.shape[0]
    occ = np.empty(m.W * m.H, np.int32)
    choice = np.zeros(max(n, 1), np.uint8)
    won = np.zeros(max(n, 1), np.uint8)
    per = None if st.period is None else np.ascontiguousarray(st.period, np.uint8)
    pha = None if st.phase is None else np.ascontiguousarray(st.phase, np.uint8)
    w = None if st.w is None else np.ascontiguousarray(st.w, np.uint8)
    h = None if st.h is None else np.ascontiguousarray(st.h, np.uint8)
    left = lib().orc_step(C.byref(m), _p(cell), _p(D), st.t, n, _p(st.xy), _p(st.heading),
                          _p(st.goal), _p(st.alive), _p(occ), _p(choice), _p(won), _p(per),
                          _p(pha), _p(w), _p(h))
    st.t += 1
    st.exited += int(left)
    return choice[:n], won[:n]
