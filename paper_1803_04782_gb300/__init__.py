"""Python binding of libsfm (include/sfm.h): argument marshalling only.

Every entry point of the C ABI is exposed under the same name (``sfm_create``,
``sfm_place``, ``sfm_step``, ...); arrays may be NumPy arrays (host memory) or
torch tensors (host or CUDA memory; the device pointer is passed through).
All computation happens in the CUDA kernels of ``csrc/``; if the shared
library is missing this module raises instead of falling back to anything.

``Sim`` is a small convenience wrapper around one context.
"""
from __future__ import annotations

import ctypes as C
import os
from typing import Optional

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_build", "libsfm.so")
_lib = None

SFM_OK, SFM_EINVAL, SFM_ENOMEM, SFM_EBUDGET, SFM_ECUDA, SFM_ECONFLICT, SFM_ETIMEOUT, SFM_ESTATE = range(8)
STATUS_NAMES = ["SFM_OK", "SFM_EINVAL", "SFM_ENOMEM", "SFM_EBUDGET", "SFM_ECUDA",
                "SFM_ECONFLICT", "SFM_ETIMEOUT", "SFM_ESTATE"]
SFM_MAX_RADIUS = 64
SFM_NSTAGES = 6
STAGES = ["bin", "field", "decide", "vote", "commit", "step"]

# Exported symbols (kept in step with include/sfm.h; checked by the tests).
EXPORTS = [
    "sfm_abi_version", "sfm_resident_bytes", "sfm_create", "sfm_destroy", "sfm_last_error", "sfm_place",
    "sfm_set_time", "sfm_step", "sfm_compute_field", "sfm_sync", "sfm_read_field",
    "sfm_compute_field_into", "sfm_read_static_field", "sfm_read_guidance", "sfm_read_peds",
    "sfm_read_decisions", "sfm_stats", "sfm_set_timing", "sfm_stage_times",
    "sfm_autotune", "sfm_set_field_footprint", "sfm_set_binning", "sfm_set_walk_periods",
    "sfm_place_sized", "sfm_snapshot", "sfm_restore", "sfm_set_ids", "sfm_set_guidance", "sfm_field_noalloc", "sfm_batch_create", "sfm_batch_place", "sfm_batch_offsets",
    "sfm_batch_autotune", "sfm_batch_test_missing_ctas", "sfm_surrogate_nparams",
    "sfm_surrogate_create", "sfm_surrogate_destroy", "sfm_surrogate_last_error",
    "sfm_surrogate_set_params", "sfm_surrogate_get_params", "sfm_surrogate_grad",
    "sfm_surrogate_forward",
    "sfm_surrogate_train", "sfm_surrogate_field", "sfm_surrogate_eval", "sfm_surrogate_set_delta",
    "sfm_surrogate_calibrate", "sfm_surrogate_step", "sfm_surrogate_counts",
    "sfm_surrogate_test_stop_copies",
]


class SfmError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{STATUS_NAMES[status] if 0 <= status < 8 else status}: {msg}")
        self.status = status


class Lattice(C.Structure):
    _fields_ = [("W", C.c_int32), ("H", C.c_int32), ("periodic_x", C.c_int32),
                ("periodic_y", C.c_int32)]


class Params(C.Structure):
    _fields_ = [("r", C.c_int32), ("bin", C.c_int32), ("kP", C.c_float), ("aP", C.c_float),
                ("gamma", C.c_float), ("kO", C.c_float), ("aO", C.c_float), ("kE", C.c_float),
                ("aE", C.c_float), ("beta", C.c_float), ("seed", C.c_uint64),
                ("hbm_budget_bytes", C.c_uint64)]


class Stats(C.Structure):
    _fields_ = [("t", C.c_int64), ("n", C.c_int64), ("alive", C.c_int64), ("exited", C.c_int64),
                ("moved_total", C.c_int64), ("max_registrants", C.c_int32),
                ("bands", C.c_int32), ("error_flags", C.c_uint32), ("pad_", C.c_int32),
                ("device_bytes", C.c_int64), ("kernel_launches", C.c_int64),
                ("decided", C.c_int64), ("near_ties", C.c_int64)]

    def as_dict(self):
        return {k: getattr(self, k) for k, _ in self._fields_ if k != "pad_"}


class SurrogateCfg(C.Structure):
    _fields_ = [("coarsen", C.c_int32), ("near_radius", C.c_int32), ("target_scale", C.c_float),
                ("lr", C.c_float), ("beta1", C.c_float), ("beta2", C.c_float), ("eps", C.c_float),
                ("taper_inner", C.c_float)]


class SurrogateReport(C.Structure):
    _fields_ = [("field_rel_err", C.c_double), ("flip_rate", C.c_double),
                ("flip_rate_raw", C.c_double), ("fallback_rate", C.c_double),
                ("ms_surrogate", C.c_double), ("ms_exact", C.c_double),
                ("ms_surrogate_field", C.c_double), ("delta", C.c_float), ("decided", C.c_int32)]


def lib():
    """Load the CUDA library (fails loudly when it has not been built)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError(f"{LIB_PATH} is missing: build it with "
                              "paper_1803_04782_gb300.build.build() (needs nvcc)")
        L = C.CDLL(LIB_PATH)
        P, I32, I64 = C.c_void_p, C.c_int32, C.c_int64
        sig = {
            "sfm_abi_version": (I32, []),
            "sfm_resident_bytes": (C.c_uint64, [C.POINTER(Lattice)]),
            "sfm_create": (C.c_int, [C.POINTER(Lattice), P, I32, C.POINTER(Params), P,
                                     C.POINTER(C.c_void_p)]),
            "sfm_destroy": (None, [P]),
            "sfm_last_error": (C.c_char_p, [P]),
            "sfm_place": (C.c_int, [P, I32, P, P, P, P, I32]),
            "sfm_set_time": (C.c_int, [P, I64]),
            "sfm_step": (C.c_int, [P, I32]),
            "sfm_compute_field": (C.c_int, [P]),
            "sfm_sync": (C.c_int, [P]),
            "sfm_read_field": (C.c_int, [P, P, I32]),
            "sfm_compute_field_into": (C.c_int, [P, P, I32]),
            "sfm_read_static_field": (C.c_int, [P, P, I32]),
            "sfm_read_guidance": (C.c_int, [P, P, I32]),
            "sfm_read_peds": (C.c_int, [P, P, P, P, I32]),
            "sfm_read_decisions": (C.c_int, [P, P, P, I32]),
            "sfm_stats": (C.c_int, [P, C.POINTER(Stats)]),
            "sfm_set_timing": (C.c_int, [P, I32]),
            "sfm_autotune": (C.c_int, [P, P]),
            "sfm_set_field_footprint": (C.c_int, [P, I32]),
            "sfm_set_binning": (C.c_int, [P, I32]),
            "sfm_set_walk_periods": (C.c_int, [P, P, P, I32]),
            "sfm_set_ids": (C.c_int, [P, P, I32]),
            "sfm_set_guidance": (C.c_int, [P, P, I32]),
            "sfm_place_sized": (C.c_int, [P, I32, P, P, P, P, P, P, I32]),
            "sfm_snapshot": (C.c_int, [P, P, C.POINTER(C.c_size_t)]),
            "sfm_restore": (C.c_int, [P, P, C.c_size_t]),
            "sfm_stage_times": (C.c_int, [P, C.POINTER(C.c_double), C.POINTER(C.c_int64)]),
            "sfm_field_noalloc": (C.c_int, [C.POINTER(Lattice), C.POINTER(Params), I32, P, P, P,
                                            P, P, P]),
            "sfm_batch_create": (C.c_int, [I32, C.POINTER(Lattice), C.POINTER(C.c_void_p),
                                           C.POINTER(Params), P, C.POINTER(C.c_void_p)]),
            "sfm_batch_place": (C.c_int, [P, P, P, P, P, P, I32]),
            "sfm_batch_offsets": (C.c_int, [P, P, P]),
            "sfm_batch_autotune": (C.c_int, [P, P]),
            "sfm_batch_test_missing_ctas": (C.c_int, [P, I32]),
            "sfm_surrogate_nparams": (I32, []),
            "sfm_surrogate_create": (C.c_int, [C.POINTER(SurrogateCfg), P, C.POINTER(C.c_void_p)]),
            "sfm_surrogate_destroy": (None, [P]),
            "sfm_surrogate_last_error": (C.c_char_p, [P]),
            "sfm_surrogate_set_params": (C.c_int, [P, P]),
            "sfm_surrogate_get_params": (C.c_int, [P, P]),
            "sfm_surrogate_grad": (C.c_int, [P, I32, I32, P, P, P, P]),
            "sfm_surrogate_train": (C.c_int, [P, P, I32, P]),
            "sfm_surrogate_field": (C.c_int, [P, P, P, I32]),
            "sfm_surrogate_eval": (C.c_int, [P, P, C.POINTER(SurrogateReport)]),
            "sfm_surrogate_forward": (C.c_int, [P, I32, I32, P, P, I32]),
            "sfm_surrogate_set_delta": (C.c_int, [P, C.c_float]),
            "sfm_surrogate_calibrate": (C.c_int, [P, P, C.c_double, P]),
            "sfm_surrogate_step": (C.c_int, [P, P, I32]),
            "sfm_surrogate_counts": (C.c_int, [P, P, P]),
            "sfm_surrogate_test_stop_copies": (C.c_int, [P, I32]),
        }
        for name, (res, args) in sig.items():
            f = getattr(L, name)
            f.restype = res
            f.argtypes = args
        _lib = L
    return _lib


def _ptr(a):
    """(pointer, on_device) of a NumPy array or torch tensor (None -> NULL)."""
    if a is None:
        return None, 0
    if isinstance(a, np.ndarray):
        if not a.flags.c_contiguous:
            raise ValueError("arrays must be C-contiguous")
        return a.ctypes.data_as(C.c_void_p), 0
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return C.c_void_p(a.data_ptr()), 1 if a.is_cuda else 0
    raise TypeError(type(a))


def _check(ctx, status):
    if status != SFM_OK:
        msg = lib().sfm_last_error(ctx)
        raise SfmError(status, msg.decode() if msg else "")


def _stream_handle(stream):
    if stream is None:
        return None
    if hasattr(stream, "cuda_stream"):
        return C.c_void_p(stream.cuda_stream)
    return C.c_void_p(int(stream))


# ---------------------------------------------------------------- C-ABI names
def sfm_abi_version() -> int:
    return lib().sfm_abi_version()


def sfm_resident_bytes(lat: Lattice) -> int:
    return int(lib().sfm_resident_bytes(C.byref(lat)))


# rows of the band buffer beyond a band's own (sfm_resident_bytes in sfm.h)
BAND_EXTRA_ROWS = 33


def band_budget(W: int, H: int, rows: int, periodic_x: int = 0, periodic_y: int = 0) -> int:
    """HBM budget that makes the field pass run in bands of ``rows`` rows."""
    lat = Lattice(int(W), int(H), int(periodic_x), int(periodic_y))
    return sfm_resident_bytes(lat) + 4 * int(W) * (int(rows) + BAND_EXTRA_ROWS)


def sfm_create(lat: Lattice, cell, prm: Params, stream=None):
    p, dev = _ptr(cell)
    out = C.c_void_p()
    st = lib().sfm_create(C.byref(lat), p, dev, C.byref(prm), _stream_handle(stream),
                          C.byref(out))
    if st != SFM_OK:
        msg = lib().sfm_last_error(None)
        raise SfmError(st, msg.decode() if msg else "")
    return out


def sfm_destroy(ctx) -> None:
    lib().sfm_destroy(ctx)


def sfm_last_error(ctx) -> str:
    m = lib().sfm_last_error(ctx)
    return m.decode() if m else ""


def sfm_place(ctx, xy, heading=None, goal=None, alive=None) -> None:
    n = int(xy.shape[0])
    pxy, dev = _ptr(xy)
    ph, _ = _ptr(heading)
    pg, _ = _ptr(goal)
    pa, _ = _ptr(alive)
    _check(ctx, lib().sfm_place(ctx, n, pxy, ph, pg, pa, dev))


def sfm_set_time(ctx, t: int) -> None:
    _check(ctx, lib().sfm_set_time(ctx, int(t)))


def sfm_step(ctx, nsteps: int = 1) -> None:
    _check(ctx, lib().sfm_step(ctx, int(nsteps)))


def sfm_compute_field(ctx) -> None:
    _check(ctx, lib().sfm_compute_field(ctx))


def sfm_sync(ctx) -> None:
    _check(ctx, lib().sfm_sync(ctx))


def sfm_read_field(ctx, dst) -> None:
    p, dev = _ptr(dst)
    _check(ctx, lib().sfm_read_field(ctx, p, dev))


def sfm_compute_field_into(ctx, dst) -> None:
    p, dev = _ptr(dst)
    _check(ctx, lib().sfm_compute_field_into(ctx, p, dev))


def sfm_read_static_field(ctx, dst) -> None:
    p, dev = _ptr(dst)
    _check(ctx, lib().sfm_read_static_field(ctx, p, dev))


def sfm_read_guidance(ctx, dst) -> None:
    p, dev = _ptr(dst)
    _check(ctx, lib().sfm_read_guidance(ctx, p, dev))


def sfm_read_peds(ctx, xy=None, heading=None, alive=None) -> None:
    devs = [_ptr(a) for a in (xy, heading, alive)]
    on_dev = max(d for _, d in devs)
    _check(ctx, lib().sfm_read_peds(ctx, devs[0][0], devs[1][0], devs[2][0], on_dev))


def sfm_read_decisions(ctx, choice=None, won=None) -> None:
    devs = [_ptr(a) for a in (choice, won)]
    on_dev = max(d for _, d in devs)
    _check(ctx, lib().sfm_read_decisions(ctx, devs[0][0], devs[1][0], on_dev))


def sfm_stats(ctx) -> dict:
    s = Stats()
    _check(ctx, lib().sfm_stats(ctx, C.byref(s)))
    return s.as_dict()


# sfm_set_field_footprint shapes 0..2; "r": the row-trimmed gather
FOOTPRINTS = ("16x16", "32x16", "32x32r")


def sfm_autotune(ctx) -> str:
    """Pick the fastest warp footprint of the field gather for this context."""
    v = C.c_int32()
    _check(ctx, lib().sfm_autotune(ctx, C.byref(v)))
    return FOOTPRINTS[v.value]


def sfm_set_timing(ctx, every) -> None:
    """every: False / 0 off, True / 1 every tick, k > 1 every k-th tick."""
    _check(ctx, lib().sfm_set_timing(ctx, int(every)))


def sfm_stage_times(ctx):
    ms = (C.c_double * SFM_NSTAGES)()
    ticks = C.c_int64()
    _check(ctx, lib().sfm_stage_times(ctx, ms, C.byref(ticks)))
    return dict(zip(STAGES, list(ms))), int(ticks.value)


def sfm_batch_create(lats, cells, prms, stream=None):
    n = len(lats)
    L = (Lattice * n)(*lats)
    P = (Params * n)(*prms)
    keep = [np.ascontiguousarray(c, np.uint8) for c in cells]
    ptrs = (C.c_void_p * n)(*[k.ctypes.data_as(C.c_void_p) for k in keep])
    out = C.c_void_p()
    st = lib().sfm_batch_create(n, L, ptrs, P, _stream_handle(stream), C.byref(out))
    if st != SFM_OK:
        msg = lib().sfm_last_error(None)
        raise SfmError(st, msg.decode() if msg else "")
    return out


def sfm_batch_place(ctx, counts, xy, heading=None, goal=None, alive=None) -> None:
    counts = np.ascontiguousarray(counts, np.int32)
    pxy, dev = _ptr(xy)
    _check(ctx, lib().sfm_batch_place(ctx, counts.ctypes.data_as(C.c_void_p), pxy,
                                      _ptr(heading)[0], _ptr(goal)[0], _ptr(alive)[0], dev))


def sfm_batch_offsets(ctx, nscenes: int):
    su = np.zeros(nscenes + 1, np.int64)
    pe = np.zeros(nscenes + 1, np.int64)
    _check(ctx, lib().sfm_batch_offsets(ctx, su.ctypes.data_as(C.c_void_p),
                                        pe.ctypes.data_as(C.c_void_p)))
    return su, pe


TABLE_STRIDES = (34, 50, 66, 82, 98, 114, 102)  # class-table row stride per radius class


def sfm_batch_autotune(ctx):
    """Footprint chosen per radius class, keyed by the class-table row stride
    (34, 50, ..., 114 for radius <= 1, 9, ..., 41; 102 for radius 42..50):
    "16x16" or "32x16"."""
    shp = np.zeros(len(TABLE_STRIDES), np.int32)
    _check(ctx, lib().sfm_batch_autotune(ctx, shp.ctypes.data_as(C.c_void_p)))
    return {sp: ("32x16" if v else "16x16") for sp, v in zip(TABLE_STRIDES, shp)}


def sfm_batch_test_missing_ctas(ctx, missing: int) -> None:
    _check(ctx, lib().sfm_batch_test_missing_ctas(ctx, int(missing)))


SFM_NOALLOC_MAX_PEDS = 1 << 20
SFM_NOALLOC_MAX_BINS = 1 << 16
SFM_NOALLOC_MAX_RADIUS = 47


def sfm_field_noalloc(lat: Lattice, prm: Params, xy, heading, alive, base, field,
                      stream=None) -> int:
    """Field superposition into ``field`` (device) without any device
    allocation; returns the sfm_status code (0 = SFM_OK).  For callers that
    cannot allocate device memory while they run; see include/sfm.h.

    Every array must be a contiguous CUDA tensor: xy int32 of shape (n, 2),
    heading and alive uint8 of n elements (or None), base and field float32
    of W*H elements each.  Anything else raises ValueError before the C call
    (the C function takes bare device pointers and cannot check them)."""
    W, H = int(lat.W), int(lat.H)

    def dev_tensor(name, a, dtype, numel=None, shape=None):
        if a is None:
            return None
        if not hasattr(a, "data_ptr") or not getattr(a, "is_cuda", False):
            raise ValueError(f"sfm_field_noalloc: {name} must be a CUDA tensor")
        if str(a.dtype) != f"torch.{dtype}":
            raise ValueError(f"sfm_field_noalloc: {name} must be {dtype}, got {a.dtype}")
        if not a.is_contiguous():
            raise ValueError(f"sfm_field_noalloc: {name} must be contiguous")
        if shape is not None and tuple(a.shape) != shape:
            raise ValueError(f"sfm_field_noalloc: {name} must have shape {shape}, got "
                             f"{tuple(a.shape)}")
        if numel is not None and a.numel() != numel:
            raise ValueError(f"sfm_field_noalloc: {name} must hold {numel} elements, got "
                             f"{a.numel()}")
        return C.c_void_p(a.data_ptr())

    if xy is None or base is None or field is None:
        raise ValueError("sfm_field_noalloc: xy, base and field are required")
    n = int(xy.shape[0]) if len(xy.shape) else -1
    pxy = dev_tensor("xy", xy, "int32", shape=(n, 2))
    ph = dev_tensor("heading", heading, "uint8", numel=n)
    pa = dev_tensor("alive", alive, "uint8", numel=n)
    pb = dev_tensor("base", base, "float32", numel=W * H)
    pf = dev_tensor("field", field, "float32", numel=W * H)
    return int(lib().sfm_field_noalloc(C.byref(lat), C.byref(prm), n, pxy, ph, pa, pb, pf,
                                       _stream_handle(stream)))


# ------------------------------------------------------------------ wrapper
def make_params(r=3, kP=1.0, aP=-0.5, gamma=0.5, kO=1.0, aO=-0.5, kE=-1.0, aE=-0.5, beta=1.0,
                seed=0, hbm_budget_bytes=0, bin=0) -> Params:
    return Params(int(r), int(bin), kP, aP, gamma, kO, aO, kE, aE, beta, int(seed) & (2**64 - 1),
                  int(hbm_budget_bytes))


class Sim:
    """One simulation context.  ``scene`` is any object with W, H, periodic_x,
    periodic_y, cell, xy, heading, goal and params attributes (for example a
    ``scenegen.Scene``); keyword arguments override its parameters."""

    def __init__(self, scene=None, *, W=None, H=None, cell=None, periodic_x=0, periodic_y=0,
                 stream=None, place=True, **params):
        if scene is not None:
            W, H, cell = scene.W, scene.H, scene.cell
            periodic_x, periodic_y = scene.periodic_x, scene.periodic_y
            p = {k: v for k, v in scene.params.items()}
            p.update(params)
        else:
            p = dict(params)
        self.W, self.H = int(W), int(H)
        self.lat = Lattice(self.W, self.H, int(periodic_x), int(periodic_y))
        self.prm = make_params(**p)
        cell = np.ascontiguousarray(cell, np.uint8) if isinstance(cell, np.ndarray) else cell
        self.ctx = sfm_create(self.lat, cell, self.prm, stream)
        self.n = 0
        if scene is not None and place:
            self.place(scene.xy, scene.heading, scene.goal)

    def close(self):
        if getattr(self, "ctx", None):
            sfm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    # state
    def place(self, xy, heading=None, goal=None, alive=None):
        if isinstance(xy, np.ndarray):
            xy = np.ascontiguousarray(xy, np.int32)
            heading = None if heading is None else np.ascontiguousarray(heading, np.uint8)
            goal = None if goal is None else np.ascontiguousarray(goal, np.uint8)
            alive = None if alive is None else np.ascontiguousarray(alive, np.uint8)
        sfm_place(self.ctx, xy, heading, goal, alive)
        self.n = int(xy.shape[0])

    def set_time(self, t):
        sfm_set_time(self.ctx, t)

    def step(self, n=1):
        sfm_step(self.ctx, n)

    def sync(self):
        sfm_sync(self.ctx)

    def compute_field(self):
        sfm_compute_field(self.ctx)

    # reads (host NumPy)
    def field(self):
        out = np.empty((self.H, self.W), np.float32)
        sfm_read_field(self.ctx, out)
        return out

    def field_banded(self):
        out = np.empty((self.H, self.W), np.float32)
        sfm_compute_field_into(self.ctx, out)
        return out

    def static_field(self):
        out = np.empty((self.H, self.W), np.float32)
        sfm_read_static_field(self.ctx, out)
        return out

    def guidance(self):
        out = np.empty((self.H, self.W), np.int32)
        sfm_read_guidance(self.ctx, out)
        return out

    def peds(self):
        xy = np.empty((self.n, 2), np.int32)
        h = np.empty(self.n, np.uint8)
        a = np.empty(self.n, np.uint8)
        sfm_read_peds(self.ctx, xy, h, a)
        return xy, h, a

    def decisions(self):
        ch = np.empty(self.n, np.uint8)
        won = np.empty(self.n, np.uint8)
        sfm_read_decisions(self.ctx, ch, won)
        return ch, won

    def stats(self):
        return sfm_stats(self.ctx)

    def autotune(self):
        return sfm_autotune(self.ctx)

    def snapshot(self) -> bytes:
        """The context's dynamic state as bytes (see sfm_snapshot)."""
        n = C.c_size_t(0)
        _check(self.ctx, lib().sfm_snapshot(self.ctx, None, C.byref(n)))
        buf = C.create_string_buffer(n.value)
        _check(self.ctx, lib().sfm_snapshot(self.ctx, buf, C.byref(n)))
        return buf.raw[:n.value]

    def restore(self, snap: bytes):
        """Continue from a snapshot of a context on the same lattice."""
        buf = C.create_string_buffer(bytes(snap), len(snap))
        _check(self.ctx, lib().sfm_restore(self.ctx, buf, len(snap)))
        self.n = int(np.frombuffer(bytes(snap)[56:64], np.int64)[0])  # header field n

    def place_sized(self, xy, heading, goal, alive, width, height):
        """Place multi-su pedestrians (odd width x height rectangles)."""
        keep = [np.ascontiguousarray(xy, np.int32), np.ascontiguousarray(heading, np.uint8),
                np.ascontiguousarray(goal, np.uint8), np.ascontiguousarray(alive, np.uint8),
                np.ascontiguousarray(width, np.uint8), np.ascontiguousarray(height, np.uint8)]
        self.n = int(keep[0].shape[0])
        _check(self.ctx, lib().sfm_place_sized(self.ctx, self.n,
                                               *[k.ctypes.data_as(C.c_void_p) for k in keep], 0))

    def set_walk_periods(self, period=None, phase=None):
        """Walk periods: pedestrian p moves only on ticks t with t % period[p]
        == phase[p]; None switches them off.  Reset by every placement."""
        if period is None:
            _check(self.ctx, lib().sfm_set_walk_periods(self.ctx, None, None, 0))
            return
        self._period = np.ascontiguousarray(period, np.uint8)
        self._phase = np.ascontiguousarray(phase, np.uint8)
        _check(self.ctx, lib().sfm_set_walk_periods(
            self.ctx, self._period.ctypes.data_as(C.c_void_p),
            self._phase.ctypes.data_as(C.c_void_p), 0))

    def set_ids(self, ids=None):
        """The pedestrians' numbers for the election (sfm_set_ids); None: the
        indices.  Reset by every placement."""
        if ids is None:
            _check(self.ctx, lib().sfm_set_ids(self.ctx, None, 0))
            return
        ids = np.ascontiguousarray(ids, np.int32)
        _check(self.ctx, lib().sfm_set_ids(self.ctx, ids.ctypes.data_as(C.c_void_p), 0))

    def set_guidance(self, D):
        """Replace the guidance distances (sfm_set_guidance), H x W int32."""
        D = np.ascontiguousarray(D, np.int32)
        assert D.size == self.W * self.H
        _check(self.ctx, lib().sfm_set_guidance(self.ctx, D.ctypes.data_as(C.c_void_p), 0))

    def set_binning(self, mode: str):
        """"auto", "grid" (scan the class grid) or "peds" (from the pedestrian list)."""
        _check(self.ctx, lib().sfm_set_binning(self.ctx, {"auto": 0, "grid": 1, "peds": 2}[mode]))

    def set_footprint(self, shape: str):
        _check(self.ctx, lib().sfm_set_field_footprint(self.ctx, FOOTPRINTS.index(shape)))

    def set_timing(self, every=True):
        """Stage events on every ``every``-th tick (True: every tick; False: off)."""
        sfm_set_timing(self.ctx, every)

    def stage_times(self):
        return sfm_stage_times(self.ctx)


class Batch:
    """A batch of independent scenes stepped by one persistent launch per tick.
    ``scenes``: objects with the attributes ``Sim`` accepts."""

    def __init__(self, scenes, stream=None, place=True):
        self.scenes = list(scenes)
        lats = [Lattice(s.W, s.H, s.periodic_x, s.periodic_y) for s in self.scenes]
        prms = [make_params(**s.params) for s in self.scenes]
        self.ctx = sfm_batch_create(lats, [s.cell for s in self.scenes], prms, stream)
        self.su_off = self.ped_off = None
        if place:
            self.place([s.xy for s in self.scenes], [s.heading for s in self.scenes],
                       [s.goal for s in self.scenes])

    def close(self):
        if getattr(self, "ctx", None):
            sfm_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def place(self, xys, headings=None, goals=None, alives=None):
        counts = [len(x) for x in xys]
        cat = lambda arrs, dt: (None if arrs is None else
                                np.ascontiguousarray(np.concatenate(arrs), dt))
        xy = np.ascontiguousarray(np.concatenate(xys).reshape(-1, 2), np.int32)
        sfm_batch_place(self.ctx, counts, xy, cat(headings, np.uint8), cat(goals, np.uint8),
                        cat(alives, np.uint8))
        self.su_off, self.ped_off = sfm_batch_offsets(self.ctx, len(self.scenes))

    def step(self, n=1):
        sfm_step(self.ctx, n)

    def sync(self):
        sfm_sync(self.ctx)

    def compute_field(self):
        sfm_compute_field(self.ctx)

    def autotune(self):
        return sfm_batch_autotune(self.ctx)

    def _split(self, flat, off, shape=None):
        out = []
        for i, s in enumerate(self.scenes):
            part = flat[off[i]:off[i + 1]]
            out.append(part.reshape(s.H, s.W) if shape == "lattice" else part)
        return out

    def fields(self):
        out = np.empty(int(self.su_off[-1]), np.float32)
        sfm_read_field(self.ctx, out)
        return self._split(out, self.su_off, "lattice")

    def static_fields(self):
        out = np.empty(int(self.su_off[-1]), np.float32)
        sfm_read_static_field(self.ctx, out)
        return self._split(out, self.su_off, "lattice")

    def guidance(self):
        out = np.empty(int(self.su_off[-1]), np.int32)
        sfm_read_guidance(self.ctx, out)
        return self._split(out, self.su_off, "lattice")

    def peds(self):
        n = int(self.ped_off[-1])
        xy = np.empty((n, 2), np.int32)
        h = np.empty(n, np.uint8)
        a = np.empty(n, np.uint8)
        sfm_read_peds(self.ctx, xy, h, a)
        return (self._split(xy, self.ped_off), self._split(h, self.ped_off),
                self._split(a, self.ped_off))

    def decisions(self):
        n = int(self.ped_off[-1])
        ch = np.empty(n, np.uint8)
        won = np.empty(n, np.uint8)
        sfm_read_decisions(self.ctx, ch, won)
        return self._split(ch, self.ped_off), self._split(won, self.ped_off)

    def stats(self):
        return sfm_stats(self.ctx)

    def set_timing(self, every=True):
        """Stage events on every ``every``-th tick (True: every tick; False: off)."""
        sfm_set_timing(self.ctx, every)

    def stage_times(self):
        return sfm_stage_times(self.ctx)


# ------------------------------------------------------------ surrogate
def _scheck(sur, status):
    if status != SFM_OK:
        m = lib().sfm_surrogate_last_error(sur)
        raise SfmError(status, m.decode() if m else "")


class Surrogate:
    """Learned field surrogate (see include/sfm.h): exact near field plus a
    BF16 convolutional far field on an s-times coarsened grid."""

    def __init__(self, coarsen=8, near_radius=3, target_scale=20.0, lr=1e-3, beta1=0.9,
                 beta2=0.999, eps=1e-8, stream=None, params=None, taper_inner=None):
        ti = float(near_radius) if taper_inner is None else float(taper_inner)
        self.cfg = SurrogateCfg(int(coarsen), int(near_radius), target_scale, lr, beta1, beta2,
                                eps, ti)
        out = C.c_void_p()
        st = lib().sfm_surrogate_create(C.byref(self.cfg), _stream_handle(stream), C.byref(out))
        if st != SFM_OK:
            m = lib().sfm_last_error(None)
            raise SfmError(st, m.decode() if m else "")
        self.h = out
        self.nparams = int(lib().sfm_surrogate_nparams())
        if params is not None:
            self.set_params(params)

    def close(self):
        if getattr(self, "h", None):
            lib().sfm_surrogate_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def set_params(self, flat):
        flat = np.ascontiguousarray(flat, np.float32)
        assert flat.size == self.nparams
        _scheck(self.h, lib().sfm_surrogate_set_params(self.h, flat.ctypes.data_as(C.c_void_p)))

    def get_params(self):
        out = np.empty(self.nparams, np.float32)
        _scheck(self.h, lib().sfm_surrogate_get_params(self.h, out.ctypes.data_as(C.c_void_p)))
        return out

    def grad(self, X, T):
        X = np.ascontiguousarray(X, np.float32)
        T = np.ascontiguousarray(T, np.float32)
        loss = C.c_float()
        g = np.empty(self.nparams, np.float32)
        _scheck(self.h, lib().sfm_surrogate_grad(self.h, X.shape[1], X.shape[2],
                                                 X.ctypes.data_as(C.c_void_p),
                                                 T.ctypes.data_as(C.c_void_p), C.byref(loss),
                                                 g.ctypes.data_as(C.c_void_p)))
        return float(loss.value), g

    def forward(self, X, tcgen05=True):
        """The network's output for a channel-planar input X [3][Hin][Win]
        (rounded to BF16), with the 3x3 32 -> 32 layers on the tcgen05 kernel
        the surrogate's ticks use, or (tcgen05=False) on the mma.sync kernel."""
        X = np.ascontiguousarray(X, np.float32)
        Y = np.empty((X.shape[1] - 10, X.shape[2] - 10), np.float32)
        _scheck(self.h, lib().sfm_surrogate_forward(self.h, X.shape[1], X.shape[2],
                                                    X.ctypes.data_as(C.c_void_p),
                                                    Y.ctypes.data_as(C.c_void_p), int(bool(tcgen05))))
        return Y

    def train(self, sim, iters):
        curve = np.zeros(int(iters), np.float32)
        _scheck(self.h, lib().sfm_surrogate_train(self.h, sim.ctx, int(iters),
                                                  curve.ctypes.data_as(C.c_void_p)))
        return curve

    def field(self, sim):
        out = np.empty((sim.H, sim.W), np.float32)
        _scheck(self.h, lib().sfm_surrogate_field(self.h, sim.ctx, out.ctypes.data_as(C.c_void_p), 0))
        return out

    def eval(self, sim):
        """Surrogate against the exact path on sim's current state (see
        sfm_surrogate_eval): field error, flip rates with and without the
        exact fallback, fallback rate, the time of each and delta."""
        r = SurrogateReport()
        _scheck(self.h, lib().sfm_surrogate_eval(self.h, sim.ctx, C.byref(r)))
        return {k: getattr(r, k) for k, _ in SurrogateReport._fields_}

    def set_delta(self, delta):
        _scheck(self.h, lib().sfm_surrogate_set_delta(self.h, float(delta)))

    def calibrate(self, sim, quantile=0.999):
        """Set delta to a quantile of the per-pedestrian candidate field error."""
        d = C.c_float()
        _scheck(self.h, lib().sfm_surrogate_calibrate(self.h, sim.ctx, float(quantile), C.byref(d)))
        return float(d.value)

    def step(self, sim, nsteps=1):
        """nsteps ticks of sim with the surrogate field and the exact fallback."""
        _scheck(self.h, lib().sfm_surrogate_step(self.h, sim.ctx, int(nsteps)))

    def test_stop_copies(self, after):
        """Test hook: the next tcgen05 layer-2 launch stops issuing copies
        after `after` tiles per CTA, so its bounded waits run out."""
        _scheck(self.h, lib().sfm_surrogate_test_stop_copies(self.h, int(after)))

    def counts(self):
        fb, dec = C.c_int64(), C.c_int64()
        _scheck(self.h, lib().sfm_surrogate_counts(self.h, C.byref(fb), C.byref(dec)))
        return int(fb.value), int(dec.value)


def flatten_params(params):
    """Public flat order W1 b1 ... W4 b4 from [(W [out,in,k,k], b [out]), ...]."""
    return np.concatenate([np.concatenate([np.asarray(W, np.float64).ravel(),
                                           np.asarray(b, np.float64).ravel()])
                           for W, b in params]).astype(np.float32)


def unflatten_params(flat, layers=((3, 32, 5), (32, 32, 3), (32, 32, 3), (32, 1, 3))):
    out, off = [], 0
    for cin, cout, k in layers:
        nw = cout * cin * k * k
        W = np.asarray(flat[off:off + nw], np.float64).reshape(cout, cin, k, k)
        off += nw
        b = np.asarray(flat[off:off + cout], np.float64)
        off += cout
        out.append((W, b))
    return out
