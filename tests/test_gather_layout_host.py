"""Shared-memory reads of the row-trimmed field gather (CPU, no GPU).

The row-trimmed gather (csrc/sfm_field3.cu) reads a pedestrian's heading-
class table without any range test: lanes and rows outside the window must
land on zero entries of the padded layout, and every read must stay inside
the tables and the zero guard in front of them.  This test enumerates, for
radii on both sides of every stride class, every
pedestrian offset the record walk keeps, every heading class (4 stored
tables and their x / y mirrors), every lane and every row group the visit
reads, and checks that each address either holds the window entry K(dx, dy)
of the pedestrian's class or a zero of the padding, and that every row in
reach is read.  The layout constants restate those of the CUDA source:
32 x 32 su footprints (lane = column), blocks of 8 rows, 7 zero rows above
and below each window, row strides of at least 2r + 32 in three classes, a
32-float guard.
"""
import numpy as np
import pytest

PAD, GUARD, BLK = 7, 32, 8
# stored table (0 none, 1 E, 2 N, 3 NE) and x / y signs of heading classes 0..8
TAB = [0, 1, 3, 2, 3, 1, 3, 2, 3]
SX = [1, 1, 1, 1, -1, -1, -1, 1, 1]
SY = [1, 1, 1, 1, 1, 1, -1, -1, -1]
# heading class -> the move Delta_k whose direction it records
HDIR = [(0, 0), (1, 0), (1, 1), (0, 1), (-1, 1), (-1, 0), (-1, -1), (0, -1), (1, -1)]


def stride(r):
    if not 1 <= r <= 40:
        return 0
    for sp in (48, 80, 112):
        if sp >= 2 * r + 32:
            return sp
    return 0


def test_mirror_classes_reproduce_every_heading():
    """Table t read at (sx dx, sy dy) is the kernel of heading class c at
    (dx, dy): the heading of t mirrored by (sx, sy) is c's heading."""
    base = {0: (0, 0), 1: (1, 0), 2: (0, 1), 3: (1, 1)}
    for c in range(9):
        hx, hy = base[TAB[c]]
        assert (SX[c] * hx, SY[c] * hy) == HDIR[c], c


def test_every_radius_of_the_gather_has_a_stride_that_fits():
    for r in range(1, 41):
        sp = stride(r)
        assert sp >= 2 * r + 32 and sp % 4 == 0
        # guard, 4 tables and 32 warps x 32 int2 of record scratch in 227 KB
        assert (GUARD + 4 * (2 * r + 1 + 2 * PAD) * sp) * 4 + 32 * 32 * 8 <= 227 * 1024


@pytest.mark.parametrize("r", [1, 3, 8, 9, 24, 25, 40])
def test_every_read_is_in_bounds_and_holds_the_right_entry(r):
    FW = FH = 32
    SP = stride(r)
    TR = 2 * r + 1 + 2 * PAD
    TS = TR * SP
    NB = FH // BLK
    col = lane = np.arange(32)
    rsub = np.arange(8)[:, None] + 0 * lane[None, :]  # rows of block b: 8b + j, every lane
    rx = np.arange(-r, FW + r)                       # kept: within r columns of the footprint
    for ry in range(-r, FH + r):                     # kept: within r rows
        b0, b1 = max(0, ry - r) // BLK, min(FH - 1, ry + r) // BLK
        assert 0 <= b0 <= b1 < NB
        gs = np.arange(b0, b1 + 1)                   # blocks in reach (the mask)
        k = BLK * gs[:, None, None] + rsub[None]                          # [b, j, lane]
        want = np.arange(max(0, ry - r), min(FH - 1, ry + r) + 1)
        assert np.isin(want, k.ravel()).all()
        for cls in range(9):
            t, sx, sy = TAB[cls], SX[cls], SY[cls]
            A = t * TS + (PAD + r - sy * ry) * SP + r - sx * rx          # [rx]
            addr = (A[:, None, None, None] + sx * col[None, None, None, :]
                    + sy * k[None] * SP)                                 # [rx, b, j, lane]
            assert addr.min() >= -(GUARD - 1) and addr.max() < 4 * TS
            dx = col[None, None, None, :] - rx[:, None, None, None]
            dy = k[None] - ry
            inwin = (np.abs(dx) <= r) & (np.abs(dy) <= r)
            a = np.where(addr >= 0, addr, 0)
            tt, rem = a // TS, a % TS
            row, cc = rem // SP, rem % SP
            zero_entry = (addr < 0) | (row < PAD) | (row > PAD + 2 * r) | (cc > 2 * r)
            ok_in = (tt == t) & (row == PAD + r + sy * dy) & (cc == r + sx * dx)
            assert np.all(np.where(inwin, ok_in, zero_entry)), (r, ry, cls)
