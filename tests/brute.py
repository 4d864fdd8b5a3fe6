"""Independent brute-force checks for tiny lattices (test-only).

These routines re-derive the model's quantities by a different enumeration
than the oracle: the field loops over *sources* and takes minimum-image offsets
to every su at once (the oracle loops over each su's window); the guidance is
a Bellman-Ford relaxation to its fixed point (the oracle runs a bucket-queue
Dijkstra).  They are only practical for lattices of a few hundred su.
"""
import math

import numpy as np

DIRS = np.array([(0, 0), (1, 0), (1, 1), (0, 1), (-1, 1),
                 (-1, 0), (-1, -1), (0, -1), (1, -1)], dtype=np.int64)


def unit(k):
    if k == 0:
        return 0.0, 0.0
    dx, dy = DIRS[k]
    n = math.hypot(dx, dy)
    return dx / n, dy / n


def _offsets(W, H, px, py, sx, sy):
    X, Y = np.meshgrid(np.arange(W), np.arange(H))
    dx = X - sx
    dy = Y - sy
    if px:
        dx = (dx + W // 2) % W - W // 2
    if py:
        dy = (dy + H // 2) % H - H // 2
    return dx.astype(np.float64), dy.astype(np.float64)


def source_kernel(W, H, px, py, r, sx, sy, k, a, gamma=0.0, hcls=0):
    """Contribution of one source at (sx, sy) to every su (H x W array)."""
    dx, dy = _offsets(W, H, px, py, sx, sy)
    cheb = np.maximum(np.abs(dx), np.abs(dy))
    inside = (cheb > 0) & (cheb <= r)
    d = np.sqrt(dx * dx + dy * dy)
    dd = np.where(inside, d, 1.0)
    hx, hy = unit(hcls)
    val = k * dd ** a * (1.0 + gamma * (hx * dx + hy * dy) / dd)
    return np.where(inside, val, 0.0)


def field(scene, xy=None, heading=None, alive=None, parts=3, params=None):
    """All-pairs field (FP64) of a scene's sources; returns (F, S)."""
    p = dict(scene.params)
    if params:
        p.update(params)
    W, H, px, py, r = scene.W, scene.H, scene.periodic_x, scene.periodic_y, int(p["r"])
    xy = scene.xy if xy is None else xy
    heading = scene.heading if heading is None else heading
    F = np.zeros((H, W))
    S = np.zeros((H, W))
    if parts & 1:
        for (yy, xx) in zip(*np.nonzero(scene.cell == 1)):
            t = source_kernel(W, H, px, py, r, xx, yy, p["kO"], p["aO"])
            F += t
            S += np.abs(t)
        for (yy, xx) in zip(*np.nonzero(scene.cell == 2)):
            t = source_kernel(W, H, px, py, r, xx, yy, p["kE"], p["aE"])
            F += t
            S += np.abs(t)
    if parts & 2:
        for i in range(len(xy)):
            if alive is not None and not alive[i]:
                continue
            t = source_kernel(W, H, px, py, r, xy[i][0], xy[i][1], p["kP"], p["aP"],
                              p["gamma"], int(heading[i]))
            F += t
            S += np.abs(t)
    return F, S


def guidance(cell, px=0, py=0, dinf=1 << 23):
    """Chamfer (5, 7) geodesic distance by Bellman-Ford relaxation to the fixed point."""
    H, W = cell.shape
    D = np.where(cell == 2, 0, dinf).astype(np.int64)
    passable = cell != 1
    while True:
        best = D.copy()
        for k in range(1, 9):
            dx, dy = DIRS[k]
            w = 7 if (dx and dy) else 5
            # value arriving at c from neighbour c - (dx, dy)
            src = np.full((H, W), dinf, np.int64)
            ys = slice(max(0, dy), H + min(0, dy))
            yd = slice(max(0, -dy), H + min(0, -dy))
            xs = slice(max(0, dx), W + min(0, dx))
            xd = slice(max(0, -dx), W + min(0, -dx))
            if px:
                sh = np.roll(D, dx, axis=1)
            else:
                sh = np.full((H, W), dinf, np.int64)
                sh[:, xs] = D[:, xd]
            if py:
                sh = np.roll(sh, dy, axis=0)
            else:
                tmp = np.full((H, W), dinf, np.int64)
                tmp[ys, :] = sh[yd, :]
                sh = tmp
            src = np.where(sh < dinf, sh + w, dinf)
            best = np.minimum(best, src)
        best = np.where(passable, best, dinf)
        best = np.where(cell == 2, 0, best)
        if np.array_equal(best, D):
            return D.astype(np.int32)
        D = best
