"""Host-side arithmetic of bench.py (CPU).

The roofline's achieved throughput divides the algorithmic work by the
gather's time; the work is the number of (su, pedestrian-in-window) pairs,
which bench.py counts from the clipped window of every live pedestrian.
Here that count is checked against a brute-force count over every su on
small closed, periodic and thin-torus lattices, with dead pedestrians.
"""
import numpy as np
import pytest

import bench
import scenegen as SG


def _brute_pairs(sc, xy, alive):
    r = int(sc.params["r"])
    ys, xs = np.mgrid[0:sc.H, 0:sc.W]
    n = 0
    for p in np.flatnonzero(alive):
        dx = xs - xy[p, 0]
        dy = ys - xy[p, 1]
        if sc.periodic_x:
            dx = (dx + sc.W // 2) % sc.W - sc.W // 2
        if sc.periodic_y:
            dy = (dy + sc.H // 2) % sc.H - sc.H // 2
        cheb = np.maximum(np.abs(dx), np.abs(dy))
        n += int(((cheb > 0) & (cheb <= r)).sum())
    return n


@pytest.mark.parametrize("kw", [
    dict(W=37, H=29, n=60, r=5, seed=1),
    dict(W=40, H=33, n=80, r=7, seed=2, periodic_x=1, exits=()),
    dict(W=30, H=30, n=70, r=4, seed=3, periodic_x=1, periodic_y=1, ring=False, exits=()),
    dict(W=11, H=50, n=40, r=5, seed=4, periodic_x=1, exits=("south",)),  # extent 2r + 1
    dict(W=20, H=16, n=30, r=12, seed=5),                                  # window wider than the lattice
])
def test_pair_count_equals_brute_force(kw):
    kw = dict(kw)
    W, H, n, r, seed = kw.pop("W"), kw.pop("H"), kw.pop("n"), kw.pop("r"), kw.pop("seed")
    sc = SG.random_scene(W, H, n, r=r, seed=seed, **kw)
    alive = np.ones(sc.n, np.uint8)
    alive[::7] = 0
    assert bench.pair_count(sc, sc.xy, alive) == _brute_pairs(sc, sc.xy, alive)


def test_default_bands_and_band_budget():
    assert bench.default_bands("floor") == 4 and bench.default_bands("floor-small") == 4
    assert bench.default_bands("corridor") == 1 and bench.default_bands("room") == 1
    sc = SG.room()
    assert bench.band_budget(sc, 1) == 0
    b4, b2 = bench.band_budget(sc, 4), bench.band_budget(sc, 2)
    assert 0 < b4 <= b2  # more bands: smaller band buffers, a smaller budget
