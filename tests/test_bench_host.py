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


def test_gather_roofline_arithmetic():
    """One table word per pair against 32 words per clock per SM; the
    algorithmic FP32 figure is 6 flops per pair, the executed one 1."""
    r = bench.gather_roofline(pairs=1.0e9, field_s=1e-3, nsm=100, mhz=2000.0, mhz_src="test",
                              kernel="k")
    assert r["bound"] == "smem"
    assert abs(r["achieved"] - 1.0) < 1e-12                 # 1e12 words/s
    assert abs(r["peak"] - 100 * 32 * 2000e6 / 1e12) < 1e-12
    assert abs(r["frac"] - 1e12 / (100 * 32 * 2e9)) < 1e-12
    a = r["algorithmic_fp32"]
    assert abs(a["achieved_tflops"] - 6.0) < 1e-12
    assert abs(a["frac"] - 6e12 / (100 * 128 * 2 * 2e9)) < 1e-12
    assert abs(r["fp32_executed"]["frac"] - a["frac"] / 6) < 1e-15


def test_reference_arm_reports_the_time_it_spent_and_the_same_config(capsys):
    """The oracle arm's ms_per_step is time actually spent on its sampled
    steps (it fits in the wall time of the run) and its config equals the
    one the GPU arm prints for the same workload."""
    import argparse
    import json
    import time

    args = argparse.Namespace(workload="room", steps=2, warmup=3, ref_sample=50, gpus=1,
                              bands=None)
    t0 = time.perf_counter()
    assert bench.run_reference(args) == 0
    wall = time.perf_counter() - t0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    assert line["impl"] == "reference"
    assert line["ms_per_step"] * args.steps / 1e3 <= wall
    cb = line["cpu_baseline"]
    assert cb["seconds_timed"] <= wall
    assert abs(line["value"] - 50 * args.steps / cb["seconds_timed"]) < 1e-6 * line["value"]
    sc, desc = bench.workload("room")
    assert line["config"] == bench.workload_config(args, sc, desc)


def test_clock_samples_are_kept_inside_the_timed_region(tmp_path):
    """The clock record keeps the nvidia-smi samples stamped inside the timed
    region (with 50 ms of slack), and falls back to all samples, saying so,
    when none lies inside."""
    import datetime
    base = datetime.datetime(2026, 1, 2, 3, 4, 5)

    def line(dt_ms, mhz, reason="Not Active"):
        ts = (base + datetime.timedelta(milliseconds=dt_ms)).strftime("%Y/%m/%d %H:%M:%S.%f")[:-3]
        return (f"{ts}, 0, GPU-abc, {mhz}, 2070, 300.0, 0x0, {reason}, Not Active, "
                f"Not Active, Not Active\n")

    t0 = base.timestamp()
    c = bench.Clocks("GPU-abc")
    c.path = str(tmp_path / "c.csv")
    with open(c.path, "w") as f:
        f.write(line(0, 900) + line(200, 2070) + line(300, 2070, "Active") + line(400, 2070)
                + line(900, 1000))

    class Done:
        def terminate(self):
            pass

        def wait(self, timeout=None):
            return 0

    c.proc = Done()
    c.t0, c.t1 = t0 + 0.15, t0 + 0.45
    out = c.stop()
    assert out["samples"] == 3 and out["window"] == "timed region"
    assert out["sm_mhz"] == 2070.0 and out["reasons"] == ["hw_slowdown"]
    c.path = str(tmp_path / "d.csv")
    with open(c.path, "w") as f:
        f.write(line(0, 900) + line(900, 1000))
    out = c.stop()
    assert out["samples"] == 2 and out["window"].startswith("whole sampling")


def test_timed_region_chunks_and_their_median():
    assert bench.chunk_sizes(400, 5) == [80] * 5
    assert bench.chunk_sizes(23, 5) == [5, 5, 5, 4, 4]
    assert bench.chunk_sizes(3, 5) == [1, 1, 1]
    r = bench.repeat_record([2, 2, 1], [4.0, 5.0, 1.5])
    assert r["ms_per_step"] == [2.0, 2.5, 1.5] and r["median_ms_per_step"] == 2.0
    assert abs(r["spread"] - 0.5) < 1e-12 and r["n"] == 3
