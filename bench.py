#!/usr/bin/env python3
"""Benchmark of the social-field pedestrian step on GB300.

Default workload: the 16384 x 16384 floor (10 % rectangular obstacles, 4 exits
of 256 su, 10^6 pedestrians, influence radius 40) with the divide-and-conquer
row bands engaged (HBM budget set so that the field is computed in >= 4
bands).  One "step" is one tick of the whole path: bins, field gather,
decision, vote, commit.

Prints ONE JSON line (rank 0).  ``--impl reference`` times the FP64 CPU oracle
instead, on bounded samples of the same workload.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

MEASURED_PEAKS = os.path.join(ROOT, "MEASURED_PEAKS.json")
FP32_LANES = 128      # FP32 lanes per SM (Blackwell)
SMEM_WORDS = 32       # shared-memory banks per SM: one 4-byte word each per clock
NOMINAL_SM_MHZ = 2070.0
# algorithmic work of one (su, pedestrian-in-window) pair in the 3-channel
# kernel-table formulation: three FP32 multiply-adds; the class-table gather
# executes one FP32 add per pair instead
FLOPS_PER_PAIR = 6.0
# stage events on every 9th tick of the timed region: an event record costs a
# few microseconds of GPU time (the stream drains before it), so recording all
# stages of every tick would add about 7 % to a floor tick; the 8 ticks in
# between fill one untimed 8-tick graph
TIMING_EVERY = 9
# DRAM bytes (read + write) per banded launch of the field gather on the
# 16384^2 floor with 4 bands, from a one-pass ncu capture of this benchmark
# (dram__bytes_read.sum + dram__bytes_write.sum); valid only while the
# gather's sources hash to the value they had when it was taken.
GATHER_TRAFFIC = {"sha1": "448dec8a766d3e7d1ab154ddb47feea4c66ca156", "bands": 4,
                  "footprint": "32x32r", "workload": "floor", "bytes_per_launch": 492707968}
GATHER_SOURCES = ("paper_1803_04782_gb300/csrc/sfm_gather.cuh",
                  "paper_1803_04782_gb300/csrc/sfm_field3.cu",
                  "paper_1803_04782_gb300/csrc/sfm_internal.h",
                  "paper_1803_04782_gb300/csrc/sfm_api.cu")  # the bands' row ranges
# the gather kernel of each footprint
GATHER_KERNEL = {"16x16": "k_field_v2", "32x16": "k_field_v2", "32x32r": "k_field_v3"}


def gather_sources_sha1() -> str:
    import hashlib
    h = hashlib.sha1()
    for f in GATHER_SOURCES:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()


def gather_traffic(workload: str, bands: int, footprint: str):
    t = GATHER_TRAFFIC
    if (gather_sources_sha1() == t["sha1"] and workload == t["workload"] and bands == t["bands"]
            and footprint == t["footprint"]):
        return t["bytes_per_launch"]
    return None


def workload(name: str):
    import scenegen as SG
    if name == "floor":
        sc = SG.floor()
        desc = "floor 16384x16384 su, 10% rectangular obstacles, 4 exits x 256 su, 1e6 peds, r=40"
    elif name == "floor-small":
        sc = SG.floor(side=4096, n=62500, exit_len=64)
        desc = "floor 4096x4096 su, 10% rectangular obstacles, 4 exits x 64 su, 62500 peds, r=40"
    elif name == "floor-mid":
        sc = SG.floor(side=8192, n=250000, exit_len=128)
        desc = "floor 8192x8192 su, 10% rectangular obstacles, 4 exits x 128 su, 250000 peds, r=40"
    elif name == "corridor":
        sc = SG.corridor()
        desc = "corridor 1000x200 su, periodic x, 20000 peds counter-flow, r=20"
    elif name == "room":
        sc = SG.room()
        desc = "room 100x100 su, 1 exit x 10 su, 200 peds, r=10"
    else:
        raise ValueError(name)
    return sc, desc


def default_bands(workload: str) -> int:
    """Row bands of the field pass when --bands is not given: the floor's
    divide-and-conquer blocking is part of its workload (at least 4 bands);
    the corridor's and the room's fields (0.8 MB and 40 KB) are not banded."""
    return 4 if workload.startswith("floor") else 1


def band_budget(sc, bands: int) -> int:
    """HBM budget that leaves room for about H/bands field rows."""
    import paper_1803_04782_gb300 as sfm
    if bands <= 1:
        return 0
    rows = -(-sc.H // bands)
    rows = -(-rows // 32) * 32
    return sfm.band_budget(sc.W, sc.H, rows) + 4096


def pair_count(sc, xy, alive) -> int:
    """(su, pedestrian-in-window) pairs of one field pass: the clipped window
    area of every live pedestrian minus its own su."""
    r = int(sc.params["r"])
    m = alive.astype(bool)
    x = xy[m, 0].astype(np.int64)
    y = xy[m, 1].astype(np.int64)
    if sc.periodic_x:
        wx = np.full(x.shape, 2 * r + 1)
    else:
        wx = np.minimum(x + r, sc.W - 1) - np.maximum(x - r, 0) + 1
    if sc.periodic_y:
        wy = np.full(y.shape, 2 * r + 1)
    else:
        wy = np.minimum(y + r, sc.H - 1) - np.maximum(y - r, 0) + 1
    return int((wx * wy - 1).sum())


class Clocks:
    """nvidia-smi sampling of SM clocks and throttle reasons during a region:
    samples every 100 ms, of which those stamped between region_begin() and
    region_end() are kept (all of them, said so, when none falls inside)."""
    Q = ("timestamp,index,uuid,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, uuid=None):
        self.uuid = uuid
        self.proc = None
        self.path = None
        self.t0 = self.t1 = None

    def region_begin(self):
        self.t0 = time.time()

    def region_end(self):
        self.t1 = time.time()

    def start(self):
        fd, self.path = tempfile.mkstemp(suffix=".csv")
        os.close(fd)
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except OSError:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows, stamps = [], []
        for line in open(self.path):
            f = [c.strip() for c in line.split(",")]
            if len(f) < 11:
                continue
            if self.uuid and self.uuid not in f[2]:
                continue
            stamps.append(sample_time(f[0]))
            rows.append(f[1:])
        os.unlink(self.path)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        if not self.uuid:
            idx = rows[0][0]
            keep = [i for i, r in enumerate(rows) if r[0] == idx]
            rows, stamps = [rows[i] for i in keep], [stamps[i] for i in keep]
        inside = [i for i, t in enumerate(stamps)
                  if t is not None and self.t0 is not None and self.t1 is not None
                  and self.t0 - 0.05 <= t <= self.t1 + 0.05]
        window = "timed region"
        if inside:
            rows = [rows[i] for i in inside]
        else:
            window = "whole sampling (no sample fell inside the timed region)"
        sm = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        mx = [float(r[3]) for r in rows if r[3].replace(".", "").isdigit()]
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        reasons = sorted({names[i] for r in rows for i in range(4) if r[6 + i] == "Active"})
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(mx) if mx else None, "reasons": reasons,
                "samples": len(rows), "window": window,
                "power_w_max": max(float(r[4]) for r in rows if r[4].replace(".", "").isdigit())
                if any(r[4].replace(".", "").isdigit() for r in rows) else None}


# consecutive chunks of the timed region, each timed on its own
REPEATS = 5


def chunk_sizes(steps: int, n: int):
    """steps split into min(n, steps) consecutive chunks, sizes within one."""
    n = max(1, min(n, steps))
    return [steps // n + (1 if k < steps % n else 0) for k in range(n)]


def repeat_record(chunks, ms):
    """ms per tick of each chunk, their median and relative spread."""
    per = [m / c for m, c in zip(ms, chunks)]
    med = statistics.median(per)
    return {"n": len(per), "ticks": chunks, "ms_per_step": per, "median_ms_per_step": med,
            "spread": (max(per) - min(per)) / med if med > 0 else 0.0}


def sample_time(stamp: str):
    """Seconds since the epoch of an nvidia-smi timestamp (local time,
    "YYYY/MM/DD HH:MM:SS.mmm"), or None."""
    import datetime
    try:
        return datetime.datetime.strptime(stamp, "%Y/%m/%d %H:%M:%S.%f").timestamp()
    except ValueError:
        return None


def peaks():
    try:
        with open(MEASURED_PEAKS) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0}, "fallback"


def sm_count(torch, dev) -> int:
    """Streaming multiprocessors of the device (its attribute, not a constant)."""
    return int(torch.cuda.get_device_properties(dev).multi_processor_count)


def max_sm_mhz(clk, pk):
    """The maximum SM clock: as nvidia-smi reported it during the timed
    region, else the measured peaks file's, else the nominal 2070."""
    if clk.get("sm_max_mhz"):
        return float(clk["sm_max_mhz"]), "nvidia-smi clocks.max.sm during the run"
    if pk.get("sm_max_mhz"):
        return float(pk["sm_max_mhz"]), "MEASURED_PEAKS.json sm_max_mhz"
    return NOMINAL_SM_MHZ, "nominal maximum"


def gather_roofline(pairs, field_s, nsm, mhz, mhz_src, kernel, traffic=None):
    """Roofline of the class-table field gather for `pairs` (su, pedestrian)
    pairs computed in `field_s` seconds.  Each pair costs one table word read
    from shared memory, and the shared-memory pipe (32 banks x 4 bytes per
    clock per SM) is the resource that binds it; the algorithmic FP32 figure
    of the 3-channel kernel-table formulation (6 flops per pair) and the FP32
    actually executed (1 add per pair) are given beside it."""
    words = pairs / field_s
    smem_peak = nsm * SMEM_WORDS * mhz * 1e6
    fp32_peak = nsm * FP32_LANES * 2 * mhz * 1e6
    return {"bound": "smem", "achieved": words / 1e12, "peak": smem_peak / 1e12,
            "unit": "T table words/s (shared memory, one 4-byte word per pair)",
            "frac": words / smem_peak, "traffic": traffic, "traffic_unit": "bytes per launch",
            "kernel": kernel, "field_ms_per_step": 1e3 * field_s, "pairs_per_step": pairs,
            "peak_basis": f"{nsm} SMs (device attribute) x {SMEM_WORDS} banks x 4 B per clock "
                          f"x {mhz:.0f} MHz ({mhz_src}); derived from unit counts, not measured",
            "algorithmic_fp32": {"flops_per_pair": FLOPS_PER_PAIR,
                                 "achieved_tflops": FLOPS_PER_PAIR * words / 1e12,
                                 "peak_tflops": fp32_peak / 1e12,
                                 "frac": FLOPS_PER_PAIR * words / fp32_peak,
                                 "basis": "3 FP32 multiply-adds per pair of the 3-channel table "
                                          "formulation (algorithmic work, not executed)"},
            "fp32_executed": {"flops_per_pair": 1.0, "achieved_tflops": words / 1e12,
                              "frac": words / fp32_peak,
                              "basis": "the gather adds one precomputed class-table word per pair"}}


# ------------------------------------------------------------------ oracle
def oracle_sample(sc, D, xy, heading, goal, alive, n_sample, t, seed=0):
    """One bounded sample of the oracle's tick, timed as it runs: n_sample
    random live pedestrians decide (the oracle evaluates the field by direct
    superposition at their 9 candidates only; it never builds the lattice
    field the GPU path writes), then vote and commit, every other pedestrian
    staying for this sample.  The state arrays are advanced in place.
    Returns (seconds spent, threads, pedestrians decided, live pedestrians,
    seconds of the decisions alone)."""
    import oracle as O
    m = O.model(sc)
    occ, _ = O.occupancy(m, sc.cell, xy, alive)
    live = np.flatnonzero(alive)
    rng = np.random.default_rng(seed + t)
    req = np.sort(rng.choice(live, size=min(n_sample, live.size), replace=False)).astype(np.int32)
    t0 = time.perf_counter()
    ch, E, T, adm = O.decide(m, sc.cell, occ, xy, heading, goal, alive, D, req)
    t1 = time.perf_counter()
    choice = np.zeros(xy.shape[0], np.uint8)
    choice[req] = ch
    won, _ = O.vote(m, t, xy, alive, choice)
    O.commit(m, sc.cell, xy, heading, alive, choice, won)
    t2 = time.perf_counter()
    return t2 - t0, O.threads(), int(req.size), int(live.size), t1 - t0


def host_cpu() -> str:
    """The host CPU's model name as lscpu reports it (else /proc/cpuinfo)."""
    try:
        out = subprocess.run(["lscpu"], capture_output=True, text=True, timeout=10).stdout
        for line in out.splitlines():
            if line.strip().startswith("Model name:"):
                return line.split(":", 1)[1].strip()
    except (OSError, subprocess.SubprocessError):
        pass
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part")):
                    return line.split(":", 1)[1].strip()
    except OSError:
        pass
    return "unknown"


def oracle_sample_desc(n_sample):
    return (f"per step: {n_sample} random live pedestrians decide (the oracle evaluates the "
            f"field by direct FP64 superposition at their 9 candidates only, not on the "
            f"lattice), vote and commit; the rest of the crowd stays for that step")


def workload_config(args, sc, desc):
    """The workload's description, identical in both arms."""
    return {"workload": desc, "W": sc.W, "H": sc.H, "n": sc.n, "r": int(sc.params["r"]),
            "bands": args.bands if args.bands is not None else default_bands(args.workload),
            "l2": "inputs larger than L2 (the field alone is 4*W*H bytes)"
            if sc.W * sc.H * 4 > 129e6 else "inputs smaller than L2"}


def reduce_over_ranks(dist, seconds, units, device="cpu"):
    """Whole-job timing over N ranks: the slowest rank's time and the units
    all ranks processed (replicas: no collective on the data path, only this
    one after the timed region).  dist None: one rank, values unchanged."""
    if dist is None:
        return float(seconds), float(units)
    import torch
    t = torch.tensor([float(seconds)], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    u = torch.tensor([float(units)], device=device, dtype=torch.float64)
    dist.all_reduce(u)
    return float(t.item()), float(u.item())


def reference_runs_here() -> bool:
    """The reference arm (the CPU oracle) runs on rank 0 only; under torchrun
    the other ranks exit 0 without work."""
    return int(os.environ.get("RANK", "0")) == 0


def run_reference(args):
    """--impl reference: the FP64 oracle on the host cores, bounded samples."""
    if not reference_runs_here():
        return 0
    import oracle as O
    O.build()
    sc, desc = workload(args.workload)
    m = O.model(sc)
    D = O.guidance(m, sc.cell)
    xy, heading, goal = sc.xy.copy(), sc.heading.copy(), sc.goal.copy()
    alive = np.ones(sc.n, np.uint8)
    n_sample = args.ref_sample
    for w in range(args.warmup):
        oracle_sample(sc, D, xy, heading, goal, alive, n_sample, w)
    secs, dec_secs, decided, lives = [], [], [], []
    thr = 0
    for k in range(args.steps):
        s, thr, ns, nl, sd = oracle_sample(sc, D, xy, heading, goal, alive, n_sample,
                                           args.warmup + k)
        secs.append(s)
        dec_secs.append(sd)
        decided.append(ns)
        lives.append(nl)
    tot = sum(secs)
    # value: pedestrian-steps the oracle actually advanced per second it ran
    value = sum(decided) / tot
    frac = sum(decided) / max(1, sum(lives))
    line = {
        "impl": "reference", "metric": "pedestrian-steps/s", "value": value,
        "unit": "ped-steps/s", "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * tot / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": workload_config(args, sc, desc),
        "parallelism": "CPU oracle, rank 0 only",
        "cpu_baseline": {"value": value, "unit": "ped-steps/s", "cores": thr, "kind": "oracle",
                         "cpu_model": host_cpu(),
                         "sample": oracle_sample_desc(n_sample),
                         "sample_peds_per_step": n_sample,
                         "sample_fraction_of_live_crowd": frac,
                         "seconds_timed": tot,
                         "seconds_deciding": sum(dec_secs)},
        # what a whole tick of the live crowd would take at the sample's
        # decision rate: an extrapolation, not a measurement
        "full_tick_s_extrapolated": (sum(dec_secs) / frac + (tot - sum(dec_secs))) / args.steps,
        "e2e": {"value": value, "unit": "ped-steps/s", "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)
    return 0


# ------------------------------------------------------------ secondary
def tick_rate(torch, sim, stream, ticks, timing_every=TIMING_EVERY):
    """Graph-replayed ticks of a placed, warmed-up context: ms per tick over
    `ticks` (CUDA events on its stream, stage events every `timing_every`-th
    tick) and the field ms per timed tick."""
    sim.set_timing(timing_every)
    sim.stage_times()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    sim.step(ticks)
    e1.record(stream)
    torch.cuda.synchronize()
    st, nt = sim.stage_times()
    sim.set_timing(False)
    return e0.elapsed_time(e1) / ticks, st["field"] / max(1, nt)


def secondary_measurements(torch, sfm, stream, nsm, mhz, mhz_src, ticks=20):
    """The other configurations, measured in the same run as the headline so
    that their numbers come from the same box and clock: the 1000x200
    corridor and the 100x100 room (autotuned, unbanded), the batch of 256
    rooms (one persistent launch per tick, autotuned), and the floor's exact
    tick with the field at each pedestrian's 9 candidates only (unbanded; the
    surrogate entry point with delta = +inf, which runs no network) beside
    its lattice tick."""
    import scenegen as SG
    out = {}
    for name in ("corridor", "room"):
        sc, desc = workload(name)
        with sfm.Sim(sc, stream=stream) as sim:
            fp = sim.autotune()
            sim.set_timing(TIMING_EVERY)
            sim.step(10)
            xy0, _, a0 = sim.peds()
            ms, fms = tick_rate(torch, sim, stream, ticks)
            pairs = pair_count(sc, xy0, a0)
            out[name] = {"workload": desc, "ped_steps_per_s": int(a0.sum()) / (ms / 1e3),
                         "ms_per_tick": ms, "field_ms": fms, "footprint": fp,
                         "roofline": gather_roofline(pairs, fms / 1e3, nsm, mhz, mhz_src,
                                                     GATHER_KERNEL.get(fp, "k_field"))}
    scenes = SG.batch(nscenes=256)
    with sfm.Batch(scenes, stream=stream) as bt:
        bt.autotune()
        bt.step(5)
        bt.sync()
        _, _, al = bt.peds()
        alive0 = sum(int(a.sum()) for a in al)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        bt.step(5)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
    out["batch"] = {"workload": "batch of 256 rooms: side U[64,2048], density U[0.05,0.4], "
                                "radius U[5,30], 1-4 exits", "ped_steps_per_s": alive0 / (ms / 1e3),
                    "ms_per_tick": ms}
    sc, desc = workload("floor")
    with sfm.Sim(sc, stream=stream) as sim:
        sim.autotune()
        sim.step(10)
        ms_lat, _ = tick_rate(torch, sim, stream, 10, timing_every=0)
        with sfm.Surrogate(coarsen=8, near_radius=3, stream=stream) as sur:
            sur.set_delta(float("inf"))
            sur.step(sim, 2)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sur.step(sim, 10)
            e1.record(stream)
            torch.cuda.synchronize()
            ms_cand = e0.elapsed_time(e1) / 10
        alive = sim.stats()["alive"]
    out["floor_candidates_only"] = {
        "workload": desc + ", unbanded", "ms_per_tick_lattice": ms_lat,
        "ms_per_tick_candidates_only": ms_cand,
        "ped_steps_per_s_candidates_only": alive / (ms_cand / 1e3),
        "how": "exact moves either way (bit for bit); the candidate-only tick computes the "
               "field at each pedestrian's 9 candidates, not on the lattice"}
    return out


# ------------------------------------------------------------------ GPU arm
def run_gpu(args):
    import torch
    import paper_1803_04782_gb300 as sfm
    from paper_1803_04782_gb300 import build as B

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU (the CPU oracle arm is --impl reference)")
    torch.cuda.set_device(local)
    B.build()
    sfm.lib()
    nsm = sm_count(torch, local)

    sc, desc = workload(args.workload)
    bands = args.bands if args.bands is not None else default_bands(args.workload)
    budget = band_budget(sc, bands)
    stream = torch.cuda.current_stream()
    sim = sfm.Sim(sc, stream=stream, hbm_budget_bytes=budget)
    n = sc.n
    if args.footprint == "auto":
        footprint = sim.autotune()
    else:  # a fixed shape (an ncu capture perturbs the autotuner's event timings)
        sim.set_footprint(args.footprint)
        footprint = args.footprint
    st0 = sim.stats()

    def barrier():
        if dist is not None:
            dist.barrier()

    # warm-up with the stage sampling on, so its first replayed tick builds
    # every graph the timed region replays (untimed and timed)
    sim.set_timing(TIMING_EVERY)
    sim.step(args.warmup)
    sim.sync()
    xy0, h0, a0 = sim.peds()
    pairs0 = pair_count(sc, xy0, a0)
    alive0 = int(a0.sum())
    stw = sim.stats()
    launches0 = stw["kernel_launches"]

    # timed region: K ticks replayed as graphs; every TIMING_EVERY-th of them
    # (the first included) replays the one-tick graph whose stage events are
    # event record nodes on the library's stream
    sim.set_timing(TIMING_EVERY)
    sim.stage_times()  # reset
    uuid = None
    try:
        uuid = str(torch.cuda.get_device_properties(local).uuid)
    except Exception:
        pass
    clocks = Clocks(uuid)
    clocks.start()
    time.sleep(0.3)
    barrier()
    torch.cuda.synchronize()
    ev0 = torch.cuda.Event(enable_timing=True)
    ev1 = torch.cuda.Event(enable_timing=True)
    clocks.region_begin()
    # the K ticks in REPEATS consecutive chunks, an event between chunks: the
    # chunks give repeated measurements of the same loop (their median and
    # spread); `value` is the whole region
    chunks = chunk_sizes(args.steps, REPEATS)
    evs = [ev0] + [torch.cuda.Event(enable_timing=True) for _ in chunks[:-1]] + [ev1]
    ev0.record(stream)
    for k, m in enumerate(chunks):
        sim.step(m)
        evs[k + 1].record(stream)
    torch.cuda.synchronize()
    clocks.region_end()
    barrier()
    clk = clocks.stop()
    elapsed = ev0.elapsed_time(ev1) / 1e3
    repeats = repeat_record(chunks, [evs[k].elapsed_time(evs[k + 1]) for k in range(len(chunks))])
    stage_ms, ticks = sim.stage_times()
    sim.set_timing(False)
    st1 = sim.stats()
    xy1, h1, a1 = sim.peds()
    # the same ticks replayed as untimed graphs (8 ticks each while that many
    # remain) without stage events: what the event nodes cost shows on small
    # lattices; after the timed region, not part of `value`
    graph_ticks = max(3, min(args.steps, 20))
    sim.step(graph_ticks)  # builds (once) the graphs the timed call replays
    torch.cuda.synchronize()
    g0 = torch.cuda.Event(enable_timing=True)
    g1 = torch.cuda.Event(enable_timing=True)
    g0.record(stream)
    sim.step(graph_ticks)
    g1.record(stream)
    torch.cuda.synchronize()
    graph_ms = g0.elapsed_time(g1) / graph_ticks
    pairs1 = pair_count(sc, xy1, a1)
    alive1 = int(a1.sum())
    launches = st1["kernel_launches"] - launches0
    # decisions of the timed ticks and the near ties among them
    decided = st1["decided"] - stw["decided"]
    near_ties = st1["near_ties"] - stw["near_ties"]
    ped_steps = 0.5 * (alive0 + alive1) * args.steps
    elapsed, ped_steps = reduce_over_ranks(dist, elapsed, ped_steps, "cuda")

    # roofline of the dominant kernel: the field gather
    pk, pk_src = peaks()
    mhz, mhz_src = max_sm_mhz(clk, pk)
    field_s = stage_ms["field"] / 1e3  # over the `ticks` timed ticks
    pairs = 0.5 * (pairs0 + pairs1)
    roofline = gather_roofline(pairs, field_s / ticks, nsm, mhz, mhz_src,
                               GATHER_KERNEL.get(footprint, "k_field"),
                               gather_traffic(args.workload, st1["bands"], footprint))
    roofline["timed_ticks"] = ticks

    # end to end through the C ABI with host buffers
    e2e_steps = min(args.steps, args.e2e_steps)
    hx = torch.from_numpy(xy1.copy()).pin_memory()
    hh = torch.from_numpy(h1.copy()).pin_memory()
    hg = torch.from_numpy(sc.goal.copy()).pin_memory()
    ha = torch.from_numpy(a1.copy()).pin_memory()
    alive_start = int(np.count_nonzero(ha.numpy()))
    torch.cuda.synchronize()
    barrier()
    t0 = time.perf_counter()
    for _ in range(e2e_steps):
        sfm.sfm_place(sim.ctx, hx, hh, hg, ha)
        sfm.sfm_step(sim.ctx, 1)
        sfm.sfm_read_peds(sim.ctx, hx, hh, ha)
    torch.cuda.synchronize()
    e2e_t = time.perf_counter() - t0
    # live pedestrians per tick: the mean of the counts before and after, as
    # for the device-timed value (the host counts outside the timed loop)
    e2e_peds = 0.5 * (alive_start + int(np.count_nonzero(ha.numpy()))) * e2e_steps
    e2e_t, e2e_peds = reduce_over_ranks(dist, e2e_t, e2e_peds, "cuda")
    e2e = {"value": e2e_peds / e2e_t, "unit": "ped-steps/s",
           "h2d_bytes_per_step": n * (8 + 1 + 1 + 1), "d2h_bytes_per_step": n * (8 + 1 + 1),
           "steps": e2e_steps}

    if rank != 0:
        sim.close()
        if dist is not None:
            dist.destroy_process_group()
        return 0

    secondary = None
    if args.workload == "floor" and world == 1 and not args.no_secondary:
        secondary = secondary_measurements(torch, sfm, stream, nsm, mhz, mhz_src)

    # CPU baseline: the oracle on a bounded sample of the same workload
    cpu = None
    if not args.no_cpu_baseline and world == 1:
        import oracle as O
        O.build()
        m = O.model(sc)
        D = O.guidance(m, sc.cell)
        s, thr, ns, nl, sd = oracle_sample(sc, D, xy1.copy(), h1.copy(), sc.goal.copy(),
                                           a1.copy(), args.ref_sample, 0)
        cpu = {"value": ns / s, "unit": "ped-steps/s", "cores": thr, "kind": "oracle",
               "cpu_model": host_cpu(),
               "sample": oracle_sample_desc(args.ref_sample) + " (one step)",
               "sample_peds": ns, "sample_fraction_of_live_crowd": ns / max(1, nl),
               "seconds_timed": s, "seconds_deciding": sd,
               "full_tick_s_extrapolated": sd * nl / max(1, ns) + (s - sd)}
    line = {
        "metric": "pedestrian-steps/s", "value": ped_steps / elapsed, "unit": "ped-steps/s",
        "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": 1e3 * elapsed / args.steps, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32", "data": "synthetic",
        "config": workload_config(args, sc, desc),
        "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
        "bands": st1["bands"], "hbm_budget_bytes": budget, "field_footprint": footprint,
        "sms": nsm,
        "su_updates_per_s": sc.W * sc.H * args.steps * world / elapsed,
        "decisions": {"timed_ticks_decided": decided, "near_ties": near_ties,
                      "near_tie_rate": near_ties / max(1, decided),
                      "rule": "best and second-best admissible energies within 1e-5 of "
                              "|F| + |own| + |guidance| (FP32, counted by the decision kernel)"},
        "stage_ms_per_step": {k: v / max(1, ticks) for k, v in stage_ms.items()},
        "stage_timing": f"CUDA events around each stage of every {TIMING_EVERY}th tick of the "
                        f"timed region ({ticks} of {args.steps} ticks)",
        "graph_ms_per_step": graph_ms,
        "repeats": repeats,
        "roofline": roofline,
        "cpu_baseline": cpu,
        "e2e": e2e,
        "secondary": secondary,
        "clocks": clk,
        "gpu_launches": int(launches),
        "peaks_source": pk_src,
        "hbm_peak_gbs": pk.get("hbm_gbs"),
    }
    print(json.dumps(line), flush=True)
    sim.close()
    if dist is not None:
        dist.destroy_process_group()
    return 0


# ------------------------------------------------------------------ batch arm
def run_batch(args):
    """256 independent rooms (side U[64,2048], density U[0.05,0.4], radius
    U[5,30], 1-4 exits) stepped together: one persistent launch per tick, the
    tick loop replayed from a CUDA graph, tiles from the autotuner.  Beside it,
    the same scenes stepped one context after another (the plain exact path)."""
    import torch
    import paper_1803_04782_gb300 as sfm
    import scenegen as SG
    from paper_1803_04782_gb300 import build as B

    if not torch.cuda.is_available():
        raise SystemExit("bench.py needs a CUDA GPU")
    B.build()
    sfm.lib()
    nsc = 256 if args.workload == "batch" else 32
    scenes = SG.batch(nscenes=nsc)
    desc = (f"batch of {nsc} rooms: side U[64,2048], density U[0.05,0.4] of free su, "
            "radius U[5,30], 1-4 exits, wall ring")
    stream = torch.cuda.current_stream()
    n = sum(s.n for s in scenes)
    su = sum(s.W * s.H for s in scenes)
    with sfm.Batch(scenes, stream=stream) as bt:
        t0 = time.perf_counter()
        shapes = bt.autotune()
        tune_s = time.perf_counter() - t0
        bt.step(args.warmup)
        bt.sync()
        xs, _, al = bt.peds()
        alive0 = sum(int(a.sum()) for a in al)
        pairs = sum(pair_count(s, x, a) for s, x, a in zip(scenes, xs, al))
        clocks = Clocks()
        clocks.start()
        time.sleep(0.3)
        torch.cuda.synchronize()
        ev0 = torch.cuda.Event(enable_timing=True)
        ev1 = torch.cuda.Event(enable_timing=True)
        clocks.region_begin()
        ev0.record(stream)
        bt.step(args.steps)
        ev1.record(stream)
        torch.cuda.synchronize()
        clocks.region_end()
        clk = clocks.stop()
        bt.sync()
        elapsed = ev0.elapsed_time(ev1) / 1e3
        _, _, al = bt.peds()
        alive1 = sum(int(a.sum()) for a in al)
        # field-only launches (bins + field) time the dominant stage
        bt.set_timing(True)
        bt.stage_times()
        for _ in range(3):
            bt.compute_field()
        st_ms, _ = bt.stage_times()
        bt.set_timing(False)
        field_s = st_ms["field"] / 3 / 1e3
        launches = bt.stats()["kernel_launches"]
    ped_steps = 0.5 * (alive0 + alive1) * args.steps
    value = ped_steps / elapsed

    # the plain exact path: each scene in its own context (footprint
    # autotuned like the batch's), (a) on one stream, one context after
    # another, and (b) spread over 16 streams so that different contexts'
    # kernels may run at the same time
    plain_steps = max(3, min(args.steps, 10))

    def plain_path(nstreams):
        streams = [stream] if nstreams == 1 else [torch.cuda.Stream() for _ in range(nstreams)]
        sims = [sfm.Sim(s, stream=streams[i % nstreams]) for i, s in enumerate(scenes)]
        for s in sims:
            s.autotune()
        # two warm-up ticks each: the first runs stage by stage, the second
        # builds every graph the timed ticks replay (no capture in the timing)
        for s in sims:
            s.step(2)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        for s in sims:
            s.step(plain_steps)
        torch.cuda.synchronize()
        t = time.perf_counter() - t0
        alive = sum(s.stats()["alive"] for s in sims)
        for s in sims:
            s.close()
        return alive * plain_steps / t

    plain_value = plain_path(1)
    plain_value_mt = plain_path(16)

    pk, _ = peaks()
    mhz, mhz_src = max_sm_mhz(clk, pk)
    line = {
        "metric": "pedestrian-steps/s", "value": value, "unit": "ped-steps/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * elapsed / args.steps,
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
        "data": "synthetic",
        "config": {"workload": desc, "scenes": nsc, "n": n, "su": su,
                   "footprint_per_radius_class": shapes, "autotune_s": tune_s,
                   "l2": "inputs larger than L2", "parallelism": "single GPU"},
        "su_updates_per_s": su * args.steps / elapsed,
        "plain_exact_path": {"value": plain_value, "unit": "ped-steps/s",
                             "how": f"{nsc} contexts stepped one after another on one stream, "
                                    f"{plain_steps} ticks"},
        "plain_exact_path_16_streams": {"value": plain_value_mt, "unit": "ped-steps/s",
                                        "how": f"{nsc} contexts on 16 streams (round robin), "
                                               f"{plain_steps} ticks, launched back to back"},
        "speedup_vs_plain": value / plain_value,
        "speedup_vs_plain_16_streams": value / plain_value_mt,
        "roofline": gather_roofline(pairs, field_s, sm_count(torch, torch.cuda.current_device()),
                                    mhz, mhz_src, "k_tick_batch (field only)"),
        "cpu_baseline": None, "e2e": None, "clocks": clk, "gpu_launches": int(launches),
    }
    print(json.dumps(line), flush=True)
    return 0


# -------------------------------------------------------------- surrogate arm
# the surrogate's training schedule: (scene, Adam steps) -- the wall-less
# torus canvas with tile densities from the sparse floor to the dense
# corridor ends, then two 4096^2 floors shaped like the benchmark's (walls,
# rectangular obstacles, 4 exits, exit-seekers) at its density and at 8x it
SURROGATE_TRAINING = (("canvas 4096^2 torus, tile densities 0.002-0.25", 60),
                      ("floor 4096^2, 62500 exit-seekers", 45),
                      ("floor 4096^2, 500000 exit-seekers", 45))


def surrogate_training_scenes():
    import scenegen as SG
    return (SG.training_canvas(side=4096, r=40, seed=500),
            SG.floor(side=4096, n=62500, exit_len=64, seed=501),
            SG.floor(side=4096, n=500000, exit_len=64, seed=502))


def train_surrogate(sfm, stream, init, lr=2e-3):
    """Trains the s = 8, r_n = 3 surrogate by the schedule above, each phase
    ticking its own context.  Returns (parameters, loss curve of each phase)."""
    curves = []
    with sfm.Surrogate(coarsen=8, near_radius=3, target_scale=20.0, lr=lr, params=init,
                       stream=stream) as sur:
        for sc, (what, iters) in zip(surrogate_training_scenes(), SURROGATE_TRAINING):
            with sfm.Sim(sc, stream=stream) as tsim:
                curves.append(sur.train(tsim, iters))
        return sur.get_params(), curves


def run_surrogate(args):
    """Learned surrogate with the exact fallback of the decisions: trained on
    the GPU by SURROGATE_TRAINING (150 Adam steps, r = 40), its margin bound
    delta calibrated (99.9th percentile of the candidate error spread) on the
    16384^2 floor three ticks before it is judged there by the exact path:
    field error, decision flip rate with and without the fallback, fallback
    rate, and three tick times -- the exact tick (lattice field), the exact
    tick with the field computed at the candidates only (delta = +inf, no
    network), and the surrogate tick.  The same near part without the
    network, and the literal fine-grid network (s = 1, no near part), are
    judged beside it."""
    import torch
    import paper_1803_04782_gb300 as sfm
    import scenegen as SG
    from paper_1803_04782_gb300 import build as B

    B.build()
    sfm.lib()
    stream = torch.cuda.current_stream()
    init = sfm.flatten_params(SG.surrogate_init(0))

    def tick_ms(fn, n):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        fn(1)
        torch.cuda.synchronize()
        e0.record(stream)
        fn(n)
        e1.record(stream)
        torch.cuda.synchronize()
        return e0.elapsed_time(e1) / n

    def judge(sur, sim, timed):
        d = sur.calibrate(sim, 0.999)
        sim.step(3)
        evs = [sur.eval(sim) for _ in range(3)]
        ev = sorted(evs, key=lambda e: e["ms_surrogate"])[1]
        out = {"delta": d, **{k: ev[k] for k in ("field_rel_err", "flip_rate", "flip_rate_raw",
                                                 "fallback_rate", "ms_surrogate", "ms_exact",
                                                 "ms_surrogate_field", "decided")}}
        if timed:
            n = max(3, min(args.steps, 10))
            out["ms_tick_surrogate"] = tick_ms(lambda k: sur.step(sim, k), n)
            fb, dec = sur.counts()
            out["fallback_rate_ticks"] = fb / max(dec, 1)
            out["ms_tick_exact"] = tick_ms(lambda k: sim.step(k), n)
            sur.set_delta(float("inf"))
            out["ms_tick_exact_candidates"] = tick_ms(lambda k: sur.step(sim, k), n)
            sur.set_delta(d)
        return out

    out = {}
    t0 = time.perf_counter()
    trained, curves = train_surrogate(sfm, stream, init)
    curve = np.concatenate(curves)
    train_s = time.perf_counter() - t0
    sc, desc = workload("floor")
    with sfm.Sim(sc, stream=stream) as fsim:
        fsim.step(args.warmup)
        for name, params in (("coarse8_near3", trained), ("near3_without_network", 0 * init)):
            with sfm.Surrogate(coarsen=8, near_radius=3, target_scale=20.0, params=params,
                               stream=stream) as sur:
                out[name] = judge(sur, fsim, timed=name == "coarse8_near3")
    out["coarse8_near3"].update({"train_iters": len(curve),
                                 "train_tiles_128": len(curve) * (4096 // 128) ** 2,
                                 "train_schedule": [list(p) for p in SURROGATE_TRAINING],
                                 "train_s": train_s, "loss_first": float(curve[0]),
                                 "loss_last": float(curve[-5:].mean())})
    # literal network: +-5 su of context, no near part (flip rate without fallback)
    canvas_s = SG.training_canvas(side=1024, r=40, seed=500)
    with sfm.Sim(canvas_s, stream=stream) as tsim, \
            sfm.Surrogate(coarsen=1, near_radius=0, target_scale=20.0, lr=2e-3, params=init,
                          stream=stream) as sur:
        sur.train(tsim, 100)
        scs, _ = workload("floor-small")
        with sfm.Sim(scs, stream=stream) as ssim:
            ssim.step(args.warmup)
            ev = sur.eval(ssim)
        out["literal_s1"] = {k: ev[k] for k in ("field_rel_err", "flip_rate_raw", "ms_surrogate",
                                                "ms_exact")}
    main_r = out["coarse8_near3"]
    speed = main_r["ms_tick_exact"] / main_r["ms_tick_surrogate"]
    speed_cand = main_r["ms_tick_exact_candidates"] / main_r["ms_tick_surrogate"]
    line = {
        "metric": "surrogate vs exact at set flip rate", "value": speed,
        "unit": "x (exact tick time / surrogate tick time)", "n_gpus": 1, "steps": 3,
        "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "bf16 weights/activations, f32 accumulation", "data": "synthetic",
        "config": {"workload": desc, "flip_rate_target": 1e-3, "delta_quantile": 0.999},
        "flip_rate": main_r["flip_rate"],
        "meets_flip_target": main_r["flip_rate"] <= 1e-3,
        "ticks_ms": {"exact_lattice": main_r["ms_tick_exact"],
                     "exact_candidates_only": main_r["ms_tick_exact_candidates"],
                     "surrogate": main_r["ms_tick_surrogate"]},
        "beats_exact_lattice": speed > 1.0,
        "speedup_vs_exact_candidates_only": speed_cand,
        "beats_exact_candidates_only": speed_cand > 1.0,
        "variants": out,
    }
    print(json.dumps(line), flush=True)
    return 0


def run_surrogate_eval(args):
    """One surrogate evaluation on the 16384^2 floor (4096^2 and 8192^2 for
    surrogate-eval-small / -mid, the cases for counter captures) with the seeded
    (untrained) network, s = 8, r_n = 3: calibrate delta (99.9th percentile)
    and judge twice; prints the second report (the case the surrogate's
    launch-list profile covers)."""
    import torch
    import paper_1803_04782_gb300 as sfm
    import scenegen as SG
    from paper_1803_04782_gb300 import build as B

    B.build()
    sfm.lib()
    stream = torch.cuda.current_stream()
    sc, desc = workload({"surrogate-eval-small": "floor-small",
                         "surrogate-eval-mid": "floor-mid"}.get(args.workload, "floor"))
    with sfm.Sim(sc, stream=stream) as sim, \
            sfm.Surrogate(coarsen=8, near_radius=3, params=sfm.flatten_params(SG.surrogate_init(0)),
                          stream=stream) as sur:
        sim.step(2)
        sur.calibrate(sim, 0.999)
        ev = [sur.eval(sim) for _ in range(2)][-1]
    print(json.dumps({"metric": "surrogate evaluation", "config": {"workload": desc}, **ev}),
          flush=True)
    return 0


def run_paper_sweep(args):
    """The paper's experiment shapes (Sec. 5) on one GB300: a periodic
    1000x1000 lattice, density 0.5 (500 000 pedestrians), 8 flow directions.
    paper-windows: field geometries 7x7 ... 77x77 (Table III, r = 3 ... 38);
    paper-periods: 7x7 fields with walk periods uniform in [1, P_max],
    P_max = 1 ... 11 (Table IV).  Each case: autotuned footprint, warm-up,
    then ticks replayed as CUDA graphs timed with CUDA events, and a second
    pass with per-stage events for the field time.  The paper's own times
    (seconds per 1000 ticks, unnamed hardware) are listed beside as context."""
    import torch
    import paper_1803_04782_gb300 as sfm
    import scenegen as SG
    from paper_1803_04782_gb300 import build as B

    B.build()
    sfm.lib()
    stream = torch.cuda.current_stream()
    if args.workload == "paper-sizes":
        return run_paper_sizes(args)
    if args.workload == "paper-sweep":
        return run_paper_grid(args)
    if args.workload == "paper-windows":
        cases = [(r, 1) for r in (3, 10, 17, 24, 31, 38)]
        paper_s = [62, 317, 738, 1424, 2187, 3238]
        what = "Table III: field geometry (2r+1)^2, 1000^2 su, density 0.5, 8 directions"
    else:
        cases = [(3, p) for p in (1, 3, 5, 7, 9, 11)]
        paper_s = [62, 64, 64, 63, 62, 62]
        what = "Table IV: maximal walk period, 1000^2 su, density 0.5, 8 directions, 7x7 fields"
    ticks = max(5, min(args.steps, 50))
    rows = []
    for (r, pmax), ps in zip(cases, paper_s):
        sc = SG.paper_scene(side=1000, density=0.5, ndir=8, r=r)
        with sfm.Sim(sc, stream=stream) as sim:
            fp = sim.autotune()
            if pmax > 1:
                per, pha = SG.walk_periods(sc.n, pmax)
                sim.set_walk_periods(per, pha)
            sim.step(max(args.warmup, 9))  # also builds the 8-tick graph
            torch.cuda.synchronize()
            xy0, _, a0 = sim.peds()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            sim.step(ticks)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / ticks
            sim.set_timing(True)
            sim.stage_times()
            sim.step(ticks)
            st_ms, nt = sim.stage_times()
            sim.set_timing(False)
            pairs = pair_count(sc, xy0, a0)
            field_ms = st_ms["field"] / max(1, nt)
            rows.append({"r": r, "window": (2 * r + 1) ** 2, "walk_period_max": pmax,
                         "footprint": fp, "ms_per_tick": ms,
                         "ped_steps_per_s": int(a0.sum()) / (ms / 1e3),
                         "su_updates_per_s": sc.W * sc.H / (ms / 1e3),
                         "field_ms": field_ms,
                         "field_tflops": FLOPS_PER_PAIR * pairs / (field_ms / 1e3) / 1e12,
                         "paper_ms_per_tick": ps, "paper_over_this": ps / ms})
    area = np.array([row["window"] for row in rows], float)
    tms = np.array([row["ms_per_tick"] for row in rows])
    slope, icpt = np.polyfit(area, tms, 1) if len(set(area)) > 1 else (0.0, float(tms.mean()))
    pred = slope * area + icpt
    r2 = 1.0 - float(((tms - pred) ** 2).sum() / max(((tms - tms.mean()) ** 2).sum(), 1e-30))
    line = {"metric": "pedestrian-steps/s", "value": rows[0]["ped_steps_per_s"],
            "unit": "ped-steps/s", "n_gpus": 1, "steps": ticks, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic", "config": {"workload": what},
            "rows": rows,
            "time_vs_window_area": {"ms_per_window_su": slope, "ms_intercept": icpt,
                                    "r2": r2 if args.workload == "paper-windows" else None}}
    print(json.dumps(line), flush=True)
    return 0


def run_paper_grid(args):
    """The paper's 360-combination sweep (Sec. 5): periodic lattices of side
    100, 200, ..., 1000 su, densities 0.1 ... 0.9, uni-, bi-, 4- and
    8-directional flows of fixed-direction walkers, 7x7 fields (r = 3), 1x1
    pedestrians, walk period 1.  One JSON line per combination (graph-
    replayed ticks timed with CUDA events after warm-up), then a summary
    line with, per flow count, the least-squares fit of the tick time to the
    number of pedestrians.  The paper plots its speed-ups for these
    combinations (its Figs. 3-6, unnamed hardware) but prints no times."""
    import torch
    import paper_1803_04782_gb300 as sfm
    import scenegen as SG
    from paper_1803_04782_gb300 import build as B

    B.build()
    sfm.lib()
    stream = torch.cuda.current_stream()
    ticks = max(5, min(args.steps, 20))
    rows = []
    for side in range(100, 1001, 100):
        for di, rho in enumerate([0.1 * k for k in range(1, 10)]):
            for nd in (1, 2, 4, 8):
                sc = SG.paper_scene(side=side, density=round(rho, 1), ndir=nd, r=3,
                                    seed=1000 + side + 10 * di + nd)
                with sfm.Sim(sc, stream=stream) as sim:
                    sim.step(max(args.warmup, 9))  # also builds the 8-tick graph
                    torch.cuda.synchronize()
                    e0 = torch.cuda.Event(enable_timing=True)
                    e1 = torch.cuda.Event(enable_timing=True)
                    e0.record(stream)
                    sim.step(ticks)
                    e1.record(stream)
                    torch.cuda.synchronize()
                    ms = e0.elapsed_time(e1) / ticks
                row = {"side": side, "density": round(rho, 1), "directions": nd, "peds": sc.n,
                       "ms_per_tick": ms, "ped_steps_per_s": sc.n / (ms / 1e3),
                       "su_updates_per_s": side * side / (ms / 1e3)}
                rows.append(row)
                print(json.dumps({"metric": "pedestrian-steps/s", "value": row["ped_steps_per_s"],
                                  "unit": "ped-steps/s", "config": {"workload": "paper sweep cell",
                                                                    **row}}), flush=True)
    fits = {}
    for nd in (1, 2, 4, 8):
        sel = [rw for rw in rows if rw["directions"] == nd]
        n = np.array([rw["peds"] for rw in sel], float)
        t = np.array([rw["ms_per_tick"] for rw in sel])
        slope, icpt = np.polyfit(n, t, 1)
        pred = slope * n + icpt
        r2 = 1.0 - float(((t - pred) ** 2).sum() / max(((t - t.mean()) ** 2).sum(), 1e-30))
        fits[str(nd)] = {"ms_per_million_peds": slope * 1e6, "ms_intercept": icpt, "r2": r2,
                         "ms_min": float(t.min()), "ms_max": float(t.max())}
    line = {"metric": "pedestrian-steps/s", "value": float(np.median([rw["ped_steps_per_s"] for rw in rows])),
            "unit": "ped-steps/s (median over the 360 combinations)", "n_gpus": 1, "steps": ticks,
            "warmup": args.warmup, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32", "data": "synthetic",
            "config": {"workload": "paper sweep: sides 100-1000 x densities 0.1-0.9 x 1/2/4/8 "
                                   "flows, periodic, 7x7 fields", "combinations": len(rows)},
            "time_vs_pedestrians": fits}
    print(json.dumps(line), flush=True)
    return 0


def run_paper_sizes(args):
    """Table V's shape: pedestrian geometry g x g (g = 1 ... 11) on a periodic
    1000^2 lattice covering half its area (500 000 / g^2 pedestrians), field
    window 7g x 7g, crossed with maximal walk periods 1 ... 11; graph-replayed
    ticks timed with CUDA events.  The paper's seconds per 1000 ticks are
    given beside (context only)."""
    import torch
    import paper_1803_04782_gb300 as sfm
    import scenegen as SG
    from paper_1803_04782_gb300 import build as B

    B.build()
    sfm.lib()
    stream = torch.cuda.current_stream()
    paper = {1: [63.5, 63.9, 64.0, 63.8, 63.7, 63.9], 3: [264.6, 261.7, 264.1, 262.9, 262.2, 261.8],
             5: [213.5, 202.0, 204.6, 201.3, 200.1, 200.8], 7: [207.7, 197.1, 195.5, 193.9, 194.5, 193.8],
             9: [197.6, 186.9, 184.4, 182.0, 184.2, 182.1], 11: [201.5, 192.5, 191.2, 191.6, 190.5, 189.6]}
    ticks = max(5, min(args.steps, 30))
    rows = []
    for g in (1, 3, 5, 7, 9, 11):
        sc, size = SG.paper_sized_scene(g=g)
        with sfm.Sim(sc, stream=stream, place=False) as sim:
            sim.place_sized(sc.xy, sc.heading, sc.goal, np.ones(sc.n, np.uint8), size, size)
            fp = sim.autotune()
            for pi, pmax in enumerate((1, 3, 5, 7, 9, 11)):
                if pmax > 1:
                    per, pha = SG.walk_periods(sc.n, pmax)
                    sim.set_walk_periods(per, pha)
                else:
                    sim.set_walk_periods(None)
                sim.step(max(args.warmup, 9))  # also builds the 8-tick graph
                torch.cuda.synchronize()
                e0 = torch.cuda.Event(enable_timing=True)
                e1 = torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                sim.step(ticks)
                e1.record(stream)
                torch.cuda.synchronize()
                ms = e0.elapsed_time(e1) / ticks
                alive = sim.stats()["alive"]
                rows.append({"ped_side": g, "peds": sc.n, "window": (7 * g) ** 2,
                             "walk_period_max": pmax, "footprint": fp, "ms_per_tick": ms,
                             "ped_steps_per_s": alive / (ms / 1e3),
                             "paper_ms_per_tick": paper[g][pi],
                             "paper_over_this": paper[g][pi] / ms})
    line = {"metric": "pedestrian-steps/s", "value": rows[0]["ped_steps_per_s"],
            "unit": "ped-steps/s", "n_gpus": 1, "steps": ticks, "warmup": args.warmup,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f32",
            "data": "synthetic",
            "config": {"workload": "Table V: pedestrian geometry x maximal walk period, 1000^2 su, "
                                   "half the area covered, 8 directions, fields 7g x 7g"},
            "rows": rows}
    print(json.dumps(line), flush=True)
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=200)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="floor",
                    choices=["floor", "floor-small", "floor-mid", "corridor", "room", "batch",
                             "batch-small",
                             "surrogate", "surrogate-eval", "surrogate-eval-small", "surrogate-eval-mid",
                             "paper-windows", "paper-periods",
                             "paper-sizes", "paper-sweep"])
    ap.add_argument("--bands", type=int, default=None,
                    help="row bands of the divide-and-conquer field pass (1 = unbanded)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--footprint", default="auto", choices=["auto", "16x16", "32x16", "32x32r"],
                    help="field gather footprint: autotuned, or fixed")
    ap.add_argument("--ref-sample", type=int, default=100000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-secondary", action="store_true",
                    help="skip the corridor / room / batch / candidate-only measurements")
    args = ap.parse_args()
    args.warmup = max(3, args.warmup)  # timing rule: at least 3 untimed warm-up ticks
    if args.impl == "reference":
        return run_reference(args)
    if args.workload.startswith("batch"):
        return run_batch(args)
    if args.workload == "surrogate":
        return run_surrogate(args)
    if args.workload in ("surrogate-eval", "surrogate-eval-small", "surrogate-eval-mid"):
        return run_surrogate_eval(args)
    if args.workload.startswith("paper-"):
        return run_paper_sweep(args)
    return run_gpu(args)


if __name__ == "__main__":
    sys.exit(main())
