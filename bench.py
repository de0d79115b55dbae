"""Benchmark: exact 2D convex hull throughput (Mpoints/s) of the gScan hot
path on GB300, one JSON line on stdout.

A step is one pass of the whole pipeline (extremes, quadrilateral filter +
compaction, radix sort, region split + second-round filter, device
finalisation) over the paper-scale workload: two hulls of 20,000,000 int32
points each, (a) uniform in the square [-2^29, 2^29)^2 and (b) uniform in
the disk of radius 2^29.  Each input (160 MB) is larger than L2, and the two
alternate, so every step reads cold inputs from HBM.

--impl reference times the CPU oracle (the project's plain monotone chain)
on the host cores instead, on a bounded sample of the same workload.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "hull Mpoints/s at 20M int32 pts (plain gScan pipeline, square + disk)"
UNIT = "Mpoints/s"
WORKLOAD = "paper-scale: 2 hulls per step, 20M uniform-square + 20M uniform-disk int32 points"
# The paper's best 20M-point times for the same two workloads (Table 3 square
# 446.4 ms, Table 5 circle 418.1 ms, GT 640): 40M points / 864.5 ms.
PAPER_MPTS = 40.0 / 0.8645
# Kernels per hull_compute with the bucket sort, two-read front: extremes,
# witnesses, fused filter (+ bin scan), placement into coarse bins, split
# into bins, bin prefixes, sort (+ second round), compaction, finalisation;
# the single-read front adds the sample polygon before its extremes pass.  A
# call rerun on the radix passes adds extremes, filter count + write, 8
# radix passes, region scan + compact, finalisation.
LAUNCHES_PER_HULL = 9
LAUNCHES_PER_RADIX_RERUN = 1 + 2 + 8 + 2 + 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=20_000_000, help="points per hull")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-clocks", action="store_true")
    ap.add_argument("--no-batched", action="store_true")
    ap.add_argument("--no-learned", action="store_true")
    ap.add_argument("--profile", action="store_true",
                    help="one untimed hull per input set, for a profiler to capture; prints no JSON")
    ap.add_argument("--profile-batched", type=int, default=0, metavar="SEG_MIN",
                    help="two untimed batched calls on a 600-instance batch (sizes log-uniform in "
                         "[1e3, 1e6], 4e7 points at most, seed 11) with the segmented path from SEG_MIN "
                         "points, for a profiler to capture; prints no JSON")
    return ap.parse_args()


def dist_env():
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    return rank, world, local


def workload(n, rank=0):
    """The two input sets of one rank.  Every rank draws its own problems
    (seeds 1+2r and 2+2r), so N ranks solve N independent pairs of hulls."""
    from paper_1508_05931_gb300 import workloads as W
    return [W.paper_square(n, 1 + 2 * rank), W.paper_disk(n, 2 + 2 * rank)]


def max_over_ranks(dist, values, device="cpu"):
    """Element-wise maximum of `values` over every rank (the slowest rank
    sets the job's time); the values themselves with one process."""
    if dist is None:
        return [float(v) for v in values]
    import torch
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.tolist()]


def job_mpts(points_per_rank_step, world, steps, seconds):
    """Whole-job throughput in Mpoints/s: the points all ranks processed
    over the slowest rank's time."""
    return world * points_per_rank_step * steps / seconds / 1e6


def cpu_info():
    model = ""
    try:
        with open("/proc/cpuinfo") as f:
            for line in f:
                if line.lower().startswith(("model name", "cpu part", "hardware")):
                    model = line.split(":", 1)[1].strip()
                    break
    except OSError:
        pass
    return model


def oracle_timing(sets, budget_s=20.0, sample_pts=None):
    """Times the oracle (single-threaded) hull on the sets; returns
    (points processed, seconds, sample description)."""
    import oracle
    oracle.build()
    done, secs, parts = 0, 0.0, []
    for pts in sets:
        p = pts if sample_pts is None else pts[:sample_pts]
        t = time.perf_counter()
        oracle.hull(p)
        dt = time.perf_counter() - t
        done += len(p)
        secs += dt
        parts.append(len(p))
        if secs > budget_s:
            break
    return done, secs, "oracle.hull (qsort + monotone chain, 1 thread) on %s points" % "+".join(map(str, parts))


def _oracle_shard_hull(job):
    """One shard's hull by the oracle: job = (shared-memory name, points in
    the set, first point, end point); returns the hull's points."""
    from multiprocessing import shared_memory
    import numpy as np
    import oracle
    name, n, a, b = job
    shm = shared_memory.SharedMemory(name=name)
    try:
        pts = np.ndarray((n, 2), dtype=np.int32, buffer=shm.buf)[a:b]
        return pts[oracle.hull(pts)].copy()
    finally:
        shm.close()


def oracle_timing_parallel(sets, cores):
    """The oracle on all host cores: every set (in shared memory) cut into
    `cores` contiguous shards whose hulls (oracle.hull, one process each) are
    merged by oracle.hull over their union (the hull of a union is the hull
    of the parts' hulls).  Returns (points, seconds, cores, description)."""
    import multiprocessing as mp
    from multiprocessing import shared_memory
    import numpy as np
    import oracle
    oracle.build()
    ctx = mp.get_context("spawn")          # the parent already drives the GPU
    done, secs = 0, 0.0
    with ctx.Pool(cores) as pool:
        for pts in sets:
            n = len(pts)
            shm = shared_memory.SharedMemory(create=True, size=max(n * 8, 8))
            try:
                np.ndarray((n, 2), dtype=np.int32, buffer=shm.buf)[:] = pts
                cuts = np.linspace(0, n, cores + 1).astype(np.int64)
                jobs = [(shm.name, n, int(cuts[i]), int(cuts[i + 1])) for i in range(cores)]
                pool.map(_oracle_shard_hull, [(shm.name, n, 0, min(n, 4))] * cores)   # workers up and warm
                t = time.perf_counter()
                parts = pool.map(_oracle_shard_hull, jobs)
                oracle.hull(np.concatenate(parts))
                secs += time.perf_counter() - t
                done += n
            finally:
                shm.close()
                shm.unlink()
    return done, secs, cores, ("oracle.hull on %d contiguous shards per set (shared memory) in %d processes, "
                               "then on the union of the shard hulls; %s points"
                               % (cores, cores, "+".join(str(len(p)) for p in sets)))


CLOCK_PAD_S = 0.5


def busy_for(step, seconds):
    """Untimed steps for about `seconds` of wall clock (each step ends with
    a synchronisation)."""
    t0 = time.perf_counter()
    while time.perf_counter() - t0 < seconds:
        step()


class ClockSampler:
    def __init__(self, enabled, index):
        self.proc = None
        # the raw samples (the JSON line carries their summary)
        self.path = os.environ.get("GBH_CLOCKS_CSV", os.path.join(tempfile.gettempdir(), "gbh_clocks_bench.csv"))
        if not enabled:
            return
        try:
            os.makedirs(os.path.dirname(self.path), exist_ok=True)
            self.f = open(self.path, "w")
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(index),
                 "--query-gpu=index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
                 "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
                 "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=self.f, stderr=subprocess.DEVNULL)
        except (OSError, FileNotFoundError):
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        self.f.close()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        with open(self.path) as f:
            for line in f:
                c = [x.strip() for x in line.split(",")]
                if len(c) < 9:
                    continue
                try:
                    sm.append(float(c[1]))
                    mx = float(c[2])
                except ValueError:
                    continue
                for nm, v in zip(names, c[5:9]):
                    if v.lower() == "active":
                        reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm),
                "window": "every 100 ms from %.1f s before to %.1f s after the timed steps, "
                          "the GPU busy with untimed steps throughout" % (CLOCK_PAD_S, CLOCK_PAD_S)}


def bench_batched(hull, torch, stream, plain_value, args):
    """4,096 uneven hulls (log-uniform sizes in [1e3, 1e6], total capped at
    2.5e8 points, square / disk / Gaussian families) in one
    hull_compute_batched call per step."""
    from paper_1508_05931_gb300 import workloads as W
    pts, offs, fam = W.batch()
    dp = torch.as_tensor(pts).cuda()
    do = torch.as_tensor(offs).cuda()
    out = torch.empty(len(pts), dtype=torch.int32, device="cuda")
    oo = torch.empty(len(offs), dtype=torch.int64, device="cuda")
    with hull.Context(torch.cuda.current_device(), autotune=True) as c:
        for _ in range(2):
            c.compute_batched(dp, do, out=out)
        torch.cuda.synchronize()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        k = max(3, args.steps // 4)
        e0.record(stream)
        for _ in range(k):
            _, oo = c.compute_batched(dp, do, out=out)
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / k
    v = len(pts) / (ms / 1e3) / 1e6
    sizes = np.diff(offs)
    tuned = {}
    try:    # the autotuner's choices (its cache: block sizes, segmented-path boundary)
        path = os.environ.get("GBHULL_AUTOTUNE_CACHE") or os.path.expanduser("~/.cache/gbhull_autotune.json")
        with open(path) as f:
            tuned = {k.split("|")[-1]: v_ for k, v_ in json.load(f).items()}
    except (OSError, ValueError):
        pass
    seg_min = tuned.get("batched_seg_min")
    paths = None
    if seg_min:
        seg = sizes >= seg_min
        paths = {"segmented": {"instances": int(seg.sum()), "points": int(sizes[seg].sum())},
                 "one_block": {"instances": int((~seg).sum()), "points": int(sizes[~seg].sum())}}
    return {"value": v, "unit": "Mpoints/s", "ms_per_batch": ms, "instances": len(offs) - 1,
            "points": int(len(pts)), "hull_vertices": int(oo[-1].item()), "steps": k,
            "vs_plain": v / plain_value, "autotuned": tuned, "paths": paths,
            "config": "4096 instances, sizes log-uniform [1e3,1e6] capped at 2.5e8 points total, "
                      "families square/disk/gaussian(2^26), seed 4; one call per step, autotuned"}


def kernel_traffic(kernel, units):
    """DRAM bytes (read + write) per launch of `kernel` from the committed
    ncu capture (profiles/<kernel>_traffic.json), scaled from the units
    (survivors) of the captured launch to `units`, or None when there is no
    capture or a source file it covers changed since."""
    import hashlib
    try:
        with open(os.path.join(ROOT, "profiles", kernel + "_traffic.json")) as f:
            rec = json.load(f)
        for src, want in rec["sources"].items():
            with open(os.path.join(ROOT, src), "rb") as f:
                if hashlib.sha256(f.read()).hexdigest() != want:
                    return None
        return (rec["dram_bytes_read"] + rec["dram_bytes_write"]) * units / rec["units"]
    except (OSError, ValueError, KeyError, AttributeError, TypeError, ZeroDivisionError):
        return None


# Kernel(s) behind each profile stage of the bucket-sort path, and the
# algorithmic bytes each moves per hull: n points, s pairs the fused filter
# passes on (the bucket sort's input), r second-round survivors (8 B per
# point, 12 B per (key, index) pair; K1 copies every 32nd point out for the
# witnesses, which read them back).
SAMPLE_STRIDE = 32
# The last field names the units a committed DRAM traffic record scales by:
# the points a launch reads, or the pairs it moves.
STAGE_KERNELS = {
    "polygon": ("k0_poly", lambda n, s, r: 0.0, "points"),
    "extremes": ("k1_extremes", lambda n, s, r: 8.0 * n + 8.0 * n / SAMPLE_STRIDE, "points"),
    "witness": ("k_witness", lambda n, s, r: 8.0 * n / SAMPLE_STRIDE, "points"),
    "filter": ("k2_fused", lambda n, s, r: 8.0 * n + 12.0 * s, "points"),
    "scatter": ("k2_place", lambda n, s, r: 24.0 * s, "pairs"),
    "split": ("k3_split + k_bin_prefix", lambda n, s, r: 24.0 * s, "pairs"),
    "sort": ("k3_bucket", lambda n, s, r: 12.0 * s + 12.0 * r, "pairs"),
    "regions": ("k4_compact", lambda n, s, r: 24.0 * r, "pairs"),
    "final": ("k5_final", lambda n, s, r: 12.0 * r, "pairs"),
}
# The single-read front (inputs of 65,536 points or more, aligned, no
# statistics): the "polygon" stage is the sample polygon (every 1024th point
# read, 8 B each); the "extremes" stage is the extremes pass that filters
# with it (8 B per point read, the q raw survivors, 12 B each, written); the
# witnesses come from the raw survivors' points (8 B each read); the fused
# filter then reads those q raw survivors and writes the s pairs.  On the
# two-read front the polygon stage is empty.
POLY_STRIDE = 1024
SINGLE_STAGE_KERNELS = dict(STAGE_KERNELS)
SINGLE_STAGE_KERNELS["polygon"] = ("k0_poly", lambda n, s, r, q: 8.0 * n / POLY_STRIDE, "points")
SINGLE_STAGE_KERNELS["extremes"] = ("k1_poly", lambda n, s, r, q: 8.0 * n + 12.0 * q, "points")
SINGLE_STAGE_KERNELS["witness"] = ("k_witness", lambda n, s, r, q: 8.0 * q, "raw")
SINGLE_STAGE_KERNELS["filter"] = ("k2_fused", lambda n, s, r, q: 12.0 * q + 12.0 * s, "raw")
DOMINANT_CANDIDATES = ("polygon", "extremes", "witness", "filter", "scatter", "split", "sort")


def roofline_of(prof, hbm, peak_src):
    """Achieved algorithmic bandwidth of every stage (CUDA events on the
    launch stream, recorded by the library between kernels) and the
    roofline entry of the dominant one (the longest stage)."""
    calls = max(prof["calls"], 1)
    n, s, r = prof["points"] / calls, prof["witness_survivors"] / calls, prof["second_round"] / calls
    single = prof.get("single_read_calls", 0) == prof["calls"] and prof["calls"] > 0
    q = prof.get("raw_survivors", 0) / calls
    table = SINGLE_STAGE_KERNELS if single else STAGE_KERNELS
    stage_ms = {k: v / calls for k, v in prof["ms"].items() if not k.startswith("-")}
    if prof["radix_calls"]:
        return {"bound": "hbm", "kernel": "mixed (calls rerun on the radix passes)", "achieved": None,
                "peak": hbm, "unit": "GB/s", "frac": None, "peak_source": peak_src, "traffic": None,
                "stage_ms_per_hull": stage_ms}
    kernels = {}
    for name, (kern, nbytes, unit) in table.items():
        ms = stage_ms.get(name, 0.0)
        b = nbytes(n, s, r, q) if single and name in ("polygon", "extremes", "witness", "filter") else nbytes(n, s, r)
        units = n if unit == "points" else (q if unit == "raw" else s)
        kernels[name] = {"kernel": kern, "ms": ms, "algorithmic_bytes": b, "units": units,
                         "gbs": b / (ms / 1e3) / 1e9 if ms > 0 else None}
    dom = max(DOMINANT_CANDIDATES, key=lambda k: kernels[k]["ms"])
    d = kernels[dom]
    achieved = d["gbs"] or 0.0
    return {"bound": "hbm", "kernel": d["kernel"], "achieved": achieved, "peak": hbm, "unit": "GB/s",
            "frac": achieved / hbm, "peak_source": peak_src,
            "front": "single-read" if single else "two-read", "raw_survivors_per_hull": q if single else None,
            "traffic": kernel_traffic(d["kernel"].split()[0], d["units"]),
            "algorithmic_bytes_per_launch": d["algorithmic_bytes"],
            "stage_ms_per_hull": stage_ms, "stages": kernels,
            "timing": "CUDA events between the kernels on the launch stream, over a second pass of the timed steps",
            "pipeline_gbs": sum(k["algorithmic_bytes"] for k in kernels.values())
            / (sum(stage_ms.values()) / 1e3) / 1e9 if sum(stage_ms.values()) > 0 else None}


def _ms_per_hull(ctx, t, out, stream, torch, k):
    for _ in range(2):
        ctx.compute_raw(t, out, stream)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(k):
        ctx.compute_raw(t, out, stream)
    e1.record(stream)
    torch.cuda.synchronize()
    return e0.elapsed_time(e1) / k


def _time_hulls(ctx, sctx, t, out, stream, torch, k):
    """ms per hull of `ctx` (no statistics: the path a caller runs), whether
    its learned polygon was used, and the first-round discard fraction of
    its filter polygon from one call of `sctx` (same proposal, statistics
    on: the two-read front, which counts the filter's survivors)."""
    ms = _ms_per_hull(ctx, t, out, stream, torch, k)
    used = ctx.last_stats()["learned_used"]
    sctx.compute_raw(t, out, stream)
    st = sctx.last_stats()
    return ms, 1.0 - st["s"] / st["n"], used


def bench_radix_fallback(hull, torch, stream, k=10):
    """The cost of the radix-pass rerun: 4M points drawn from 40 distinct
    points (coordinates in [-1000, 1000), seed 9), whose duplicates fill a
    bin the bucket sort cannot split, so the call is rerun on the radix
    passes; beside it a 4M uniform disk (seed 12) that the bucket sort takes
    itself.  ms per hull (one call per step) and whether the rerun ran."""
    from paper_1508_05931_gb300 import workloads as W
    rng = np.random.default_rng(9)
    few = rng.integers(-1000, 1000, size=(40, 2)).astype(np.int32)
    cases = [("duplicates_4M", few[rng.integers(0, 40, size=4_000_000)]),
             ("disk_4M", W.uniform_disk(4_000_000, 2.0 ** 29, 12))]
    res = {}
    for name, pts in cases:
        t = torch.as_tensor(np.ascontiguousarray(pts)).cuda()
        o = torch.empty(t.shape[0], dtype=torch.int32, device="cuda")
        with hull.Context(torch.cuda.current_device()) as c:
            ms = _ms_per_hull(c, t, o, stream, torch, k)
        with hull.Context(torch.cuda.current_device(), collect_stats=True) as c:
            c.compute_raw(t, o, stream)
            fb = c.last_stats()["sort_fallback"]
        res[name] = {"ms_per_hull": ms, "sort_fallback": int(fb), "n": int(len(pts))}
    res["rerun_over_disk"] = res["duplicates_4M"]["ms_per_hull"] / res["disk_4M"]["ms_per_hull"]
    return res


def bench_configs(hull, torch, stream, hbm, peak_src, k=20):
    """The other two plain configurations, one hull per step: 100,000
    points uniform in [-2^20, 2^20)^2 (seed 0; its 800 KB stay in L2 between
    steps) and the 4M near-circle ring (seed 3; 32 MB).  Device time per
    hull, throughput, stage times and the roofline entry of each."""
    from paper_1508_05931_gb300 import workloads as W
    res = {}
    for name, pts in (("small_square_100k", W.small_square()), ("near_circle_4M", W.adversarial_ring())):
        t = torch.as_tensor(pts).cuda()
        o = torch.empty(t.shape[0], dtype=torch.int32, device="cuda")
        with hull.Context(torch.cuda.current_device()) as c:
            for _ in range(3):
                c.compute_raw(t, o, stream)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k):
                c.compute_raw(t, o, stream)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            c.set_profiling(True)
            for _ in range(k):
                c.compute_raw(t, o, stream)
            torch.cuda.synchronize()
            prof = c.profile()
        with hull.Context(torch.cuda.current_device(), collect_stats=True) as c:
            c.compute_raw(t, o, stream)
            torch.cuda.synchronize()
            st = c.last_stats()
        res[name] = {"value": len(pts) / (ms / 1e3) / 1e6, "unit": UNIT, "ms_per_hull": ms, "n": len(pts),
                     "first_round_survivors": st["s"], "witness_survivors": st["s_witness"],
                     "second_round": st["r_lower"] + st["r_upper"], "hull_vertices": st["h"],
                     "roofline": roofline_of(prof, hbm, peak_src)}
    return res


def bench_reverse_round(hull, torch, stream, dev_sets, dev_outs):
    """The mirrored second round (opt-in, hull_config.reverse_round) against
    the paper's single second round: ms per hull and second-round survivors
    r on the two 20M sets and the 4M near-circle ring (many near-hull
    points: the case the extra round was aimed at)."""
    from paper_1508_05931_gb300 import workloads as W
    ring = torch.as_tensor(W.adversarial_ring()).cuda()
    ring_out = torch.empty(ring.shape[0], dtype=torch.int32, device="cuda")
    cases = [("square_20M", dev_sets[0], dev_outs[0]), ("disk_20M", dev_sets[1], dev_outs[1]),
             ("near_circle_4M", ring, ring_out)]
    res = {}
    for rev in (False, True):
        with hull.Context(torch.cuda.current_device(), collect_stats=True, reverse_round=rev) as c:
            for name, t, o in cases:
                ms, _, _ = _time_hulls(c, c, t, o, stream, torch, 5)
                st = c.last_stats()
                res.setdefault(name, {})["on" if rev else "off"] = {"ms": ms, "r": st["r_lower"] + st["r_upper"],
                                                                   "h": st["h"]}
    return res


def bench_angular_front(hull, torch, stream, dev_sets):
    """The paper's own ordering (steps 1-7 with the sort by angle about
    P_miny and Figure 2's forward and backward walks) through its stage entry
    point, and the whole angular hull (steps 1-8), on the two 20M sets: ms
    per call (the entries reuse the context's scratch and synchronise),
    first-round and second-round survivors, hull size.  Its failure never
    touches the main line."""
    res = {}
    try:
        with hull.Context(torch.cuda.current_device()) as c:
            for name, t in zip(("square_20M", "disk_20M"), dev_sets):
                order, keep, l = c.stage_angular(t, stream)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(3):
                    order, keep, l = c.stage_angular(t, stream)
                torch.cuda.synchronize()
                ms = (time.perf_counter() - t0) / 3 * 1e3
                hull_idx = c.compute_angular(t, stream)
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                for _ in range(3):
                    hull_idx = c.compute_angular(t, stream)
                torch.cuda.synchronize()
                hull_ms = (time.perf_counter() - t0) / 3 * 1e3
                res[name] = {"ms": ms, "m": int(order.shape[0]), "kept": int(keep.sum().item()),
                             "l_pos": int(l), "hull_ms": hull_ms, "h": int(hull_idx.shape[0]),
                             "timing": "host clock around 3 synchronising calls"}
    except Exception as exc:       # a section of its own: report, do not fail the run
        res["error"] = str(exc)[:200]
    return res


def bench_second_round_ablation(hull, torch, stream, dev_sets):
    """Section 3.4's chunked second round (BLOCK_SIZE = 1024, one block per
    region, one thread per run, as the paper runs it) against the exact scan
    on the same sorted survivors (steps 1-4 on the device): ms and kept
    points, and the share of the input left after each round (Figure 9's
    quantity)."""
    res = {}
    names = ("square_20M", "disk_20M")
    with hull.Context(torch.cuda.current_device()) as c:
        for name, t in zip(names, dev_sets):
            xy, idx = c.stage_sorted_survivors(t, stream)
            row = {"n": int(t.shape[0]), "s": int(xy.shape[0]),
                   "after_round1_pct": 100.0 * xy.shape[0] / t.shape[0]}
            for label, fn in (("exact", lambda: c.stage_second_round(xy, idx, stream)),
                              ("chunked_1024", lambda: c.stage_second_round_chunked(xy, idx, 1024, stream))):
                lo, up = fn()
                torch.cuda.synchronize()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                for _ in range(3):
                    lo, up = fn()
                e1.record(stream)
                torch.cuda.synchronize()
                r = int(lo.shape[0] + up.shape[0])
                row[label] = {"ms": e0.elapsed_time(e1) / 3, "r": r, "after_round2_pct": 100.0 * r / t.shape[0]}
            res[name] = row
    return res


def bench_learned(hull, torch, stream, args):
    """Learned filter proposal vs the plain quadrilateral on the anisotropic
    families at 20M points (single hull: on the path a caller runs, the
    single-read front, where the proposal does not run, and on the two-read
    front, where it does) and as a 1,024-instance batch of the same 20M
    points.  The network is trained first, on the GPU, by the library's own
    kernels (fixed seeds)."""
    from paper_1508_05931_gb300 import learned as L
    dev = torch.cuda.current_device()
    res = {"families": {}}
    with hull.Context(dev, proposal=1, collect_stats=True) as lcs, hull.Context(dev, collect_stats=True) as pcs, \
            hull.Context(dev, proposal=1) as lc, hull.Context(dev) as pc:
        t0 = time.perf_counter()
        X, Y = L.make_dataset(lcs, 192, seed0=1000, lo=1e5, hi=4e5)
        t1 = time.perf_counter()
        losses = L.train(lcs, X, Y, steps=3000, lr=2e-3, batch=64)
        torch.cuda.synchronize()
        lc.mlp_set_params(lcs.mlp_get_params())
        res["training"] = {"instances": 192, "steps": 3000, "data_s": t1 - t0,
                           "train_s": time.perf_counter() - t1,
                           "loss_first": float(np.mean(losses[:20])), "loss_last": float(np.mean(losses[-50:]))}
        out = torch.empty(20_000_000, dtype=torch.int32, device="cuda")
        names = ["anisotropic_gaussian", "elliptic_disk", "gaussian_clusters"]
        k = max(3, args.steps // 4)
        tot_p = tot_l = 0.0
        for fam in range(3):
            pts = torch.as_tensor(L.instance(fam, 20_000_000, 5 + fam)).cuda()
            mp, dp_, _ = _time_hulls(pc, pcs, pts, out, stream, torch, k)
            ml, dl, used = _time_hulls(lc, lcs, pts, out, stream, torch, k)
            # the two-read front (statistics on), where the proposal runs
            mp2 = _ms_per_hull(pcs, pts, out, stream, torch, k)
            ml2 = _ms_per_hull(lcs, pts, out, stream, torch, k)
            used2 = lcs.last_stats()["learned_used"]
            tot_p += mp; tot_l += ml
            res["families"][names[fam]] = {"plain_ms": mp, "learned_ms": ml, "speedup": mp / ml,
                                           "plain_discard": dp_, "learned_discard": dl, "learned_used": used,
                                           "plain_mpts": 20.0 / mp * 1e3, "learned_mpts": 20.0 / ml * 1e3,
                                           "two_read_front": {"plain_ms": mp2, "learned_ms": ml2,
                                                              "speedup": mp2 / ml2, "learned_used": used2}}
            del pts
        res["single_hull"] = {"plain_mpts": 60.0 / tot_p * 1e3, "learned_mpts": 60.0 / tot_l * 1e3,
                              "speedup": tot_p / tot_l}
        # 1,024-instance batch of the same families (19,531 points each)
        parts = [L.instance(i % 3, 19531, 7000 + i) for i in range(1024)]
        offs = np.zeros(1025, np.int64)
        offs[1:] = np.cumsum([len(p) for p in parts])
        bp = torch.as_tensor(np.concatenate(parts)).cuda()
        bo = torch.as_tensor(offs).cuda()
        bout = torch.empty(len(bp), dtype=torch.int32, device="cuda")
        bres = {}
        for name, c in (("plain", pc), ("learned", lc)):
            for _ in range(2):
                c.compute_batched(bp, bo, out=bout)
            torch.cuda.synchronize()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            for _ in range(k):
                c.compute_batched(bp, bo, out=bout)
            e1.record(stream)
            torch.cuda.synchronize()
            ms = e0.elapsed_time(e1) / k
            bres[name] = {"ms": ms, "mpts": len(bp) / (ms / 1e3) / 1e6}
        bres["speedup"] = bres["plain"]["ms"] / bres["learned"]["ms"]
        bres["instances"] = 1024
        bres["points"] = int(len(bp))
        res["batch_1024"] = bres
    return res


def run_reference(args, rank, world):
    if rank != 0:
        return
    sets = workload(args.n)
    sample = min(1_000_000, args.n)
    times = []
    import oracle
    oracle.build()
    for i in range(args.warmup + args.steps):
        t = time.perf_counter()
        for pts in sets:
            oracle.hull(pts[:sample])
        dt = time.perf_counter() - t
        if i >= args.warmup:
            times.append(dt)
    pts_step = sample * len(sets)
    secs = sum(times)
    value = pts_step * len(times) / secs / 1e6
    desc = "first %d points of each 20M set per step (oracle.hull, 1 thread)" % sample
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / len(times),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": value / PAPER_MPTS,
            "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "sample": desc},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle", "sample": desc,
                             "cpu": cpu_info()},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def main():
    args = parse()
    rank, world, local = dist_env()
    if args.impl == "reference":
        run_reference(args, rank, world)
        return
    import torch
    from paper_1508_05931_gb300 import build as _b
    _b.build_library()
    from paper_1508_05931_gb300 import hull

    torch.cuda.set_device(local)
    if args.profile_batched:
        from paper_1508_05931_gb300 import workloads as W
        pts, offs, _ = W.batch(b=600, seed=11, cap=4e7)
        dp, do = torch.as_tensor(pts).cuda(), torch.as_tensor(offs).cuda()
        bout = torch.empty(len(pts), dtype=torch.int32, device="cuda")
        with hull.Context(local, batched_seg_min=args.profile_batched) as c:
            for _ in range(2):
                c.compute_batched(dp, do, out=bout)
        torch.cuda.synchronize()
        return
    dist = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl")

    def barrier():
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()

    sets = workload(args.n, rank)
    dev_sets = [torch.as_tensor(p).cuda() for p in sets]
    out = torch.empty(args.n, dtype=torch.int32, device="cuda")
    dev_outs = [torch.empty(len(p), dtype=torch.int32, device="cuda") for p in sets]
    ctx = hull.Context(local)
    stream = torch.cuda.current_stream()
    if args.profile:
        for t in dev_sets:
            ctx.compute_raw(t, out, stream)
        torch.cuda.synchronize()
        ctx.close()
        return

    def step():
        # One hull_compute_multi call per step: the step's hulls run on the
        # library's two lanes.
        ctx.compute_multi(dev_sets, dev_outs, stream)

    for _ in range(max(args.warmup, 3)):
        step()
    # The clock samples (every 100 ms) bracket the timed steps: untimed steps
    # keep the GPU busy for CLOCK_PAD_S before and after them, so that a
    # timed region shorter than the sampling interval still has samples
    # taken under the same load around it.
    sampler = ClockSampler(not args.no_clocks and rank == 0, local)
    if sampler.proc is not None:
        busy_for(step, CLOCK_PAD_S)
    barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(args.steps):
        step()
    e1.record(stream)
    barrier()
    if sampler.proc is not None:
        busy_for(step, CLOCK_PAD_S)
    clocks = sampler.stop()
    ms = e0.elapsed_time(e1)
    # Stage durations: the same steps again with the library's CUDA events
    # between kernels (on the launch stream).  The events cost a few percent
    # of the step, so `value` is timed without them.
    ctx.set_profiling(True)
    for _ in range(args.steps):
        step()
    torch.cuda.synchronize()
    prof = ctx.profile()
    ctx.set_profiling(False)
    ms = max_over_ranks(dist, [ms], "cuda")[0]
    pts_step = sum(len(p) for p in sets)
    value = job_mpts(pts_step, world, args.steps, ms / 1e3)

    # e2e: the same steps through the host entry point (pinned host input,
    # H2D copy, compute, D2H of the vertex indices inside the timed region):
    # one hull_compute_host_multi call per step, which copies the second set
    # while the first one's hull is computed.
    host_sets = [torch.as_tensor(p).pin_memory() for p in sets]
    host_outs = [torch.empty(len(p), dtype=torch.int32).pin_memory() for p in sets]
    h_counts = []

    def host_step():
        h_counts.clear()
        for r in ctx.compute_host_multi(host_sets, outs=host_outs, stream=stream):
            h_counts.append(len(r))

    for _ in range(2):
        host_step()
    barrier()
    t0 = time.perf_counter()
    k_e2e = max(3, args.steps // 2)
    for _ in range(k_e2e):
        host_step()
    barrier()
    e2e_s = max_over_ranks(dist, [time.perf_counter() - t0], "cuda")[0]
    e2e_val = job_mpts(pts_step, world, k_e2e, e2e_s)

    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except (OSError, ValueError):
        pass
    hbm = float(peaks.get("hbm_gbs", 6800.0))
    peak_src = "measured" if "hbm_gbs" in peaks else "fallback"

    roofline = roofline_of(prof, hbm, peak_src)
    calls = max(prof["calls"], 1)
    # First-round survivors: the fused filter counts them only for a context
    # that collects statistics (one untimed hull per set).
    first_round, witness = [], []
    with hull.Context(local, collect_stats=True) as sc:
        for t in dev_sets:
            sc.compute_raw(t, out, stream)
            torch.cuda.synchronize()
            st = sc.last_stats()
            first_round.append(st["s"])
            witness.append(st["s_witness"])

    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": value / PAPER_MPTS, "dtype": "int32", "data": "synthetic",
            "config": {"workload": WORKLOAD, "points_per_step": pts_step, "hulls_per_step": len(sets),
                       "l2": "inputs larger than L2 (160 MB each, alternating)",
                       "parallelism": "replicas" if world > 1 else "single GPU",
                       "survivors_per_hull": sum(first_round) / len(first_round),
                       "witness_survivors_per_hull": prof["witness_survivors"] / calls,
                       "second_round_per_hull": prof["second_round"] / calls},
            "gpu_launches": prof["calls"] * LAUNCHES_PER_HULL + prof.get("single_read_calls", 0)
            + prof["radix_calls"] * LAUNCHES_PER_RADIX_RERUN,
            "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": 8 * pts_step,
                    "d2h_bytes_per_step": 4 * sum(h_counts), "api": "hull_compute_host_multi"},
            "roofline": roofline}
    if clocks:
        line["clocks"] = clocks
    # The batched and learned sections and the CPU baseline are single-GPU
    # measurements: with several ranks only the replicated plain pipeline runs.
    if world == 1 and not args.no_batched:
        line["batched"] = bench_batched(hull, torch, stream, value, args)
    if world == 1 and not args.no_learned:
        line["learned"] = bench_learned(hull, torch, stream, args)
    if world == 1:
        line["configs"] = bench_configs(hull, torch, stream, hbm, peak_src)
        line["radix_fallback"] = bench_radix_fallback(hull, torch, stream)
    if world == 1 and not args.no_batched:
        line["reverse_round"] = bench_reverse_round(hull, torch, stream, dev_sets, dev_outs)
        line["second_round_ablation"] = bench_second_round_ablation(hull, torch, stream, dev_sets)
        line["angular_front"] = bench_angular_front(hull, torch, stream, dev_sets)
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        done, secs, desc = oracle_timing(sets)
        line["cpu_baseline"] = {"value": done / secs / 1e6, "unit": UNIT, "cores": 1, "kind": "oracle",
                                "sample": desc, "cpu": cpu_info(), "nproc": os.cpu_count()}
        pdone, psecs, pcores, pdesc = oracle_timing_parallel(sets, os.cpu_count() or 1)
        line["cpu_baseline_all_cores"] = {"value": pdone / psecs / 1e6, "unit": UNIT, "cores": pcores,
                                          "kind": "oracle", "sample": pdesc}
    ctx.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
