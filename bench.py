"""Benchmark: radius-search throughput on the 12M-point ALS tile.

Workload (one step = the whole hot path once): build the 2D dense grid index
(1 m voxels) of a 12,000,000-point synthetic ALS tile (500 m x 500 m, UTM
offsets, terrain + buildings + trees), then the two-pass fixed-radius sphere
search with every point as a query (count, scan, fill with rows sorted by
original id) at r = 1 m.  Inputs are resident in HBM when the timed region
starts; they are 288 MB, larger than the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                  [--workload tile|batched|serving]

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on
the host cores instead (bounded sample of the same workload).  The other
workloads: `batched` = 256 tiles (~60M points) through the graph-captured
pipeline (build + radius r = 1 m + k-NN k = 16), binary32-offset and binary64
storage side by side; `serving` = 8 resident indexes under a Poisson stream
of radius / k-NN requests (p50 / p99 latency and queries/s).
"""
from __future__ import annotations

import argparse
import hashlib
import json
import math
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "radius-search queries/s (12M-pt ALS tile, every point a query, r=1 m)"
UNIT = "queries/s"
N_POINTS = 12_000_000
RADIUS = 1.0
CELL = 1.0


def _peaks():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons while running."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.thread = threading.Thread(target=self._read, daemon=True)
            self.thread.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self) -> dict:
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def _src_hash(names) -> str:
    h = hashlib.sha256()
    for n in names:
        with open(os.path.join(ROOT, "paper_2502_11602_gb300", "csrc", n), "rb") as f:
            h.update(f.read())
    return h.hexdigest()[:16]


def _traffic(kernel: str, src_files) -> float | None:
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current source of the kernel."""
    path = os.path.join(ROOT, "profiles", "traffic_radius_als12m.txt")
    try:
        with open(path) as f:
            t = json.load(f)
        ent = t[kernel]
        if ent.get("src_hash") != _src_hash(src_files):
            return None
        return float(ent["dram_bytes_per_launch"])
    except Exception:
        return None


def _setup_dist(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if args.impl == "ours" else "gloo"
        dist.init_process_group(backend=backend)
    return rank, world, local, dist


def _max_over_ranks(x: float, dist, device) -> float:
    """The slowest rank's value (every rank gets it); x itself on one rank."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def _sum_over_ranks(x: float, dist, device) -> float:
    """Total over ranks (units of work processed by the whole job)."""
    if dist is None:
        return x
    import torch
    t = torch.tensor([x], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.SUM)
    return float(t.item())


def _tile_config(n: int, precision: str, world: int) -> dict:
    """The tile workload's config (the same dict on both arms)."""
    return {"workload": "ALS tile 12M pts, 500x500 m, 2D dense grid 1 m, sphere r=1 m, all points as queries",
            "n_points": n, "radius_m": RADIUS, "cell_m": CELL, "precision": precision,
            "l2": "inputs larger than L2 (288 MB points, 129 MB L2)", "parallelism": f"replicas x{world}"}


def _single_core(xyz, sample_queries: int, seed: int = 6) -> dict:
    """The oracle on one thread: the whole small ALS tile (100k points, every
    point a query, r = 1 m) and a seeded 1 % query sample of the large tile,
    extrapolated to every point as a query (labelled as such)."""
    import numpy as np

    import cloudgen
    import oracle
    small = cloudgen.als_uniform()
    t0 = time.perf_counter()
    six = oracle.Index(small, CELL)
    six.radius_search(small, RADIUS, oracle.SPHERE, threads=1)
    t_small = time.perf_counter() - t0
    ix = oracle.Index(xyz, CELL)
    q = xyz[np.random.default_rng(seed).integers(0, len(xyz), sample_queries)]
    t0 = time.perf_counter()
    ix.radius_search(q, RADIUS, oracle.SPHERE, threads=1)
    t_q = time.perf_counter() - t0
    return {"cores": 1,
            "small_tile_queries_per_s": len(small) / t_small,
            "small_tile": f"{len(small)} points, build + every point a query, one thread ({t_small:.2f} s)",
            "large_tile_sample_queries_per_s": sample_queries / t_q,
            "large_tile_sample": f"{sample_queries} seeded random queries of the {len(xyz)}-point tile "
                                 f"(1 %), one thread ({t_q:.2f} s); queries only, extrapolation: "
                                 f"{len(xyz) / (sample_queries / t_q):.0f} s for every point as a query"}


def _cpu_baseline(xyz, sample_queries: int, seed: int = 5):
    """The oracle as it stands, on the host cores: full single-threaded build
    plus a seeded sample of queries on all cores, extrapolated to N queries."""
    import numpy as np

    import oracle
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ix = oracle.Index(xyz, CELL)
    t_build = time.perf_counter() - t0
    rng = np.random.default_rng(seed)
    q = xyz[rng.integers(0, len(xyz), sample_queries)]
    t0 = time.perf_counter()
    off, ind = ix.radius_search(q, RADIUS, oracle.SPHERE, threads=cores)
    t_q = time.perf_counter() - t0
    t_all = t_build + t_q * len(xyz) / sample_queries
    return {"value": len(xyz) / t_all, "unit": UNIT, "cores": cores, "kind": "oracle",
            "sample": f"full single-threaded oracle build of the {len(xyz)}-point tile ({t_build:.1f} s) + "
                      f"{sample_queries} seeded random queries on {cores} threads ({t_q:.1f} s), "
                      f"query time extrapolated to all {len(xyz)} queries",
            "build_s": t_build, "query_sample_s": t_q,
            "single_core": _single_core(xyz, len(xyz) // 100)}


def run_reference(args):
    import numpy as np

    import cloudgen
    import oracle
    rank, world, local, dist = _setup_dist(args)
    if rank != 0:
        if dist is not None:
            dist.destroy_process_group()
        return
    xyz = cloudgen.als_urban(N_POINTS)
    cores = os.cpu_count() or 1
    t0 = time.perf_counter()
    ix = oracle.Index(xyz, CELL)
    t_build = time.perf_counter() - t0
    S = args.ref_sample
    rng = np.random.default_rng(17)
    times = []
    for step in range(args.warmup + args.steps):
        q = xyz[rng.integers(0, len(xyz), S)]
        t0 = time.perf_counter()
        ix.radius_search(q, RADIUS, oracle.SPHERE, threads=cores)
        dt = time.perf_counter() - t0
        if step >= args.warmup:
            times.append(dt)
    t_q = statistics.mean(times)
    # the timed region: each step is one sample of S queries (count + fill,
    # rows sorted) against the resident oracle index
    value = S / t_q
    t_full = t_build + t_q * len(xyz) / S  # a whole step, extrapolated (labelled below)
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_q * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": _tile_config(len(xyz), args.precision, args.gpus),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"each step: {S} seeded random queries of the {len(xyz)}-point tile on "
                                       f"{cores} threads against the oracle index built once before the timed "
                                       f"region ({t_build:.1f} s, one thread); value = sample queries / step time"},
            "extrapolated_full_step": {"ms": t_full * 1e3, "queries_per_s": len(xyz) / t_full,
                                       "how": "oracle build + the sample's per-query time x every point as a query "
                                              "(not timed as one region)"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def _alg_tests(xyz, r: float, cell: float) -> int:
    """Candidate tests of Algorithm 1 with every point as a query on a 2D
    dense grid: for each query, the points of every voxel that meets its
    kernel's bounding box [c - r, c + r] in x and y (z is not indexed).
    Counted with a summed-area table of the voxel counts."""
    import numpy as np
    lo = xyz[:, :2].min(0)
    hi = xyz[:, :2].max(0)
    nx, ny = (np.floor((hi - lo) / cell).astype(np.int64) + 1).tolist()
    ij = np.floor((xyz[:, :2] - lo) / cell).astype(np.int64)
    cnt = np.bincount(ij[:, 0] * ny + ij[:, 1], minlength=nx * ny).reshape(nx, ny)
    sat = np.zeros((nx + 1, ny + 1), np.int64)
    sat[1:, 1:] = cnt.cumsum(0).cumsum(1)
    total = 0
    for a in range(0, len(xyz), 4_000_000):
        c = xyz[a:a + 4_000_000, :2]
        i0 = np.clip(np.floor((c[:, 0] - r - lo[0]) / cell).astype(np.int64), 0, nx - 1)
        i1 = np.clip(np.floor((c[:, 0] + r - lo[0]) / cell).astype(np.int64), 0, nx - 1)
        j0 = np.clip(np.floor((c[:, 1] - r - lo[1]) / cell).astype(np.int64), 0, ny - 1)
        j1 = np.clip(np.floor((c[:, 1] + r - lo[1]) / cell).astype(np.int64), 0, ny - 1)
        total += int((sat[i1 + 1, j1 + 1] - sat[i0, j1 + 1] - sat[i1 + 1, j0] + sat[i0, j0]).sum())
    return total


# binary32 lane operations of one sphere test: 3 subtractions, 1 multiply,
# 2 fused multiply-adds, 1 comparison
OPS_PER_TEST = 7
# sources of the kernels whose DRAM traffic profiles/traffic_radius_als12m.txt records
TRAFFIC_SRC = ["cg_radius2.cu", "cg_f32x2.cuh", "cg_query.cu", "cg_query.cuh", "cg_internal.cuh", "cg_zwin.cu"]
COUNT_PHASES = ("radius_count5_512", "radius_count5_1k", "radius_count5_2k", "radius_count2", "radius_v1_count")
FILL_PHASES = ("radius_fill5_512", "radius_fill5_1k", "radius_fill5_2k", "radius_fill2", "radius_v1_fill",
               "radius_row_sort")


def run_ours(args):
    import numpy as np
    import torch

    import cloudgen
    import paper_2502_11602_gb300 as cg

    rank, world, local, dist = _setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    # weak scaling: each rank owns an independent tile (replicas, no exchange)
    npts = args.points
    side = 500.0 * math.sqrt(npts / N_POINTS)  # same density as the 12M tile
    xyz = cloudgen.als_urban(npts, extent=(side, side), seed=cloudgen.CONFIG_SEED + 1 + 1000 * rank,
                             n_buildings=max(1, round(200 * npts / N_POINTS)),
                             n_trees=max(1, round(3000 * npts / N_POINTS)))
    n = xyz.shape[0]
    x = torch.from_numpy(xyz).to(dev)
    stream = torch.cuda.current_stream(dev)
    cg.load()

    prec = cg.FP32_OFFSET if args.precision == "fp32" else cg.FP64

    def step(record=None, p=prec):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record is not None else None
        if ev: ev[0].record(stream)
        h = cg.cg_build(x, CELL, CELL, 2, cg.DENSE, p)
        if ev: ev[1].record(stream)
        off = torch.empty(n + 1, dtype=torch.int64, device=dev)
        total = cg.cg_all_points_count(h, RADIUS, cg.SPHERE, off)
        if ev: ev[2].record(stream)
        ind = torch.empty(total, dtype=torch.int32, device=dev)
        cg.cg_all_points_fill(h, RADIUS, cg.SPHERE, off, ind)
        if ev: ev[3].record(stream)
        cg.cg_index_free(h)
        if record is not None:
            record.append(ev)
        return total

    # the sampler starts before the warm-up: nvidia-smi's start-up stalls
    # CUDA calls of this process for tens of ms and must not fall in the
    # timed region
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)
    for _ in range(args.warmup):
        total = step()
    torch.cuda.synchronize()

    records = []
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    cg.cg_profile_read(reset=True)
    cg.cg_profile_enable(True)
    launches0 = cg.cg_launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        total = step(records)
    t1.record(stream)
    torch.cuda.synchronize()
    launches = (cg.cg_launch_count() - launches0) / args.steps
    cg.cg_profile_enable(False)
    phases = cg.cg_profile_read(reset=True)
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = _max_over_ranks(t0.elapsed_time(t1) / args.steps, dist, dev)
    build_ms = statistics.mean(r[0].elapsed_time(r[1]) for r in records)
    count_ms = statistics.mean(r[1].elapsed_time(r[2]) for r in records)
    fill_ms = statistics.mean(r[2].elapsed_time(r[3]) for r in records)

    # end to end through the public API: pinned host points in, CSR out.
    # Serial: one step at a time, synchronized.  Pipelined (the reported
    # figure): step i+1's points go up on one copy stream while step i
    # computes, and step i's CSR comes back on another while step i+1
    # computes; every step still moves its own inputs and results.
    host_in = torch.from_numpy(xyz).pin_memory()
    host_off = [torch.empty(n + 1, dtype=torch.int64).pin_memory() for _ in range(2)]
    host_ind = [torch.empty(total, dtype=torch.int32).pin_memory() for _ in range(2)]
    serial = []
    for it in range(3):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        xd = torch.empty((n, 3), dtype=torch.float64, device=dev)
        xd.copy_(host_in, non_blocking=True)
        ix = cg.Index(xd, CELL, CELL, 2, cg.DENSE, prec)
        off, ind = ix.radius_search(None, RADIUS, cg.SPHERE, check=False)
        host_off[0].copy_(off, non_blocking=True)
        host_ind[0][:ind.numel()].copy_(ind, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        ix.close()
        del xd, off, ind
        if it > 0:
            serial.append(a.elapsed_time(b))
    # all three on pool streams: work on the legacy default stream would wait
    # for the copies of blocking streams
    comp, up, down = torch.cuda.Stream(dev), torch.cuda.Stream(dev), torch.cuda.Stream(dev)
    xin = [torch.empty((n, 3), dtype=torch.float64, device=dev) for _ in range(2)]
    ready = [torch.cuda.Event() for _ in range(2)]
    freed = [torch.cuda.Event() for _ in range(2)]
    for e in freed:
        e.record(comp)

    def upload(i):
        up.wait_event(freed[i % 2])
        with torch.cuda.stream(up):
            xin[i % 2].copy_(host_in, non_blocking=True)
        ready[i % 2].record(up)

    e2e_steps = max(4, min(args.steps, 10))
    torch.cuda.synchronize()
    a = torch.cuda.Event(enable_timing=True)
    b = torch.cuda.Event(enable_timing=True)
    with torch.cuda.stream(comp):
        a.record(comp)
        upload(0)
        for i in range(e2e_steps):
            comp.wait_event(ready[i % 2])
            ix = cg.Index(xin[i % 2], CELL, CELL, 2, cg.DENSE, prec)  # copies the points
            freed[i % 2].record(comp)
            if i + 1 < e2e_steps:
                upload(i + 1)
            off, ind = ix.radius_search(None, RADIUS, cg.SPHERE, check=False)
            down.wait_stream(comp)
            with torch.cuda.stream(down):
                host_off[i % 2].copy_(off, non_blocking=True)
                host_ind[i % 2][:ind.numel()].copy_(ind, non_blocking=True)
            off.record_stream(down)
            ind.record_stream(down)
            ix.close()
            del off, ind
        comp.wait_stream(down)
        b.record(comp)
    torch.cuda.synchronize()
    e2e_ms = a.elapsed_time(b) / e2e_steps
    e2e_serial_ms = statistics.mean(serial)

    n_all = _sum_over_ranks(n, dist, dev)          # queries of the whole job
    total_all = _sum_over_ranks(total, dist, dev)  # neighbours of the whole job
    value = n_all / (ms * 1e-3)
    peak, peak_kind = _peaks()
    per_step = {k: v[1] / args.steps for k, v in phases.items()}
    # the count (fill) kernels of one pass run concurrently on forked
    # streams: their device time is the span of the enclosing trace scope
    count_k = per_step.get("radius_count_kernels", sum(per_step.get(k, 0.0) for k in COUNT_PHASES))
    fill_k = per_step.get("radius_fill_kernels", sum(per_step.get(k, 0.0) for k in FILL_PHASES))
    ncell = int(math.floor((xyz[:, 0].max() - xyz[:, 0].min()) / CELL) + 1) * \
        int(math.floor((xyz[:, 1].max() - xyz[:, 1].min()) / CELL) + 1)
    tests = _alg_tests(xyz, RADIUS, CELL)
    # the count kernels are bound by the binary32 tests, not by memory; the
    # fill kernels by writing the CSR; the longer of the two is reported as
    # the dominant kernel, the other beside it
    sm_mhz = float(clk.get("sm_max_mhz") or 2070.0)
    alu_peak = 152 * 128 * sm_mhz * 1e6 / 1e12  # T lane-ops/s
    achieved = OPS_PER_TEST * tests / (count_k * 1e-3) / 1e12
    roof_count = {"bound": "alu", "kernel": "concurrent " + "+".join(k for k in COUNT_PHASES if k in per_step),
                  "achieved": achieved, "peak": alu_peak, "unit": "T lane-ops/s", "frac": achieved / alu_peak,
                  "peak_kind": "derived: 152 SMs x 128 FP32 lanes x max SM clock",
                  "traffic": _traffic("radius_count_kernels", TRAFFIC_SRC),
                  "algorithmic_tests": tests, "ops_per_test": OPS_PER_TEST, "ms_per_launch": count_k}
    alg = 16 * n + 4 * (ncell + 1) + 8 * (n + 1) + 4 * total
    achieved = alg / (fill_k * 1e-3) / 1e9
    roof_fill = {"bound": "hbm", "kernel": "concurrent " + "+".join(k for k in FILL_PHASES if k in per_step),
                 "achieved": achieved, "peak": peak, "peak_kind": peak_kind, "unit": "GB/s",
                 "frac": achieved / peak,
                 "traffic": _traffic("radius_fill_kernels", TRAFFIC_SRC),
                 "algorithmic_bytes": alg, "ms_per_launch": fill_k}
    roof, roof_other = (roof_count, roof_fill) if count_k >= fill_k else (roof_fill, roof_count)

    # the whole step against HBM, from the bytes-touched model of one build +
    # count + fill (binary32 records): build reads the points (24 B) and
    # writes keys, sorted keys and ids (12 B), records (16 B) and the exact
    # copy (24 B); each query pass reads the records (16 B/pt) and the cell
    # table; count writes counts and the offsets (4 + 8 B/query); fill reads
    # the offsets (8 B/query) and writes 4 B per neighbour
    model = {"build": 24 * n + 12 * n + 16 * n + 24 * n,
             "count": 16 * n + 4 * (ncell + 1) + 12 * n,
             "fill": 16 * n + 4 * (ncell + 1) + 8 * n + 4 * total}
    model_bytes = sum(model.values())
    hbm_model = {"bytes_per_step": model_bytes, "terms": model,
                 "achieved_gbs": model_bytes / (ms * 1e-3) / 1e9, "peak_gbs": peak, "peak_kind": peak_kind,
                 "frac": model_bytes / (ms * 1e-3) / 1e9 / peak,
                 "alu_floor_ms": OPS_PER_TEST * tests / (152 * 128 * 2070e6) * 1e3}

    # secondary measurements on the same tile: k-NN (k = 16) and the binary64 path
    h = cg.cg_build(x, CELL, CELL, 2, cg.DENSE, prec)
    # the candidate tests the count kernels run (height ranges cut Algorithm
    # 1's voxel scan), from one count pass
    _off = torch.empty(n + 1, dtype=torch.int64, device=dev)
    cg.cg_all_points_count(h, RADIUS, cg.SPHERE, _off)
    rstats = cg.cg_radius_stats(h)
    del _off
    roof_count["executed_tests"] = rstats["tested_pairs"]
    roof_count["executed_over_algorithmic"] = rstats["tested_pairs"] / tests if tests else None
    roof_count["executed_lane_ops_per_s"] = OPS_PER_TEST * rstats["tested_pairs"] / (count_k * 1e-3) / 1e12
    kidx = torch.empty((n, 16), dtype=torch.int32, device=dev)
    kd2 = torch.empty((n, 16), dtype=torch.float64, device=dev)
    kt = []
    for it in range(3):
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        cg.cg_all_points_knn(h, 16, kidx, kd2)
        b.record(stream)
        torch.cuda.synchronize()
        if it > 0:
            kt.append(a.elapsed_time(b))
    cg.cg_index_status(h)
    cg.cg_index_free(h)
    del kidx, kd2
    fp64_ms = None
    if prec == cg.FP32_OFFSET and not args.no_fp64:
        step(p=cg.FP64)
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(2):
            step(p=cg.FP64)
        b.record(stream)
        torch.cuda.synchronize()
        fp64_ms = a.elapsed_time(b) / 2

    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == cg.FP32_OFFSET else "f64", "data": "synthetic",
        "config": _tile_config(n, args.precision, world),
        "neighbors_per_s": total_all / (ms * 1e-3), "neighbors_per_step": total_all,
        "stages_ms": {"build": build_ms, "count": count_ms, "fill": fill_ms},
        "kernels_ms_per_step": per_step,
        "e2e": {"value": n_all / (_max_over_ranks(e2e_ms, dist, dev) * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                "pipelined_steps": e2e_steps, "serial_ms_per_step": e2e_serial_ms,
                "h2d_bytes_per_step": n * 24, "d2h_bytes_per_step": (n + 1) * 8 + total * 4},
        "roofline": roof, "roofline_other": roof_other, "hbm_model": hbm_model, "clocks": clk,
        "gpu_launches": launches,
        "knn16": {"queries_per_s": n_all / (_max_over_ranks(statistics.mean(kt), dist, dev) * 1e-3),
                  "ms": statistics.mean(kt)},
    }
    if fp64_ms is not None:
        line["fp64_path"] = {"queries_per_s": n_all / (_max_over_ranks(fp64_ms, dist, dev) * 1e-3),
                             "ms_per_step": fp64_ms}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(xyz, args.cpu_sample)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_batched(args):
    """256 tiles (~60M points) through the graph-captured pipeline: build +
    all-points radius r = 1 m + all-points k-NN k = 16, one graph replay per
    step, binary32-offset storage against binary64 storage."""
    import numpy as np
    import torch

    import cloudgen
    import paper_2502_11602_gb300 as cg
    from paper_2502_11602_gb300 import autotune

    rank, world, local, dist = _setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    stream = torch.cuda.current_stream(dev)
    xyz, off = cloudgen.batched_tiles(args.tiles, args.batch_points, seed=cloudgen.CONFIG_SEED + 3 + 1000 * rank)
    n = len(xyz)
    x = torch.from_numpy(xyz).to(dev)
    cache = os.path.join(ROOT, "_build", "autotune.json")
    cells, report = autotune.tune(xyz, off, radius=1.0, k=16, precision=cg.FP32_OFFSET, cache_path=cache)
    # launch shapes for the captured batch, timed on the batch itself
    shapes, launch_report = autotune.tune_pipeline(x, off, cells, radius=1.0, k=16, precision=cg.FP32_OFFSET,
                                                   cache_path=cache)
    tuning = dict(cg.cg_get_tuning(), **shapes)
    out = {}
    clocks = ClockSampler(local)
    clocks.start()
    time.sleep(1.0)
    for name, prec, tun in (("fp32", cg.FP32_OFFSET, tuning), ("fp32_default_shapes", cg.FP32_OFFSET, None),
                            ("fp64", cg.FP64, None)):
        cg.cg_set_tuning(tun)  # launch shapes are fixed when the pipeline's graph is captured
        pipe = cg.Pipeline(x, off, cells, radius=1.0, k=16, precision=prec)
        for _ in range(args.warmup):
            total = pipe.run()
        if dist is not None:
            dist.barrier()
        torch.cuda.synchronize()
        l0 = cg.cg_launch_count()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        for _ in range(args.steps):
            pipe.run(sync=False)
        b.record(stream)
        torch.cuda.synchronize()
        launches = (cg.cg_launch_count() - l0) / args.steps
        total = pipe.run()  # synchronising check: no re-plan, no device error
        assert pipe.info()["replans"] == 0
        ms = _max_over_ranks(a.elapsed_time(b) / args.steps, dist, dev)
        info = pipe.info()
        if name == "fp32_default_shapes":
            out[name] = {"ms_per_step": ms, "queries_per_s": world * n / (ms * 1e-3)}
            pipe.close()
            continue
        # end to end: pinned host points in, CSR and k-NN out, every step
        host_in = torch.from_numpy(xyz).pin_memory()
        outs = pipe.outputs()
        host = {k: torch.empty(v.shape, dtype=v.dtype).pin_memory() for k, v in outs.items()}
        et = []
        for it in range(3):
            torch.cuda.synchronize()
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            x.copy_(host_in, non_blocking=True)
            t = pipe.run()
            o = pipe.outputs()
            for k, v in o.items():
                host[k][:v.shape[0]].copy_(v, non_blocking=True)
            e1.record(stream)
            torch.cuda.synchronize()
            if it > 0:
                et.append(e0.elapsed_time(e1))
        e2e_ms = statistics.mean(et)
        out[name] = {"ms_per_step": ms, "queries_per_s": world * n / (ms * 1e-3),
                     "neighbors_per_s": world * total / (ms * 1e-3), "neighbors_per_step": total,
                     "graph_kernels": info["graph_kernels"], "gpu_launches": launches,
                     "device_bytes": info["device_bytes"],
                     "e2e_ms": e2e_ms, "e2e_queries_per_s": world * n / (e2e_ms * 1e-3),
                     "d2h_bytes": int(sum(v.numel() * v.element_size() for v in o.values()))}
        pipe.close()
        del host_in, host, outs, o
    clk = clocks.stop()
    cg.cg_set_tuning(None)
    f = out["fp32"]
    line = {
        "metric": "batched radius+kNN queries/s (256 ALS tiles, ~60M pts, r=1 m, k=16, one graph replay per step)",
        "value": f["queries_per_s"], "unit": "queries/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": f["ms_per_step"], "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": f"{args.tiles} ALS-like tiles, {n} pts, density 5-60 pts/m2, log-uniform sizes "
                               "10k-2M, 2D dense grids, cell autotuned per density bucket, sphere r=1 m, k=16",
                   "n_points": n, "tiles": args.tiles, "cells_used": sorted(set(cells.tolist())),
                   "autotune_report": {str(k): v for k, v in report.items()},
                   "launch_tuning": tuning,
                   "launch_tuning_report": {str(k): v for k, v in launch_report.items()},
                   "l2": "inputs larger than L2 (1.4 GB points)"},
        "fp32_offset": f, "fp64": out["fp64"],
        "fp32_default_shapes": out["fp32_default_shapes"],
        "tuned_over_default_shapes": out["fp32_default_shapes"]["ms_per_step"] / f["ms_per_step"],
        "fp32_over_fp64": out["fp64"]["ms_per_step"] / f["ms_per_step"],
        "e2e": {"value": f["e2e_queries_per_s"], "unit": "queries/s", "h2d_bytes_per_step": n * 24,
                "d2h_bytes_per_step": f["d2h_bytes"]},
        "clocks": clk, "gpu_launches": f["gpu_launches"],
    }
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_serving(args):
    """8 resident indexes (ALS and TLS clouds of 5-30M points, binary32
    offsets) under a Poisson stream of requests: query sets of log-uniform
    size in [1k, 1M] drawn from the index's points, each a sphere radius
    (U[0.25, 3] m on ALS, U[0.05, 0.5] m on TLS) or a k-NN with k in
    {8, 16, 32} (even odds).  Offered load
    swept in steps up to saturation; p50 / p99 latency and queries/s."""
    import numpy as np
    import torch

    import cloudgen
    import paper_2502_11602_gb300 as cg

    rank, world, local, dist = _setup_dist(args)
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    rng = np.random.default_rng(cloudgen.CONFIG_SEED + 4 + 1000 * rank)
    sizes = [int(v) for v in np.round(np.exp(rng.uniform(np.log(5e6), np.log(30e6), 8)) * args.serve_scale)]
    clouds, indexes, cells = [], [], []
    for i, m in enumerate(sizes):
        if i % 2 == 0:
            side = 500.0 * math.sqrt(m / N_POINTS)
            c = cloudgen.als_urban(m, extent=(side, side), seed=cloudgen.CONFIG_SEED + 40 + i,
                                   n_buildings=max(1, round(200 * m / N_POINTS)),
                                   n_trees=max(1, round(3000 * m / N_POINTS)))
            cell, dim = 1.0, 2
        else:
            c = cloudgen.tls_street(m, seed=cloudgen.CONFIG_SEED + 40 + i)
            cell, dim = 0.25, 3
        x = torch.from_numpy(c).to(dev)
        indexes.append(cg.Index(x, cell, cell, dim=dim, precision=cg.FP32_OFFSET))
        clouds.append(x)
        cells.append(cell)
    # requests, queries staged on the device beforehand
    nreq = args.serve_requests
    reqs = []
    for i in range(nreq):
        j = int(rng.integers(0, 8))
        nq = int(np.exp(rng.uniform(np.log(1e3), np.log(1e6))))
        sel = torch.from_numpy(rng.integers(0, clouds[j].shape[0], nq)).to(dev)
        q = clouds[j][sel].contiguous()
        if rng.random() < 0.5:
            # ALS indexes: r ~ U[0.25, 3] m; TLS indexes (3D, up to 250k
            # pts/m^2 near a scanner): the TLS radii, r ~ U[0.05, 0.5] m
            r = float(rng.uniform(0.25, 3.0)) if j % 2 == 0 else float(rng.uniform(0.05, 0.5))
            reqs.append((j, q, "radius", r))
        else:
            reqs.append((j, q, "knn", int(rng.choice([8, 16, 32]))))
    torch.cuda.synchronize()
    budget = int(args.serve_budget_gb * (1 << 30))

    def run_at(rate):
        import threading
        srv = cg.Server(indexes, slots=args.serve_slots, memory_budget=budget)
        gaps = rng.exponential(1.0 / rate, nreq)
        ids = []
        done = []

        def submitter():
            t = time.perf_counter()
            for (j, q, kind, p), g in zip(reqs, gaps):
                t += g
                d = t - time.perf_counter()
                if d > 0:
                    time.sleep(d)
                ids.append(srv.submit_radius(j, q, p) if kind == "radius" else srv.submit_knn(j, q, p))

        th = threading.Thread(target=submitter)
        t0 = time.perf_counter()
        th.start()
        failed = 0
        for _ in range(nreq):
            rid = srv.wait_any()
            try:
                srv.wait(rid, copy=False)
            except cg.CheeseError:
                failed += 1
            srv.release(rid)
            done.append(time.perf_counter())
        th.join()
        wall = time.perf_counter() - t0
        st = srv.stats()
        srv.close()
        return {"offered_req_per_s": rate, "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "max_ms": st["max_ms"],
                "queries_per_s": st["queries_per_s"], "requests": st["requests_done"], "failed": failed,
                "max_in_flight": st["max_in_flight"], "preemptions": st["preemptions"],
                "memory_peak_gb": st["memory_peak"] / 2 ** 30, "wall_s": wall}

    # warm-up, then a closed burst (everything at once) gives the capacity
    run_at(1e6)
    sat = run_at(1e6)
    cap_rps = sat["requests"] / max(sat["wall_s"], 1e-9)
    sweep = [run_at(f * cap_rps) for f in (0.25, 0.5, 0.75, 0.9)]
    line = {
        "metric": "serving queries/s and p50/p99 latency (8 resident indexes, Poisson radius/kNN requests)",
        "value": sat["queries_per_s"], "unit": "queries/s", "n_gpus": world, "steps": nreq, "warmup": nreq,
        "ms_per_step": None, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f32+f64", "data": "synthetic",
        "config": {"workload": "8 indexes (4 ALS 2D cell 1 m, 4 TLS 3D cell 0.25 m), binary32 offsets; requests "
                               "nq log-uniform [1k, 1M], r ~ U[0.25, 3] m (ALS) / U[0.05, 0.5] m (TLS) or "
                               "k in {8,16,32}",
                   "index_points": sizes, "slots": args.serve_slots, "memory_budget_gb": args.serve_budget_gb},
        "saturation": sat, "sweep": sweep,
    }
    for ix in indexes:
        ix.close()
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


def run_latency(args):
    """Per-call latency of small query batches through the public API (the
    paper times single random queries): batches of 1 .. 100k random queries
    drawn near the 12M tile's points, sphere r = 1 m (count + fill) and
    k-NN k = 16, median over repetitions, per call and per query."""
    import numpy as np
    import torch

    import cloudgen
    import paper_2502_11602_gb300 as cg

    dev = torch.device("cuda", 0)
    xyz = cloudgen.als_urban(args.points)
    ix = cg.Index(torch.from_numpy(xyz).to(dev), CELL)
    rng = np.random.default_rng(11)
    rows = []
    for B in (1, 10, 100, 1000, 10_000, 100_000):
        reps = 50 if B <= 1000 else 10
        qs = [torch.from_numpy(np.ascontiguousarray(
            xyz[rng.integers(0, len(xyz), B)] + rng.normal(0, 0.5, (B, 3)))).to(dev) for _ in range(reps + 3)]
        torch.cuda.synchronize()
        out = {}
        for kind in ("radius", "knn"):
            ts = []
            for i, q in enumerate(qs):
                t0 = time.perf_counter()
                if kind == "radius":
                    off, ind = ix.radius_search(q, RADIUS, check=False)
                else:
                    idx, d2 = ix.knn(q, 16, check=False)
                torch.cuda.synchronize()
                if i >= 3:
                    ts.append(time.perf_counter() - t0)
            med = statistics.median(ts)
            out[kind] = {"us_per_call": med * 1e6, "us_per_query": med * 1e6 / B, "queries_per_s": B / med}
        rows.append({"batch": B, **out})
    ix.close()
    line = {"metric": "query latency through the public API (12M ALS tile, sphere r=1 m, k-NN k=16)",
            "value": rows[0]["radius"]["us_per_call"], "unit": "us per single-query call", "n_gpus": 1,
            "higher_is_better": False, "data": "synthetic",
            "config": {"workload": "12M ALS tile, 2D dense 1 m; random queries within 0.5 m of the points; "
                                   "host-timed, synchronised, median of 10-50 calls per batch size"},
            "batches": rows}
    print(json.dumps(line), flush=True)


def run_memory(args):
    """Device memory of the index per flavour, dimension and cell size on the
    12M tile, against the 8 n bytes (one pointer per point) the paper takes
    as the minimum of a point index."""
    import torch

    import cloudgen
    import paper_2502_11602_gb300 as cg

    dev = torch.device("cuda", 0)
    xyz = cloudgen.als_urban(args.points)
    n = len(xyz)
    x = torch.from_numpy(xyz).to(dev)
    rows = []
    names = {cg.DENSE: "dense", cg.SPARSE: "sparse", cg.MIXED: "mixed"}
    for dim in (2, 3):
        for cell in (0.5, 1.0, 2.0):
            for fl in (cg.DENSE, cg.SPARSE, cg.MIXED):
                torch.cuda.synchronize()
                t0 = time.perf_counter()
                ix = cg.Index(x, cell, cell, dim=dim, flavor=fl)
                torch.cuda.synchronize()
                t_build = time.perf_counter() - t0
                info = ix.info()
                # records (16 n) + exact copy (24 n) are point data, and so is
                # the height-sorted copy of 2D grids (16 n + 4 n ids); the rest
                # indexes them
                zcopy = 20 * n if dim == 2 else 0
                tables = info["device_bytes"] - 40 * n - zcopy
                rows.append({"dim": dim, "cell_m": cell, "flavor": names[fl], "ncell": info["ncell"],
                             "nonempty": info["nonempty"], "device_MiB": info["device_bytes"] / 2 ** 20,
                             "index_MiB": tables / 2 ** 20, "index_over_8n": tables / (8.0 * n),
                             "height_copy_MiB": zcopy / 2 ** 20,
                             "build_ms": t_build * 1e3})
                ix.close()
    line = {"metric": "index device memory vs the 8 n-byte minimum (12M ALS tile)", "value": None,
            "unit": "MiB", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": "12M ALS tile; index bytes = device bytes minus the 16 n B binary32 records "
                                   "and the 24 n B exact copy", "n_points": n, "min_8n_MiB": 8 * n / 2 ** 20},
            "rows": rows}
    print(json.dumps(line), flush=True)


def run_knn(args):
    """All-points k-NN on the 12M tile (every point a query, the k closest
    under (d2, id), binary64 d2 out) for k = 1 .. 64: device time per pass
    (CUDA events, mean of `steps` after `warmup`) and, per k, the library's
    own phase split (the box classes, the bounded search, the ring path)."""
    import torch

    import cloudgen
    import paper_2502_11602_gb300 as cg

    dev = torch.device("cuda", 0)
    xyz = cloudgen.als_urban(args.points)
    n = len(xyz)
    x = torch.from_numpy(xyz).to(dev)
    h = cg.cg_build(x, CELL, CELL, 2, cg.DENSE, cg.FP32_OFFSET)
    stream = torch.cuda.current_stream()
    rows = []
    ks = [int(v) for v in args.knn_k.split(",")]
    for k in ks:
        idx = torch.empty((n, k), dtype=torch.int32, device=dev)
        d2 = torch.empty((n, k), dtype=torch.float64, device=dev)
        for _ in range(max(args.warmup, 1)):
            cg.cg_all_points_knn(h, k, idx, d2)
        torch.cuda.synchronize()
        ts = []
        for _ in range(args.steps):
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record(stream)
            cg.cg_all_points_knn(h, k, idx, d2)
            b.record(stream)
            torch.cuda.synchronize()
            ts.append(a.elapsed_time(b))
        cg.cg_index_status(h)
        cg.cg_profile_enable(True)
        cg.cg_all_points_knn(h, k, idx, d2)
        torch.cuda.synchronize()
        phases = {name: round(ms, 4) for name, (_, ms) in cg.cg_profile_read().items()}
        cg.cg_profile_enable(False)
        ms = statistics.mean(ts)
        rows.append({"k": k, "ms": ms, "queries_per_s": n / (ms * 1e-3), "phases_ms": phases})
        del idx, d2
    cg.cg_index_free(h)
    line = {"metric": "all-points k-NN queries/s (12M ALS tile, every point a query)",
            "value": next((r for r in rows if r["k"] == 16), rows[0])["queries_per_s"], "unit": "queries/s", "n_gpus": 1, "steps": args.steps,
            "warmup": args.warmup, "higher_is_better": True, "data": "synthetic",
            "config": {"workload": f"ALS tile {n} pts, 2D dense grid 1 m, binary32 offsets, k-NN all points",
                       "n_points": n},
            "by_k": rows}
    print(json.dumps(line), flush=True)


def run_sz(args):
    """Slice thickness of the 3D mixed flavour (Section 3.3.3) on the street
    canyon cloud: the z voxel side s_z swept at a fixed 0.25 m xy side; per
    setting the build time, device memory, dense slices, and the radius
    (r = 0.1 m, count + fill) and k-NN (k = 16) times on 1M of the cloud's
    points as queries; the binary64 results are identical in every setting."""
    import numpy as np
    import torch

    import cloudgen
    import paper_2502_11602_gb300 as cg

    dev = torch.device("cuda", 0)
    n = args.points if args.points != N_POINTS else 20_000_000
    xyz = cloudgen.tls_street(n)
    x = torch.from_numpy(xyz).to(dev)
    q = torch.from_numpy(cloudgen.sample_queries(xyz, 1_000_000, seed=cloudgen.CONFIG_SEED + 2)).to(dev)
    rows, ref = [], None
    for sz in (0.125, 0.25, 0.5, 1.0, 2.0):
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        ix = cg.Index(x, 0.25, sz, dim=3, flavor=cg.MIXED)
        torch.cuda.synchronize()
        t_build = time.perf_counter() - t0
        info = ix.info()
        def timed(fn):
            fn()
            torch.cuda.synchronize()
            a = torch.cuda.Event(enable_timing=True)
            b = torch.cuda.Event(enable_timing=True)
            a.record()
            out = fn()
            b.record()
            torch.cuda.synchronize()
            return a.elapsed_time(b), out
        t_rad, (off, ind) = timed(lambda: ix.radius_search(q, 0.1))
        t_knn, (kidx, _) = timed(lambda: ix.knn(q, 16))
        sig = (int(off[-1]), int(ind.sum()), int(kidx.sum()))
        ref = ref or sig
        rows.append({"s_z_m": sz, "slices": info["nslices"], "dense_slices": info["dense_slices"],
                     "nonempty": info["nonempty"], "device_MiB": info["device_bytes"] / 2 ** 20,
                     "build_ms": t_build * 1e3, "radius_ms": t_rad, "knn16_ms": t_knn, "same_result": sig == ref})
        ix.close()
    line = {"metric": "3D mixed flavour: slice thickness s_z sweep (street canyon cloud)", "value": None,
            "unit": "ms", "n_gpus": 1, "data": "synthetic",
            "config": {"workload": f"TLS street canyon {n} pts, 3D mixed, xy voxel 0.25 m, 1M queries drawn "
                                   "from the cloud, sphere r = 0.1 m and k = 16", "n_points": n},
            "rows": rows}
    print(json.dumps(line), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", choices=["ours", "reference"], default="ours")
    ap.add_argument("--precision", choices=["fp32", "fp64"], default="fp32")
    ap.add_argument("--cpu-sample", type=int, default=2_000_000)
    ap.add_argument("--ref-sample", type=int, default=100_000)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--points", type=int, default=N_POINTS, help="tile size (profiling cases only)")
    ap.add_argument("--no-fp64", action="store_true", help="skip the binary64 comparison on the tile")
    ap.add_argument("--workload", choices=["tile", "batched", "serving", "latency", "memory", "sz", "knn"], default="tile")
    ap.add_argument("--tiles", type=int, default=256)
    ap.add_argument("--knn-k", default="1,8,16,32,64", help="k values of the knn workload")
    ap.add_argument("--batch-points", type=int, default=60_000_000)
    ap.add_argument("--serve-requests", type=int, default=120)
    ap.add_argument("--serve-slots", type=int, default=4)
    ap.add_argument("--serve-budget-gb", type=float, default=48.0)
    ap.add_argument("--serve-scale", type=float, default=1.0, help="index sizes x this (smaller test runs)")
    args = ap.parse_args()
    if args.impl == "reference":
        if args.workload != "tile":
            print(json.dumps({"impl": "reference", "unavailable": "the oracle arm covers the tile workload only"}))
            return
        run_reference(args)
    elif args.workload == "batched":
        run_batched(args)
    elif args.workload == "serving":
        run_serving(args)
    elif args.workload == "latency":
        run_latency(args)
    elif args.workload == "knn":
        run_knn(args)
    elif args.workload == "sz":
        run_sz(args)
    elif args.workload == "memory":
        run_memory(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
