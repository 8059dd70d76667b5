"""Benchmark: radius-search throughput on the 12M-point ALS tile.

Workload (one step = the whole hot path once): build the 2D dense grid index
(1 m voxels) of a 12,000,000-point synthetic ALS tile (500 m x 500 m, UTM
offsets, terrain + buildings + trees), then the two-pass fixed-radius sphere
search with every point as a query (count, scan, fill with rows sorted by
original id) at r = 1 m.  Inputs are resident in HBM when the timed region
starts; they are 288 MB, larger than the 129 MB L2.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

Prints one JSON line (rank 0).  `--impl reference` times the CPU oracle on
the host cores instead (bounded sample of the same workload).
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
    path = os.path.join(ROOT, "profiles", "traffic.json")
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
            "build_s": t_build, "query_sample_s": t_q}


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
    t_step = t_build + t_q * len(xyz) / S  # one full step: build + every point a query
    value = len(xyz) / t_step
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": t_step * 1e3, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic", "impl": "reference",
            "config": {"workload": "ALS tile 12M pts, 500x500 m, 2D dense grid 1 m, sphere r=1 m, all points as queries",
                       "n_points": len(xyz), "radius_m": RADIUS, "cell_m": CELL},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "sample": f"oracle build of the full tile once ({t_build:.1f} s, 1 thread); each step "
                                       f"{S} seeded random queries on {cores} threads, extrapolated to all queries"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


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

    def step(record=None):
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(4)] if record is not None else None
        if ev: ev[0].record(stream)
        h = cg.cg_build(x, CELL, CELL, 2, cg.DENSE, prec)
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

    for _ in range(args.warmup):
        total = step()
    torch.cuda.synchronize()

    records = []
    clocks = ClockSampler(local)
    clocks.start()
    if dist is not None:
        dist.barrier()
    torch.cuda.synchronize()
    launches0 = cg.cg_launch_count()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    t0.record(stream)
    for _ in range(args.steps):
        total = step(records)
    t1.record(stream)
    torch.cuda.synchronize()
    launches = (cg.cg_launch_count() - launches0) / args.steps
    if dist is not None:
        dist.barrier()
    clk = clocks.stop()
    ms = t0.elapsed_time(t1) / args.steps
    if dist is not None:
        tt = torch.tensor([ms], device=dev)
        dist.all_reduce(tt, op=dist.ReduceOp.MAX)
        ms = float(tt.item())
    build_ms = statistics.mean(r[0].elapsed_time(r[1]) for r in records)
    count_ms = statistics.mean(r[1].elapsed_time(r[2]) for r in records)
    fill_ms = statistics.mean(r[2].elapsed_time(r[3]) for r in records)

    # end to end through the public API: pinned host points in, CSR out
    host_in = torch.from_numpy(xyz).pin_memory()
    host_off = torch.empty(n + 1, dtype=torch.int64).pin_memory()
    host_ind = torch.empty(total, dtype=torch.int32).pin_memory()
    e2e_times = []
    for it in range(max(2, min(args.steps, 5)) + 1):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record(stream)
        xd = torch.empty((n, 3), dtype=torch.float64, device=dev)
        xd.copy_(host_in, non_blocking=True)
        ix = cg.Index(xd, CELL, CELL, 2, cg.DENSE, prec)
        off, ind = ix.radius_search(None, RADIUS, cg.SPHERE, check=False)
        host_off.copy_(off, non_blocking=True)
        host_ind.copy_(ind, non_blocking=True)
        b.record(stream)
        torch.cuda.synchronize()
        ix.close()
        del xd, off, ind
        if it > 0:
            e2e_times.append(a.elapsed_time(b))
    e2e_ms = statistics.mean(e2e_times)

    value = world * n / (ms * 1e-3)
    peak, peak_kind = _peaks()
    # dominant kernel: the fill pass (largest share of the step)
    stages = {"build": build_ms, "count": count_ms, "fill": fill_ms}
    dom = max(("count", "fill"), key=lambda s: stages[s])
    bytes_per_point = 16  # binary32 record: x~, y~, z~, id
    info_ncell = int(math.floor(side / CELL) + 1) ** 2
    if dom == "fill":
        alg = bytes_per_point * n + 4 * (info_ncell + 1) + 8 * (n + 1) + 4 * total
        kname, files = "radius_fill", ["cg_query.cu", "cg_internal.cuh"]
        dur = fill_ms
    else:
        alg = bytes_per_point * n + 4 * (info_ncell + 1) + 4 * n + 16 * (n + 1)
        kname, files = "radius_count", ["cg_query.cu", "cg_internal.cuh"]
        dur = count_ms
    achieved = alg / (dur * 1e-3) / 1e9
    roof = {"bound": "hbm", "kernel": kname, "achieved": achieved, "peak": peak, "peak_kind": peak_kind,
            "unit": "GB/s", "frac": achieved / peak, "traffic": _traffic(kname, files),
            "algorithmic_bytes": alg, "ms_per_launch": dur}
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms, "higher_is_better": True, "scaling": "weak",
        "vs_baseline": None, "dtype": "f32+f64" if prec == cg.FP32_OFFSET else "f64", "data": "synthetic",
        "config": {"workload": "ALS tile 12M pts, 500x500 m, 2D dense grid 1 m, sphere r=1 m, all points as queries",
                   "n_points": n, "radius_m": RADIUS, "cell_m": CELL, "precision": args.precision,
                   "l2": "inputs larger than L2 (288 MB points, 129 MB L2)", "parallelism": f"replicas x{world}"},
        "neighbors_per_s": world * total / (ms * 1e-3), "neighbors_per_step": total,
        "stages_ms": stages,
        "e2e": {"value": world * n / (e2e_ms * 1e-3), "unit": UNIT, "ms_per_step": e2e_ms,
                "h2d_bytes_per_step": n * 24, "d2h_bytes_per_step": (n + 1) * 8 + total * 4},
        "roofline": roof, "clocks": clk, "gpu_launches": launches,
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = _cpu_baseline(xyz, args.cpu_sample)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()


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
    args = ap.parse_args()
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
