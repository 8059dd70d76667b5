"""Autotuner for batched tiles: cell size, chunk height and launch shapes.

Tiles are grouped by point density (points per m^2 of their xy bounding box,
one bucket per factor of two).  For every bucket not yet in the cache, one
representative tile (the bucket's median size) is indexed and searched at
each candidate cell size through the library (build + all-points radius
count and fill, plus k-NN when k > 0), and the fastest cell size is kept.
Results are cached in a JSON file keyed by GPU name, dimension, radius,
kernel, k, precision and bucket, so later runs make no measurement.

The cell size only changes speed: the neighbour sets are fixed by the
predicate, whatever the grid (Section 3: any voxel size gives the same
kernel search result).
"""
from __future__ import annotations

import json
import math
import os

import numpy as np
import torch

CANDIDATES = (0.5, 1.0, 2.0)


def default_cache_path() -> str:
    base = os.environ.get("XDG_CACHE_HOME", os.path.join(os.path.expanduser("~"), ".cache"))
    return os.path.join(base, "cheesegpu", "autotune.json")


def density_bucket(xyz: np.ndarray) -> int:
    """floor(log2(points per m^2 of the xy bounding box))."""
    ext = xyz[:, :2].max(0) - xyz[:, :2].min(0)
    area = max(float(ext[0]) * float(ext[1]), 1e-6)
    return int(math.floor(math.log2(max(len(xyz) / area, 1e-6))))


def _key(gpu: str, dim: int, radius: float, kernel: int, k: int, precision: int, bucket: int) -> str:
    return f"{gpu}|dim{dim}|r{radius:g}|kern{kernel}|k{k}|prec{precision}|d{bucket}"


def _time_cell(cg, tile: torch.Tensor, cell: float, dim: int, radius: float, kernel: int, k: int,
               precision: int, reps: int = 3) -> float:
    times = []
    for it in range(reps + 1):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        ix = cg.Index(tile, cell, cell, dim=dim, precision=precision)
        ix.radius_search(None, radius, kernel, check=False)
        if k > 0:
            ix.knn(None, k, check=False)
        b.record()
        torch.cuda.synchronize()
        ix.close()
        if it > 0:
            times.append(a.elapsed_time(b))
    return float(np.median(times))


def tune(xyz: np.ndarray, tile_offsets, radius: float, kernel: int = 0, k: int = 0, dim: int = 2,
         precision: int = 1, candidates=CANDIDATES, cache_path: str | None = None,
         device: str = "cuda:0") -> tuple[np.ndarray, dict]:
    """Cell size per tile, and a report {bucket: {cell: ms, ..., "best": cell}}
    for the buckets measured by this call (cached buckets are not re-timed)."""
    import paper_2502_11602_gb300 as cg

    off = np.asarray(tile_offsets, dtype=np.int64)
    T = len(off) - 1
    cache_path = cache_path or default_cache_path()
    try:
        with open(cache_path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    gpu = torch.cuda.get_device_name(torch.device(device))
    buckets = np.array([density_bucket(xyz[off[t]:off[t + 1]]) for t in range(T)])
    report = {}
    for bk in sorted(set(buckets.tolist())):
        key = _key(gpu, dim, radius, kernel, k, precision, bk)
        if key in cache:
            continue
        members = np.nonzero(buckets == bk)[0]
        sizes = off[members + 1] - off[members]
        rep = int(members[np.argsort(sizes)[len(sizes) // 2]])
        tile = torch.from_numpy(np.ascontiguousarray(xyz[off[rep]:off[rep + 1]])).to(device)
        ms = {str(c): _time_cell(cg, tile, float(c), dim, radius, kernel, k, precision) for c in candidates}
        best = float(min(ms, key=ms.get))
        cache[key] = best
        report[bk] = dict(ms, best=best, tile=rep, points=int(off[rep + 1] - off[rep]))
        del tile
    if report:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    cells = np.array([cache[_key(gpu, dim, radius, kernel, k, precision, int(b))] for b in buckets])
    return cells, report


# ------------------------------------------------------------ launch shapes
#
# The radius kernels' launch shapes (warps per CTA and warps sharing a voxel
# group, per size class) and the height span of an all-points chunk (binary32
# 2D grids) are this design's "threads per query" and "staging depth": they
# set how many lanes share a group's staged candidates and how many queries
# one staging serves.  Like the cell size they change only speed.

CHUNK_HEIGHTS = (4.0, 8.0, 12.0)
SHAPES = (0, 1, 2)


def _time_radius(cg, ix, radius: float, kernel: int, reps: int = 5) -> float:
    times = []
    for it in range(reps + 1):
        torch.cuda.synchronize()
        a = torch.cuda.Event(enable_timing=True)
        b = torch.cuda.Event(enable_timing=True)
        a.record()
        ix.radius_search(None, radius, kernel, check=False)
        b.record()
        torch.cuda.synchronize()
        if it > 0:
            times.append(a.elapsed_time(b))
    return float(np.min(times))


def tune_launch(xyz: np.ndarray, tile_offsets, cells, radius: float, kernel: int = 0, dim: int = 2,
                precision: int = 1, cache_path: str | None = None, device: str = "cuda:0") -> tuple[dict, dict]:
    """Launch tuning per density bucket (coordinate descent: chunk height,
    then the count kernels' shape, then the fill kernels'), each bucket's
    median tile searched at its cell size; cached like the cell sizes.
    Returns the tuning of the bucket holding the most points (one tuning
    serves a whole batch, whose tiles share each launch) and a report
    {bucket: {"tuning": ..., "ms": {setting: ms}}} of the buckets measured."""
    import paper_2502_11602_gb300 as cg

    off = np.asarray(tile_offsets, dtype=np.int64)
    T = len(off) - 1
    cells = np.asarray(cells, dtype=np.float64)
    cache_path = cache_path or default_cache_path()
    try:
        with open(cache_path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    gpu = torch.cuda.get_device_name(torch.device(device))
    buckets = np.array([density_bucket(xyz[off[t]:off[t + 1]]) for t in range(T)])
    saved = cg.cg_get_tuning()
    report = {}
    try:
        for bk in sorted(set(buckets.tolist())):
            key = _key(gpu, dim, radius, kernel, 0, precision, bk) + "|launch"
            if key in cache:
                continue
            members = np.nonzero(buckets == bk)[0]
            sizes = off[members + 1] - off[members]
            rep = int(members[np.argmax(sizes)])  # the largest: launch overheads matter least
            tile = torch.from_numpy(np.ascontiguousarray(xyz[off[rep]:off[rep + 1]])).to(device)
            ix = cg.Index(tile, float(cells[rep]), float(cells[rep]), dim=dim, precision=precision)
            best = {"radius_chunk_height": 8.0, "count_shape": 0, "fill_shape": 0}
            ms = {}

            def trial(**kw):
                t = dict(best, **kw)
                cg.cg_set_tuning(t)
                v = _time_radius(cg, ix, radius, kernel)
                ms[",".join(f"{k}={t[k]:g}" for k in sorted(t))] = v
                return v

            chunked = dim == 2 and precision == 1 and kernel in (0, 1)
            for field, values in (("radius_chunk_height", CHUNK_HEIGHTS if chunked else (8.0,)),
                                  ("count_shape", SHAPES), ("fill_shape", SHAPES)):
                times = {v: trial(**{field: v}) for v in values}
                best[field] = min(times, key=times.get)
            ix.close()
            del tile
            cache[key] = best
            report[bk] = {"tuning": dict(best), "ms": ms, "tile": rep, "points": int(off[rep + 1] - off[rep])}
    finally:
        cg.cg_set_tuning(saved)
    if report:
        os.makedirs(os.path.dirname(cache_path), exist_ok=True)
        tmp = cache_path + f".tmp{os.getpid()}"
        with open(tmp, "w") as f:
            json.dump(cache, f, indent=1, sort_keys=True)
        os.replace(tmp, cache_path)
    pts = {}
    for t in range(T):
        pts[int(buckets[t])] = pts.get(int(buckets[t]), 0) + int(off[t + 1] - off[t])
    main = max(pts, key=pts.get)
    batch = dict(cache[_key(gpu, dim, radius, kernel, 0, precision, main) + "|launch"])
    return batch, report


def tune_pipeline(x: torch.Tensor, tile_offsets, cells, radius: float, k: int = 0, precision: int = 1,
                  cache_path: str | None = None, margin: float = 0.02, reps: int = 3) -> tuple[dict, dict]:
    """Launch shapes for a captured batch, timed on the batch itself: a
    pipeline is captured per candidate (coordinate descent over the count
    shapes, then the fill shapes) and replayed; a candidate replaces the
    default only if it is faster by more than `margin`.  Cached per GPU and
    batch (tiles, points, radius, k, precision).  Returns (tuning, report
    {setting: ms}); the library's tuning is left as it was."""
    import paper_2502_11602_gb300 as cg

    off = np.asarray(tile_offsets, dtype=np.int64)
    cache_path = cache_path or default_cache_path()
    try:
        with open(cache_path) as f:
            cache = json.load(f)
    except (OSError, ValueError):
        cache = {}
    gpu = torch.cuda.get_device_name(x.device)
    key = f"{gpu}|pipeline|T{len(off) - 1}|n{int(off[-1])}|r{radius:g}|k{k}|prec{precision}"
    if key in cache:
        return dict(cache[key]), {}
    saved = cg.cg_get_tuning()
    report = {}

    def timed(t) -> float:
        cg.cg_set_tuning(t)
        pipe = cg.Pipeline(x, off, cells, radius=radius, k=k, precision=precision)
        try:
            pipe.run()
            ts = []
            for _ in range(reps):
                torch.cuda.synchronize()
                a = torch.cuda.Event(enable_timing=True)
                b = torch.cuda.Event(enable_timing=True)
                a.record()
                pipe.run(sync=False)
                b.record()
                torch.cuda.synchronize()
                ts.append(a.elapsed_time(b))
        finally:
            pipe.close()
        v = float(np.median(ts))
        report[f"count_shape={t['count_shape']},fill_shape={t['fill_shape']}"] = v
        return v

    try:
        best = {"count_shape": 0, "fill_shape": 0}
        base = timed(dict(saved, **best))
        best_ms = base
        for field in ("count_shape", "fill_shape"):
            for v in SHAPES:
                if v == best[field]:
                    continue
                cand = dict(best, **{field: v})
                ms = timed(dict(saved, **cand))
                if ms < best_ms * (1.0 - margin):
                    best, best_ms = cand, ms
    finally:
        cg.cg_set_tuning(saved)
    cache[key] = best
    os.makedirs(os.path.dirname(cache_path), exist_ok=True)
    tmp = cache_path + f".tmp{os.getpid()}"
    with open(tmp, "w") as f:
        json.dump(cache, f, indent=1, sort_keys=True)
    os.replace(tmp, cache_path)
    return dict(best), report
