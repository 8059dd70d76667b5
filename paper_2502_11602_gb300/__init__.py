"""cheesegpu: GB300 (sm_103a) Cheesemap neighbour search behind a C ABI.

Thin Python binding over ``libcheesegpu.so`` (``include/cheesegpu.h``).  It
only marshals arguments: torch tensors provide device memory and streams,
every step of the build and of the queries runs in the library's CUDA
kernels.  There is no CPU fallback: if the library cannot be loaded, every
call raises.

Functions with the C ABI's names (``cg_build``, ``cg_radius_count``, ...) take
the same arguments as the C calls, with tensors for device pointers; the
``Index`` class is a convenience wrapper around them.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

from . import _build

DENSE, SPARSE, MIXED = 0, 1, 2
SPHERE, CUBE, CYLINDER = 0, 1, 2
FP64, FP32_OFFSET = 0, 1
GROW_MONOTONE, GROW_DENSITY = 0, 1

STATUS = {0: "CG_OK", 1: "CG_ERR_INVALID", 2: "CG_ERR_OOM", 3: "CG_ERR_CUDA", 4: "CG_ERR_TIMEOUT",
          5: "CG_ERR_OVERFLOW", 6: "CG_ERR_INTERNAL", 7: "CG_ERR_UNIMPLEMENTED"}

EXPORTS = ["cg_set_allocator", "cg_last_error", "cg_version", "cg_launch_count", "cg_build", "cg_build_batched",
           "cg_index_info", "cg_index_status", "cg_index_free", "cg_radius_count", "cg_radius_fill", "cg_radius_search",
           "cg_radius_search_into", "cg_free_device", "cg_all_points_count", "cg_all_points_fill", "cg_knn",
           "cg_all_points_knn", "cg_knn_grow", "cg_offsets_scan_noalloc", "cg_pipeline_create", "cg_pipeline_run",
           "cg_pipeline_outputs", "cg_pipeline_info", "cg_pipeline_free", "cg_server_create", "cg_server_submit",
           "cg_server_wait", "cg_server_wait_any", "cg_server_release", "cg_server_stats", "cg_server_free",
           "cg_profile_enable", "cg_profile_read", "cg_set_tuning", "cg_get_tuning", "cg_radius_stats"]

REQ_RADIUS, REQ_KNN = 0, 1

# The library's small-batch paths: calls of up to SMALL_BATCH external
# queries, rows of up to SMALL_ROW_CAP neighbours kept per query.
SMALL_BATCH, SMALL_ROW_CAP = 1024, 2048
SMALL_GUESS = 256  # output entries reserved per query by a small radius call


class CheeseError(RuntimeError):
    def __init__(self, code: int, msg: str):
        super().__init__(f"{STATUS.get(code, code)}: {msg}")
        self.code = code


class IndexInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("dim", ctypes.c_int32), ("flavor", ctypes.c_int32),
                ("precision", ctypes.c_int32), ("ntiles", ctypes.c_int32), ("ncell", ctypes.c_int64),
                ("nonempty", ctypes.c_int64), ("nslices", ctypes.c_int64),
                ("dense_slices", ctypes.c_int64), ("device_bytes", ctypes.c_int64),
                ("lo", ctypes.c_double * 3), ("hi", ctypes.c_double * 3), ("nc", ctypes.c_int64 * 3),
                ("cell", ctypes.c_double * 3), ("origin", ctypes.c_double * 3),
                ("enc_err", ctypes.c_double)]


class Tuning(ctypes.Structure):
    _fields_ = [("radius_chunk_height", ctypes.c_float), ("radius_chunk_max", ctypes.c_uint32),
                ("count_shape", ctypes.c_int32), ("fill_shape", ctypes.c_int32)]


def cg_set_tuning(tuning: dict | None = None):
    """Process-wide launch tuning (None restores the defaults); keys as
    cg_tuning_t: radius_chunk_height, radius_chunk_max, count_shape, fill_shape."""
    if tuning is None:
        _check(load().cg_set_tuning(None))
        return
    t = Tuning(**cg_get_tuning())
    for k, v in tuning.items():
        setattr(t, k, v)
    _check(load().cg_set_tuning(ctypes.byref(t)))


class RadiusStats(ctypes.Structure):
    _fields_ = [("tested_pairs", ctypes.c_int64), ("general_groups", ctypes.c_int64), ("groups", ctypes.c_int64)]


def cg_radius_stats(h: int) -> dict:
    s = RadiusStats()
    _check(load().cg_radius_stats(h, ctypes.byref(s)))
    return {f: getattr(s, f) for f, _ in RadiusStats._fields_}


def cg_get_tuning() -> dict:
    t = Tuning()
    _check(load().cg_get_tuning(ctypes.byref(t)))
    return {f: getattr(t, f) for f, _ in Tuning._fields_}


class PipelineOpts(ctypes.Structure):
    _fields_ = [("radius", ctypes.c_double), ("kernel", ctypes.c_int32), ("k", ctypes.c_int32),
                ("headroom", ctypes.c_double)]


class PipelineInfo(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int64), ("ntiles", ctypes.c_int32), ("k", ctypes.c_int32),
                ("graph_kernels", ctypes.c_int32), ("graph_nodes", ctypes.c_int32),
                ("replans", ctypes.c_int64), ("capacity_indices", ctypes.c_int64),
                ("capacity_voxels", ctypes.c_int64), ("ncell", ctypes.c_int64),
                ("device_bytes", ctypes.c_int64)]


class ServerOpts(ctypes.Structure):
    _fields_ = [("slots", ctypes.c_int32), ("memory_budget", ctypes.c_int64)]


class Request(ctypes.Structure):
    _fields_ = [("index", ctypes.c_int32), ("op", ctypes.c_int32), ("kernel", ctypes.c_int32),
                ("k", ctypes.c_int32), ("radius", ctypes.c_double), ("q_dev", ctypes.c_void_p),
                ("nq", ctypes.c_int64)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("nq", ctypes.c_int64), ("total", ctypes.c_int64),
                ("offsets", ctypes.c_void_p), ("indices", ctypes.c_void_p), ("knn_idx", ctypes.c_void_p),
                ("knn_d2", ctypes.c_void_p), ("queue_ms", ctypes.c_double), ("latency_ms", ctypes.c_double)]


class ServerStats(ctypes.Structure):
    _fields_ = [("requests_done", ctypes.c_int64), ("requests_failed", ctypes.c_int64),
                ("queries_done", ctypes.c_int64), ("queued", ctypes.c_int64), ("in_flight", ctypes.c_int32),
                ("max_in_flight", ctypes.c_int32), ("memory_budget", ctypes.c_int64),
                ("memory_in_use", ctypes.c_int64), ("memory_peak", ctypes.c_int64),
                ("preemptions", ctypes.c_int64), ("p50_ms", ctypes.c_double), ("p99_ms", ctypes.c_double),
                ("max_ms", ctypes.c_double), ("queries_per_s", ctypes.c_double)]


_lib = None
_lock = threading.Lock()


def library_path() -> str:
    return _build.LIB


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Loads libcheesegpu.so (building it first if needed)."""
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        path = _build.build() if build_if_missing else _build.LIB
        if not os.path.exists(path):
            raise RuntimeError(f"cheesegpu library not found at {path}")
        lib = ctypes.CDLL(path)
        P, I64, I32, D, I = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int32, ctypes.c_double, ctypes.c_int
        sig = {
            "cg_set_allocator": [P, P, P],
            "cg_last_error": [],
            "cg_version": [],
            "cg_launch_count": [],
            "cg_build": [P, I64, D, D, I, I, I, P, P],
            "cg_build_batched": [P, P, I32, P, I, I, I, P, P],
            "cg_index_info": [P, P],
            "cg_index_free": [P],
            "cg_index_status": [P, P],
            "cg_radius_count": [P, P, I64, D, I, P, P, P],
            "cg_radius_fill": [P, P, I64, D, I, P, P, P],
            "cg_radius_search": [P, P, I64, D, I, P, P, P, P],
            "cg_radius_search_into": [P, P, I64, D, I, P, P, I64, P, P],
            "cg_free_device": [P, P],
            "cg_all_points_count": [P, D, I, P, P, P],
            "cg_all_points_fill": [P, D, I, P, P, P],
            "cg_knn": [P, P, I64, I32, P, P, P],
            "cg_all_points_knn": [P, I32, P, P, P],
            "cg_knn_grow": [P, P, I64, I32, I32, P, P, P, P],
            "cg_offsets_scan_noalloc": [P, I64, P, P],
            "cg_pipeline_create": [P, P, I32, P, I, I, P, P, P],
            "cg_pipeline_run": [P, P, P],
            "cg_pipeline_outputs": [P, P, P, P, P],
            "cg_pipeline_info": [P, P],
            "cg_pipeline_free": [P],
            "cg_server_create": [P, I32, P, P],
            "cg_server_submit": [P, P, P],
            "cg_server_wait": [P, I64, D, P],
            "cg_server_wait_any": [P, D, P],
            "cg_server_release": [P, I64],
            "cg_server_stats": [P, P],
            "cg_server_free": [P],
            "cg_profile_enable": [I],
            "cg_profile_read": [P, ctypes.c_size_t, P, I],
            "cg_set_tuning": [P],
            "cg_radius_stats": [P, P],
            "cg_get_tuning": [P],
        }
        for name, args in sig.items():
            f = getattr(lib, name)
            f.argtypes = args
            f.restype = ctypes.c_char_p if name in ("cg_last_error", "cg_version") else ctypes.c_int
        lib.cg_launch_count.restype = ctypes.c_uint64
        _lib = lib
        return lib


def _check(code: int):
    if code != 0:
        msg = load().cg_last_error().decode()
        raise CheeseError(code, msg)


def _ptr(t) -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError("expected a CUDA tensor")
    if not t.is_contiguous():
        raise ValueError("expected a contiguous tensor")
    return t.data_ptr()


def _stream(stream=None) -> int:
    if stream is not None:
        return stream.cuda_stream
    raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)  # the current stream's handle, without a Stream object
    if raw is not None:
        return raw(torch.cuda.current_device())
    return torch.cuda.current_stream().cuda_stream


def _points(x: torch.Tensor) -> torch.Tensor:
    if x.dtype != torch.float64 or x.dim() != 2 or x.shape[1] != 3:
        raise ValueError("points must be a float64 tensor of shape (n, 3)")
    return x.contiguous()


# ---------------------------------------------------------------- C ABI names


def cg_version() -> str:
    return load().cg_version().decode()


def cg_launch_count() -> int:
    """Kernels launched by the library so far in this process."""
    return int(load().cg_launch_count())


def cg_build(xyz: torch.Tensor, cell_xy: float, cell_z: float | None = None, dim: int = 2,
             flavor: int = DENSE, precision: int = FP32_OFFSET, stream=None) -> int:
    xyz = _points(xyz)
    h = ctypes.c_void_p()
    _check(load().cg_build(_ptr(xyz), xyz.shape[0], float(cell_xy),
                           float(cell_z if cell_z is not None else cell_xy), dim, flavor, precision,
                           _stream(stream), ctypes.byref(h)))
    return h.value


def cg_build_batched(xyz: torch.Tensor, tile_offsets, cells, dim: int = 2, flavor: int = DENSE,
                     precision: int = FP32_OFFSET, stream=None) -> int:
    import numpy as np
    xyz = _points(xyz)
    toff = np.ascontiguousarray(tile_offsets, dtype=np.int64)
    cel = np.ascontiguousarray(cells, dtype=np.float64)
    h = ctypes.c_void_p()
    _check(load().cg_build_batched(_ptr(xyz), toff.ctypes.data, len(toff) - 1, cel.ctypes.data, dim,
                                   flavor, precision, _stream(stream), ctypes.byref(h)))
    return h.value


def cg_index_info(h: int) -> dict:
    info = IndexInfo()
    _check(load().cg_index_info(h, ctypes.byref(info)))
    return {f: (list(getattr(info, f)) if isinstance(getattr(info, f), ctypes.Array) else getattr(info, f))
            for f, _ in IndexInfo._fields_}


def cg_index_status(h: int, stream=None):
    _check(load().cg_index_status(h, _stream(stream)))


def cg_index_free(h: int):
    _check(load().cg_index_free(h))


def cg_radius_count(h, q, r, kernel, offsets, want_total=True, stream=None):
    tot = ctypes.c_int64(0)
    _check(load().cg_radius_count(h, _ptr(q), q.shape[0], float(r), kernel, _ptr(offsets),
                                  ctypes.byref(tot) if want_total else None, _stream(stream)))
    return tot.value if want_total else None


def cg_radius_search_into(h, q, r, kernel, offsets, indices, capacity, stream=None):
    """Count + fill into `indices` (capacity entries): (fits, total).  When the
    rows do not fit, the count stands and cg_radius_fill completes it."""
    tot = ctypes.c_int64(0)
    rc = load().cg_radius_search_into(h, _ptr(q), q.shape[0], float(r), kernel, _ptr(offsets), _ptr(indices),
                                      int(capacity), ctypes.byref(tot), _stream(stream))
    if rc == 5:  # CG_ERR_OVERFLOW
        return False, tot.value
    _check(rc)
    return True, tot.value


def cg_radius_fill(h, q, r, kernel, offsets, indices, stream=None):
    _check(load().cg_radius_fill(h, _ptr(q), q.shape[0], float(r), kernel, _ptr(offsets),
                                 _ptr(indices), _stream(stream)))


def cg_all_points_count(h, r, kernel, offsets, want_total=True, stream=None):
    tot = ctypes.c_int64(0)
    _check(load().cg_all_points_count(h, float(r), kernel, _ptr(offsets),
                                      ctypes.byref(tot) if want_total else None, _stream(stream)))
    return tot.value if want_total else None


def cg_all_points_fill(h, r, kernel, offsets, indices, stream=None):
    _check(load().cg_all_points_fill(h, float(r), kernel, _ptr(offsets), _ptr(indices),
                                     _stream(stream)))


def cg_knn(h, q, k, idx, d2=None, stream=None):
    _check(load().cg_knn(h, _ptr(q), q.shape[0], int(k), _ptr(idx), _ptr(d2), _stream(stream)))


def cg_knn_grow(h, q, k, policy, idx, d2=None, visited=None, stream=None):
    _check(load().cg_knn_grow(h, _ptr(q), q.shape[0], int(k), int(policy), _ptr(idx), _ptr(d2), _ptr(visited),
                              _stream(stream)))


def cg_all_points_knn(h, k, idx, d2=None, stream=None):
    _check(load().cg_all_points_knn(h, int(k), _ptr(idx), _ptr(d2), _stream(stream)))


def cg_pipeline_create(xyz: torch.Tensor, tile_offsets, cells, dim: int, precision: int, radius: float,
                       kernel: int = SPHERE, k: int = 0, headroom: float = 0.0, stream=None) -> int:
    import numpy as np
    if xyz.dtype != torch.float64 or xyz.dim() != 2 or xyz.shape[1] != 3 or not xyz.is_contiguous():
        raise ValueError("points must be a contiguous float64 tensor of shape (n, 3)")
    toff = np.ascontiguousarray(tile_offsets, dtype=np.int64)
    cel = np.ascontiguousarray(cells, dtype=np.float64)
    opts = PipelineOpts(float(radius), int(kernel), int(k), float(headroom))
    h = ctypes.c_void_p()
    _check(load().cg_pipeline_create(_ptr(xyz), toff.ctypes.data, len(toff) - 1, cel.ctypes.data, dim, precision,
                                     ctypes.byref(opts), _stream(stream), ctypes.byref(h)))
    return h.value


def cg_pipeline_run(h: int, want_total: bool = True, stream=None):
    tot = ctypes.c_int64(0)
    _check(load().cg_pipeline_run(h, _stream(stream), ctypes.byref(tot) if want_total else None))
    return tot.value if want_total else None


def cg_pipeline_outputs(h: int) -> tuple[int, int, int, int]:
    ptrs = [ctypes.c_void_p() for _ in range(4)]
    _check(load().cg_pipeline_outputs(h, *[ctypes.byref(p) for p in ptrs]))
    return tuple(p.value or 0 for p in ptrs)


def cg_pipeline_info(h: int) -> dict:
    info = PipelineInfo()
    _check(load().cg_pipeline_info(h, ctypes.byref(info)))
    return {f: getattr(info, f) for f, _ in PipelineInfo._fields_}


def cg_pipeline_free(h: int):
    _check(load().cg_pipeline_free(h))


class _DeviceArray:
    """A zero-copy view of library-owned device memory (CUDA array interface)."""

    def __init__(self, ptr: int, shape, typestr: str):
        self.__cuda_array_interface__ = {"shape": tuple(shape), "typestr": typestr, "data": (ptr, False),
                                         "version": 2, "strides": None}


def _view(ptr: int, shape, typestr: str, device) -> torch.Tensor:
    if ptr == 0 or 0 in tuple(shape):
        dt = {"<i8": torch.int64, "<i4": torch.int32, "<f8": torch.float64}[typestr]
        return torch.empty(shape, dtype=dt, device=device)
    return torch.as_tensor(_DeviceArray(ptr, shape, typestr), device=device)


def cg_profile_enable(on: bool = True):
    """Device-time tracing of the library's kernel phases (CUDA events)."""
    _check(load().cg_profile_enable(1 if on else 0))


def cg_profile_read(reset: bool = True) -> dict:
    """{phase: (launches, total_ms)} since the last reset (waits for the GPU)."""
    import json
    n = ctypes.c_size_t(0)
    _check(load().cg_profile_read(None, 0, ctypes.byref(n), 0))
    buf = ctypes.create_string_buffer(n.value + 256)
    _check(load().cg_profile_read(buf, len(buf), ctypes.byref(n), 1 if reset else 0))
    return {k: (int(v[0]), float(v[1])) for k, v in json.loads(buf.value.decode()).items()}


# ------------------------------------------------------------- convenience


def cg_server_create(index_handles, slots: int = 4, memory_budget: int = 0) -> int:
    arr = (ctypes.c_void_p * len(index_handles))(*index_handles)
    opts = ServerOpts(int(slots), int(memory_budget))
    h = ctypes.c_void_p()
    _check(load().cg_server_create(arr, len(index_handles), ctypes.byref(opts), ctypes.byref(h)))
    return h.value


def cg_server_submit(h: int, index: int, q: torch.Tensor, op: int, radius: float = 0.0, kernel: int = SPHERE,
                     k: int = 0) -> int:
    req = Request(int(index), int(op), int(kernel), int(k), float(radius), _ptr(q) if q.shape[0] else None,
                  int(q.shape[0]))
    rid = ctypes.c_int64(0)
    _check(load().cg_server_submit(h, ctypes.byref(req), ctypes.byref(rid)))
    return rid.value


def cg_server_wait(h: int, rid: int, timeout_s: float = -1.0) -> Result:
    res = Result()
    code = load().cg_server_wait(h, rid, float(timeout_s), ctypes.byref(res))
    _check(code)
    return res


def cg_server_wait_any(h: int, timeout_s: float = -1.0) -> int:
    rid = ctypes.c_int64(0)
    _check(load().cg_server_wait_any(h, float(timeout_s), ctypes.byref(rid)))
    return rid.value


def cg_server_release(h: int, rid: int):
    _check(load().cg_server_release(h, rid))


def cg_server_stats(h: int) -> dict:
    st = ServerStats()
    _check(load().cg_server_stats(h, ctypes.byref(st)))
    return {f: getattr(st, f) for f, _ in ServerStats._fields_}


def cg_server_free(h: int):
    _check(load().cg_server_free(h))


class Server:
    """Continuous-batching request loop over device-resident ``Index``es."""

    def __init__(self, indexes, slots: int = 4, memory_budget: int = 0):
        self.indexes = list(indexes)  # kept alive while the server runs
        self.device = self.indexes[0].device
        self.h = cg_server_create([ix.h for ix in self.indexes], slots, memory_budget)
        self._queries = {}

    def submit_radius(self, index: int, q: torch.Tensor, r: float, kernel: int = SPHERE) -> int:
        q = _points(q)
        rid = cg_server_submit(self.h, index, q, REQ_RADIUS, radius=r, kernel=kernel)
        self._queries[rid] = (q, None)
        return rid

    def submit_knn(self, index: int, q: torch.Tensor, k: int) -> int:
        q = _points(q)
        rid = cg_server_submit(self.h, index, q, REQ_KNN, k=k)
        self._queries[rid] = (q, k)
        return rid

    def wait(self, rid: int, timeout_s: float = -1.0, copy: bool = True) -> dict:
        """The request's result (device tensors, copied out of server memory
        when ``copy``), latency and queueing time in ms."""
        res = cg_server_wait(self.h, rid, timeout_s)
        q, k = self._queries[rid]
        out = {"latency_ms": res.latency_ms, "queue_ms": res.queue_ms, "nq": res.nq}
        if k is None:
            off = _view(res.offsets or 0, (res.nq + 1,), "<i8", self.device)
            ind = _view(res.indices or 0, (res.total,), "<i4", self.device)
            out["offsets"], out["indices"] = (off.clone(), ind.clone()) if copy else (off, ind)
        else:
            idx = _view(res.knn_idx or 0, (res.nq, k), "<i4", self.device)
            d2 = _view(res.knn_d2 or 0, (res.nq, k), "<f8", self.device)
            out["idx"], out["d2"] = (idx.clone(), d2.clone()) if copy else (idx, d2)
        return out

    def wait_any(self, timeout_s: float = -1.0) -> int:
        """Id of the next finished request (completion order)."""
        return cg_server_wait_any(self.h, timeout_s)

    def release(self, rid: int):
        cg_server_release(self.h, rid)
        self._queries.pop(rid, None)

    def stats(self) -> dict:
        return cg_server_stats(self.h)

    def close(self):
        if getattr(self, "h", None):
            cg_server_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Pipeline:
    """Graph-captured batched pipeline (build + all-points radius search +
    all-points k-NN) over the tiles of ``xyz``; ``run()`` replays it on the
    current contents of ``xyz`` (same tile sizes)."""

    def __init__(self, xyz: torch.Tensor, tile_offsets, cells, radius: float, kernel: int = SPHERE, k: int = 0,
                 dim: int = 2, precision: int = FP32_OFFSET, headroom: float = 0.0, stream=None):
        self.xyz = xyz  # the pipeline reads this buffer on every replay
        self.n = xyz.shape[0]
        self.k = k
        self.device = xyz.device
        self.total = None
        self.h = cg_pipeline_create(xyz, tile_offsets, cells, dim, precision, radius, kernel, k, headroom, stream)

    def run(self, stream=None, sync: bool = True):
        t = cg_pipeline_run(self.h, sync, stream)
        if sync:
            self.total = t
        return t

    def outputs(self) -> dict:
        """Views of the last replay's outputs (pipeline-owned memory: copy
        what must outlive the next run).  Needs a synchronising run."""
        if self.total is None:
            raise RuntimeError("outputs need a run with sync=True")
        off, ind, kidx, kd2 = cg_pipeline_outputs(self.h)
        out = {"offsets": _view(off, (self.n + 1,), "<i8", self.device),
               "indices": _view(ind, (self.total,), "<i4", self.device)}
        if self.k > 0:
            out["knn_idx"] = _view(kidx, (self.n, self.k), "<i4", self.device)
            out["knn_d2"] = _view(kd2, (self.n, self.k), "<f8", self.device)
        return out

    def info(self) -> dict:
        return cg_pipeline_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            cg_pipeline_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass



class Index:
    """A device-resident grid index (owns the library handle)."""

    def __init__(self, xyz: torch.Tensor, cell_xy: float, cell_z: float | None = None, dim: int = 2,
                 flavor: int = DENSE, precision: int = FP32_OFFSET, stream=None):
        self.n = xyz.shape[0]
        self.h = cg_build(xyz, cell_xy, cell_z, dim, flavor, precision, stream)
        self.device = xyz.device

    @classmethod
    def batched(cls, xyz, tile_offsets, cells, dim=2, flavor=DENSE, precision=FP32_OFFSET, stream=None):
        self = cls.__new__(cls)
        self.n = xyz.shape[0]
        self.h = cg_build_batched(xyz, tile_offsets, cells, dim, flavor, precision, stream)
        self.device = xyz.device
        return self

    def info(self) -> dict:
        return cg_index_info(self.h)

    def close(self):
        if getattr(self, "h", None):
            cg_index_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def radius_search(self, q: torch.Tensor | None, r: float, kernel: int = SPHERE, stream=None,
                      check: bool = True):
        """CSR (offsets int64 [nq+1], indices int32 [total]); q=None: every point."""
        nq = self.n if q is None else q.shape[0]
        if q is not None and 0 < nq <= SMALL_BATCH:
            # small calls: count and fill in one call (one synchronisation)
            # into a buffer of SMALL_GUESS entries per query; longer results
            # take one more (unsynchronised) fill into a buffer of their size
            q = _points(q)
            cap = nq * SMALL_GUESS + 1024
            offsets = torch.empty(nq + 1, dtype=torch.int64, device=self.device)
            indices = torch.empty(cap, dtype=torch.int32, device=self.device)
            fits, total = cg_radius_search_into(self.h, q, r, kernel, offsets, indices, cap, stream=stream)
            if not fits:
                indices = torch.empty(max(total, 1), dtype=torch.int32, device=self.device)
                cg_radius_fill(self.h, q, r, kernel, offsets, indices, stream=stream)
            if check:
                cg_index_status(self.h, stream)
            return offsets, indices[:total]
        offsets = torch.empty(nq + 1, dtype=torch.int64, device=self.device)
        if q is None:
            total = cg_all_points_count(self.h, r, kernel, offsets, stream=stream)
        else:
            q = _points(q)
            total = cg_radius_count(self.h, q, r, kernel, offsets, stream=stream)
        indices = torch.empty(max(total, 1), dtype=torch.int32, device=self.device)
        if q is None:
            cg_all_points_fill(self.h, r, kernel, offsets, indices, stream=stream)
        else:
            cg_radius_fill(self.h, q, r, kernel, offsets, indices, stream=stream)
        if check:
            cg_index_status(self.h, stream)
        return offsets, indices[:total]

    def knn_grow(self, q: torch.Tensor, k: int, policy: int = GROW_MONOTONE, stream=None, check: bool = True):
        """Algorithm 2 step by step under a growth policy: (idx, d2, visited)."""
        q = _points(q)
        nq = q.shape[0]
        idx = torch.empty((nq, k), dtype=torch.int32, device=self.device)
        d2 = torch.empty((nq, k), dtype=torch.float64, device=self.device)
        vis = torch.empty(nq, dtype=torch.int64, device=self.device)
        cg_knn_grow(self.h, q, k, policy, idx, d2, vis, stream=stream)
        if check:
            cg_index_status(self.h, stream)
        return idx, d2, vis

    def knn(self, q: torch.Tensor | None, k: int, with_d2: bool = True, stream=None,
            check: bool = True):
        nq = self.n if q is None else q.shape[0]
        idx = torch.empty((nq, k), dtype=torch.int32, device=self.device)
        d2 = torch.empty((nq, k), dtype=torch.float64, device=self.device) if with_d2 else None
        if q is None:
            cg_all_points_knn(self.h, k, idx, d2, stream=stream)
        else:
            cg_knn(self.h, _points(q), k, idx, d2, stream=stream)
        if check:
            cg_index_status(self.h, stream)
        return idx, d2
