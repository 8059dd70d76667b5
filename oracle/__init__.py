"""CPU oracle for the Cheesemap grid index and its queries (arXiv 2502.11602).

TEST INFRASTRUCTURE ONLY.  This package wraps ``cheese_oracle.c``, a plain,
single-threaded C restatement of Section 3 of the paper (grid of Eqs.
grid-size / chs-point-to-idcs / indices-to-global, the dense, sparse and mixed
flavours of Section 3.3, Algorithm 1 and Algorithm 2) plus brute force.  Only
the tests, ``__graft_entry__.smoke()`` and the CPU-baseline leg of
``bench.py`` may import it; the CUDA library never does, and the two share no
code.

Conventions: points and queries are float64 arrays of shape ``(n, 3)``
(C-contiguous, AoS), results use original 0-based indices.  Predicates:
sphere ``fl(fl(fl(dx*dx)+fl(dy*dy))+fl(dz*dz)) <= fl(r*r)``, cube
``max(fl(dx*dx), fl(dy*dy), fl(dz*dz)) <= fl(r*r)``, k-NN order
``(d2, index)``.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "cheese_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None

DENSE, SPARSE, MIXED = 0, 1, 2
SPHERE, CUBE, CYLINDER = 0, 1, 2
GROW_MONOTONE, GROW_DENSITY = 0, 1

_CFLAGS = ["-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-shared", "-fPIC"]


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (no FMA contraction); returns the .so path."""
    os.makedirs(_BUILD, exist_ok=True)
    if force or not os.path.exists(_LIB_PATH) or os.path.getmtime(_LIB_PATH) < os.path.getmtime(_SRC):
        tmp = _LIB_PATH + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", *_CFLAGS, "-o", tmp, _SRC, "-lm", "-lpthread"])
        os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is not None:
            return _lib
        lib = ctypes.CDLL(build())
        P = ctypes.c_void_p
        I64 = ctypes.c_int64
        D = ctypes.c_double
        I = ctypes.c_int
        sig = {
            "og_d2": (D, [P, P]),
            "og_cube2": (D, [P, P]),
            "og_bbox": (None, [P, I64, P, P]),
            "og_grid_size": (I64, [D, D, D]),
            "og_voxel_coord": (I64, [D, D, D]),
            "og_build": (P, [P, I64, D, D, I, I]),
            "og_free": (None, [P]),
            "og_info": (None, [P, P, P, P, P, P, P]),
            "og_slice_dense": (I, [P, I64]),
            "og_voxel_count": (I64, [P, I64, I64, I64]),
            "og_voxel_stored": (I, [P, I64, I64, I64]),
            "og_kernel_search": (I64, [P, P, D, I, P]),
            "og_radius_count": (None, [P, P, I64, D, I, P]),
            "og_radius_fill": (None, [P, P, I64, D, I, P, P]),
            "og_knn_one": (None, [P, P, I64, P, P]),
            "og_knn": (None, [P, P, I64, I64, P, P]),
            "og_brute_radius_one": (I64, [P, I64, P, D, I, P]),
            "og_brute_knn_one": (None, [P, I64, P, I64, P, P]),
            "og_radius_count_mt": (None, [P, P, I64, D, I, P, I]),
            "og_radius_fill_mt": (None, [P, P, I64, D, I, P, P, I]),
            "og_knn_mt": (None, [P, P, I64, I64, P, P, I]),
            "og_knn_policy_mt": (None, [P, P, I64, I64, I, P, P, P, I]),
        }
        for name, (res, args) in sig.items():
            f = getattr(lib, name)
            f.restype = res
            f.argtypes = args
        _lib = lib
        return lib


def _pts(a) -> np.ndarray:
    a = np.ascontiguousarray(a, dtype=np.float64)
    if a.ndim != 2 or a.shape[1] != 3:
        raise ValueError("points must have shape (n, 3)")
    return a


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(ctypes.c_void_p)


def d2(p, c) -> float:
    """Sphere predicate value for one pair (fixed evaluation order)."""
    p = np.ascontiguousarray(p, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    return _load().og_d2(_ptr(p), _ptr(c))


def cube2(p, c) -> float:
    p = np.ascontiguousarray(p, dtype=np.float64)
    c = np.ascontiguousarray(c, dtype=np.float64)
    return _load().og_cube2(_ptr(p), _ptr(c))


def grid_size(lo: float, hi: float, s: float) -> int:
    """Eq. grid-size of Section 3.2."""
    return int(_load().og_grid_size(lo, hi, s))


def voxel_coord(p: float, lo: float, s: float) -> int:
    """Eq. chs-point-to-idcs of Section 3.2 (0-based)."""
    return int(_load().og_voxel_coord(p, lo, s))


def bbox(xyz):
    xyz = _pts(xyz)
    lo = np.zeros(3)
    hi = np.zeros(3)
    _load().og_bbox(_ptr(xyz), xyz.shape[0], _ptr(lo), _ptr(hi))
    return lo, hi


class Index:
    """Grid index of Section 3 over ``xyz`` (kept alive by this object)."""

    def __init__(self, xyz, cell_xy: float, cell_z: float | None = None, dim: int = 2,
                 flavor: int = DENSE):
        lib = _load()
        self.xyz = _pts(xyz)
        self.n = self.xyz.shape[0]
        self.cell_xy = float(cell_xy)
        self.cell_z = float(cell_z if cell_z is not None else cell_xy)
        self.dim = dim
        self.flavor = flavor
        self._h = lib.og_build(_ptr(self.xyz), self.n, self.cell_xy, self.cell_z, dim, flavor)
        if not self._h:
            raise ValueError("oracle index build failed (invalid arguments or out of memory)")

    def __del__(self):
        h = getattr(self, "_h", None)
        if h:
            _load().og_free(h)
            self._h = None

    def info(self) -> dict:
        nc = np.zeros(3, np.int64)
        lo = np.zeros(3)
        hi = np.zeros(3)
        ncell = ctypes.c_int64()
        ne = ctypes.c_int64()
        nsl = ctypes.c_int64()
        _load().og_info(self._h, _ptr(nc), _ptr(lo), _ptr(hi), ctypes.byref(ncell),
                        ctypes.byref(ne), ctypes.byref(nsl))
        return {"nc": tuple(int(v) for v in nc), "lo": lo, "hi": hi, "ncell": ncell.value,
                "nonempty": ne.value, "nslices": nsl.value}

    def slice_dense(self, sl: int) -> bool:
        return bool(_load().og_slice_dense(self._h, sl))

    def voxel_count(self, i: int, j: int, k: int = 0) -> int:
        return int(_load().og_voxel_count(self._h, i, j, k))

    def voxel_stored(self, i: int, j: int, k: int = 0) -> bool:
        return bool(_load().og_voxel_stored(self._h, i, j, k))

    def kernel_search(self, c, r: float, kernel: int = SPHERE) -> np.ndarray:
        """Algorithm 1 for one query: ascending original ids inside the kernel."""
        c = np.ascontiguousarray(c, dtype=np.float64)
        out = np.empty(self.n, np.int64)
        m = _load().og_kernel_search(self._h, _ptr(c), float(r), kernel, _ptr(out))
        return out[:m].copy()

    def radius_count(self, q, r: float, kernel: int = SPHERE, threads: int = 1) -> np.ndarray:
        q = _pts(q)
        counts = np.empty(q.shape[0], np.int64)
        if threads <= 1:
            _load().og_radius_count(self._h, _ptr(q), q.shape[0], float(r), kernel, _ptr(counts))
        else:
            _load().og_radius_count_mt(self._h, _ptr(q), q.shape[0], float(r), kernel,
                                       _ptr(counts), threads)
        return counts

    def radius_search(self, q, r: float, kernel: int = SPHERE, threads: int = 1):
        """CSR (offsets int64[nq+1], indices int32[total]), rows ascending."""
        q = _pts(q)
        counts = self.radius_count(q, r, kernel, threads)
        offsets = np.zeros(q.shape[0] + 1, np.int64)
        np.cumsum(counts, out=offsets[1:])
        indices = np.empty(int(offsets[-1]), np.int32)
        if threads <= 1:
            _load().og_radius_fill(self._h, _ptr(q), q.shape[0], float(r), kernel, _ptr(offsets),
                                   _ptr(indices))
        else:
            _load().og_radius_fill_mt(self._h, _ptr(q), q.shape[0], float(r), kernel,
                                      _ptr(offsets), _ptr(indices), threads)
        return offsets, indices

    def knn(self, q, k: int, threads: int = 1):
        """Algorithm 2: (idx int32[nq,k], d2 float64[nq,k]); -1 / inf padding."""
        q = _pts(q)
        idx = np.empty((q.shape[0], k), np.int32)
        dd = np.empty((q.shape[0], k), np.float64)
        if threads <= 1:
            _load().og_knn(self._h, _ptr(q), q.shape[0], k, _ptr(idx), _ptr(dd))
        else:
            _load().og_knn_mt(self._h, _ptr(q), q.shape[0], k, _ptr(idx), _ptr(dd), threads)
        return idx, dd

    def knn_policy(self, q, k: int, policy: int = GROW_MONOTONE, threads: int = 1):
        """Algorithm 2 under a growth policy (GROW_MONOTONE: r + s;
        GROW_DENSITY: the density step of Section 3.4.2): (idx, d2, visited)
        with visited[i] the voxels of query i's final taboo box."""
        q = _pts(q)
        idx = np.empty((q.shape[0], k), np.int32)
        dd = np.empty((q.shape[0], k), np.float64)
        vis = np.empty(q.shape[0], np.int64)
        _load().og_knn_policy_mt(self._h, _ptr(q), q.shape[0], k, int(policy), _ptr(idx), _ptr(dd), _ptr(vis),
                                 max(1, threads))
        return idx, dd, vis


def brute_radius(xyz, c, r: float, kernel: int = SPHERE) -> np.ndarray:
    """O(N) scan: every point inside the kernel, ascending ids."""
    xyz = _pts(xyz)
    c = np.ascontiguousarray(c, dtype=np.float64)
    out = np.empty(xyz.shape[0], np.int64)
    m = _load().og_brute_radius_one(_ptr(xyz), xyz.shape[0], _ptr(c), float(r), kernel, _ptr(out))
    return out[:m].copy()


def brute_knn(xyz, c, k: int):
    """O(N log N): the first min(k, N) points under (d2, id)."""
    xyz = _pts(xyz)
    c = np.ascontiguousarray(c, dtype=np.float64)
    idx = np.empty(k, np.int32)
    dd = np.empty(k, np.float64)
    _load().og_brute_knn_one(_ptr(xyz), xyz.shape[0], _ptr(c), k, _ptr(idx), _ptr(dd))
    return idx, dd
