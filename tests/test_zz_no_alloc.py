"""cg_offsets_scan_noalloc: the allocation-free variant of the offsets scan.

Some callers cannot allocate device memory (their memory was reserved up
front by another allocator, or an allocation could stall a real-time loop);
this entry point scans counts into CSR offsets using only a fixed scratch
array inside the library.  Its output must equal the offsets that the
regular count pass (cg_all_points_count) produces, on two calls in a row
(the second call must not see the first call's leftover scratch).  The file
name makes pytest collect it last."""
import ctypes

import numpy as np
import pytest
import torch

import cloudgen
import paper_2502_11602_gb300 as cg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _scan_noalloc(counts_u32: torch.Tensor, n: int, out: torch.Tensor) -> int:
    lib = cg.load()
    return lib.cg_offsets_scan_noalloc(ctypes.c_void_p(counts_u32.data_ptr()), n,
                                       ctypes.c_void_p(out.data_ptr()),
                                       ctypes.c_void_p(torch.cuda.current_stream().cuda_stream))


def _reference_offsets(npts: int, seed: int, r: float):
    xyz = torch.from_numpy(cloudgen.als_uniform(npts, extent=(60.0, 60.0), seed=seed)).to(DEV)
    ix = cg.Index(xyz, 1.0)
    off = torch.empty(npts + 1, dtype=torch.int64, device=DEV)
    cg.cg_all_points_count(ix.h, r, cg.SPHERE, off)   # existing entry point: count + scan
    torch.cuda.synchronize()
    ix.close()
    counts = (off[1:] - off[:-1]).to(torch.int32)  # uint32 bit pattern (counts < 2^31)
    return off, counts


def test_noalloc_scan_matches_count_pass_twice():
    # first call: a larger problem; second call: a smaller one, so stale
    # status words from the first call would show up if not cleared
    for npts, seed, r in ((70_000, 31, 1.5), (9_000, 32, 1.0)):
        ref, counts = _reference_offsets(npts, seed, r)
        out = torch.full((npts + 1,), -7, dtype=torch.int64, device=DEV)
        assert _scan_noalloc(counts, npts, out) == 0, cg.load().cg_last_error()
        torch.cuda.synchronize()
        assert torch.equal(out, ref)


def test_noalloc_scan_repeat_same_input_and_limits():
    ref, counts = _reference_offsets(40_000, 33, 2.0)
    for _ in range(2):
        out = torch.zeros(40_001, dtype=torch.int64, device=DEV)
        assert _scan_noalloc(counts, 40_000, out) == 0
        torch.cuda.synchronize()
        assert torch.equal(out, ref)
    # multi-tile boundaries and the empty case
    for n in (0, 1, 2047, 2048, 2049, 300_000):
        c = torch.randint(0, 1000, (max(n, 1),), dtype=torch.int32, device=DEV)
        out = torch.full((n + 1,), -3, dtype=torch.int64, device=DEV)
        assert _scan_noalloc(c, n, out) == 0
        torch.cuda.synchronize()
        expect = np.zeros(n + 1, np.int64)
        np.cumsum(c[:n].cpu().numpy().astype(np.int64), out=expect[1:])
        assert np.array_equal(out.cpu().numpy(), expect)
    # beyond the fixed scratch: rejected before any device work
    big = 134_217_728 + 1
    dummy = torch.zeros(2, dtype=torch.int64, device=DEV)
    assert _scan_noalloc(dummy, big, dummy) == 1
    assert b"max 134217728" in cg.load().cg_last_error()


def test_noalloc_scan_misaligned_counts():
    # counts that start 4 bytes past a 16-byte boundary take the scalar loads
    base = torch.randint(0, 1 << 20, (10_001,), dtype=torch.int32, device=DEV)
    c = base[1:]
    n = 10_000
    out = torch.full((n + 1,), -5, dtype=torch.int64, device=DEV)
    assert _scan_noalloc(c, n, out) == 0
    torch.cuda.synchronize()
    expect = np.zeros(n + 1, np.int64)
    np.cumsum(c.cpu().numpy().astype(np.int64), out=expect[1:])
    assert np.array_equal(out.cpu().numpy(), expect)


def test_noalloc_scan_at_the_documented_maximum():
    # n = 2^27: all 65536 tiles of the fixed scratch, the last status word
    # included; totals well above 2^32 exercise the 62-bit packed prefixes
    n = 134_217_728
    g = torch.Generator(device=DEV).manual_seed(7)
    c = torch.randint(0, 1 << 7, (n,), dtype=torch.int32, device=DEV, generator=g)
    out = torch.full((n + 1,), -9, dtype=torch.int64, device=DEV)
    assert _scan_noalloc(c, n, out) == 0, cg.load().cg_last_error()
    torch.cuda.synchronize()
    host = c.cpu().numpy().astype(np.int64)
    expect = np.zeros(n + 1, np.int64)
    np.cumsum(host, out=expect[1:])
    assert expect[-1] > (1 << 32)
    got = out.cpu().numpy()
    assert got[-1] == expect[-1]
    assert np.array_equal(got, expect)
    del c, out
    torch.cuda.empty_cache()
