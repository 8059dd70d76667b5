"""Parity of the radius search on height-sorted columns (binary32 records
on 2D grids, sphere and cube: all-points voxel groups cut into height
chunks, each column restricted to a chunk's height range) with the oracle,
on clouds built to reach the edge cases:

* columns far taller than the kernel (most of a column outside the range);
* runs longer than the warp sort (sorted by a CTA) and longer than the
  height sort's limit (kept in id order, taken whole);
* dense patches whose groups fall in each size class, and groups too large
  for any class (the general kernel);
* external queries whose groups hold queries at very different heights,
  and queries outside the tile.

Offsets and indices must equal the oracle's element by element."""
import numpy as np
import pytest
import torch

import cloudgen
import oracle
import paper_2502_11602_gb300 as cg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
UTM = np.array([508000.0, 5440000.0, 100.0])


def _towers_cloud(seed=5):
    """Terrain at 20 pts/m2 over 40 m x 40 m plus vertical structures."""
    rng = np.random.default_rng(seed)
    parts = [np.column_stack([rng.uniform(0, 40, 32000), rng.uniform(0, 40, 32000), rng.normal(0, 0.3, 32000)])]

    def column(cx, cy, n, h, w=0.9):
        return np.column_stack([cx + rng.uniform(0, w, n), cy + rng.uniform(0, w, n), rng.uniform(0, h, n)])

    parts.append(column(5.05, 5.05, 3000, 60.0))    # run > 2048: kept in id order
    parts.append(column(10.05, 10.05, 1200, 30.0))  # sorted by a CTA
    parts.append(column(15.05, 15.05, 400, 10.0))   # sorted by a CTA (> 256)
    parts.append(column(20.05, 5.05, 200, 12.0))    # a warp
    # a wall: thin in x, 8 m long in y, 15 m tall
    n = 6000
    parts.append(np.column_stack([25.3 + rng.normal(0, 0.02, n), rng.uniform(20, 28, n), rng.uniform(0, 15, n)]))
    # dense patches for the larger size classes and the general kernel
    for (x0, y0, dens) in ((30.0, 30.0, 60), (33.0, 34.0, 150), (5.0, 30.0, 400)):
        m = int(dens * 9)
        parts.append(np.column_stack([x0 + rng.uniform(0, 3, m), y0 + rng.uniform(0, 3, m), rng.normal(0, 0.5, m)]))
    xyz = np.concatenate(parts) + UTM
    return xyz[rng.permutation(len(xyz))]


@pytest.fixture(scope="module")
def towers():
    return _towers_cloud()


def _compare(ix, ref, q, r, kernel):
    off, ind = ix.radius_search(None if q is None else torch.from_numpy(q).to(DEV), r, kernel)
    torch.cuda.synchronize()
    o_off, o_ind = ref.radius_search(ref.xyz if q is None else q, r, kernel, threads=8)
    g_off = off.cpu().numpy()
    bad = np.nonzero(g_off != o_off)[0]
    assert bad.size == 0, f"offsets differ first at {bad[:5]}"
    assert np.array_equal(ind.cpu().numpy(), o_ind)
    return int(o_off[-1])


@pytest.mark.parametrize("flavor", [cg.DENSE, cg.SPARSE, cg.MIXED])
@pytest.mark.parametrize("kernel", [cg.SPHERE, cg.CUBE])
def test_towers_all_points(towers, flavor, kernel):
    ref = oracle.Index(towers, 1.0, 1.0, dim=2, flavor=flavor)
    ix = cg.Index(torch.from_numpy(towers).to(DEV), 1.0, dim=2, flavor=flavor, precision=cg.FP32_OFFSET)
    try:
        for r in (0.3, 1.0):
            _compare(ix, ref, None, r, kernel)
    finally:
        ix.close()


@pytest.mark.parametrize("kernel", [cg.SPHERE, cg.CUBE])
def test_towers_larger_radius_and_cell(towers, kernel):
    # r = 2 on 1 m voxels (5 x 5 columns per group) and r = 1.5 on 0.5 m voxels
    ref = oracle.Index(towers, 1.0, 1.0, dim=2)
    ix = cg.Index(torch.from_numpy(towers).to(DEV), 1.0, dim=2, precision=cg.FP32_OFFSET)
    try:
        _compare(ix, ref, None, 2.0, kernel)
    finally:
        ix.close()
    ref = oracle.Index(towers, 0.5, 0.5, dim=2)
    ix = cg.Index(torch.from_numpy(towers).to(DEV), 0.5, dim=2, precision=cg.FP32_OFFSET)
    try:
        _compare(ix, ref, None, 1.5, kernel)
    finally:
        ix.close()


@pytest.mark.parametrize("kernel", [cg.SPHERE, cg.CUBE])
def test_towers_external_queries(towers, kernel):
    rng = np.random.default_rng(9)
    q = np.concatenate([
        towers[rng.integers(0, len(towers), 20000)] + rng.normal(0, 0.4, (20000, 3)),
        # the tall columns' footprints at random heights: groups mix heights
        np.column_stack([5.5 + rng.uniform(-1, 1, 3000), 5.5 + rng.uniform(-1, 1, 3000),
                         rng.uniform(-5, 70, 3000)]) + UTM,
        UTM + rng.uniform(-10, 50, (2000, 3)),           # partly outside the tile
    ])
    ref = oracle.Index(towers, 1.0, 1.0, dim=2)
    ix = cg.Index(torch.from_numpy(towers).to(DEV), 1.0, dim=2, precision=cg.FP32_OFFSET)
    try:
        for r in (0.5, 1.0):
            _compare(ix, ref, q, r, kernel)
    finally:
        ix.close()


def test_als_tile_height_chunks_match_binary64_path():
    # the height-chunked binary32 path and the binary64 path on one cloud
    xyz = cloudgen.als_urban(400_000, extent=(100.0, 100.0), seed=77)
    out = {}
    for prec in (cg.FP32_OFFSET, cg.FP64):
        ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0, dim=2, precision=prec)
        try:
            off, ind = ix.radius_search(None, 1.0, cg.SPHERE)
            out[prec] = (off.cpu().numpy(), ind.cpu().numpy())
        finally:
            ix.close()
    assert np.array_equal(out[cg.FP32_OFFSET][0], out[cg.FP64][0])
    assert np.array_equal(out[cg.FP32_OFFSET][1], out[cg.FP64][1])
    # and a sample against the oracle
    ref = oracle.Index(xyz, 1.0, 1.0, dim=2)
    rng = np.random.default_rng(3)
    sel = np.sort(rng.choice(len(xyz), 20000, replace=False))
    o_off, o_ind = ref.radius_search(xyz[sel], 1.0, oracle.SPHERE, threads=8)
    g_off, g_ind = out[cg.FP32_OFFSET]
    for t, i in enumerate(sel):
        assert np.array_equal(g_ind[g_off[i]:g_off[i + 1]], o_ind[o_off[t]:o_off[t + 1]])


@pytest.mark.parametrize("kernel", [cg.SPHERE, cg.CUBE])
def test_spatially_ordered_ids(towers, kernel):
    # ids in scan order (sorted by x, then y): a group's candidate ids fall in
    # a few narrow ranges, so the id sort of a group takes its crowded path
    xyz = towers[np.lexsort((towers[:, 1], np.floor(towers[:, 0] * 4.0)))]
    ref = oracle.Index(xyz, 1.0, 1.0, dim=2)
    ix = cg.Index(torch.from_numpy(np.ascontiguousarray(xyz)).to(DEV), 1.0, dim=2, precision=cg.FP32_OFFSET)
    try:
        for r in (0.5, 1.0, 2.0):
            _compare(ix, ref, None, r, kernel)
    finally:
        ix.close()


@pytest.mark.parametrize("flavor", [cg.DENSE, cg.SPARSE])
def test_towers_knn_all_points(towers, flavor):
    # all-points k-NN on height chunks of the height-sorted columns (k <= 32)
    # and on the voxel groups (k > 32): ids and binary64 d2 as the oracle's
    ref = oracle.Index(towers, 1.0, 1.0, dim=2, flavor=flavor)
    ix = cg.Index(torch.from_numpy(towers).to(DEV), 1.0, dim=2, flavor=flavor, precision=cg.FP32_OFFSET)
    rows = np.random.default_rng(2).choice(len(towers), 20000, replace=False)
    try:
        for k in (1, 8, 16, 32, 40):
            idx, d2 = ix.knn(None, k)
            r_idx, r_d2 = ref.knn(towers[rows], k, threads=8)
            assert np.array_equal(idx.cpu().numpy()[rows], r_idx), k
            assert np.array_equal(d2.cpu().numpy()[rows], r_d2), k
    finally:
        ix.close()
