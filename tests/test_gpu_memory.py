"""The index's device memory (cg_index_info.device_bytes) equals the sum of
its documented buffers, for every flavour, dimension and precision:

  status words        256 B
  tile table          168 B per tile
  xyz64               24 n   (the caller's coordinates, exact rechecks)
  records             16 n   (binary32 offsets + id)  or  32 n (binary64)
  sid                 4 n    (original id per sorted position)
  ukeys, ustart       4 m + 4 (m + 1)      (m = non-empty voxels)
  height order        16 n + 4 n           (binary32 records on 2D grids)
  dense table         4 (ncell + 1)
  sparse / mixed hash 8 * 2^ceil(log2(max(64, 2 m)))
  mixed tables        slices B + 4 slices + 8 max(1, dense voxels)

so the memory-footprint report of the bench (index bytes against the 8 n
minimum of Section 5) reads a figure whose parts are known."""
import math

import numpy as np
import pytest
import torch

import cloudgen
import paper_2502_11602_gb300 as cg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _expected(info) -> int:
    n, m, ncell = info["n"], info["nonempty"], info["ncell"]
    b = 256 + 168 * info["ntiles"] + 24 * n + 4 * n + 4 * m + 4 * (m + 1)
    b += 16 * n if info["precision"] == cg.FP32_OFFSET else 32 * n
    if info["precision"] == cg.FP32_OFFSET and info["dim"] == 2:
        b += 16 * n + 4 * n
    if info["flavor"] == cg.DENSE:
        b += 4 * (ncell + 1)
    else:
        b += 8 * (1 << math.ceil(math.log2(max(64, 2 * m))))
    if info["flavor"] == cg.MIXED:
        slices = info["nslices"]
        per_slice = ncell // slices
        b += slices + 4 * slices + 8 * max(1, info["dense_slices"] * per_slice)
    return b


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
@pytest.mark.parametrize("flavor", [cg.DENSE, cg.SPARSE, cg.MIXED])
@pytest.mark.parametrize("dim", [2, 3])
def test_device_bytes_equal_documented_layout(dim, flavor, prec):
    xyz = cloudgen.als_uniform(50_000, extent=(60.0, 60.0), seed=9)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0, 0.5, dim=dim, flavor=flavor, precision=prec)
    try:
        info = ix.info()
    finally:
        ix.close()
    assert info["device_bytes"] == _expected(info)


def test_mixed_3d_dense_slices_counted():
    # a cloud whose lowest slices are full and upper slices sparse: the mixed
    # tables hold exactly the dense slices' voxels
    rng = np.random.default_rng(3)
    ground = np.column_stack([rng.uniform(0, 20, 40_000), rng.uniform(0, 20, 40_000), rng.uniform(0, 1.0, 40_000)])
    sky = np.column_stack([rng.uniform(0, 20, 300), rng.uniform(0, 20, 300), rng.uniform(1.0, 10.0, 300)])
    xyz = np.concatenate([ground, sky])
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0, 0.5, dim=3, flavor=cg.MIXED)
    try:
        info = ix.info()
    finally:
        ix.close()
    assert 1 <= info["dense_slices"] < info["nslices"]
    assert info["device_bytes"] == _expected(info)
