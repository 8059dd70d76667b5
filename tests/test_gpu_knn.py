"""Parity of the CUDA k-NN with the oracle: ids and binary64 d2 identical,
ordered by (d2, id), padding -1 / inf when fewer than k points exist."""
import numpy as np
import pytest
import torch

import cloudgen
import oracle
import paper_2502_11602_gb300 as cg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _check(xyz, q, k, cell, cell_z=None, dim=2, flavor=cg.DENSE, prec=cg.FP32_OFFSET):
    ref = oracle.Index(xyz, cell, cell_z or cell, dim=dim, flavor=flavor)
    o_idx, o_d2 = ref.knn(xyz if q is None else q, k, threads=8)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), cell, cell_z, dim=dim, flavor=flavor, precision=prec)
    g_idx, g_d2 = ix.knn(None if q is None else torch.from_numpy(q).to(DEV), k)
    torch.cuda.synchronize()
    g_idx = g_idx.cpu().numpy()
    g_d2 = g_d2.cpu().numpy()
    ix.close()
    bad = np.nonzero(np.any(g_idx != o_idx, axis=1))[0]
    assert bad.size == 0, f"{bad.size} rows differ, first {bad[:3]}: {g_idx[bad[0]]} vs {o_idx[bad[0]]}"
    assert np.array_equal(g_d2, o_d2)


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 8, 9, 16, 17, 32, 33, 64])
def test_small_als_tile_all_points(prec, k):
    xyz = cloudgen.als_uniform(60_000, extent=(75.0, 75.0))
    _check(xyz, None, k, 1.0, prec=prec)


@pytest.mark.parametrize("flavor", [cg.DENSE, cg.SPARSE, cg.MIXED])
@pytest.mark.parametrize("dim", [2, 3])
def test_flavours_and_dims(flavor, dim):
    xyz = cloudgen.als_uniform(20_000, extent=(40.0, 40.0), seed=12)
    _check(xyz, None, 16, 0.6, 0.4, dim=dim, flavor=flavor)


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
def test_ties_duplicates_and_lattice(prec):
    xyz = cloudgen.adversarial_cloud(12_000, seed=9)
    _check(xyz, None, 24, 1.0, dim=3, prec=prec)
    lat = cloudgen.lattice_cloud(8, offset=(508000.0, 5440000.0, 100.0))
    _check(lat, None, 27, 1.0, dim=3, prec=prec)
    _check(lat, None, 64, 2.0, dim=2, prec=prec)


def test_external_queries_and_far_away():
    xyz = cloudgen.als_uniform(30_000, extent=(50.0, 50.0), seed=14)
    rng = np.random.default_rng(3)
    q = np.concatenate([xyz[rng.integers(0, len(xyz), 2000)] + rng.normal(0, 0.4, (2000, 3)),
                        xyz.min(0) + rng.uniform(-30, 80, (500, 3)),
                        np.array([xyz.max(0) + 5e3])])
    for flavor in (cg.DENSE, cg.SPARSE):
        for prec in (cg.FP32_OFFSET, cg.FP64):
            _check(xyz, q, 12, 1.0, flavor=flavor, prec=prec)


def test_fewer_points_than_k_and_k64():
    xyz = cloudgen.random_cloud(20, extent=(3.0, 3.0, 1.0), seed=4)
    _check(xyz, None, 32, 1.0)
    _check(xyz, None, 64, 0.5, dim=3)
    big = cloudgen.als_uniform(15_000, extent=(30.0, 30.0), seed=15)
    _check(big, None, 64, 1.0)


def test_sparse_regions_need_wider_rings():
    # clusters far apart: most queries must look beyond the first ring
    rng = np.random.default_rng(6)
    c = rng.uniform(0, 200, (60, 3)) * [1, 1, 0.05]
    xyz = np.concatenate([cc + rng.normal(0, 0.5, (40, 3)) for cc in c]) + [508000.0, 5440000.0, 0.0]
    _check(np.ascontiguousarray(xyz), None, 50, 1.0)
