"""Parity of the CUDA radius search (count + scan + fill) with the oracle.

Every comparison is element by element on the CSR output: offsets and
indices must be identical (integer results: bit-exact)."""
import numpy as np
import pytest
import torch

import cloudgen
import oracle
import paper_2502_11602_gb300 as cg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _gpu_csr(ix, q, r, kernel):
    off, ind = ix.radius_search(None if q is None else torch.from_numpy(q).to(DEV), r, kernel)
    torch.cuda.synchronize()
    return off.cpu().numpy(), ind.cpu().numpy()


def _check(xyz, q, r, cell, cell_z=None, dim=2, flavor=cg.DENSE, prec=cg.FP32_OFFSET,
           kernel=cg.SPHERE, threads=8):
    ref = oracle.Index(xyz, cell, cell_z or cell, dim=dim, flavor=flavor)
    o_off, o_ind = ref.radius_search(xyz if q is None else q, r, kernel, threads=threads)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), cell, cell_z, dim=dim, flavor=flavor, precision=prec)
    g_off, g_ind = _gpu_csr(ix, q, r, kernel)
    ix.close()
    assert g_off.shape == o_off.shape
    bad = np.nonzero(g_off != o_off)[0]
    assert bad.size == 0, f"offsets differ first at {bad[:5]}"
    assert np.array_equal(g_ind, o_ind)
    return int(o_off[-1])


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
def test_small_als_tile_all_points(prec):
    # the 100k-point tile, 2D dense grid, 1 m voxels, sphere r = 1 m
    xyz = cloudgen.als_uniform()
    total = _check(xyz, None, 1.0, 1.0, prec=prec)
    assert 25 * len(xyz) < total < 40 * len(xyz)


@pytest.mark.parametrize("flavor", [cg.DENSE, cg.SPARSE, cg.MIXED])
@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kernel", [cg.SPHERE, cg.CUBE])
def test_flavours_dims_kernels(flavor, dim, kernel):
    xyz = cloudgen.als_uniform(30_000, extent=(40.0, 40.0), seed=3)
    _check(xyz, None, 1.3, 0.7, 0.5, dim=dim, flavor=flavor, kernel=kernel)


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
def test_adversarial_cloud(prec):
    # duplicates, points on voxel faces, tight clusters at a UTM offset
    xyz = cloudgen.adversarial_cloud(20_000, seed=21)
    for r in (0.5, 1.0, 2.0):
        _check(xyz, None, r, 1.0, dim=3, prec=prec)
        _check(xyz, None, r, 1.0, dim=2, flavor=cg.SPARSE, prec=prec, kernel=cg.CUBE)


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
def test_lattice_exact_boundaries(prec):
    # integer lattice: many pairs at exactly d^2 == r^2 (3-4-0, 5-0-0, ...)
    xyz = cloudgen.lattice_cloud(12, offset=(508000.0, 5440000.0, 100.0))
    for r in (1.0, 2.0, 5.0):
        _check(xyz, None, r, 1.0, dim=3, prec=prec)
        _check(xyz, None, r, 1.0, dim=2, prec=prec, kernel=cg.CUBE)


def test_external_queries_inside_and_outside():
    xyz = cloudgen.als_uniform(40_000, extent=(50.0, 50.0), seed=8)
    rng = np.random.default_rng(1)
    q = np.concatenate([
        xyz[rng.integers(0, len(xyz), 3000)] + rng.normal(0, 0.3, (3000, 3)),
        xyz.min(0) + rng.uniform(-20, 70, (1000, 3)),   # partly outside the bbox
        np.array([[0.0, 0.0, 0.0], xyz.max(0) + 1e4]),   # very far away
    ])
    for flavor in (cg.DENSE, cg.SPARSE, cg.MIXED):
        for prec in (cg.FP32_OFFSET, cg.FP64):
            _check(xyz, q, 1.5, 1.0, flavor=flavor, prec=prec)


def test_heavy_blocks_multi_chunk_rows():
    # dense clusters: staged candidates exceed one shared-memory chunk, rows
    # are assembled from several sorted runs and sorted afterwards
    rng = np.random.default_rng(4)
    a = rng.normal(0, 0.15, (30_000, 3)) + [508000.0, 5440000.0, 0.0]
    b = rng.uniform(0, 20, (10_000, 3)) + [507990.0, 5439990.0, 0.0]
    xyz = np.ascontiguousarray(np.concatenate([a, b]))
    _check(xyz, None, 0.5, 1.0)
    _check(xyz, None, 2.0, 1.0, dim=3, kernel=cg.CUBE, prec=cg.FP64)


def test_repeated_fill_and_stream_order():
    xyz = cloudgen.als_uniform(20_000, extent=(40.0, 40.0), seed=5)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0)
    a = _gpu_csr(ix, None, 1.0, cg.SPHERE)
    b = _gpu_csr(ix, None, 1.0, cg.SPHERE)
    c = _gpu_csr(ix, None, 2.0, cg.CUBE)
    d = _gpu_csr(ix, None, 1.0, cg.SPHERE)
    assert np.array_equal(a[1], b[1]) and np.array_equal(a[1], d[1])
    ref = oracle.Index(xyz, 1.0).radius_search(xyz, 2.0, oracle.CUBE, threads=8)
    assert np.array_equal(c[0], ref[0]) and np.array_equal(c[1], ref[1])
    ix.close()


def test_single_point_and_tiny():
    xyz = np.array([[508000.5, 5440000.5, 3.0]])
    _check(xyz, None, 1.0, 1.0)
    xyz = np.array([[0.0, 0.0, 0.0], [0.0, 0.0, 0.0], [1.0, 0.0, 0.0]])
    _check(xyz, None, 1.0, 1.0, dim=3)


def test_invalid_arguments_raise():
    xyz = torch.from_numpy(cloudgen.als_uniform(1000, extent=(10.0, 10.0), seed=2)).to(DEV)
    ix = cg.Index(xyz, 1.0)
    off = torch.empty(1001, dtype=torch.int64, device=DEV)
    with pytest.raises(cg.CheeseError):
        cg.cg_all_points_count(ix.h, -1.0, cg.SPHERE, off)
    with pytest.raises(cg.CheeseError):
        cg.cg_all_points_count(ix.h, float("inf"), cg.SPHERE, off)
    bad = xyz.clone()
    bad[5, 1] = float("nan")
    with pytest.raises(cg.CheeseError):
        cg.Index(bad, 1.0)
    q = xyz[:10].clone()
    q[3, 0] = float("nan")
    with pytest.raises(cg.CheeseError):
        ix.radius_search(q, 1.0)
    ix.close()


def test_als_12m_tile_sampled_parity():
    """Full-size ALS tile (12M points, 500 m x 500 m), the benchmark's launch:
    all points as queries at r = 1 m.  Rows of a seeded sample of queries
    are compared with the oracle one by one; the totals must agree with the
    invariants (symmetry sample, every point its own neighbour)."""
    xyz = cloudgen.als_urban()
    x = torch.from_numpy(xyz).to(DEV)
    ix = cg.Index(x, 1.0)
    off, ind = ix.radius_search(None, 1.0)
    torch.cuda.synchronize()
    ref = oracle.Index(xyz, 1.0)
    rng = np.random.default_rng(77)
    sample = rng.integers(0, len(xyz), 4000)
    o_off, o_ind = ref.radius_search(xyz[sample], 1.0, threads=8)
    g_off = off.cpu().numpy()
    g_ind = ind.cpu().numpy()
    for t, q in enumerate(sample):
        row = g_ind[g_off[q]:g_off[q + 1]]
        assert np.array_equal(row, o_ind[o_off[t]:o_off[t + 1]]), f"row {q}"
        assert q in set(row.tolist())
    # symmetry on the sampled rows
    for q in sample[:300]:
        for j in g_ind[g_off[q]:g_off[q + 1]][:50]:
            assert q in set(g_ind[g_off[j]:g_off[j + 1]].tolist())
    ix.close()


@pytest.mark.parametrize("kernel", [cg.SPHERE, cg.CUBE])
def test_tall_columns_and_stacked_layers(kernel):
    # vertical structures spanning > 32 search radii in z (z-groups wider
    # than r), stacked ground / roof layers and points below the origin
    rng = np.random.default_rng(10)
    n = 30_000
    ground = np.stack([rng.uniform(0, 30, n), rng.uniform(0, 30, n), rng.normal(-3.0, 0.05, n)], 1)
    roof = np.stack([rng.uniform(5, 15, n // 2), rng.uniform(5, 15, n // 2), rng.normal(12.0, 0.05, n // 2)], 1)
    poles = []
    for px, py in rng.uniform(0, 30, (40, 2)):
        m = 800
        poles.append(np.stack([px + rng.normal(0, 0.05, m), py + rng.normal(0, 0.05, m), rng.uniform(-3, 120, m)], 1))
    xyz = np.ascontiguousarray(np.concatenate([ground, roof] + poles) + [508000.0, 5440000.0, 0.0])
    for r in (0.4, 1.0, 2.5):
        _check(xyz, None, r, 1.0, kernel=kernel)


def test_query_buffer_rewritten_in_place_is_planned_again():
    # the same device buffer (same pointer, same size) with new contents must
    # give the new contents' results, for radius search and k-NN alike
    xyz = cloudgen.als_uniform(30_000, extent=(40.0, 40.0), seed=12)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0)
    ref = oracle.Index(xyz, 1.0)
    rng = np.random.default_rng(5)
    q = torch.empty((2000, 3), dtype=torch.float64, device=DEV)
    for trial in range(3):
        qh = xyz[rng.integers(0, len(xyz), 2000)] + rng.normal(0, 0.5, (2000, 3))
        q.copy_(torch.from_numpy(qh))
        off, ind = ix.radius_search(q, 1.2)
        o_off, o_ind = ref.radius_search(qh, 1.2, threads=8)
        assert np.array_equal(off.cpu().numpy(), o_off) and np.array_equal(ind.cpu().numpy(), o_ind)
        idx, d2 = ix.knn(q, 8)
        r_idx, r_d2 = ref.knn(qh, 8, threads=8)
        assert np.array_equal(idx.cpu().numpy(), r_idx) and np.array_equal(d2.cpu().numpy(), r_d2)
    ix.close()


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
@pytest.mark.parametrize("dim,flavor", [(2, cg.DENSE), (3, cg.DENSE), (3, cg.SPARSE), (3, cg.MIXED)])
def test_cylinder_kernel(prec, dim, flavor):
    # vertical cylinder: every height within the horizontal radius (on a 3D
    # grid every z slice of the voxel columns is searched)
    xyz = cloudgen.als_uniform(20_000, extent=(30.0, 30.0), seed=14)
    rng = np.random.default_rng(6)
    poles = np.stack([rng.uniform(0, 30, 4000), rng.uniform(0, 30, 4000), rng.uniform(-3, 25, 4000)], 1)
    xyz = np.ascontiguousarray(np.concatenate([xyz, poles + xyz.min(0) * [1, 1, 0]]))
    for r in (0.4, 1.0, 2.2):
        _check(xyz, None, r, 1.0, 0.5, dim=dim, flavor=flavor, prec=prec, kernel=cg.CYLINDER)
    q = xyz[rng.integers(0, len(xyz), 500)] + rng.normal(0, 2.0, (500, 3))
    _check(xyz, q, 1.5, 1.0, 0.5, dim=dim, flavor=flavor, prec=prec, kernel=cg.CYLINDER)
