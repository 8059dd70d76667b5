"""Parity at the workloads' full sizes, on outputs the oracle can check one
by one: sampled query rows (radius CSR rows and k-NN rows are compared with
the oracle's element by element) and whole sampled tiles of the batch.

* ALS tile: 12M points over 500 m x 500 m (the benchmark's tile), 2D grids
  of 1 m voxels in all three flavours; sphere r = 1 m with every point a
  query, cube r = 2 m and k-NN k = 16 / 32.
* TLS street canyon: 20M points, 3D grids of 0.25 m voxels, dense and
  sparse; sphere radii 0.05 - 0.5 m and k-NN k = 16 on 5M queries drawn
  from the cloud.
* Batch: 256 tiles, ~60M points, the captured pipeline (r = 1 m, k = 16)
  with autotuned cell sizes; four whole tiles against the oracle.
"""
import numpy as np
import pytest
import torch

import cloudgen
import oracle
import paper_2502_11602_gb300 as cg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _rows_equal(g_off, g_ind, rows, o_off, o_ind):
    for t, q in enumerate(rows):
        a = g_ind[g_off[q]:g_off[q + 1]]
        b = o_ind[o_off[t]:o_off[t + 1]]
        assert np.array_equal(a, b), f"row {q}"


@pytest.fixture(scope="module")
def als():
    return cloudgen.als_urban()


@pytest.mark.parametrize("flavor", [cg.DENSE, cg.SPARSE, cg.MIXED])
def test_als_12m_all_points_sphere_every_flavour(als, flavor):
    xyz = als
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0, flavor=flavor)
    off, ind = ix.radius_search(None, 1.0)
    g_off, g_ind = off.cpu().numpy(), ind.cpu().numpy()
    ix.close()
    rng = np.random.default_rng(100 + flavor)
    rows = rng.integers(0, len(xyz), 3000)
    o_off, o_ind = oracle.Index(xyz, 1.0).radius_search(xyz[rows], 1.0, threads=16)
    _rows_equal(g_off, g_ind, rows, o_off, o_ind)


def test_als_12m_cube_and_knn(als):
    xyz = als
    x = torch.from_numpy(xyz).to(DEV)
    ix = cg.Index(x, 1.0)
    ref = oracle.Index(xyz, 1.0)
    rng = np.random.default_rng(7)
    q = cloudgen.sample_queries(xyz, 40_000, seed=8) + rng.normal(0, 0.3, (40_000, 3))
    off, ind = ix.radius_search(torch.from_numpy(q).to(DEV), 2.0, cg.CUBE)
    o_off, o_ind = ref.radius_search(q, 2.0, oracle.CUBE, threads=16)
    assert np.array_equal(off.cpu().numpy(), o_off) and np.array_equal(ind.cpu().numpy(), o_ind)
    rows = rng.integers(0, len(xyz), 4000)
    for k in (16, 32):
        idx, d2 = ix.knn(None, k)
        idx, d2 = idx.cpu().numpy(), d2.cpu().numpy()
        r_idx, r_d2 = ref.knn(xyz[rows], k, threads=16)
        assert np.array_equal(idx[rows], r_idx) and np.array_equal(d2[rows], r_d2), f"k={k}"
    ix.close()


@pytest.fixture(scope="module")
def tls():
    return cloudgen.tls_street()


@pytest.mark.parametrize("flavor", [cg.DENSE, cg.SPARSE])
def test_tls_20m_3d_radii_and_knn(tls, flavor):
    xyz = tls
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 0.25, 0.25, dim=3, flavor=flavor)
    ref = oracle.Index(xyz, 0.25, 0.25, dim=3)
    q_all = cloudgen.sample_queries(xyz, 5_000_000, seed=cloudgen.CONFIG_SEED + 2)
    qd = torch.from_numpy(q_all).to(DEV)
    rng = np.random.default_rng(20 + flavor)
    for r, m in ((0.05, 50_000), (0.1, 50_000), (0.25, 20_000), (0.5, 5_000)):
        sel = rng.integers(0, len(q_all), m)
        off, ind = ix.radius_search(qd[torch.from_numpy(sel).to(DEV)].contiguous(), r)
        o_off, o_ind = ref.radius_search(q_all[sel], r, threads=16)
        assert np.array_equal(off.cpu().numpy(), o_off), f"r={r} counts"
        assert np.array_equal(ind.cpu().numpy(), o_ind), f"r={r} indices"
    # the vertical cylinder spans every z slice of the 3D grid's columns
    sel = rng.integers(0, len(q_all), 5_000)
    off, ind = ix.radius_search(qd[torch.from_numpy(sel).to(DEV)].contiguous(), 0.05, cg.CYLINDER)
    o_off, o_ind = ref.radius_search(q_all[sel], 0.05, oracle.CYLINDER, threads=16)
    assert np.array_equal(off.cpu().numpy(), o_off) and np.array_equal(ind.cpu().numpy(), o_ind), "cylinder"
    idx, d2 = ix.knn(qd, 16)
    rows = rng.integers(0, len(q_all), 5000)
    r_idx, r_d2 = ref.knn(q_all[rows], 16, threads=16)
    assert np.array_equal(idx.cpu().numpy()[rows], r_idx)
    assert np.array_equal(d2.cpu().numpy()[rows], r_d2)
    ix.close()


def test_batched_60m_pipeline_whole_tiles(tmp_path):
    from paper_2502_11602_gb300 import autotune
    xyz, off = cloudgen.batched_tiles()
    cells, _ = autotune.tune(xyz, off, radius=1.0, k=16, cache_path=str(tmp_path / "tune.json"))
    x = torch.from_numpy(xyz).to(DEV)
    pipe = cg.Pipeline(x, off, cells, radius=1.0, k=16)
    pipe.run()
    out = pipe.outputs()
    g_off = out["offsets"].cpu().numpy()
    g_ind = out["indices"].cpu().numpy()
    k_idx = out["knn_idx"].cpu().numpy()
    k_d2 = out["knn_d2"].cpu().numpy()
    pipe.close()
    sizes = np.diff(off)
    rng = np.random.default_rng(3)
    tiles = {int(np.argmin(sizes)), int(np.argmax(sizes))} | set(rng.integers(0, len(sizes), 2).tolist())
    for t in sorted(tiles):
        a, b = off[t], off[t + 1]
        tile = xyz[a:b]
        ref = oracle.Index(tile, cells[t])
        o_off, o_ind = ref.radius_search(tile, 1.0, threads=16)
        assert np.array_equal(g_off[a:b + 1] - g_off[a], o_off), f"tile {t} counts"
        assert np.array_equal(g_ind[g_off[a]:g_off[b]], o_ind + a), f"tile {t} indices"
        r_idx, r_d2 = ref.knn(tile, 16, threads=16)
        assert np.array_equal(k_idx[a:b], np.where(r_idx >= 0, r_idx + a, -1)), f"tile {t} knn"
        assert np.array_equal(k_d2[a:b], r_d2), f"tile {t} knn d2"
