"""Batched tiles: one index over many independent tiles (own bounding box,
origin, grid and cell size each); every point queries its own tile.  Each
tile's rows must equal the oracle run on that tile alone (ids shifted by
the tile's offset in the concatenated array)."""
import numpy as np
import pytest
import torch

import cloudgen
import oracle
import paper_2502_11602_gb300 as cg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _tiles(ntiles, total, seed):
    sizes = cloudgen.batched_tile_sizes(ntiles, total, lo=200, hi=20_000, seed=seed)
    rng = np.random.default_rng(seed)
    parts, cells = [], []
    for t, n in enumerate(sizes):
        dens = rng.uniform(5.0, 60.0)
        side = float(np.sqrt(n / dens))
        org = (400000.0 + 1000.0 * rng.integers(0, 50), 5000000.0 + 1000.0 * rng.integers(0, 50), 0.0)
        parts.append(cloudgen.als_uniform(int(n), (side, side), seed=seed * 100 + t, offset=org))
        cells.append(float(rng.choice([0.5, 1.0, 2.0])))
    off = np.zeros(ntiles + 1, np.int64)
    np.cumsum(sizes, out=off[1:])
    return np.ascontiguousarray(np.concatenate(parts)), off, np.array(cells)


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
def test_batched_radius_and_knn_match_per_tile_oracle(prec):
    xyz, off, cells = _tiles(24, 150_000, seed=5)
    ix = cg.Index.batched(torch.from_numpy(xyz).to(DEV), off, cells, precision=prec)
    info = ix.info()
    assert info["ntiles"] == 24 and info["n"] == len(xyz)
    g_off, g_ind = ix.radius_search(None, 1.0)
    k_idx, k_d2 = ix.knn(None, 16)
    g_off = g_off.cpu().numpy(); g_ind = g_ind.cpu().numpy()
    k_idx = k_idx.cpu().numpy(); k_d2 = k_d2.cpu().numpy()
    for t in range(24):
        a, b = off[t], off[t + 1]
        tile = xyz[a:b]
        ref = oracle.Index(tile, cells[t])
        o_off, o_ind = ref.radius_search(tile, 1.0, threads=8)
        rows = g_off[a:b + 1] - g_off[a]
        assert np.array_equal(rows, o_off), f"tile {t} counts"
        assert np.array_equal(g_ind[g_off[a]:g_off[b]], o_ind + a), f"tile {t} indices"
        r_idx, r_d2 = ref.knn(tile, 16, threads=8)
        r_idx = np.where(r_idx >= 0, r_idx + a, -1)
        assert np.array_equal(k_idx[a:b], r_idx), f"tile {t} knn ids"
        assert np.array_equal(k_d2[a:b], r_d2), f"tile {t} knn d2"
    ix.close()


def test_batched_rejects_external_queries_and_bad_offsets():
    xyz, off, cells = _tiles(4, 8_000, seed=6)
    x = torch.from_numpy(xyz).to(DEV)
    ix = cg.Index.batched(x, off, cells)
    with pytest.raises(cg.CheeseError):
        ix.radius_search(x[:10].contiguous(), 1.0)
    ix.close()
    bad = off.copy(); bad[2] = bad[1]
    with pytest.raises(cg.CheeseError):
        cg.Index.batched(x, bad, cells)
