"""Graph-captured batched pipeline: build + all-points radius search +
all-points k-NN over every tile, replayed on new coordinates of the same
tile layout.  Every replay's outputs must equal the oracle run on each tile
alone (ids shifted by the tile's offset), including replays that force a
re-plan (a tile's grid changes, or the neighbour count outgrows the
capacity chosen at creation)."""
import numpy as np
import pytest
import torch

import cloudgen
import oracle
import paper_2502_11602_gb300 as cg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _tiles(ntiles, total, seed, lo=300, hi=30_000):
    sizes = cloudgen.batched_tile_sizes(ntiles, total, lo=lo, hi=hi, seed=seed)
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


def _compare(pipe, xyz, off, cells, r, kernel=cg.SPHERE, k=0, dim=2):
    out = pipe.outputs()
    g_off = out["offsets"].cpu().numpy()
    g_ind = out["indices"].cpu().numpy()
    assert g_off[0] == 0 and g_off[-1] == pipe.total == len(g_ind)
    if k:
        k_idx = out["knn_idx"].cpu().numpy()
        k_d2 = out["knn_d2"].cpu().numpy()
    for t in range(len(off) - 1):
        a, b = off[t], off[t + 1]
        tile = xyz[a:b]
        ref = oracle.Index(tile, cells[t], cells[t], dim=dim)
        o_off, o_ind = ref.radius_search(tile, r, kernel, threads=8)
        assert np.array_equal(g_off[a:b + 1] - g_off[a], o_off), f"tile {t} counts"
        assert np.array_equal(g_ind[g_off[a]:g_off[b]], o_ind + a), f"tile {t} indices"
        if k:
            r_idx, r_d2 = ref.knn(tile, k, threads=8)
            assert np.array_equal(k_idx[a:b], np.where(r_idx >= 0, r_idx + a, -1)), f"tile {t} knn ids"
            assert np.array_equal(k_d2[a:b], r_d2), f"tile {t} knn d2"


def _upload(x_dev, xyz):
    x_dev.copy_(torch.from_numpy(xyz))
    torch.cuda.synchronize()


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
def test_pipeline_replays_match_oracle(prec):
    xyz, off, cells = _tiles(12, 120_000, seed=31)
    x = torch.from_numpy(xyz).to(DEV)
    pipe = cg.Pipeline(x, off, cells, radius=1.0, k=16, precision=prec)
    info = pipe.info()
    assert info["ntiles"] == 12 and info["n"] == len(xyz) and info["graph_kernels"] > 10
    pipe.run()
    _compare(pipe, xyz, off, cells, 1.0, k=16)
    # new coordinates, same grids: points shuffled inside each tile and new
    # heights (2D index: z is not indexed)
    rng = np.random.default_rng(2)
    xyz2 = xyz.copy()
    for t in range(12):
        a, b = off[t], off[t + 1]
        xyz2[a:b] = xyz2[a:b][rng.permutation(b - a)]
    xyz2[:, 2] += rng.normal(0.0, 0.3, len(xyz2))
    _upload(x, xyz2)
    pipe.run()
    assert pipe.info()["replans"] == 0
    _compare(pipe, xyz2, off, cells, 1.0, k=16)
    # one tile shrinks: its grid changes, the replay re-plans
    xyz3 = xyz2.copy()
    a, b = off[4], off[5]
    c = xyz3[a:b, :2].mean(0)
    xyz3[a:b, :2] = c + 0.6 * (xyz3[a:b, :2] - c)
    _upload(x, xyz3)
    pipe.run()
    assert pipe.info()["replans"] == 1
    _compare(pipe, xyz3, off, cells, 1.0, k=16)
    pipe.close()


def test_pipeline_capacity_replan():
    # same bounding boxes, but most points of one tile pulled into a small
    # cluster: the neighbour count outgrows the planned output capacity
    xyz, off, cells = _tiles(6, 40_000, seed=32)
    x = torch.from_numpy(xyz).to(DEV)
    pipe = cg.Pipeline(x, off, cells, radius=1.0, k=8, headroom=1.0)
    pipe.run()
    _compare(pipe, xyz, off, cells, 1.0, k=8)
    cap = pipe.info()["capacity_indices"]
    t = int(np.argmax(np.diff(off)))
    a, b = off[t], off[t + 1]
    xyz2 = xyz.copy()
    lo, hi = xyz2[a:b].min(0), xyz2[a:b].max(0)
    rng = np.random.default_rng(3)
    keep = 4
    xyz2[a + keep:b, :2] = lo[:2] + (hi[:2] - lo[:2]) * 0.5 + rng.normal(0, 0.8, (b - a - keep, 2))
    xyz2[a + keep:b, :2] = np.clip(xyz2[a + keep:b, :2], lo[:2], hi[:2])
    xyz2[a:a + keep, :2] = [[lo[0], lo[1]], [hi[0], hi[1]], [lo[0], hi[1]], [hi[0], lo[1]]]
    _upload(x, xyz2)
    pipe.run()
    info = pipe.info()
    assert info["replans"] == 1 and pipe.total > cap
    _compare(pipe, xyz2, off, cells, 1.0, k=8)
    pipe.close()


def test_pipeline_async_replays_and_launch_count():
    xyz, off, cells = _tiles(8, 60_000, seed=33)
    x = torch.from_numpy(xyz).to(DEV)
    pipe = cg.Pipeline(x, off, cells, radius=1.5, kernel=cg.CUBE, k=4)
    kern = pipe.info()["graph_kernels"]
    c0 = cg.cg_launch_count()
    for _ in range(3):
        pipe.run(sync=False)
    pipe.run()
    # four graph replays, plus the synchronous run's readback kernel (status
    # word and CSR total, through mapped host memory)
    assert cg.cg_launch_count() - c0 == 4 * kern + 1
    _compare(pipe, xyz, off, cells, 1.5, kernel=cg.CUBE, k=4)
    pipe.close()


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
def test_pipeline_3d_sphere_no_knn(prec):
    xyz, off, cells = _tiles(5, 30_000, seed=34)
    x = torch.from_numpy(xyz).to(DEV)
    pipe = cg.Pipeline(x, off, cells, radius=0.8, k=0, dim=3, precision=prec)
    pipe.run()
    assert "knn_idx" not in pipe.outputs()
    _compare(pipe, xyz, off, cells, 0.8, dim=3)
    pipe.close()


def test_pipeline_rejects_bad_options():
    xyz, off, cells = _tiles(3, 3_000, seed=35)
    x = torch.from_numpy(xyz).to(DEV)
    with pytest.raises(cg.CheeseError):
        cg.Pipeline(x, off, cells, radius=-1.0)
    with pytest.raises(cg.CheeseError):
        cg.Pipeline(x, off, cells, radius=1.0, k=65)
    with pytest.raises(cg.CheeseError):
        cg.Pipeline(x, off, cells, radius=1.0, headroom=0.5)
