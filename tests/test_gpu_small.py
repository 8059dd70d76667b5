"""Small query batches (at most 1024 external queries): the radius search
runs one warp per query without a query plan, and k-NN runs Algorithm 2 one
warp per query.  Results must equal the oracle's element by element for 1,
10, 100 and 1000 queries, every kernel, flavour, dimension and precision,
with queries inside, outside and far from the cloud, and equal the regular
path's results for the same queries (reached with a larger batch)."""
import numpy as np
import pytest
import torch

import cloudgen
import oracle
import paper_2502_11602_gb300 as cg

pytestmark = pytest.mark.gpu

DEV = "cuda:0"


def _queries(xyz, m, seed):
    rng = np.random.default_rng(seed)
    q = xyz[rng.integers(0, len(xyz), m)] + rng.normal(0, 0.4, (m, 3))
    if m >= 10:
        q[-1] = xyz.max(0) + 3e3            # far away
        q[-2] = xyz.min(0) - [5.0, 5.0, 50.0]  # outside the box
    return np.ascontiguousarray(q)


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
@pytest.mark.parametrize("dim,flavor", [(2, cg.DENSE), (2, cg.MIXED), (3, cg.SPARSE), (3, cg.DENSE)])
def test_small_radius_batches(prec, dim, flavor):
    xyz = cloudgen.adversarial_cloud(20_000, seed=31)
    ref = oracle.Index(xyz, 1.0, 0.5, dim=dim, flavor=flavor)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0, 0.5, dim=dim, flavor=flavor, precision=prec)
    try:
        for m in (1, 10, 100, 1000):
            q = _queries(xyz, m, seed=m + dim)
            for kern in (cg.SPHERE, cg.CUBE, cg.CYLINDER):
                r = 0.3 if kern == cg.CYLINDER and dim == 3 else 1.2
                off, ind = ix.radius_search(torch.from_numpy(q).to(DEV), r, kern)
                o_off, o_ind = ref.radius_search(q, r, kern, threads=8)
                assert np.array_equal(off.cpu().numpy(), o_off), (m, kern)
                assert np.array_equal(ind.cpu().numpy(), o_ind), (m, kern)
    finally:
        ix.close()


def test_small_radius_equals_regular_path():
    xyz = cloudgen.als_uniform(50_000, extent=(60.0, 60.0), seed=5)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0)
    try:
        q = _queries(xyz, 3000, seed=1)
        qd = torch.from_numpy(q).to(DEV)
        off_big, ind_big = ix.radius_search(qd, 1.0)   # 3000 queries: the regular path
        off_big, ind_big = off_big.cpu().numpy(), ind_big.cpu().numpy()
        for a in range(0, 3000, 1000):                   # the same queries, 1000 at a time
            off, ind = ix.radius_search(qd[a:a + 1000].contiguous(), 1.0)
            off, ind = off.cpu().numpy(), ind.cpu().numpy()
            assert np.array_equal(off, off_big[a:a + 1001] - off_big[a])
            assert np.array_equal(ind, ind_big[off_big[a]:off_big[a + 1000]])
    finally:
        ix.close()


def test_small_radius_long_rows_take_the_regular_path():
    # rows longer than the warp's buffer (2048): a dense blob, r = 1 m
    rng = np.random.default_rng(2)
    xyz = np.ascontiguousarray(rng.normal(0, 0.3, (30_000, 3)) + [508000.0, 5440000.0, 0.0])
    q = np.ascontiguousarray(xyz[:20] + 0.01)
    ref = oracle.Index(xyz, 1.0)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0)
    try:
        off, ind = ix.radius_search(torch.from_numpy(q).to(DEV), 1.0)
        o_off, o_ind = ref.radius_search(q, 1.0, threads=8)
        assert int(np.diff(o_off).max()) > 2048
        assert np.array_equal(off.cpu().numpy(), o_off) and np.array_equal(ind.cpu().numpy(), o_ind)
    finally:
        ix.close()


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
@pytest.mark.parametrize("dim", [2, 3])
def test_small_knn_batches(prec, dim):
    xyz = cloudgen.adversarial_cloud(20_000, seed=33)
    ref = oracle.Index(xyz, 1.0, 0.5, dim=dim)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0, 0.5, dim=dim, precision=prec)
    try:
        for m in (1, 10, 100, 1000):
            q = _queries(xyz, m, seed=50 + m)
            for k in (1, 16, 64):
                idx, d2 = ix.knn(torch.from_numpy(q).to(DEV), k)
                r_idx, r_d2 = ref.knn(q, k, threads=8)
                assert np.array_equal(idx.cpu().numpy(), r_idx), (m, k)
                assert np.array_equal(d2.cpu().numpy(), r_d2), (m, k)
    finally:
        ix.close()


def test_search_into_capacity_and_overflow():
    # cg_radius_search_into: rows that fit are written by the one call; a
    # buffer that is too small gives CG_ERR_OVERFLOW with the total, and the
    # count stands for a fill into a buffer of that size
    xyz = cloudgen.als_uniform(50_000, extent=(60.0, 60.0), seed=8)
    ref = oracle.Index(xyz, 1.0)
    ix = cg.Index(torch.from_numpy(xyz).to(DEV), 1.0)
    try:
        for m in (1, 300, 3000):  # the last one beyond the small path
            q = _queries(xyz, m, seed=70 + m)
            qd = torch.from_numpy(q).to(DEV)
            o_off, o_ind = ref.radius_search(q, 1.0, threads=8)
            off = torch.empty(m + 1, dtype=torch.int64, device=DEV)
            big = torch.full((int(o_off[-1]) + 10,), -1, dtype=torch.int32, device=DEV)
            fits, total = cg.cg_radius_search_into(ix.h, qd, 1.0, cg.SPHERE, off, big, big.numel())
            assert fits and total == int(o_off[-1])
            assert np.array_equal(off.cpu().numpy(), o_off)
            assert np.array_equal(big[:total].cpu().numpy(), o_ind)
            small = torch.empty(max(total // 2, 1), dtype=torch.int32, device=DEV)
            fits, total2 = cg.cg_radius_search_into(ix.h, qd, 1.0, cg.SPHERE, off, small, small.numel())
            assert not fits and total2 == total
            out = torch.empty(total, dtype=torch.int32, device=DEV)
            cg.cg_radius_fill(ix.h, qd, 1.0, cg.SPHERE, off, out)
            cg.cg_index_status(ix.h)
            assert np.array_equal(out.cpu().numpy(), o_ind)
    finally:
        ix.close()
