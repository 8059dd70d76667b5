"""Pins for Algorithm 2's two radius-growth policies in the oracle
(Section 3.4.2: the monotone step r + s, and the density step of the second
phase, read as r = (3 k / (4 pi rho))^(1/3)).

The policy may change only the sequence of radii and the voxels visited,
never the result: both must equal brute force.  The visited-voxel count is
pinned by a closed form, and the direction of Section 3.5's observation
(the density step explores fewer voxels in most cases) is checked on a
uniform random cloud like the paper's."""
import numpy as np
import pytest

import cloudgen
import oracle

POLICIES = (oracle.GROW_MONOTONE, oracle.GROW_DENSITY)


def _brute(xyz, q, k):
    out_i = np.empty((len(q), k), np.int32)
    out_d = np.empty((len(q), k), np.float64)
    for t, c in enumerate(q):
        out_i[t], out_d[t] = oracle.brute_knn(xyz, c, k)
    return out_i, out_d


@pytest.mark.parametrize("policy", POLICIES)
@pytest.mark.parametrize("dim,flavor", [(2, oracle.DENSE), (3, oracle.DENSE), (3, oracle.SPARSE),
                                        (3, oracle.MIXED)])
def test_policies_equal_brute_force(policy, dim, flavor):
    rng = np.random.default_rng(31 + dim)
    xyz = cloudgen.adversarial_cloud(3000, seed=5)
    q = np.concatenate([xyz[rng.integers(0, len(xyz), 150)] + rng.normal(0, 0.3, (150, 3)),
                        xyz.min(0) + rng.uniform(-5, 15, (30, 3))])
    ix = oracle.Index(xyz, 0.7, 0.5, dim=dim, flavor=flavor)
    for k in (1, 7, 32, 64):
        idx, d2, vis = ix.knn_policy(q, k, policy)
        b_idx, b_d2 = _brute(xyz, q, k)
        assert np.array_equal(idx, b_idx), k
        assert np.array_equal(d2, b_d2), k
        assert (vis >= 1).all()


@pytest.mark.parametrize("policy", POLICIES)
def test_policies_with_fewer_points_than_k(policy):
    xyz = cloudgen.random_cloud(20, extent=(4.0, 4.0, 2.0), seed=2)
    ix = oracle.Index(xyz, 0.5, 0.5, dim=3)
    q = np.array([[1.0, 1.0, 1.0], [30.0, -4.0, 0.0]])
    idx, d2, vis = ix.knn_policy(q, 25, policy)
    b_idx, b_d2 = _brute(xyz, q, 25)
    assert np.array_equal(idx, b_idx) and np.array_equal(d2, b_d2)
    assert (idx[:, 20:] == -1).all()
    nc = ix.info()["nc"]
    assert (vis == nc[0] * nc[1] * nc[2]).all()  # every voxel visited


def test_visited_box_closed_form():
    # unit lattice (points at integer coordinates, -6 .. 6), unit voxels, k = 1
    xyz = cloudgen.lattice_cloud(6)
    ix = oracle.Index(xyz, 1.0, 1.0, dim=3)
    ix2 = oracle.Index(xyz, 1.0, 1.0, dim=2)
    # a query on a lattice point: the first radius is 0 (it lies on a voxel
    # wall), the box is its voxel widened by one voxel on each side (3 per
    # axis) and the point itself ends the search
    on = np.array([[0.0, 0.0, 0.0], [-3.0, 2.0, 4.0]])
    # a query at a voxel centre, between lattice points: r = 1/2 finds no
    # point (the nearest are sqrt(3)/2 away) and 4 voxels per axis; P^ is
    # empty, so both policies step to r = 3/2: 6 voxels per axis, and the
    # eight nearest points end the search
    mid = np.array([[0.5, 0.5, 0.5], [-2.5, 1.5, 3.5]])
    for policy in POLICIES:
        assert ix.knn_policy(on, 1, policy)[2].tolist() == [27, 27]
        assert ix.knn_policy(mid, 1, policy)[2].tolist() == [216, 216]
        # 2D grid: the z range of a column is unbounded, the box is 3 x 3 or
        # 6 x 6 columns
        assert ix2.knn_policy(on, 1, policy)[2].tolist() == [9, 9]
        assert ix2.knn_policy(mid, 1, policy)[2].tolist() == [36, 36]


def test_density_step_explores_fewer_voxels_on_random_points():
    # Section 3.5 (uniform random points): the density step explores fewer
    # voxels than the monotone one in most cases; same results always
    rng = np.random.default_rng(0)
    xyz = rng.uniform([0, 0, 0], [60, 60, 30], (100_000, 3))
    ix = oracle.Index(xyz, 1.0, 1.0, dim=3)
    q = xyz[rng.integers(0, len(xyz), 4000)]
    for k in (16, 50):
        a = ix.knn_policy(q, k, oracle.GROW_MONOTONE, threads=4)
        b = ix.knn_policy(q, k, oracle.GROW_DENSITY, threads=4)
        assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
        fewer = (b[2] < a[2]).mean()
        worse = (b[2] > a[2]).mean()
        assert fewer > 0.5 and worse < fewer, (k, fewer, worse)
        assert b[2].mean() < a[2].mean()
