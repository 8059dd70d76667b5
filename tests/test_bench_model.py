"""The work counts behind the bench line's rooflines, checked on the CPU.

* `bench._alg_tests` (the Algorithm 1 candidate tests that the count
  kernels' ALU roofline divides by) against a brute-force enumeration: for
  every query, every point whose voxel lies in the query's voxel range.
* The same count against the oracle's own enumeration: the candidates the
  oracle visits are a superset of the neighbours it returns, and the sphere
  neighbours of every query are among the counted candidates.
"""
import math

import numpy as np

import bench
import cloudgen
import oracle


def _brute_tests(xyz, r, cell):
    lo = xyz[:, :2].min(0)
    hi = xyz[:, :2].max(0)
    n = (np.floor((hi - lo) / cell).astype(np.int64) + 1)
    vox = np.floor((xyz[:, :2] - lo) / cell).astype(np.int64)
    total = 0
    for c in xyz[:, :2]:
        a0 = np.clip(np.floor((c - r - lo) / cell).astype(np.int64), 0, n - 1)
        a1 = np.clip(np.floor((c + r - lo) / cell).astype(np.int64), 0, n - 1)
        inside = (vox[:, 0] >= a0[0]) & (vox[:, 0] <= a1[0]) & (vox[:, 1] >= a0[1]) & (vox[:, 1] <= a1[1])
        total += int(inside.sum())
    return total


def test_alg_tests_matches_brute_force():
    for seed, (npts, side, r, cell) in enumerate([(1500, 20.0, 1.0, 1.0), (1200, 12.0, 0.7, 0.5),
                                                  (900, 30.0, 2.5, 1.0)]):
        xyz = cloudgen.als_uniform(npts, extent=(side, side), seed=cloudgen.CONFIG_SEED + 300 + seed)
        assert bench._alg_tests(xyz, r, cell) == _brute_tests(xyz, r, cell)


def test_alg_tests_bound_the_neighbours():
    xyz = cloudgen.als_uniform(3000, extent=(25.0, 25.0), seed=cloudgen.CONFIG_SEED + 310)
    r = 1.0
    tests = bench._alg_tests(xyz, r, 1.0)
    off, _ = oracle.Index(xyz, 1.0).radius_search(xyz, r)
    neighbours = int(off[-1])
    assert neighbours <= tests
    # a 3x3 block of unit voxels around each query against the disc's area
    assert tests <= 9.0 / math.pi * neighbours * 1.5
