"""GPU parity on the predicates' rounding boundary: the triples of
``exact_rounding.standard_cases`` (points on which the specified binary64
evaluation order and a contracted, re-associated, unrounded, root-compared or
strictly compared one disagree) searched through the C ABI in both storage
precisions and both grid dimensions.  Each query's row must be its own point
exactly when the exact-rational specification says so, and must equal the
oracle's row; k-NN must report the specified binary64 value."""
import os
import sys
from fractions import Fraction

import numpy as np
import pytest
import torch

import oracle
import paper_2502_11602_gb300 as cg

sys.path.insert(0, os.path.dirname(__file__))
import exact_rounding as ex  # noqa: E402

pytestmark = pytest.mark.gpu

DEV = "cuda:0"
KERNEL = {ex.SPHERE: cg.SPHERE, ex.CUBE: cg.CUBE, ex.CYLINDER: cg.CYLINDER}


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
@pytest.mark.parametrize("origin", list(ex.ORIGINS))
def test_boundary_triples_radius(origin, prec, dim):
    cases = [cs for cs in ex.standard_cases() if cs[2] == origin]
    pts = np.array([cs[4] for cs in cases])
    ix = cg.Index(torch.from_numpy(pts).to(DEV), 1.0, 1.0, dim=dim, precision=prec)
    ref = oracle.Index(pts, 1.0, 1.0, dim=dim)
    bad = []
    try:
        for i, (kind, alt, _, c, _, r, inside) in enumerate(cases):
            q = torch.from_numpy(c.reshape(1, 3).copy()).to(DEV)
            off, ind = ix.radius_search(q, r, KERNEL[kind])
            row = ind.cpu().numpy().tolist()
            assert int(off[-1]) == len(row)
            want = [i] if inside else []
            if row != want or ref.kernel_search(c, r, kind).tolist() != want:
                bad.append((ex.KINDS[kind], alt, i, row, want))
    finally:
        ix.close()
    assert bad == []


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
@pytest.mark.parametrize("origin", list(ex.ORIGINS))
def test_boundary_triples_batched_queries(origin, prec):
    # the same cases as one multi-query call per radius value: the query
    # plan and voxel groups see them together (radii differ, so one call
    # per case radius, every query of the origin in each call)
    cases = [cs for cs in ex.standard_cases() if cs[2] == origin and cs[0] == ex.SPHERE]
    pts = np.array([cs[4] for cs in cases])
    qs = np.array([cs[3] for cs in cases])
    ix = cg.Index(torch.from_numpy(pts).to(DEV), 1.0, 1.0, dim=2, precision=prec)
    ref = oracle.Index(pts, 1.0, 1.0, dim=2)
    qd = torch.from_numpy(qs).to(DEV)
    try:
        for i, (_, _, _, c, _, r, inside) in enumerate(cases[:16]):
            off, ind = ix.radius_search(qd, r, cg.SPHERE)
            o_off, o_ind = ref.radius_search(qs, r, oracle.SPHERE)
            assert np.array_equal(off.cpu().numpy(), o_off)
            assert np.array_equal(ind.cpu().numpy(), o_ind)
            row_i = ind.cpu().numpy()[off[i]:off[i + 1]].tolist()
            assert row_i == ([i] if inside else [])
    finally:
        ix.close()


@pytest.mark.parametrize("prec", [cg.FP32_OFFSET, cg.FP64])
@pytest.mark.parametrize("origin", list(ex.ORIGINS))
def test_boundary_triples_knn_distance(origin, prec):
    cases = [cs for cs in ex.standard_cases() if cs[2] == origin and cs[0] == ex.SPHERE]
    pts = np.array([cs[4] for cs in cases])
    qs = np.array([cs[3] for cs in cases])
    ix = cg.Index(torch.from_numpy(pts).to(DEV), 1.0, 1.0, dim=2, precision=prec)
    try:
        idx, d2 = ix.knn(torch.from_numpy(qs).to(DEV), 1)
        idx = idx.cpu().numpy()
        d2 = d2.cpu().numpy()
    finally:
        ix.close()
    for i, cs in enumerate(cases):
        assert idx[i, 0] == i
        assert Fraction(float(d2[i, 0])) == ex.sphere_d2(cs[4] - cs[3])
