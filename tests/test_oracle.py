"""Pins for the CPU oracle: values printed in the paper, closed forms,
brute force on tiny clouds and exact invariants.  None of these re-types the
oracle's own formulas; each is chosen so that a plausible slip in the oracle
(a dropped axis, a wrong sign, an off-by-one voxel, a wrong flavour rule, a
broken tie order) fails at least one of them."""
import itertools
import json
import math
import os

import numpy as np
import pytest

import cloudgen
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _golden(name):
    with open(os.path.join(GOLDEN, name)) as f:
        return json.load(f)


def _round_sig(x, digits):
    """Round to the precision the paper prints (e.g. 251.00e3: 2 decimals of
    the mantissa in engineering form)."""
    e = int(math.floor(math.log10(abs(x)) / 3) * 3)
    return round(x / 10 ** e, digits) * 10 ** e


# ---------------------------------------------------------------- grid size


def test_grid_size_dalesC_printed_counts():
    g = _golden("grid_size_pins.json")["dalesC"]
    ex, ey, ez = g["extent_m"]
    s = g["cell_m"]
    nx = oracle.grid_size(0.0, ex, s)
    ny = oracle.grid_size(0.0, ey, s)
    nz = oracle.grid_size(0.0, ez, s)
    assert (nx, ny, nz) == (501, 501, 169)
    assert _round_sig(nx * ny, g["voxels_2d_digits"]) == pytest.approx(g["voxels_2d_printed"])
    assert _round_sig(nx * ny * nz, g["voxels_3d_digits"]) == pytest.approx(g["voxels_3d_printed"])
    # 428 empty voxels are 0.17 % of the 2D grid
    assert round(100.0 * g["empty_2d"] / (nx * ny), 2) == pytest.approx(g["empty_2d_pct_printed"])


def test_grid_size_lille_consistent_layers():
    g = _golden("grid_size_pins.json")["lille"]
    # a 3D grid has exactly n_z layers of the 2D grid: the printed ratio is an integer
    nz = g["voxels_3d_printed"] / g["voxels_2d_printed"]
    assert abs(nz - round(nz)) < 0.01 and round(nz) == 43


def test_grid_size_through_index_bbox():
    # a cloud whose bbox is exactly the dalesC box: the index must size its grid to it
    xyz = np.array([[0.0, 0.0, 0.0], [500.0, 500.0, 168.4], [250.0, 3.0, 7.0]])
    ix2 = oracle.Index(xyz, 1.0, 1.0, dim=2)
    ix3 = oracle.Index(xyz, 1.0, 1.0, dim=3)
    assert ix2.info()["ncell"] == 251001
    assert ix3.info()["ncell"] == 42419169
    assert ix3.info()["nc"] == (501, 501, 169)


def test_voxel_coord_zero_based_and_top_corner():
    # Eq. chs-point-to-idcs is 0-based: p- maps to 0; p+ maps to n_a - 1
    assert oracle.voxel_coord(0.0, 0.0, 1.0) == 0
    assert oracle.voxel_coord(0.999, 0.0, 1.0) == 0
    assert oracle.voxel_coord(1.0, 0.0, 1.0) == 1
    assert oracle.voxel_coord(500.0, 0.0, 1.0) == oracle.grid_size(0.0, 500.0, 1.0) - 1
    assert oracle.voxel_coord(168.4, 0.0, 1.0) == oracle.grid_size(0.0, 168.4, 1.0) - 1
    assert oracle.voxel_coord(508003.0, 508000.0, 0.5) == 6


# ---------------------------------------------------------- worked examples


def test_kernel_search_worked_example_range_and_circle():
    ex = _golden("kernel_search_example.json")
    (cx, cy), r = ex["center"], ex["radius"]
    # bounding box of the kernel and its voxel range (Algorithm 1, first steps)
    (x0, y0), (x1, y1) = ex["kernel_bbox"]
    assert (cx - r, cy - r) == pytest.approx((x0, y0))
    assert (cx + r, cy + r) == pytest.approx((x1, y1))
    i0, i1 = oracle.voxel_coord(cx - r, 0.0, 1.0), oracle.voxel_coord(cx + r, 0.0, 1.0)
    j0, j1 = oracle.voxel_coord(cy - r, 0.0, 1.0), oracle.voxel_coord(cy + r, 0.0, 1.0)
    assert [i0, i1] == ex["bbox_voxels"]["i"] and [j0, j1] == ex["bbox_voxels"]["j"]
    # one point at the spot of each bbox voxel nearest to c: it is inside the
    # circle exactly when the voxel meets the circle
    pts, cells = [], []
    for i in range(i0, i1 + 1):
        for j in range(j0, j1 + 1):
            px = min(max(cx, i), i + 1)
            py = min(max(cy, j), j + 1)
            pts.append([px, py, 0.0])
            cells.append((i, j))
    pts.append([0.0, 0.0, 0.0])
    pts.append([8.0, 5.0, 0.0])  # grid corners: an 8 x 5 (+1 for the closed top) grid
    pts = np.array(pts)
    ix = oracle.Index(pts, 1.0, 1.0, dim=2)
    hit = ix.kernel_search(np.array([cx, cy, 0.0]), r)
    hit_cells = {cells[h] for h in hit if h < len(cells)}
    assert len(hit_cells) == ex["voxels_meeting_circle_count"]
    missing = sorted(set(cells) - hit_cells)
    assert [list(m) for m in missing] == ex["voxels_missing_circle"]


@pytest.mark.parametrize("flavor", [oracle.SPARSE, oracle.MIXED, oracle.DENSE])
def test_sparse_worked_example(flavor):
    ex = _golden("sparse_example.json")
    (ecx, ecy), (a, b) = ex["ellipse"]["center"], ex["ellipse"]["semi_axes"]
    g = np.arange(0, 800) * 0.01
    h = np.arange(0, 500) * 0.01
    X, Y = np.meshgrid(g, h, indexing="ij")
    X = X.ravel(); Y = Y.ravel()
    keep = ((X - ecx) / a) ** 2 + ((Y - ecy) / b) ** 2 > 1.0
    xyz = np.stack([X[keep], Y[keep], np.zeros(keep.sum())], 1)
    ix = oracle.Index(xyz, 1.0, 1.0, dim=2, flavor=flavor)
    assert ix.info()["nc"][:2] == tuple(ex["grid"])
    empty = sorted([i, j] for i in range(8) for j in range(5) if ix.voxel_count(i, j) == 0)
    assert empty == sorted(ex["empty_voxels"])
    if flavor == oracle.SPARSE:
        stored = sorted([i, j] for i in range(8) for j in range(5) if not ix.voxel_stored(i, j))
        assert stored == sorted(ex["empty_voxels"])
        assert ix.info()["nonempty"] == 40 - 4
    if flavor == oracle.MIXED:
        # 36 of 40 voxels (90 %) are non-empty: the single 2D slice turns dense
        assert ix.slice_dense(0)


# ------------------------------------------------------ closed-form lattice


def _lattice_ball_count(rad2):
    """Integer triples with x^2 + y^2 + z^2 <= rad2 (pure integer arithmetic)."""
    m = int(math.isqrt(rad2))
    return sum(1 for x in range(-m, m + 1) for y in range(-m, m + 1) for z in range(-m, m + 1)
               if x * x + y * y + z * z <= rad2)


@pytest.mark.parametrize("dim,flavor", [(2, 0), (3, 0), (2, 1), (3, 1), (3, 2)])
def test_lattice_sphere_and_cube_counts(dim, flavor):
    # lattice at UTM-like integer offsets: every difference is exact, so the
    # counts are integer facts independent of rounding
    off = (508000.0, 5440000.0, 100.0)
    xyz = cloudgen.lattice_cloud(6, offset=off)
    ix = oracle.Index(xyz, 1.0, 1.0, dim=dim, flavor=flavor)
    c = np.array(off)
    for r in (1, 2, 3, 5):
        got = ix.kernel_search(c, float(r), oracle.SPHERE)
        assert len(got) == _lattice_ball_count(r * r)
        # radius exactly on lattice distances (3,4,0): the boundary is included
        cube = ix.kernel_search(c, float(r), oracle.CUBE)
        assert len(cube) == (2 * r + 1) ** 3
    # just below 5: the 3-4-0 shell (and 5-0-0) drops out
    assert len(ix.kernel_search(c, 5.0 - 1e-9)) == _lattice_ball_count(24)
    # a query off every lattice coordinate axis: shift in z only
    c2 = c + np.array([0.0, 0.0, 0.5])
    # points with x^2 + y^2 + (z - 0.5)^2 <= 4  <=> 4x^2+4y^2+(2z-1)^2 <= 16
    expect = sum(1 for x in range(-6, 7) for y in range(-6, 7) for z in range(-6, 7)
                 if 4 * x * x + 4 * y * y + (2 * z - 1) ** 2 <= 16)
    assert len(ix.kernel_search(c2, 2.0)) == expect


@pytest.mark.parametrize("dim,flavor", [(2, 0), (3, 0), (3, 1), (3, 2)])
def test_lattice_cylinder_counts(dim, flavor):
    # vertical cylinder (Section 2's xy-only kernel): every z level of the
    # lattice inside the disk x^2 + y^2 <= r^2, whatever the query's height
    off = (508000.0, 5440000.0, 100.0)
    xyz = cloudgen.lattice_cloud(6, offset=off)
    ix = oracle.Index(xyz, 1.0, 1.0, dim=dim, flavor=flavor)
    for dz in (0.0, 4.0, 40.0):  # queries above the cloud still see every level
        c = np.array(off) + np.array([0.0, 0.0, dz])
        for r in (1, 2, 5):
            disk = sum(1 for x in range(-6, 7) for y in range(-6, 7) if x * x + y * y <= r * r)
            assert len(ix.kernel_search(c, float(r), oracle.CYLINDER)) == disk * 13


def test_cylinder_contains_sphere_and_equals_it_on_a_plane():
    xyz = cloudgen.adversarial_cloud(3000, seed=41)
    ix = oracle.Index(xyz, 1.0, 1.0, dim=3)
    rng = np.random.default_rng(2)
    for c in xyz[rng.integers(0, len(xyz), 30)]:
        sph = set(ix.kernel_search(c, 1.3, oracle.SPHERE).tolist())
        cyl = set(ix.kernel_search(c, 1.3, oracle.CYLINDER).tolist())
        assert sph <= cyl
    flat = xyz.copy()
    flat[:, 2] = 7.25
    ixf = oracle.Index(flat, 1.0, 1.0, dim=3)
    for c in flat[rng.integers(0, len(flat), 30)]:
        assert np.array_equal(ixf.kernel_search(c, 0.8, oracle.CYLINDER), ixf.kernel_search(c, 0.8, oracle.SPHERE))


def test_lattice_knn_shells():
    off = (508000.0, 5440000.0, 100.0)
    xyz = cloudgen.lattice_cloud(4, offset=off)
    ix = oracle.Index(xyz, 1.0, 1.0, dim=3)
    idx, d2 = ix.knn(np.array([off]), 27)
    # the 3x3x3 block around the centre: 1 at d2 = 0, 6 at 1, 12 at 2, 8 at 3
    assert list(d2[0]) == [0.0] * 1 + [1.0] * 6 + [2.0] * 12 + [3.0] * 8
    # ties are ordered by original index
    for v in (1.0, 2.0, 3.0):
        sel = idx[0][d2[0] == v]
        assert list(sel) == sorted(sel)
    # every returned point really sits at its reported integer distance
    for t in range(27):
        p = xyz[idx[0, t]] - np.array(off)
        assert int(round(p @ p)) == d2[0, t]


def test_knn_fewer_points_than_k():
    xyz = np.array([[0.0, 0.0, 0.0], [3.0, 0.0, 0.0], [0.0, 4.0, 0.0]])
    ix = oracle.Index(xyz, 1.0)
    idx, d2 = ix.knn(np.array([[0.0, 0.0, 0.0]]), 5)
    assert list(idx[0]) == [0, 1, 2, -1, -1]
    assert list(d2[0][:3]) == [0.0, 9.0, 16.0] and np.all(np.isinf(d2[0][3:]))


# ------------------------------------------------------------ brute force

CASES = [(d, f) for d in (2, 3) for f in (oracle.DENSE, oracle.SPARSE, oracle.MIXED)]


@pytest.mark.parametrize("dim,flavor", CASES)
def test_index_matches_brute_force(dim, flavor):
    xyz = cloudgen.adversarial_cloud(2000, seed=11 + dim * 3 + flavor)
    ix = oracle.Index(xyz, 1.0, 0.5, dim=dim, flavor=flavor)
    rng = np.random.default_rng(5)
    qs = np.concatenate([xyz[rng.integers(0, len(xyz), 40)],
                         xyz[:5] + rng.normal(0, 3.0, (5, 3)),       # some outside the bbox
                         np.array([xyz.min(0) - 50.0])])            # far outside
    for c in qs:
        for r in (0.3, 1.0, 2.5):
            for kern in (oracle.SPHERE, oracle.CUBE, oracle.CYLINDER):
                assert np.array_equal(ix.kernel_search(c, r, kern), oracle.brute_radius(xyz, c, r, kern))
        for k in (1, 7, 33):
            a_i, a_d = ix.knn(c[None, :], k)
            b_i, b_d = oracle.brute_knn(xyz, c, k)
            assert np.array_equal(a_i[0], b_i) and np.array_equal(a_d[0], b_d)


def test_points_exactly_on_sphere():
    # a centre and points at exactly representable distance r along axes and
    # on 3-4-5 triangles scaled by 2^-3, placed at a UTM-like offset
    c = np.array([508123.0, 5440321.0, 12.0])
    r = 0.625  # = 5 * 2^-3
    pts = [c + [0.625, 0, 0], c + [0, -0.625, 0], c + [0.375, 0.5, 0], c + [0, 0.375, -0.5],
           c + [0.375, 0.5, 1e-9], c + [0.375, 0.5, 1e-7], c + [0.626, 0, 0]]
    xyz = np.array(pts)
    ix = oracle.Index(xyz, 0.25, 0.25, dim=3)
    got = ix.kernel_search(c, r)
    # point 4: dz^2 ~ 1e-18 is below half an ulp of r^2 = 0.390625 (ulp 2^-54),
    # so the binary64 sum rounds back onto the sphere and the point is inside;
    # point 5: dz^2 ~ 1e-14 survives the rounding and the point is outside
    assert list(got) == [0, 1, 2, 3, 4]


# -------------------------------------------------------------- invariants


@pytest.fixture(scope="module")
def small_tile():
    xyz = cloudgen.als_uniform(6000, extent=(25.0, 25.0), seed=99)
    return xyz, oracle.Index(xyz, 1.0)


def test_symmetry(small_tile):
    xyz, ix = small_tile
    off, ind = ix.radius_search(xyz, 1.2)
    rows = np.repeat(np.arange(len(xyz)), np.diff(off))
    a = set(zip(rows.tolist(), ind.tolist()))
    assert all((j, i) in a for (i, j) in a)
    # every point is its own neighbour
    assert all((i, i) in a for i in range(len(xyz)))


def test_cube_contains_sphere(small_tile):
    xyz, ix = small_tile
    s_off, s_ind = ix.radius_search(xyz[:500], 1.0, oracle.SPHERE)
    c_off, c_ind = ix.radius_search(xyz[:500], 1.0, oracle.CUBE)
    for q in range(500):
        s = set(s_ind[s_off[q]:s_off[q + 1]].tolist())
        c = set(c_ind[c_off[q]:c_off[q + 1]].tolist())
        assert s <= c


def test_rows_sorted_and_unique(small_tile):
    xyz, ix = small_tile
    off, ind = ix.radius_search(xyz[:800], 2.0)
    for q in range(800):
        row = ind[off[q]:off[q + 1]]
        assert np.all(np.diff(row) > 0)


def test_results_independent_of_cell_and_flavour(small_tile):
    xyz, ix = small_tile
    q = xyz[:300]
    ref = ix.radius_search(q, 1.5)
    for cell, dim, fl in [(0.5, 2, oracle.SPARSE), (2.0, 3, oracle.MIXED), (0.3, 3, oracle.DENSE)]:
        other = oracle.Index(xyz, cell, cell, dim=dim, flavor=fl).radius_search(q, 1.5)
        assert np.array_equal(ref[0], other[0]) and np.array_equal(ref[1], other[1])


def test_knn_prefix_and_self_first(small_tile):
    xyz, ix = small_tile
    q = xyz[:200]
    i8, d8 = ix.knn(q, 8)
    i20, d20 = ix.knn(q, 20)
    assert np.array_equal(i8, i20[:, :8]) and np.array_equal(d8, d20[:, :8])
    assert np.all(np.diff(d20, axis=1) >= 0)
    # generated points are distinct here, so each query's nearest is itself
    assert np.array_equal(i8[:, 0], np.arange(200)) and np.all(d8[:, 0] == 0)


def test_knn_matches_radius_count(small_tile):
    # the k nearest all lie within the k-th distance, and the radius query at
    # that distance returns at least k points
    xyz, ix = small_tile
    idx, dd = ix.knn(xyz[:100], 12)
    for q in range(100):
        rr = math.sqrt(dd[q, -1])
        row = ix.kernel_search(xyz[q], rr * (1 + 1e-12))
        assert set(idx[q].tolist()) <= set(row.tolist())


def test_mixed_slice_rule_80_percent():
    # 3D lattice 4 x 4 x 3 voxels; layer 0 fully occupied (16/16), layer 1 at
    # 13/16 (81 %), layer 2 at 12/16 (75 %) -> dense, dense, sparse
    pts = []
    for i, j in itertools.product(range(4), range(4)):
        pts.append([i + 0.5, j + 0.5, 0.5])
    for t, (i, j) in enumerate(itertools.product(range(4), range(4))):
        if t < 13:
            pts.append([i + 0.5, j + 0.5, 1.5])
        if t < 12:
            pts.append([i + 0.5, j + 0.5, 2.5])
    pts.append([0.0, 0.0, 0.0])
    pts.append([2.9, 3.9, 2.9])  # voxel (2, 3, 2): already occupied
    ix = oracle.Index(np.array(pts), 1.0, 1.0, dim=3, flavor=oracle.MIXED)
    assert ix.info()["nslices"] == 3
    assert [ix.slice_dense(s) for s in range(3)] == [True, True, False]
    # results are the same as dense and sparse
    q = np.array(pts[:20])
    ref = oracle.Index(np.array(pts), 1.0, 1.0, dim=3).radius_search(q, 1.1)
    got = ix.radius_search(q, 1.1)
    assert np.array_equal(ref[1], got[1])


def test_multithreaded_driver_equals_single(small_tile):
    xyz, ix = small_tile
    a = ix.radius_search(xyz, 1.0, threads=1)
    b = ix.radius_search(xyz, 1.0, threads=4)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])
    ka = ix.knn(xyz[:500], 9, threads=1)
    kb = ix.knn(xyz[:500], 9, threads=3)
    assert np.array_equal(ka[0], kb[0]) and np.array_equal(ka[1], kb[1])


def test_mixed_slice_rule_exactly_80_percent():
    # 5 x 4 voxels per layer: 16 of 20 non-empty is exactly 80 % -> dense;
    # 15 of 20 -> sparse (the rule is "at least 80 %", Section 3.3.3)
    pts = []
    holes = {(1, 1), (1, 2), (2, 1), (2, 2)}
    for i, j in itertools.product(range(5), range(4)):
        if (i, j) not in holes:
            pts.append([i + 0.5, j + 0.5, 0.5])
        if (i, j) not in holes | {(3, 1)}:
            pts.append([i + 0.5, j + 0.5, 1.5])
    pts.append([0.0, 0.0, 0.0])
    ix = oracle.Index(np.array(pts), 1.0, 1.0, dim=3, flavor=oracle.MIXED)
    assert ix.info()["nc"] == (5, 4, 2)
    assert [ix.slice_dense(s) for s in range(2)] == [True, False]
