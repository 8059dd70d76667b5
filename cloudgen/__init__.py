"""Seeded synthetic LiDAR-like point clouds.

These generators stand in for the public datasets of the paper's evaluation
(DALES ALS tiles, Paris-Lille-3D MLS, Semantic3D TLS; Section 4), which are
not available here.  They reproduce shape, extent, density and structure, not
the datasets' contents.  This module holds none of the search method's
arithmetic: it only makes inputs, which both the CUDA path and the oracle
consume.

Every generator is deterministic in its ``seed`` (numpy PCG64 plus a
SplitMix64 lattice hash for the terrain), returns float64 AoS ``(n, 3)``
arrays, and shuffles the points with the same seed so that the original point
order carries no spatial information.
"""
from __future__ import annotations

import math

import numpy as np

UTM_OFFSET = (508000.0, 5440000.0, 0.0)
CONFIG_SEED = 0x5EED0000

_M64 = np.uint64(0xFFFFFFFFFFFFFFFF)


def splitmix64(x: np.ndarray) -> np.ndarray:
    """SplitMix64 finaliser (Steele, Lea, Flood 2014) on uint64 arrays."""
    with np.errstate(over="ignore"):
        z = (x + np.uint64(0x9E3779B97F4A7C15)) & _M64
        z = ((z ^ (z >> np.uint64(30))) * np.uint64(0xBF58476D1CE4E5B9)) & _M64
        z = ((z ^ (z >> np.uint64(27))) * np.uint64(0x94D049BB133111EB)) & _M64
        return z ^ (z >> np.uint64(31))


def _lattice_value(seed: int, octave: int, i: np.ndarray, j: np.ndarray) -> np.ndarray:
    """Uniform value in [-1, 1] hashed from (seed, octave, i, j)."""
    with np.errstate(over="ignore"):
        h = splitmix64(np.uint64(seed) ^ (np.uint64(octave) * np.uint64(0xD1B54A32D192ED03)))
        h = splitmix64(h ^ (i.astype(np.int64).astype(np.uint64) * np.uint64(0x9E3779B97F4A7C15)))
        h = splitmix64(h ^ (j.astype(np.int64).astype(np.uint64) * np.uint64(0xC2B2AE3D27D4EB4F)))
    return (h >> np.uint64(11)).astype(np.float64) * (2.0 / 9007199254740992.0) - 1.0


def _quintic(t: np.ndarray) -> np.ndarray:
    return t * t * t * (t * (t * 6.0 - 15.0) + 10.0)


def terrain(x: np.ndarray, y: np.ndarray, seed: int, amplitude: float = 5.0) -> np.ndarray:
    """Five-octave value noise (lattice 64, 32, 16, 8, 4 m; weights 0.5^o),
    quintic-smoothstep interpolation, scaled to +-amplitude metres."""
    z = np.zeros_like(x)
    total = 0.0
    for o, spacing in enumerate((64.0, 32.0, 16.0, 8.0, 4.0)):
        w = 0.5 ** o
        total += w
        u = x / spacing
        v = y / spacing
        i0 = np.floor(u)
        j0 = np.floor(v)
        fu = _quintic(u - i0)
        fv = _quintic(v - j0)
        a = _lattice_value(seed, o, i0, j0)
        b = _lattice_value(seed, o, i0 + 1, j0)
        c = _lattice_value(seed, o, i0, j0 + 1)
        d = _lattice_value(seed, o, i0 + 1, j0 + 1)
        z += w * ((a * (1 - fu) + b * fu) * (1 - fv) + (c * (1 - fu) + d * fu) * fv)
    return z * (amplitude / total)


def _finish(xyz: np.ndarray, rng: np.random.Generator, offset) -> np.ndarray:
    xyz = xyz[rng.permutation(xyz.shape[0])]
    xyz += np.asarray(offset, np.float64)[None, :]
    return np.ascontiguousarray(xyz)


def als_uniform(n: int = 100_000, extent=(100.0, 100.0), seed: int = CONFIG_SEED + 0,
                offset=UTM_OFFSET, noise: float = 0.05) -> np.ndarray:
    """Small ALS-like tile: uniform xy over ``extent``, z = terrain + N(0, noise)."""
    rng = np.random.default_rng(seed)
    x = rng.uniform(0.0, extent[0], n)
    y = rng.uniform(0.0, extent[1], n)
    z = terrain(x, y, seed) + rng.normal(0.0, noise, n)
    return _finish(np.stack([x, y, z], axis=1), rng, offset)


def als_urban(n: int = 12_000_000, extent=(500.0, 500.0), seed: int = CONFIG_SEED + 1,
              offset=UTM_OFFSET, n_buildings: int = 200, n_trees: int = 3000,
              noise: float = 0.05, wall_factor: float = 0.2) -> np.ndarray:
    """ALS-scale urban tile: terrain, axis-aligned box buildings (roof and wall
    points) and trees (Gaussian crowns).  The point budget is split in
    proportion to each surface's sampled area (walls weighted by
    ``wall_factor``, as a near-nadir scanner sees them obliquely); the total is
    exactly ``n``."""
    rng = np.random.default_rng(seed)
    ex, ey = extent
    bw = rng.uniform(10.0, 40.0, n_buildings)
    bd = rng.uniform(10.0, 40.0, n_buildings)
    bh = rng.uniform(5.0, 30.0, n_buildings)
    bx = rng.uniform(0.0, ex - bw)
    by = rng.uniform(0.0, ey - bd)
    th = rng.uniform(5.0, 20.0, n_trees)
    tx = rng.uniform(0.0, ex, n_trees)
    ty = rng.uniform(0.0, ey, n_trees)
    crown_r = 0.25 * th

    roof_area = bw * bd
    wall_area = 2.0 * (bw + bd) * bh * wall_factor
    tree_area = math.pi * crown_r ** 2
    ground_area = ex * ey
    areas = np.array([ground_area, roof_area.sum(), wall_area.sum(), tree_area.sum()])
    share = np.floor(n * areas / areas.sum()).astype(np.int64)
    share[0] += n - share.sum()
    n_ground, n_roof, n_wall, n_tree = (int(v) for v in share)

    # ground (including under roofs: the tile keeps a complete terrain layer)
    gx = rng.uniform(0.0, ex, n_ground)
    gy = rng.uniform(0.0, ey, n_ground)
    gz = terrain(gx, gy, seed) + rng.normal(0.0, noise, n_ground)

    # roofs: pick a building by roof area, uniform on its roof
    b = rng.choice(n_buildings, n_roof, p=roof_area / roof_area.sum())
    rx = bx[b] + rng.uniform(0.0, 1.0, n_roof) * bw[b]
    ry = by[b] + rng.uniform(0.0, 1.0, n_roof) * bd[b]
    rz = terrain(bx[b] + 0.5 * bw[b], by[b] + 0.5 * bd[b], seed) + bh[b] + rng.normal(0.0, noise, n_roof)

    # walls: pick a building by wall area, then a wall by its length
    b = rng.choice(n_buildings, n_wall, p=wall_area / wall_area.sum())
    t = rng.uniform(0.0, 1.0, n_wall) * 2.0 * (bw[b] + bd[b])
    h = rng.uniform(0.0, 1.0, n_wall) * bh[b]
    wx = np.where(t < bw[b], bx[b] + t,
         np.where(t < bw[b] + bd[b], bx[b] + bw[b],
         np.where(t < 2 * bw[b] + bd[b], bx[b] + bw[b] - (t - bw[b] - bd[b]), bx[b])))
    wy = np.where(t < bw[b], by[b],
         np.where(t < bw[b] + bd[b], by[b] + (t - bw[b]),
         np.where(t < 2 * bw[b] + bd[b], by[b] + bd[b], by[b] + bd[b] - (t - 2 * bw[b] - bd[b]))))
    wx = wx + rng.normal(0.0, noise, n_wall)
    wy = wy + rng.normal(0.0, noise, n_wall)
    wz = terrain(bx[b] + 0.5 * bw[b], by[b] + 0.5 * bd[b], seed) + h

    # trees: Gaussian crown around the stem, vertical scatter over the crown
    tt = rng.choice(n_trees, n_tree, p=tree_area / tree_area.sum())
    cx = tx[tt] + rng.normal(0.0, 0.5, n_tree) * crown_r[tt]
    cy = ty[tt] + rng.normal(0.0, 0.5, n_tree) * crown_r[tt]
    cz = terrain(tx[tt], ty[tt], seed) + th[tt] * np.clip(rng.normal(0.7, 0.15, n_tree), 0.05, 1.0)
    cx = np.clip(cx, 0.0, ex)
    cy = np.clip(cy, 0.0, ey)

    xyz = np.concatenate([
        np.stack([gx, gy, gz], 1), np.stack([rx, ry, rz], 1),
        np.stack([np.clip(wx, 0.0, ex), np.clip(wy, 0.0, ey), wz], 1), np.stack([cx, cy, cz], 1)])
    assert xyz.shape[0] == n
    return _finish(xyz, rng, offset)


def _radial_plane(rng, m: int, h: float, rmax: float, smin: float, angular: float):
    """Radii on a plane at distance h from a scanner, density ~ 1/d^2 with
    d^2 = rho^2 + h^2 (a constant-angular-step scanner), clipped so that the
    spacing d*angular never drops below smin.  Returns (rho, phi)."""
    # pdf(rho) ~ rho / (rho^2 + h^2): inverse CDF in closed form
    u = rng.uniform(0.0, 1.0, m)
    a = h * h
    b = rmax * rmax + h * h
    rho = np.sqrt(np.maximum(a * (b / a) ** u - a, 0.0))
    phi = rng.uniform(0.0, 2.0 * math.pi, m)
    return rho, phi


def tls_street(n: int = 20_000_000, seed: int = CONFIG_SEED + 2, offset=UTM_OFFSET,
               length: float = 300.0, width: float = 20.0, facade_h: float = 20.0,
               n_scanners: int = 8, n_poles: int = 500) -> np.ndarray:
    """TLS/MLS-like street canyon: ground plane, two facade planes, cylindrical
    poles, sampled from ``n_scanners`` positions at 1.8 m height with density
    ~ 1/d^2 from the scanner (spacing clipped to 0.002 - 0.5 m)."""
    rng = np.random.default_rng(seed)
    sx = (np.arange(n_scanners) + 0.5) * (length / n_scanners)
    sh = 1.8
    hw = 0.5 * width
    per = np.full(n_scanners, n // n_scanners, np.int64)
    per[: n - per.sum()] += 1
    # poles along both sidewalks
    px = rng.uniform(0.0, length, n_poles)
    py = np.where(rng.uniform(0.0, 1.0, n_poles) < 0.5, -hw + 1.5, hw - 1.5)
    pr = rng.uniform(0.1, 0.3, n_poles)
    ph = rng.uniform(3.0, 10.0, n_poles)
    out = []
    for s in range(n_scanners):
        m = int(per[s])
        m_ground = int(0.45 * m)
        m_fac = int(0.45 * m)
        m_pole = m - m_ground - m_fac
        # ground: plane z = 0 at distance sh below the scanner
        rho, phi = _radial_plane(rng, m_ground, sh, 60.0, 0.002, 0.001)
        gx = sx[s] + rho * np.cos(phi)
        gy = rho * np.sin(phi)
        keep = (gx >= 0) & (gx <= length) & (np.abs(gy) <= hw)
        gx = np.where(keep, gx, rng.uniform(0.0, length, m_ground))
        gy = np.where(keep, gy, rng.uniform(-hw, hw, m_ground))
        gz = rng.normal(0.0, 0.005, m_ground)
        # facades: planes y = +-hw at distance hw from the scanner
        side = np.where(rng.uniform(0.0, 1.0, m_fac) < 0.5, -1.0, 1.0)
        rho, phi = _radial_plane(rng, m_fac, hw, 60.0, 0.002, 0.001)
        fx = sx[s] + rho * np.cos(phi)
        fz = sh + rho * np.sin(phi)
        keep = (fx >= 0) & (fx <= length) & (fz >= 0) & (fz <= facade_h)
        fx = np.where(keep, fx, rng.uniform(0.0, length, m_fac))
        fz = np.where(keep, fz, rng.uniform(0.0, facade_h, m_fac))
        fy = side * hw + rng.normal(0.0, 0.005, m_fac)
        # poles: choose a pole with weight ~ 1/d^2 to this scanner, uniform on it
        d2 = (px - sx[s]) ** 2 + py ** 2
        w = 1.0 / np.maximum(d2, 1.0)
        pi = rng.choice(n_poles, m_pole, p=w / w.sum())
        ang = rng.uniform(0.0, 2.0 * math.pi, m_pole)
        qx = px[pi] + pr[pi] * np.cos(ang)
        qy = py[pi] + pr[pi] * np.sin(ang)
        qz = rng.uniform(0.0, 1.0, m_pole) * ph[pi]
        out.append(np.stack([gx, gy, gz], 1))
        out.append(np.stack([fx, fy, fz], 1))
        out.append(np.stack([qx, qy, qz], 1))
    xyz = np.concatenate(out)
    assert xyz.shape[0] == n
    return _finish(xyz, rng, offset)


def batched_tile_sizes(ntiles: int = 256, total: int = 60_000_000, lo: int = 10_000,
                       hi: int = 2_000_000, seed: int = CONFIG_SEED + 3) -> np.ndarray:
    """Log-uniform tile sizes in [lo, hi], rescaled by one common factor so
    that they sum to about ``total`` and clamped back to [lo, hi]."""
    rng = np.random.default_rng(seed)
    s = np.exp(rng.uniform(math.log(lo), math.log(hi), ntiles))
    s = s * (total / s.sum())
    return np.clip(np.round(s), lo, hi).astype(np.int64)


def batched_tiles(ntiles: int = 256, total: int = 60_000_000, seed: int = CONFIG_SEED + 3):
    """Batch of ALS-like tiles (generator of ``als_uniform``) at density
    U(5, 60) pts/m^2, side sqrt(n / density), each with its own UTM-like
    origin.  Returns (xyz float64 (sum n, 3), offsets int64 [ntiles+1])."""
    rng = np.random.default_rng(seed)
    sizes = batched_tile_sizes(ntiles, total, seed=seed)
    dens = rng.uniform(5.0, 60.0, ntiles)
    parts = []
    for t in range(ntiles):
        side = math.sqrt(sizes[t] / dens[t])
        org = (400000.0 + 1000.0 * rng.integers(0, 500), 5000000.0 + 1000.0 * rng.integers(0, 500), 0.0)
        parts.append(als_uniform(int(sizes[t]), (side, side), seed=seed * 1000 + t, offset=org))
    offsets = np.zeros(ntiles + 1, np.int64)
    np.cumsum(sizes, out=offsets[1:])
    return np.ascontiguousarray(np.concatenate(parts)), offsets


def sample_queries(xyz: np.ndarray, m: int, seed: int) -> np.ndarray:
    """``m`` query points drawn uniformly (with replacement) from the cloud."""
    rng = np.random.default_rng(seed)
    return np.ascontiguousarray(xyz[rng.integers(0, xyz.shape[0], m)])


def random_cloud(n: int, extent=(10.0, 10.0, 3.0), seed: int = 1, offset=(0.0, 0.0, 0.0)):
    """Uniform random points in a box (tests)."""
    rng = np.random.default_rng(seed)
    xyz = rng.uniform(0.0, 1.0, (n, 3)) * np.asarray(extent)[None, :]
    return np.ascontiguousarray(xyz + np.asarray(offset)[None, :])


def lattice_cloud(half: int, offset=(0.0, 0.0, 0.0), spacing: float = 1.0) -> np.ndarray:
    """Integer lattice {-half..half}^3 * spacing + offset, shuffled order fixed
    by a seed.  With integer offsets every coordinate difference is exact."""
    g = np.arange(-half, half + 1, dtype=np.float64) * spacing
    x, y, z = np.meshgrid(g, g, g, indexing="ij")
    xyz = np.stack([x.ravel(), y.ravel(), z.ravel()], 1) + np.asarray(offset)[None, :]
    rng = np.random.default_rng(12345)
    return np.ascontiguousarray(xyz[rng.permutation(xyz.shape[0])])


def adversarial_cloud(n: int, seed: int = 7, cell: float = 1.0, offset=UTM_OFFSET) -> np.ndarray:
    """Hard cases for a grid: exact duplicates, points on voxel faces (integer
    multiples of ``cell`` from the corner), clusters, and ordinary points."""
    rng = np.random.default_rng(seed)
    k = n // 4
    base = rng.uniform(0.0, 8.0, (n - 3 * k, 3))
    faces = rng.integers(0, 9, (k, 3)).astype(np.float64) * cell
    faces[:, 2] += rng.uniform(0.0, 2.0, k)
    dup_src = base[rng.integers(0, base.shape[0], k)]
    clus = 4.0 + rng.normal(0.0, 0.05, (k, 3))
    xyz = np.concatenate([base, faces, dup_src, clus])
    xyz[0] = 0.0  # pin the bounding-box corner to a lattice point
    return _finish(xyz, rng, offset)
