"""Exact-rational model of the fixed predicates, for pinning rounding order.

Test infrastructure.  The predicates of the method (Section 2's sphere, cube
and vertical cylinder, with the evaluation order fixed by the project
statement) are evaluated here step by step on ``fractions.Fraction`` values,
each step rounded to binary64 by ``rn64`` (round to nearest, ties to even),
written from the IEEE 754 definition.  Nothing here calls the oracle or the
CUDA library, and neither of them imports this module.

``boundary_cases`` searches, with a seeded generator, for (centre, point,
radius) triples on which the specified evaluation order and a plausible
wrong one (a fused multiply-add, a re-associated sum, exact arithmetic, a
comparison of roots, a strict comparison) disagree
about membership.  A predicate that deviates from the specified order in
that way fails at least one of them.
"""
from __future__ import annotations

import math
import functools
from fractions import Fraction

import numpy as np

SPHERE, CUBE, CYLINDER = 0, 1, 2

_EMIN = -1074  # exponent of the smallest binary64 subnormal


def rn64(x: Fraction) -> Fraction:
    """Round an exact rational to the nearest binary64 value, ties to even."""
    if x == 0:
        return Fraction(0)
    neg = x < 0
    a = -x if neg else x
    num, den = a.numerator, a.denominator
    e = num.bit_length() - den.bit_length()  # 2^e <= a < 2^(e+1) after fix-up
    if (num << max(0, -e)) < (den << max(0, e)):
        e -= 1
    q = max(e - 52, _EMIN)                   # weight of the last kept bit
    if q >= 0:
        m, rem = divmod(num, den << q)
        half = den << q
    else:
        m, rem = divmod(num << -q, den)
        half = den
    twice = 2 * rem
    if twice > half or (twice == half and (m & 1)):
        m += 1
    v = Fraction(m) * (Fraction(2) ** q)
    return -v if neg else v


def F(v: float) -> Fraction:
    return Fraction(float(v))


# ------------------------------------------------------- predicate values


def sphere_d2(d) -> Fraction:
    """fl(fl(fl(dx^2) + fl(dy^2)) + fl(dz^2)), every step rounded."""
    dx, dy, dz = (F(t) for t in d)
    a, b, c = rn64(dx * dx), rn64(dy * dy), rn64(dz * dz)
    return rn64(rn64(a + b) + c)


def cube_m2(d) -> Fraction:
    """max(fl(dx^2), fl(dy^2), fl(dz^2))."""
    return max(rn64(F(t) * F(t)) for t in d)


def cyl_d2(d) -> Fraction:
    """fl(fl(dx^2) + fl(dy^2)); z does not enter."""
    dx, dy = F(d[0]), F(d[1])
    return rn64(rn64(dx * dx) + rn64(dy * dy))


def r2_of(r: float) -> Fraction:
    return rn64(F(r) * F(r))


def spec_inside(kind: int, d, r: float) -> bool:
    v = {SPHERE: sphere_d2, CUBE: cube_m2, CYLINDER: cyl_d2}[kind](d)
    return v <= r2_of(r)


# ---------------------------------------- plausible wrong evaluation orders


def _sq(t):
    return F(t) * F(t)


def _alt_values(kind: int):
    """Wrong predicate values (exact rationals) by name, per kernel."""
    if kind == SPHERE:
        def fma_z(d):       # fl(s + dz*dz) with dz*dz unrounded
            a, b = rn64(_sq(d[0])), rn64(_sq(d[1]))
            return rn64(rn64(a + b) + _sq(d[2]))

        def fma_xy_a(d):    # fma(dy, dy, fl(dx^2)), then + fl(dz^2)
            s = rn64(rn64(_sq(d[0])) + _sq(d[1]))
            return rn64(s + rn64(_sq(d[2])))

        def fma_xy_b(d):    # fma(dx, dx, fl(dy^2)), then + fl(dz^2)
            s = rn64(rn64(_sq(d[1])) + _sq(d[0]))
            return rn64(s + rn64(_sq(d[2])))

        def fma_all_a(d):   # both additions contracted
            s = rn64(rn64(_sq(d[0])) + _sq(d[1]))
            return rn64(s + _sq(d[2]))

        def fma_all_b(d):
            s = rn64(rn64(_sq(d[1])) + _sq(d[0]))
            return rn64(s + _sq(d[2]))

        def reassoc_yz(d):  # dx^2 + (dy^2 + dz^2)
            a, b, c = (rn64(_sq(t)) for t in d)
            return rn64(a + rn64(b + c))

        def reassoc_xz(d):  # (dx^2 + dz^2) + dy^2
            a, b, c = (rn64(_sq(t)) for t in d)
            return rn64(rn64(a + c) + b)

        def exact(d):       # no rounding at all (extended precision)
            return _sq(d[0]) + _sq(d[1]) + _sq(d[2])

        return {"fma_z": fma_z, "fma_xy_a": fma_xy_a, "fma_xy_b": fma_xy_b,
                "fma_all_a": fma_all_a, "fma_all_b": fma_all_b,
                "reassoc_yz": reassoc_yz, "reassoc_xz": reassoc_xz, "exact": exact}
    if kind == CYLINDER:
        def fma_a(d):
            return rn64(rn64(_sq(d[0])) + _sq(d[1]))

        def fma_b(d):
            return rn64(rn64(_sq(d[1])) + _sq(d[0]))

        def exact(d):
            return _sq(d[0]) + _sq(d[1])

        return {"fma_a": fma_a, "fma_b": fma_b, "exact": exact}
    return {}


def _alt_members(kind: int):
    """Wrong membership rules that are not a different value compared with
    fl(r*r): roots, absolute values, a strict comparison."""
    val = {SPHERE: sphere_d2, CUBE: cube_m2, CYLINDER: cyl_d2}[kind]

    def sqrt_cmp(d, r):      # fl(sqrt(v)) <= r
        return math.sqrt(float(val(d))) <= r

    def strict(d, r):        # v < fl(r*r)
        return val(d) < r2_of(r)

    if kind == CUBE:
        # For normal binary64 values, x -> fl(x*x) is strictly increasing (the
        # exact squares of neighbouring doubles lie more than one unit in the
        # last place apart), so fl(dx^2) <= fl(r^2) holds exactly when
        # |dx| <= r, and fl(sqrt(fl(x^2))) = |x|: the absolute-value and
        # root comparisons agree with the specified rule everywhere and
        # cannot be told apart by any case.  Only the strict comparison can.
        return {"strict": strict}
    return {"sqrt_cmp": sqrt_cmp, "strict": strict}


def alternatives(kind: int) -> list[str]:
    return sorted(_alt_values(kind)) + sorted(_alt_members(kind))


def _radii_near(x: float, steps: int = 6):
    """Doubles within a few units in the last place of x (x > 0)."""
    out = [x]
    lo = hi = x
    for _ in range(steps):
        lo = math.nextafter(lo, 0.0)
        hi = math.nextafter(hi, math.inf)
        out += [lo, hi]
    return [t for t in out if t > 0]


def _radius_with_r2_in(lo: Fraction, hi: Fraction):
    """A double r with lo <= fl(r*r) < hi, or None."""
    for r in _radii_near(math.sqrt(float(lo)), 8):
        t = r2_of(r)
        if lo <= t < hi:
            return r
    return None


def _direction(rng, kind):
    if kind == CUBE:                 # one axis dominant, the others smaller
        v = rng.uniform(-0.9, 0.9, 3)
        ax = int(rng.integers(0, 3))
        v[ax] = rng.choice([-1.0, 1.0])
        return v
    v = rng.normal(size=3)
    if kind == CYLINDER:
        v[2] = rng.uniform(-3.0, 3.0)  # any height: the cylinder ignores it
        n = math.hypot(v[0], v[1])
        return np.array([v[0] / n, v[1] / n, v[2]])
    return v / np.linalg.norm(v)


def _try_one(kind, alt, d, rng):
    """A radius on which the specified rule and `alt` disagree for offset d."""
    vals = _alt_values(kind)
    if alt in vals:
        s = {SPHERE: sphere_d2, CUBE: cube_m2, CYLINDER: cyl_d2}[kind](d)
        a = vals[alt](d)
        if s == a:
            return None
        lo, hi = (s, a) if s < a else (a, s)
        return _radius_with_r2_in(lo, hi)
    wrong = _alt_members(kind)[alt]
    base = {SPHERE: sphere_d2, CUBE: cube_m2, CYLINDER: cyl_d2}[kind](d)
    cands = _radii_near(math.sqrt(float(base)), 8)
    rng.shuffle(cands)
    for r in cands:
        if spec_inside(kind, d, r) != wrong(d, r):
            return r
    return None


def boundary_cases(kind: int, alt: str, n: int, seed: int, origin=(0.0, 0.0, 0.0),
                   spacing: float = 16.0, start: int = 0, max_tries: int = 20000):
    """n triples (centre c, point p, radius r, inside) with p - c exact in
    binary64, on which the specified rule and `alt` disagree.

    Centre i sits on a grid of `spacing` metres from `origin` (slot
    start + i), so triples laid out together never see each other's points
    for radii below spacing / 2.  `inside` is the specified membership,
    decided here in exact rational arithmetic."""
    rng = np.random.default_rng(seed)
    out = []
    tries = 0
    while len(out) < n:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"no boundary case found for {kind}/{alt}")
        slot = start + len(out)
        c = np.array([origin[0] + spacing * (slot % 32) + rng.uniform(0.25, 0.75),
                      origin[1] + spacing * (slot // 32) + rng.uniform(0.25, 0.75),
                      origin[2] + rng.uniform(0.25, 0.75)])
        rho = rng.uniform(0.3, 2.5)
        p = c + rho * _direction(rng, kind)
        d = p - c
        # p - c must be exact (Sterbenz holds for these magnitudes; checked)
        if any(Fraction(float(p[a])) - Fraction(float(c[a])) != F(d[a]) for a in range(3)):
            continue
        r = _try_one(kind, alt, d, rng)
        if r is None or r >= spacing / 2:
            continue
        out.append((c.copy(), p.copy(), float(r), spec_inside(kind, d, r)))
    return out


ORIGINS = {"utm": (508000.0, 5440000.0, 100.0), "local": (0.0, 0.0, 0.0)}
KINDS = {SPHERE: "sphere", CUBE: "cube", CYLINDER: "cylinder"}
PER_ORIGIN = 4


@functools.lru_cache(maxsize=None)
def standard_cases():
    """(kind, alt, origin, c, p, r, inside) for every kernel, wrong rule and
    origin; seeded, so the oracle's pins and the GPU parity tests see the
    same triples.  Every case of an origin has its own grid slot."""
    out = []
    slot = {o: 0 for o in ORIGINS}
    for kind in KINDS:
        for ai, alt in enumerate(alternatives(kind)):
            for oi, (oname, org) in enumerate(ORIGINS.items()):
                seed = 0x5EED1000 + 1000 * kind + 10 * ai + oi
                for c, p, r, inside in boundary_cases(kind, alt, PER_ORIGIN, seed, origin=org,
                                                      start=slot[oname]):
                    out.append((kind, alt, oname, c, p, r, inside))
                slot[oname] += PER_ORIGIN
    return tuple(out)
