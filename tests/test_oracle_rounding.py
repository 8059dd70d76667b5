"""Pins for the oracle's rounding order: the binary64 predicates are
evaluated in one fixed order with no fused multiply-add (Section 2's kernels;
the sphere is fl(fl(fl(dx^2) + fl(dy^2)) + fl(dz^2)) <= fl(r^2)).

The expected membership of every case comes from ``exact_rounding``: exact
rationals rounded step by step by a round-to-nearest-even written from the
IEEE definition, never from the oracle's own formulas.  The cases sit on the
boundary where the specified order and a plausible wrong one (a contraction,
a re-associated sum, unrounded arithmetic, a root comparison, a strict
comparison) disagree, so that an oracle built with
contraction switched on or with the terms re-associated fails here; the
mutation tests below build such oracles and check that they do."""
import ctypes
import math
import os
import platform
import subprocess
import sys
from fractions import Fraction

import numpy as np
import pytest

import oracle

sys.path.insert(0, os.path.dirname(__file__))
import exact_rounding as ex  # noqa: E402

ORIGINS = ex.ORIGINS
KINDS = ex.KINDS
PER_ORIGIN = ex.PER_ORIGIN
all_cases = ex.standard_cases


# ----------------------------------------------------- the checker itself


def test_rn64_agrees_with_ieee_hardware():
    # Python floats are IEEE binary64 with round-to-nearest-even: each
    # product and sum of two floats rounded by rn64 must equal the machine's
    rng = np.random.default_rng(7)
    xs = np.concatenate([rng.normal(0, 1, 3000) * 10.0 ** rng.integers(-8, 8, 3000),
                         [1.0, 3.0, 0.1, 2.0 ** -1074, 2.0 ** -1022, 1e308, -5.5]])
    ys = np.roll(xs, 17)
    for a, b in zip(xs.tolist(), ys.tolist()):
        if abs(a * b) < 1e300:
            assert ex.rn64(Fraction(a) * Fraction(b)) == Fraction(a * b)
        assert ex.rn64(Fraction(a) + Fraction(b)) == Fraction(a + b)
    # ties go to even
    one = Fraction(1)
    u = Fraction(2) ** -53
    assert ex.rn64(one + u) == one                 # halfway, 1 is even
    assert ex.rn64(one + 3 * u) == one + 4 * u     # halfway, rounds up to even
    assert ex.rn64(Fraction(2) ** -1075) == 0      # half the smallest subnormal


def test_cube_rule_equals_absolute_comparison():
    # the reason the cube has only the strict comparison as a wrong rule:
    # fl(x^2) <= fl(r^2) exactly when |x| <= r, for normal doubles, including
    # neighbouring pairs one unit in the last place apart
    rng = np.random.default_rng(11)
    xs = rng.uniform(0.05, 4.0, 4000) * 10.0 ** rng.integers(-3, 4, 4000)
    for x in xs.tolist():
        for r in (x, np.nextafter(x, 0.0), np.nextafter(x, np.inf)):
            r = float(r)
            assert (ex.rn64(Fraction(x) ** 2) <= ex.r2_of(r)) == (x <= r)
            assert math.sqrt(float(ex.rn64(Fraction(x) ** 2))) == x


def test_cases_straddle_each_wrong_rule():
    cases = all_cases()
    for kind in KINDS:
        for alt in ex.alternatives(kind):
            got = [cs for cs in cases if cs[0] == kind and cs[1] == alt]
            assert len(got) == PER_ORIGIN * len(ORIGINS), (kind, alt)
    # both memberships occur among the cases
    assert {cs[6] for cs in cases} == {True, False}


# ------------------------------------------------------------ the oracle


def _load(path):
    lib = ctypes.CDLL(path)
    P, D, I64, I = ctypes.c_void_p, ctypes.c_double, ctypes.c_int64, ctypes.c_int
    for name in ("og_d2", "og_cube2", "og_cyl2"):
        getattr(lib, name).restype = D
        getattr(lib, name).argtypes = [P, P]
    lib.og_brute_radius_one.restype = I64
    lib.og_brute_radius_one.argtypes = [P, I64, P, D, I, P]
    return lib


def _ptr(a):
    return a.ctypes.data_as(ctypes.c_void_p)


def _mismatches(lib):
    """Every case where a library's value or membership differs from the
    exact-rational specification."""
    bad = []
    fn = {ex.SPHERE: (lib.og_d2, ex.sphere_d2), ex.CUBE: (lib.og_cube2, ex.cube_m2),
          ex.CYLINDER: (lib.og_cyl2, ex.cyl_d2)}
    for kind, alt, oname, c, p, r, inside in all_cases():
        c = np.ascontiguousarray(c, dtype=np.float64)
        p = np.ascontiguousarray(p, dtype=np.float64)
        f, spec = fn[kind]
        val = f(_ptr(p), _ptr(c))
        if Fraction(val) != spec(p - c):
            bad.append((KINDS[kind], alt, oname, "value"))
        got = lib.og_brute_radius_one(_ptr(p.reshape(1, 3)), 1, _ptr(c), r, kind, None)
        if bool(got) != inside:
            bad.append((KINDS[kind], alt, oname, "membership"))
    return bad


def test_oracle_predicates_follow_the_specified_rounding():
    assert _mismatches(_load(oracle.build())) == []


@pytest.mark.parametrize("dim", [2, 3])
@pytest.mark.parametrize("kind", list(KINDS))
def test_oracle_index_search_on_boundary_cases(kind, dim):
    # Algorithm 1 through the grid index: one query per case, its own point
    # the only one within reach
    cases = [cs for cs in all_cases() if cs[0] == kind]
    for oname in ORIGINS:
        sub = [cs for cs in cases if cs[2] == oname]
        pts = np.array([cs[4] for cs in sub])
        ix = oracle.Index(pts, 1.0, 1.0, dim=dim)
        for i, (_, alt, _, c, _, r, inside) in enumerate(sub):
            row = ix.kernel_search(c, r, kind).tolist()
            assert row == ([i] if inside else []), (KINDS[kind], alt, oname, i)


def test_oracle_knn_distances_are_the_specified_values():
    # k-NN reports the sphere value itself: it must be the specified one
    for oname in ORIGINS:
        sub = [cs for cs in all_cases() if cs[0] == ex.SPHERE and cs[2] == oname]
        pts = np.array([cs[4] for cs in sub])
        qs = np.array([cs[3] for cs in sub])
        ix = oracle.Index(pts, 1.0, 1.0, dim=2)
        idx, d2 = ix.knn(qs, 1)
        for i, cs in enumerate(sub):
            assert idx[i, 0] == i
            assert Fraction(float(d2[i, 0])) == ex.sphere_d2(cs[4] - cs[3])


# ------------------------------------------- planted mistakes must be seen


_SRC = os.path.join(os.path.dirname(oracle.__file__), "cheese_oracle.c")
_D2_BODY = "  double sxy = dx * dx + dy * dy;\n  return sxy + dz * dz;\n"
_CUBE_CMP = "if (kernel == OG_CUBE) return og_cube2(p, c) <= r2;"


def _fma_flags():
    if platform.machine() in ("x86_64", "AMD64"):
        try:
            with open("/proc/cpuinfo") as f:
                if " fma" not in f.read():
                    return None
        except OSError:
            return None
        return ["-mfma"]
    return []  # aarch64 has fused multiply-add in its base instruction set


def _build_variant(tmp_path, name, src_edit=None, extra=(), contract="off"):
    with open(_SRC) as f:
        src = f.read()
    if src_edit is not None:
        old, new = src_edit
        assert old in src, f"planting {name}: pattern not found"
        src = src.replace(old, new)
    cpath = tmp_path / f"{name}.c"
    cpath.write_text(src)
    so = tmp_path / f"lib{name}.so"
    subprocess.check_call(["gcc", "-O2", "-std=c11", f"-ffp-contract={contract}", "-fno-fast-math",
                           *extra, "-shared", "-fPIC", "-o", str(so), str(cpath), "-lm", "-lpthread"])
    return _load(str(so))


def test_planted_contraction_is_detected(tmp_path):
    flags = _fma_flags()
    if flags is None:
        pytest.skip("this CPU has no fused multiply-add")
    lib = _build_variant(tmp_path, "contract", extra=flags, contract="fast")
    bad = _mismatches(lib)
    kinds = {b[0] for b in bad}
    assert "sphere" in kinds and "cylinder" in kinds, bad


def test_planted_reassociation_is_detected(tmp_path):
    lib = _build_variant(tmp_path, "reassoc",
                         src_edit=(_D2_BODY, "  return dx * dx + (dy * dy + dz * dz);\n"))
    bad = _mismatches(lib)
    assert any(b[0] == "sphere" for b in bad), bad


def test_planted_strict_cube_comparison_is_detected(tmp_path):
    lib = _build_variant(tmp_path, "cubestrict",
                         src_edit=(_CUBE_CMP, "if (kernel == OG_CUBE) return og_cube2(p, c) < r2;"))
    bad = _mismatches(lib)
    assert any(b[0] == "cube" and b[3] == "membership" for b in bad), bad


def test_unplanted_rebuild_is_clean(tmp_path):
    # the same build recipe with nothing planted passes: the detections above
    # come from the planted change, not from the recipe
    assert _mismatches(_build_variant(tmp_path, "clean")) == []
