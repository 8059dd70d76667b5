// cg_f32x2.cuh -- candidate tests shared by the radius kernels (internal):
// the exact binary64 predicates and the packed binary32 (f32x2) arithmetic of
// the binary32-offset path.
#pragma once
#include "cg_query.cuh"

namespace cg {
namespace {

// The fixed binary64 predicates (Section 2's sphere, cube and vertical
// cylinder): dx = fl(p - c) per axis, then
//   sphere   fl(fl(fl(dx^2) + fl(dy^2)) + fl(dz^2)) <= r2
//   cylinder fl(fl(dx^2) + fl(dy^2)) <= r2
//   cube     max(fl(dx^2), fl(dy^2), fl(dz^2)) <= r2
// with every operation rounded on its own (no contraction).
template <int KERN>
__device__ __forceinline__ bool exact_in(const double* __restrict__ p, const double* __restrict__ c, double r2) {
  double dx = __dsub_rn(__ldg(p), __ldg(c));
  double dy = __dsub_rn(__ldg(p + 1), __ldg(c + 1));
  double dz = __dsub_rn(__ldg(p + 2), __ldg(c + 2));
  if (KERN == CG_SPHERE)
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) <= r2;
  if (KERN == CG_CYLINDER) return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= r2;
  return fmax(fmax(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) <= r2;
}
template <int KERN>
__device__ __forceinline__ bool exact_in4(const double4_32a& p, const double4_32a& c, double r2) {
  double dx = __dsub_rn(p.x, c.x), dy = __dsub_rn(p.y, c.y), dz = __dsub_rn(p.z, c.z);
  if (KERN == CG_SPHERE)
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) <= r2;
  if (KERN == CG_CYLINDER) return __dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)) <= r2;
  return fmax(fmax(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz)) <= r2;
}

__device__ __forceinline__ unsigned long long pk(float a, float b) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a), "f"(b));
  return r;
}
__device__ __forceinline__ void upk(unsigned long long r, float& a, float& b) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(r));
}
__device__ __forceinline__ unsigned long long sub2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long mul2(unsigned long long a, unsigned long long b) {
  unsigned long long r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}
__device__ __forceinline__ unsigned long long fma2(unsigned long long a, unsigned long long b, unsigned long long c) {
  unsigned long long r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}

// The binary32 values of a candidate pair (packed): squared distance for the
// sphere, its xy part for the cylinder, largest squared axis offset for the
// cube.
template <int KERN>
__device__ __forceinline__ unsigned long long pair_vals(const ulonglong2& xy, unsigned long long zz,
                                                        unsigned long long QX, unsigned long long QY,
                                                        unsigned long long QZ) {
  const unsigned long long DX = sub2(xy.x, QX), DY = sub2(xy.y, QY);
  if (KERN == CG_CYLINDER) return fma2(DY, DY, mul2(DX, DX));
  const unsigned long long DZ = sub2(zz, QZ);
  if (KERN == CG_SPHERE) return fma2(DZ, DZ, fma2(DY, DY, mul2(DX, DX)));
  float a0, a1, b0, b1, c0, c1;
  upk(mul2(DX, DX), a0, a1);
  upk(mul2(DY, DY), b0, b1);
  upk(mul2(DZ, DZ), c0, c1);
  return pk(fmaxf(fmaxf(a0, b0), c0), fmaxf(fmaxf(a1, b1), c1));
}
template <int KERN>
__device__ __forceinline__ void pair_test(const ulonglong2& xy, unsigned long long zz, unsigned long long QX,
                                          unsigned long long QY, unsigned long long QZ, float& v0, float& v1) {
  upk(pair_vals<KERN>(xy, zz, QX, QY, QZ), v0, v1);
}

// m << 1 with the sign bit of x shifted in (one funnel shift).
__device__ __forceinline__ uint32_t push_sign(uint32_t m, float x) {
  uint32_t d;
  asm("shf.l.wrap.b32 %0, %1, %2, 1;" : "=r"(d) : "r"(__float_as_uint(x)), "r"(m));
  return d;
}

// The comparison constants of word_masks for a threshold t (t < FLT_MAX).
__device__ __forceinline__ unsigned long long above(float t) {
  const float T = t < 0.f ? 0.f : __uint_as_float(__float_as_uint(t) + 1u);
  return pk(T, T);
}

}  // namespace
}  // namespace cg
