// cg_query.cuh -- query-side structures shared by the radius and k-NN
// kernels (internal).
#pragma once
#include "cg_index.h"

namespace cg {

// Decision thresholds of the binary32 path (see make_thresholds).
struct Thresholds {
  double r2;      // fl64(r * r)
  float s_lo;     // sphere: binary32 value <= s_lo  -> inside for sure
  float s_hi;     // sphere: binary32 value >  s_hi  -> outside for sure
  float c_lo;     // cube, per axis
  float c_hi;
  float r_f;      // r rounded up to binary32
  float e_q;      // encode error bound of the queries used here
  float pad_[2];
};

// Error model of the binary32 offset test (derivation in the design notes):
// e_p, e_q bound |x~ - (x - O)| for indexed points and queries per axis.
__host__ __device__ Thresholds make_thresholds(double r, double e_p, double e_q);

// Queries of one call, in block order.
struct QuerySet {
  int all_points;              // queries are the indexed points
  uint32_t nq;
  uint32_t nblocks;
  const uint32_t* blk_beg;     // [nblocks+1] block start in query order
  const uint32_t* blk_key;     // [nblocks] voxel key of the block
  const float4* qrec;          // [nq] x~, y~, z~, id bits (binary32)
  const double4_32a* qrec64;       // [nq] x, y, z, id bits (binary64)
  const double* q64;           // [nq][3] original order, exact coordinates
};

// Builds (or reuses) the plan of an external query set on ix->plan.
cg_status prepare_queries(cg_index* ix, const double* q, int64_t nq, cudaStream_t st);
QuerySet query_set(cg_index* ix, const double* q, int64_t nq, bool all_points);

}  // namespace cg
