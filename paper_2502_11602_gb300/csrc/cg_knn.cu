// cg_knn.cu -- exact k-NN (placeholder until the ring kernel lands)
#include "cg_query.cuh"
namespace cg {
cg_status knn_pass(cg_index* ix, bool all_points, const double* q, int64_t nq, int k, int32_t* idx,
                   double* d2, cudaStream_t st) {
  (void)ix; (void)all_points; (void)q; (void)nq; (void)k; (void)idx; (void)d2; (void)st;
  return fail(CG_ERR_UNIMPLEMENTED, "k-NN not built yet");
}
}  // namespace cg
