// cg_sort.cuh -- device-wide scan and radix sort used by the build and the
// query passes (internal).
#pragma once
#include "cg_internal.cuh"

namespace cg {

// Scratch bytes for exclusive_scan_* over n elements.
size_t scan_scratch_bytes(int64_t n);

// out[0..n] = exclusive prefix sums of in[0..n); out[n] = total.
cudaError_t exclusive_scan_u32_i64(const uint32_t* in, int64_t* out, int64_t n, void* scratch,
                                   uint32_t* err, cudaStream_t st);
cudaError_t exclusive_scan_u32_u32(const uint32_t* in, uint32_t* out, int64_t n, void* scratch,
                                   uint32_t* err, cudaStream_t st);

// Scratch bytes for radix_sort_pairs over n keys.
size_t radix_sort_scratch_bytes(int64_t n);

// Stable LSD radix sort of keys[0..n) (only the low key_bits bits are
// examined); writes the sorted keys and, for each sorted position, the
// input position of its key (the permutation).  keys is not modified.
cudaError_t radix_sort_pairs(const uint32_t* keys, int64_t n, int key_bits, uint32_t* keys_sorted,
                             uint32_t* vals_sorted, void* scratch, uint32_t* err,
                             cudaStream_t st);

}  // namespace cg
