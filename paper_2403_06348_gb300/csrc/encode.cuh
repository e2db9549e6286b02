// Host-side launchers of the encode kernels (encode.cu).
#pragma once

#include "alto_internal.cuh"

namespace alto {

cudaError_t launch_linearize(const DecodePlan &dp, const uint32_t *coords, uint64_t nnz,
                             const uint64_t *dims_dev, uint64_t *keys, uint32_t *status, int num_sms,
                             cudaStream_t s);

// ||X||^2 with duplicate positions summed into one cell (keys must be sorted).
uint64_t norm_chunks(uint64_t nnz);
cudaError_t launch_norm(int kw, const uint64_t *keys, const float *vals, uint64_t nnz, double *head,
                        double *tail, uint8_t *flags, double *norm_sq, int num_sms, cudaStream_t s);

// Device workspace of launch_radix_sort (look-back words, digit counts, tickets).
size_t sort_workspace_bytes(uint64_t nnz);

// Stable LSD radix sort of nnz (position, value) pairs on their low nbits
// bits. keys[0] holds the positions, vals_in the values; the result lands in
// keys[*final_buf] / vals[*final_buf]. work holds sort_workspace_bytes(nnz)
// bytes. A bounded look-back wait that expires sets kStatusTimeout in *status.
// skip_constant reads the digit counts back (one stream synchronisation) and
// leaves out every pass whose digit is the same for all positions.
// *passes_run (may be NULL) counts the passes launched.
cudaError_t launch_radix_sort(int kw, int nbits, uint64_t nnz, uint64_t *keys[2], float *vals[2],
                              const float *vals_in, void *work, uint32_t *status, bool skip_constant,
                              int *final_buf, int *passes_run, int num_sms, cudaStream_t s);

cudaError_t launch_partition(const DecodePlan &dp, const uint64_t *keys, uint64_t nnz, uint64_t L,
                             uint32_t *intervals, uint32_t *max_len, int num_sms, cudaStream_t s);

cudaError_t launch_hot_rows(const DecodePlan &dp, const uint64_t *keys, uint64_t nnz,
                            const uint64_t *dims, uint64_t L, uint32_t *const *counts_dev_ptrs,
                            uint32_t *const *counts_host_ptrs, uint32_t *scratch, uint64_t *list,
                            uint32_t *const *hot_rows, uint32_t *nhot, int num_sms,
                            cudaStream_t s);

cudaError_t launch_decode(const DecodePlan &dp, const uint64_t *keys, uint64_t nnz, uint32_t *coords,
                          int num_sms, cudaStream_t s);

}  // namespace alto
