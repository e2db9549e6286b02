// MTTKRP kernel arguments and launchers (mttkrp.cu).
#pragma once

#include "alto_internal.cuh"

namespace alto {

struct MttkrpArgs {
  DecodePlan dp;
  const uint64_t *keys;        // ordered positions [nnz][kw]
  const float *vals;           // ordered values [nnz]
  uint64_t nnz;
  uint64_t L;                  // line segments
  const uint32_t *intervals;   // [L][N][2]
  const void *factors[kMaxModes];
  float *out;                  // [I_mode][R]
  int mode;
  int R;
  // ATOMIC variant: hot rows staged in shared memory
  const uint64_t *htab;        // (slot << 32 | row), empty = ~0
  const uint32_t *slot_rows;   // row of every slot
  int hbits;
  int nslots;
  // PULL variant
  float *partials;             // Temp_l of every segment, back to back
  const uint64_t *part_off;    // first partial row of each segment [L]
};

// Shared memory the segment kernel needs.
size_t mttkrp_smem_bytes(bool pull, int R, int nslots, int hbits, uint32_t max_interval);

// Largest dynamic shared memory a block may use on this device.
size_t mttkrp_smem_limit();

cudaError_t launch_mttkrp(const MttkrpArgs &a, int cpl, bool bf16, bool pull, size_t smem,
                          int num_sms, cudaStream_t s);

cudaError_t launch_pull_reduce(const float *partials, const uint64_t *row_ptr, const uint64_t *prow,
                               uint64_t I, int R, float *out, int num_sms, cudaStream_t s);

}  // namespace alto
