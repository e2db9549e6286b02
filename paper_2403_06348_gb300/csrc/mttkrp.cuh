// MTTKRP kernel arguments and launchers (mttkrp*.cu).
#pragma once

#include "alto_internal.cuh"

namespace alto {

constexpr int kMttkrpThreads = 1024;  // one persistent CTA per SM

struct MttkrpArgs {
  DecodePlan dp;               // permuted: coordinate 0 is the output mode
  const uint64_t *keys;        // ordered positions [nnz][kw]
  const float *vals;           // ordered values [nnz]
  uint64_t nnz;
  uint64_t L;                  // line segments
  const uint32_t *intervals;   // [L][N][2] (original mode order)
  const void *factors[kMaxModes];  // permuted like dp; factors[0] unused
  float *out;                  // [I_mode][R]
  int mode;                    // output mode in the original order
  int R;
  int flush_every;             // ATOMIC: segments between flushes of the hot table
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

// cpl = factor columns per lane (R / cpl lanes work on one nonzero).
cudaError_t launch_mttkrp(const MttkrpArgs &a, int cpl, bool bf16, bool pull, size_t smem,
                          int num_sms, cudaStream_t s);

// Specialisations by the number of modes (0 = any number, decided at run time).
template <int NT>
cudaError_t launch_mttkrp_nt(const MttkrpArgs &a, int cpl, bool bf16, bool pull, size_t smem,
                             int num_sms, cudaStream_t s);

cudaError_t launch_pull_reduce(const float *partials, const uint64_t *row_ptr, const uint64_t *prow,
                               uint64_t I, int R, float *out, int num_sms, cudaStream_t s);

}  // namespace alto
