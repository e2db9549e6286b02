// Grouped MTTKRP: many encoded tensors, each with its own output mode, rank
// and number of modes, streamed by one persistent launch (group.cu). The CP-ALS
// batch (batch.cu) runs its MTTKRP step through the same kernel.
#pragma once

#include "alto_internal.cuh"

namespace alto {

// One MTTKRP problem of a grouped launch, in device memory.
struct GroupProb {
  BlockPlan bp;                 // decode by blocks (N = 3, 4, 5); out_rank unused
  const DecodePlan32 *dp;       // runs by rank (any N), device memory
  const uint64_t *keys;         // ordered positions [nnz][kw]
  const float *vals;            // [nnz]
  uint64_t nnz;
  uint64_t L;                   // line segments (the units of work)
  const uint32_t *intervals;    // [L][N][2], original mode order
  const void *fac[kMaxModes];   // factor matrix of every rank (row-major I x R)
  float *out;                   // output rows of the current mode, zero on entry
  const int *cur_mode;          // CP-ALS batch: current mode (else null: `mode`)
  const int *done;              // CP-ALS batch: nonzero once the run stopped
  uint64_t dims[kMaxModes];     // by mode
  uint32_t max_interval[kMaxModes];  // by mode
  int rank_of[kMaxModes];
  // hot rows of each mode (by mode; nslots 0 = none): open-addressing table
  // (slot << 32 | row, empty = ~0) and the row of every slot
  const uint64_t *htab[kMaxModes];
  const uint32_t *slot_rows[kMaxModes];
  int hbits[kMaxModes];
  int nslots[kMaxModes];
  int N, kw, R, mode;
};

// Dynamic shared memory the grouped kernel stages output rows in: a segment
// whose interval of the output mode holds at most this many bytes of rows
// (interval length x R x 4) keeps its Temp in shared memory and flushes it at
// the end; any other segment stages the mode's hot rows (table and slots in
// the same space) and adds its other runs straight to the output.
size_t group_stage_bytes();

// Sets the kernel's shared-memory limit (once; call before stream capture).
cudaError_t configure_group_mttkrp();

// Units u = 0 .. unit_off[P] - 1 (P = *nprobs) are (problem, segment) pairs:
// problem p = unit_prob[u] owns units unit_off[p] .. unit_off[p+1] - 1. CTAs
// take units in turn from ctr[0] (zero on entry); the last CTA to finish puts
// ctr[0] and ctr[1] back to 0, so the same counters serve the next launch.
cudaError_t launch_group_mttkrp(const GroupProb *probs, const uint64_t *unit_off,
                                const uint32_t *unit_prob, const int *nprobs, unsigned *ctr, bool bf16,
                                int num_sms, cudaStream_t s);

}  // namespace alto

struct alto_tensor;

namespace alto {

// Puts the handle's decode runs, in rank order, on the device (once).
alto_status ensure_rank_runs(alto_tensor *h, cudaStream_t s);

// The problem fields that come from the handle (everything but the mode,
// the factors and the output). Builds, for every mode whose segments do not
// all fit the staging space, the handle's grouped hot-row table; waits for s.
alto_status fill_group_prob(alto_tensor *h, int R, GroupProb *q, cudaStream_t s);

}  // namespace alto
