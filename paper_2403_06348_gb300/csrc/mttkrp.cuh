// MTTKRP kernel arguments and launchers (mttkrp*.cu).
#pragma once

#include "alto_internal.cuh"

namespace alto {

// Persistent CTAs: kMttkrpBlocksPerSm CTAs of kMttkrpThreads threads per SM.
// Three CTAs of 512 threads (48 warps, at most 40 registers a thread) hide
// more gather latency than one CTA of 1024 threads at 64 registers.
#ifndef ALTO_MTTKRP_THREADS
#define ALTO_MTTKRP_THREADS 512
#endif
#ifndef ALTO_MTTKRP_BLOCKS_PER_SM
#define ALTO_MTTKRP_BLOCKS_PER_SM 3
#endif
constexpr int kMttkrpThreads = ALTO_MTTKRP_THREADS;
constexpr int kMttkrpBlocksPerSm = ALTO_MTTKRP_BLOCKS_PER_SM;

// Coordinates inside the kernel are in rank order (modes sorted by length).
struct MttkrpArgs {
  BlockPlan bp;                // decode by blocks (kernels specialised on N)
  DecodePlan32 dp;             // decode by 32-bit runs, rows in rank order (any N)
  const uint64_t *keys;        // ordered positions [nnz][kw]
  const float *vals;           // ordered values [nnz]
  uint64_t nnz;
  uint64_t L;                  // line segments
  const uint32_t *intervals;   // [L][N][2] (original mode order)
  const void *factors[kMaxModes];  // by rank; the output rank's entry is unused
  const void *fin[kMaxModes];      // the N-1 input factors, ranks in order without the output
  float *out;                  // [I_mode][R]
  int mode;                    // output mode in the original order
  int out_rank;                // its rank
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
  // CP-APR model update Phi (Alg. 5)
  const float *bmat;           // B of the output mode [I_n][R]
  const float *pimat;          // precomputed Pi [nnz][R] (PRE) or null (OTF)
  float eps;
  const int *skip;             // nonzero: return at once (inner loop converged)
  // output-oriented traversal (Alg. 4): pos_out of the output mode [nnz]
  const uint32_t *perm;
  // in-tile output-oriented traversal (TILED): htab holds nbins hot rows, the
  // first nslots of them staged in shared memory, the rest ("warm") summed in
  // kWarmReps fp64 replicas [kWarmReps][nbins][R] (zero between launches)
  int nbins;
  double *warm;
  uint32_t *status;            // device status word (kStatusTimeout)
  // byte-table decode (one-word positions): the table [8][256] in global
  // memory, copied into shared memory by the kernels that use it; null: none
  const uint64_t *lut;
  LutPlan lp;
};

// Shared memory the segment kernel needs.
size_t mttkrp_smem_bytes(bool pull, int R, int nslots, int hbits, uint32_t max_interval);

// Largest dynamic shared memory a block may use on this device.
size_t mttkrp_smem_limit();

// Shared memory one segment-kernel CTA may use for its staging table.
size_t mttkrp_stage_budget();

// cpl = factor columns per lane (R / cpl lanes work on one nonzero).
cudaError_t launch_mttkrp(const MttkrpArgs &a, int cpl, bool bf16, bool pull, size_t smem,
                          int num_sms, cudaStream_t s);

// Specialisations by the number of modes (0 = any number, decided at run time).
template <int NT>
cudaError_t launch_mttkrp_nt(const MttkrpArgs &a, int cpl, bool bf16, bool pull, size_t smem,
                             int num_sms, cudaStream_t s);

cudaError_t launch_pull_reduce(const float *partials, const uint64_t *row_ptr, const uint64_t *prow,
                               uint64_t I, int R, float *out, int num_sms, cudaStream_t s,
                               const int *skip = nullptr);

// Phi (Alg. 5) for a.mode: a.bmat set, a.pimat set for PRE.
cudaError_t launch_phi(const MttkrpArgs &a, bool pull, bool pre, size_t smem, int num_sms,
                       cudaStream_t s);

// Largest nnz with a stored output-oriented order (32-bit entries).
constexpr uint64_t kPosOutMaxNnz = 0xFFFFFFFFull - 4096;

// MTTKRP over the stored output-oriented order of a.mode (a.keys / a.vals in
// that order, a.perm its ordered positions); a.htab .. a.nslots the staged hot
// rows (nslots 0: none), smem = mttkrp_smem_bytes(false, R, nslots, hbits, 0).
cudaError_t launch_mttkrp_out(const MttkrpArgs &a, int cpl, bool bf16, size_t smem, int num_sms,
                              cudaStream_t s);

template <int NT>
cudaError_t launch_mttkrp_out_nt(const MttkrpArgs &a, int cpl, bool bf16, size_t smem, int num_sms,
                                 cudaStream_t s);

// Phi (Alg. 5) over the stored order: a.bmat set, a.pimat set for PRE.
cudaError_t launch_phi_out(const MttkrpArgs &a, bool pre, size_t smem, int num_sms, cudaStream_t s);

template <int NT>
cudaError_t launch_phi_out_nt(const MttkrpArgs &a, bool pre, size_t smem, int num_sms, cudaStream_t s);

template <int NT>
cudaError_t launch_phi_nt(const MttkrpArgs &a, bool pull, bool pre, size_t smem, int num_sms,
                          cudaStream_t s);

// MTTKRP over the one ALTO copy, output-oriented inside each tile (tile.cuh):
// a.htab / a.nbins / a.nslots / a.slot_rows the mode's hot rows, a.warm the
// replicas when nbins > nslots (then followed by launch_warm_reduce).
cudaError_t launch_mttkrp_tile(const MttkrpArgs &a, int cpl, bool bf16, bool group, int num_sms,
                               cudaStream_t s);

template <int NT>
cudaError_t launch_mttkrp_tile_nt(const MttkrpArgs &a, int cpl, bool bf16, bool group, int num_sms,
                                  cudaStream_t s);

// Shared memory of one TILED CTA for nmodes, key width kw, rank R, cpl.
size_t tile_smem_bytes(int nmodes, int kw, int R, int cpl, int nslots, int hbits, int nbins, bool lut);

// out(row of warm slot i, :) = sum of the kWarmReps replicas of slot i, for
// slots nslots..nbins-1; the replicas are zeroed again for the next launch.
cudaError_t launch_warm_reduce(double *warm, const uint32_t *slot_rows, int nslots, int nbins, int R,
                               float *out, int num_sms, cudaStream_t s);

// Replicas of the warm rows used by the TILED kernel.
constexpr int kTileWarmReps = 16;

}  // namespace alto
