// The encoded-tensor handle behind alto_handle_t and the pieces of the C ABI
// layer that more than one translation unit needs.
#pragma once

#include <cstdarg>
#include <string>
#include <vector>

#include "alto_internal.cuh"

struct alto_tensor;

namespace alto {

// Sets the calling thread's error message (alto_last_error) and returns st.
alto_status fail(alto_status st, const char *fmt, ...);

#define CUDA_TRY(expr)                                                                       \
  do {                                                                                       \
    cudaError_t e_ = (expr);                                                                 \
    if (e_ != cudaSuccess) return fail(ALTO_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_)); \
  } while (0)

struct ProfEvt {
  int kind;
  cudaEvent_t a, b;
};

struct PullPlan {
  bool valid = false;
  uint64_t *part_off = nullptr;  // [L]
  uint64_t *row_ptr = nullptr;   // [I+1]
  uint64_t *prow = nullptr;      // [entries]
  uint64_t total_rows = 0;
  uint64_t entries = 0;
};

struct HotTable {
  int nslots = -1;
  int hbits = 0;
  uint64_t *htab = nullptr;
};

struct Buf {
  void *p = nullptr;
  size_t bytes = 0;
};

}  // namespace alto

namespace alto {

// Device memory of a handle: its allocator if it has one, else
// cudaMallocAsync / cudaFreeAsync on stream s; counted in bytes_held.
void *dalloc(alto_tensor *h, size_t bytes, cudaStream_t s);
void dfree(alto_tensor *h, void *p, size_t bytes, cudaStream_t s);

// ALTO_ERR_INVALID_ARG unless the current device is the one h was encoded on
// (its buffers, plans and tables live there).
alto_status check_device(const alto_tensor *h);

// Re-partitions the handle into L segments (Section IV-A) on stream s; waits
// for s (the interval lengths come back to the host).
alto_status repartition(alto_tensor *h, uint64_t L, cudaStream_t s);

// A hot-row table of mode n for grouped launches holding the first nslots
// sampled hot rows (at most the number sampled); tables of up to five sizes
// are kept in the handle until alto_free. Waits for s.
alto_status ensure_group_hot(alto_tensor *h, int n, int nslots, cudaStream_t s,
                             const HotTable **out);

// Largest segment of the stored order that one CTA sorts in shared memory;
// by default the order's segments are at most this long.
constexpr uint64_t kPosOutSegCap = 8192;

// pos_out of Alg. 4 for one mode: inside every segment l of L, the ordered
// positions by increasing coordinate of `mode`, ties in line order, as nnz
// uint32 positions in *out (needs nnz < 2^32), and in that order the line
// positions (keys_out, nnz * kw words) and values (vals_out), both allocated
// by the caller. Scratch and *out come from the handle's allocator; *out is
// the caller's (4 * nnz bytes).
alto_status build_pos_out(alto_tensor *h, int mode, uint64_t L, uint32_t **out, uint64_t *keys_out,
                          float *vals_out, cudaStream_t s);

// keys_out[p] = keys[perm[p]], vals_out[p] = vals[perm[p]] (the line
// positions and values in the stored order).
cudaError_t launch_gather_out(const uint32_t *perm, const uint64_t *keys, const float *vals,
                              uint64_t nnz, int kw, uint64_t *keys_out, float *vals_out, int num_sms,
                              cudaStream_t s);

}  // namespace alto

struct alto_tensor {
  using DecodePlan = alto::DecodePlan;
  using DecodePlan32 = alto::DecodePlan32;
  using BlockPlan = alto::BlockPlan;
  using HotTable = alto::HotTable;
  using PullPlan = alto::PullPlan;
  using Buf = alto::Buf;
  using ProfEvt = alto::ProfEvt;
  int N = 0, nbits = 0, kw = 1;
  uint64_t M = 0;
  uint64_t dims[alto::kMaxModes] = {};
  int bits[alto::kMaxModes] = {};
  uint64_t mask_lo[alto::kMaxModes] = {}, mask_hi[alto::kMaxModes] = {};
  DecodePlan dp{};
  DecodePlan32 dp32{};
  BlockPlan bp{};
  int rank_of[alto::kMaxModes] = {};   // rank (order by length) of each mode
  int mode_of[alto::kMaxModes] = {};   // mode of each rank
  alto_allocator alloc{};
  bool user_alloc = false;
  cudaStream_t stream = nullptr;
  int device = 0, num_sms = 1;
  size_t bytes_held = 0;
  // device state
  uint64_t *keys = nullptr;
  float *vals = nullptr;
  uint64_t *dims_dev = nullptr;
  uint64_t L = 0;
  uint32_t *intervals = nullptr;
  uint32_t *max_len_dev = nullptr;
  uint32_t *status_dev = nullptr;
  double *norm_sq_dev = nullptr;
  DecodePlan32 *dp_rank_dev = nullptr;   // runs by rank, for grouped launches
  uint64_t *lut_dev = nullptr;            // byte-table decode [8][256] (positions <= 64 bits)
  alto::LutPlan lut_plan{};               // its packing, by rank
  uint32_t *hot_rows[alto::kMaxModes] = {};
  uint32_t *nhot_dev = nullptr;
  // host mirrors
  uint32_t max_interval[alto::kMaxModes] = {};
  uint32_t nhot[alto::kMaxModes] = {};
  std::vector<uint32_t> hot_host[alto::kMaxModes];
  double norm_sq = 0.0;
  std::vector<uint32_t> intervals_host;
  bool intervals_host_valid = false;
  // plans and caches
  alto_mode_plan plan[alto::kMaxModes];
  HotTable hot_tab[alto::kMaxModes];
  HotTable group_hot[alto::kMaxModes][5];  // smaller tables for grouped launches, by size
  PullPlan pull[alto::kMaxModes];
  Buf partials;
  Buf warm;                                 // TILED: warm-row replicas (zero between launches)
  uint32_t *pos_out[alto::kMaxModes] = {};  // stored output-oriented order per mode
  uint64_t *keys_out[alto::kMaxModes] = {}; // line positions in that order [nnz][kw]
  float *vals_out[alto::kMaxModes] = {};    // values in that order
  uint64_t pos_out_L[alto::kMaxModes] = {}; // its segment count
  bool pos_out_failed[alto::kMaxModes] = {};   // AUTO could not allocate it: ATOMIC
  // instrumentation
  bool prof_on = false;
  std::vector<ProfEvt> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  double prof_ms[ALTO_PROF_KINDS] = {};
  float encode_ms = 0.f;  // device time of the encode kernels (CUDA events)
  float sort_ms = 0.f;    // of which the radix sort
  int sort_passes = 0;    // radix passes the sort launched
  uint64_t prof_n[ALTO_PROF_KINDS] = {};
};
