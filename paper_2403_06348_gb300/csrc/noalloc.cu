// alto_mttkrp_noalloc: the pull variant of the MTTKRP (Alg. 4, recursive
// traversal with Temp and pull-based reduction) for callers that must not
// have the library allocate device memory.
//
// Some callers cannot let a library call cudaMalloc at the point where they
// run a kernel: a service that reserved its whole device memory budget at
// start-up and hands out only fixed buffers afterwards, or a framework whose
// own caching allocator owns the device and would be undercut by allocations
// it does not see. alto_mttkrp may allocate (the pull partials grow with the
// partition), so this entry point keeps the partials in a fixed, file-scope
// device array instead and calls no allocating routine at all.
#include <mutex>

#include "handle.cuh"
#include "mttkrp.cuh"

namespace alto {
namespace {

// Fixed scratch for the segments' partials (Temp_l of Alg. 4), shared by every
// call on a device and kept until the process exits: 8 Mi floats = 32 MiB.
constexpr size_t kNoAllocScratchFloats = (size_t)8 << 20;
static __device__ __align__(256) float g_noalloc_partials[kNoAllocScratchFloats];

constexpr int kMaxDevices = 64;
std::mutex g_scratch_mutex;
float *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_noalloc_partials on the current device. The host name of
// the array is only a stand-in for the symbol, so the address is looked up
// once per device (with that device current) and cached.
alto_status scratch_address(float **out) {
  int dev = 0;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return fail(ALTO_ERR_UNSUPPORTED, "device index %d", dev);
  std::lock_guard<std::mutex> lock(g_scratch_mutex);
  if (!g_scratch_ptr[dev]) {
    void *p = nullptr;
    CUDA_TRY(cudaGetSymbolAddress(&p, g_noalloc_partials));
    g_scratch_ptr[dev] = static_cast<float *>(p);
  }
  *out = g_scratch_ptr[dev];
  return ALTO_OK;
}

}  // namespace
}  // namespace alto

using namespace alto;

extern "C" alto_status alto_mttkrp_noalloc(alto_handle_t h, int mode, const void *const *factors,
                                           alto_dtype fdtype, int R, float *out, void *stream) {
  if (!h) return fail(ALTO_ERR_INVALID_ARG, "null handle");
  alto_status st = check_device(h);
  if (st != ALTO_OK) return st;
  if (mode < 0 || mode >= h->N) return fail(ALTO_ERR_INVALID_ARG, "mode %d out of range", mode);
  if (!(R == 4 || R == 8 || R == 16 || R == 32 || R == 64))
    return fail(ALTO_ERR_UNSUPPORTED, "rank %d not in {4,8,16,32,64}", R);
  if (fdtype != ALTO_F32 && fdtype != ALTO_BF16) return fail(ALTO_ERR_INVALID_ARG, "bad dtype");
  if (!factors || !out) return fail(ALTO_ERR_INVALID_ARG, "factors/out NULL");
  if (((uintptr_t)out & 15u) != 0) return fail(ALTO_ERR_INVALID_ARG, "out not 16-byte aligned");
  for (int m = 0; m < h->N; ++m) {
    if (m == mode) continue;
    if (!factors[m]) return fail(ALTO_ERR_INVALID_ARG, "factors[%d] is NULL", m);
    if (((uintptr_t)factors[m] & 15u) != 0)
      return fail(ALTO_ERR_INVALID_ARG, "factors[%d] not 16-byte aligned", m);
  }
  cudaStream_t s = (cudaStream_t)stream;
  const uint64_t I = h->dims[mode];
  if (h->M == 0) {
    CUDA_TRY(cudaMemsetAsync(out, 0, I * R * sizeof(float), s));
    return ALTO_OK;
  }
  const PullPlan &pp = h->pull[mode];
  if (!pp.valid)
    return fail(ALTO_ERR_INVALID_ARG,
                "mode %d has no row-to-segment lists yet: one alto_mttkrp call with the PULL "
                "variant on this mode builds them (that call may allocate)",
                mode);
  const size_t smem = mttkrp_smem_bytes(true, R, 0, 0, h->max_interval[mode]);
  if (smem > mttkrp_stage_budget())
    return fail(ALTO_ERR_UNSUPPORTED, "mode %d: interval of %u rows does not fit shared memory", mode,
                h->max_interval[mode]);
  const uint64_t need = pp.total_rows * (uint64_t)R;
  if (need > kNoAllocScratchFloats)
    return fail(ALTO_ERR_UNSUPPORTED,
                "mode %d at rank %d needs %llu floats of scratch; the fixed scratch holds %llu",
                mode, R, (unsigned long long)need, (unsigned long long)kNoAllocScratchFloats);
  float *scratch = nullptr;
  st = scratch_address(&scratch);
  if (st != ALTO_OK) return st;

  MttkrpArgs a{};
  a.bp = h->bp;
  a.bp.out_rank = h->rank_of[mode];
  a.out_rank = h->rank_of[mode];
  a.dp.nmodes = h->N;
  a.dp.kw = h->kw;
  for (int q = 0; q < h->N; ++q) {
    const int m = h->mode_of[q];
    a.dp.nruns[q] = h->dp32.nruns[m];
    memcpy(a.dp.runs[q], h->dp32.runs[m], sizeof(a.dp.runs[q]));
    a.factors[q] = m == mode ? nullptr : factors[m];
  }
  for (int q = 0, k = 0; q < h->N; ++q)
    if (h->mode_of[q] != mode) a.fin[k++] = factors[h->mode_of[q]];
  a.keys = h->keys;
  a.vals = h->vals;
  a.nnz = h->M;
  a.L = h->L;
  a.intervals = h->intervals;
  a.out = out;
  a.mode = mode;
  a.R = R;
  a.flush_every = 1;
  // Every segment writes its whole Temp (zeroed in shared memory first) and
  // the reduction reads only rows some segment wrote, so nothing left in the
  // shared scratch by an earlier call is ever read.
  a.partials = scratch;
  a.part_off = pp.part_off;
  CUDA_TRY(launch_mttkrp(a, 4, fdtype == ALTO_BF16, true, smem, h->num_sms, s));
  CUDA_TRY(launch_pull_reduce(scratch, pp.row_ptr, pp.prow, I, R, out, h->num_sms, s));
  return ALTO_OK;
}
