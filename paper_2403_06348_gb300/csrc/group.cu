// Grouped MTTKRP (Alg. 3 with the conflict resolution of Alg. 4) over many
// encoded tensors in one persistent launch.
//
// The units of work are the line segments of every problem (Section IV-A: each
// segment holds the same number of nonzeros of its tensor). CTAs take units in
// turn from a global counter, so problems of very different size share the
// GPU without a launch each. Inside a unit the kernel runs the same batch and
// round structure as the single-tensor kernel (one warp decodes 32 ordered
// nonzeros, groups of R/4 lanes gather, multiply and merge runs of equal
// output row); rank, number of modes and key width are read per unit.
// Conflict resolution per unit: when the segment's interval of the output mode
// fits shared memory, its Temp is staged there and flushed once with vector
// atomics (rows stay in shared memory for the whole segment, as in Alg. 4);
// otherwise runs go straight to the output with vector atomics.
#include <cstring>
#include <vector>

#include "group.cuh"
#include "handle.cuh"
#include "mttkrp_kernel.cuh"

namespace alto {

namespace {

// Everything one unit needs, filled by thread 0 and read from shared memory.
struct GroupUnit {
  BlockPlan bp;
  const uint64_t *keys;
  const float *vals;
  float *out;
  const void *fin[kMaxModes];  // input factors: ranks in order without the output rank
  const uint64_t *htab;        // hot rows of the output mode (global)
  const uint32_t *slot_rows;
  uint64_t s0, s1;
  uint32_t Ts, len;
  int p, N, kw, R, ro, staged, active, hbits, nslots;
};

constexpr size_t kGroupStaticReserve = 8192;  // GroupUnit + DecodePlan32 + scalars

// Two CTAs of 512 threads per SM: the per-unit state (pointers, bounds, the
// staging mode) needs more registers than the single-tensor kernel's 40.
constexpr int kGroupThreads = 512;
constexpr int kGroupBlocksPerSm = 2;

}  // namespace

size_t group_stage_bytes() {
  static int per_sm = 0;
  if (!per_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  }
  size_t b = (size_t)per_sm / kGroupBlocksPerSm - 2048 - kGroupStaticReserve;
  return b < mttkrp_smem_limit() - kGroupStaticReserve ? b : mttkrp_smem_limit() - kGroupStaticReserve;
}

template <int NT, int KW, bool BF16>
__device__ __noinline__ void group_segment(const GroupUnit &g, const DecodePlan32 &dp,
                                              float *temp, const uint64_t *shtab) {
  constexpr int NMAX = NT ? NT : kMaxModes;
  constexpr int NIN = NMAX > 1 ? NMAX - 1 : 1;
  constexpr int CPL = 4;
  const int N = NT ? NT : g.N;
  const int R = g.R;
  const int tpn = R / CPL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int grp = lane / tpn, sub = lane - grp * tpn;
  const int ro = g.ro;
  const uint32_t rowb = (uint32_t)R * (BF16 ? 2u : 4u);
  const uint32_t inb = lane_byte_offset<CPL, BF16>(sub);
  const char *fb[NIN];
#pragma unroll
  for (int k = 0; k < NIN; ++k)
    fb[k] = k + 1 < N ? static_cast<const char *>(g.fin[k]) + inb : nullptr;
  const uint64_t s0 = g.s0, s1 = g.s1;
  const uint64_t *keys = g.keys;
  const float *vals = g.vals;
  float *out = g.out;
  const bool staged = g.staged != 0;
  const bool hot = !staged && g.nslots > 0;
  const int hbits = g.hbits;
  const uint32_t Ts = g.Ts;

  uint64_t nlo = 0, nhi = 0;
  float nv = 0.f;
  auto fetch = [&](uint64_t xx) {
    if (xx < s1) {
      if (KW == 1) {
        nlo = __ldcs(reinterpret_cast<const unsigned long long *>(keys) + xx);
      } else {
        const ulonglong2 kk = __ldcs(reinterpret_cast<const ulonglong2 *>(keys) + xx);
        nlo = kk.x;
        nhi = kk.y;
      }
      nv = __ldcs(vals + xx);
    }
  };
  fetch(s0 + (uint64_t)warp * 32 + lane);
  for (uint64_t base = s0 + (uint64_t)warp * 32; base < s1; base += (uint64_t)nwarps * 32) {
    const uint64_t x = base + lane;
    const bool valid = x < s1;
    const uint64_t lo = nlo, hi = nhi;
    const float v = valid ? nv : 0.f;
    fetch(x + (uint64_t)nwarps * 32);
    uint32_t c[NMAX];
    if constexpr (NT > 0)
      decode_blocks<KW, NMAX, 0>(g.bp, lo, hi, c);
    else
      decode_runs<KW, NMAX>(dp, N, lo, hi, c);
    uint32_t row = c[0];
    uint32_t in[NIN];
#pragma unroll
    for (int n = 1; n < NMAX; ++n)
      if (n == ro) row = c[n];
#pragma unroll
    for (int k = 0; k < NIN; ++k) in[k] = (NMAX > 1 && k + 1 < NMAX) ? (k < ro ? c[k] : c[k + 1]) : 0u;
    int slot = -1;
    if (valid) slot = staged ? (int)(row - Ts) : (hot ? hot_lookup(shtab, hbits, row) : -1);
    const uint64_t rem = s1 - base;
    // many small tensors stage heavily shared rows: rotate the flush order per
    // group so groups on the same row add to different columns
    if (rem >= 32)
      group_rounds<NMAX, CPL, BF16, false, kAprOff, true>(fb, out, R, N, tpn, grp, sub, v, slot, row,
                                                          in, 32, temp, rowb);
    else
      group_rounds<NMAX, CPL, BF16, true, kAprOff, true>(fb, out, R, N, tpn, grp, sub, v, slot, row,
                                                         in, (int)rem, temp, rowb);
  }
}

template <bool BF16>
__global__ void __launch_bounds__(kGroupThreads, kGroupBlocksPerSm)
    group_mttkrp_kernel(const GroupProb *__restrict__ probs, const uint64_t *__restrict__ unit_off,
                        const uint32_t *__restrict__ unit_prob, const int *__restrict__ nprobs,
                        unsigned *ctr, uint32_t stage_bytes) {
  extern __shared__ __align__(16) unsigned char sm[];
  float *temp = reinterpret_cast<float *>(sm);
  __shared__ GroupUnit g;
  __shared__ DecodePlan32 sdp;
  __shared__ int dp_of;
  __shared__ unsigned unit;
  const int P = *nprobs;
  const uint64_t U = P > 0 ? unit_off[P] : 0;
  if (threadIdx.x == 0) dp_of = -1;
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) unit = atomicAdd(&ctr[0], 1u);
    __syncthreads();
    const uint64_t u = unit;
    if (u >= U) break;
    if (threadIdx.x == 0) {
      const int p = (int)unit_prob[u];
      const GroupProb &q = probs[p];
      const int mode = q.cur_mode ? *q.cur_mode : q.mode;
      const bool stopped = q.done ? (*q.done != 0) : false;
      const uint64_t l = u - unit_off[p];
      const uint64_t nnz = q.nnz, L = q.L;
      g.p = p;
      g.s0 = (l * nnz) / L;
      g.s1 = ((l + 1) * nnz) / L;
      g.active = (!stopped && g.s1 > g.s0) ? 1 : 0;
      const int N = q.N, ro = q.rank_of[mode], R = q.R;
      g.N = N;
      g.kw = q.kw;
      g.R = R;
      g.ro = ro;
      g.keys = q.keys;
      g.vals = q.vals;
      g.out = q.out;
      for (int k = 0; k + 1 < N; ++k) g.fin[k] = q.fac[k < ro ? k : k + 1];
      g.bp = q.bp;
      uint32_t Ts = 0, len = 0;
      if (g.active) {
        Ts = q.intervals[(l * (uint64_t)N + mode) * 2];
        len = q.intervals[(l * (uint64_t)N + mode) * 2 + 1] - Ts + 1u;
      }
      g.Ts = Ts;
      g.len = len;
      g.staged = (g.active && (uint64_t)len * (uint64_t)R * 4u <= stage_bytes) ? 1 : 0;
      g.nslots = g.staged ? 0 : q.nslots[mode];
      g.hbits = q.hbits[mode];
      g.htab = q.htab[mode];
      g.slot_rows = q.slot_rows[mode];
    }
    __syncthreads();
    if (!g.active) continue;
    const int N = g.N;
    if ((N < 3 || N > 5) && dp_of != g.p) {
      const uint32_t *src = reinterpret_cast<const uint32_t *>(probs[g.p].dp);
      uint32_t *dst = reinterpret_cast<uint32_t *>(&sdp);
      for (int i = threadIdx.x; i < (int)(sizeof(DecodePlan32) / 4); i += blockDim.x) dst[i] = src[i];
      __syncthreads();
      if (threadIdx.x == 0) dp_of = g.p;
    }
    const int R = g.R;
    uint64_t *shtab = reinterpret_cast<uint64_t *>(temp + (size_t)g.nslots * R);
    if (g.staged) {
      for (uint32_t i = threadIdx.x; i < g.len * (uint32_t)R; i += blockDim.x) temp[i] = 0.f;
      __syncthreads();
    } else if (g.nslots > 0) {
      const int hsize = 1 << g.hbits;
      for (int i = threadIdx.x; i < hsize; i += blockDim.x) shtab[i] = g.htab[i];
      for (int i = threadIdx.x; i < g.nslots * R; i += blockDim.x) temp[i] = 0.f;
      __syncthreads();
    }
    const bool k2 = g.kw == 2;
    switch (N) {
      case 3:
        k2 ? group_segment<3, 2, BF16>(g, sdp, temp, shtab) : group_segment<3, 1, BF16>(g, sdp, temp, shtab);
        break;
      case 4:
        k2 ? group_segment<4, 2, BF16>(g, sdp, temp, shtab) : group_segment<4, 1, BF16>(g, sdp, temp, shtab);
        break;
      case 5:
        k2 ? group_segment<5, 2, BF16>(g, sdp, temp, shtab) : group_segment<5, 1, BF16>(g, sdp, temp, shtab);
        break;
      default:
        k2 ? group_segment<0, 2, BF16>(g, sdp, temp, shtab) : group_segment<0, 1, BF16>(g, sdp, temp, shtab);
        break;
    }
    if (!g.staged && g.nslots > 0) {
      __syncthreads();
      const float4 *t4 = reinterpret_cast<const float4 *>(temp);
      const int per_row = R / 4;
      const int n4 = g.nslots * per_row;
      float *out = g.out;
      const uint32_t *rows = g.slot_rows;
      for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        const float4 t = t4[i];
        if (t.x != 0.f || t.y != 0.f || t.z != 0.f || t.w != 0.f) {
          const int sl = i / per_row;
          const int c4 = ((i - sl * per_row) * 4) ^ slot_swizzle(sl, R);
          red_v4(out + (uint64_t)rows[sl] * (uint64_t)R + c4, t.x, t.y, t.z, t.w);
        }
      }
    }
    if (g.staged) {
      __syncthreads();
      const float4 *t4 = reinterpret_cast<const float4 *>(temp);
      const uint32_t per_row = (uint32_t)R / 4;
      const uint32_t n4 = g.len * per_row;
      float *out = g.out;
      const uint32_t Ts = g.Ts;
      for (uint32_t i = threadIdx.x; i < n4; i += blockDim.x) {
        const float4 t = t4[i];
        if (t.x != 0.f || t.y != 0.f || t.z != 0.f || t.w != 0.f) {
          const uint32_t row = i / per_row;
          const int c4 = (int)((i - row * per_row) * 4) ^ slot_swizzle((int)row, R);
          red_v4(out + (uint64_t)(Ts + row) * (uint64_t)R + c4, t.x, t.y, t.z, t.w);
        }
      }
    }
  }
  // The counter goes back to zero for the next launch once every CTA has
  // drawn past the last unit.
  if (threadIdx.x == 0) {
    const unsigned finished = atomicAdd(&ctr[1], 1u);
    if (finished == gridDim.x - 1) {
      atomicExch(&ctr[0], 0u);
      atomicExch(&ctr[1], 0u);
    }
  }
}

cudaError_t configure_group_mttkrp() {
  static int configured = 0;
  if (configured) return cudaSuccess;
  const int smem = (int)group_stage_bytes();
  cudaError_t e = cudaFuncSetAttribute(group_mttkrp_kernel<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess)
    e = cudaFuncSetAttribute(group_mttkrp_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e == cudaSuccess) configured = 1;
  return e;
}

cudaError_t launch_group_mttkrp(const GroupProb *probs, const uint64_t *unit_off,
                                const uint32_t *unit_prob, const int *nprobs, unsigned *ctr, bool bf16,
                                int num_sms, cudaStream_t s) {
  auto kern = bf16 ? group_mttkrp_kernel<true> : group_mttkrp_kernel<false>;
  const size_t smem = group_stage_bytes();
  cudaError_t e = configure_group_mttkrp();
  if (e != cudaSuccess) return e;
  kern<<<(unsigned)(num_sms * kGroupBlocksPerSm), kGroupThreads, smem, s>>>(probs, unit_off, unit_prob, nprobs, ctr,
                                                       (uint32_t)smem);
  note_launches(1);
  return cudaGetLastError();
}

// The rank-ordered runs of a handle, kept on the device for grouped launches.
alto_status ensure_rank_runs(alto_tensor *h, cudaStream_t s) {
  if (h->dp_rank_dev) return ALTO_OK;
  DecodePlan32 d{};
  d.nmodes = h->N;
  d.kw = h->kw;
  for (int q = 0; q < h->N; ++q) {
    const int m = h->mode_of[q];
    d.nruns[q] = h->dp32.nruns[m];
    memcpy(d.runs[q], h->dp32.runs[m], sizeof(d.runs[q]));
  }
  void *p = dalloc(h, sizeof(DecodePlan32), s);
  if (!p) return fail(ALTO_ERR_OOM, "decode runs (%zu bytes)", sizeof(DecodePlan32));
  h->dp_rank_dev = static_cast<DecodePlan32 *>(p);
  CUDA_TRY(cudaMemcpyAsync(p, &d, sizeof(d), cudaMemcpyHostToDevice, s));
  return ALTO_OK;
}

alto_status fill_group_prob(alto_tensor *h, int R, GroupProb *q, cudaStream_t s) {
  *q = GroupProb{};
  q->bp = h->bp;
  q->dp = h->dp_rank_dev;
  q->keys = h->keys;
  q->vals = h->vals;
  q->nnz = h->M;
  q->L = h->L;
  q->intervals = h->intervals;
  q->N = h->N;
  q->kw = h->kw;
  q->R = R;
  const size_t budget = group_stage_bytes();
  for (int m = 0; m < h->N; ++m) {
    q->dims[m] = h->dims[m];
    q->max_interval[m] = h->max_interval[m];
    q->rank_of[m] = h->rank_of[m];
    // modes whose every segment is staged need no hot rows
    if ((uint64_t)h->max_interval[m] * R * 4u <= budget || h->nhot[m] == 0) continue;
    int k = (int)h->nhot[m];
    int hbits = 1;
    for (;;) {
      hbits = 1;
      while ((1 << hbits) < 2 * k) ++hbits;
      if (k == 0 || (size_t)k * R * 4 + ((size_t)1 << hbits) * 8 <= budget) break;
      k = k * 7 / 8;
    }
    if (k == 0) continue;
    const HotTable *t = nullptr;
    alto_status st = ensure_group_hot(h, m, k, s, &t);
    if (st != ALTO_OK) return st;
    q->htab[m] = t->htab;
    q->slot_rows[m] = h->hot_rows[m];
    q->hbits[m] = t->hbits;
    q->nslots[m] = t->nslots;
  }
  return ALTO_OK;
}

}  // namespace alto

using namespace alto;

extern "C" alto_status alto_mttkrp_grouped(int n, const alto_handle_t *hs, const int *modes,
                                           const void *const *const *factors, const int *Rs,
                                           alto_dtype fdtype, float *const *outs, void *stream) {
  if (n < 0) return fail(ALTO_ERR_INVALID_ARG, "n = %d", n);
  if (n == 0) return ALTO_OK;
  if (!hs || !modes || !factors || !Rs || !outs) return fail(ALTO_ERR_INVALID_ARG, "NULL array");
  if (fdtype != ALTO_F32 && fdtype != ALTO_BF16) return fail(ALTO_ERR_INVALID_ARG, "bad dtype");
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<GroupProb> probs(n);
  std::vector<uint64_t> unit_off(n + 1, 0);
  int num_sms = 1;
  for (int i = 0; i < n; ++i) {
    alto_tensor *h = hs[i];
    if (!h) return fail(ALTO_ERR_INVALID_ARG, "problem %d: null handle", i);
    if (check_device(h) != ALTO_OK)
      return fail(ALTO_ERR_INVALID_ARG, "problem %d: handle encoded on device %d, not the current one", i,
                  h->device);
    const int mode = modes[i], R = Rs[i];
    if (mode < 0 || mode >= h->N) return fail(ALTO_ERR_INVALID_ARG, "problem %d: mode %d", i, mode);
    if (!(R == 4 || R == 8 || R == 16 || R == 32 || R == 64))
      return fail(ALTO_ERR_UNSUPPORTED, "problem %d: rank %d not in {4,8,16,32,64}", i, R);
    if (!factors[i] || !outs[i]) return fail(ALTO_ERR_INVALID_ARG, "problem %d: NULL factors/out", i);
    if (((uintptr_t)outs[i] & 15u) != 0)
      return fail(ALTO_ERR_INVALID_ARG, "problem %d: out not 16-byte aligned", i);
    for (int m = 0; m < h->N; ++m) {
      if (m == mode) continue;
      if (!factors[i][m]) return fail(ALTO_ERR_INVALID_ARG, "problem %d: factors[%d] NULL", i, m);
      if (((uintptr_t)factors[i][m] & 15u) != 0)
        return fail(ALTO_ERR_INVALID_ARG, "problem %d: factors[%d] not 16-byte aligned", i, m);
    }
    num_sms = h->num_sms;
    alto_status st = ensure_rank_runs(h, s);
    if (st != ALTO_OK) return st;
    st = fill_group_prob(h, R, &probs[i], s);
    if (st != ALTO_OK) return st;
    probs[i].mode = mode;
    probs[i].out = outs[i];
    for (int q = 0; q < h->N; ++q) {
      const int m = h->mode_of[q];
      probs[i].fac[q] = m == mode ? nullptr : factors[i][m];
    }
    unit_off[i + 1] = unit_off[i] + (h->M ? h->L : 0);
  }
  const uint64_t U = unit_off[n];
  if (U > 0xFFFFFFF0ull) return fail(ALTO_ERR_UNSUPPORTED, "%llu segments in one launch", (unsigned long long)U);
  std::vector<uint32_t> unit_prob(U);
  for (int i = 0; i < n; ++i)
    for (uint64_t u = unit_off[i]; u < unit_off[i + 1]; ++u) unit_prob[u] = (uint32_t)i;
  // one temporary block: probs | unit_off | unit_prob | nprobs + counters
  const size_t o_probs = 0;
  const size_t o_off = (o_probs + n * sizeof(GroupProb) + 255) & ~(size_t)255;
  const size_t o_prob = (o_off + (n + 1) * sizeof(uint64_t) + 255) & ~(size_t)255;
  const size_t o_int = (o_prob + U * sizeof(uint32_t) + 255) & ~(size_t)255;
  const size_t bytes = o_int + 16;
  char *ws = nullptr;
  CUDA_TRY(cudaMallocAsync(reinterpret_cast<void **>(&ws), bytes, s));
  const int header[4] = {n, 0, 0, 0};
  cudaError_t e = cudaMemcpyAsync(ws + o_probs, probs.data(), n * sizeof(GroupProb),
                                  cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(ws + o_off, unit_off.data(), (n + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && U)
    e = cudaMemcpyAsync(ws + o_prob, unit_prob.data(), U * sizeof(uint32_t), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(ws + o_int, header, sizeof(header), cudaMemcpyHostToDevice, s);
  for (int i = 0; i < n && e == cudaSuccess; ++i) {
    const alto_tensor *h = hs[i];
    e = cudaMemsetAsync(outs[i], 0, h->dims[modes[i]] * (size_t)Rs[i] * sizeof(float), s);
  }
  if (e == cudaSuccess && U)
    e = launch_group_mttkrp(reinterpret_cast<const GroupProb *>(ws + o_probs),
                            reinterpret_cast<const uint64_t *>(ws + o_off),
                            reinterpret_cast<const uint32_t *>(ws + o_prob),
                            reinterpret_cast<const int *>(ws + o_int),
                            reinterpret_cast<unsigned *>(ws + o_int + 4), fdtype == ALTO_BF16, num_sms, s);
  cudaFreeAsync(ws, s);
  if (e != cudaSuccess) return fail(ALTO_ERR_CUDA, "grouped MTTKRP: %s", cudaGetErrorString(e));
  return ALTO_OK;
}
