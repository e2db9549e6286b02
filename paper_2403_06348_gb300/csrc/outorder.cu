// The stored output-oriented order pos_out of Alg. 4 and the dispatch of its
// MTTKRP kernel by number of modes (kernels in outorder.cuh, out_n*.cu).
//
// pos_out of a mode is the per-segment stable sort of positions by the mode's
// coordinate. Segments of at most kPosOutSegCap nonzeros (the default count
// of the stored order guarantees it) are sorted one per CTA in shared memory; otherwise the whole line goes through one
// stable LSD radix sort whose key of ordered position x is (segment of x,
// coordinate) and whose sorted values are the positions: segments are
// contiguous and the sort is stable, so the result is the same.
#include "encode.cuh"
#include "handle.cuh"
#include "mttkrp.cuh"

namespace alto {

// The 32-bit runs of one mode (EXTRACT of Alg. 3 for that mode only).
struct ModeRuns32 {
  int nruns;
  Run32 runs[kMaxRuns32];
};

template <int KW>
__device__ __forceinline__ uint32_t decode_mode(const ModeRuns32 &mr, uint64_t lo, uint64_t hi) {
  uint32_t v = 0;
#pragma unroll
  for (int r = 0; r < kMaxRuns32; ++r) {
    if (r < mr.nruns) {
      const Run32 &br = mr.runs[r];
      uint32_t x = window32<KW>(lo, hi, br.start) & br.mask[0];
#pragma unroll
      for (int j = 0; j < 5; ++j)
        if (j < br.steps) x = (x | (x >> br.sh[j])) & br.mask[j + 1];
      v |= x << br.outshift;
    }
  }
  return v;
}

static ModeRuns32 mode_runs(const alto_tensor *h, int mode) {
  ModeRuns32 mr{};
  mr.nruns = h->dp32.nruns[mode];
  for (int r = 0; r < mr.nruns; ++r) mr.runs[r] = h->dp32.runs[mode][r];
  return mr;
}

// key[x] = l(x) << bits | i_mode(x), pos[x] = x, where l(x) is the segment
// [floor(l M / L), floor((l + 1) M / L)) holding x: l(x) = floor(((x + 1) L - 1) / M).
template <int KW>
__global__ void __launch_bounds__(256) pos_key_kernel(const __grid_constant__ ModeRuns32 mr,
                                                      const uint64_t *__restrict__ keys, uint64_t nnz,
                                                      uint64_t L, int bits, uint64_t *__restrict__ ck,
                                                      uint32_t *__restrict__ pos) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nnz;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t i = decode_mode<KW>(mr, keys[x * KW], KW == 2 ? keys[x * KW + 1] : 0ull);
    const uint64_t l = ((x + 1) * L - 1) / nnz;
    ck[x] = (l << bits) | i;
    pos[x] = (uint32_t)x;
  }
}

// Segments of at most kSegCap nonzeros are sorted inside one CTA each: the
// segment's (coordinate - segment minimum, local index) pairs sit in shared
// memory and go through a stable LSD radix sort with 8-bit digits, as many
// passes as the segment's coordinate range needs. Per pass, warp w ranks the
// items of its contiguous share by digit (match_any; one writer per digit and
// warp), a scan over the digit-major (digit, warp) count table gives every
// warp's first slot per digit, and a second walk scatters the items.
constexpr int kSegThreads = 512;
constexpr int kSegWarps = kSegThreads / 32;
constexpr uint32_t kSegCap = kPosOutSegCap;  // two sorting CTAs fit one SM
constexpr size_t kSegSmem = (size_t)kSegCap * (4 + 2) * 2 + (size_t)256 * kSegWarps * 4;

__device__ __forceinline__ unsigned seg_lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <int KW>
__global__ void __launch_bounds__(kSegThreads) pos_seg_kernel(const __grid_constant__ ModeRuns32 mr,
                                                              const uint64_t *__restrict__ keys,
                                                              const float *__restrict__ vals,
                                                              uint64_t nnz, uint64_t L,
                                                              uint32_t *__restrict__ pos_out,
                                                              uint64_t *__restrict__ keys_out,
                                                              float *__restrict__ vals_out) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint32_t *ka = reinterpret_cast<uint32_t *>(sm);
  uint32_t *kb = ka + kSegCap;
  uint16_t *ia = reinterpret_cast<uint16_t *>(kb + kSegCap);
  uint16_t *ib = ia + kSegCap;
  uint32_t *wc = reinterpret_cast<uint32_t *>(ib + kSegCap);  // [256][kSegWarps]
  __shared__ uint32_t red[2][kSegWarps];
  __shared__ uint32_t part[kSegThreads / 32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const unsigned full = 0xffffffffu;
  for (uint64_t l = blockIdx.x; l < L; l += gridDim.x) {
    const uint64_t s0 = l * nnz / L, s1 = (l + 1) * nnz / L;
    const uint32_t S = (uint32_t)(s1 - s0);
    uint32_t mn = 0xFFFFFFFFu, mx = 0;
#pragma unroll 8
    for (uint32_t j = threadIdx.x; j < S; j += kSegThreads) {
      const uint64_t x = s0 + j;
      const uint32_t i = decode_mode<KW>(mr, keys[x * KW], KW == 2 ? keys[x * KW + 1] : 0ull);
      ka[j] = i;
      ia[j] = (uint16_t)j;
      mn = min(mn, i);
      mx = max(mx, i);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      mn = min(mn, __shfl_xor_sync(full, mn, o));
      mx = max(mx, __shfl_xor_sync(full, mx, o));
    }
    if (lane == 0) {
      red[0][warp] = mn;
      red[1][warp] = mx;
    }
    __syncthreads();
    mn = 0xFFFFFFFFu;
    mx = 0;
    for (int w = 0; w < kSegWarps; ++w) {
      mn = min(mn, red[0][w]);
      mx = max(mx, red[1][w]);
    }
    const uint32_t range = S ? mx - mn : 0u;
    const int passes = (32 - __clz(range) + 7) / 8;  // __clz(0) = 32: no pass
    // warp w's share [w * per, min(S, (w + 1) * per)), walked in rounds of 32
    const uint32_t per = (S + kSegWarps - 1) / kSegWarps;
    const uint32_t w0 = min(S, warp * per), w1 = min(S, w0 + per);
    for (int p = 0; p < passes; ++p) {
      const int shift = 8 * p;
      for (int i = threadIdx.x; i < 256 * kSegWarps; i += kSegThreads) wc[i] = 0;
      __syncthreads();
      for (uint32_t base = w0; base < w1; base += 32) {
        const uint32_t j = base + lane;
        const uint32_t d = j < w1 ? ((ka[j] - mn) >> shift) & 0xFFu : 256u;
        const unsigned peers = __match_any_sync(full, d);
        if (d < 256u && (peers & seg_lanemask_lt()) == 0) wc[d * kSegWarps + warp] += __popc(peers);
        __syncwarp();
      }
      __syncthreads();
      {
        // exclusive scan of the 256 x kSegWarps table, digit-major: thread t
        // owns entries [8t, 8t + 8)
        constexpr int kPer = 256 * kSegWarps / kSegThreads;
        uint32_t v[kPer], sum = 0;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          v[k] = wc[threadIdx.x * kPer + k];
          sum += v[k];
        }
        uint32_t inc = sum;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
          const uint32_t y = __shfl_up_sync(full, inc, o);
          if (lane >= o) inc += y;
        }
        if (lane == 31) part[warp] = inc;
        __syncthreads();
        uint32_t before = 0;
        for (int w = 0; w < warp; ++w) before += part[w];
        uint32_t run = before + inc - sum;
#pragma unroll
        for (int k = 0; k < kPer; ++k) {
          wc[threadIdx.x * kPer + k] = run;
          run += v[k];
        }
      }
      __syncthreads();
      for (uint32_t base = w0; base < w1; base += 32) {
        const uint32_t j = base + lane;
        const bool ok = j < w1;
        const uint32_t key = ok ? ka[j] : 0u;
        const uint32_t d = ok ? ((key - mn) >> shift) & 0xFFu : 256u;
        const unsigned peers = __match_any_sync(full, d);
        uint32_t slot = 0;
        if (ok) slot = wc[d * kSegWarps + warp] + __popc(peers & seg_lanemask_lt());
        __syncwarp();
        if (ok && (peers & seg_lanemask_lt()) == 0) wc[d * kSegWarps + warp] += __popc(peers);
        if (ok) {
          kb[slot] = key;
          ib[slot] = ia[j];
        }
        __syncwarp();
      }
      __syncthreads();
      uint32_t *tk = ka;
      ka = kb;
      kb = tk;
      uint16_t *ti = ia;
      ia = ib;
      ib = ti;
    }
    // the order, and the segment's line positions and values in it (the
    // segment was just read: its keys come from L2)
#pragma unroll 4
    for (uint32_t j = threadIdx.x; j < S; j += kSegThreads) {
      const uint64_t x = s0 + ia[j];
      pos_out[s0 + j] = (uint32_t)x;
#pragma unroll
      for (int w = 0; w < KW; ++w) keys_out[(s0 + j) * KW + w] = keys[x * KW + w];
      vals_out[s0 + j] = vals[x];
    }
    __syncthreads();
  }
}

static int bit_width_u64(uint64_t v) {
  int b = 0;
  while (v) {
    ++b;
    v >>= 1;
  }
  return b;
}

alto_status build_pos_out(alto_tensor *h, int mode, uint64_t L, uint32_t **out, uint64_t *keys_out,
                          float *vals_out, cudaStream_t s) {
  *out = nullptr;
  const uint64_t M = h->M;
  if (M > kPosOutMaxNnz)
    return fail(ALTO_ERR_UNSUPPORTED, "pos_out holds 32-bit positions: nnz %llu too large",
                (unsigned long long)M);
  if (L < 1 || L > M) L = M ? std::min<uint64_t>(std::max<uint64_t>(L, 1), M) : 1;
  const int bits = h->bits[mode];
  const int nbits = bit_width_u64(L - 1) + bits;  // <= 32 + 32
  uint64_t *kbuf[2] = {nullptr, nullptr};
  float *vbuf[2] = {nullptr, nullptr};
  uint32_t *pos = nullptr;
  void *sort_work = nullptr;
  const size_t sort_bytes = sort_workspace_bytes(M);
  auto release = [&](int keep) {
    for (int b = 0; b < 2; ++b) {
      dfree(h, kbuf[b], M * 8, s);
      if (b != keep) dfree(h, vbuf[b], M * 4, s);
    }
    dfree(h, pos, M * 4, s);
    dfree(h, sort_work, sort_bytes, s);
  };
  uint32_t *res = static_cast<uint32_t *>(dalloc(h, std::max<uint64_t>(M, 1) * 4, s));
  if (!res) return fail(ALTO_ERR_OOM, "pos_out of %llu entries", (unsigned long long)M);
  if (M == 0) {
    *out = res;
    return ALTO_OK;
  }
  if ((M + L - 1) / L <= kSegCap) {
    // every segment fits one CTA's shared memory
    static bool attr_set = false;
    if (!attr_set) {
      cudaError_t e1 = cudaFuncSetAttribute(pos_seg_kernel<1>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kSegSmem);
      cudaError_t e2 = cudaFuncSetAttribute(pos_seg_kernel<2>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kSegSmem);
      if (e1 != cudaSuccess || e2 != cudaSuccess) {
        dfree(h, res, M * 4, s);
        return fail(ALTO_ERR_CUDA, "pos_out: shared memory attribute");
      }
      attr_set = true;
    }
    const int grid = (int)std::min<uint64_t>(L, (uint64_t)h->num_sms * 2);
    const ModeRuns32 mr = mode_runs(h, mode);
    if (h->kw == 1)
      pos_seg_kernel<1><<<grid, kSegThreads, kSegSmem, s>>>(mr, h->keys, h->vals, M, L, res, keys_out,
                                                            vals_out);
    else
      pos_seg_kernel<2><<<grid, kSegThreads, kSegSmem, s>>>(mr, h->keys, h->vals, M, L, res, keys_out,
                                                            vals_out);
    note_launches(1);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) {
      dfree(h, res, M * 4, s);
      return fail(ALTO_ERR_CUDA, "pos_out: %s", cudaGetErrorString(e));
    }
    *out = res;
    return ALTO_OK;
  }
  for (int b = 0; b < 2; ++b) {
    kbuf[b] = static_cast<uint64_t *>(dalloc(h, M * 8, s));
    vbuf[b] = b == 0 ? reinterpret_cast<float *>(res) : static_cast<float *>(dalloc(h, M * 4, s));
  }
  pos = static_cast<uint32_t *>(dalloc(h, M * 4, s));
  sort_work = dalloc(h, sort_bytes, s);
  if (!kbuf[0] || !kbuf[1] || !vbuf[1] || !pos || !sort_work) {
    release(-1);
    return fail(ALTO_ERR_OOM, "pos_out sort scratch for %llu entries", (unsigned long long)M);
  }
  const int grid = (int)std::min<uint64_t>((M + 255) / 256, (uint64_t)h->num_sms * 8);
  const ModeRuns32 mr = mode_runs(h, mode);
  if (h->kw == 1)
    pos_key_kernel<1><<<grid, 256, 0, s>>>(mr, h->keys, M, L, bits, kbuf[0], pos);
  else
    pos_key_kernel<2><<<grid, 256, 0, s>>>(mr, h->keys, M, L, bits, kbuf[0], pos);
  note_launches(1);
  cudaError_t e = cudaGetLastError();
  int fbuf = 0;
  // the positions travel through the sort as 32-bit payload words, bit for bit
  if (e == cudaSuccess)
    e = launch_radix_sort(1, nbits, M, kbuf, vbuf, reinterpret_cast<const float *>(pos), sort_work,
                          h->status_dev, false, &fbuf, nullptr, h->num_sms, s);
  if (e != cudaSuccess) {
    release(-1);
    return fail(ALTO_ERR_CUDA, "pos_out: %s", cudaGetErrorString(e));
  }
  if (fbuf == 0) {
    release(0);
  } else {
    // result in vbuf[1]: keep it, free the buffer that was allocated as res
    dfree(h, res, M * 4, s);
    vbuf[0] = nullptr;
    res = reinterpret_cast<uint32_t *>(vbuf[1]);
    release(1);
  }
  e = launch_gather_out(res, h->keys, h->vals, M, h->kw, keys_out, vals_out, h->num_sms, s);
  if (e != cudaSuccess) {
    dfree(h, res, M * 4, s);
    return fail(ALTO_ERR_CUDA, "pos_out copy: %s", cudaGetErrorString(e));
  }
  *out = res;
  return ALTO_OK;
}

template <int KW>
__global__ void __launch_bounds__(256) gather_out_kernel(const uint32_t *__restrict__ perm,
                                                         const uint64_t *__restrict__ keys,
                                                         const float *__restrict__ vals, uint64_t nnz,
                                                         uint64_t *__restrict__ keys_out,
                                                         float *__restrict__ vals_out) {
  for (uint64_t p = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; p < nnz;
       p += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x = perm[p];
#pragma unroll
    for (int w = 0; w < KW; ++w) keys_out[p * KW + w] = keys[x * KW + w];
    vals_out[p] = vals[x];
  }
}

cudaError_t launch_gather_out(const uint32_t *perm, const uint64_t *keys, const float *vals,
                              uint64_t nnz, int kw, uint64_t *keys_out, float *vals_out, int num_sms,
                              cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  const int grid = (int)std::min<uint64_t>((nnz + 255) / 256, (uint64_t)num_sms * 16);
  if (kw == 1)
    gather_out_kernel<1><<<grid, 256, 0, s>>>(perm, keys, vals, nnz, keys_out, vals_out);
  else
    gather_out_kernel<2><<<grid, 256, 0, s>>>(perm, keys, vals, nnz, keys_out, vals_out);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mttkrp_out(const MttkrpArgs &a, int cpl, bool bf16, size_t smem, int num_sms,
                              cudaStream_t s) {
  if (a.nnz == 0) return cudaSuccess;
  switch (a.dp.nmodes) {
    case 3: return launch_mttkrp_out_nt<3>(a, cpl, bf16, smem, num_sms, s);
    case 4: return launch_mttkrp_out_nt<4>(a, cpl, bf16, smem, num_sms, s);
    case 5: return launch_mttkrp_out_nt<5>(a, cpl, bf16, smem, num_sms, s);
    default: return launch_mttkrp_out_nt<0>(a, cpl, bf16, smem, num_sms, s);
  }
}

cudaError_t launch_phi_out(const MttkrpArgs &a, bool pre, size_t smem, int num_sms, cudaStream_t s) {
  if (a.nnz == 0) return cudaSuccess;
  switch (a.dp.nmodes) {
    case 3: return launch_phi_out_nt<3>(a, pre, smem, num_sms, s);
    case 4: return launch_phi_out_nt<4>(a, pre, smem, num_sms, s);
    case 5: return launch_phi_out_nt<5>(a, pre, smem, num_sms, s);
    default: return launch_phi_out_nt<0>(a, pre, smem, num_sms, s);
  }
}

}  // namespace alto
