// The MTTKRP segment kernel (Alg. 3 with the conflict resolution of Alg. 4),
// included by the per-mode-count instantiation units mttkrp_n*.cu.
//
// One persistent CTA per SM walks line segments. Each warp takes 32
// consecutive ordered nonzeros: lane j loads and de-linearizes nonzero j
// (once), then groups of tpn = R / CPL lanes take tpn consecutive nonzeros of
// the batch each. Lane `sub` of a group owns the 16-byte column vectors
// sub, sub + tpn, sub + 2*tpn, ..., so each vector instruction of a group
// reads or atomically adds one contiguous 16*tpn-byte piece of a row. Runs of
// equal output row inside a group are summed in registers before they leave
// the warp.
//
// ATOMIC: hot rows (sampled at encode time) accumulate in a shared-memory
//   table found through an open-addressing hash; the table is flushed with
//   vector atomics every `flush_every` segments. Other rows go straight to
//   the output with red.global.add.v4.f32.
// PULL: the segment's Temp over its mode interval [T^s, T^e] lives in shared
//   memory (index i_mode - T^s) and is written out as the segment's partial
//   for pull_reduce_kernel.
#pragma once

#include "mttkrp.cuh"

namespace alto {

__device__ __forceinline__ int hot_lookup(const uint64_t *htab, int hbits, uint32_t row) {
  const uint32_t mask = (1u << hbits) - 1u;
  uint32_t h = (row * 0x9E3779B1u) >> (32 - hbits);
  for (int probe = 0; probe <= (int)mask; ++probe) {
    const uint64_t e = htab[h];
    const uint32_t r = (uint32_t)e;
    if (r == row) return (int)(e >> 32);
    if (r == kEmptyRow) return -1;
    h = (h + 1u) & mask;
  }
  return -1;
}

// Vector v of a lane covers columns 4 * (sub + v * tpn) .. +3.
template <int CPL, bool BF16>
__device__ __forceinline__ void load_row(const void *base, uint32_t row, int R, int sub, int tpn,
                                         float (&f)[CPL]) {
  const uint64_t off = (uint64_t)row * (uint64_t)R;
#pragma unroll
  for (int v = 0; v < CPL / 4; ++v) {
    const int col = 4 * (sub + v * tpn);
    if constexpr (!BF16) {
      const float4 q = __ldg(reinterpret_cast<const float4 *>(static_cast<const float *>(base) + off + col));
      f[4 * v + 0] = q.x;
      f[4 * v + 1] = q.y;
      f[4 * v + 2] = q.z;
      f[4 * v + 3] = q.w;
    } else {
      const uint2 q =
          __ldg(reinterpret_cast<const uint2 *>(static_cast<const __nv_bfloat16 *>(base) + off + col));
      f[4 * v + 0] = bf16lo(q.x);
      f[4 * v + 1] = bf16hi(q.x);
      f[4 * v + 2] = bf16lo(q.y);
      f[4 * v + 3] = bf16hi(q.y);
    }
  }
}

__device__ __forceinline__ void red_v4(float *addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b), "f"(c),
               "f"(d));
}

// Shared-memory rows start on bank 0 whatever the slot; XOR-ing the column
// with the slot's low bits spreads the rows of different slots that one
// instruction touches over different banks. The 16-byte vectors stay whole.
__device__ __forceinline__ int slot_swizzle(int slot, int R) {
  const int m = (R >= 32 ? 8 : R / 4) - 1;
  return (slot & m) << 2;
}

template <int CPL>
__device__ __forceinline__ void flush_run(const float (&run)[CPL], uint32_t row, int slot,
                                          float *temp, float *out, int R, int sub, int tpn) {
  if (slot >= 0) {
    float *t = temp + (size_t)slot * R;
    const int sw = slot_swizzle(slot, R);
#pragma unroll
    for (int v = 0; v < CPL / 4; ++v) {
      const int col = (4 * (sub + v * tpn)) ^ sw;
#pragma unroll
      for (int k = 0; k < 4; ++k) atomicAdd(t + col + k, run[4 * v + k]);
    }
  } else {
    float *o = out + (uint64_t)row * (uint64_t)R;
#pragma unroll
    for (int v = 0; v < CPL / 4; ++v)
      red_v4(o + 4 * (sub + v * tpn), run[4 * v], run[4 * v + 1], run[4 * v + 2], run[4 * v + 3]);
  }
}

// EXTRACT (Alg. 3), generic number of modes: the precomputed 32-bit runs of
// every rank, unrolled, masks and shifts from the constant bank.
template <int KW, int NMAX>
__device__ __forceinline__ void decode_runs(const DecodePlan32 &dp, int N, uint64_t lo, uint64_t hi,
                                            uint32_t (&c)[NMAX]) {
#pragma unroll
  for (int n = 0; n < NMAX; ++n) {
    uint32_t v = 0;
    if (n < N) {
      const int nr = dp.nruns[n];
#pragma unroll
      for (int r = 0; r < kMaxRuns32; ++r) {
        if (r < nr) {
          const Run32 &br = dp.runs[n][r];
          uint32_t x = window32<KW>(lo, hi, br.start) & br.mask[0];
#pragma unroll
          for (int j = 0; j < 5; ++j)
            if (j < br.steps) x = (x | (x >> br.sh[j])) & br.mask[j + 1];
          v |= x << br.outshift;
        }
      }
    }
    c[n] = v;
  }
}

// EXTRACT (Alg. 3) for a known number of modes N: rank q collects its bits
// from blocks j <= q, block j being an (N - j)-way interleave, so every stride
// is a compile-time constant and each block costs one window, one mask and a
// fixed number of doubling steps.
template <int KW, int K>
__device__ __forceinline__ uint32_t block_bits(const BlockPlan &bp, int j, int qmj, uint64_t lo,
                                               uint64_t hi) {
  const int st = bp.base[j] + qmj;
  const uint64_t w = (KW == 1) ? (lo >> st) : window64(lo, hi, st);
  uint32_t v = (uint32_t)compact_fixed<K>(w & bp.mask[j]) << bp.off[j];
  if (KW == 2 && bp.mask2[j]) {
    const uint64_t w2 = window64(lo, hi, st + bp.shift2[j]);
    v |= (uint32_t)compact_fixed<K>(w2 & bp.mask2[j]) << bp.off2[j];
  }
  return v;
}

template <int KW, int N, int Q, int J>
struct RankBits {
  static __device__ __forceinline__ uint32_t get(const BlockPlan &bp, uint64_t lo, uint64_t hi) {
    uint32_t v = 0;
    if (bp.mask[J]) v = block_bits<KW, N - J>(bp, J, Q - J, lo, hi);
    if constexpr (J < Q) v |= RankBits<KW, N, Q, J + 1>::get(bp, lo, hi);
    return v;
  }
};

template <int KW, int N, int Q>
__device__ __forceinline__ void decode_blocks(const BlockPlan &bp, uint64_t lo, uint64_t hi,
                                              uint32_t (&c)[N]) {
  c[Q] = RankBits<KW, N, Q, 0>::get(bp, lo, hi);
  if constexpr (Q + 1 < N) decode_blocks<KW, N, Q + 1>(bp, lo, hi, c);
}

template <int NT, int KW, int CPL, bool BF16, bool PULL>
__global__ void __launch_bounds__(kMttkrpThreads, kMttkrpBlocksPerSm) mttkrp_kernel(const __grid_constant__ MttkrpArgs a) {
  constexpr int NMAX = NT ? NT : kMaxModes;
  const int N = NT ? NT : a.dp.nmodes;
  extern __shared__ __align__(16) unsigned char sm[];
  float *temp = reinterpret_cast<float *>(sm);
  const int R = a.R;
  const int tpn = R / CPL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int grp = lane / tpn, sub = lane - grp * tpn;
  const unsigned full = 0xffffffffu;
  const int ro = a.out_rank;

  uint64_t *htab = nullptr;
  if (!PULL) {
    htab = reinterpret_cast<uint64_t *>(temp + (size_t)a.nslots * R);
    const int hsize = 1 << a.hbits;
    for (int i = threadIdx.x; i < hsize; i += blockDim.x) htab[i] = a.htab[i];
    for (int i = threadIdx.x; i < a.nslots * R; i += blockDim.x) temp[i] = 0.f;
    __syncthreads();
  }

  int since_flush = 0;
  for (uint64_t l = blockIdx.x; l < a.L; l += gridDim.x) {
    const uint64_t s0 = (l * a.nnz) / a.L, s1 = ((l + 1) * a.nnz) / a.L;
    uint32_t Ts = 0, len = 0;
    if (PULL) {
      if (s1 > s0) {
        Ts = a.intervals[(l * (uint64_t)N + a.mode) * 2];
        len = a.intervals[(l * (uint64_t)N + a.mode) * 2 + 1] - Ts + 1u;
      }
      for (uint32_t i = threadIdx.x; i < len * (uint32_t)R; i += blockDim.x) temp[i] = 0.f;
      __syncthreads();
    }
    // the next batch's positions and values are loaded while this one runs
    uint64_t nlo = 0, nhi = 0;
    float nv = 0.f;
    auto fetch = [&](uint64_t xx) {
      if (xx < s1) {
        if (KW == 1) {
          nlo = __ldcs(reinterpret_cast<const unsigned long long *>(a.keys) + xx);
        } else {
          const ulonglong2 kk = __ldcs(reinterpret_cast<const ulonglong2 *>(a.keys) + xx);
          nlo = kk.x;
          nhi = kk.y;
        }
        nv = __ldcs(a.vals + xx);
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
        decode_blocks<KW, NMAX, 0>(a.bp, lo, hi, c);
      else
        decode_runs<KW, NMAX>(a.dp, N, lo, hi, c);
      uint32_t row = 0;
#pragma unroll
      for (int n = 0; n < NMAX; ++n)
        if (n == ro) row = c[n];
      int slot = -1;
      if (valid) slot = PULL ? (int)(row - Ts) : hot_lookup(htab, a.hbits, row);
      const uint64_t rem = s1 - base;
      const int nvalid = rem < 32 ? (int)rem : 32;

      float run[CPL];
#pragma unroll
      for (int k = 0; k < CPL; ++k) run[k] = 0.f;
      uint32_t run_row = kEmptyRow;
      int run_slot = -1;
      for (int q = 0; q < tpn; ++q) {
        const int j = grp * tpn + q;
        const float vj = __shfl_sync(full, v, j);
        const int sj = __shfl_sync(full, slot, j);
        const uint32_t rj = __shfl_sync(full, row, j);
        uint32_t cj[NMAX];
#pragma unroll
        for (int n = 0; n < NMAX; ++n) cj[n] = (n < N && n != ro) ? __shfl_sync(full, c[n], j) : 0u;
        if (j < nvalid) {
          float p[CPL];
#pragma unroll
          for (int k = 0; k < CPL; ++k) p[k] = vj;
#pragma unroll
          for (int m = 0; m < NMAX; ++m) {
            if (m < N && m != ro) {
              float f[CPL];
              load_row<CPL, BF16>(a.factors[m], cj[m], R, sub, tpn, f);
#pragma unroll
              for (int k = 0; k < CPL; ++k) p[k] *= f[k];
            }
          }
          if (rj == run_row) {
#pragma unroll
            for (int k = 0; k < CPL; ++k) run[k] += p[k];
          } else {
            if (run_row != kEmptyRow) flush_run<CPL>(run, run_row, run_slot, temp, a.out, R, sub, tpn);
#pragma unroll
            for (int k = 0; k < CPL; ++k) run[k] = p[k];
            run_row = rj;
            run_slot = sj;
          }
        }
      }
      if (run_row != kEmptyRow) flush_run<CPL>(run, run_row, run_slot, temp, a.out, R, sub, tpn);
    }
    if (PULL) {
      __syncthreads();
      if (len) {
        float4 *dst = reinterpret_cast<float4 *>(a.partials + a.part_off[l] * (uint64_t)R);
        const uint32_t per_row = (uint32_t)R / 4;
        const uint32_t n4 = len * per_row;
        for (uint32_t i = threadIdx.x; i < n4; i += blockDim.x) {
          const uint32_t row = i / per_row, c4 = (i - row * per_row) * 4;
          dst[i] = *reinterpret_cast<const float4 *>(temp + row * R + (c4 ^ slot_swizzle(row, R)));
        }
      }
      __syncthreads();
    } else if (++since_flush >= a.flush_every || l + gridDim.x >= a.L) {
      since_flush = 0;
      __syncthreads();
      float4 *t4 = reinterpret_cast<float4 *>(temp);
      const int n4 = a.nslots * R / 4;
      const int per_row = R / 4;
      for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        const float4 t = t4[i];
        if (t.x != 0.f || t.y != 0.f || t.z != 0.f || t.w != 0.f) {
          const int sl = i / per_row, c4 = ((i - sl * per_row) * 4) ^ slot_swizzle(sl, R);
          red_v4(a.out + (uint64_t)a.slot_rows[sl] * (uint64_t)R + c4, t.x, t.y, t.z, t.w);
          t4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      __syncthreads();
    }
  }
}

template <int NT, int KW, int CPL, bool BF16, bool PULL>
static cudaError_t launch_one(const MttkrpArgs &a, size_t smem, int num_sms, cudaStream_t s) {
  auto kern = mttkrp_kernel<NT, KW, CPL, BF16, PULL>;
  static int configured = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mttkrp_smem_limit());
    if (e != cudaSuccess) return e;
    configured = 1;
  }
  uint64_t grid = (uint64_t)num_sms * kMttkrpBlocksPerSm;
  if (grid > a.L) grid = a.L;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kMttkrpThreads, smem, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

template <int NT, int KW, int CPL>
static cudaError_t launch_kc(const MttkrpArgs &a, bool bf16, bool pull, size_t smem, int num_sms,
                             cudaStream_t s) {
  if (bf16)
    return pull ? launch_one<NT, KW, CPL, true, true>(a, smem, num_sms, s)
                : launch_one<NT, KW, CPL, true, false>(a, smem, num_sms, s);
  return pull ? launch_one<NT, KW, CPL, false, true>(a, smem, num_sms, s)
              : launch_one<NT, KW, CPL, false, false>(a, smem, num_sms, s);
}

template <int NT>
cudaError_t launch_mttkrp_nt(const MttkrpArgs &a, int cpl, bool bf16, bool pull, size_t smem,
                             int num_sms, cudaStream_t s) {
  if (a.dp.kw == 1) {
    if (cpl == 4) return launch_kc<NT, 1, 4>(a, bf16, pull, smem, num_sms, s);
    if (cpl == 8) return launch_kc<NT, 1, 8>(a, bf16, pull, smem, num_sms, s);
    return launch_kc<NT, 1, 16>(a, bf16, pull, smem, num_sms, s);
  }
  if (cpl == 4) return launch_kc<NT, 2, 4>(a, bf16, pull, smem, num_sms, s);
  if (cpl == 8) return launch_kc<NT, 2, 8>(a, bf16, pull, smem, num_sms, s);
  return launch_kc<NT, 2, 16>(a, bf16, pull, smem, num_sms, s);
}

}  // namespace alto
