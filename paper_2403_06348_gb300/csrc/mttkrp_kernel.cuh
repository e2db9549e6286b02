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

#ifndef ALTO_HOT_ROTATE
#define ALTO_HOT_ROTATE 1
#endif

// First column of a lane's v-th 4-column vector. CPL = 8: the lane's columns
// are contiguous (8 sub .. 8 sub + 7, one 32-byte load per row); otherwise
// vector v covers columns 4 (sub + v tpn) .. + 3.
template <int CPL>
__device__ __forceinline__ int lane_col(int sub, int v, int tpn) {
  return CPL == 8 ? 8 * sub + 4 * v : 4 * (sub + v * tpn);
}

// Byte offset of a lane's first column in a factor row.
template <int CPL, bool BF16>
__device__ __forceinline__ uint32_t lane_byte_offset(int sub) {
  return (uint32_t)lane_col<CPL>(sub, 0, 1) * (BF16 ? 2u : 4u);
}

// Shared-memory flushes: at step k, the lanes of group g add element
// (k + g) mod 4 of their 4-column vector, so groups flushing in the same
// instruction use different banks (each group's lanes cover a whole row).
template <int CPL, bool ROT = (CPL >= 8)>
__device__ __forceinline__ void flush_run(const float (&run)[CPL], uint32_t row, int slot,
                                          float *temp, float *out, int R, int sub, int tpn,
                                          int grp) {
  if (slot >= 0) {
    float *t = temp + (size_t)slot * R;
    const int sw = slot_swizzle(slot, R);
    const int rot = (ALTO_HOT_ROTATE && ROT) ? (grp & 3) : 0;
#pragma unroll
    for (int v = 0; v < CPL / 4; ++v) {
      const int col = lane_col<CPL>(sub, v, tpn) ^ sw;
      float e0 = run[4 * v], e1 = run[4 * v + 1], e2 = run[4 * v + 2], e3 = run[4 * v + 3];
      if (rot & 1) {
        const float x = e0;
        e0 = e1;
        e1 = e2;
        e2 = e3;
        e3 = x;
      }
      if (rot & 2) {
        const float x = e0, y = e1;
        e0 = e2;
        e1 = e3;
        e2 = x;
        e3 = y;
      }
      atomicAdd(t + col + (rot & 3), e0);
      atomicAdd(t + col + ((rot + 1) & 3), e1);
      atomicAdd(t + col + ((rot + 2) & 3), e2);
      atomicAdd(t + col + ((rot + 3) & 3), e3);
    }
  } else {
    float *o = out + (uint64_t)row * (uint64_t)R;
#pragma unroll
    for (int v = 0; v < CPL / 4; ++v)
      red_v4(o + lane_col<CPL>(sub, v, tpn), run[4 * v], run[4 * v + 1], run[4 * v + 2], run[4 * v + 3]);
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

// p = vj * (the product over the N-1 input factors of row ij[k]), this lane's
// CPL columns of it. fb[k] is input factor k plus the lane's byte offset.
template <int NMAX, int CPL, bool BF16>
__device__ __forceinline__ void gather_product(const char *const (&fb)[NMAX > 1 ? NMAX - 1 : 1],
                                               const uint32_t (&ij)[NMAX > 1 ? NMAX - 1 : 1],
                                               uint32_t rowb, int tpn, int N, float vj,
                                               float (&p)[CPL]) {
  constexpr int NIN = NMAX > 1 ? NMAX - 1 : 1;
#pragma unroll
  for (int k = 0; k < NIN; ++k) {
    if (k + 1 < N) {
      const char *rb = fb[k] + (uint64_t)ij[k] * rowb;
      float f[CPL];
      if constexpr (CPL == 8 && !BF16) {
        asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
            : "=f"(f[0]), "=f"(f[1]), "=f"(f[2]), "=f"(f[3]), "=f"(f[4]), "=f"(f[5]), "=f"(f[6]),
              "=f"(f[7])
            : "l"(rb));
      } else if constexpr (CPL == 8) {
        const uint4 qv = __ldg(reinterpret_cast<const uint4 *>(rb));
        f[0] = bf16lo(qv.x);
        f[1] = bf16hi(qv.x);
        f[2] = bf16lo(qv.y);
        f[3] = bf16hi(qv.y);
        f[4] = bf16lo(qv.z);
        f[5] = bf16hi(qv.z);
        f[6] = bf16lo(qv.w);
        f[7] = bf16hi(qv.w);
      } else {
#pragma unroll
      for (int w = 0; w < CPL / 4; ++w) {
        const int voff = w * tpn * (BF16 ? 8 : 16);
        if constexpr (!BF16) {
          const float4 qv = __ldg(reinterpret_cast<const float4 *>(rb + voff));
          f[4 * w] = qv.x;
          f[4 * w + 1] = qv.y;
          f[4 * w + 2] = qv.z;
          f[4 * w + 3] = qv.w;
        } else {
          const uint2 qv = __ldg(reinterpret_cast<const uint2 *>(rb + voff));
          f[4 * w] = bf16lo(qv.x);
          f[4 * w + 1] = bf16hi(qv.x);
          f[4 * w + 2] = bf16lo(qv.y);
          f[4 * w + 3] = bf16hi(qv.y);
        }
      }
      }
#pragma unroll
      for (int c = 0; c < CPL; ++c) p[c] = (k == 0 ? vj : p[c]) * f[c];
    } else if (k == 0) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) p[c] = vj;
    }
  }
}

#ifndef ALTO_MTTKRP_RUNS
#define ALTO_MTTKRP_RUNS 1
#endif

// The rounds of one batch: round q gives group grp the batch's nonzero
// j = grp * tpn + q; the group gathers its N-1 input rows (lane `sub` holds the
// column vectors sub, sub + tpn, ...), multiplies, and sums runs of equal
// output row in registers before flushing them. TAIL batches check j < nvalid.
// fb[k] is the k-th input factor plus this lane's byte offset (inb).
//
// APR != 0 computes the CP-APR model update Phi (Alg. 5) instead: the group's
// Khatri-Rao row krp (the product of the gathered rows, or row pos0 + j of the
// precomputed Pi when APR == kAprPre) is dotted with row rj of B over the
// group's lanes, and the run receives v / max(B(rj,:) . krp, eps) * krp.
constexpr int kAprOff = 0, kAprOtf = 1, kAprPre = 2;

struct AprArgs {
  const float *bmat;   // B of the output mode [I_n][R]
  const float *pimat;  // Pi [nnz][R] in ALTO order (kAprPre)
  float eps;
  uint64_t pos0;       // ordered position of the batch's first nonzero
};

template <int NMAX, int CPL, bool BF16, bool TAIL, int APR = kAprOff, bool ROT = (CPL >= 8)>
__device__ __forceinline__ void group_rounds(const char *const (&fb)[NMAX > 1 ? NMAX - 1 : 1],
                                             float *out, int R, int N, int tpn, int grp, int sub,
                                             float v, int slot, uint32_t row,
                                             const uint32_t (&in)[NMAX > 1 ? NMAX - 1 : 1], int nvalid,
                                             float *temp, uint32_t rowb, const AprArgs &apr = AprArgs{}) {
  static_assert(APR == kAprOff || (CPL == 4 && !BF16), "Phi uses 4 fp32 columns per lane");
  constexpr int NIN = NMAX > 1 ? NMAX - 1 : 1;
  const unsigned full = 0xffffffffu;
  float run[CPL];
#pragma unroll
  for (int k = 0; k < CPL; ++k) run[k] = 0.f;
  uint32_t run_row = kEmptyRow;
  int run_slot = -1;
#pragma unroll(CPL <= 8 ? 2 : 1)
  for (int q = 0; q < tpn; ++q) {
    const int j = grp * tpn + q;
    const float vj = __shfl_sync(full, v, j);
    const int sj = __shfl_sync(full, slot, j);
    const uint32_t rj = __shfl_sync(full, row, j);
    uint32_t ij[NIN];
#pragma unroll
    for (int k = 0; k < NIN; ++k)
      ij[k] = (APR != kAprPre && k + 1 < N) ? __shfl_sync(full, in[k], j) : 0u;
    float p[CPL];
    if constexpr (APR != kAprOff) {
      const bool live = !TAIL || j < nvalid;
      float kr[4] = {1.f, 1.f, 1.f, 1.f};
      if (APR == kAprPre) {
        if (live) {
          const float4 qv = __ldg(reinterpret_cast<const float4 *>(apr.pimat) +
                                  (apr.pos0 + (uint64_t)j) * (uint64_t)(R / 4) + sub);
          kr[0] = qv.x;
          kr[1] = qv.y;
          kr[2] = qv.z;
          kr[3] = qv.w;
        }
      } else {
#pragma unroll
        for (int k = 0; k < NIN; ++k) {
          if (k + 1 < N) {
            const float4 qv = __ldg(reinterpret_cast<const float4 *>(fb[k] + (uint64_t)ij[k] * rowb));
            kr[0] *= qv.x;
            kr[1] *= qv.y;
            kr[2] *= qv.z;
            kr[3] *= qv.w;
          }
        }
      }
      const float4 bv = __ldg(reinterpret_cast<const float4 *>(apr.bmat) + (uint64_t)rj * (R / 4) + sub);
      float dot = kr[0] * bv.x + kr[1] * bv.y + kr[2] * bv.z + kr[3] * bv.w;
      for (int o = 1; o < tpn; o <<= 1) dot += __shfl_xor_sync(full, dot, o);
      if (!live) continue;
      const float scale = vj / fmaxf(dot, apr.eps);
#pragma unroll
      for (int c = 0; c < 4; ++c) p[c] = scale * kr[c];
    } else {
      if (TAIL && j >= nvalid) continue;
      gather_product<NMAX, CPL, BF16>(fb, ij, rowb, tpn, N, vj, p);
    }
    if (ALTO_MTTKRP_RUNS && rj == run_row) {
#pragma unroll
      for (int c = 0; c < CPL; ++c) run[c] += p[c];
    } else {
      if (run_row != kEmptyRow) flush_run<CPL, ROT>(run, run_row, run_slot, temp, out, R, sub, tpn, grp);
#pragma unroll
      for (int c = 0; c < CPL; ++c) run[c] = p[c];
      run_row = rj;
      run_slot = sj;
    }
  }
  if (run_row != kEmptyRow) flush_run<CPL, ROT>(run, run_row, run_slot, temp, out, R, sub, tpn, grp);
}

// Wider lanes (8 or 16 columns) keep twice the values in registers: those
// builds run two CTAs per SM (64 registers) instead of three (40).
template <int CPL>
constexpr int mttkrp_min_blocks() {
  return CPL >= 8 ? 2 : kMttkrpBlocksPerSm;
}

template <int NT, int KW, int CPL, bool BF16, bool PULL, int APR = kAprOff>
__global__ void __launch_bounds__(kMttkrpThreads, mttkrp_min_blocks<CPL>())
    mttkrp_kernel(const __grid_constant__ MttkrpArgs a) {
  if (APR != kAprOff && a.skip && *a.skip) return;  // CP-APR inner loop already converged
  constexpr int NMAX = NT ? NT : kMaxModes;
  const int N = NT ? NT : a.dp.nmodes;
  extern __shared__ __align__(16) unsigned char sm[];
  float *temp = reinterpret_cast<float *>(sm);
  const int R = a.R;
  const int tpn = R / CPL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int grp = lane / tpn, sub = lane - grp * tpn;
  const int ro = a.out_rank;
  // byte offset of this lane's first column vector, and the row strides
  const uint32_t rowb = (uint32_t)R * (BF16 ? 2u : 4u);
  const uint32_t inb = lane_byte_offset<CPL, BF16>(sub);
  constexpr int NIN = NMAX > 1 ? NMAX - 1 : 1;
  const char *fb[NIN];
#pragma unroll
  for (int k = 0; k < NIN; ++k) fb[k] = static_cast<const char *>(a.fin[k]) + inb;

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
      // the output row and the N-1 input coordinates in a fixed order
      uint32_t row = c[0];
      uint32_t in[NIN];
#pragma unroll
      for (int n = 1; n < NMAX; ++n)
        if (n == ro) row = c[n];
#pragma unroll
      for (int k = 0; k < NIN; ++k) in[k] = (NMAX > 1 && k + 1 < NMAX) ? (k < ro ? c[k] : c[k + 1]) : 0u;
      int slot = -1;
      if (valid) slot = PULL ? (int)(row - Ts) : hot_lookup(htab, a.hbits, row);
      const uint64_t rem = s1 - base;
      AprArgs apr{};
      if constexpr (APR != kAprOff) apr = AprArgs{a.bmat, a.pimat, a.eps, base};
      if (rem >= 32)
        group_rounds<NMAX, CPL, BF16, false, APR>(fb, a.out, R, N, tpn, grp, sub, v, slot, row, in,
                                                  32, temp, rowb, apr);
      else
        group_rounds<NMAX, CPL, BF16, true, APR>(fb, a.out, R, N, tpn, grp, sub, v, slot, row, in,
                                                 (int)rem, temp, rowb, apr);
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

// ---------------------------------------------------------------------------
// One thread per nonzero ("threads per nonzero" = 1). A thread decodes its
// nonzero, then walks the row in chunks of 8 columns: one 32-byte load per
// input factor row (a whole sector), 8 products per input mode, and the chunk
// leaves through two 16-byte vector atomics (cold row) or 8 shared-memory
// atomics (hot row / Temp). No shuffles; each warp keeps 32 independent row
// gathers in flight. The staging table here swizzles every column by the low
// bits of its slot, so threads on different rows use different banks.
// ---------------------------------------------------------------------------
__device__ __forceinline__ int lpn_swizzle(int slot, int R) { return slot & ((R < 32 ? R : 32) - 1); }

template <bool BF16>
__device__ __forceinline__ void load8(const void *base, uint64_t off, float (&f)[8]) {
  if constexpr (!BF16) {
    const float *p = static_cast<const float *>(base) + off;
    asm("ld.global.nc.v8.f32 {%0, %1, %2, %3, %4, %5, %6, %7}, [%8];"
        : "=f"(f[0]), "=f"(f[1]), "=f"(f[2]), "=f"(f[3]), "=f"(f[4]), "=f"(f[5]), "=f"(f[6]), "=f"(f[7])
        : "l"(p));
  } else {
    const uint4 q = __ldg(reinterpret_cast<const uint4 *>(static_cast<const __nv_bfloat16 *>(base) + off));
    f[0] = bf16lo(q.x);
    f[1] = bf16hi(q.x);
    f[2] = bf16lo(q.y);
    f[3] = bf16hi(q.y);
    f[4] = bf16lo(q.z);
    f[5] = bf16hi(q.z);
    f[6] = bf16lo(q.w);
    f[7] = bf16hi(q.w);
  }
}

template <int NT, int KW, bool BF16, bool PULL>
__global__ void __launch_bounds__(kMttkrpThreads, kMttkrpBlocksPerSm)
    mttkrp_lpn_kernel(const __grid_constant__ MttkrpArgs a) {
  constexpr int NMAX = NT ? NT : kMaxModes;
  const int N = NT ? NT : a.dp.nmodes;
  extern __shared__ __align__(16) unsigned char sm[];
  float *temp = reinterpret_cast<float *>(sm);
  const int R = a.R;
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
    for (uint64_t x = s0 + threadIdx.x; x < s1; x += blockDim.x) {
      uint64_t lo, hi = 0;
      if (KW == 1) {
        lo = __ldcs(reinterpret_cast<const unsigned long long *>(a.keys) + x);
      } else {
        const ulonglong2 kk = __ldcs(reinterpret_cast<const ulonglong2 *>(a.keys) + x);
        lo = kk.x;
        hi = kk.y;
      }
      const float v = __ldcs(a.vals + x);
      uint32_t c[NMAX];
      if constexpr (NT > 0)
        decode_blocks<KW, NMAX, 0>(a.bp, lo, hi, c);
      else
        decode_runs<KW, NMAX>(a.dp, N, lo, hi, c);
      uint32_t row = 0;
#pragma unroll
      for (int n = 0; n < NMAX; ++n)
        if (n == ro) row = c[n];
      const int slot = PULL ? (int)(row - Ts) : hot_lookup(htab, a.hbits, row);
      const int sw = slot >= 0 ? lpn_swizzle(slot, R) : 0;
      float *trow = temp + (size_t)(slot >= 0 ? slot : 0) * R;
      float *orow = a.out + (uint64_t)row * (uint64_t)R;
      for (int cc = 0; cc < R; cc += 8) {
        float p[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) p[k] = v;
#pragma unroll
        for (int m = 0; m < NMAX; ++m) {
          if (m < N && m != ro) {
            float f[8];
            load8<BF16>(a.factors[m], (uint64_t)c[m] * (uint64_t)R + cc, f);
#pragma unroll
            for (int k = 0; k < 8; ++k) p[k] *= f[k];
          }
        }
        if (slot >= 0) {
#pragma unroll
          for (int k = 0; k < 8; ++k) atomicAdd(trow + ((cc + k) ^ sw), p[k]);
        } else {
          red_v4(orow + cc, p[0], p[1], p[2], p[3]);
          red_v4(orow + cc + 4, p[4], p[5], p[6], p[7]);
        }
      }
    }
    if (PULL) {
      __syncthreads();
      if (len) {
        float *dst = a.partials + a.part_off[l] * (uint64_t)R;
        const uint32_t n = len * (uint32_t)R;
        for (uint32_t i = threadIdx.x; i < n; i += blockDim.x) {
          const uint32_t r = i / (uint32_t)R, col = i - r * (uint32_t)R;
          dst[i] = temp[r * R + (col ^ lpn_swizzle((int)r, R))];
        }
      }
      __syncthreads();
    } else if (++since_flush >= a.flush_every || l + gridDim.x >= a.L) {
      since_flush = 0;
      __syncthreads();
      const int n = a.nslots * R;
      for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const float t = temp[i];
        if (t != 0.f) {
          const int sl = i / R, col = (i - sl * R) ^ lpn_swizzle(sl, R);
          atomicAdd(a.out + (uint64_t)a.slot_rows[sl] * (uint64_t)R + col, t);
          temp[i] = 0.f;
        }
      }
      __syncthreads();
    }
  }
}

// CTAs of kMttkrpThreads that fit one SM with `smem` bytes of dynamic shared
// memory (at most kMttkrpBlocksPerSm).
template <typename K>
static int resident_ctas(K kern, size_t smem) {
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kMttkrpThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  return per_sm < 1 ? 1 : (per_sm > kMttkrpBlocksPerSm ? kMttkrpBlocksPerSm : per_sm);
}

template <int NT, int KW, bool BF16, bool PULL>
static cudaError_t launch_lpn(const MttkrpArgs &a, size_t smem, int num_sms, cudaStream_t s) {
  auto kern = mttkrp_lpn_kernel<NT, KW, BF16, PULL>;
  static int configured = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mttkrp_smem_limit());
    if (e != cudaSuccess) return e;
    configured = 1;
  }
  uint64_t grid = (uint64_t)num_sms * resident_ctas(kern, smem);
  if (grid > a.L) grid = a.L;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kMttkrpThreads, smem, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

template <int NT, int KW>
static cudaError_t launch_lpn_k(const MttkrpArgs &a, bool bf16, bool pull, size_t smem, int num_sms,
                                cudaStream_t s) {
  if (bf16)
    return pull ? launch_lpn<NT, KW, true, true>(a, smem, num_sms, s)
                : launch_lpn<NT, KW, true, false>(a, smem, num_sms, s);
  return pull ? launch_lpn<NT, KW, false, true>(a, smem, num_sms, s)
              : launch_lpn<NT, KW, false, false>(a, smem, num_sms, s);
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
  uint64_t grid = (uint64_t)num_sms * resident_ctas(kern, smem);
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

// The CP-APR model update Phi (Alg. 5) through the same kernel: 4 fp32
// columns per lane, ATOMIC (hot rows staged) or PULL, the Khatri-Rao rows
// gathered on the fly (OTF) or read from a precomputed Pi (PRE).
template <int NT, int KW, bool PULL, int APR>
static cudaError_t launch_phi_one(const MttkrpArgs &a, size_t smem, int num_sms, cudaStream_t s) {
  auto kern = mttkrp_kernel<NT, KW, 4, false, PULL, APR>;
  static int configured = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mttkrp_smem_limit());
    if (e != cudaSuccess) return e;
    configured = 1;
  }
  uint64_t grid = (uint64_t)num_sms * resident_ctas(kern, smem);
  if (grid > a.L) grid = a.L;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kMttkrpThreads, smem, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

template <int NT>
cudaError_t launch_phi_nt(const MttkrpArgs &a, bool pull, bool pre, size_t smem, int num_sms,
                          cudaStream_t s) {
  if (a.dp.kw == 1) {
    if (pull) return pre ? launch_phi_one<NT, 1, true, kAprPre>(a, smem, num_sms, s)
                         : launch_phi_one<NT, 1, true, kAprOtf>(a, smem, num_sms, s);
    return pre ? launch_phi_one<NT, 1, false, kAprPre>(a, smem, num_sms, s)
               : launch_phi_one<NT, 1, false, kAprOtf>(a, smem, num_sms, s);
  }
  if (pull) return pre ? launch_phi_one<NT, 2, true, kAprPre>(a, smem, num_sms, s)
                       : launch_phi_one<NT, 2, true, kAprOtf>(a, smem, num_sms, s);
  return pre ? launch_phi_one<NT, 2, false, kAprPre>(a, smem, num_sms, s)
             : launch_phi_one<NT, 2, false, kAprOtf>(a, smem, num_sms, s);
}

template <int NT>
cudaError_t launch_mttkrp_nt(const MttkrpArgs &a, int cpl, bool bf16, bool pull, size_t smem,
                             int num_sms, cudaStream_t s) {
  if (cpl == a.R && a.R >= 8)
    return a.dp.kw == 1 ? launch_lpn_k<NT, 1>(a, bf16, pull, smem, num_sms, s)
                        : launch_lpn_k<NT, 2>(a, bf16, pull, smem, num_sms, s);
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
