// Internal definitions shared by the ALTO kernels and the C ABI layer.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cstdint>
#include <cstddef>

#include "alto.h"

namespace alto {

constexpr int kMaxModes = ALTO_MAX_MODES;
constexpr int kMaxRuns = 12;          // strided runs per mode (see BitRun)
constexpr uint32_t kEmptyRow = 0xFFFFFFFFu;

// Device status word bits (latched per handle).
constexpr uint32_t kStatusCoordRange = 1u;
constexpr uint32_t kStatusNotSpd = 2u;
constexpr uint32_t kStatusTimeout = 4u;
constexpr uint32_t kStatusPinv = 8u;  // a CP-ALS solve used the pseudo-inverse

// One strided run of a mode's bits inside the linear index (Section III-A):
// bits g0 .. g0+count-1 of the coordinate sit at key positions
// shift, shift+stride, ..., shift+(count-1)*stride. Inside one bit group block
// with k active modes the stride is k. Runs are split so that every run lies
// in the 64-bit window starting at `shift`.
struct BitRun {
  uint8_t shift;
  uint8_t stride;
  uint8_t count;
  uint8_t outshift;  // g0
};

struct DecodePlan {
  int nmodes;
  int kw;                          // 64-bit words per position (1 or 2)
  int nruns[kMaxModes];
  BitRun runs[kMaxModes][kMaxRuns];
};

// The bit plan by blocks (Section III-A): sort the modes by length (rank 0 =
// shortest); block j holds the bit groups g with bits(rank j-1) <= g <
// bits(rank j), each group holding bit g of ranks j..N-1 in rank order, so
// block j is an (N - j)-way interleave and bit g of rank q >= j sits at
// base[j] + (g - off[j]) * (N - j) + (q - j). Decoding rank q therefore takes,
// for every block j <= q, a window starting at base[j] + q - j, keeps cnt[j]
// bits at stride N - j (mask[j]) and compacts them with a stride known at
// compile time. A block wider than 64 bits (two-word positions) is cut in two
// windows: the second starts shift2[j] bits later and holds cnt2[j] bits.
struct BlockPlan {
  int nmodes;
  int kw;
  int out_rank;                 // rank of the MTTKRP output mode
  uint8_t base[kMaxModes];
  uint8_t off[kMaxModes];       // coordinate bit of the block's first bit
  uint8_t shift2[kMaxModes];
  uint8_t off2[kMaxModes];
  uint64_t mask[kMaxModes];     // cnt[j] bits at stride N - j from bit 0
  uint64_t mask2[kMaxModes];    // second window (0 if none)
};

// The same bit plan cut into runs that fit a 32-bit window, with the masks
// and shifts of the compaction precomputed on the host: the run's bits sit at
// window bits 0, k, 2k, ... (count of them); x = window & mask[0], then for
// each step j, x = (x | x >> sh[j]) & mask[j + 1] doubles the packed groups.
constexpr int kMaxRuns32 = 16;
struct Run32 {
  uint32_t mask[6];
  uint8_t sh[5];
  uint8_t start;     // key bit of the first bit of the run
  uint8_t steps;     // number of doubling steps
  uint8_t outshift;  // coordinate bit of the first bit of the run
};

struct DecodePlan32 {
  int nmodes;
  int kw;
  int nruns[kMaxModes];
  Run32 runs[kMaxModes][kMaxRuns32];
};


// ---------------------------------------------------------------------------
// Stride compaction (PEXT of a regularly spaced mask) and expansion (PDEP).
// For stride K the bits at 0, K, 2K, ... are gathered into consecutive bits by
// doubling groups: after step j, groups of 2^j bits sit at multiples of K*2^j.
// ---------------------------------------------------------------------------
__host__ __device__ constexpr uint64_t stride_mask(int K, int j) {
  uint64_t m = 0;
  const int g = 1 << j;
  const int sp = K * g;
  for (int p = 0; p < 64; p += sp)
    for (int b = 0; b < g && p + b < 64; ++b) m |= (uint64_t)1 << (p + b);
  return m;
}

__device__ __forceinline__ uint64_t low_mask64(int cnt) {
  return cnt >= 64 ? ~0ull : ((1ull << cnt) - 1ull);
}

// Shifts by a compile-time amount; amounts >= 64 give 0 (such steps only
// occur for run lengths that cannot fit a 64-bit window).
template <int S>
__device__ __forceinline__ uint64_t shr_c(uint64_t x) {
  if constexpr (S >= 64) return 0; else return x >> S;
}
template <int S>
__device__ __forceinline__ uint64_t shl_c(uint64_t x) {
  if constexpr (S >= 64) return 0; else return x << S;
}

template <int K>
__device__ __forceinline__ uint64_t compact_k(uint64_t x, int cnt) {
  x &= stride_mask(K, 0);
  if (cnt > 1) x = (x | shr_c<(K - 1) << 0>(x)) & stride_mask(K, 1);
  if (cnt > 2) x = (x | shr_c<(K - 1) << 1>(x)) & stride_mask(K, 2);
  if (cnt > 4) x = (x | shr_c<(K - 1) << 2>(x)) & stride_mask(K, 3);
  if (cnt > 8) x = (x | shr_c<(K - 1) << 3>(x)) & stride_mask(K, 4);
  if (cnt > 16) x = (x | shr_c<(K - 1) << 4>(x)) & stride_mask(K, 5);
  return x & low_mask64(cnt);
}

template <int K>
__device__ __forceinline__ uint64_t expand_k(uint64_t x, int cnt) {
  x &= low_mask64(cnt);
  if (cnt > 16) x = (x | shl_c<(K - 1) << 4>(x)) & stride_mask(K, 4);
  if (cnt > 8) x = (x | shl_c<(K - 1) << 3>(x)) & stride_mask(K, 3);
  if (cnt > 4) x = (x | shl_c<(K - 1) << 2>(x)) & stride_mask(K, 2);
  if (cnt > 2) x = (x | shl_c<(K - 1) << 1>(x)) & stride_mask(K, 1);
  if (cnt > 1) x = (x | shl_c<(K - 1) << 0>(x)) & stride_mask(K, 0);
  return x;
}

__device__ __forceinline__ uint64_t compact_stride(uint64_t w, int k, int cnt) {
  switch (k) {
    case 1: return w & low_mask64(cnt);
    case 2: return compact_k<2>(w, cnt);
    case 3: return compact_k<3>(w, cnt);
    case 4: return compact_k<4>(w, cnt);
    case 5: return compact_k<5>(w, cnt);
    case 6: return compact_k<6>(w, cnt);
    case 7: return compact_k<7>(w, cnt);
    default: return compact_k<8>(w, cnt);
  }
}

__device__ __forceinline__ uint64_t expand_stride(uint64_t v, int k, int cnt) {
  switch (k) {
    case 1: return v & low_mask64(cnt);
    case 2: return expand_k<2>(v, cnt);
    case 3: return expand_k<3>(v, cnt);
    case 4: return expand_k<4>(v, cnt);
    case 5: return expand_k<5>(v, cnt);
    case 6: return expand_k<6>(v, cnt);
    case 7: return expand_k<7>(v, cnt);
    default: return expand_k<8>(v, cnt);
  }
}

// Gathers bits 0, K, 2K, ... of x (already masked to those positions) into
// the low bits: fixed doubling steps with immediate masks.
template <int K>
__device__ __forceinline__ uint64_t compact_fixed(uint64_t x) {
  if constexpr (K == 1) {
    return x;
  } else {
    constexpr int kMaxCnt = (63 / K + 1) < 32 ? (63 / K + 1) : 32;
    if constexpr (kMaxCnt > 1) x = (x | shr_c<(K - 1) << 0>(x)) & stride_mask(K, 1);
    if constexpr (kMaxCnt > 2) x = (x | shr_c<(K - 1) << 1>(x)) & stride_mask(K, 2);
    if constexpr (kMaxCnt > 4) x = (x | shr_c<(K - 1) << 2>(x)) & stride_mask(K, 3);
    if constexpr (kMaxCnt > 8) x = (x | shr_c<(K - 1) << 3>(x)) & stride_mask(K, 4);
    if constexpr (kMaxCnt > 16) x = (x | shr_c<(K - 1) << 4>(x)) & stride_mask(K, 5);
    return x;
  }
}

// 64-bit window of a 128-bit position starting at bit s.
__device__ __forceinline__ uint64_t window64(uint64_t lo, uint64_t hi, int s) {
  if (s == 0) return lo;
  if (s < 64) return (lo >> s) | (hi << (64 - s));
  return hi >> (s - 64);
}

template <int KW>
__device__ __forceinline__ uint32_t window32(uint64_t lo, uint64_t hi, int s) {
  if (KW == 1) return (uint32_t)(lo >> s);
  return (uint32_t)window64(lo, hi, s);
}

// De-linearize one position into all coordinates (EXTRACT of Alg. 3).
template <int KW>
__device__ __forceinline__ void decode_all(const DecodePlan &dp, uint64_t lo, uint64_t hi,
                                           uint32_t (&c)[kMaxModes]) {
#pragma unroll
  for (int n = 0; n < kMaxModes; ++n) {
    uint32_t v = 0;
    if (n < dp.nmodes) {
      const int nr = dp.nruns[n];
      for (int r = 0; r < nr; ++r) {
        const BitRun br = dp.runs[n][r];
        const uint64_t w = (KW == 1) ? (br.shift ? (lo >> br.shift) : lo)
                                     : window64(lo, hi, br.shift);
        v |= (uint32_t)compact_stride(w, br.stride, br.count) << br.outshift;
      }
    }
    c[n] = v;
  }
}

// ---------------------------------------------------------------------------
// Byte-table de-linearization (EXTRACT of Alg. 3) for positions of at most 64
// bits. The position's bits are a fixed permutation of the coordinates' bits,
// so every byte of the position contributes disjoint bits: table[b][v] holds
// the bits that byte value v at byte b contributes, with the coordinates
// packed by rank (rank q at bit off[q], bits[q] wide). A position's packed
// coordinates are the OR of its eight bytes' entries.
// ---------------------------------------------------------------------------
constexpr int kLutEntries = 8 * 256;
constexpr size_t kLutBytes = (size_t)kLutEntries * sizeof(uint64_t);

struct LutPlan {
  uint8_t off[kMaxModes];   // bit of rank q in the packed word
  uint8_t bits[kMaxModes];  // its width
};

template <int NMAX>
__device__ __forceinline__ void decode_lut(const uint64_t *__restrict__ T, const LutPlan &lp, uint64_t key,
                                           uint32_t (&c)[NMAX]) {
  const uint32_t l = (uint32_t)key, h = (uint32_t)(key >> 32);
  const uint64_t p = (T[l & 255u] | T[256 + ((l >> 8) & 255u)] | T[512 + ((l >> 16) & 255u)] |
                      T[768 + (l >> 24)]) |
                     (T[1024 + (h & 255u)] | T[1280 + ((h >> 8) & 255u)] | T[1536 + ((h >> 16) & 255u)] |
                      T[1792 + (h >> 24)]);
#pragma unroll
  for (int q = 0; q < NMAX; ++q)
    c[q] = (uint32_t)(p >> lp.off[q]) & (uint32_t)((1ull << lp.bits[q]) - 1ull);
}

// ---------------------------------------------------------------------------
// Raw vector memory helpers (inline PTX)
// ---------------------------------------------------------------------------
__device__ __forceinline__ void red_add_v4(float *addr, float a, float b, float c, float d) {
  asm volatile("red.global.add.v4.f32 [%0], {%1, %2, %3, %4};" ::"l"(addr), "f"(a), "f"(b),
               "f"(c), "f"(d)
               : "memory");
}

__device__ __forceinline__ float4 ldg_nc_f4(const float *p) {
  float4 v;
  asm volatile("ld.global.nc.v4.f32 {%0, %1, %2, %3}, [%4];"
               : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w)
               : "l"(p));
  return v;
}

__device__ __forceinline__ uint2 ldg_nc_u2(const void *p) {
  uint2 v;
  asm volatile("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(v.x), "=r"(v.y) : "l"(p));
  return v;
}

__device__ __forceinline__ uint4 ldg_nc_u4(const void *p) {
  uint4 v;
  asm volatile("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];"
               : "=r"(v.x), "=r"(v.y), "=r"(v.z), "=r"(v.w)
               : "l"(p));
  return v;
}

// Streaming (evict-first) loads for the once-read nonzero stream.
__device__ __forceinline__ uint64_t ldg_stream_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.global.cs.u64 %0, [%1];" : "=l"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ ulonglong2 ldg_stream_u128(const uint64_t *p) {
  ulonglong2 v;
  asm volatile("ld.global.cs.v2.u64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p));
  return v;
}

__device__ __forceinline__ float ldg_stream_f32(const float *p) {
  float v;
  asm volatile("ld.global.cs.f32 %0, [%1];" : "=f"(v) : "l"(p));
  return v;
}

__device__ __forceinline__ float bf16lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf16hi(uint32_t u) { return __uint_as_float(u & 0xFFFF0000u); }

// Process-wide count of kernels launched by the library (api.cu).
void note_launches(int n);

}  // namespace alto
