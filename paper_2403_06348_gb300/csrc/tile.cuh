// MTTKRP over the one ALTO copy with the output-oriented traversal of Alg. 4
// done inside each tile of the line, included by the per-mode-count
// instantiation units tile_n*.cu.
//
// Alg. 4's output-oriented branch visits a segment's nonzeros by increasing
// output coordinate, so that the updates of one output row are summed before
// they reach memory. Here no ordered copy is stored: every tile of
// kTileNnz consecutive nonzeros of the ALTO line is regrouped on chip.
//
//  1. The tile's positions and values arrive in shared memory through one
//     bulk asynchronous copy (cp.async.bulk, completion on an mbarrier); the
//     copy of the next tile is in flight while this one is processed.
//  2. Every nonzero is de-linearized once (EXTRACT of Alg. 3) by one thread,
//     and its output row is looked up in the mode's hot-row table (the most
//     frequent rows, sampled at encode time).
//  3. GROUP: a counting sort over bins (one per hot row, one for all other
//     rows) makes the nonzeros of each hot row consecutive; the other rows
//     keep line order. Without GROUP the tile stays in line order.
//  4. The decoded records (output row code, input coordinates, value) are
//     written to shared memory; each group of R / CPL lanes walks a
//     contiguous piece of them, gathers the N-1 input rows (CPL columns per
//     lane, 16- or 32-byte loads), multiplies in packed f32x2 arithmetic and
//     carries the run of equal output rows in registers.
//  5. A run leaves when its row changes: staged hot rows (the first nslots)
//     into shared memory, flushed once per CTA at the end; the remaining hot
//     rows ("warm") into one of kWarmReps fp64 replicas (fp64 atomics; a
//     small kernel adds the replicas into the output afterwards): a warm row
//     takes an addition from every tile that holds it, too long a chain for
//     fp32; all other rows straight into the output (red.global.add.v4.f32).
#pragma once

#include "mttkrp_kernel.cuh"
#include "async_copy.cuh"

namespace alto {

constexpr int kTileThreads = 512;
#ifndef ALTO_TILE_NPT
#define ALTO_TILE_NPT 4
#endif
constexpr int kTileNpt = ALTO_TILE_NPT;                 // nonzeros decoded per thread
constexpr int kTileNnz = kTileThreads * kTileNpt;      // nonzeros per tile
constexpr uint32_t kHotCode = 0x80000000u;             // record row code of a hot row
constexpr int kWarmReps = kTileWarmReps;               // fp32 replicas of the warm rows

// Record: output row code, the N-1 input coordinates (rank order without
// the output rank) and the value, padded to 16-byte multiples.
template <int NMAX>
constexpr int tile_rec_words() {
  return NMAX + 1 <= 4 ? 4 : (NMAX + 1 <= 8 ? 8 : 12);
}

__host__ __device__ constexpr uint32_t tile_round(uint32_t x, uint32_t a) { return (x + a - 1) / a * a; }

// Shared-memory layout of one CTA (host and device compute the same).
struct TileLayout {
  uint32_t buf;    // bytes of one of the two tile buffers (raw tile, then records)
  uint32_t stage;  // staged hot rows [nslots][R] fp32
  uint32_t htab;   // hot-row hash table [2^hbits] (slot << 32 | row)
  uint32_t bins;   // bin counts / offsets [nbins + 1] and 32 scan words
  uint32_t bar;    // two mbarriers
  uint32_t lut;    // byte-table decode [8][256] (one-word positions), if used
  uint32_t total;
};

// ngroups = groups of R / CPL lanes per CTA: the record slots hold the tile
// plus one skew slot per group (and one spare).
__host__ __device__ inline TileLayout tile_layout(int kw, int rec_bytes, int ngroups, int R, int nslots,
                                                  int hbits, int nbins, bool lut) {
  TileLayout L{};
  const uint32_t raw = (uint32_t)kTileNnz * (8u * kw + 4u);
  const uint32_t rec = ((uint32_t)kTileNnz + (uint32_t)ngroups + 1u) * (uint32_t)rec_bytes;
  L.buf = tile_round(raw > rec ? raw : rec, 128);
  L.stage = 2 * L.buf;
  L.htab = L.stage + tile_round((uint32_t)nslots * (uint32_t)R * 4u, 16);
  L.bins = L.htab + (1u << hbits) * 8u;
  L.bar = tile_round(L.bins + ((uint32_t)nbins + 1u + 32u) * 4u, 16);
  L.lut = L.bar + 16;
  L.total = L.lut + (lut ? (uint32_t)kLutBytes : 0u);
  return L;
}

constexpr uint64_t kTileWaitNs = 2000000000ull;  // 2 s: a tile copy takes microseconds

__device__ __forceinline__ unsigned tile_lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// ---------------------------------------------------------------------------
// Packed f32x2 arithmetic (two fp32 lanes per 64-bit register pair)
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t f2_mul(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_fma(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t f2_add(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}
__device__ __forceinline__ uint64_t f2_splat(float v) {
  const uint64_t u = __float_as_uint(v);
  return u | (u << 32);
}
__device__ __forceinline__ float f2_lo(uint64_t a) { return __uint_as_float((uint32_t)a); }
__device__ __forceinline__ float f2_hi(uint64_t a) { return __uint_as_float((uint32_t)(a >> 32)); }

// bf16 pair (low half first) -> packed fp32 pair.
__device__ __forceinline__ uint64_t bf2_to_f2(uint32_t u) {
  return (uint64_t)(u << 16) | ((uint64_t)(u & 0xFFFF0000u) << 32);
}

// This lane's CPL consecutive columns (starting at column CPL * sub) of one
// factor row as CPL / 2 packed pairs; rb points at the lane's first column.
template <int CPL, bool BF16>
__device__ __forceinline__ void load_row_f2(const char *rb, uint64_t (&f)[CPL / 2]) {
  if constexpr (!BF16 && CPL == 8) {
    asm("ld.global.nc.v4.u64 {%0, %1, %2, %3}, [%4];"
        : "=l"(f[0]), "=l"(f[1]), "=l"(f[2]), "=l"(f[3])
        : "l"(rb));
  } else if constexpr (!BF16 && CPL == 4) {
    asm("ld.global.nc.v2.u64 {%0, %1}, [%2];" : "=l"(f[0]), "=l"(f[1]) : "l"(rb));
  } else if constexpr (BF16 && CPL == 8) {
    uint32_t q0, q1, q2, q3;
    asm("ld.global.nc.v4.u32 {%0, %1, %2, %3}, [%4];" : "=r"(q0), "=r"(q1), "=r"(q2), "=r"(q3) : "l"(rb));
    f[0] = bf2_to_f2(q0);
    f[1] = bf2_to_f2(q1);
    f[2] = bf2_to_f2(q2);
    f[3] = bf2_to_f2(q3);
  } else {
    uint32_t q0, q1;
    asm("ld.global.nc.v2.u32 {%0, %1}, [%2];" : "=r"(q0), "=r"(q1) : "l"(rb));
    f[0] = bf2_to_f2(q0);
    f[1] = bf2_to_f2(q1);
  }
}

// A finished run leaves: staged hot row -> shared memory; warm row -> its
// replica; other rows -> the output.
template <int CPL>
__device__ __forceinline__ void tile_flush(const uint64_t (&run)[CPL / 2], uint32_t code,
                                           const MttkrpArgs &a, float *stage, int sub, int tpn, int grp) {
  float f[CPL];
#pragma unroll
  for (int c = 0; c < CPL / 2; ++c) {
    f[2 * c] = f2_lo(run[c]);
    f[2 * c + 1] = f2_hi(run[c]);
  }
  if (code & kHotCode) {
    const int idx = (int)(code & ~kHotCode);
    if (idx < a.nslots) {
      flush_run<CPL>(f, 0u, idx, stage, a.out, a.R, sub, tpn, grp);
      return;
    }
    // fp64: a warm row takes one addition per tile that holds it, tens of
    // thousands on a Zipf head, too long a chain for fp32
    double *w = a.warm + ((size_t)(blockIdx.x % kWarmReps) * (size_t)a.nbins + (size_t)idx) * (size_t)a.R;
#pragma unroll
    for (int c = 0; c < CPL; ++c) atomicAdd(w + CPL * sub + c, (double)f[c]);
    return;
  }
  float *o = a.out + (uint64_t)code * (uint64_t)a.R;
#pragma unroll
  for (int v = 0; v < CPL / 4; ++v)
    red_v4(o + CPL * sub + 4 * v, f[4 * v], f[4 * v + 1], f[4 * v + 2], f[4 * v + 3]);
}

// Gathers this lane's columns of the N-1 input rows of record w.
template <int NT, int CPL, bool BF16, int NIN>
__device__ __forceinline__ void tile_gather(const uint32_t *w, const char *const (&fb)[NIN], uint32_t rowb,
                                            uint64_t (&g)[NIN][CPL / 2]) {
#pragma unroll
  for (int q = 0; q < NIN; ++q) load_row_f2<CPL, BF16>(fb[q] + (uint64_t)w[1 + q] * rowb, g[q]);
}

// Reads the RW words of a record.
template <int RW>
__device__ __forceinline__ void tile_rec(const uint32_t *rp, uint32_t (&w)[RW]) {
#pragma unroll
  for (int q = 0; q < RW / 4; ++q) {
    const uint4 u = reinterpret_cast<const uint4 *>(rp)[q];
    w[4 * q] = u.x;
    w[4 * q + 1] = u.y;
    w[4 * q + 2] = u.z;
    w[4 * q + 3] = u.w;
  }
}

// Walks n records starting at rp, stride `step` records. MERGE: runs of
// equal row code are summed in registers and leave when the code changes;
// otherwise every record leaves on its own (rows without a hot code go
// straight to the output).
template <int NT, int CPL, bool BF16, int RW, bool MERGE, int NIN>
__device__ __forceinline__ void tile_walk(const uint32_t *rp, int step, int n, const char *const (&fb)[NIN],
                                          uint32_t rowb, int N, const MttkrpArgs &a, float *stage, int sub,
                                          int tpn, int grp) {
  uint64_t run[CPL / 2];
#pragma unroll
  for (int c = 0; c < CPL / 2; ++c) run[c] = 0ull;
  uint32_t run_code = kEmptyRow;
  if constexpr (NT > 0) {
#pragma unroll 2
    for (int i = 0; i < n; ++i) {
      uint32_t w[RW];
      tile_rec<RW>(rp + (size_t)i * step * RW, w);
      uint64_t g[NIN][CPL / 2];
      tile_gather<NT, CPL, BF16, NIN>(w, fb, rowb, g);
      // t = v * A_0 ... A_{N-3}; contribution = t * A_{N-2}
      uint64_t tv[CPL / 2];
      const uint64_t vv = f2_splat(__uint_as_float(w[RW - 1]));
#pragma unroll
      for (int c = 0; c < CPL / 2; ++c) tv[c] = vv;
#pragma unroll
      for (int q = 0; q + 1 < NIN; ++q)
#pragma unroll
        for (int c = 0; c < CPL / 2; ++c) tv[c] = f2_mul(tv[c], g[q][c]);
      if constexpr (MERGE) {
        if (w[0] != run_code) {
          if (run_code != kEmptyRow) tile_flush<CPL>(run, run_code, a, stage, sub, tpn, grp);
#pragma unroll
          for (int c = 0; c < CPL / 2; ++c) run[c] = 0ull;
          run_code = w[0];
        }
#pragma unroll
        for (int c = 0; c < CPL / 2; ++c) run[c] = f2_fma(tv[c], g[NIN - 1][c], run[c]);
      } else {
        uint64_t pr[CPL / 2];
#pragma unroll
        for (int c = 0; c < CPL / 2; ++c) pr[c] = f2_mul(tv[c], g[NIN - 1][c]);
        float *o = a.out + (uint64_t)w[0] * (uint64_t)a.R + CPL * sub;
#pragma unroll
        for (int v = 0; v < CPL / 4; ++v)
          red_v4(o + 4 * v, f2_lo(pr[2 * v]), f2_hi(pr[2 * v]), f2_lo(pr[2 * v + 1]), f2_hi(pr[2 * v + 1]));
      }
    }
  } else {
    for (int i = 0; i < n; ++i) {
      uint32_t w[RW];
      tile_rec<RW>(rp + (size_t)i * step * RW, w);
      uint64_t tv[CPL / 2];
      const uint64_t vv = f2_splat(__uint_as_float(w[RW - 1]));
#pragma unroll
      for (int c = 0; c < CPL / 2; ++c) tv[c] = vv;
#pragma unroll
      for (int q = 0; q < NIN; ++q) {
        if (q + 1 < N) {
          uint64_t f[CPL / 2];
          load_row_f2<CPL, BF16>(fb[q] + (uint64_t)w[1 + q] * rowb, f);
#pragma unroll
          for (int c = 0; c < CPL / 2; ++c) tv[c] = f2_mul(tv[c], f[c]);
        }
      }
      if (MERGE) {
        if (w[0] != run_code) {
          if (run_code != kEmptyRow) tile_flush<CPL>(run, run_code, a, stage, sub, tpn, grp);
#pragma unroll
          for (int c = 0; c < CPL / 2; ++c) run[c] = 0ull;
          run_code = w[0];
        }
#pragma unroll
        for (int c = 0; c < CPL / 2; ++c) run[c] = f2_add(run[c], tv[c]);
      } else {
        float *o = a.out + (uint64_t)w[0] * (uint64_t)a.R + CPL * sub;
#pragma unroll
        for (int v = 0; v < CPL / 4; ++v)
          red_v4(o + 4 * v, f2_lo(tv[2 * v]), f2_hi(tv[2 * v]), f2_lo(tv[2 * v + 1]), f2_hi(tv[2 * v + 1]));
      }
    }
  }
  if (MERGE && run_code != kEmptyRow) tile_flush<CPL>(run, run_code, a, stage, sub, tpn, grp);
}

// ---------------------------------------------------------------------------
// The kernel
// ---------------------------------------------------------------------------
template <int NT, int KW, int CPL, bool BF16, bool GROUP>
__global__ void __launch_bounds__(kTileThreads, 2) mttkrp_tile_kernel(const __grid_constant__ MttkrpArgs a) {
  constexpr int NMAX = NT ? NT : kMaxModes;
  constexpr int NIN = NMAX > 1 ? NMAX - 1 : 1;
  constexpr int RW = tile_rec_words<NMAX>();
  const int N = NT ? NT : a.dp.nmodes;
  const int R = a.R;
  const int tpn = R / CPL;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int grp = lane / tpn, sub = lane - grp * tpn;
  const int ro = a.out_rank;
  const unsigned full = 0xffffffffu;
  const bool use_lut = KW == 1 && a.lut != nullptr;
  const TileLayout lay = tile_layout(KW, RW * 4, kTileThreads / tpn, R, a.nslots, a.hbits, a.nbins, use_lut);

  extern __shared__ __align__(16) unsigned char sm[];
  float *stage = reinterpret_cast<float *>(sm + lay.stage);
  uint64_t *htab = reinterpret_cast<uint64_t *>(sm + lay.htab);
  uint32_t *bins = reinterpret_cast<uint32_t *>(sm + lay.bins);
  uint32_t *scan_w = bins + a.nbins + 1;
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + lay.bar);
  uint64_t *lut = reinterpret_cast<uint64_t *>(sm + lay.lut);
  if (use_lut)
    for (int i = tid; i < kLutEntries; i += kTileThreads) lut[i] = a.lut[i];

  const int hsize = 1 << a.hbits;
  for (int i = tid; i < hsize; i += kTileThreads) htab[i] = a.htab[i];
  for (int i = tid; i < a.nslots * R; i += kTileThreads) stage[i] = 0.f;
  for (int i = tid; i <= a.nbins; i += kTileThreads) bins[i] = 0u;

  const uint64_t ntiles = (a.nnz + kTileNnz - 1) / kTileNnz;
  const uint64_t nfull = a.nnz / kTileNnz;
  constexpr uint32_t kKeyBytes = (uint32_t)kTileNnz * 8u * KW;
  constexpr uint32_t kValBytes = (uint32_t)kTileNnz * 4u;
  auto issue = [&](uint64_t t, int b) {
    unsigned char *buf = sm + (size_t)b * lay.buf;
    mbar_expect_tx(&bar[b], kKeyBytes + kValBytes);
    bulk_g2s(buf, a.keys + t * (uint64_t)kTileNnz * KW, kKeyBytes, &bar[b]);
    bulk_g2s(buf + kKeyBytes, a.vals + t * (uint64_t)kTileNnz, kValBytes, &bar[b]);
  };
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
    if ((uint64_t)blockIdx.x < nfull) issue(blockIdx.x, 0);
  }
  __syncthreads();

  // the N-1 input factors plus this lane's byte offset
  const uint32_t rowb = (uint32_t)R * (BF16 ? 2u : 4u);
  const char *fb[NIN];
#pragma unroll
  for (int k = 0; k < NIN; ++k)
    fb[k] = static_cast<const char *>(a.fin[k]) + (uint32_t)(CPL * sub) * (BF16 ? 2u : 4u);

  uint32_t parity = 0;  // bit b: phase of bar[b] to wait for
  int it = 0;
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++it) {
    const int b = it & 1;
    unsigned char *buf = sm + (size_t)b * lay.buf;
    const uint64_t s0 = t * (uint64_t)kTileNnz;
    const int cnt = (int)((a.nnz - s0) < (uint64_t)kTileNnz ? (a.nnz - s0) : (uint64_t)kTileNnz);
    const bool bulk = t < nfull;
    bool ok = true;
    const uint32_t ph = (parity >> b) & 1u;
    if (bulk) {
      ok = mbar_wait_bounded(&bar[b], ph, kTileWaitNs);
      parity ^= 1u << b;
    }
    // every thread has left the previous tile (its buffer is free again)
    if (!__syncthreads_and(ok)) {
      // this tile's copy (the only one in flight) did not complete: report
      // it, give the copy one more bounded wait so that it does not land in
      // the shared memory of a finished CTA, and stop
      if (tid == 0) {
        atomicOr(a.status, kStatusTimeout);
        mbar_wait_bounded(&bar[b], ph, kTileWaitNs);
      }
      return;
    }
    if (tid == 0 && t + gridDim.x < nfull) {
      fence_proxy_async_smem();  // generic reads of buffer b^1 before the async write
      issue(t + gridDim.x, b ^ 1);
    }

    // ---- decode (EXTRACT of Alg. 3), hot-row lookup --------------------
    uint32_t code[kTileNpt];
    uint32_t inr[kTileNpt][NIN];
    float val[kTileNpt];
#pragma unroll
    for (int k = 0; k < kTileNpt; ++k) {
      const int x = tid + k * kTileThreads;
      uint64_t lo = 0, hi = 0;
      float v = 0.f;
      if (x < cnt) {
        if (bulk) {
          if (KW == 1) {
            lo = reinterpret_cast<const uint64_t *>(buf)[x];
          } else {
            const ulonglong2 kk = reinterpret_cast<const ulonglong2 *>(buf)[x];
            lo = kk.x;
            hi = kk.y;
          }
          v = reinterpret_cast<const float *>(buf + kKeyBytes)[x];
        } else {
          if (KW == 1) {
            lo = __ldcs(reinterpret_cast<const unsigned long long *>(a.keys) + s0 + x);
          } else {
            const ulonglong2 kk = __ldcs(reinterpret_cast<const ulonglong2 *>(a.keys) + s0 + x);
            lo = kk.x;
            hi = kk.y;
          }
          v = __ldcs(a.vals + s0 + x);
        }
      }
      uint32_t c[NMAX];
      if (use_lut)
        decode_lut<NMAX>(lut, a.lp, lo, c);
      else if constexpr (NT > 0)
        decode_blocks<KW, NMAX, 0>(a.bp, lo, hi, c);
      else
        decode_runs<KW, NMAX>(a.dp, N, lo, hi, c);
      uint32_t row = c[0];
#pragma unroll
      for (int n = 1; n < NMAX; ++n)
        if (n == ro) row = c[n];
#pragma unroll
      for (int q = 0; q < NIN; ++q) inr[k][q] = (NMAX > 1 && q + 1 < NMAX) ? (q < ro ? c[q] : c[q + 1]) : 0u;
      int idx = -1;
      if (x < cnt && a.nbins > 0) idx = hot_lookup(htab, a.hbits, row);
      code[k] = idx >= 0 ? (kHotCode | (uint32_t)idx) : row;
      val[k] = v;
    }

    uint32_t pos[kTileNpt];
    uint32_t bins_hot_count = 0;
    if constexpr (GROUP) {
      // ---- counting sort by bin: hot row idx -> bin idx, others -> nbins --
      uint32_t rank[kTileNpt], bin[kTileNpt];
#pragma unroll
      for (int k = 0; k < kTileNpt; ++k) {
        const int x = tid + k * kTileThreads;
        bin[k] = x < cnt ? ((code[k] & kHotCode) ? (code[k] & ~kHotCode) : (uint32_t)a.nbins) : 0xFFFFFFFFu;
        const unsigned peers = __match_any_sync(full, bin[k]);
        const int leader = __ffs(peers) - 1;
        uint32_t base = 0;
        if (lane == leader && bin[k] != 0xFFFFFFFFu) base = atomicAdd(&bins[bin[k]], (uint32_t)__popc(peers));
        base = __shfl_sync(full, base, leader);
        rank[k] = base + (uint32_t)__popc(peers & tile_lanemask_lt());
      }
      __syncthreads();
      // exclusive scan of bins[0..nbins] in place: each thread a contiguous
      // chunk, warp scan of the chunk sums, then the warps' totals
      const int nb = a.nbins + 1;
      const int per = (nb + kTileThreads - 1) / kTileThreads;
      const int i0 = tid * per;
      uint32_t sum = 0;
      for (int i = i0; i < i0 + per && i < nb; ++i) sum += bins[i];
      uint32_t incl = sum;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(full, incl, o);
        if (lane >= o) incl += y;
      }
      if (lane == 31) scan_w[warp] = incl;
      __syncthreads();
      uint32_t wt = lane < kTileThreads / 32 ? scan_w[lane] : 0u;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        const uint32_t y = __shfl_up_sync(full, wt, o);
        if (lane >= o) wt += y;
      }
      const uint32_t wbase = __shfl_sync(full, wt, (warp + 31) & 31) * (warp > 0 ? 1u : 0u);
      uint32_t run_off = wbase + incl - sum;
      for (int i = i0; i < i0 + per && i < nb; ++i) {
        const uint32_t c0 = bins[i];
        bins[i] = run_off;
        run_off += c0;
      }
      __syncthreads();
      bins_hot_count = bins[a.nbins];  // records of hot rows (they sort first)
#pragma unroll
      for (int k = 0; k < kTileNpt; ++k) {
        const int x = tid + k * kTileThreads;
        pos[k] = x < cnt ? bins[bin[k]] + rank[k] : 0u;
      }
    } else {
      __syncthreads();  // the raw tile is read before records overwrite it
#pragma unroll
      for (int k = 0; k < kTileNpt; ++k) pos[k] = (uint32_t)(tid + k * kTileThreads);
    }
    // ---- records into the tile buffer -----------------------------------
    // Sorted order (GROUP): hot bins [0, nhot) first, then the other rows;
    // in line order (no GROUP) the whole tile is the merged part. Group g
    // walks the contiguous piece [g * hpiece, (g + 1) * hpiece) of the hot part
    // (runs merged; piece g skewed by g slots so that the groups of a warp
    // read different banks) and the records nhot + g, nhot + g + G, ... of
    // the rest (one update each; consecutive groups read consecutive slots).
    const int ngroups = kTileThreads / tpn;
    const int nhot = GROUP ? (int)bins_hot_count : cnt;  // line order: one merged part
    const int hpiece = (nhot + ngroups - 1) / ngroups;
    const int cold_base = nhot + (hpiece ? (nhot + hpiece - 1) / hpiece : 0);
    uint32_t *rec = reinterpret_cast<uint32_t *>(buf);
#pragma unroll
    for (int k = 0; k < kTileNpt; ++k) {
      const int x = tid + k * kTileThreads;
      if (x < cnt) {
        const int pk = (int)pos[k];
        const int phys = pk < nhot ? pk + pk / hpiece : cold_base + (pk - nhot);
        uint32_t w[RW];
        w[0] = code[k];
#pragma unroll
        for (int q = 0; q < NIN; ++q) w[1 + q] = inr[k][q];
#pragma unroll
        for (int q = NIN + 1; q < RW - 1; ++q) w[q] = 0u;
        w[RW - 1] = __float_as_uint(val[k]);
        uint4 *dst = reinterpret_cast<uint4 *>(rec + (size_t)phys * RW);
#pragma unroll
        for (int q = 0; q < RW / 4; ++q) dst[q] = make_uint4(w[4 * q], w[4 * q + 1], w[4 * q + 2], w[4 * q + 3]);
      }
    }
    __syncthreads();
    if constexpr (GROUP) {
      for (int i = tid; i <= a.nbins; i += kTileThreads) bins[i] = 0u;  // for the next tile
    }

    // ---- gather, multiply, merge runs (Alg. 4 output-oriented updates) --
    const int gw = warp * (32 / tpn) + grp;
    if (nhot > 0) {
      const int j0 = gw * hpiece;
      const int j1 = (j0 + hpiece) < nhot ? (j0 + hpiece) : nhot;
      if (j0 < j1)
        tile_walk<NT, CPL, BF16, RW, true>(rec + (size_t)(j0 + gw) * RW, 1, j1 - j0, fb, rowb, N, a, stage,
                                           sub, tpn, grp);
    }
    if (cnt > nhot) {
      const int c0 = nhot + gw;
      if (c0 < cnt)
        tile_walk<NT, CPL, BF16, RW, false>(rec + (size_t)(cold_base + gw) * RW, ngroups,
                                            (cnt - c0 + ngroups - 1) / ngroups, fb, rowb, N, a, stage, sub,
                                            tpn, grp);
    }
  }

  // the staged hot rows leave once per CTA
  if (a.nslots > 0) {
    __syncthreads();
    const float4 *t4 = reinterpret_cast<const float4 *>(stage);
    const int n4 = a.nslots * R / 4;
    const int per_row = R / 4;
    for (int i = tid; i < n4; i += kTileThreads) {
      const float4 v4 = t4[i];
      if (v4.x != 0.f || v4.y != 0.f || v4.z != 0.f || v4.w != 0.f) {
        const int sl = i / per_row, c4 = ((i - sl * per_row) * 4) ^ slot_swizzle(sl, R);
        red_v4(a.out + (uint64_t)a.slot_rows[sl] * (uint64_t)R + c4, v4.x, v4.y, v4.z, v4.w);
      }
    }
  }
}

template <int NT, int KW, int CPL, bool BF16, bool GROUP>
static cudaError_t launch_tile_one(const MttkrpArgs &a, int num_sms, cudaStream_t s) {
  auto kern = mttkrp_tile_kernel<NT, KW, CPL, BF16, GROUP>;
  constexpr int RW = tile_rec_words<NT ? NT : kMaxModes>();
  const TileLayout lay = tile_layout(KW, RW * 4, kTileThreads / (a.R / CPL), a.R, a.nslots, a.hbits, a.nbins,
                                     KW == 1 && a.lut != nullptr);
  static int configured = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mttkrp_smem_limit());
    if (e != cudaSuccess) return e;
    configured = 1;
  }
  int per_sm = 0;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kTileThreads, lay.total) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  if (per_sm < 1) per_sm = 1;
  const uint64_t ntiles = (a.nnz + kTileNnz - 1) / kTileNnz;
  uint64_t grid = (uint64_t)num_sms * (uint64_t)per_sm;
  if (grid > ntiles) grid = ntiles;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kTileThreads, lay.total, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

template <int NT, int KW, int CPL>
static cudaError_t launch_tile_kc(const MttkrpArgs &a, bool bf16, bool group, int num_sms, cudaStream_t s) {
  if (bf16)
    return group ? launch_tile_one<NT, KW, CPL, true, true>(a, num_sms, s)
                 : launch_tile_one<NT, KW, CPL, true, false>(a, num_sms, s);
  return group ? launch_tile_one<NT, KW, CPL, false, true>(a, num_sms, s)
               : launch_tile_one<NT, KW, CPL, false, false>(a, num_sms, s);
}

template <int NT>
cudaError_t launch_mttkrp_tile_nt(const MttkrpArgs &a, int cpl, bool bf16, bool group, int num_sms,
                                  cudaStream_t s) {
  if (a.dp.kw == 1)
    return cpl == 8 ? launch_tile_kc<NT, 1, 8>(a, bf16, group, num_sms, s)
                    : launch_tile_kc<NT, 1, 4>(a, bf16, group, num_sms, s);
  return cpl == 8 ? launch_tile_kc<NT, 2, 8>(a, bf16, group, num_sms, s)
                  : launch_tile_kc<NT, 2, 4>(a, bf16, group, num_sms, s);
}

}  // namespace alto
