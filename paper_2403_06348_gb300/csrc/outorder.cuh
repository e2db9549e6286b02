// MTTKRP with output-oriented traversal (Alg. 4, the pos_out branch),
// included by the per-mode-count instantiation units out_n*.cu.
//
// The stored order (pos_out / val_out of Alg. 4: the line positions and values
// of every segment's nonzeros by increasing output coordinate) puts nonzeros
// of one output row next to each other. Warps take chunks of 32 * B consecutive entries of pos_out
// (B = out_batches<CPL>()); inside a chunk, each group of tpn = R / CPL lanes
// owns a contiguous piece of tpn * B entries and walks it in B batches of tpn
// nonzeros. The run of equal output row is carried in registers across
// the batches of the piece and leaves with one vector atomic per run (the
// paper's boundary update), so the number of global updates is the number of
// distinct rows per piece instead of the number of nonzeros. No shared memory.
#pragma once

#include "mttkrp_kernel.cuh"

namespace alto {

// Batches per piece at 4 columns per lane; 8-column lanes (half the lanes per
// nonzero) take twice as many, so a piece holds 4 R entries either way.
#ifndef ALTO_OUT_BATCHES
#define ALTO_OUT_BATCHES 16
#endif
#ifndef ALTO_OUT_UNROLL
#define ALTO_OUT_UNROLL 2  // rounds (nonzeros of a group) unrolled together
#endif
#ifndef ALTO_OUT_MIN_BLOCKS
#define ALTO_OUT_MIN_BLOCKS 0  // 0: as the segment kernel (3 CTAs per SM, 2 for 8 columns)
#endif
constexpr int kOutUnroll = ALTO_OUT_UNROLL;
#ifndef ALTO_OUT_PREFETCH
#define ALTO_OUT_PREFETCH 1  // steps of the nonzero stream in flight per warp (deeper rings spill)
#endif
constexpr int kOutPrefetch = ALTO_OUT_PREFETCH;

template <int CPL>
constexpr int out_batches() {
  return ALTO_OUT_BATCHES * (CPL / 4);
}
// entries are 32-bit and a chunk may run up to one chunk past the end
static_assert(32ull * ALTO_OUT_BATCHES * 2 <= 0xFFFFFFFFull - kPosOutMaxNnz, "chunk overruns 32 bits");

// A run of at least kStageMinRun nonzeros may belong to a hot row whose runs
// span many pieces: it is looked up in the staged table (shared memory) and
// added there if found. Shorter runs go straight to the output; the lookup
// stays off the path of the many short runs of cold rows.
constexpr int kStageMinRun = 8;

template <int CPL>
__device__ __forceinline__ void flush_out_run(const float (&run)[CPL], uint32_t row, int n, bool staged,
                                              const uint64_t *htab, const MttkrpArgs &a, float *temp,
                                              int sub, int tpn, int grp) {
  const int slot = (staged && n >= kStageMinRun) ? hot_lookup(htab, a.hbits, row) : -1;
  flush_run<CPL>(run, row, slot, temp, a.out, a.R, sub, tpn, grp);
}

// APR != kAprOff computes the CP-APR model update Phi (Alg. 5) with the same
// traversal: the group's Khatri-Rao row (gathered, or row x of the
// precomputed Pi, x the nonzero's line position) dotted with B(i_n, :) over
// the group's lanes, and the run receives v / max(dot, eps) * krp.
template <int NT, int KW, int CPL, bool BF16, int APR = kAprOff>
__global__ void __launch_bounds__(kMttkrpThreads,
                                  ALTO_OUT_MIN_BLOCKS ? ALTO_OUT_MIN_BLOCKS : mttkrp_min_blocks<CPL>())
    mttkrp_out_kernel(const __grid_constant__ MttkrpArgs a) {
  static_assert(APR == kAprOff || (CPL == 4 && !BF16), "Phi uses 4 fp32 columns per lane");
  if (APR != kAprOff && a.skip && *a.skip) return;  // CP-APR inner loop already converged
  constexpr int NMAX = NT ? NT : kMaxModes;
  constexpr int NIN = NMAX > 1 ? NMAX - 1 : 1;
  constexpr int kOutBatches = out_batches<CPL>();
  const int N = NT ? NT : a.dp.nmodes;
  const int R = a.R;
  const int tpn = R / CPL;
  const int lane = threadIdx.x & 31;
  const int grp = lane / tpn, sub = lane - grp * tpn;
  const int ro = a.out_rank;
  const unsigned full = 0xffffffffu;
  const uint32_t rowb = (uint32_t)R * (BF16 ? 2u : 4u);
  const uint32_t inb = lane_byte_offset<CPL, BF16>(sub);
  const char *fb[NIN];
#pragma unroll
  for (int k = 0; k < NIN; ++k) fb[k] = static_cast<const char *>(a.fin[k]) + inb;

  // The sampled hot rows of the mode are staged in shared memory for the
  // whole launch: a Zipf head spans thousands of pieces, and adding each
  // piece's run to global memory would chain that many fp32 additions.
  extern __shared__ __align__(16) unsigned char sm[];
  float *temp = reinterpret_cast<float *>(sm);
  uint64_t *htab = reinterpret_cast<uint64_t *>(temp + (size_t)a.nslots * R);
  const bool staged = a.nslots > 0;
  // the byte table of the one-word decode follows the hot-row table
  const bool use_lut = KW == 1 && a.lut != nullptr;
  uint64_t *lut = htab + ((size_t)1 << a.hbits);
  if (use_lut) {
    for (int i = threadIdx.x; i < kLutEntries; i += blockDim.x) lut[i] = a.lut[i];
    if (!staged) __syncthreads();
  }
  if (staged) {
    const int hsize = 1 << a.hbits;
    for (int i = threadIdx.x; i < hsize; i += blockDim.x) htab[i] = a.htab[i];
    for (int i = threadIdx.x; i < a.nslots * R; i += blockDim.x) temp[i] = 0.f;
    __syncthreads();
  }

  // 32-bit entry arithmetic: pos_out exists only for nnz <= kPosOutMaxNnz
  const uint32_t nnz = (uint32_t)a.nnz;
  const uint32_t warp_id = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const uint32_t nwarps = (gridDim.x * blockDim.x) >> 5;
  constexpr uint32_t chunk = 32u * kOutBatches;
  const uint32_t nchunks = (nnz + chunk - 1) / chunk;
  const uint32_t piece = (uint32_t)tpn * kOutBatches;

  // The warp's steps t = 0, 1, ... are (chunk warp_id + (t / B) nwarps,
  // batch t % B); the entries of the next kOutPrefetch steps are in flight
  // while a step is processed (a ring shifted by one each step).
  auto step_pos = [&](uint32_t t, uint32_t &p) -> bool {
    const uint32_t c = warp_id + (t / (uint32_t)kOutBatches) * nwarps;
    p = c * chunk + (uint32_t)grp * piece + (uint32_t)sub + (t % (uint32_t)kOutBatches) * (uint32_t)tpn;
    return c < nchunks && p < nnz;
  };
  uint64_t qlo[kOutPrefetch], qhi[kOutPrefetch];
  float qv[kOutPrefetch];
  uint32_t qx[kOutPrefetch];  // PRE: the nonzero's line position (its row of Pi)
  auto load_step = [&](uint32_t t, int slot) {
    uint32_t p;
    qlo[slot] = 0;
    qhi[slot] = 0;
    qv[slot] = 0.f;
    qx[slot] = 0;
    if (step_pos(t, p)) {
      if (KW == 1) {
        qlo[slot] = __ldcs(reinterpret_cast<const unsigned long long *>(a.keys) + p);
      } else {
        const ulonglong2 kk = __ldcs(reinterpret_cast<const ulonglong2 *>(a.keys) + p);
        qlo[slot] = kk.x;
        qhi[slot] = kk.y;
      }
      qv[slot] = __ldcs(a.vals + p);
      if (APR == kAprPre) qx[slot] = __ldcs(a.perm + p);
    }
  };
  uint32_t t_next = 0;
#pragma unroll
  for (int d = 0; d < kOutPrefetch; ++d) load_step(t_next++, d);

  for (uint32_t ch = warp_id; ch < nchunks; ch += nwarps) {
    // entry of the stored order this lane uses in batch b: p0 + b * tpn
    // (a.keys / a.vals hold the line positions and values in that order)
    const uint32_t p0 = ch * chunk + (uint32_t)grp * piece + (uint32_t)sub;

    float run[CPL];
#pragma unroll
    for (int c = 0; c < CPL; ++c) run[c] = 0.f;
    uint32_t run_row = kEmptyRow;
    int run_n = 0;  // nonzeros in the run
    for (int b = 0; b < kOutBatches; ++b) {
      const bool valid = p0 + (uint32_t)(b * tpn) < nnz;
      const uint64_t lo = qlo[0], hi = qhi[0];
      const float v = qv[0];
      const uint32_t xb = qx[0];
#pragma unroll
      for (int d = 0; d + 1 < kOutPrefetch; ++d) {
        qlo[d] = qlo[d + 1];
        qhi[d] = qhi[d + 1];
        qv[d] = qv[d + 1];
        qx[d] = qx[d + 1];
      }
      load_step(t_next++, kOutPrefetch - 1);
      uint32_t c[NMAX];
      if (use_lut)
        decode_lut<NMAX>(lut, a.lp, lo, c);
      else if constexpr (NT > 0)
        decode_blocks<KW, NMAX, 0>(a.bp, lo, hi, c);
      else
        decode_runs<KW, NMAX>(a.dp, N, lo, hi, c);
      uint32_t row = c[0];
      uint32_t in[NIN];
#pragma unroll
      for (int n = 1; n < NMAX; ++n)
        if (n == ro) row = c[n];
#pragma unroll
      for (int k = 0; k < NIN; ++k) in[k] = (NMAX > 1 && k + 1 < NMAX) ? (k < ro ? c[k] : c[k + 1]) : 0u;
      const unsigned live = __ballot_sync(full, valid);
      if (!live) continue;  // past the end (last chunk); the step ring stays in order
#pragma unroll(CPL <= 8 ? kOutUnroll : 1)
      for (int q = 0; q < tpn; ++q) {
        const int j = grp * tpn + q;
        const float vj = __shfl_sync(full, v, j);
        const uint32_t rj = __shfl_sync(full, row, j);
        uint32_t ij[NIN];
#pragma unroll
        for (int k = 0; k < NIN; ++k)
          ij[k] = (APR != kAprPre && k + 1 < N) ? __shfl_sync(full, in[k], j) : 0u;
        const bool live_j = (live >> j) & 1u;
        float p[CPL];
        if constexpr (APR != kAprOff) {
          float kr[4] = {1.f, 1.f, 1.f, 1.f};
          if (APR == kAprPre) {
            const uint32_t xj = __shfl_sync(full, xb, j);
            if (live_j) {
              const float4 qv = __ldg(reinterpret_cast<const float4 *>(a.pimat) +
                                      (uint64_t)xj * (uint64_t)(R / 4) + sub);
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
          const float4 bv = __ldg(reinterpret_cast<const float4 *>(a.bmat) + (uint64_t)rj * (R / 4) + sub);
          float dot = kr[0] * bv.x + kr[1] * bv.y + kr[2] * bv.z + kr[3] * bv.w;
          for (int o = 1; o < tpn; o <<= 1) dot += __shfl_xor_sync(full, dot, o);
          if (!live_j) continue;
          const float scale = vj / fmaxf(dot, a.eps);
#pragma unroll
          for (int cc = 0; cc < 4; ++cc) p[cc] = scale * kr[cc];
        } else {
          if (!live_j) continue;
          gather_product<NMAX, CPL, BF16>(fb, ij, rowb, tpn, N, vj, p);
        }
        if (rj == run_row) {
#pragma unroll
          for (int cc = 0; cc < CPL; ++cc) run[cc] += p[cc];
          ++run_n;
        } else {
          if (run_row != kEmptyRow) flush_out_run<CPL>(run, run_row, run_n, staged, htab, a, temp, sub, tpn, grp);
#pragma unroll
          for (int cc = 0; cc < CPL; ++cc) run[cc] = p[cc];
          run_row = rj;
          run_n = 1;
        }
      }
    }
    if (run_row != kEmptyRow) flush_out_run<CPL>(run, run_row, run_n, staged, htab, a, temp, sub, tpn, grp);
  }
  if (staged) {  // the staged hot rows leave once per CTA
    __syncthreads();
    const float4 *t4 = reinterpret_cast<const float4 *>(temp);
    const int n4 = a.nslots * R / 4;
    const int per_row = R / 4;
    for (int i = threadIdx.x; i < n4; i += blockDim.x) {
      const float4 t = t4[i];
      if (t.x != 0.f || t.y != 0.f || t.z != 0.f || t.w != 0.f) {
        const int sl = i / per_row, c4 = ((i - sl * per_row) * 4) ^ slot_swizzle(sl, R);
        red_v4(a.out + (uint64_t)a.slot_rows[sl] * (uint64_t)R + c4, t.x, t.y, t.z, t.w);
      }
    }
  }
}

template <int NT, int KW, int CPL, bool BF16, int APR = kAprOff>
static cudaError_t launch_out_one(const MttkrpArgs &a, size_t smem, int num_sms, cudaStream_t s) {
  auto kern = mttkrp_out_kernel<NT, KW, CPL, BF16, APR>;
  static int configured = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mttkrp_smem_limit());
    if (e != cudaSuccess) return e;
    configured = 1;
  }
  constexpr uint64_t chunk = 32ull * out_batches<CPL>();
  const uint64_t chunks = (a.nnz + chunk - 1) / chunk;
  const uint64_t warps_per_cta = kMttkrpThreads / 32;
  uint64_t grid = (uint64_t)num_sms * resident_ctas(kern, smem);
  const uint64_t need = (chunks + warps_per_cta - 1) / warps_per_cta;
  if (grid > need) grid = need;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, kMttkrpThreads, smem, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

template <int NT>
cudaError_t launch_mttkrp_out_nt(const MttkrpArgs &a, int cpl, bool bf16, size_t smem, int num_sms,
                                 cudaStream_t s) {
  if (a.dp.kw == 1) {
    if (cpl == 8) return bf16 ? launch_out_one<NT, 1, 8, true>(a, smem, num_sms, s)
                              : launch_out_one<NT, 1, 8, false>(a, smem, num_sms, s);
    return bf16 ? launch_out_one<NT, 1, 4, true>(a, smem, num_sms, s)
                : launch_out_one<NT, 1, 4, false>(a, smem, num_sms, s);
  }
  if (cpl == 8) return bf16 ? launch_out_one<NT, 2, 8, true>(a, smem, num_sms, s)
                            : launch_out_one<NT, 2, 8, false>(a, smem, num_sms, s);
  return bf16 ? launch_out_one<NT, 2, 4, true>(a, smem, num_sms, s)
              : launch_out_one<NT, 2, 4, false>(a, smem, num_sms, s);
}

template <int NT>
cudaError_t launch_phi_out_nt(const MttkrpArgs &a, bool pre, size_t smem, int num_sms, cudaStream_t s) {
  if (a.dp.kw == 1)
    return pre ? launch_out_one<NT, 1, 4, false, kAprPre>(a, smem, num_sms, s)
               : launch_out_one<NT, 1, 4, false, kAprOtf>(a, smem, num_sms, s);
  return pre ? launch_out_one<NT, 2, 4, false, kAprPre>(a, smem, num_sms, s)
             : launch_out_one<NT, 2, 4, false, kAprOtf>(a, smem, num_sms, s);
}

}  // namespace alto
