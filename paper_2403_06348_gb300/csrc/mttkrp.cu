// Mode-agnostic MTTKRP over one ALTO copy (Alg. 3, Alg. 4).
//
// One CTA works on one line segment at a time (persistent over segments).
// Each warp takes 32 consecutive nonzeros of the segment: lane j loads and
// de-linearizes nonzero j (one decode per nonzero), then groups of
// tpn = R / CPL lanes each take tpn consecutive nonzeros of the batch; a lane
// owns CPL consecutive columns, so a group reads whole factor rows with
// coalesced 16-byte loads. Runs of equal output row inside a group are summed
// in registers before they leave the warp.
//
// ATOMIC: hot rows (picked at encode time) accumulate in a shared-memory
//   table found through an open-addressing hash; the table is flushed with
//   vector atomics after every segment. Other rows go straight to the output
//   with red.global.add.v4.f32.
// PULL: the segment's Temp over its mode interval [T^s, T^e] lives in shared
//   memory (index i_mode - T^s), is written out as the segment's partial, and
//   pull_reduce_kernel sums, for every output row b, the partials of the
//   segments whose interval contains b.
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

template <int CPL, bool BF16>
__device__ __forceinline__ void load_factor_row(const void *base, uint32_t row, int R, int col,
                                                float (&f)[CPL]) {
  const uint64_t off = (uint64_t)row * (uint64_t)R + (uint64_t)col;
  if constexpr (!BF16) {
    const float *p = static_cast<const float *>(base) + off;
#pragma unroll
    for (int v = 0; v < CPL / 4; ++v) {
      const float4 q = ldg_nc_f4(p + 4 * v);
      f[4 * v + 0] = q.x;
      f[4 * v + 1] = q.y;
      f[4 * v + 2] = q.z;
      f[4 * v + 3] = q.w;
    }
  } else {
    const __nv_bfloat16 *p = static_cast<const __nv_bfloat16 *>(base) + off;
    if constexpr (CPL == 4) {
      const uint2 q = ldg_nc_u2(p);
      f[0] = bf16lo(q.x);
      f[1] = bf16hi(q.x);
      f[2] = bf16lo(q.y);
      f[3] = bf16hi(q.y);
    } else {
      const uint4 q = ldg_nc_u4(p);
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
}

template <int CPL>
__device__ __forceinline__ void flush_run(const float (&run)[CPL], uint32_t row, int slot,
                                          float *temp, float *out, int R, int col) {
  if (slot >= 0) {
    float *t = temp + (size_t)slot * R + col;
#pragma unroll
    for (int k = 0; k < CPL; ++k) atomicAdd(t + k, run[k]);
  } else {
    float *o = out + (uint64_t)row * (uint64_t)R + (uint64_t)col;
#pragma unroll
    for (int v = 0; v < CPL / 4; ++v)
      red_add_v4(o + 4 * v, run[4 * v], run[4 * v + 1], run[4 * v + 2], run[4 * v + 3]);
  }
}

template <int KW, int CPL, bool BF16, bool PULL>
__global__ void __launch_bounds__(256) mttkrp_kernel(const __grid_constant__ MttkrpArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  float *temp = reinterpret_cast<float *>(sm);
  const int R = a.R;
  const int tpn = R / CPL;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
  const int grp = lane / tpn, col = (lane % tpn) * CPL;
  const int N = a.dp.nmodes;
  const int mode = a.mode;
  const unsigned full = 0xffffffffu;

  uint64_t *htab = nullptr;
  if (!PULL) {
    htab = reinterpret_cast<uint64_t *>(temp + (size_t)a.nslots * R);
    const int hsize = 1 << a.hbits;
    for (int i = threadIdx.x; i < hsize; i += blockDim.x) htab[i] = a.htab[i];
    for (int i = threadIdx.x; i < a.nslots * R; i += blockDim.x) temp[i] = 0.f;
    __syncthreads();
  }

  for (uint64_t l = blockIdx.x; l < a.L; l += gridDim.x) {
    const uint64_t s0 = (l * a.nnz) / a.L, s1 = ((l + 1) * a.nnz) / a.L;
    uint32_t Ts = 0, len = 0;
    if (PULL) {
      if (s1 > s0) {
        Ts = a.intervals[(l * N + mode) * 2];
        len = a.intervals[(l * N + mode) * 2 + 1] - Ts + 1u;
      }
      for (uint32_t i = threadIdx.x; i < len * (uint32_t)R; i += blockDim.x) temp[i] = 0.f;
      __syncthreads();
    }
    for (uint64_t base = s0 + (uint64_t)warp * 32; base < s1; base += (uint64_t)nwarps * 32) {
      const uint64_t x = base + lane;
      const bool valid = x < s1;
      uint64_t lo = 0, hi = 0;
      float v = 0.f;
      if (valid) {
        if (KW == 1) {
          lo = ldg_stream_u64(a.keys + x);
        } else {
          const ulonglong2 kk = ldg_stream_u128(a.keys + 2 * x);
          lo = kk.x;
          hi = kk.y;
        }
        v = ldg_stream_f32(a.vals + x);
      }
      uint32_t c[kMaxModes];
      decode_all<KW>(a.dp, lo, hi, c);
      uint32_t row = 0;
#pragma unroll
      for (int n = 0; n < kMaxModes; ++n)
        if (n == mode) row = c[n];
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
        uint32_t cj[kMaxModes];
#pragma unroll
        for (int n = 0; n < kMaxModes; ++n) cj[n] = (n < N) ? __shfl_sync(full, c[n], j) : 0u;
        if (j < nvalid) {
          float p[CPL];
#pragma unroll
          for (int k = 0; k < CPL; ++k) p[k] = vj;
          uint32_t rj = 0;
#pragma unroll
          for (int m = 0; m < kMaxModes; ++m) {
            if (m < N) {
              if (m == mode) {
                rj = cj[m];
              } else {
                float f[CPL];
                load_factor_row<CPL, BF16>(a.factors[m], cj[m], R, col, f);
#pragma unroll
                for (int k = 0; k < CPL; ++k) p[k] *= f[k];
              }
            }
          }
          if (rj == run_row) {
#pragma unroll
            for (int k = 0; k < CPL; ++k) run[k] += p[k];
          } else {
            if (run_row != kEmptyRow) flush_run<CPL>(run, run_row, run_slot, temp, a.out, R, col);
#pragma unroll
            for (int k = 0; k < CPL; ++k) run[k] = p[k];
            run_row = rj;
            run_slot = sj;
          }
        }
      }
      if (run_row != kEmptyRow) flush_run<CPL>(run, run_row, run_slot, temp, a.out, R, col);
    }
    __syncthreads();
    if (PULL) {
      if (len) {
        float4 *dst = reinterpret_cast<float4 *>(a.partials + a.part_off[l] * (uint64_t)R);
        const float4 *src = reinterpret_cast<const float4 *>(temp);
        const uint32_t n4 = len * (uint32_t)R / 4;
        for (uint32_t i = threadIdx.x; i < n4; i += blockDim.x) dst[i] = src[i];
      }
      __syncthreads();
    } else {
      float4 *t4 = reinterpret_cast<float4 *>(temp);
      const int n4 = a.nslots * R / 4;
      const int per_row = R / 4;
      for (int i = threadIdx.x; i < n4; i += blockDim.x) {
        const float4 t = t4[i];
        if (t.x != 0.f || t.y != 0.f || t.z != 0.f || t.w != 0.f) {
          const int sl = i / per_row, c4 = (i - sl * per_row) * 4;
          red_add_v4(a.out + (uint64_t)a.slot_rows[sl] * (uint64_t)R + c4, t.x, t.y, t.z, t.w);
          t4[i] = make_float4(0.f, 0.f, 0.f, 0.f);
        }
      }
      __syncthreads();
    }
  }
}

// out(b,:) = sum over segments l with b in [T^s_l, T^e_l] of Temp_l(b - T^s_l, :)
// (Alg. 4, pull-based reduction); prow lists, per row, the partial rows to add.
__global__ void __launch_bounds__(256) pull_reduce_kernel(const float *__restrict__ partials,
                                                          const uint64_t *__restrict__ row_ptr,
                                                          const uint64_t *__restrict__ prow,
                                                          uint64_t I, int R, float *__restrict__ out) {
  const int per_row = R / 4;
  const uint64_t total = I * (uint64_t)per_row;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t b = t / per_row;
    const int c4 = (int)(t - b * per_row) * 4;
    double s0 = 0, s1 = 0, s2 = 0, s3 = 0;
    for (uint64_t e = row_ptr[b]; e < row_ptr[b + 1]; ++e) {
      const float4 p = *reinterpret_cast<const float4 *>(partials + prow[e] * (uint64_t)R + c4);
      s0 += p.x;
      s1 += p.y;
      s2 += p.z;
      s3 += p.w;
    }
    *reinterpret_cast<float4 *>(out + b * (uint64_t)R + c4) =
        make_float4((float)s0, (float)s1, (float)s2, (float)s3);
  }
}

size_t mttkrp_smem_bytes(bool pull, int R, int nslots, int hbits, uint32_t max_interval) {
  if (pull) return (size_t)max_interval * (size_t)R * sizeof(float);
  return (size_t)nslots * R * sizeof(float) + ((size_t)1 << hbits) * sizeof(uint64_t);
}

size_t mttkrp_smem_limit() {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  return (size_t)v;
}

template <int KW, int CPL, bool BF16, bool PULL>
static cudaError_t launch_one(const MttkrpArgs &a, size_t smem, int num_sms, cudaStream_t s) {
  auto kern = mttkrp_kernel<KW, CPL, BF16, PULL>;
  static int configured = 0;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)mttkrp_smem_limit());
    if (e != cudaSuccess) return e;
    configured = 1;
  }
  int per_sm = 0;
  cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, 256, smem);
  if (e != cudaSuccess) return e;
  if (per_sm < 1) per_sm = 1;
  uint64_t grid = (uint64_t)num_sms * (uint64_t)per_sm;
  if (grid > a.L) grid = a.L;
  if (grid < 1) grid = 1;
  kern<<<(unsigned)grid, 256, smem, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

template <int KW, int CPL>
static cudaError_t dispatch2(const MttkrpArgs &a, bool bf16, bool pull, size_t smem, int num_sms,
                             cudaStream_t s) {
  if (bf16) {
    return pull ? launch_one<KW, CPL, true, true>(a, smem, num_sms, s)
                : launch_one<KW, CPL, true, false>(a, smem, num_sms, s);
  }
  return pull ? launch_one<KW, CPL, false, true>(a, smem, num_sms, s)
              : launch_one<KW, CPL, false, false>(a, smem, num_sms, s);
}

cudaError_t launch_mttkrp(const MttkrpArgs &a, int cpl, bool bf16, bool pull, size_t smem,
                          int num_sms, cudaStream_t s) {
  if (a.nnz == 0) return cudaSuccess;
  if (a.dp.kw == 1)
    return cpl == 4 ? dispatch2<1, 4>(a, bf16, pull, smem, num_sms, s)
                    : dispatch2<1, 8>(a, bf16, pull, smem, num_sms, s);
  return cpl == 4 ? dispatch2<2, 4>(a, bf16, pull, smem, num_sms, s)
                  : dispatch2<2, 8>(a, bf16, pull, smem, num_sms, s);
}

cudaError_t launch_pull_reduce(const float *partials, const uint64_t *row_ptr, const uint64_t *prow,
                               uint64_t I, int R, float *out, int num_sms, cudaStream_t s) {
  const uint64_t total = I * (uint64_t)(R / 4);
  uint64_t grid = (total + 255) / 256;
  if (grid > (uint64_t)num_sms * 16) grid = (uint64_t)num_sms * 16;
  if (grid < 1) grid = 1;
  pull_reduce_kernel<<<(unsigned)grid, 256, 0, s>>>(partials, row_ptr, prow, I, R, out);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace alto
