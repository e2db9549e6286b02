// CP-ALS glue of Alg. 1 around the MTTKRP.
//
// Per mode n (factors stored as B_m with A_m = B_m diag(s_m)):
//   prepare_kernel  one CTA, fp64: V = Hadamard product of the other Grams,
//                   Cholesky V = L L^T, V^-1, Sn = prod_{m != n} s_m and
//                   W = diag(Sn) V^-1. MTTKRP over the stored B's gives
//                   M_B = M diag(1/Sn), so M V^-1 = M_B W.
//   (MTTKRP)
//   update_kernel   B_n = M_B W in one pass over M_B, accumulating B_n^T B_n
//                   and sum_i M_B(i,r) B_n(i,r) (fp32 partial sums over at most
//                   1024 rows, fp64 combine).
//   finish_kernel   one CTA, fp64: lambda_r = ||B_n(:,r)||, s_n = 1/lambda
//                   (1 for a zero column), the new Gram diag(s_n) B^T B
//                   diag(s_n), and after the last mode the fit.
// gram_kernel gives the Grams of the initial factors; scale_kernel writes the
// normalised A_m = B_m diag(s_m) once at the end of a run.
// Every per-iteration kernel returns at once when the run has stopped
// (done_at <= it).
#include "cpals_body.cuh"

namespace alto {

constexpr int kGramRows = 32;

__global__ void __launch_bounds__(256) gram_kernel(const float *__restrict__ A, uint64_t I, int R,
                                                   double *__restrict__ G) {
  __shared__ __align__(16) float tile[kGramRows * ALTO_MAX_RANK];
  __shared__ double red[ALTO_MAX_RANK * ALTO_MAX_RANK];
  const int B = R / 4, BB = B * B, RG = 256 / BB;
  const int tid = threadIdx.x, tb = tid % BB, rg = tid / BB, bi = tb / B, bj = tb % B;
  for (int i = tid; i < R * R; i += 256) red[i] = 0.0;
  float acc[4][4];
  double dacc[4][4];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      acc[a][b] = 0.f;
      dacc[a][b] = 0.0;
    }
  int steps = 0;
  const float4 *A4 = reinterpret_cast<const float4 *>(A);
  float4 *t4 = reinterpret_cast<float4 *>(tile);
  for (uint64_t r0 = (uint64_t)blockIdx.x * kGramRows; r0 < I; r0 += (uint64_t)gridDim.x * kGramRows) {
    const int nrows = (I - r0) < (uint64_t)kGramRows ? (int)(I - r0) : kGramRows;
    __syncthreads();
    for (int i = tid; i < nrows * B; i += 256) t4[i] = A4[r0 * B + i];
    __syncthreads();
    for (int r = rg; r < nrows; r += RG) {
      const float4 x = t4[r * B + bi], y = t4[r * B + bj];
      const float xa[4] = {x.x, x.y, x.z, x.w}, ya[4] = {y.x, y.y, y.z, y.w};
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) acc[a][b] = fmaf(xa[a], ya[b], acc[a][b]);
    }
    if (++steps == 32) {
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int b = 0; b < 4; ++b) {
          dacc[a][b] += (double)acc[a][b];
          acc[a][b] = 0.f;
        }
      steps = 0;
    }
  }
  __syncthreads();
  // lanes holding the same block (equal modulo BB) are summed in the warp first
  const int lane = tid & 31;
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      double v = dacc[a][b] + (double)acc[a][b];
      for (int o = 16; o >= BB; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      if (BB >= 32 || lane < BB) atomicAdd(&red[(bi * 4 + a) * R + bj * 4 + b], v);
    }
  __syncthreads();
  for (int i = tid; i < R * R; i += 256)
    if (red[i] != 0.0) atomicAdd(&G[i], red[i]);
}

__global__ void __launch_bounds__(256) prepare_kernel(const CpArgs a) {
  extern __shared__ __align__(16) double sd[];
  prepare_body(a, sd);
}

__global__ void __launch_bounds__(kUpdThreads, 2) update_kernel(const float *__restrict__ M,
                                                             const float *__restrict__ W,
                                                             float *__restrict__ Bout, uint64_t I, int R,
                                                             double *__restrict__ BtB, double *__restrict__ dot,
                                                             const int *__restrict__ done_at, int it) {
  if (*done_at <= it) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const uint64_t TR = 4096 / R;
  update_body<true>(const_cast<float *>(M), W, Bout, I, R, BtB, dot, blockIdx.x, gridDim.x, (I + TR - 1) / TR,
              false, smraw);
}

__global__ void __launch_bounds__(256) finish_kernel(const CpArgs a) { finish_body(a); }

__global__ void __launch_bounds__(256) scale_kernel(float *__restrict__ B, const double *__restrict__ s,
                                                    uint64_t I, int R) {
  const int per_row = R / 4;
  const uint64_t total = I * (uint64_t)per_row;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const int c4 = (int)(t % per_row) * 4;
    float4 *p = reinterpret_cast<float4 *>(B) + t;
    float4 v = *p;
    v.x *= (float)s[c4];
    v.y *= (float)s[c4 + 1];
    v.z *= (float)s[c4 + 2];
    v.w *= (float)s[c4 + 3];
    *p = v;
  }
}

static int grid_rows(uint64_t I, int rows_per_step, int num_sms, int per_sm) {
  uint64_t g = (I + rows_per_step - 1) / rows_per_step;
  const uint64_t cap = (uint64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_gram(const float *A, uint64_t I, int R, double *G, int num_sms, cudaStream_t s) {
  if (I == 0) return cudaSuccess;
  gram_kernel<<<grid_rows(I, kGramRows * 8, num_sms, 4), 256, 0, s>>>(A, I, R, G);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_prepare(const CpArgs &a, cudaStream_t s) {
  static bool configured = false;
  const size_t max_smem = (size_t)3 * ALTO_MAX_RANK * ALTO_MAX_RANK * sizeof(double);
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(prepare_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)max_smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  prepare_kernel<<<1, 256, (size_t)3 * a.R * a.R * sizeof(double), s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}


cudaError_t launch_update(const float *M, const float *W, float *B, uint64_t I, int R, double *BtB,
                          double *dot, const int *done_at, int it, int num_sms, cudaStream_t s) {
  if (I == 0) return cudaSuccess;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)update_smem(ALTO_MAX_RANK));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, update_kernel, kUpdThreads, update_smem(R));
  update_kernel<<<grid_rows(I, 4096 / R, num_sms, per_sm > 0 ? per_sm : 1), kUpdThreads,
                  update_smem(R), s>>>(M, W, B, I, R, BtB, dot, done_at, it);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_finish(const CpArgs &a, cudaStream_t s) {
  finish_kernel<<<1, 256, 0, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_scale(float *B, const double *s_m, uint64_t I, int R, int num_sms, cudaStream_t s) {
  if (I == 0) return cudaSuccess;
  const uint64_t total = I * (uint64_t)(R / 4);
  uint64_t g = (total + 255) / 256;
  if (g > (uint64_t)num_sms * 16) g = (uint64_t)num_sms * 16;
  scale_kernel<<<(unsigned)(g ? g : 1), 256, 0, s>>>(B, s_m, I, R);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace alto
