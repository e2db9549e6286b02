// CP-APR with multiplicative updates (Alg. 2): the kernels around Phi.
//
// Per mode n of an outer iteration (the driver is cpapr_run in api.cu):
//   shift_scale   B = (A^(n) + S) diag(lambda)
//   pi            (PRE only) Pi rows of every nonzero, once per mode
//   l_max times:  inner_begin (zero Phi and the KKT maximum), Phi (Alg. 5,
//                 mttkrp_kernel with APR), kkt (max |min(B, 1 - Phi)|), mu
//                 (stop, or B *= Phi)
//   colsum + normalize: lambda = e^T B, A^(n) = B diag(lambda)^-1
// Every inner-loop kernel returns at once when the loop has already stopped,
// so a mode costs l_max launches of near-empty kernels after convergence
// instead of a device-to-host round trip per inner iteration.
#include "apr.cuh"

namespace alto {

namespace {

int grid_for(uint64_t work, int threads, int num_sms, int per_sm) {
  uint64_t g = (work + threads - 1) / threads;
  const uint64_t cap = (uint64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  return (int)(g < 1 ? 1 : g);
}

}  // namespace

__global__ void __launch_bounds__(256) colsum_kernel(const float *__restrict__ A, uint64_t I, int R,
                                                     double *__restrict__ sums) {
  __shared__ double part[ALTO_MAX_RANK];
  for (int r = threadIdx.x; r < R; r += blockDim.x) part[r] = 0.0;
  __syncthreads();
  // thread t sums column t % R over rows t / R, t / R + rows_per_step, ...
  const int rows_per_block = 256 / R;
  const int c = threadIdx.x % R, r0 = threadIdx.x / R;
  double acc = 0.0;
  if (r0 < rows_per_block)
    for (uint64_t i = (uint64_t)blockIdx.x * rows_per_block + r0; i < I;
         i += (uint64_t)gridDim.x * rows_per_block)
      acc += (double)A[i * (uint64_t)R + c];
  if (r0 < rows_per_block) atomicAdd(&part[c], acc);
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x)
    if (part[r] != 0.0) atomicAdd(&sums[r], part[r]);
}

__global__ void __launch_bounds__(256) normalize_kernel(float *__restrict__ A, uint64_t I, int R,
                                                        const double *__restrict__ sums,
                                                        double *__restrict__ lam) {
  if (lam && blockIdx.x == 0)
    for (int r = threadIdx.x; r < R; r += blockDim.x) lam[r] *= sums[r];
  const uint64_t total = I * (uint64_t)R;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const double sr = sums[t % R];
    if (sr > 0.0) A[t] = (float)((double)A[t] / sr);
  }
}

__global__ void __launch_bounds__(256) shift_scale_kernel(const float *__restrict__ A,
                                                          const float *__restrict__ phi_prev,
                                                          uint64_t I, int R, const double *__restrict__ lam,
                                                          int shift, float kappa, float kappa_tol,
                                                          float *__restrict__ B) {
  const uint64_t total = I * (uint64_t)R;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const float a = A[t];
    const float s = (shift && a < kappa_tol && phi_prev[t] > 1.f) ? kappa : 0.f;
    B[t] = (float)((double)(a + s) * lam[t % R]);
  }
}

__global__ void __launch_bounds__(256) inner_begin_kernel(float *__restrict__ phi, uint64_t I, int R,
                                                          int zero_phi, unsigned *kkt_bits,
                                                          const int *__restrict__ done) {
  if (*done) return;
  if (blockIdx.x == 0 && threadIdx.x == 0) *kkt_bits = 0u;
  if (!zero_phi) return;
  const uint64_t n4 = I * (uint64_t)R / 4;
  float4 *p4 = reinterpret_cast<float4 *>(phi);
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < n4;
       t += (uint64_t)gridDim.x * blockDim.x)
    p4[t] = make_float4(0.f, 0.f, 0.f, 0.f);
}

__global__ void __launch_bounds__(256) kkt_kernel(const float *__restrict__ B,
                                                  const float *__restrict__ phi, uint64_t I, int R,
                                                  unsigned *kkt_bits, const int *__restrict__ done) {
  if (*done) return;
  __shared__ float wmax[8];
  float m = 0.f;
  const uint64_t total = I * (uint64_t)R;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x)
    m = fmaxf(m, fabsf(fminf(B[t], 1.f - phi[t])));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) m = fmaxf(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) wmax[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.f;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b = fmaxf(b, wmax[w]);
    // non-negative floats order like their bit patterns
    atomicMax(kkt_bits, __float_as_uint(b));
  }
}

__global__ void __launch_bounds__(256) mu_kernel(float *__restrict__ B, const float *__restrict__ phi,
                                                 uint64_t I, int R, const unsigned *kkt_bits, float tau,
                                                 int *done, int *stepped, int *steps) {
  if (*done) return;
  if (__uint_as_float(*kkt_bits) < tau) {
    if (blockIdx.x == 0 && threadIdx.x == 0) *done = 1;
    return;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *stepped = 1;
    ++*steps;
  }
  const uint64_t total = I * (uint64_t)R;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x)
    B[t] *= phi[t];
}

__global__ void __launch_bounds__(256) pi_kernel(const __grid_constant__ DecodePlan dp,
                                                 const uint64_t *__restrict__ keys, uint64_t nnz,
                                                 int mode, const __grid_constant__ FactorPtrs f, int R,
                                                 float *__restrict__ pi) {
  const int per = R / 4;
  const uint64_t total = nnz * (uint64_t)per;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x = t / per;
    const int c4 = (int)(t - x * per) * 4;
    const uint64_t lo = keys[x * dp.kw], hi = dp.kw == 2 ? keys[x * 2 + 1] : 0ull;
    uint32_t c[kMaxModes];
    if (dp.kw == 1)
      decode_all<1>(dp, lo, hi, c);
    else
      decode_all<2>(dp, lo, hi, c);
    float4 k = make_float4(1.f, 1.f, 1.f, 1.f);
    for (int m = 0; m < dp.nmodes; ++m) {
      if (m == mode) continue;
      const float4 a = *reinterpret_cast<const float4 *>(f.p[m] + (uint64_t)c[m] * R + c4);
      k.x *= a.x;
      k.y *= a.y;
      k.z *= a.z;
      k.w *= a.w;
    }
    *reinterpret_cast<float4 *>(pi + x * (uint64_t)R + c4) = k;
  }
}

__global__ void __launch_bounds__(256) loglik_kernel(const __grid_constant__ DecodePlan dp,
                                                     const uint64_t *__restrict__ keys,
                                                     const float *__restrict__ vals, uint64_t nnz,
                                                     const __grid_constant__ FactorPtrs f,
                                                     const double *__restrict__ lam, int R,
                                                     double *acc) {
  __shared__ double wsum[8];
  double s = 0.0;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nnz;
       x += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t lo = keys[x * dp.kw], hi = dp.kw == 2 ? keys[x * 2 + 1] : 0ull;
    uint32_t c[kMaxModes];
    if (dp.kw == 1)
      decode_all<1>(dp, lo, hi, c);
    else
      decode_all<2>(dp, lo, hi, c);
    double m = 0.0;
    for (int r = 0; r < R; ++r) {
      double p = lam[r];
      for (int q = 0; q < dp.nmodes; ++q) p *= (double)f.p[q][(uint64_t)c[q] * R + r];
      m += p;
    }
    s += (double)vals[x] * log(m > 1e-300 ? m : 1e-300);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  if ((threadIdx.x & 31) == 0) wsum[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    double b = 0.0;
    for (int w = 0; w < (int)(blockDim.x >> 5); ++w) b += wsum[w];
    atomicAdd(acc, b);
  }
}

cudaError_t launch_colsum(const float *A, uint64_t I, int R, double *sums, int num_sms,
                          cudaStream_t s) {
  if (I == 0) return cudaSuccess;
  colsum_kernel<<<grid_for(I, 256 / R, num_sms, 4), 256, 0, s>>>(A, I, R, sums);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_normalize(float *A, uint64_t I, int R, const double *sums, double *lam,
                             int num_sms, cudaStream_t s) {
  normalize_kernel<<<grid_for(I * R, 256, num_sms, 8), 256, 0, s>>>(A, I, R, sums, lam);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_shift_scale(const float *A, const float *phi_prev, uint64_t I, int R,
                               const double *lam, int shift, float kappa, float kappa_tol, float *B,
                               int num_sms, cudaStream_t s) {
  if (I == 0) return cudaSuccess;
  shift_scale_kernel<<<grid_for(I * R, 256, num_sms, 8), 256, 0, s>>>(A, phi_prev, I, R, lam, shift,
                                                                      kappa, kappa_tol, B);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_inner_begin(float *phi, uint64_t I, int R, bool zero_phi, unsigned *kkt_bits,
                               const int *done, int num_sms, cudaStream_t s) {
  inner_begin_kernel<<<grid_for(I * R / 4, 256, num_sms, 8), 256, 0, s>>>(phi, I, R, zero_phi ? 1 : 0,
                                                                          kkt_bits, done);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_kkt(const float *B, const float *phi, uint64_t I, int R, unsigned *kkt_bits,
                       const int *done, int num_sms, cudaStream_t s) {
  kkt_kernel<<<grid_for(I * R, 256, num_sms, 8), 256, 0, s>>>(B, phi, I, R, kkt_bits, done);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_mu(float *B, const float *phi, uint64_t I, int R, const unsigned *kkt_bits,
                      float tau, int *done, int *stepped, int *steps, int num_sms, cudaStream_t s) {
  mu_kernel<<<grid_for(I * R, 256, num_sms, 8), 256, 0, s>>>(B, phi, I, R, kkt_bits, tau, done,
                                                             stepped, steps);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_pi(const DecodePlan &dp, const uint64_t *keys, uint64_t nnz, int mode,
                      const FactorPtrs &factors, int R, float *pi, int num_sms, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  pi_kernel<<<grid_for(nnz * (R / 4), 256, num_sms, 8), 256, 0, s>>>(dp, keys, nnz, mode, factors, R,
                                                                     pi);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_loglik(const DecodePlan &dp, const uint64_t *keys, const float *vals, uint64_t nnz,
                          const FactorPtrs &factors, const double *lam, int R, double *acc,
                          int num_sms, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  loglik_kernel<<<grid_for(nnz, 256, num_sms, 8), 256, 0, s>>>(dp, keys, vals, nnz, factors, lam, R,
                                                               acc);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace alto
