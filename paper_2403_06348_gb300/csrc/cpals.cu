// CP-ALS glue of Alg. 1 around the MTTKRP:
//   gram_kernel   G = A^T A (fp32 products, fp32 partial sums over at most
//                 1024 rows, fp64 combine)
//   solve_kernel  one CTA, fp64: V = Hadamard of the other Grams, Cholesky
//                 V = L L^T, V^-1, lambda_r = ||(M V^-1)(:,r)|| from
//                 V^-1 (M^T M) V^-1, W = V^-1 diag(1/lambda), the new Gram
//                 diag(1/lambda) V^-1 M^T M V^-1 diag(1/lambda), and after the
//                 last mode the fit
//   rmul_kernel   A^(n) = M W (fp32), i.e. the normalised M V^-1.
// Every kernel returns at once when the run stopped early (done_at <= it).
#include "cpals.cuh"

#include <climits>

namespace alto {

constexpr int kGramRows = 32;  // rows staged per step

__global__ void __launch_bounds__(256) gram_kernel(const float *__restrict__ A, uint64_t I, int R,
                                                   double *__restrict__ G,
                                                   const int *__restrict__ done_at, int it) {
  if (done_at && *done_at <= it) return;
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
    if (++steps == 32) {  // at most 32*32 rows per fp32 partial
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
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int b = 0; b < 4; ++b) {
      dacc[a][b] += (double)acc[a][b];
      atomicAdd(&red[(bi * 4 + a) * R + bj * 4 + b], dacc[a][b]);
    }
  __syncthreads();
  for (int i = tid; i < R * R; i += 256)
    if (red[i] != 0.0) atomicAdd(&G[i], red[i]);
}

// One CTA of 256 threads; all matrices R x R in shared memory (fp64).
__global__ void __launch_bounds__(256) solve_kernel(const SolveArgs a) {
  if (*a.done_at <= a.it) return;
  extern __shared__ __align__(16) double sd[];
  const int R = a.R, RR = R * R, tid = threadIdx.x;
  double *V = sd;            // V, then its Cholesky factor L (lower)
  double *Vi = V + RR;       // V^-1
  double *T = Vi + RR;       // scratch
  double *Gr = T + RR;       // V^-1 MtM V^-1
  double *lam = Gr + RR;     // R
  double *scl = lam + R;     // R: 1/lambda or 1
  __shared__ int fail;
  if (tid == 0) fail = 0;
  // V = *_{m != n} G_m
  for (int e = tid; e < RR; e += 256) {
    double v = 1.0;
    for (int m = 0; m < a.N; ++m)
      if (m != a.n) v *= a.G[(size_t)m * RR + e];
    V[e] = v;
  }
  __syncthreads();
  // Cholesky, column by column (lower triangle of V overwritten by L)
  for (int k = 0; k < R; ++k) {
    if (tid == 0) {
      const double d = V[k * R + k];
      if (!(d > 0.0) || !isfinite(d)) fail = 1;
      V[k * R + k] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    const double dk = V[k * R + k];
    for (int i = k + 1 + tid; i < R; i += 256) V[i * R + k] /= dk;
    __syncthreads();
    const int m = R - k - 1;
    for (int p = tid; p < m * m; p += 256) {
      const int i = k + 1 + p / m, j = k + 1 + p % m;
      if (j <= i) V[i * R + j] -= V[i * R + k] * V[j * R + k];
    }
    __syncthreads();
  }
  if (fail) {
    if (tid == 0) {
      atomicOr(a.status, kStatusNotSpd);
      *a.done_at = a.it;  // stop: later kernels of this and further iterations skip
    }
    return;
  }
  // V^-1 = L^-T L^-1, one column per thread
  for (int j = tid; j < R; j += 256) {
    for (int i = 0; i < R; ++i) {  // forward: L y = e_j
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= V[i * R + k] * T[k * R + j];
      T[i * R + j] = s / V[i * R + i];
    }
    for (int i = R - 1; i >= 0; --i) {  // backward: L^T x = y
      double s = T[i * R + j];
      for (int k = i + 1; k < R; ++k) s -= V[k * R + i] * Vi[k * R + j];
      Vi[i * R + j] = s / V[i * R + i];
    }
  }
  __syncthreads();
  // Gr = V^-1 MtM V^-1 (= (M V^-1)^T (M V^-1))
  for (int e = tid; e < RR; e += 256) {
    const int i = e / R, j = e % R;
    double s = 0.0;
    for (int k = 0; k < R; ++k) s += Vi[i * R + k] * a.MtM[k * R + j];
    T[e] = s;
  }
  __syncthreads();
  for (int e = tid; e < RR; e += 256) {
    const int i = e / R, j = e % R;
    double s = 0.0;
    for (int k = 0; k < R; ++k) s += T[i * R + k] * Vi[k * R + j];
    Gr[e] = s;
  }
  __syncthreads();
  for (int r = tid; r < R; r += 256) {
    const double g = Gr[r * R + r];
    const double l = g > 0.0 ? sqrt(g) : 0.0;
    lam[r] = l;
    scl[r] = l > 0.0 ? 1.0 / l : 1.0;
    a.lambda[r] = l;
  }
  __syncthreads();
  for (int e = tid; e < RR; e += 256) {
    const int i = e / R, j = e % R;
    a.W[e] = (float)(Vi[e] * scl[j]);
    a.G_out[e] = Gr[e] * scl[i] * scl[j];
  }
  __syncthreads();
  if (!a.last_mode) return;
  // fit = 1 - sqrt(max(0, ||X||^2 + lam^T (*_m G_m) lam - 2 <X, X_hat>)) / ||X||
  // <X, X_hat> = sum_r lam_r sum_i M(i,r) A(i,r) = sum_r lam_r (MtM V^-1)_{rr} scl_r
  __shared__ double part[2][256];
  double s1 = 0.0, s2 = 0.0;
  for (int e = tid; e < RR; e += 256) {
    const int i = e / R, j = e % R;
    double h = 1.0;
    for (int m = 0; m < a.N; ++m) h *= (m == a.n) ? a.G_out[e] : a.G[(size_t)m * RR + e];
    s1 += lam[i] * lam[j] * h;
  }
  for (int r = tid; r < R; r += 256) {
    double d = 0.0;
    for (int k = 0; k < R; ++k) d += a.MtM[r * R + k] * Vi[k * R + r];
    s2 += lam[r] * d * scl[r];
  }
  part[0][tid] = s1;
  part[1][tid] = s2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) {
      part[0][tid] += part[0][tid + o];
      part[1][tid] += part[1][tid + o];
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double nx = *a.norm_sq;
    const double resid = nx + part[0][0] - 2.0 * part[1][0];
    const double fit = nx > 0.0 ? 1.0 - sqrt(resid > 0.0 ? resid : 0.0) / sqrt(nx) : 0.0;
    a.fits[a.it] = fit;
    *a.iters_done = a.it + 1;
    if (a.tol > 0.0 && a.it > 0 && fabs(fit - a.fits[a.it - 1]) < a.tol) *a.done_at = a.it + 1;
  }
}

// A = M W: thread (row, 4 columns), M rows staged in shared memory.
__global__ void __launch_bounds__(256) rmul_kernel(const float *__restrict__ M, const float *__restrict__ W,
                                                   float *__restrict__ A, uint64_t I, int R,
                                                   const int *__restrict__ done_at, int it) {
  if (done_at && *done_at <= it) return;
  __shared__ __align__(16) float w[ALTO_MAX_RANK * ALTO_MAX_RANK];
  __shared__ __align__(16) float m[1024];
  const int B = R / 4;
  const int rows = 1024 / R;  // rows per step (256 threads x 4 columns)
  const int tid = threadIdx.x;
  for (int i = tid; i < R * R; i += 256) w[i] = W[i];
  const int lr = tid / B, c4 = (tid % B) * 4;
  const float4 *M4 = reinterpret_cast<const float4 *>(M);
  float4 *m4 = reinterpret_cast<float4 *>(m);
  for (uint64_t r0 = (uint64_t)blockIdx.x * rows; r0 < I; r0 += (uint64_t)gridDim.x * rows) {
    const int nrows = (I - r0) < (uint64_t)rows ? (int)(I - r0) : rows;
    __syncthreads();
    if (tid < nrows * B) m4[tid] = M4[r0 * B + tid];
    __syncthreads();
    if (lr < nrows) {
      float o0 = 0.f, o1 = 0.f, o2 = 0.f, o3 = 0.f;
      const float *mr = m + lr * R;
      for (int k = 0; k < R; ++k) {
        const float mk = mr[k];
        const float4 wk = *reinterpret_cast<const float4 *>(w + k * R + c4);
        o0 = fmaf(mk, wk.x, o0);
        o1 = fmaf(mk, wk.y, o1);
        o2 = fmaf(mk, wk.z, o2);
        o3 = fmaf(mk, wk.w, o3);
      }
      *reinterpret_cast<float4 *>(A + (r0 + lr) * (uint64_t)R + c4) = make_float4(o0, o1, o2, o3);
    }
  }
}

static int grid_rows(uint64_t I, int rows_per_step, int num_sms, int per_sm) {
  uint64_t g = (I + rows_per_step - 1) / rows_per_step;
  const uint64_t cap = (uint64_t)num_sms * per_sm;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

cudaError_t launch_gram(const float *A, uint64_t I, int R, double *G, const int *done_at, int it,
                        int num_sms, cudaStream_t s) {
  if (I == 0) return cudaSuccess;
  gram_kernel<<<grid_rows(I, kGramRows * 8, num_sms, 4), 256, 0, s>>>(A, I, R, G, done_at, it);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_solve(const SolveArgs &a, cudaStream_t s) {
  const size_t smem = (size_t)(4 * a.R * a.R + 2 * a.R) * sizeof(double);
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(solve_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)((4 * ALTO_MAX_RANK * ALTO_MAX_RANK + 2 * ALTO_MAX_RANK) *
                                               sizeof(double)));
    if (e != cudaSuccess) return e;
    configured = true;
  }
  solve_kernel<<<1, 256, smem, s>>>(a);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_rmul(const float *M, const float *W, float *A, uint64_t I, int R,
                        const int *done_at, int it, int num_sms, cudaStream_t s) {
  if (I == 0) return cudaSuccess;
  rmul_kernel<<<grid_rows(I, 1024 / R, num_sms, 8), 256, 0, s>>>(M, W, A, I, R, done_at, it);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace alto
