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
#include "cpals.cuh"

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

// Cholesky of the R x R matrix in V (lower triangle overwritten by L).
// Returns false if a pivot is not positive and finite.
__device__ bool block_cholesky(double *V, int R, int *fail) {
  const int tid = threadIdx.x;
  for (int k = 0; k < R; ++k) {
    if (tid == 0) {
      const double d = V[k * R + k];
      if (!(d > 0.0) || !isfinite(d)) *fail = 1;
      V[k * R + k] = sqrt(d > 0.0 ? d : 1.0);
    }
    __syncthreads();
    const double dk = V[k * R + k];
    for (int i = k + 1 + tid; i < R; i += blockDim.x) V[i * R + k] /= dk;
    __syncthreads();
    const int m = R - k - 1;
    for (int p = tid; p < m * m; p += blockDim.x) {
      const int i = k + 1 + p / m, j = k + 1 + p % m;
      if (j <= i) V[i * R + j] -= V[i * R + k] * V[j * R + k];
    }
    __syncthreads();
  }
  return *fail == 0;
}

__global__ void __launch_bounds__(256) prepare_kernel(const CpArgs a) {
  if (*a.done_at <= a.it) return;
  extern __shared__ __align__(16) double sd[];
  const int R = a.R, RR = R * R, tid = threadIdx.x;
  double *V = sd;       // V, then L
  double *Vi = V + RR;  // V^-1
  double *T = Vi + RR;  // forward-solve scratch
  __shared__ int fail;
  if (tid == 0) fail = 0;
  for (int e = tid; e < RR; e += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < a.N; ++m)
      if (m != a.n) v *= a.G[(size_t)m * RR + e];
    V[e] = v;
  }
  __syncthreads();
  if (!block_cholesky(V, R, &fail)) {
    if (tid == 0) {
      atomicOr(a.status, kStatusNotSpd);
      *a.done_at = a.it;
    }
    return;
  }
  for (int j = tid; j < R; j += blockDim.x) {
    for (int i = 0; i < R; ++i) {  // L y = e_j
      double s = (i == j) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) s -= V[i * R + k] * T[k * R + j];
      T[i * R + j] = s / V[i * R + i];
    }
    for (int i = R - 1; i >= 0; --i) {  // L^T x = y
      double s = T[i * R + j];
      for (int k = i + 1; k < R; ++k) s -= V[k * R + i] * Vi[k * R + j];
      Vi[i * R + j] = s / V[i * R + i];
    }
  }
  for (int r = tid; r < R; r += blockDim.x) {
    double p = 1.0;
    for (int m = 0; m < a.N; ++m)
      if (m != a.n) p *= a.s[(size_t)m * R + r];
    a.Sn[r] = p;
  }
  __syncthreads();
  for (int e = tid; e < RR; e += blockDim.x) {
    const int i = e / R;
    a.W[e] = (float)(a.Sn[i] * Vi[e]);
  }
}

// B = M W with B^T B and the column dot products of M and B, one pass.
// A tile of TR = 4096 / R rows: every thread computes a 4-row x 4-column block
// of B from the transposed M tile and W (two 16-byte shared loads per 16
// FMAs), adds its block's column products M(r,c) B(r,c), stores B, and then
// accumulates a 4 x 4 block of B^T B over its share of the tile's rows.
// fp32 partial sums cover at most 32 tiles per thread before they move to
// fp64.
constexpr int kUpdThreads = 256;

__global__ void __launch_bounds__(kUpdThreads) update_kernel(const float *__restrict__ M,
                                                             const float *__restrict__ W,
                                                             float *__restrict__ Bout, uint64_t I, int R,
                                                             double *__restrict__ BtB, double *__restrict__ dot,
                                                             const int *__restrict__ done_at, int it) {
  if (*done_at <= it) return;
  extern __shared__ __align__(16) unsigned char smraw[];
  const int TR = 4096 / R;       // rows per tile
  const int TRP = TR + 4;        // padded row count of the transposed tile
  const int RP = R + 4;          // padded row length of the B tile
  double *red = reinterpret_cast<double *>(smraw);       // R*R + R
  float *w = reinterpret_cast<float *>(red + R * R + R);  // R*R
  float *mt = w + R * R;                                  // R * TRP (M tile, transposed)
  float *bt = mt + R * TRP;                               // TR * RP (B tile)
  const int tid = threadIdx.x;
  const int B4 = R / 4;                      // column blocks
  const int cb = tid % B4, rb = tid / B4;    // phase 1: rows 4*rb .. 4*rb+3, cols 4*cb ..
  const int BB = B4 * B4, RG = kUpdThreads / BB;
  const int tb = tid % BB, rg = tid / BB, bi = tb / B4, bj = tb % B4;
  for (int i = tid; i < R * R + R; i += kUpdThreads) red[i] = 0.0;
  for (int i = tid; i < R * R; i += kUpdThreads) w[i] = W[i];
  float g[4][4], dp[4];
  double dg[4][4], ddp[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    dp[x] = 0.f;
    ddp[x] = 0.0;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      g[x][y] = 0.f;
      dg[x][y] = 0.0;
    }
  }
  int tiles = 0;
  const float4 *M4 = reinterpret_cast<const float4 *>(M);
  for (uint64_t r0 = (uint64_t)blockIdx.x * TR; r0 < I; r0 += (uint64_t)gridDim.x * TR) {
    const int nrows = (I - r0) < (uint64_t)TR ? (int)(I - r0) : TR;
    __syncthreads();
    // transpose the M tile into shared memory (rows beyond nrows are zero)
    for (int i = tid; i < TR * B4; i += kUpdThreads) {
      const int r = i / B4, c = (i - r * B4) * 4;
      const float4 m = r < nrows ? M4[(r0 + r) * B4 + (i - r * B4)] : make_float4(0.f, 0.f, 0.f, 0.f);
      mt[(c + 0) * TRP + r] = m.x;
      mt[(c + 1) * TRP + r] = m.y;
      mt[(c + 2) * TRP + r] = m.z;
      mt[(c + 3) * TRP + r] = m.w;
    }
    __syncthreads();
    float o[4][4];
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) o[x][y] = 0.f;
    for (int k = 0; k < R; ++k) {
      const float4 mk = *reinterpret_cast<const float4 *>(mt + k * TRP + 4 * rb);
      const float4 wk = *reinterpret_cast<const float4 *>(w + k * R + 4 * cb);
      const float ma[4] = {mk.x, mk.y, mk.z, mk.w}, wa[4] = {wk.x, wk.y, wk.z, wk.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) o[x][y] = fmaf(ma[x], wa[y], o[x][y]);
    }
    // column products with M, store B (global and shared)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const float4 mc = *reinterpret_cast<const float4 *>(mt + (4 * cb + y) * TRP + 4 * rb);
      const float ma[4] = {mc.x, mc.y, mc.z, mc.w};
#pragma unroll
      for (int x = 0; x < 4; ++x) dp[y] = fmaf(ma[x], o[x][y], dp[y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int r = 4 * rb + x;
      const float4 ov = make_float4(o[x][0], o[x][1], o[x][2], o[x][3]);
      *reinterpret_cast<float4 *>(bt + r * RP + 4 * cb) = ov;
      if (r < nrows) *reinterpret_cast<float4 *>(Bout + (r0 + r) * (uint64_t)R + 4 * cb) = ov;
    }
    __syncthreads();
    for (int r = rg; r < nrows; r += RG) {
      const float4 xv = *reinterpret_cast<const float4 *>(bt + r * RP + 4 * bi);
      const float4 yv = *reinterpret_cast<const float4 *>(bt + r * RP + 4 * bj);
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) g[x][y] = fmaf(xa[x], ya[y], g[x][y]);
    }
    if (++tiles == 32) {
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        ddp[x] += (double)dp[x];
        dp[x] = 0.f;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          dg[x][y] += (double)g[x][y];
          g[x][y] = 0.f;
        }
      }
      tiles = 0;
    }
  }
  __syncthreads();
#pragma unroll
  for (int x = 0; x < 4; ++x) {
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      dg[x][y] += (double)g[x][y];
      atomicAdd(&red[(4 * bi + x) * R + 4 * bj + y], dg[x][y]);
    }
    atomicAdd(&red[R * R + 4 * cb + x], ddp[x] + (double)dp[x]);
  }
  __syncthreads();
  for (int i = tid; i < R * R; i += kUpdThreads)
    if (red[i] != 0.0) atomicAdd(&BtB[i], red[i]);
  for (int i = tid; i < R; i += kUpdThreads)
    if (red[R * R + i] != 0.0) atomicAdd(&dot[i], red[R * R + i]);
}

__global__ void __launch_bounds__(256) finish_kernel(const CpArgs a) {
  if (*a.done_at <= a.it) return;
  const int R = a.R, RR = R * R, tid = threadIdx.x;
  __shared__ double lam[ALTO_MAX_RANK], sn[ALTO_MAX_RANK];
  __shared__ double part[2][256];
  double *sv = a.s + (size_t)a.n * R;
  double *Gn = a.G + (size_t)a.n * RR;
  for (int r = tid; r < R; r += blockDim.x) {
    const double g = a.BtB[r * R + r];
    const double l = g > 0.0 ? sqrt(g) : 0.0;
    lam[r] = l;
    sn[r] = l > 0.0 ? 1.0 / l : 1.0;
    a.lambda[r] = l;
    sv[r] = sn[r];
  }
  __syncthreads();
  for (int e = tid; e < RR; e += blockDim.x) Gn[e] = a.BtB[e] * sn[e / R] * sn[e % R];
  __syncthreads();
  if (!a.last_mode) return;
  // fit = 1 - sqrt(max(0, ||X||^2 + lam^T (*_m G_m) lam - 2 <X, X_hat>)) / ||X||,
  // <X, X_hat> = sum_r lam_r sum_i M(i,r) A_n(i,r) = sum_r Sn_r sum_i M_B(i,r) B_n(i,r)
  double s1 = 0.0, s2 = 0.0;
  for (int e = tid; e < RR; e += blockDim.x) {
    double h = 1.0;
    for (int m = 0; m < a.N; ++m) h *= a.G[(size_t)m * RR + e];
    s1 += lam[e / R] * lam[e % R] * h;
  }
  for (int r = tid; r < R; r += blockDim.x) s2 += a.Sn[r] * a.dot[r];
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

static size_t update_smem(int R) {
  const int TR = 4096 / R;
  return (size_t)(R * R + R) * sizeof(double) +
         (size_t)(R * R + R * (TR + 4) + TR * (R + 4)) * sizeof(float);
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
