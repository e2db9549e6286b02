// CP-ALS glue of Alg. 1 around the MTTKRP.
//
// Per mode n (factors stored as B_m with A_m = B_m diag(s_m)):
//   prepare_kernel  one CTA, fp64: V = Hadamard product of the other Grams,
//                   Cholesky V = L L^T, X = L^-1, Sn = prod_{m != n} s_m and
//                   the solve factors W1 = diag(Sn) X^T, W2 = X (V^-1 =
//                   X^T X is never formed). MTTKRP over the stored B's gives
//                   M_B = M diag(1/Sn), so M V^-1 = (M_B W1) W2.
//   (MTTKRP)
//   update_kernel   B_n = (M_B W1) W2 in one pass over M_B (update_tc_kernel
//                   on the tensor cores for R = 16, 32), accumulating B_n^T B_n
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

// B_n = (M_B W1) W2 with B_n^T B_n and the column dot products
// sum_i M_B(i,r) B_n(i,r) in the same pass over M_B (the solve step of Alg. 1
// and the Gram and fit terms it needs, formed from the B_n values that are
// stored).
//
// A tile is TR = 4096 / R rows (16 KB), loaded into registers one tile ahead
// and stored transposed in shared memory. Thread (rb, cb) computes the 4 x 4
// block of Y = M_B W1 at rows 4 rb.., columns 4 cb.. (R steps of 16 FMA),
// puts it in shared memory, computes its block of B_n = Y W2 the same way and
// part of the dot products; the block also goes to shared memory, from which
// every thread then accumulates one 4 x 4 block (bi <= bj) of B_n^T B_n over a
// share of the tile's rows (the blocks on and above the diagonal spread over
// all 256 threads). fp32 partial sums move to fp64 every kUgFlush tiles: the
// Gram blocks into per-thread slots in shared memory, the dot products into
// shared fp64 accumulators; at the end the CTA sums them into BtB and dot.
constexpr int kUgThreads = 256;
constexpr int kUgFlush = 32;
#ifndef ALTO_UG_MIN_BLOCKS
#define ALTO_UG_MIN_BLOCKS 2
#endif

template <int R>
__global__ void __launch_bounds__(kUgThreads, ALTO_UG_MIN_BLOCKS)
    update_kernel(const float *__restrict__ M, const float *__restrict__ W, float *__restrict__ Bout,
                  uint64_t I, double *__restrict__ BtB, double *__restrict__ dot,
                  const int *__restrict__ done_at, int it) {
  if (*done_at <= it) return;
  constexpr int TR = 4096 / R, TRP = TR + 4, RP = R + 4, B4 = R / 4;
  constexpr int BB = B4 * (B4 + 1) / 2;
  constexpr int kPer = 4096 / 4 / kUgThreads;  // float4 of a tile per thread
  extern __shared__ __align__(16) unsigned char smraw[];
  double *slot = reinterpret_cast<double *>(smraw);           // [kUgThreads][16]
  double *dsum = slot + kUgThreads * 16;                       // [R]
  float *w = reinterpret_cast<float *>(dsum + R);              // 2 R * R: W1, W2
  float *mt = w + 2 * R * R;                                   // R * TRP (M tile, column-major)
  float *bt = mt + R * TRP;                                    // TR * RP (B tile, row-major;
                                                               // first M W1, column-major)
  const int tid = threadIdx.x;
  const int cb = tid % B4, rb = tid / B4;
  // Gram block of this thread: block b = tid mod BB of the upper triangle,
  // rows qg, qg + nb, ... of the tile (nb threads share block b)
  const int b = tid % BB, qg = tid / BB, nb = (kUgThreads - 1 - b) / BB + 1;
  int bi = 0, rem = b;
  while (rem >= B4 - bi) {
    rem -= B4 - bi;
    ++bi;
  }
  const int bj = bi + rem;
  for (int i = tid; i < 2 * R * R; i += kUgThreads) w[i] = W[i];
  for (int i = tid; i < R; i += kUgThreads) dsum[i] = 0.0;
#pragma unroll
  for (int i = 0; i < 16; ++i) slot[tid * 16 + i] = 0.0;
  float g[4][4], dp[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    dp[x] = 0.f;
#pragma unroll
    for (int y = 0; y < 4; ++y) g[x][y] = 0.f;
  }
  auto flush = [&]() {
#pragma unroll
    for (int x = 0; x < 4; ++x) {
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        slot[tid * 16 + 4 * x + y] += (double)g[x][y];
        g[x][y] = 0.f;
      }
      atomicAdd(&dsum[4 * cb + x], (double)dp[x]);
      dp[x] = 0.f;
    }
  };
  const float4 *M4 = reinterpret_cast<const float4 *>(M);
  const uint64_t ntiles = (I + TR - 1) / TR;
  float4 nxt[kPer];
  auto load_tile = [&](uint64_t tt) {
    const uint64_t rr0 = tt * (uint64_t)TR;
    const int nr = (I - rr0) < (uint64_t)TR ? (int)(I - rr0) : TR;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int i = tid + j * kUgThreads, r = i / B4;
      nxt[j] = r < nr ? __ldcs(M4 + (rr0 + r) * B4 + (i - r * B4)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  int tiles = 0;
  if ((uint64_t)blockIdx.x < ntiles) load_tile(blockIdx.x);
  for (uint64_t t = blockIdx.x; t < ntiles; t += gridDim.x) {
    const uint64_t r0 = t * (uint64_t)TR;
    const int nrows = (I - r0) < (uint64_t)TR ? (int)(I - r0) : TR;
    __syncthreads();  // the previous tile's reads of mt and bt are done
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int i = tid + j * kUgThreads;
      const int r = i / B4, c = (i - r * B4) * 4;
      const float4 m = nxt[j];
      mt[(c + 0) * TRP + r] = m.x;
      mt[(c + 1) * TRP + r] = m.y;
      mt[(c + 2) * TRP + r] = m.z;
      mt[(c + 3) * TRP + r] = m.w;
    }
    if (t + gridDim.x < ntiles) load_tile(t + gridDim.x);
    __syncthreads();
    // B_n block: rows 4 rb .. 4 rb + 3, columns 4 cb .. 4 cb + 3, as
    // (M W1) W2 with the block of M W1 passing through shared memory
    float o[4][4];
    block_product(mt, TRP, w, R, rb, cb, o);
#pragma unroll
    for (int y = 0; y < 4; ++y)
      *reinterpret_cast<float4 *>(bt + (4 * cb + y) * TRP + 4 * rb) = make_float4(o[0][y], o[1][y], o[2][y], o[3][y]);
    __syncthreads();
    block_product(bt, TRP, w + R * R, R, rb, cb, o);
    __syncthreads();  // every read of M W1 is done before B overwrites it
    // dot products with M_B (rows past nrows are 0 in both)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const float4 mc = *reinterpret_cast<const float4 *>(mt + (4 * cb + y) * TRP + 4 * rb);
      dp[y] = fmaf(mc.x, o[0][y], fmaf(mc.y, o[1][y], fmaf(mc.z, o[2][y], fmaf(mc.w, o[3][y], dp[y]))));
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int r = 4 * rb + x;
      const float4 ov = make_float4(o[x][0], o[x][1], o[x][2], o[x][3]);
      *reinterpret_cast<float4 *>(bt + r * RP + 4 * cb) = ov;
      if (r < nrows) __stcs(reinterpret_cast<float4 *>(Bout + (r0 + r) * (uint64_t)R + 4 * cb), ov);
    }
    __syncthreads();
    // Gram block (bi, bj) of B_n over this thread's rows
    for (int r = qg; r < nrows; r += nb) {
      const float4 xv = *reinterpret_cast<const float4 *>(bt + r * RP + 4 * bi);
      const float4 yv = *reinterpret_cast<const float4 *>(bt + r * RP + 4 * bj);
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) g[x][y] = fmaf(xa[x], ya[y], g[x][y]);
    }
    if (++tiles == kUgFlush) {
      flush();
      tiles = 0;
    }
  }
  flush();
  __syncthreads();
  // the first thread of every block sums the block's slots into BtB
  if (tid < BB) {
#pragma unroll
    for (int e = 0; e < 16; ++e) {
      double v = 0.0;
      for (int k = tid; k < kUgThreads; k += BB) v += slot[k * 16 + e];
      const int x = e / 4, y = e % 4;
      if (v != 0.0) {
        atomicAdd(&BtB[(4 * bi + x) * R + 4 * bj + y], v);
        if (bi != bj) atomicAdd(&BtB[(4 * bj + y) * R + 4 * bi + x], v);
      }
    }
  }
  for (int i = tid; i < R; i += kUgThreads)
    if (dsum[i] != 0.0) atomicAdd(&dot[i], dsum[i]);
}

template <int R>
constexpr size_t update_smem_r() {
  return (size_t)(kUgThreads * 16 + R) * sizeof(double) +
         (size_t)(2 * R * R + R * (4096 / R + 4) + (4096 / R) * (R + 4)) * sizeof(float);
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

// B(:, r) *= rscale[r] when finish_body asked for it (its s_n is then 1).
__global__ void __launch_bounds__(256) renorm_kernel(float *__restrict__ B, const double *__restrict__ rscale,
                                                     const int *__restrict__ renorm, uint64_t I, int R) {
  if (!*renorm) return;
  const int per_row = R / 4;
  const uint64_t total = I * (uint64_t)per_row;
  for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
       t += (uint64_t)gridDim.x * blockDim.x) {
    const int c4 = (int)(t % per_row) * 4;
    float4 *p = reinterpret_cast<float4 *>(B) + t;
    float4 v = *p;
    v.x *= (float)rscale[c4];
    v.y *= (float)rscale[c4 + 1];
    v.z *= (float)rscale[c4 + 2];
    v.w *= (float)rscale[c4 + 3];
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


template <int R>
static cudaError_t launch_update_r(const float *M, const float *W, float *B, uint64_t I, double *BtB,
                                   double *dot, const int *done_at, int it, int num_sms, cudaStream_t s) {
  auto kern = update_kernel<R>;
  constexpr size_t smem = update_smem_r<R>();
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  int per_sm = 1;
  if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kUgThreads, smem) != cudaSuccess) {
    cudaGetLastError();
    per_sm = 1;
  }
  kern<<<grid_rows(I, 4096 / R, num_sms, per_sm > 0 ? per_sm : 1), kUgThreads, smem, s>>>(M, W, B, I, BtB,
                                                                                         dot, done_at, it);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_update(const float *M, const float *W, float *B, uint64_t I, int R, double *BtB,
                          double *dot, const int *done_at, int it, int num_sms, cudaStream_t s) {
  if (I == 0) return cudaSuccess;
  switch (R) {
    case 4: return launch_update_r<4>(M, W, B, I, BtB, dot, done_at, it, num_sms, s);
    case 8: return launch_update_r<8>(M, W, B, I, BtB, dot, done_at, it, num_sms, s);
    case 16: return launch_update_r<16>(M, W, B, I, BtB, dot, done_at, it, num_sms, s);
    case 32: return launch_update_r<32>(M, W, B, I, BtB, dot, done_at, it, num_sms, s);
    default: return launch_update_r<64>(M, W, B, I, BtB, dot, done_at, it, num_sms, s);
  }
}

cudaError_t launch_renorm(float *B, const double *rscale, const int *renorm, uint64_t I, int R, int num_sms,
                          cudaStream_t s) {
  if (I == 0) return cudaSuccess;
  const uint64_t total = I * (uint64_t)(R / 4);
  uint64_t g = (total + 255) / 256;
  if (g > (uint64_t)num_sms * 8) g = (uint64_t)num_sms * 8;
  renorm_kernel<<<(unsigned)(g ? g : 1), 256, 0, s>>>(B, rscale, renorm, I, R);
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
