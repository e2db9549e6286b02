// CP-ALS update step on the tensor cores (tcgen05, TF32 with an error-
// compensating split): B_n = (M_B W1) W2 in one pass over M_B (W1 W2 the
// solve factors of V^-1 from the prepare step), with B_n^T B_n and
// the column dot products sum_i M_B(i,r) B_n(i,r) (the solve step of Alg. 1
// and the Gram and fit terms it needs, formed from the B_n values stored).
//
// All products are dense contractions with a short inner dimension:
//   Y tile  (128 rows x R)  = M tile (128 x R) . W1 (R x R)
//   B tile  (128 rows x R)  = Y tile . W2
//   Gram    (R x R)        += sum over tiles of B tile^T B tile
// Every operand x is split into two TF32 numbers, x = hi + lo with
// hi = rna_tf32(x) and lo = rna_tf32(x - hi), and a product a b is formed as
// hi_a hi_b + hi_a lo_b + lo_a hi_b (three MMAs into one fp32 accumulator in
// tensor memory); the dropped terms are below 2^-21 |a b|.
//
// One CTA of 128 threads owns 128 rows at a time, thread i row i:
//   1. the M rows are split into the K-major operand layout in shared memory;
//   2. one thread issues the Y MMAs (M = 128, N = R, K = 8 per instruction);
//      every thread reads its row of Y back (tcgen05.ld) and puts it, split,
//      in place of its M row; one thread issues the B MMAs the same way;
//   3. every thread reads its row of B back, stores it, adds
//      its products M(i,r) B(i,r) to fp32 dot sums, and writes it, split, into
//      the Gram operand: G[(q, r)][k] = B[q R + k][r] for chunk q = i / R;
//   4. one thread issues the Gram MMAs G G^T (M = N = 128, K = R): the
//      diagonal R x R blocks of the product are the chunks' B^T B.
// Every 32 tiles the diagonal blocks and the dot sums move to fp64 in shared
// memory; at the end the CTA adds them to BtB and dot. Every mbarrier wait is
// bounded (2 s); on expiry the CTA reports kStatusTimeout, waits once more for
// its MMAs, frees its tensor memory and returns.
#include "cpals.cuh"

#include "async_copy.cuh"

namespace alto {

namespace {

constexpr int kTcThreads = 128;       // one tile row per thread
constexpr int kTcRows = 128;          // rows per tile (the MMA's M)
constexpr int kTcFlush = 32;          // tiles between fp64 flushes
constexpr uint32_t kTcCols = 256;     // tensor-memory columns per CTA
constexpr uint32_t kTcGramCol = 128;  // first column of the Gram accumulator
constexpr uint64_t kTcWaitNs = 2000000000ull;
constexpr uint32_t kLboG = 144;       // A and Gram operands: K-direction core-matrix
                                      // stride (128 + 16: the eight 16-byte chunks of a
                                      // row, or one column of eight rows, fall in
                                      // different banks)

// --- tcgen05 (inline PTX) ----------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *dst, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(dst)),
               "r"(ncols)
               : "memory");
}

__device__ __forceinline__ void tmem_relinquish() {
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}

__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}

__device__ __forceinline__ void tc_fence_before() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tc_fence_after() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// D[tmem] (+)= A B^T, A and B read from shared memory through descriptors
__device__ __forceinline__ void mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc, uint32_t idesc,
                                         uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.u32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}

// bar receives one arrival once every MMA issued before by this thread is done
__device__ __forceinline__ void mma_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(bar))
               : "memory");
}

// lane j of the warp gets columns [col, col + 32) of tensor-memory lane
// (warp's lane quarter) + j
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32]) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, "
      "[%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
        "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
        "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, "
      "%13, %14, %15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
        "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// shared-memory matrix descriptor, no swizzle: core matrices of 8 rows x 16
// bytes (128 contiguous bytes), lbo = byte stride between core matrices along
// K, sbo = byte stride between groups of 8 rows
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor: fp32 accumulator, TF32 A and B, both K-major
constexpr uint32_t idesc_tf32(int m, int n) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

// x rounded to the nearest TF32 value (10 explicit mantissa bits), ties away
// from zero, as an fp32 bit pattern with the 13 low bits clear: add half a
// TF32 unit to the magnitude bits, then truncate (integer operations only)
__device__ __forceinline__ float tf32_rna(float x) {
  return __uint_as_float((__float_as_uint(x) + 0x1000u) & 0xFFFFE000u);
}

// byte offset of element (row, k) in a K-major operand (no swizzle)
__device__ __forceinline__ uint32_t op_off(int row, int k, uint32_t lbo, uint32_t sbo) {
  return (uint32_t)(row >> 3) * sbo + (uint32_t)(k >> 2) * lbo + (uint32_t)(row & 7) * 16u + (uint32_t)(k & 3) * 4u;
}

template <int R>
struct TcLayout {
  static constexpr uint32_t kSboW = (R / 4) * 128;      // W operand: N = R rows, K = R
  static constexpr uint32_t kSboA = (R / 4) * kLboG;    // M (then Y) tile: 128 rows, K = R
  static constexpr uint32_t kSboG = (R / 4) * kLboG;    // Gram operand: 128 rows, K = R
  static constexpr uint32_t kW = (R / 8) * kSboW;       // bytes of one W half
  static constexpr uint32_t kA = (kTcRows / 8) * kSboA;
  static constexpr uint32_t kG = (kTcRows / 8) * kSboG;
  // W1 (hi, lo), W2 (hi, lo), the A operand (M, then Y; hi, lo), the Gram operand (hi, lo)
  static constexpr uint32_t w1h = 0, w1l = kW, w2h = 2 * kW, w2l = 3 * kW;
  static constexpr uint32_t ah = 4 * kW, al = ah + kA, gh = al + kA, gl = gh + kG;
  static constexpr uint32_t bar = gl + kG;                    // two mbarriers
  static constexpr uint32_t tmem = bar + 16;                  // allocated address
  // at least 80 KB, so that at most two CTAs (2 x 256 tensor-memory columns)
  // share an SM and no allocation waits
  static constexpr uint32_t total = tmem + 16 > 80 * 1024 ? tmem + 16 : 80 * 1024;
};

// Moves the diagonal R x R blocks D of the Gram accumulator (chunk q: lanes
// and columns [q R, q R + R)) and the dot sums into the fp64 registers greg
// (elements tid + 128 j of B^T B) and dreg (dot r = tid), through the free
// Gram operand buffers (stage, dstage) in shared memory: no shared atomics.
// The accumulator holds hi hi^T + 2 hi lo^T; its symmetric part (D + D^T) / 2
// is hi hi^T + hi lo^T + lo hi^T.
template <int R>
__device__ __forceinline__ void flush_sums(uint32_t tbase, float *stage, float *dstage, float (&dacc)[R],
                                           double (&greg)[R * R / kTcThreads], double &dreg, int warp,
                                           int lane, bool gram) {
  const int tid = threadIdx.x;
  if (gram) {
    const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16) + kTcGramCol + 32u * warp;
    const int i = 32 * warp + lane;  // tensor-memory lane = (q, r)
    const int r = i % R, q = i / R;
    const int first = q * R - 32 * warp;  // first needed column inside the 32 loaded
    float v[32];
    tmem_ld32(taddr, v);
    // stage[q][r][c], rows padded to R + 1 (one column of the lanes: distinct banks)
#pragma unroll
    for (int c = 0; c < 32; ++c)
      if (c >= first && c < first + R) stage[(q * R + r) * (R + 1) + (c - first)] = v[c];
  }
#pragma unroll
  for (int r = 0; r < R; ++r) {
    float v = dacc[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    if (lane == 0) dstage[warp * R + r] = v;
    dacc[r] = 0.f;
  }
  __syncthreads();
#pragma unroll
  for (int j = 0; j < R * R / kTcThreads; ++j) {
    if (!gram) break;
    const int e = tid + kTcThreads * j, r = e / R, c = e % R;
    double acc = 0.0;
#pragma unroll
    for (int q = 0; q < kTcRows / R; ++q)
      acc += (double)stage[(q * R + r) * (R + 1) + c] + (double)stage[(q * R + c) * (R + 1) + r];
    greg[j] += 0.5 * acc;
  }
  if (tid < R) {
    double acc = 0.0;
#pragma unroll
    for (int w = 0; w < kTcThreads / 32; ++w) acc += (double)dstage[w * R + tid];
    dreg += acc;
  }
  __syncthreads();  // the buffers serve as Gram operands again
}

// chunk (row, 4 c .. 4 c + 3) of the A operand, split into its hi and lo halves
template <int R>
__device__ __forceinline__ void split_chunk(unsigned char *sm, int row, int c, float4 x) {
  using L = TcLayout<R>;
  float4 h, l;
  h.x = tf32_rna(x.x);
  h.y = tf32_rna(x.y);
  h.z = tf32_rna(x.z);
  h.w = tf32_rna(x.w);
  l.x = tf32_rna(x.x - h.x);
  l.y = tf32_rna(x.y - h.y);
  l.z = tf32_rna(x.z - h.z);
  l.w = tf32_rna(x.w - h.w);
  const uint32_t o = op_off(row, 4 * c, kLboG, L::kSboA);
  *reinterpret_cast<float4 *>(sm + L::ah + o) = h;
  *reinterpret_cast<float4 *>(sm + L::al + o) = l;
}

// row `row` of the A operand, whole (hi + lo)
template <int R>
__device__ __forceinline__ void read_row(const unsigned char *sm, int row, float (&x)[R]) {
  using L = TcLayout<R>;
#pragma unroll
  for (int c = 0; c < R / 4; ++c) {
    const uint32_t o = op_off(row, 4 * c, kLboG, L::kSboA);
    const float4 h = *reinterpret_cast<const float4 *>(sm + L::ah + o);
    const float4 l = *reinterpret_cast<const float4 *>(sm + L::al + o);
    x[4 * c] = h.x + l.x;
    x[4 * c + 1] = h.y + l.y;
    x[4 * c + 2] = h.z + l.z;
    x[4 * c + 3] = h.w + l.w;
  }
}

// D (columns 0..R-1) = A operand x the W operand at wh (hi; lo follows it),
// issued by thread 0 after the barrier the caller passed; every thread then
// waits (bounded) for the MMAs. Returns false (on every thread) on expiry;
// `pending` tells whether a completion is still owed on bar.
template <int R>
__device__ __forceinline__ bool tc_product(uint32_t sbase, uint32_t wh, uint32_t tbase, uint32_t idesc,
                                           uint64_t *bar, uint32_t &phase, bool &pending) {
  using L = TcLayout<R>;
  if (threadIdx.x == 0) {
    tc_fence_after();
#pragma unroll
    for (int s = 0; s < R / 8; ++s) {
      const uint64_t a_h = smem_desc(sbase + L::ah + s * 2 * kLboG, kLboG, L::kSboA);
      const uint64_t a_l = smem_desc(sbase + L::al + s * 2 * kLboG, kLboG, L::kSboA);
      const uint64_t w_h = smem_desc(sbase + wh + s * 256, 128, L::kSboW);
      const uint64_t w_l = smem_desc(sbase + wh + L::kW + s * 256, 128, L::kSboW);
      mma_tf32(tbase, a_h, w_h, idesc, s > 0);
      mma_tf32(tbase, a_h, w_l, idesc, 1);
      mma_tf32(tbase, a_l, w_h, idesc, 1);
    }
    mma_commit(bar);
  }
  pending = true;
  if (!__syncthreads_and(mbar_wait_bounded(bar, phase, kTcWaitNs))) return false;  // the phase stays owed
  phase ^= 1;
  pending = false;
  tc_fence_after();
  return true;
}

// this thread's row (tensor-memory lane) of columns 0..R-1
template <int R>
__device__ __forceinline__ void tc_row(uint32_t tbase, int warp, float (&v)[R]) {
  const uint32_t taddr = tbase + ((uint32_t)(32 * warp) << 16);
  if constexpr (R == 32)
    tmem_ld32(taddr, v);
  else
    tmem_ld16(taddr, v);
}

template <int R>
__global__ void __launch_bounds__(kTcThreads, 2)
    update_tc_kernel(const float *__restrict__ M, const float *__restrict__ W, float *__restrict__ Bout,
                     uint64_t I, double *__restrict__ BtB, double *__restrict__ dot,
                     const int *__restrict__ done_at, int it, uint32_t *status) {
  static_assert(R == 16 || R == 32, "tensor-core update: R = 16 or 32");
  using L = TcLayout<R>;
  if (*done_at <= it) return;
  extern __shared__ __align__(128) unsigned char sm[];
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + L::bar);
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + L::tmem);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const uint32_t sbase = smem_u32(sm);

  if (warp == 0) {
    tmem_alloc(tslot, kTcCols);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bar[0], 1);
    mbar_init(&bar[1], 1);
    fence_mbar_init();
  }
  // W1 and W2 operands: element (n, k) = W[k][n], split
  for (int e = tid; e < 2 * R * R; e += kTcThreads) {
    const int f = e / (R * R), k = (e % (R * R)) / R, n = e % R;
    const float x = W[e];
    const float h = tf32_rna(x);
    const uint32_t o = op_off(n, k, 128, L::kSboW) + (f ? L::w2h : L::w1h);
    *reinterpret_cast<float *>(sm + o) = h;
    *reinterpret_cast<float *>(sm + o + L::kW) = tf32_rna(x - h);
  }
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;

  constexpr uint32_t idB = idesc_tf32(kTcRows, R);
  constexpr uint32_t idG = idesc_tf32(kTcRows, kTcRows);
  const uint64_t ntiles = (I + kTcRows - 1) / kTcRows;
  float dacc[R];
#pragma unroll
  for (int r = 0; r < R; ++r) dacc[r] = 0.f;
  double greg[R * R / kTcThreads], dreg = 0.0;
#pragma unroll
  for (int j = 0; j < R * R / kTcThreads; ++j) greg[j] = 0.0;
  float *stage = reinterpret_cast<float *>(sm + L::gh), *dstage = reinterpret_cast<float *>(sm + L::gl);
  // the tile's rows arrive coalesced: warp w loads rows 32 w .. 32 w + 31,
  // lane j the 16-byte chunks e = 32 v + j (row e / (R/4), chunk e % (R/4))
  constexpr int kChunks = R / 4;
  auto load_tile = [&](uint64_t t, float4 (&m)[kChunks]) {
#pragma unroll
    for (int v = 0; v < kChunks; ++v) {
      const int e = 32 * v + lane;
      const uint64_t row = t * kTcRows + 32 * warp + e / kChunks;
      m[v] = (t < ntiles && row < I) ? __ldcs(reinterpret_cast<const float4 *>(M + row * R) + e % kChunks)
                                     : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  uint32_t ph0 = 0, ph1 = 0;
  bool b_pending = false, gram_pending = false;
  int since_flush = 0;
  // one tile; cur holds its rows, nxt receives the rows of the tile after
  auto tile = [&](uint64_t t, float4 (&cur)[kChunks], float4 (&nxt)[kChunks]) -> bool {
    // 1. this tile's M rows into the A operand, the next tile's rows in flight
#pragma unroll
    for (int v = 0; v < kChunks; ++v) {
      const int e = 32 * v + lane;
      split_chunk<R>(sm, 32 * warp + e / kChunks, e % kChunks, cur[v]);
    }
    load_tile(t + gridDim.x, nxt);
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    // 2. Y tile = M tile W1; then B tile = Y tile W2
    float m[R], b[R];
    read_row<R>(sm, tid, m);  // this thread's M row, for the dot products
    if (!tc_product<R>(sbase, L::w1h, tbase, idB, &bar[0], ph0, b_pending)) return false;
    tc_row<R>(tbase, warp, b);
    // the Y row replaces the M row in the A operand (the MMAs reading it are done)
#pragma unroll
    for (int c = 0; c < kChunks; ++c)
      split_chunk<R>(sm, tid, c, make_float4(b[4 * c], b[4 * c + 1], b[4 * c + 2], b[4 * c + 3]));
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    if (!tc_product<R>(sbase, L::w2h, tbase, idB, &bar[0], ph0, b_pending)) return false;
    // 3. the B row of this thread: store, dot products, Gram operand
    tc_row<R>(tbase, warp, b);
    const uint64_t row = t * kTcRows + tid;
    if (row < I) {
      float4 *dst = reinterpret_cast<float4 *>(Bout + row * R);
#pragma unroll
      for (int c = 0; c < kChunks; ++c)
        __stcs(dst + c, make_float4(b[4 * c], b[4 * c + 1], b[4 * c + 2], b[4 * c + 3]));
    }
#pragma unroll
    for (int r = 0; r < R; ++r) dacc[r] = fmaf(m[r], b[r], dacc[r]);
    if (gram_pending) {
      // the previous Gram MMAs still read the Gram operand
      if (!__syncthreads_and(mbar_wait_bounded(&bar[1], ph1, kTcWaitNs))) return false;  // owed
      ph1 ^= 1;
      gram_pending = false;
    }
    if (since_flush == kTcFlush) {
      tc_fence_after();
      flush_sums<R>(tbase, stage, dstage, dacc, greg, dreg, warp, lane, true);
      since_flush = 0;
    }
    {
      // G[(q, r)][k] = B[q R + k][r]: hi, and 2 lo (see flush_sums)
      const int q = tid / R, k = tid % R;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const float h = tf32_rna(b[r]);
        const uint32_t o = op_off(q * R + r, k, kLboG, L::kSboG);
        *reinterpret_cast<float *>(sm + L::gh + o) = h;
        *reinterpret_cast<float *>(sm + L::gl + o) = 2.f * tf32_rna(b[r] - h);
      }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    // 4. the chunks' Gram blocks: G G^T + 2 G lo^T
    if (tid == 0) {
      tc_fence_after();
#pragma unroll
      for (int s = 0; s < R / 8; ++s) {
        const uint64_t g_h = smem_desc(sbase + L::gh + s * 2 * kLboG, kLboG, L::kSboG);
        const uint64_t g_l = smem_desc(sbase + L::gl + s * 2 * kLboG, kLboG, L::kSboG);
        mma_tf32(tbase + kTcGramCol, g_h, g_h, idG, (since_flush > 0 || s > 0) ? 1u : 0u);
        mma_tf32(tbase + kTcGramCol, g_h, g_l, idG, 1);
      }
      mma_commit(&bar[1]);
    }
    gram_pending = true;
    ++since_flush;
    return true;
  };
  float4 m0[kChunks], m1[kChunks];
  load_tile(blockIdx.x, m0);
  bool ok = true;
  for (uint64_t t = blockIdx.x; t < ntiles; t += 2ull * gridDim.x) {
    if (!(ok = tile(t, m0, m1))) break;
    if (t + gridDim.x >= ntiles) break;
    if (!(ok = tile(t + gridDim.x, m1, m0))) break;
  }
  if (!ok) {
    // an MMA did not complete in time: report it, give the MMAs one more
    // bounded wait, free the tensor memory and stop
    if (tid == 0) {
      atomicOr(status, kStatusTimeout);
      if (b_pending) mbar_wait_bounded(&bar[0], ph0, kTcWaitNs);
      if (gram_pending) mbar_wait_bounded(&bar[1], ph1, kTcWaitNs);
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
      tc_fence_after();
      tmem_dealloc(tbase, kTcCols);
    }
    return;
  }
  if (gram_pending && !__syncthreads_and(mbar_wait_bounded(&bar[1], ph1, kTcWaitNs))) {
    if (tid == 0) atomicOr(status, kStatusTimeout);
    since_flush = 0;  // the accumulator is not complete: not read
  }
  tc_fence_after();
  flush_sums<R>(tbase, stage, dstage, dacc, greg, dreg, warp, lane, since_flush > 0);
  tc_fence_before();
  __syncthreads();
  if (warp == 0) {
    tc_fence_after();
    tmem_dealloc(tbase, kTcCols);
  }
#pragma unroll
  for (int j = 0; j < R * R / kTcThreads; ++j)
    if (greg[j] != 0.0) atomicAdd(&BtB[tid + kTcThreads * j], greg[j]);
  if (tid < R && dreg != 0.0) atomicAdd(&dot[tid], dreg);
}

template <int R>
cudaError_t launch_update_tc_r(const float *M, const float *W, float *B, uint64_t I, double *BtB, double *dot,
                               const int *done_at, int it, uint32_t *status, int num_sms, cudaStream_t s) {
  using L = TcLayout<R>;
  static bool configured = false;
  if (!configured) {
    cudaError_t e = cudaFuncSetAttribute(update_tc_kernel<R>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)L::total);
    if (e != cudaSuccess) return e;
    configured = true;
  }
  const uint64_t ntiles = (I + kTcRows - 1) / kTcRows;
  const uint64_t cap = (uint64_t)num_sms * 2;
  const int grid = (int)(ntiles < cap ? ntiles : cap);
  update_tc_kernel<R><<<grid, kTcThreads, L::total, s>>>(M, W, B, I, BtB, dot, done_at, it, status);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace

bool update_tc_supported(int R) { return R == 16 || R == 32; }

cudaError_t launch_update_tc(const float *M, const float *W, float *B, uint64_t I, int R, double *BtB,
                             double *dot, const int *done_at, int it, uint32_t *status, int num_sms,
                             cudaStream_t s) {
  if (I == 0) return cudaSuccess;
  if (R == 32) return launch_update_tc_r<32>(M, W, B, I, BtB, dot, done_at, it, status, num_sms, s);
  if (R == 16) return launch_update_tc_r<16>(M, W, B, I, BtB, dot, done_at, it, status, num_sms, s);
  return cudaErrorInvalidValue;
}

}  // namespace alto
