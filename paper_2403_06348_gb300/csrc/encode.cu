// ALTO encode kernels (Section III-A: linearization and ordering; Section IV-A:
// balanced line segments and mode intervals) plus the hot-row sampling used by
// the ATOMIC MTTKRP variant.
#include "encode.cuh"

#include <algorithm>
#include <vector>

namespace alto {

// ---------------------------------------------------------------------------
// Linearization: position = OR over modes of PDEP(i_n, mask_n), built from the
// strided runs of the bit plan. Also sums ||X||^2 and checks coordinate range
// (an out-of-range coordinate sets a status bit and is clamped to 0, so every
// key stays decodable to in-range rows).
// ---------------------------------------------------------------------------
template <int KW>
__global__ void __launch_bounds__(256) linearize_kernel(const __grid_constant__ DecodePlan dp,
                                                        const uint32_t *__restrict__ coords,
                                                        uint64_t nnz, const uint64_t *__restrict__ dims_dev,
                                                        uint64_t *__restrict__ keys,
                                                        uint32_t *__restrict__ status) {
  bool bad = false;
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nnz;
       x += (uint64_t)gridDim.x * blockDim.x) {
    uint64_t lo = 0, hi = 0;
#pragma unroll
    for (int n = 0; n < kMaxModes; ++n) {
      if (n < dp.nmodes) {
        uint32_t c = coords[(uint64_t)n * nnz + x];
        if ((uint64_t)c >= dims_dev[n]) {
          bad = true;
          c = 0;
        }
        for (int r = 0; r < dp.nruns[n]; ++r) {
          const BitRun br = dp.runs[n][r];
          const uint64_t e = expand_stride((uint64_t)(c >> br.outshift), br.stride, br.count);
          if (KW == 1) {
            lo |= e << br.shift;
          } else {
            if (br.shift < 64) {
              lo |= e << br.shift;
              if (br.shift) hi |= e >> (64 - br.shift);
            } else {
              hi |= e << (br.shift - 64);
            }
          }
        }
      }
    }
    keys[x * KW] = lo;
    if (KW == 2) keys[x * KW + 1] = hi;
  }
  if (bad) atomicOr(status, kStatusCoordRange);
}

// ---------------------------------------------------------------------------
// ||X||^2 over cells: after the sort, entries with equal coordinates form runs
// of equal positions; every run is one cell whose value is the run's sum.
// norm_runs_kernel: one thread per chunk of kNormChunk entries squares the
// runs that start and end inside its chunk and leaves the partial sums of runs
// that cross its edges; norm_span_kernel: the chunk where a crossing run starts
// adds up the pieces and squares the total.
// ---------------------------------------------------------------------------
constexpr int kNormChunk = 32;
constexpr uint8_t kContLeft = 1, kContRight = 2, kSingleRun = 4;

template <int KW>
__device__ __forceinline__ bool same_key(const uint64_t *k, uint64_t a, uint64_t b) {
  if (KW == 1) return k[a] == k[b];
  return k[2 * a] == k[2 * b] && k[2 * a + 1] == k[2 * b + 1];
}

__device__ __forceinline__ void block_add_double(double v, double *out) {
  __shared__ double red[32];
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (lane == 0) red[warp] = v;
  __syncthreads();
  if (warp == 0) {
    double s = lane < (int)(blockDim.x >> 5) ? red[lane] : 0.0;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if (lane == 0 && s != 0.0) atomicAdd(out, s);
  }
}

template <int KW>
__global__ void __launch_bounds__(256) norm_runs_kernel(const uint64_t *__restrict__ keys,
                                                        const float *__restrict__ vals, uint64_t nnz,
                                                        uint64_t nchunks, double *__restrict__ head,
                                                        double *__restrict__ tail,
                                                        uint8_t *__restrict__ flags,
                                                        double *__restrict__ norm_sq) {
  double acc = 0.0;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t first = c * kNormChunk;
    const uint64_t last = (first + kNormChunk < nnz ? first + kNormChunk : nnz) - 1;
    const bool cl = first > 0 && same_key<KW>(keys, first, first - 1);
    const bool cr = last + 1 < nnz && same_key<KW>(keys, last, last + 1);
    double run = (double)vals[first], hd = 0.0;
    bool first_run = true;
    for (uint64_t x = first + 1; x <= last; ++x) {
      if (same_key<KW>(keys, x, x - 1)) {
        run += (double)vals[x];
      } else {
        if (first_run && cl)
          hd = run;
        else
          acc += run * run;
        first_run = false;
        run = (double)vals[x];
      }
    }
    if (first_run) hd = run;
    if (!cr && !(first_run && cl)) acc += run * run;
    head[c] = hd;
    tail[c] = run;
    flags[c] = (cl ? kContLeft : 0) | (cr ? kContRight : 0) | (first_run ? kSingleRun : 0);
  }
  block_add_double(acc, norm_sq);
}

__global__ void __launch_bounds__(256) norm_span_kernel(const double *__restrict__ head,
                                                        const double *__restrict__ tail,
                                                        const uint8_t *__restrict__ flags,
                                                        uint64_t nchunks, double *__restrict__ norm_sq) {
  double acc = 0.0;
  for (uint64_t c = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
       c += (uint64_t)gridDim.x * blockDim.x) {
    const uint8_t f = flags[c];
    if ((f & kContRight) && !((f & kSingleRun) && (f & kContLeft))) {
      double S = tail[c];
      for (uint64_t k = c + 1; k < nchunks; ++k) {
        const uint8_t fk = flags[k];
        S += head[k];
        if (!((fk & kSingleRun) && (fk & kContRight))) break;
      }
      acc += S * S;
    }
  }
  block_add_double(acc, norm_sq);
}

// ---------------------------------------------------------------------------
// Stable LSD radix sort of (position, value) pairs with 8-bit digits.
// One histogram kernel reads the positions once and counts the digits of
// every pass. Then one kernel per pass ranks each tile of 4096 items in
// shared memory, finds the tile's first output slot per digit by a chained
// scan over the tiles (each tile publishes its own digit counts, then looks
// back over its predecessors until it meets a running total, and publishes
// its own), and writes the tile out through shared memory, one digit run
// after the other. Tiles are handed out in start order through a ticket
// counter, so a tile only waits on tiles whose CTAs already run; every wait
// is bounded (2 s) and reports kStatusTimeout.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096
constexpr int kRadix = 256;
constexpr int kMaxSortPasses = 16;                     // 128-bit positions
constexpr int kHistItems = 8;
constexpr uint64_t kLookLimitNs = 2000000000ull;
constexpr int kLookWindow = 8;

// look-back word: bits 63-62 kind (1 = the tile's own count, 2 = running
// total through the tile), bits 61-56 the pass (1-based), bits 31-0 the count
constexpr uint64_t kLookOwn = 1ull << 62;
constexpr uint64_t kLookTotal = 2ull << 62;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

// lanes of the warp holding the same digit (d < 512; 256 marks "no item"):
// nine ballots, one per bit, intersected
__device__ __forceinline__ unsigned digit_peers(uint32_t d) {
  unsigned m = 0xffffffffu;
#pragma unroll
  for (int b = 0; b < 9; ++b) {
    const bool set = (d >> b) & 1u;
    const unsigned bal = __ballot_sync(0xffffffffu, set);
    m &= set ? bal : ~bal;
  }
  return m;
}

__device__ __forceinline__ uint64_t ld_relaxed_u64(const uint64_t *p) {
  uint64_t v;
  asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(uint64_t *p, uint64_t v) {
  asm volatile("st.relaxed.gpu.global.u64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

__device__ __forceinline__ uint64_t sort_clock_ns() {
  uint64_t t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}

template <int KW>
__device__ __forceinline__ uint32_t sort_digit(const uint64_t (&k)[KW], int bit) {
  const uint64_t kd = (KW == 2 && bit >= 64) ? k[KW - 1] : k[0];
  return (uint32_t)((kd >> (bit & 63)) & 0xFFu);
}

// hist[p * 256 + d] += number of positions whose digit p is d, p < passes.
// One shared-memory atomic per digit: the counts need no ranks, and peers
// found by ballots cost more issue slots than the atomics' conflicts.
template <int KW>
__global__ void __launch_bounds__(kSortThreads) radix_hist_kernel(const uint64_t *__restrict__ keys,
                                                                  uint64_t nnz, int passes,
                                                                  uint32_t *__restrict__ hist) {
  __shared__ uint32_t sh[kMaxSortPasses * kRadix];
  for (int i = threadIdx.x; i < passes * kRadix; i += kSortThreads) sh[i] = 0;
  __syncthreads();
  const uint64_t step = (uint64_t)gridDim.x * kSortThreads * kHistItems;
  for (uint64_t base = (uint64_t)blockIdx.x * kSortThreads * kHistItems; base < nnz; base += step) {
    uint64_t k[kHistItems][KW];
#pragma unroll
    for (int i = 0; i < kHistItems; ++i) {
      const uint64_t x = base + (uint64_t)i * kSortThreads + threadIdx.x;
#pragma unroll
      for (int w = 0; w < KW; ++w) k[i][w] = x < nnz ? __ldcs(keys + x * KW + w) : 0ull;
    }
#pragma unroll
    for (int i = 0; i < kHistItems; ++i) {
      if (base + (uint64_t)i * kSortThreads + threadIdx.x >= nnz) continue;
      for (int p = 0; p < passes; ++p) atomicAdd(&sh[p * kRadix + sort_digit<KW>(k[i], 8 * p)], 1u);
    }
  }
  __syncthreads();
  for (int i = threadIdx.x; i < passes * kRadix; i += kSortThreads)
    if (sh[i]) atomicAdd(&hist[i], sh[i]);
}

// --- exclusive scan over the block (values and total < 2^32) ---------------
__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v) {
  __shared__ uint32_t warp_sums[32];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  uint32_t inc = v;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const uint32_t y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) warp_sums[warp] = inc;
  __syncthreads();
  if (warp == 0) {
    const int nw = (blockDim.x + 31) >> 5;
    uint32_t s = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
      if (lane >= o) s += y;
    }
    warp_sums[lane] = s;  // inclusive
  }
  __syncthreads();
  const uint32_t warp_prefix = warp ? warp_sums[warp - 1] : 0u;
  __syncthreads();
  return warp_prefix + inc - v;
}

// One pass: digit (keys >> bit) & 0xFF of every position, stable.
// hist = this pass's 256 digit counts; look = ntiles x 256 words, zero or
// left by other passes; ticket = this pass's counter, zero.
template <int KW>
__global__ void __launch_bounds__(kSortThreads, 2) radix_pass_kernel(
    const uint64_t *__restrict__ keys_in, const float *__restrict__ vals_in, uint64_t nnz, int bit,
    uint32_t pass_tag, const uint32_t *__restrict__ hist, uint64_t *look, uint32_t *ticket,
    uint32_t *status, uint64_t *__restrict__ keys_out, float *__restrict__ vals_out) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(sm);                         // kSortTile * KW
  float *sv = reinterpret_cast<float *>(sk + (size_t)kSortTile * KW);     // kSortTile
  uint32_t *wcount = reinterpret_cast<uint32_t *>(sv + kSortTile);        // 8 * 256
  uint32_t *dstart = wcount + 8 * kRadix;                                  // 256
  uint32_t *gbase = dstart + kRadix;                                       // 256
  __shared__ uint32_t s_tile;

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  if (threadIdx.x == 0) s_tile = atomicAdd(ticket, 1u);
  for (int i = threadIdx.x; i < 8 * kRadix; i += kSortThreads) wcount[i] = 0;
  __syncthreads();
  const uint32_t t = s_tile;
  const uint64_t tile_base = (uint64_t)t * kSortTile;

  // warp w owns items [w*512, w*512+512) of the tile, in 16 rounds of 32
  uint64_t k[kSortItems][KW];
  float v[kSortItems];
  uint32_t rank[kSortItems];
  uint32_t dig[kSortItems];
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const uint64_t x = tile_base + (uint64_t)warp * (32 * kSortItems) + r * 32 + lane;
    const bool valid = x < nnz;
#pragma unroll
    for (int w = 0; w < KW; ++w) k[r][w] = valid ? __ldcs(keys_in + x * KW + w) : 0ull;
    v[r] = valid ? __ldcs(vals_in + x) : 0.f;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const uint64_t x = tile_base + (uint64_t)warp * (32 * kSortItems) + r * 32 + lane;
    const bool valid = x < nnz;
    const uint32_t d = valid ? sort_digit<KW>(k[r], bit) : (uint32_t)kRadix;
    dig[r] = d;
    const unsigned peers = digit_peers(d);
    const int leader = __ffs(peers) - 1;
    uint32_t basev = 0;
    if (lane == leader && valid) {
      basev = wcount[warp * kRadix + d];
      wcount[warp * kRadix + d] = basev + (uint32_t)__popc(peers);
    }
    basev = __shfl_sync(0xffffffffu, basev, leader);
    rank[r] = basev + (uint32_t)__popc(peers & lanemask_lt());
    __syncwarp();
  }
  __syncthreads();
  const int d = threadIdx.x;  // thread d looks after digit d from here on
  const uint64_t tag = (uint64_t)pass_tag << 56;
  uint64_t *mine = look + (uint64_t)t * kRadix + d;
  uint32_t run = 0;
#pragma unroll
  for (int w = 0; w < 8; ++w) {
    const uint32_t c = wcount[w * kRadix + d];
    wcount[w * kRadix + d] = run;
    run += c;
  }
  // the tile's own count goes out first, so that later tiles can pass it
  st_relaxed_u64(mine, (t == 0 ? kLookTotal : kLookOwn) | tag | run);
  dstart[d] = block_exclusive_scan(run);
  const uint32_t digit_base = block_exclusive_scan(hist[d]);
  // the tile in sorted order in shared memory (slots inside the tile only)
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const uint32_t dd = dig[r];
    if (dd < kRadix) {
      const uint32_t pos = dstart[dd] + wcount[warp * kRadix + dd] + rank[r];
#pragma unroll
      for (int w = 0; w < KW; ++w) sk[(size_t)pos * KW + w] = k[r][w];
      sv[pos] = v[r];
    }
  }
  // look back over the preceding tiles, kLookWindow words per round trip:
  // own counts are summed until a running total ends the walk
  uint32_t before = 0;
  if (t > 0) {
    int64_t j = (int64_t)t - 1;
    bool done = false;
    uint32_t idle = 0;
    uint64_t t0 = 0;
    while (!done) {
      uint64_t wv[kLookWindow];
#pragma unroll
      for (int i = 0; i < kLookWindow; ++i)
        wv[i] = j - i >= 0 ? ld_relaxed_u64(look + (uint64_t)(j - i) * kRadix + d) : 0ull;
      int used = 0;
      bool gap = false;
#pragma unroll
      for (int i = 0; i < kLookWindow; ++i) {
        if (done || gap) continue;
        const uint64_t x = wv[i];
        if (j - i < 0) {
          done = true;  // past tile 0, which always holds a total
        } else if ((x >> 62) != 0 && ((x >> 56) & 0x3Fu) == pass_tag) {
          before += (uint32_t)x;
          ++used;
          done = (x >> 62) == 2;
        } else {
          gap = true;   // not published yet
        }
      }
      j -= used;
      if (!done && used == 0) {
        __nanosleep(64);
        if ((++idle & 15u) == 0) {
          const uint64_t now = sort_clock_ns();
          if (t0 == 0) {
            t0 = now;
          } else if (now - t0 > kLookLimitNs) {
            atomicOr(status, kStatusTimeout);
            break;
          }
        }
      }
    }
    st_relaxed_u64(mine, kLookTotal | tag | (uint32_t)(before + run));
  }
  gbase[d] = digit_base + before;
  __syncthreads();
  const uint64_t rem = nnz - tile_base;
  const uint32_t count = rem < (uint64_t)kSortTile ? (uint32_t)rem : (uint32_t)kSortTile;
#pragma unroll 4
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t idx = i * kSortThreads + threadIdx.x;
    if (idx < count) {
      uint64_t kk[KW];
#pragma unroll
      for (int w = 0; w < KW; ++w) kk[w] = sk[(size_t)idx * KW + w];
      const uint32_t d = sort_digit<KW>(kk, bit);
      const uint64_t dst = (uint64_t)gbase[d] + (idx - dstart[d]);
      // a timed-out look-back leaves wrong offsets: stay inside the arrays
      if (dst < nnz) {
#pragma unroll
        for (int w = 0; w < KW; ++w) keys_out[dst * KW + w] = kk[w];
        vals_out[dst] = sv[idx];
      }
    }
  }
}

// ---------------------------------------------------------------------------
// Partition (Section IV-A): segment l = [floor(l*M/L), floor((l+1)*M/L)),
// closed per-mode interval [min, max] of its decoded coordinates.
// ---------------------------------------------------------------------------
template <int KW>
__global__ void __launch_bounds__(256) partition_kernel(const __grid_constant__ DecodePlan dp,
                                                        const uint64_t *__restrict__ keys,
                                                        uint64_t nnz, uint64_t L,
                                                        uint32_t *__restrict__ intervals,
                                                        uint32_t *__restrict__ max_len) {
  __shared__ uint32_t smin[8][kMaxModes], smax[8][kMaxModes];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int N = dp.nmodes;
  for (uint64_t l = blockIdx.x; l < L; l += gridDim.x) {
    const uint64_t s0 = (l * nnz) / L, s1 = ((l + 1) * nnz) / L;
    uint32_t mn[kMaxModes], mx[kMaxModes];
#pragma unroll
    for (int n = 0; n < kMaxModes; ++n) {
      mn[n] = kEmptyRow;
      mx[n] = 0;
    }
    for (uint64_t x = s0 + threadIdx.x; x < s1; x += blockDim.x) {
      const uint64_t lo = keys[x * KW];
      const uint64_t hi = KW == 2 ? keys[x * KW + 1] : 0ull;
      uint32_t c[kMaxModes];
      decode_all<KW>(dp, lo, hi, c);
#pragma unroll
      for (int n = 0; n < kMaxModes; ++n) {
        mn[n] = min(mn[n], c[n]);
        mx[n] = max(mx[n], c[n]);
      }
    }
#pragma unroll
    for (int n = 0; n < kMaxModes; ++n) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        mn[n] = min(mn[n], __shfl_xor_sync(0xffffffffu, mn[n], o));
        mx[n] = max(mx[n], __shfl_xor_sync(0xffffffffu, mx[n], o));
      }
    }
    if (lane == 0) {
#pragma unroll
      for (int n = 0; n < kMaxModes; ++n) {
        smin[warp][n] = mn[n];
        smax[warp][n] = mx[n];
      }
    }
    __syncthreads();
    if (threadIdx.x < N) {
      const int n = threadIdx.x;
      uint32_t a = kEmptyRow, b = 0;
      for (int w = 0; w < (int)(blockDim.x >> 5); ++w) {
        a = min(a, smin[w][n]);
        b = max(b, smax[w][n]);
      }
      if (s1 <= s0) {
        a = kEmptyRow;
        b = 0;
      }
      intervals[(l * N + n) * 2] = a;
      intervals[(l * N + n) * 2 + 1] = b;
      if (s1 > s0) atomicMax(&max_len[n], b - a + 1);
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// Hot rows: row counts of every mode on a strided sample of the ordered
// nonzeros; rows whose estimated count clears a threshold are kept, at most
// ALTO_MAX_HOT per mode, most frequent first.
// ---------------------------------------------------------------------------
template <int KW>
__global__ void __launch_bounds__(256) sample_counts_kernel(const __grid_constant__ DecodePlan dp,
                                                            const uint64_t *__restrict__ keys,
                                                            uint64_t nnz, uint64_t stride,
                                                            uint64_t nsamples,
                                                            uint32_t *const *__restrict__ counts) {
  for (uint64_t s = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; s < nsamples;
       s += (uint64_t)gridDim.x * blockDim.x) {
    const uint64_t x = s * stride;
    const uint64_t lo = keys[x * KW];
    const uint64_t hi = KW == 2 ? keys[x * KW + 1] : 0ull;
    uint32_t c[kMaxModes];
    decode_all<KW>(dp, lo, hi, c);
#pragma unroll
    for (int n = 0; n < kMaxModes; ++n) {
      if (n < dp.nmodes) {
        const unsigned peers = __match_any_sync(__activemask(), c[n]);
        if ((peers & lanemask_lt()) == 0) atomicAdd(&counts[n][c[n]], (uint32_t)__popc(peers));
      }
    }
  }
}

__global__ void count_buckets_kernel(const uint32_t *__restrict__ counts, uint64_t I,
                                     uint32_t min_count, uint32_t *__restrict__ buckets) {
  __shared__ uint32_t h[33];
  if (threadIdx.x < 33) h[threadIdx.x] = 0;
  __syncthreads();
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = counts[i];
    if (c >= min_count && c > 0) atomicAdd(&h[31 - __clz(c)], 1u);
  }
  __syncthreads();
  if (threadIdx.x < 33 && h[threadIdx.x]) atomicAdd(&buckets[threadIdx.x], h[threadIdx.x]);
}

__global__ void pick_threshold_kernel(const uint32_t *__restrict__ buckets, uint32_t min_count,
                                      uint32_t cap, uint32_t *__restrict__ thr) {
  if (threadIdx.x == 0 && blockIdx.x == 0) {
    uint32_t acc = 0;
    int b = 32;
    while (b > 0 && acc + buckets[b - 1] <= cap) {
      acc += buckets[b - 1];
      --b;
    }
    // rows with count >= 2^b (b = first bucket kept) fit in cap
    // when even the top bucket alone exceeds cap, take part of it
    uint32_t t = b >= 32 ? 0x80000000u : (1u << b);
    if (b == 0) t = 1u;
    *thr = t > min_count ? t : min_count;
  }
}

__global__ void collect_hot_kernel(const uint32_t *__restrict__ counts, uint64_t I,
                                   const uint32_t *__restrict__ thr, uint32_t cap,
                                   uint64_t *__restrict__ list, uint32_t *__restrict__ nlist) {
  const uint32_t t = *thr;
  for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < I;
       i += (uint64_t)gridDim.x * blockDim.x) {
    const uint32_t c = counts[i];
    if (c >= t && c > 0) {
      const uint32_t p = atomicAdd(nlist, 1u);
      // descending count, then ascending row: sort ascending on (~count, row)
      if (p < cap) list[p] = ((uint64_t)(~c) << 32) | (uint64_t)i;
    }
  }
}

// single block bitonic sort of up to ALTO_MAX_HOT 64-bit keys; writes rows
__global__ void __launch_bounds__(1024) sort_hot_kernel(const uint64_t *__restrict__ list,
                                                        const uint32_t *__restrict__ nlist,
                                                        uint32_t cap, uint32_t *__restrict__ rows,
                                                        uint32_t *__restrict__ nhot) {
  __shared__ uint64_t s[ALTO_MAX_HOT];
  uint32_t n = *nlist;
  if (n > cap) n = cap;
  for (int i = threadIdx.x; i < ALTO_MAX_HOT; i += blockDim.x) s[i] = i < (int)n ? list[i] : ~0ull;
  __syncthreads();
  for (int k = 2; k <= ALTO_MAX_HOT; k <<= 1) {
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int i = threadIdx.x; i < ALTO_MAX_HOT; i += blockDim.x) {
        const int p = i ^ j;
        if (p > i) {
          const uint64_t a = s[i], b = s[p];
          const bool up = (i & k) == 0;
          if ((a > b) == up) {
            s[i] = b;
            s[p] = a;
          }
        }
      }
      __syncthreads();
    }
  }
  for (int i = threadIdx.x; i < (int)n; i += blockDim.x) rows[i] = (uint32_t)(s[i] & 0xFFFFFFFFull);
  if (threadIdx.x == 0) *nhot = n;
}

// ---------------------------------------------------------------------------
// Full de-linearization (test aid)
// ---------------------------------------------------------------------------
template <int KW>
__global__ void decode_kernel(const __grid_constant__ DecodePlan dp, const uint64_t *__restrict__ keys,
                              uint64_t nnz, uint32_t *__restrict__ coords) {
  for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < nnz;
       x += (uint64_t)gridDim.x * blockDim.x) {
    uint32_t c[kMaxModes];
    decode_all<KW>(dp, keys[x * KW], KW == 2 ? keys[x * KW + 1] : 0ull, c);
#pragma unroll
    for (int n = 0; n < kMaxModes; ++n)
      if (n < dp.nmodes) coords[(uint64_t)n * nnz + x] = c[n];
  }
}

// ---------------------------------------------------------------------------
// host-side launchers
// ---------------------------------------------------------------------------
static int grid_for(uint64_t work, int threads, int max_blocks) {
  uint64_t b = (work + threads - 1) / threads;
  if (b < 1) b = 1;
  if (b > (uint64_t)max_blocks) b = max_blocks;
  return (int)b;
}

cudaError_t launch_linearize(const DecodePlan &dp, const uint32_t *coords, uint64_t nnz,
                             const uint64_t *dims_dev, uint64_t *keys, uint32_t *status, int num_sms,
                             cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  const int grid = grid_for(nnz, 256, num_sms * 8);
  if (dp.kw == 1)
    linearize_kernel<1><<<grid, 256, 0, s>>>(dp, coords, nnz, dims_dev, keys, status);
  else
    linearize_kernel<2><<<grid, 256, 0, s>>>(dp, coords, nnz, dims_dev, keys, status);
  note_launches(1);
  return cudaGetLastError();
}

uint64_t norm_chunks(uint64_t nnz) { return (nnz + kNormChunk - 1) / kNormChunk; }

cudaError_t launch_norm(int kw, const uint64_t *keys, const float *vals, uint64_t nnz, double *head,
                        double *tail, uint8_t *flags, double *norm_sq, int num_sms, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  const uint64_t nc = norm_chunks(nnz);
  const int grid = grid_for(nc, 256, num_sms * 8);
  if (kw == 1)
    norm_runs_kernel<1><<<grid, 256, 0, s>>>(keys, vals, nnz, nc, head, tail, flags, norm_sq);
  else
    norm_runs_kernel<2><<<grid, 256, 0, s>>>(keys, vals, nnz, nc, head, tail, flags, norm_sq);
  norm_span_kernel<<<grid, 256, 0, s>>>(head, tail, flags, nc, norm_sq);
  note_launches(2);
  return cudaGetLastError();
}

size_t sort_workspace_bytes(uint64_t nnz) {
  const uint64_t ntiles = (nnz + kSortTile - 1) / kSortTile;
  return (size_t)ntiles * kRadix * 8 + (size_t)kMaxSortPasses * kRadix * 4 + kMaxSortPasses * 4;
}

static size_t pass_smem(int kw) {
  return (size_t)kSortTile * (8 * kw + 4) + (8 * kRadix + 2 * kRadix) * 4;
}

template <int KW>
static cudaError_t radix_sort_t(int passes, uint64_t nnz, uint64_t *keys[2], float *vals[2],
                                const float *vals_in, void *work, uint32_t *status,
                                bool skip_constant, int *final_buf, int *passes_run, int num_sms,
                                cudaStream_t s) {
  static bool attr_set = false;
  if (!attr_set) {
    cudaError_t e = cudaFuncSetAttribute(radix_pass_kernel<KW>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)pass_smem(KW));
    if (e != cudaSuccess) return e;
    attr_set = true;
  }
  const uint32_t ntiles = (uint32_t)((nnz + kSortTile - 1) / kSortTile);
  uint64_t *look = static_cast<uint64_t *>(work);
  uint32_t *hist = reinterpret_cast<uint32_t *>(look + (size_t)ntiles * kRadix);
  uint32_t *tickets = hist + kMaxSortPasses * kRadix;
  cudaError_t e = cudaMemsetAsync(work, 0, sort_workspace_bytes(nnz), s);
  if (e != cudaSuccess) return e;
  const uint64_t per_block = (uint64_t)kSortThreads * kHistItems;
  const uint64_t hist_blocks = (nnz + per_block - 1) / per_block;
  const int hgrid = (int)std::min<uint64_t>(hist_blocks, (uint64_t)num_sms * 4);
  radix_hist_kernel<KW><<<hgrid, kSortThreads, 0, s>>>(keys[0], nnz, passes, hist);
  note_launches(1);
  if ((e = cudaGetLastError()) != cudaSuccess) return e;
  bool skip[kMaxSortPasses] = {};
  if (skip_constant) {
    // a digit that one value covers leaves the order as it is
    std::vector<uint32_t> hh((size_t)passes * kRadix);
    if ((e = cudaMemcpyAsync(hh.data(), hist, hh.size() * 4, cudaMemcpyDeviceToHost, s)) != cudaSuccess ||
        (e = cudaStreamSynchronize(s)) != cudaSuccess)
      return e;
    for (int p = 0; p < passes; ++p)
      for (int d = 0; d < kRadix; ++d)
        if (hh[(size_t)p * kRadix + d] == nnz) skip[p] = true;
  }
  int cur = 0;
  const float *vin = vals_in;
  for (int p = 0; p < passes; ++p) {
    if (skip[p]) continue;
    const int nxt = cur ^ 1;
    radix_pass_kernel<KW><<<ntiles, kSortThreads, pass_smem(KW), s>>>(
        keys[cur], vin, nnz, 8 * p, (uint32_t)(p + 1), hist + (size_t)p * kRadix, look, tickets + p,
        status, keys[nxt], vals[nxt]);
    note_launches(1);
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    cur = nxt;
    vin = vals[cur];
    if (passes_run) ++*passes_run;
  }
  if (vin == vals_in) {
    // no pass moved anything: the values are still the caller's
    if ((e = cudaMemcpyAsync(vals[0], vals_in, nnz * sizeof(float), cudaMemcpyDeviceToDevice, s)) !=
        cudaSuccess)
      return e;
  }
  *final_buf = cur;
  return cudaSuccess;
}

cudaError_t launch_radix_sort(int kw, int nbits, uint64_t nnz, uint64_t *keys[2], float *vals[2],
                              const float *vals_in, void *work, uint32_t *status, bool skip_constant,
                              int *final_buf, int *passes_run, int num_sms, cudaStream_t s) {
  // keys[0] holds the input positions; vals_in the input values. The result
  // ends in keys[*final_buf] / vals[*final_buf].
  *final_buf = 0;
  if (passes_run) *passes_run = 0;
  if (nnz == 0) return cudaSuccess;
  const int passes = (nbits + 7) / 8;
  if (passes == 0)
    return cudaMemcpyAsync(vals[0], vals_in, nnz * sizeof(float), cudaMemcpyDeviceToDevice, s);
  if (kw == 1)
    return radix_sort_t<1>(passes, nnz, keys, vals, vals_in, work, status, skip_constant, final_buf,
                           passes_run, num_sms, s);
  return radix_sort_t<2>(passes, nnz, keys, vals, vals_in, work, status, skip_constant, final_buf,
                         passes_run, num_sms, s);
}

cudaError_t launch_partition(const DecodePlan &dp, const uint64_t *keys, uint64_t nnz, uint64_t L,
                             uint32_t *intervals, uint32_t *max_len, int num_sms, cudaStream_t s) {
  const int grid = (int)(L < (uint64_t)num_sms * 16 ? L : (uint64_t)num_sms * 16);
  if (dp.kw == 1)
    partition_kernel<1><<<grid, 256, 0, s>>>(dp, keys, nnz, L, intervals, max_len);
  else
    partition_kernel<2><<<grid, 256, 0, s>>>(dp, keys, nnz, L, intervals, max_len);
  note_launches(1);
  return cudaGetLastError();
}

cudaError_t launch_hot_rows(const DecodePlan &dp, const uint64_t *keys, uint64_t nnz,
                            const uint64_t *dims, uint64_t L, uint32_t *const *counts_dev_ptrs,
                            uint32_t *const *counts_host_ptrs, uint32_t *scratch /*64 words*/,
                            uint64_t *list /*ALTO_MAX_HOT*/, uint32_t *const *hot_rows,
                            uint32_t *nhot /*per mode*/, int num_sms, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  const uint64_t max_samples = 1ull << 21;
  const uint64_t stride = nnz > max_samples ? (nnz + max_samples - 1) / max_samples : 1;
  const uint64_t nsamples = (nnz + stride - 1) / stride;
  const int grid = grid_for(nsamples, 256, num_sms * 8);
  if (dp.kw == 1)
    sample_counts_kernel<1><<<grid, 256, 0, s>>>(dp, keys, nnz, stride, nsamples, counts_dev_ptrs);
  else
    sample_counts_kernel<2><<<grid, 256, 0, s>>>(dp, keys, nnz, stride, nsamples, counts_dev_ptrs);
  note_launches(1);
  // a row is a candidate when its estimated count reaches one per segment
  uint64_t mc = (L + stride - 1) / stride;
  if (mc < 2) mc = 2;
  const uint32_t min_count = (uint32_t)(mc > 0xFFFFFFFFull ? 0xFFFFFFFFull : mc);
  for (int n = 0; n < dp.nmodes; ++n) {
    uint32_t *buckets = scratch;       // 33
    uint32_t *thr = scratch + 40;      // 1
    uint32_t *nlist = scratch + 41;    // 1
    cudaError_t e = cudaMemsetAsync(scratch, 0, 64 * sizeof(uint32_t), s);
    if (e != cudaSuccess) return e;
    const int g = grid_for(dims[n], 256, num_sms * 8);
    count_buckets_kernel<<<g, 256, 0, s>>>(counts_host_ptrs[n], dims[n], min_count, buckets);
    pick_threshold_kernel<<<1, 32, 0, s>>>(buckets, min_count, ALTO_MAX_HOT, thr);
    collect_hot_kernel<<<g, 256, 0, s>>>(counts_host_ptrs[n], dims[n], thr, ALTO_MAX_HOT, list,
                                         nlist);
    sort_hot_kernel<<<1, 1024, 0, s>>>(list, nlist, ALTO_MAX_HOT, hot_rows[n], nhot + n);
    note_launches(4);
    e = cudaGetLastError();
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

cudaError_t launch_decode(const DecodePlan &dp, const uint64_t *keys, uint64_t nnz, uint32_t *coords,
                          int num_sms, cudaStream_t s) {
  if (nnz == 0) return cudaSuccess;
  const int grid = grid_for(nnz, 256, num_sms * 8);
  if (dp.kw == 1)
    decode_kernel<1><<<grid, 256, 0, s>>>(dp, keys, nnz, coords);
  else
    decode_kernel<2><<<grid, 256, 0, s>>>(dp, keys, nnz, coords);
  note_launches(1);
  return cudaGetLastError();
}

}  // namespace alto
