// ALTO encode kernels (Section III-A: linearization and ordering; Section IV-A:
// balanced line segments and mode intervals) plus the hot-row sampling used by
// the ATOMIC MTTKRP variant.
#include "encode.cuh"

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
// Stable LSD radix sort of (position, value) pairs, 8-bit digits,
// reduce-then-scan per pass: upsweep (per-tile digit counts), exclusive scan
// of the digit-major count table, downsweep (stable local ranks, staged in
// shared memory, coalesced write-out). No inter-CTA waiting anywhere.
// ---------------------------------------------------------------------------
constexpr int kSortThreads = 256;
constexpr int kSortItems = 16;
constexpr int kSortTile = kSortThreads * kSortItems;  // 4096
constexpr int kRadix = 256;

__device__ __forceinline__ unsigned lanemask_lt() {
  unsigned m;
  asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
  return m;
}

template <int KW>
__global__ void __launch_bounds__(kSortThreads) radix_upsweep(const uint64_t *__restrict__ keys,
                                                             uint64_t nnz, int word, int shift,
                                                             uint32_t ntiles,
                                                             uint32_t *__restrict__ table) {
  __shared__ uint32_t hist[kRadix];
  const uint32_t t = blockIdx.x;
  hist[threadIdx.x] = 0;
  __syncthreads();
  const uint64_t base = (uint64_t)t * kSortTile;
  // all of the thread's digits first (16 loads in flight), then the counts
  uint32_t dig[kSortItems];
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint64_t x = base + (uint64_t)i * kSortThreads + threadIdx.x;
    dig[i] = x < nnz ? (uint32_t)((keys[x * KW + word] >> shift) & 0xFFu) : kRadix;
  }
#pragma unroll
  for (int i = 0; i < kSortItems; ++i) {
    const uint32_t d = dig[i];
    const bool valid = d < kRadix;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
    if (valid && (peers & lanemask_lt()) == 0) atomicAdd(&hist[d], (uint32_t)__popc(peers));
  }
  __syncthreads();
  table[(uint64_t)threadIdx.x * ntiles + t] = hist[threadIdx.x];
}

// --- exclusive scan of a uint32 table (values and total < 2^32) ------------
constexpr int kScanThreads = 1024;
constexpr int kScanItems = 4;
constexpr int kScanBlock = kScanThreads * kScanItems;

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t *total) {
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
  if (total) *total = warp_sums[((blockDim.x + 31) >> 5) - 1];
  __syncthreads();
  return warp_prefix + inc - v;
}

__global__ void __launch_bounds__(kScanThreads) scan_reduce(const uint32_t *__restrict__ in,
                                                            uint64_t n,
                                                            uint32_t *__restrict__ sums) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanBlock;
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    const uint64_t x = base + (uint64_t)i * kScanThreads + threadIdx.x;
    if (x < n) s += in[x];
  }
  uint32_t total;
  block_exclusive_scan(s, &total);
  if (threadIdx.x == 0) sums[blockIdx.x] = total;
}

__global__ void __launch_bounds__(kScanThreads) scan_top(uint32_t *__restrict__ sums, uint32_t n) {
  // single block: exclusive scan of n block sums in place
  const uint32_t per = (n + kScanThreads - 1) / kScanThreads;
  const uint32_t b = threadIdx.x * per;
  uint32_t s = 0;
  for (uint32_t i = 0; i < per && b + i < n; ++i) s += sums[b + i];
  uint32_t run = block_exclusive_scan(s, nullptr);
  for (uint32_t i = 0; i < per && b + i < n; ++i) {
    const uint32_t v = sums[b + i];
    sums[b + i] = run;
    run += v;
  }
}

__global__ void __launch_bounds__(kScanThreads) scan_down(const uint32_t *__restrict__ in, uint64_t n,
                                                          const uint32_t *__restrict__ sums,
                                                          uint32_t *__restrict__ out) {
  const uint64_t base = (uint64_t)blockIdx.x * kScanBlock + (uint64_t)threadIdx.x * kScanItems;
  uint32_t v[kScanItems];
  uint32_t s = 0;
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    v[i] = (base + i < n) ? in[base + i] : 0u;
    s += v[i];
  }
  uint32_t run = block_exclusive_scan(s, nullptr) + sums[blockIdx.x];
#pragma unroll
  for (int i = 0; i < kScanItems; ++i) {
    if (base + i < n) out[base + i] = run;
    run += v[i];
  }
}

template <int KW>
struct SortItem {
  uint64_t k[KW];
};

template <int KW>
__global__ void __launch_bounds__(kSortThreads) radix_downsweep(
    const uint64_t *__restrict__ keys_in, const float *__restrict__ vals_in, uint64_t nnz,
    int word, int shift, uint32_t ntiles, const uint32_t *__restrict__ offsets,
    uint64_t *__restrict__ keys_out, float *__restrict__ vals_out) {
  extern __shared__ __align__(16) unsigned char sm[];
  uint64_t *sk = reinterpret_cast<uint64_t *>(sm);                         // kSortTile * KW
  float *sv = reinterpret_cast<float *>(sk + (size_t)kSortTile * KW);     // kSortTile
  uint32_t *wcount = reinterpret_cast<uint32_t *>(sv + kSortTile);        // 8 * 256
  uint32_t *dstart = wcount + 8 * kRadix;                                  // 256
  uint32_t *gbase = dstart + kRadix;                                       // 256

  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const uint32_t t = blockIdx.x;
  const uint64_t tile_base = (uint64_t)t * kSortTile;
  for (int i = threadIdx.x; i < 8 * kRadix; i += kSortThreads) wcount[i] = 0;
  gbase[threadIdx.x] = offsets[(uint64_t)threadIdx.x * ntiles + t];
  __syncthreads();

  // warp w owns items [w*512, w*512+512) of the tile, in 16 rounds of 32
  uint64_t k[kSortItems][KW];
  float v[kSortItems];
  uint32_t rank[kSortItems];
  uint32_t dig[kSortItems];
  // all of the thread's items first (loads in flight together), then the ranks
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const uint64_t x = tile_base + (uint64_t)warp * (32 * kSortItems) + r * 32 + lane;
    const bool valid = x < nnz;
#pragma unroll
    for (int w = 0; w < KW; ++w) k[r][w] = valid ? keys_in[x * KW + w] : 0ull;
    v[r] = valid ? vals_in[x] : 0.f;
  }
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const uint64_t x = tile_base + (uint64_t)warp * (32 * kSortItems) + r * 32 + lane;
    const bool valid = x < nnz;
    const uint64_t kd = (KW == 2 && word) ? k[r][KW - 1] : k[r][0];
    const uint32_t d = valid ? (uint32_t)((kd >> shift) & 0xFFu) : kRadix;
    dig[r] = d;
    const unsigned peers = __match_any_sync(0xffffffffu, d);
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
  // per-digit exclusive offsets across warps, then across digits
  {
    const int d = threadIdx.x;
    uint32_t run = 0;
#pragma unroll
    for (int w = 0; w < 8; ++w) {
      const uint32_t c = wcount[w * kRadix + d];
      wcount[w * kRadix + d] = run;
      run += c;
    }
    const uint32_t ex = block_exclusive_scan(run, nullptr);
    dstart[d] = ex;
  }
  __syncthreads();
#pragma unroll
  for (int r = 0; r < kSortItems; ++r) {
    const uint32_t d = dig[r];
    if (d < kRadix) {
      const uint32_t pos = dstart[d] + wcount[warp * kRadix + d] + rank[r];
#pragma unroll
      for (int w = 0; w < KW; ++w) sk[(size_t)pos * KW + w] = k[r][w];
      sv[pos] = v[r];
    }
  }
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
      const uint64_t kd = (KW == 2 && word) ? kk[KW - 1] : kk[0];
      const uint32_t d = (uint32_t)((kd >> shift) & 0xFFu);
      const uint64_t dst = (uint64_t)gbase[d] + (idx - dstart[d]);
#pragma unroll
      for (int w = 0; w < KW; ++w) keys_out[dst * KW + w] = kk[w];
      vals_out[dst] = sv[idx];
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

size_t sort_table_entries(uint64_t nnz) {
  const uint64_t ntiles = (nnz + kSortTile - 1) / kSortTile;
  return (size_t)ntiles * kRadix;
}

size_t sort_scan_blocks(uint64_t nnz) {
  return (sort_table_entries(nnz) + kScanBlock - 1) / kScanBlock;
}

static size_t downsweep_smem(int kw) {
  return (size_t)kSortTile * (8 * kw + 4) + (8 * kRadix + 2 * kRadix) * 4;
}

cudaError_t launch_radix_sort(int kw, int nbits, uint64_t nnz, uint64_t *keys[2], float *vals[2],
                              const float *vals_in, uint32_t *table, uint32_t *table_scan,
                              uint32_t *block_sums, int *final_buf, cudaStream_t s) {
  // keys[0] holds the input positions; vals_in the input values. The result
  // ends in keys[*final_buf] / vals[*final_buf].
  *final_buf = 0;
  if (nnz == 0) return cudaSuccess;
  const int passes = (nbits + 7) / 8;
  if (passes == 0) {
    cudaError_t e = cudaMemcpyAsync(vals[0], vals_in, nnz * sizeof(float),
                                    cudaMemcpyDeviceToDevice, s);
    return e;
  }
  const uint32_t ntiles = (uint32_t)((nnz + kSortTile - 1) / kSortTile);
  const uint64_t entries = (uint64_t)ntiles * kRadix;
  const uint32_t nblocks = (uint32_t)((entries + kScanBlock - 1) / kScanBlock);
  const size_t smem = downsweep_smem(kw);
  static bool attr_set[3] = {false, false, false};
  if (!attr_set[kw]) {
    cudaError_t e = kw == 1 ? cudaFuncSetAttribute(radix_downsweep<1>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)downsweep_smem(1))
                            : cudaFuncSetAttribute(radix_downsweep<2>,
                                                   cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                   (int)downsweep_smem(2));
    if (e != cudaSuccess) return e;
    attr_set[kw] = true;
  }
  int cur = 0;
  const float *vin = vals_in;
  for (int p = 0; p < passes; ++p) {
    const int bit = p * 8;
    const int word = bit >> 6, shift = bit & 63;
    if (kw == 1)
      radix_upsweep<1><<<ntiles, kSortThreads, 0, s>>>(keys[cur], nnz, word, shift, ntiles, table);
    else
      radix_upsweep<2><<<ntiles, kSortThreads, 0, s>>>(keys[cur], nnz, word, shift, ntiles, table);
    scan_reduce<<<nblocks, kScanThreads, 0, s>>>(table, entries, block_sums);
    scan_top<<<1, kScanThreads, 0, s>>>(block_sums, nblocks);
    scan_down<<<nblocks, kScanThreads, 0, s>>>(table, entries, block_sums, table_scan);
    const int nxt = cur ^ 1;
    if (kw == 1)
      radix_downsweep<1><<<ntiles, kSortThreads, smem, s>>>(keys[cur], vin, nnz, word, shift, ntiles,
                                                            table_scan, keys[nxt], vals[nxt]);
    else
      radix_downsweep<2><<<ntiles, kSortThreads, smem, s>>>(keys[cur], vin, nnz, word, shift, ntiles,
                                                            table_scan, keys[nxt], vals[nxt]);
    note_launches(5);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    cur = nxt;
    vin = vals[cur];
  }
  *final_buf = cur;
  return cudaSuccess;
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
