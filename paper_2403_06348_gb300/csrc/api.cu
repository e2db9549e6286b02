// C ABI of the ALTO library: handle management, the bit plan of Section III-A,
// and the orchestration of the encode, MTTKRP and CP-ALS kernels.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "alto_internal.cuh"
#include "apr.cuh"
#include "cpals.cuh"
#include "handle.cuh"
#include "encode.cuh"
#include "mttkrp.cuh"

using namespace alto;

namespace {
std::atomic<uint64_t> g_launches{0};
}  // namespace

void alto::note_launches(int n) { g_launches.fetch_add((uint64_t)n, std::memory_order_relaxed); }

namespace {

thread_local std::string g_last_error;

}  // namespace

alto_status alto::fail(alto_status st, const char *fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  g_last_error = buf;
  return st;
}


void *alto::dalloc(alto_tensor *h, size_t bytes, cudaStream_t s) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (h->user_alloc) {
    p = h->alloc.alloc(bytes, (void *)s, h->alloc.ctx);
  } else if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) h->bytes_held += bytes;
  return p;
}

void alto::dfree(alto_tensor *h, void *p, size_t bytes, cudaStream_t s) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  if (h->user_alloc)
    h->alloc.free(p, bytes, (void *)s, h->alloc.ctx);
  else
    cudaFreeAsync(p, s);
  h->bytes_held -= bytes;
}

namespace {

cudaEvent_t prof_event(alto_tensor *h) {
  if (!h->prof_pool.empty()) {
    cudaEvent_t e = h->prof_pool.back();
    h->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Brackets the kernels launched in its scope with CUDA events on stream s.
struct ProfScope {
  alto_tensor *h;
  int kind;
  cudaStream_t s;
  cudaEvent_t a = nullptr;
  ProfScope(alto_tensor *h_, int kind_, cudaStream_t s_) : h(h_), kind(kind_), s(s_) {
    if (h->prof_on && (a = prof_event(h)) != nullptr) cudaEventRecord(a, s);
  }
  ~ProfScope() {
    if (!a) return;
    cudaEvent_t b = prof_event(h);
    if (!b) {
      h->prof_pool.push_back(a);
      return;
    }
    cudaEventRecord(b, s);
    h->prof_pending.push_back(ProfEvt{kind, a, b});
  }
};

template <typename T>
alto_status alloc_n(alto_tensor *h, T **p, size_t n, cudaStream_t s, const char *what) {
  *p = static_cast<T *>(dalloc(h, n * sizeof(T), s));
  if (!*p) return fail(ALTO_ERR_OOM, "allocation of %zu bytes for %s failed", n * sizeof(T), what);
  return ALTO_OK;
}

int mode_bits(uint64_t I) {
  if (I <= 1) return 0;
  return 64 - __builtin_clzll(I - 1);
}

// Section III-A bit plan: groups from the LSB, shortest mode lowest.
alto_status build_bit_plan(alto_tensor *h) {
  const int N = h->N;
  int order[kMaxModes];
  for (int n = 0; n < N; ++n) {
    order[n] = n;
    h->bits[n] = mode_bits(h->dims[n]);
  }
  std::stable_sort(order, order + N, [&](int a, int b) { return h->dims[a] < h->dims[b]; });
  int pos[kMaxModes][32];
  int p = 0, maxb = 0;
  for (int n = 0; n < N; ++n) maxb = std::max(maxb, h->bits[n]);
  for (int g = 0; g < maxb; ++g)
    for (int k = 0; k < N; ++k) {
      const int n = order[k];
      if (h->bits[n] > g) pos[n][g] = p++;
    }
  h->nbits = p;
  if (p > 128) return fail(ALTO_ERR_UNSUPPORTED, "%d index bits exceed 128", p);
  h->kw = p <= 64 ? 1 : 2;
  DecodePlan &dp = h->dp;
  memset(&dp, 0, sizeof(dp));
  dp.nmodes = N;
  dp.kw = h->kw;
  for (int n = 0; n < N; ++n) {
    h->mask_lo[n] = h->mask_hi[n] = 0;
    for (int g = 0; g < h->bits[n]; ++g) {
      if (pos[n][g] < 64)
        h->mask_lo[n] |= 1ull << pos[n][g];
      else
        h->mask_hi[n] |= 1ull << (pos[n][g] - 64);
    }
    // split the mode's positions into arithmetic runs inside 64-bit windows
    int nr = 0, g = 0;
    while (g < h->bits[n]) {
      const int start = pos[n][g];
      int stride = 1, cnt = 1;
      if (g + 1 < h->bits[n]) {
        const int d = pos[n][g + 1] - start;
        if (d <= 8 && pos[n][g + 1] - start < 64) {
          stride = d;
          cnt = 2;
          while (g + cnt < h->bits[n] && pos[n][g + cnt] - pos[n][g + cnt - 1] == stride &&
                 pos[n][g + cnt] - start < 64)
            ++cnt;
        }
      }
      if (nr >= kMaxRuns) return fail(ALTO_ERR_UNSUPPORTED, "bit plan needs too many runs");
      dp.runs[n][nr].shift = (uint8_t)start;
      dp.runs[n][nr].stride = (uint8_t)stride;
      dp.runs[n][nr].count = (uint8_t)cnt;
      dp.runs[n][nr].outshift = (uint8_t)g;
      ++nr;
      g += cnt;
    }
    dp.nruns[n] = nr;
  }
  // 32-bit runs with precomputed compaction masks (the MTTKRP decode)
  DecodePlan32 &d32 = h->dp32;
  memset(&d32, 0, sizeof(d32));
  d32.nmodes = N;
  d32.kw = h->kw;
  for (int n = 0; n < N; ++n) {
    int nr = 0, g = 0;
    while (g < h->bits[n]) {
      const int start = pos[n][g];
      int k = 1, cnt = 1;
      if (g + 1 < h->bits[n] && pos[n][g + 1] - start < 32) {
        k = pos[n][g + 1] - start;
        cnt = 2;
        while (g + cnt < h->bits[n] && pos[n][g + cnt] - pos[n][g + cnt - 1] == k &&
               pos[n][g + cnt] - start < 32)
          ++cnt;
      }
      if (nr >= kMaxRuns32) return fail(ALTO_ERR_UNSUPPORTED, "bit plan needs too many runs");
      Run32 &r = d32.runs[n][nr++];
      r.start = (uint8_t)start;
      r.outshift = (uint8_t)g;
      int steps = 0;
      while ((1 << steps) < cnt) ++steps;
      r.steps = (uint8_t)steps;
      uint32_t m0 = 0;
      for (int t = 0; t < cnt; ++t) m0 |= 1u << (k * t);
      r.mask[0] = m0;
      for (int j = 0; j < steps; ++j) {
        r.sh[j] = (uint8_t)((k - 1) << j);
        // after step j: groups of 2^(j+1) bits at multiples of k * 2^(j+1)
        uint32_t m = 0;
        const int gsz = 1 << (j + 1), sp = k * gsz;
        for (int p = 0; p < 32; p += sp)
          for (int b = 0; b < gsz && p + b < 32; ++b) m |= 1u << (p + b);
        r.mask[j + 1] = m;
      }
      g += cnt;
    }
    d32.nruns[n] = nr;
  }
  // the block view of the same plan (Section III-A), ranks = modes by length
  BlockPlan &bp = h->bp;
  memset(&bp, 0, sizeof(bp));
  bp.nmodes = N;
  bp.kw = h->kw;
  for (int q = 0; q < N; ++q) {
    h->mode_of[q] = order[q];
    h->rank_of[order[q]] = q;
  }
  int base = 0, prev_bits = 0;
  for (int j = 0; j < N; ++j) {
    const int k = N - j;
    const int cnt = h->bits[order[j]] - prev_bits;
    bp.base[j] = (uint8_t)base;
    bp.off[j] = (uint8_t)prev_bits;
    const int h1 = std::min(cnt, 63 / k + 1);
    for (int t = 0; t < h1; ++t) bp.mask[j] |= 1ull << (k * t);
    if (cnt > h1) {
      bp.shift2[j] = (uint8_t)(h1 * k);
      bp.off2[j] = (uint8_t)(prev_bits + h1);
      for (int t = 0; t < cnt - h1; ++t) bp.mask2[j] |= 1ull << (k * t);
      if (h->kw == 1) return fail(ALTO_ERR_UNSUPPORTED, "internal: block wider than 64 bits");
    }
    base += cnt * k;
    prev_bits = h->bits[order[j]];
  }
  return ALTO_OK;
}

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

uint64_t default_parts(uint64_t M, int num_sms) {
  if (M == 0) return 1;
  uint64_t L = (M + 16383) / 16384;
  const uint64_t want = std::min<uint64_t>((M + 1023) / 1024, 2ull * (uint64_t)num_sms);
  return std::max<uint64_t>(std::max<uint64_t>(L, want), 1);
}

void free_pull(alto_tensor *h, int n, cudaStream_t s) {
  PullPlan &pp = h->pull[n];
  if (pp.part_off) dfree(h, pp.part_off, h->L * sizeof(uint64_t), s);
  if (pp.row_ptr) dfree(h, pp.row_ptr, (h->dims[n] + 1) * sizeof(uint64_t), s);
  if (pp.prow) dfree(h, pp.prow, pp.entries * sizeof(uint64_t), s);
  pp = PullPlan();
}

void free_hot(alto_tensor *h, int n, cudaStream_t s) {
  HotTable &ht = h->hot_tab[n];
  if (ht.htab) dfree(h, ht.htab, ((size_t)1 << ht.hbits) * sizeof(uint64_t), s);
  ht = HotTable();
}

alto_status run_partition(alto_tensor *h, uint64_t L, cudaStream_t s) {
  if (h->intervals) dfree(h, h->intervals, h->L * h->N * 2 * sizeof(uint32_t), s);
  h->intervals = nullptr;
  h->L = L;
  alto_status st = alloc_n(h, &h->intervals, (size_t)L * h->N * 2, s, "intervals");
  if (st != ALTO_OK) return st;
  CUDA_TRY(cudaMemsetAsync(h->max_len_dev, 0, kMaxModes * sizeof(uint32_t), s));
  if (h->M == 0) {
    CUDA_TRY(cudaMemsetAsync(h->intervals, 0xFF, (size_t)L * h->N * 2 * sizeof(uint32_t), s));
    // empty interval convention: (2^32-1, 0)
    std::vector<uint32_t> iv((size_t)L * h->N * 2);
    for (size_t i = 0; i < iv.size(); i += 2) {
      iv[i] = kEmptyRow;
      iv[i + 1] = 0;
    }
    CUDA_TRY(cudaMemcpyAsync(h->intervals, iv.data(), iv.size() * 4, cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaStreamSynchronize(s));
  } else {
    CUDA_TRY(launch_partition(h->dp, h->keys, h->M, L, h->intervals, h->max_len_dev, h->num_sms, s));
  }
  CUDA_TRY(cudaMemcpyAsync(h->max_interval, h->max_len_dev, kMaxModes * sizeof(uint32_t),
                           cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  h->intervals_host_valid = false;
  for (int n = 0; n < h->N; ++n) free_pull(h, n, s);
  return ALTO_OK;
}

alto_status ensure_intervals_host(alto_tensor *h, cudaStream_t s) {
  if (h->intervals_host_valid) return ALTO_OK;
  h->intervals_host.resize((size_t)h->L * h->N * 2);
  CUDA_TRY(cudaMemcpyAsync(h->intervals_host.data(), h->intervals,
                           h->intervals_host.size() * sizeof(uint32_t), cudaMemcpyDeviceToHost, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  h->intervals_host_valid = true;
  return ALTO_OK;
}

// Row -> segment lists of the pull reduction (Alg. 4), built on the host from
// the mode intervals; every row lists its partial rows in segment order.
alto_status ensure_pull(alto_tensor *h, int n, cudaStream_t s) {
  PullPlan &pp = h->pull[n];
  if (pp.valid) return ALTO_OK;
  alto_status st = ensure_intervals_host(h, s);
  if (st != ALTO_OK) return st;
  const uint64_t L = h->L, I = h->dims[n];
  const int N = h->N;
  std::vector<uint64_t> part_off(L);
  std::vector<uint64_t> cnt(I + 1, 0);
  uint64_t total = 0;
  for (uint64_t l = 0; l < L; ++l) {
    const uint32_t a = h->intervals_host[(l * N + n) * 2], b = h->intervals_host[(l * N + n) * 2 + 1];
    part_off[l] = total;
    if (a <= b) {
      total += (uint64_t)(b - a) + 1;
      for (uint64_t r = a; r <= b; ++r) cnt[r + 1]++;
    }
  }
  for (uint64_t i = 0; i < I; ++i) cnt[i + 1] += cnt[i];
  std::vector<uint64_t> fillpos(cnt.begin(), cnt.end() - 1);
  std::vector<uint64_t> prow(total);
  for (uint64_t l = 0; l < L; ++l) {
    const uint32_t a = h->intervals_host[(l * N + n) * 2], b = h->intervals_host[(l * N + n) * 2 + 1];
    if (a <= b)
      for (uint64_t r = a; r <= b; ++r) prow[fillpos[r]++] = part_off[l] + (r - a);
  }
  pp.total_rows = total;
  pp.entries = total;
  if ((st = alloc_n(h, &pp.part_off, L, s, "pull offsets")) != ALTO_OK) return st;
  if ((st = alloc_n(h, &pp.row_ptr, I + 1, s, "pull row pointers")) != ALTO_OK) return st;
  if ((st = alloc_n(h, &pp.prow, std::max<uint64_t>(total, 1), s, "pull lists")) != ALTO_OK) return st;
  CUDA_TRY(cudaMemcpyAsync(pp.part_off, part_off.data(), L * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(pp.row_ptr, cnt.data(), (I + 1) * 8, cudaMemcpyHostToDevice, s));
  if (total) CUDA_TRY(cudaMemcpyAsync(pp.prow, prow.data(), total * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));  // host vectors go out of scope
  pp.valid = true;
  return ALTO_OK;
}

// Hash table of the first nslots hot rows of mode n (open addressing).
alto_status build_hot_table(alto_tensor *h, int n, int nslots, HotTable &ht, cudaStream_t s) {
  if (ht.nslots == nslots && ht.htab) return ALTO_OK;
  if (ht.htab) dfree(h, ht.htab, ((size_t)1 << ht.hbits) * sizeof(uint64_t), s);
  ht = HotTable();
  int hbits = 1;
  while ((1 << hbits) < 2 * std::max(nslots, 1)) ++hbits;
  const size_t hsize = (size_t)1 << hbits;
  std::vector<uint64_t> tab(hsize, ~0ull);
  for (int sl = 0; sl < nslots; ++sl) {
    const uint32_t row = h->hot_host[n][sl];
    uint32_t k = (row * 0x9E3779B1u) >> (32 - hbits);
    while ((uint32_t)tab[k] != kEmptyRow) k = (k + 1) & (uint32_t)(hsize - 1);
    tab[k] = ((uint64_t)sl << 32) | row;
  }
  alto_status st = alloc_n(h, &ht.htab, hsize, s, "hot table");
  if (st != ALTO_OK) return st;
  CUDA_TRY(cudaMemcpyAsync(ht.htab, tab.data(), hsize * 8, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  ht.nslots = nslots;
  ht.hbits = hbits;
  return ALTO_OK;
}

// The byte table of the one-word decode (positions of at most 64 bits),
// built on the host from the bit plan on first use and kept in the handle.
alto_status ensure_lut(alto_tensor *h, cudaStream_t s) {
  if (h->kw != 1 || h->lut_dev) return ALTO_OK;
  LutPlan lp{};
  int off = 0;
  for (int q = 0; q < h->N; ++q) {
    const int b = h->bits[h->mode_of[q]];
    lp.off[q] = (uint8_t)(b ? off : 0);
    lp.bits[q] = (uint8_t)b;
    off += b;
  }
  std::vector<uint64_t> tab(kLutEntries, 0);
  for (int b = 0; b < 8; ++b)
    for (int v = 0; v < 256; ++v) {
      const uint64_t key = (uint64_t)v << (8 * b);
      uint64_t packed = 0;
      for (int n = 0; n < h->N; ++n) {
        uint64_t c = 0;
        int k = 0;
        for (int i = 0; i < 64; ++i)
          if ((h->mask_lo[n] >> i) & 1ull) c |= ((key >> i) & 1ull) << k++;
        packed |= c << lp.off[h->rank_of[n]];
      }
      tab[b * 256 + v] = packed;
    }
  uint64_t *d = nullptr;
  alto_status st = alloc_n(h, &d, kLutEntries, s, "decode table");
  if (st != ALTO_OK) return st;
  CUDA_TRY(cudaMemcpyAsync(d, tab.data(), kLutBytes, cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  h->lut_dev = d;
  h->lut_plan = lp;
  return ALTO_OK;
}

alto_status ensure_hot_table(alto_tensor *h, int n, int nslots, cudaStream_t s) {
  return build_hot_table(h, n, nslots, h->hot_tab[n], s);
}

bool rank_ok(int R) { return R == 4 || R == 8 || R == 16 || R == 32 || R == 64; }

size_t stage_budget() { return mttkrp_stage_budget(); }

int hot_slots_within(int R, int want, size_t budget) {
  int k = want;
  while (k > 0) {
    int hbits = 1;
    while ((1 << hbits) < 2 * k) ++hbits;
    if (mttkrp_smem_bytes(false, R, k, hbits, 0) <= budget) break;
    k = k * 7 / 8;
  }
  return std::max(k, 0);
}

// Hot rows outside the table take every one of their updates as a global
// atomic, summed in fp32 in arrival order; a table of at least kMinHotSlots
// rows keeps those rows' update counts (and so their rounding) small on skewed
// modes. The table fits the shared memory of kMttkrpBlocksPerSm CTAs per SM
// when it can; a larger one runs fewer CTAs per SM.
constexpr int kMinHotSlots = 512;

int hot_slots_that_fit(int R, int want) {
  int k = hot_slots_within(R, want, stage_budget());
  const int kmin = std::min(want, kMinHotSlots);
  if (k < kmin) k = hot_slots_within(R, kmin, mttkrp_smem_limit());
  return k;
}

// Hot rows the OUTPUT kernels stage: the most frequent sampled rows, as many
// as fit the shared memory of three CTAs per SM, at most kOutHotSlots. Runs of
// other rows meet at most their number of pieces of additions in fp32.
constexpr int kOutHotSlots = 256;

int out_hot_slots(const alto_tensor *h, int mode, int R) {
  return hot_slots_within(R, std::min<int>((int)h->nhot[mode], kOutHotSlots), stage_budget());
}

// The staged hot rows of mode n for an OUTPUT launch; *smem its shared memory.
alto_status out_staging(alto_tensor *h, int n, int R, MttkrpArgs &a, size_t *smem, cudaStream_t s) {
  const int nslots = out_hot_slots(h, n, R);
  alto_status st = ensure_hot_table(h, n, nslots, s);
  if (st != ALTO_OK) return st;
  const HotTable &ht = h->hot_tab[n];
  a.htab = ht.htab;
  a.slot_rows = h->hot_rows[n];
  a.hbits = ht.hbits;
  a.nslots = ht.nslots;
  *smem = mttkrp_smem_bytes(false, R, ht.nslots, ht.hbits, 0);
  return ALTO_OK;
}

// In-tile output-oriented traversal (TILED): the mode's most frequent rows
// get bins (at most kTileBins); as many of them as fit two CTAs per SM are
// staged in shared memory, the rest go to the warm replicas.
constexpr int kTileBins = 1024;

int hbits_for(int k) {
  int hb = 1;
  while ((1 << hb) < 2 * std::max(k, 1)) ++hb;
  return hb;
}

int tile_bins(const alto_tensor *h, int mode) { return std::min<int>((int)h->nhot[mode], kTileBins); }

// The byte-table decode is used when positions take one word and the table
// fits beside the rest of the layout.
bool tile_lut(const alto_tensor *h, int mode, int R, int cpl) {
  const int nb = tile_bins(h, mode);
  return h->kw == 1 && tile_smem_bytes(h->N, h->kw, R, cpl, 0, hbits_for(nb), nb, true) <= mttkrp_smem_limit();
}

int tile_slots(const alto_tensor *h, int mode, int R, int cpl) {
  const int nb = tile_bins(h, mode);
  const int hb = hbits_for(nb);
  static int per_sm = 0;
  if (!per_sm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&per_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
  }
  const size_t base = tile_smem_bytes(h->N, h->kw, R, cpl, 0, hb, nb, tile_lut(h, mode, R, cpl));
  size_t target = (size_t)per_sm / 2 - 1024;  // two CTAs per SM
  if (target > mttkrp_smem_limit()) target = mttkrp_smem_limit();
  if (base >= target) return 0;
  const size_t k = (target - base) / ((size_t)R * 4);
  return (int)std::min<size_t>(k, (size_t)nb);
}

bool tile_variant(int v) { return v == ALTO_VARIANT_TILED || v == ALTO_VARIANT_TILED_LINE; }

// Whether a TILED CTA (no staged rows) fits the shared memory of one block.
bool tile_fits(const alto_tensor *h, int mode, int R, int cpl) {
  const int nb = tile_bins(h, mode);
  return tile_smem_bytes(h->N, h->kw, R, cpl, 0, hbits_for(nb), nb, false) <= mttkrp_smem_limit();
}

alto_status resolve_plan(alto_tensor *h, int mode, int R, alto_mode_plan *out) {
  alto_mode_plan p = h->plan[mode];
  if (tile_variant(p.variant) && h->dims[mode] > 0x80000000ull) p.variant = ALTO_VARIANT_ATOMIC;
  if (tile_variant(p.variant)) {
    const bool wide = R >= 8 && (p.cols_per_lane == 0 || p.cols_per_lane >= 8);
    p.cols_per_lane = wide ? 8 : 4;
    // more lanes per nonzero means fewer groups and fewer skew slots
    if (!tile_fits(h, mode, R, p.cols_per_lane) && R >= 8) p.cols_per_lane = 8;
    if (!tile_fits(h, mode, R, p.cols_per_lane)) p.variant = ALTO_VARIANT_ATOMIC;
  }
  if (tile_variant(p.variant)) {
    const int fit = tile_slots(h, mode, R, p.cols_per_lane);
    p.hot_rows = p.hot_rows >= 0 ? std::min(p.hot_rows, fit) : fit;
    *out = p;
    return ALTO_OK;
  }
  if (p.cols_per_lane != 4 && p.cols_per_lane != 8 && p.cols_per_lane != 16 &&
      p.cols_per_lane != 32 && p.cols_per_lane != 64)
    p.cols_per_lane = 4;
  while (R % p.cols_per_lane) p.cols_per_lane /= 2;
  // one thread per nonzero needs R >= 8 (8-column chunks)
  if (p.cols_per_lane == R && R < 8) p.cols_per_lane = 4;
  if (p.cols_per_lane > 16 && p.cols_per_lane != R) p.cols_per_lane = 16;
  if (p.variant == ALTO_VARIANT_OUTPUT) {
    p.cols_per_lane = (p.cols_per_lane >= 8 && R >= 8) ? 8 : 4;
    p.hot_rows = out_hot_slots(h, mode, R);
    *out = p;
    return ALTO_OK;
  }
  const size_t pull_smem = mttkrp_smem_bytes(true, R, 0, 0, h->max_interval[mode]);
  const bool pull_fits = pull_smem <= mttkrp_smem_limit() && h->M > 0;
  if (p.variant == ALTO_VARIANT_AUTO) {
    // The output-oriented traversal through the stored order whenever the
    // order can be held: on this GPU it beats the recursive one (PULL) even
    // for modes of high fiber reuse. Otherwise the paper's rule: PULL when
    // the reuse pays for buffered accumulation and the interval fits, else
    // ATOMIC.
    const double reuse = (double)h->M / (double)h->dims[mode];
    if (h->M <= kPosOutMaxNnz && !h->pos_out_failed[mode])
      p.variant = ALTO_VARIANT_OUTPUT;
    else if (reuse > 4.0 && pull_fits)
      p.variant = ALTO_VARIANT_PULL;
    else
      p.variant = ALTO_VARIANT_ATOMIC;
    if (p.variant == ALTO_VARIANT_OUTPUT) {
      p.cols_per_lane = (p.cols_per_lane >= 8 && R >= 8) ? 8 : 4;
      p.hot_rows = out_hot_slots(h, mode, R);
      *out = p;
      return ALTO_OK;
    }
  }
  if (p.variant == ALTO_VARIANT_PULL && !pull_fits)
    return fail(ALTO_ERR_UNSUPPORTED, "mode %d: interval of %u rows does not fit shared memory",
                mode, h->max_interval[mode]);
  if (p.variant == ALTO_VARIANT_ATOMIC) {
    const int avail = (int)h->nhot[mode];
    const int want = (p.hot_rows < 0 || p.hot_rows > avail) ? avail : p.hot_rows;
    p.hot_rows = hot_slots_that_fit(R, want);
  } else {
    p.hot_rows = 0;
  }
  *out = p;
  return ALTO_OK;
}

void free_pos_out(alto_tensor *h, int n, cudaStream_t s) {
  const uint64_t M1 = std::max<uint64_t>(h->M, 1);
  dfree(h, h->pos_out[n], M1 * 4, s);
  dfree(h, h->keys_out[n], M1 * h->kw * 8, s);
  dfree(h, h->vals_out[n], M1 * 4, s);
  h->pos_out[n] = nullptr;
  h->keys_out[n] = nullptr;
  h->vals_out[n] = nullptr;
  h->pos_out_L[n] = 0;
}

// Builds (or rebuilds) the stored order of mode n with L segments (0 = the
// current count) and keeps it in the handle.
alto_status set_pos_out(alto_tensor *h, int n, uint64_t L, cudaStream_t s) {
  // default: the handle's segments, cut finer where they exceed what one CTA
  // sorts in shared memory
  if (L == 0) L = std::max<uint64_t>(h->L, (h->M + kPosOutSegCap - 1) / kPosOutSegCap);
  const uint64_t M1 = std::max<uint64_t>(h->M, 1);
  uint32_t *po = nullptr;
  uint64_t *ko = nullptr;
  float *vo = nullptr;
  alto_status st;
  {
    ProfScope ps(h, ALTO_PROF_POS_OUT, s);
    ko = static_cast<uint64_t *>(dalloc(h, M1 * h->kw * 8, s));
    vo = static_cast<float *>(dalloc(h, M1 * 4, s));
    if (!ko || !vo)
      st = fail(ALTO_ERR_OOM, "output-ordered copy of %llu nonzeros", (unsigned long long)h->M);
    else
      st = build_pos_out(h, n, L, &po, ko, vo, s);
  }
  if (st != ALTO_OK) {
    dfree(h, po, M1 * 4, s);
    dfree(h, ko, M1 * h->kw * 8, s);
    dfree(h, vo, M1 * 4, s);
    return st;
  }
  free_pos_out(h, n, s);
  h->pos_out[n] = po;
  h->keys_out[n] = ko;
  h->vals_out[n] = vo;
  h->pos_out_L[n] = h->M ? std::min<uint64_t>(std::max<uint64_t>(L, 1), h->M) : 1;
  return ALTO_OK;
}


alto_status check_handle(alto_tensor *h) {
  if (!h) return fail(ALTO_ERR_INVALID_ARG, "null handle");
  return check_device(h);
}

alto_status mttkrp_impl(alto_tensor *h, int mode, const void *const *factors, bool bf16, int R,
                        float *out, cudaStream_t s) {
  alto_mode_plan p;
  alto_status st = resolve_plan(h, mode, R, &p);
  if (st != ALTO_OK) return st;
  const uint64_t I = h->dims[mode];
  MttkrpArgs a{};
  // the kernel works on coordinates in rank order (modes sorted by length)
  a.bp = h->bp;
  a.bp.out_rank = h->rank_of[mode];
  a.out_rank = h->rank_of[mode];
  a.dp.nmodes = h->N;
  a.dp.kw = h->kw;
  for (int q = 0; q < h->N; ++q) {
    const int m = h->mode_of[q];
    a.dp.nruns[q] = h->dp32.nruns[m];
    memcpy(a.dp.runs[q], h->dp32.runs[m], sizeof(a.dp.runs[q]));
    a.factors[q] = m == mode ? nullptr : factors[m];
  }
  for (int q = 0, k = 0; q < h->N; ++q)
    if (h->mode_of[q] != mode) a.fin[k++] = factors[h->mode_of[q]];
  a.keys = h->keys;
  a.vals = h->vals;
  a.nnz = h->M;
  a.L = h->L;
  a.intervals = h->intervals;
  a.out = out;
  a.mode = mode;
  a.R = R;
  {
    const uint64_t per_seg = std::max<uint64_t>(h->M / std::max<uint64_t>(h->L, 1), 1);
    a.flush_every = (int)std::max<uint64_t>(1, 32768 / per_seg);
  }
  if (h->M == 0) {
    CUDA_TRY(cudaMemsetAsync(out, 0, I * R * sizeof(float), s));
    return ALTO_OK;
  }
  if (p.variant == ALTO_VARIANT_OUTPUT && !h->pos_out[mode] &&
      (st = set_pos_out(h, mode, 0, s)) != ALTO_OK) {
    // AUTO falls back to ATOMIC when the order cannot be held; OUTPUT asked
    // for by name reports the error
    if (st != ALTO_ERR_OOM || h->plan[mode].variant != ALTO_VARIANT_AUTO) return st;
    h->pos_out_failed[mode] = true;
    if ((st = resolve_plan(h, mode, R, &p)) != ALTO_OK) return st;
  }
  if (p.variant == ALTO_VARIANT_OUTPUT) {
    if (p.cols_per_lane == 8 && !bf16)
      for (int m = 0; m < h->N; ++m)
        if (m != mode && ((uintptr_t)factors[m] & 31u) != 0) p.cols_per_lane = 4;
    a.perm = h->pos_out[mode];
    a.keys = h->keys_out[mode];
    a.vals = h->vals_out[mode];
    size_t smem = 0;
    if ((st = out_staging(h, mode, R, a, &smem, s)) != ALTO_OK) return st;
    if (h->kw == 1 && smem + kLutBytes <= mttkrp_stage_budget()) {
      if ((st = ensure_lut(h, s)) != ALTO_OK) return st;
      a.lut = h->lut_dev;
      a.lp = h->lut_plan;
      smem += kLutBytes;
    }
    {
      ProfScope ps(h, ALTO_PROF_ZERO, s);
      CUDA_TRY(cudaMemsetAsync(out, 0, I * R * sizeof(float), s));
    }
    ProfScope ps(h, ALTO_PROF_MTTKRP, s);
    CUDA_TRY(launch_mttkrp_out(a, p.cols_per_lane, bf16, smem, h->num_sms, s));
    return ALTO_OK;
  }
  if (tile_variant(p.variant)) {
    if (p.cols_per_lane == 8 && !bf16)
      for (int m = 0; m < h->N; ++m)
        if (m != mode && ((uintptr_t)factors[m] & 31u) != 0) p.cols_per_lane = 4;
    if (!tile_fits(h, mode, R, p.cols_per_lane)) {
      // 16-byte aligned factors force 4 columns per lane, whose layout does
      // not fit here: run the mode as ATOMIC instead
      const alto_mode_plan saved = h->plan[mode];
      h->plan[mode] = alto_mode_plan{ALTO_VARIANT_ATOMIC, 4, -1};
      st = resolve_plan(h, mode, R, &p);
      h->plan[mode] = saved;
      if (st != ALTO_OK) return st;
    }
  }
  if (tile_variant(p.variant)) {
    const int nb = tile_bins(h, mode);
    const int nslots = std::min({p.hot_rows, tile_slots(h, mode, R, p.cols_per_lane), nb});
    const HotTable *tab = nullptr;
    if ((st = ensure_group_hot(h, mode, nb, s, &tab)) != ALTO_OK) return st;
    a.htab = tab->htab;
    a.hbits = tab->hbits;
    a.nbins = tab->nslots;
    a.nslots = std::min(nslots, a.nbins);
    a.slot_rows = h->hot_rows[mode];
    a.status = h->status_dev;
    if (tile_lut(h, mode, R, p.cols_per_lane)) {
      if ((st = ensure_lut(h, s)) != ALTO_OK) return st;
      a.lut = h->lut_dev;
      a.lp = h->lut_plan;
    }
    if (a.nbins > a.nslots) {
      const size_t need = (size_t)kTileWarmReps * (size_t)a.nbins * (size_t)R * sizeof(double);
      if (h->warm.bytes < need) {
        dfree(h, h->warm.p, h->warm.bytes, s);
        h->warm.p = dalloc(h, need, s);
        h->warm.bytes = h->warm.p ? need : 0;
        if (!h->warm.p) return fail(ALTO_ERR_OOM, "warm-row replicas of %zu bytes", need);
        // zero once; every launch leaves the replicas zero again
        CUDA_TRY(cudaMemsetAsync(h->warm.p, 0, need, s));
      }
      a.warm = static_cast<double *>(h->warm.p);
    }
    {
      ProfScope ps(h, ALTO_PROF_ZERO, s);
      CUDA_TRY(cudaMemsetAsync(out, 0, I * R * sizeof(float), s));
    }
    ProfScope ps(h, ALTO_PROF_MTTKRP, s);
    CUDA_TRY(launch_mttkrp_tile(a, p.cols_per_lane, bf16, p.variant == ALTO_VARIANT_TILED, h->num_sms, s));
    if (a.nbins > a.nslots)
      CUDA_TRY(launch_warm_reduce(a.warm, a.slot_rows, a.nslots, a.nbins, R, out, h->num_sms, s));
    return ALTO_OK;
  }
  if (p.variant == ALTO_VARIANT_PULL) {
    if ((st = ensure_pull(h, mode, s)) != ALTO_OK) return st;
    const PullPlan &pp = h->pull[mode];
    const size_t need = pp.total_rows * (size_t)R * sizeof(float);
    if (h->partials.bytes < need) {
      dfree(h, h->partials.p, h->partials.bytes, s);
      h->partials.p = dalloc(h, need, s);
      h->partials.bytes = h->partials.p ? need : 0;
      if (!h->partials.p) return fail(ALTO_ERR_OOM, "pull partials of %zu bytes", need);
    }
    a.partials = static_cast<float *>(h->partials.p);
    a.part_off = pp.part_off;
    const size_t smem = mttkrp_smem_bytes(true, R, 0, 0, h->max_interval[mode]);
    if (p.cols_per_lane == R || (p.cols_per_lane == 8 && !bf16))
      for (int m = 0; m < h->N; ++m)
        if (m != mode && ((uintptr_t)factors[m] & 31u) != 0) p.cols_per_lane = 4;
    {
      ProfScope ps(h, ALTO_PROF_MTTKRP, s);
      CUDA_TRY(launch_mttkrp(a, p.cols_per_lane, bf16, true, smem, h->num_sms, s));
    }
    {
      ProfScope ps(h, ALTO_PROF_PULL_REDUCE, s);
      CUDA_TRY(launch_pull_reduce(a.partials, pp.row_ptr, pp.prow, I, R, out, h->num_sms, s));
    }
  } else {
    if (p.cols_per_lane == R || (p.cols_per_lane == 8 && !bf16)) {
      // 32-byte loads (one thread per nonzero, or 8 columns per lane in fp32):
      // factors need 32-byte alignment
      for (int m = 0; m < h->N; ++m)
        if (m != mode && ((uintptr_t)factors[m] & 31u) != 0) p.cols_per_lane = 4;
    }
    if ((st = ensure_hot_table(h, mode, p.hot_rows, s)) != ALTO_OK) return st;
    const HotTable &ht = h->hot_tab[mode];
    a.htab = ht.htab;
    a.slot_rows = h->hot_rows[mode];
    a.hbits = ht.hbits;
    a.nslots = ht.nslots;
    const size_t smem = mttkrp_smem_bytes(false, R, ht.nslots, ht.hbits, 0);
    {
      ProfScope ps(h, ALTO_PROF_ZERO, s);
      CUDA_TRY(cudaMemsetAsync(out, 0, I * R * sizeof(float), s));
    }
    {
      ProfScope ps(h, ALTO_PROF_MTTKRP, s);
      CUDA_TRY(launch_mttkrp(a, p.cols_per_lane, bf16, false, smem, h->num_sms, s));
    }
  }
  return ALTO_OK;
}

bool aligned16(const void *p) { return ((uintptr_t)p & 15u) == 0; }

// Phi^(n) of Alg. 5 into phi (which the ATOMIC and OUTPUT variants need
// zeroed; the caller's inner_begin kernel does that) with the same per-mode
// conflict resolution as the MTTKRP: hot rows staged (ATOMIC), segment Temp
// and the pull reduction (PULL), or the stored output-oriented order
// (OUTPUT). 4 fp32 columns per lane.
alto_status phi_impl(alto_tensor *h, int mode, const float *const *A, const float *B,
                     const float *pimat, float eps, int R, float *phi, const int *skip,
                     cudaStream_t s) {
  alto_mode_plan p;
  alto_status st = resolve_plan(h, mode, R, &p);
  if (st != ALTO_OK) return st;
  if (p.variant == ALTO_VARIANT_OUTPUT && !h->pos_out[mode] && h->M > 0 &&
      (st = set_pos_out(h, mode, 0, s)) != ALTO_OK) {
    if (st != ALTO_ERR_OOM || h->plan[mode].variant != ALTO_VARIANT_AUTO) return st;
    h->pos_out_failed[mode] = true;  // AUTO: ATOMIC from now on
    if ((st = resolve_plan(h, mode, R, &p)) != ALTO_OK) return st;
  }
  MttkrpArgs a{};
  a.bp = h->bp;
  a.bp.out_rank = h->rank_of[mode];
  a.out_rank = h->rank_of[mode];
  a.dp.nmodes = h->N;
  a.dp.kw = h->kw;
  for (int q = 0; q < h->N; ++q) {
    const int m = h->mode_of[q];
    a.dp.nruns[q] = h->dp32.nruns[m];
    memcpy(a.dp.runs[q], h->dp32.runs[m], sizeof(a.dp.runs[q]));
    a.factors[q] = m == mode ? nullptr : A[m];
  }
  for (int q = 0, k = 0; q < h->N; ++q)
    if (h->mode_of[q] != mode) a.fin[k++] = A[h->mode_of[q]];
  a.keys = h->keys;
  a.vals = h->vals;
  a.nnz = h->M;
  a.L = h->L;
  a.intervals = h->intervals;
  a.out = phi;
  a.mode = mode;
  a.R = R;
  a.bmat = B;
  a.pimat = pimat;
  a.eps = eps;
  a.skip = skip;
  {
    const uint64_t per_seg = std::max<uint64_t>(h->M / std::max<uint64_t>(h->L, 1), 1);
    a.flush_every = (int)std::max<uint64_t>(1, 32768 / per_seg);
  }
  if (h->M == 0) return ALTO_OK;
  const bool pre = pimat != nullptr;
  if (p.variant == ALTO_VARIANT_OUTPUT) {
    a.perm = h->pos_out[mode];
    a.keys = h->keys_out[mode];
    a.vals = h->vals_out[mode];
    size_t smem = 0;
    if ((st = out_staging(h, mode, R, a, &smem, s)) != ALTO_OK) return st;
    CUDA_TRY(launch_phi_out(a, pre, smem, h->num_sms, s));
  } else if (p.variant == ALTO_VARIANT_PULL) {
    if ((st = ensure_pull(h, mode, s)) != ALTO_OK) return st;
    const PullPlan &pp = h->pull[mode];
    const size_t need = pp.total_rows * (size_t)R * sizeof(float);
    if (h->partials.bytes < need) {
      dfree(h, h->partials.p, h->partials.bytes, s);
      h->partials.p = dalloc(h, need, s);
      h->partials.bytes = h->partials.p ? need : 0;
      if (!h->partials.p) return fail(ALTO_ERR_OOM, "pull partials of %zu bytes", need);
    }
    a.partials = static_cast<float *>(h->partials.p);
    a.part_off = pp.part_off;
    const size_t smem = mttkrp_smem_bytes(true, R, 0, 0, h->max_interval[mode]);
    CUDA_TRY(launch_phi(a, true, pre, smem, h->num_sms, s));
    CUDA_TRY(launch_pull_reduce(a.partials, pp.row_ptr, pp.prow, h->dims[mode], R, phi, h->num_sms,
                                s, skip));
  } else {
    if ((st = ensure_hot_table(h, mode, p.hot_rows, s)) != ALTO_OK) return st;
    const HotTable &ht = h->hot_tab[mode];
    a.htab = ht.htab;
    a.slot_rows = h->hot_rows[mode];
    a.hbits = ht.hbits;
    a.nslots = ht.nslots;
    const size_t smem = mttkrp_smem_bytes(false, R, ht.nslots, ht.hbits, 0);
    CUDA_TRY(launch_phi(a, false, pre, smem, h->num_sms, s));
  }
  return ALTO_OK;
}

}  // namespace

alto_status alto::check_device(const alto_tensor *h) {
  int dev = -1;
  CUDA_TRY(cudaGetDevice(&dev));
  if (dev != h->device)
    return fail(ALTO_ERR_INVALID_ARG, "handle encoded on device %d, called with device %d current",
                h->device, dev);
  return ALTO_OK;
}

alto_status alto::repartition(alto_tensor *h, uint64_t L, cudaStream_t s) {
  return run_partition(h, L, s);
}

alto_status alto::ensure_group_hot(alto_tensor *h, int n, int nslots, cudaStream_t s,
                                   const HotTable **out) {
  nslots = std::min<int>(nslots, (int)h->nhot[n]);
  HotTable *slot = nullptr;
  for (HotTable &t : h->group_hot[n]) {
    if (t.htab && t.nslots == nslots) {
      *out = &t;
      return ALTO_OK;
    }
    if (!t.htab && !slot) slot = &t;
  }
  if (!slot) slot = &h->group_hot[n][0];  // more than five sizes: reuse the first
  alto_status st = build_hot_table(h, n, nslots, *slot, s);
  *out = slot;
  return st;
}

extern "C" {

const char *alto_last_error(void) { return g_last_error.c_str(); }

int alto_version(void) { return 100; }

alto_status alto_encode(const uint32_t *coords, const float *vals, const uint64_t *dims, int nmodes,
                        uint64_t nnz, const alto_allocator *alloc, void *stream, alto_handle_t *out) {
  g_last_error.clear();
  if (!out) return fail(ALTO_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (nmodes < 1 || nmodes > ALTO_MAX_MODES)
    return fail(ALTO_ERR_INVALID_ARG, "nmodes %d not in 1..%d", nmodes, ALTO_MAX_MODES);
  if (!dims) return fail(ALTO_ERR_INVALID_ARG, "dims is NULL");
  for (int n = 0; n < nmodes; ++n)
    if (dims[n] < 1 || dims[n] > 0xFFFFFFFFull)
      return fail(ALTO_ERR_INVALID_ARG, "dims[%d] = %llu not in [1, 2^32)", n,
                  (unsigned long long)dims[n]);
  if (nnz >= 0xFFFFFFFFull) return fail(ALTO_ERR_UNSUPPORTED, "nnz must be < 2^32");
  if (nnz > 0 && (!coords || !vals)) return fail(ALTO_ERR_INVALID_ARG, "coords/vals NULL");
  if (alloc && (!alloc->alloc || !alloc->free))
    return fail(ALTO_ERR_INVALID_ARG, "allocator without alloc/free");

  alto_tensor *h = new alto_tensor();
  h->N = nmodes;
  h->M = nnz;
  for (int n = 0; n < nmodes; ++n) h->dims[n] = dims[n];
  if (alloc) {
    h->alloc = *alloc;
    h->user_alloc = true;
  }
  for (int n = 0; n < kMaxModes; ++n) {
    h->plan[n].variant = ALTO_VARIANT_AUTO;
    h->plan[n].cols_per_lane = 0;
    h->plan[n].hot_rows = -1;
  }
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  alto_status st = build_bit_plan(h);
  if (st != ALTO_OK) {
    delete h;
    return st;
  }
  auto bail = [&](alto_status code) {
    alto_free(h);
    return code;
  };
  if (cudaGetDevice(&h->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, h->device) != cudaSuccess) {
    cudaGetLastError();
    delete h;
    return fail(ALTO_ERR_CUDA, "no CUDA device");
  }
  const uint64_t M = nnz;
  const int N = nmodes, kw = h->kw;

  // resident state
  if ((st = alloc_n(h, &h->dims_dev, kMaxModes, s, "dims")) != ALTO_OK) return bail(st);
  if ((st = alloc_n(h, &h->status_dev, 4, s, "status")) != ALTO_OK) return bail(st);
  if ((st = alloc_n(h, &h->norm_sq_dev, 1, s, "norm")) != ALTO_OK) return bail(st);
  if ((st = alloc_n(h, &h->max_len_dev, kMaxModes, s, "max interval")) != ALTO_OK) return bail(st);
  if ((st = alloc_n(h, &h->nhot_dev, kMaxModes, s, "hot counts")) != ALTO_OK) return bail(st);
  for (int n = 0; n < N; ++n)
    if ((st = alloc_n(h, &h->hot_rows[n], ALTO_MAX_HOT, s, "hot rows")) != ALTO_OK) return bail(st);
  uint64_t dims_pad[kMaxModes] = {};
  for (int n = 0; n < N; ++n) dims_pad[n] = dims[n];
  if (cudaMemcpyAsync(h->dims_dev, dims_pad, sizeof(dims_pad), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemsetAsync(h->status_dev, 0, 4 * sizeof(uint32_t), s) != cudaSuccess ||
      cudaMemsetAsync(h->norm_sq_dev, 0, sizeof(double), s) != cudaSuccess ||
      cudaMemsetAsync(h->nhot_dev, 0, kMaxModes * sizeof(uint32_t), s) != cudaSuccess)
    return bail(fail(ALTO_ERR_CUDA, "initialising handle state"));

  // temporaries
  uint32_t *coords_d = const_cast<uint32_t *>(coords);
  float *vals_d = const_cast<float *>(vals);
  bool own_coords = false, own_vals = false;
  uint64_t *kbuf[2] = {nullptr, nullptr};
  float *vbuf[2] = {nullptr, nullptr};
  void *sort_work = nullptr;
  uint32_t *counts = nullptr, *hot_scratch = nullptr;
  uint32_t **counts_ptrs_dev = nullptr;
  uint64_t *hot_list = nullptr;
  uint64_t sum_dims = 0;
  for (int n = 0; n < N; ++n) sum_dims += dims[n];
  const size_t sort_bytes = sort_workspace_bytes(M);
  cudaEvent_t evs[4] = {};  // encode start, sort start, sort end, encode end
  auto cleanup = [&]() {
    for (cudaEvent_t &ev : evs)
      if (ev) cudaEventDestroy(ev), ev = nullptr;
    if (own_coords) dfree(h, coords_d, (size_t)N * M * 4, s);
    if (own_vals) dfree(h, vals_d, M * 4, s);
    for (int b = 0; b < 2; ++b) {
      if (kbuf[b] && kbuf[b] != h->keys) dfree(h, kbuf[b], M * kw * 8, s);
      if (vbuf[b] && vbuf[b] != h->vals) dfree(h, vbuf[b], M * 4, s);
    }
    dfree(h, sort_work, sort_bytes, s);
    dfree(h, counts, sum_dims * 4, s);
    dfree(h, hot_scratch, 64 * 4, s);
    dfree(h, counts_ptrs_dev, kMaxModes * sizeof(void *), s);
    dfree(h, hot_list, ALTO_MAX_HOT * 8, s);
  };
  auto bail2 = [&](alto_status code) {
    cleanup();
    cudaStreamSynchronize(s);
    alto_free(h);
    return code;
  };

  if (M > 0) {
    if (!is_device_ptr(coords)) {
      if ((st = alloc_n(h, &coords_d, (size_t)N * M, s, "coords copy")) != ALTO_OK) return bail2(st);
      own_coords = true;
      if (cudaMemcpyAsync(coords_d, coords, (size_t)N * M * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return bail2(fail(ALTO_ERR_CUDA, "copying coords"));
    }
    if (!is_device_ptr(vals)) {
      if ((st = alloc_n(h, &vals_d, M, s, "vals copy")) != ALTO_OK) return bail2(st);
      own_vals = true;
      if (cudaMemcpyAsync(vals_d, vals, M * 4, cudaMemcpyHostToDevice, s) != cudaSuccess)
        return bail2(fail(ALTO_ERR_CUDA, "copying vals"));
    }
  }
  for (int b = 0; b < 2; ++b) {
    if ((st = alloc_n(h, &kbuf[b], (size_t)M * kw, s, "keys")) != ALTO_OK) return bail2(st);
    if ((st = alloc_n(h, &vbuf[b], M, s, "values")) != ALTO_OK) return bail2(st);
  }
  if (M > 0 && !(sort_work = dalloc(h, sort_bytes, s))) return bail2(fail(ALTO_ERR_OOM, "sort workspace"));

  for (cudaEvent_t &ev : evs)
    if (cudaEventCreate(&ev) != cudaSuccess) return bail2(fail(ALTO_ERR_CUDA, "encode events"));
  cudaEventRecord(evs[0], s);
  cudaError_t e = launch_linearize(h->dp, coords_d, M, h->dims_dev, kbuf[0], h->status_dev,
                                   h->num_sms, s);
  if (e != cudaSuccess) return bail2(fail(ALTO_ERR_CUDA, "linearize: %s", cudaGetErrorString(e)));
  int fb = 0;
  cudaEventRecord(evs[1], s);
  e = launch_radix_sort(kw, h->nbits, M, kbuf, vbuf, vals_d, sort_work, h->status_dev, true, &fb,
                        &h->sort_passes, h->num_sms, s);
  if (e != cudaSuccess) return bail2(fail(ALTO_ERR_CUDA, "radix sort: %s", cudaGetErrorString(e)));
  cudaEventRecord(evs[2], s);
  h->keys = kbuf[fb];
  h->vals = vbuf[fb];
  {
    // ||X||^2 over cells (duplicates summed); scratch reuses the other key buffer
    const uint64_t nc = norm_chunks(M);
    char *scr = reinterpret_cast<char *>(kbuf[fb ^ 1]);
    const size_t need = nc * (8 + 8 + 1);
    char *tmp = nullptr;
    if (need > (size_t)M * kw * 8) {
      tmp = static_cast<char *>(dalloc(h, need, s));
      if (!tmp) return bail2(fail(ALTO_ERR_OOM, "norm scratch"));
      scr = tmp;
    }
    e = launch_norm(kw, h->keys, h->vals, M, reinterpret_cast<double *>(scr),
                    reinterpret_cast<double *>(scr + nc * 8), reinterpret_cast<uint8_t *>(scr + nc * 16),
                    h->norm_sq_dev, h->num_sms, s);
    if (tmp) dfree(h, tmp, need, s);
    if (e != cudaSuccess) return bail2(fail(ALTO_ERR_CUDA, "norm: %s", cudaGetErrorString(e)));
  }

  if ((st = run_partition(h, default_parts(M, h->num_sms), s)) != ALTO_OK) return bail2(st);

  // hot rows per mode
  if (M > 0) {
    if ((st = alloc_n(h, &counts, sum_dims, s, "row counts")) != ALTO_OK) return bail2(st);
    if ((st = alloc_n(h, &hot_scratch, 64, s, "hot scratch")) != ALTO_OK) return bail2(st);
    if ((st = alloc_n(h, &counts_ptrs_dev, kMaxModes, s, "count pointers")) != ALTO_OK) return bail2(st);
    if ((st = alloc_n(h, &hot_list, ALTO_MAX_HOT, s, "hot list")) != ALTO_OK) return bail2(st);
    uint32_t *cp[kMaxModes] = {};
    uint64_t off = 0;
    for (int n = 0; n < N; ++n) {
      cp[n] = counts + off;
      off += dims[n];
    }
    if (cudaMemsetAsync(counts, 0, sum_dims * 4, s) != cudaSuccess ||
        cudaMemcpyAsync(counts_ptrs_dev, cp, sizeof(cp), cudaMemcpyHostToDevice, s) != cudaSuccess)
      return bail2(fail(ALTO_ERR_CUDA, "hot-row setup"));
    e = launch_hot_rows(h->dp, h->keys, M, h->dims, h->L, counts_ptrs_dev, cp, hot_scratch, hot_list,
                        h->hot_rows, h->nhot_dev, h->num_sms, s);
    if (e != cudaSuccess) return bail2(fail(ALTO_ERR_CUDA, "hot rows: %s", cudaGetErrorString(e)));
  }
  uint32_t status = 0;
  cudaEventRecord(evs[3], s);
  if (cudaMemcpyAsync(&status, h->status_dev, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(&h->norm_sq, h->norm_sq_dev, 8, cudaMemcpyDeviceToHost, s) != cudaSuccess ||
      cudaMemcpyAsync(h->nhot, h->nhot_dev, kMaxModes * 4, cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return bail2(fail(ALTO_ERR_CUDA, "reading back encode results"));
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return bail2(fail(ALTO_ERR_CUDA, "encode: %s", cudaGetErrorString(e)));
  if (status & kStatusCoordRange) return bail2(fail(ALTO_ERR_COORD_RANGE, "coordinate >= dims"));
  if (status & kStatusTimeout) return bail2(fail(ALTO_ERR_TIMEOUT, "radix sort: a look-back wait expired"));
  if (cudaEventElapsedTime(&h->encode_ms, evs[0], evs[3]) != cudaSuccess ||
      cudaEventElapsedTime(&h->sort_ms, evs[1], evs[2]) != cudaSuccess)
    return bail2(fail(ALTO_ERR_CUDA, "encode timing"));
  for (int n = 0; n < N; ++n) {
    h->hot_host[n].resize(h->nhot[n]);
    if (h->nhot[n] &&
        cudaMemcpy(h->hot_host[n].data(), h->hot_rows[n], h->nhot[n] * 4, cudaMemcpyDeviceToHost) != cudaSuccess)
      return bail2(fail(ALTO_ERR_CUDA, "reading hot rows"));
  }
  cleanup();
  e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    alto_free(h);
    return fail(ALTO_ERR_CUDA, "encode cleanup: %s", cudaGetErrorString(e));
  }
  *out = h;
  return ALTO_OK;
}

void alto_free(alto_handle_t h) {
  if (!h) return;
  cudaStream_t s = h->stream;
  for (auto &pe : h->prof_pending) {
    cudaEventDestroy(pe.a);
    cudaEventDestroy(pe.b);
  }
  for (auto e : h->prof_pool) cudaEventDestroy(e);
  for (int n = 0; n < kMaxModes; ++n) {
    free_pull(h, n, s);
    free_hot(h, n, s);
    free_pos_out(h, n, s);
    for (HotTable &t : h->group_hot[n])
      if (t.htab) dfree(h, t.htab, ((size_t)1 << t.hbits) * sizeof(uint64_t), s);
    if (h->hot_rows[n]) dfree(h, h->hot_rows[n], ALTO_MAX_HOT * 4, s);
  }
  dfree(h, h->partials.p, h->partials.bytes, s);
  dfree(h, h->warm.p, h->warm.bytes, s);
  dfree(h, h->keys, h->M * h->kw * 8, s);
  dfree(h, h->vals, h->M * 4, s);
  dfree(h, h->dims_dev, kMaxModes * 8, s);
  dfree(h, h->intervals, h->L * h->N * 2 * 4, s);
  dfree(h, h->max_len_dev, kMaxModes * 4, s);
  dfree(h, h->status_dev, 4 * 4, s);
  dfree(h, h->norm_sq_dev, 8, s);
  dfree(h, h->nhot_dev, kMaxModes * 4, s);
  dfree(h, h->dp_rank_dev, sizeof(DecodePlan32), s);
  dfree(h, h->lut_dev, kLutBytes, s);
  delete h;
}

alto_status alto_profile_enable(alto_handle_t h, int on) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  h->prof_on = on != 0;
  return ALTO_OK;
}

alto_status alto_profile_read(alto_handle_t h, alto_profile *out, int reset) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  for (auto &pe : h->prof_pending) {
    float ms = 0.f;
    CUDA_TRY(cudaEventSynchronize(pe.b));
    CUDA_TRY(cudaEventElapsedTime(&ms, pe.a, pe.b));
    h->prof_ms[pe.kind] += ms;
    h->prof_n[pe.kind] += 1;
    h->prof_pool.push_back(pe.a);
    h->prof_pool.push_back(pe.b);
  }
  h->prof_pending.clear();
  if (out)
    for (int k = 0; k < ALTO_PROF_KINDS; ++k) {
      out->launches[k] = h->prof_n[k];
      out->ms[k] = h->prof_ms[k];
    }
  if (reset)
    for (int k = 0; k < ALTO_PROF_KINDS; ++k) {
      h->prof_n[k] = 0;
      h->prof_ms[k] = 0.0;
    }
  return ALTO_OK;
}

uint64_t alto_kernel_launches(void) { return g_launches.load(std::memory_order_relaxed); }

alto_status alto_query(alto_handle_t h, alto_info *info) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (!info) return fail(ALTO_ERR_INVALID_ARG, "info is NULL");
  uint32_t status = 0;
  CUDA_TRY(cudaMemcpyAsync(&status, h->status_dev, 4, cudaMemcpyDeviceToHost, h->stream));
  CUDA_TRY(cudaStreamSynchronize(h->stream));
  memset(info, 0, sizeof(*info));
  info->nmodes = h->N;
  info->nbits = h->nbits;
  info->key_words = h->kw;
  info->status = (status & kStatusCoordRange)  ? ALTO_ERR_COORD_RANGE
                 : (status & kStatusNotSpd)    ? ALTO_ERR_NOT_SPD
                 : (status & kStatusTimeout)   ? ALTO_ERR_TIMEOUT
                                               : ALTO_OK;
  info->nnz = h->M;
  info->nparts = h->L;
  for (int n = 0; n < h->N; ++n) {
    info->dims[n] = h->dims[n];
    info->bits[n] = h->bits[n];
    info->mask_lo[n] = h->mask_lo[n];
    info->mask_hi[n] = h->mask_hi[n];
    info->max_interval[n] = h->max_interval[n];
    info->nhot[n] = h->nhot[n];
  }
  info->norm_sq = h->norm_sq;
  info->device_bytes = h->bytes_held;
  info->encode_ms = h->encode_ms;
  info->sort_ms = h->sort_ms;
  info->sort_passes = h->sort_passes;
  return ALTO_OK;
}

alto_status alto_set_partitions(alto_handle_t h, uint64_t nparts, void *stream) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (nparts < 1 || nparts > 0xFFFFFFFFull) return fail(ALTO_ERR_INVALID_ARG, "nparts out of range");
  h->stream = (cudaStream_t)stream;
  return run_partition(h, nparts, h->stream);
}

alto_status alto_copy_partition(alto_handle_t h, uint64_t *starts, uint32_t *intervals) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (starts)
    for (uint64_t l = 0; l <= h->L; ++l) starts[l] = (l * h->M) / h->L;
  if (intervals) {
    if ((st = ensure_intervals_host(h, h->stream)) != ALTO_OK) return st;
    memcpy(intervals, h->intervals_host.data(), h->intervals_host.size() * 4);
  }
  return ALTO_OK;
}

alto_status alto_copy_encoded(alto_handle_t h, uint64_t *keys, float *vals, void *stream) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  if (h->M == 0) return ALTO_OK;
  if (keys)
    CUDA_TRY(cudaMemcpyAsync(keys, h->keys, h->M * h->kw * 8, cudaMemcpyDeviceToDevice, s));
  if (vals) CUDA_TRY(cudaMemcpyAsync(vals, h->vals, h->M * 4, cudaMemcpyDeviceToDevice, s));
  return ALTO_OK;
}

alto_status alto_decode(alto_handle_t h, uint32_t *coords, float *vals, void *stream) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (!coords && h->M) return fail(ALTO_ERR_INVALID_ARG, "coords is NULL");
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  CUDA_TRY(launch_decode(h->dp, h->keys, h->M, coords, h->num_sms, s));
  if (vals && h->M) CUDA_TRY(cudaMemcpyAsync(vals, h->vals, h->M * 4, cudaMemcpyDeviceToDevice, s));
  return ALTO_OK;
}

alto_status alto_copy_hot_rows(alto_handle_t h, int mode, uint32_t *rows, uint32_t cap,
                               uint32_t *count) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (mode < 0 || mode >= h->N) return fail(ALTO_ERR_INVALID_ARG, "mode %d out of range", mode);
  if (count) *count = h->nhot[mode];
  if (rows) {
    const uint32_t k = std::min<uint32_t>(cap, h->nhot[mode]);
    memcpy(rows, h->hot_host[mode].data(), k * 4);
  }
  return ALTO_OK;
}

alto_status alto_set_mode_plan(alto_handle_t h, int mode, const alto_mode_plan *plan) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (mode < 0 || mode >= h->N || !plan) return fail(ALTO_ERR_INVALID_ARG, "bad mode or plan");
  if (plan->variant < ALTO_VARIANT_AUTO || plan->variant > ALTO_VARIANT_TILED_LINE)
    return fail(ALTO_ERR_INVALID_ARG, "unknown variant %d", plan->variant);
  if (plan->cols_per_lane != 0 && plan->cols_per_lane != 4 && plan->cols_per_lane != 8 &&
      plan->cols_per_lane != 16 && plan->cols_per_lane != 32 && plan->cols_per_lane != 64)
    return fail(ALTO_ERR_INVALID_ARG, "cols_per_lane must be 0, 4, 8, 16, 32 or 64");
  h->plan[mode] = *plan;
  return ALTO_OK;
}

alto_status alto_get_mode_plan(alto_handle_t h, int mode, int R, alto_mode_plan *plan) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (mode < 0 || mode >= h->N || !plan) return fail(ALTO_ERR_INVALID_ARG, "bad mode or plan");
  if (!rank_ok(R)) return fail(ALTO_ERR_UNSUPPORTED, "rank %d not in {4,8,16,32,64}", R);
  return resolve_plan(h, mode, R, plan);
}

alto_status alto_build_pos_out(alto_handle_t h, int mode, uint64_t nparts, void *stream) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (mode < -1 || mode >= h->N) return fail(ALTO_ERR_INVALID_ARG, "bad mode %d", mode);
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  for (int n = 0; n < h->N; ++n)
    if (mode < 0 || n == mode)
      if ((st = set_pos_out(h, n, nparts, s)) != ALTO_OK) return st;
  return ALTO_OK;
}

alto_status alto_copy_pos_out(alto_handle_t h, int mode, uint32_t *dst, uint64_t *nparts,
                              void *stream) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (mode < 0 || mode >= h->N || !dst) return fail(ALTO_ERR_INVALID_ARG, "bad mode or dst");
  if (!h->pos_out[mode]) return fail(ALTO_ERR_INVALID_ARG, "no stored order for mode %d", mode);
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  if (nparts) *nparts = h->pos_out_L[mode];
  if (h->M == 0) return ALTO_OK;
  CUDA_TRY(cudaMemcpyAsync(dst, h->pos_out[mode], h->M * 4, cudaMemcpyDefault, s));
  if (!is_device_ptr(dst)) CUDA_TRY(cudaStreamSynchronize(s));
  return ALTO_OK;
}

alto_status alto_free_pos_out(alto_handle_t h, int mode) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (mode < -1 || mode >= h->N) return fail(ALTO_ERR_INVALID_ARG, "bad mode %d", mode);
  for (int n = 0; n < h->N; ++n)
    if (mode < 0 || n == mode) free_pos_out(h, n, h->stream);
  return ALTO_OK;
}

alto_status alto_mttkrp(alto_handle_t h, int mode, const void *const *factors, alto_dtype fdtype,
                        int R, float *out, void *stream) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (mode < 0 || mode >= h->N) return fail(ALTO_ERR_INVALID_ARG, "mode %d out of range", mode);
  if (!rank_ok(R)) return fail(ALTO_ERR_UNSUPPORTED, "rank %d not in {4,8,16,32,64}", R);
  if (fdtype != ALTO_F32 && fdtype != ALTO_BF16) return fail(ALTO_ERR_INVALID_ARG, "bad dtype");
  if (!factors || !out) return fail(ALTO_ERR_INVALID_ARG, "factors/out NULL");
  if (!aligned16(out)) return fail(ALTO_ERR_INVALID_ARG, "out not 16-byte aligned");
  for (int m = 0; m < h->N; ++m) {
    if (m == mode) continue;
    if (!factors[m]) return fail(ALTO_ERR_INVALID_ARG, "factors[%d] is NULL", m);
    if (!aligned16(factors[m])) return fail(ALTO_ERR_INVALID_ARG, "factors[%d] not 16-byte aligned", m);
  }
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  return mttkrp_impl(h, mode, factors, fdtype == ALTO_BF16, R, out, s);
}

alto_status cpals_run(alto_handle_t h, int R, int iters, float *const *factors, double *lambda,
                      double *fits, double tol, int *iters_done, void *stream) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (!rank_ok(R)) return fail(ALTO_ERR_UNSUPPORTED, "rank %d not in {4,8,16,32,64}", R);
  if (iters < 1) return fail(ALTO_ERR_INVALID_ARG, "iters must be >= 1");
  if (h->M == 0) return fail(ALTO_ERR_INVALID_ARG, "CP-ALS needs nnz > 0");
  if (!factors || !lambda) return fail(ALTO_ERR_INVALID_ARG, "factors/lambda NULL");
  if (!(tol >= 0.0)) return fail(ALTO_ERR_INVALID_ARG, "tol must be >= 0");
  const int N = h->N;
  int ndev = 0;
  for (int m = 0; m < N; ++m) {
    if (!factors[m]) return fail(ALTO_ERR_INVALID_ARG, "factors[%d] is NULL", m);
    if (!aligned16(factors[m])) return fail(ALTO_ERR_INVALID_ARG, "factors[%d] not 16-byte aligned", m);
    ndev += is_device_ptr(factors[m]) ? 1 : 0;
  }
  if (ndev != 0 && ndev != N) return fail(ALTO_ERR_INVALID_ARG, "factors mix host and device memory");
  const bool host_factors = ndev == 0;
  const bool host_lambda = !is_device_ptr(lambda);
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;

  uint64_t maxI = 0, sumI = 0;
  for (int m = 0; m < N; ++m) {
    maxI = std::max(maxI, h->dims[m]);
    sumI += h->dims[m];
  }
  const size_t RR = (size_t)R * R;
  // one workspace: M | G[N] | s[N] | Sn | BtB | dot | W | fits | lambda | ints | device factors
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_M = take(maxI * R * 4), o_G = take(N * RR * 8), o_s = take((size_t)N * R * 8),
               o_Sn = take((size_t)R * 8), o_BtB = take(RR * 8), o_dot = take((size_t)R * 8),
               o_W = take(2 * RR * 4), o_fits = take((size_t)iters * 8), o_lam = take((size_t)R * 8),
               o_wcol = take((size_t)R * 8), o_rscale = take((size_t)R * 8),
               o_int = take(16), o_fac = take(host_factors ? sumI * R * 4 : 0);
  char *ws = static_cast<char *>(dalloc(h, off, s));
  if (!ws) return fail(ALTO_ERR_OOM, "CP-ALS workspace of %zu bytes", off);
  float *Mbuf = reinterpret_cast<float *>(ws + o_M);
  double *G = reinterpret_cast<double *>(ws + o_G);
  double *scl = reinterpret_cast<double *>(ws + o_s);
  double *Sn = reinterpret_cast<double *>(ws + o_Sn);
  double *BtB = reinterpret_cast<double *>(ws + o_BtB);
  double *dot = reinterpret_cast<double *>(ws + o_dot);
  float *W = reinterpret_cast<float *>(ws + o_W);
  double *fits_d = reinterpret_cast<double *>(ws + o_fits);
  double *lam_d = host_lambda ? reinterpret_cast<double *>(ws + o_lam) : lambda;
  int *done_at = reinterpret_cast<int *>(ws + o_int);
  int *iters_done_d = done_at + 1;
  int *renorm_d = done_at + 2;
  float *A[kMaxModes];
  {
    size_t fo = o_fac;
    for (int m = 0; m < N; ++m) {
      if (host_factors) {
        A[m] = reinterpret_cast<float *>(ws + fo);
        fo += h->dims[m] * R * 4;
      } else {
        A[m] = factors[m];
      }
    }
  }
  auto finish = [&](alto_status code) {
    dfree(h, ws, off, s);
    return code;
  };
#define CP_TRY(expr)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return finish(fail(ALTO_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_))); \
  } while (0)
  if (host_factors)
    for (int m = 0; m < N; ++m)
      CP_TRY(cudaMemcpyAsync(A[m], factors[m], h->dims[m] * R * 4, cudaMemcpyHostToDevice, s));
  {
    std::vector<double> ones((size_t)N * R, 1.0);
    CP_TRY(cudaMemcpyAsync(scl, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice, s));
  }
  CP_TRY(cudaMemsetAsync(done_at, 0x7F, sizeof(int), s));
  CP_TRY(cudaMemsetAsync(iters_done_d, 0, 2 * sizeof(int), s));  // iterations done, renorm flag
  CP_TRY(cudaMemsetAsync(G, 0, N * RR * 8, s));
  CP_TRY(cudaMemsetAsync(fits_d, 0, (size_t)iters * 8, s));
  for (int m = 0; m < N; ++m) {
    ProfScope ps(h, ALTO_PROF_GRAM, s);
    CP_TRY(launch_gram(A[m], h->dims[m], R, G + m * RR, h->num_sms, s));
  }
  const void *fptr[kMaxModes];
  for (int m = 0; m < N; ++m) fptr[m] = A[m];
  CpArgs ca{};
  ca.G = G;
  ca.s = scl;
  ca.Sn = Sn;
  ca.BtB = BtB;
  ca.dot = dot;
  ca.W = W;
  ca.wcol = reinterpret_cast<double *>(ws + o_wcol);
  ca.rscale = reinterpret_cast<double *>(ws + o_rscale);
  ca.renorm = renorm_d;
  ca.lambda = lam_d;
  ca.fits = fits_d;
  ca.norm_sq = h->norm_sq_dev;
  ca.done_at = done_at;
  ca.iters_done = iters_done_d;
  ca.status = h->status_dev;
  ca.N = N;
  ca.R = R;
  ca.tol = tol;
  for (int it = 0; it < iters; ++it) {
    for (int n = 0; n < N; ++n) {
      ca.n = n;
      ca.it = it;
      ca.last_mode = n == N - 1;
      {
        ProfScope ps(h, ALTO_PROF_SOLVE, s);
        CP_TRY(launch_prepare(ca, s));
      }
      st = mttkrp_impl(h, n, fptr, false, R, Mbuf, s);
      if (st != ALTO_OK) return finish(st);
      CP_TRY(cudaMemsetAsync(BtB, 0, RR * 8, s));
      CP_TRY(cudaMemsetAsync(dot, 0, (size_t)R * 8, s));
      {
        ProfScope ps(h, ALTO_PROF_RMUL, s);
        if (update_tc_supported(R))
          CP_TRY(launch_update_tc(Mbuf, W, A[n], h->dims[n], R, BtB, dot, done_at, it, h->status_dev,
                                  h->num_sms, s));
        else
          CP_TRY(launch_update(Mbuf, W, A[n], h->dims[n], R, BtB, dot, done_at, it, h->num_sms, s));
      }
      {
        ProfScope ps(h, ALTO_PROF_SOLVE, s);
        CP_TRY(launch_finish(ca, s));
      }
      CP_TRY(launch_renorm(A[n], ca.rscale, renorm_d, h->dims[n], R, h->num_sms, s));
    }
    if (tol > 0.0 && it + 1 < iters) {
      int d = INT_MAX;
      CP_TRY(cudaMemcpyAsync(&d, done_at, sizeof(int), cudaMemcpyDeviceToHost, s));
      CP_TRY(cudaStreamSynchronize(s));
      if (d <= it + 1) break;
    }
  }
  for (int m = 0; m < N; ++m) {
    ProfScope ps(h, ALTO_PROF_RMUL, s);
    CP_TRY(launch_scale(A[m], scl + (size_t)m * R, h->dims[m], R, h->num_sms, s));
  }
  if (host_lambda) CP_TRY(cudaMemcpyAsync(lambda, lam_d, (size_t)R * 8, cudaMemcpyDeviceToHost, s));
  if (host_factors)
    for (int m = 0; m < N; ++m)
      CP_TRY(cudaMemcpyAsync(factors[m], A[m], h->dims[m] * R * 4, cudaMemcpyDeviceToHost, s));
  int nd = 0;
  uint32_t status = 0;
  if (fits) CP_TRY(cudaMemcpyAsync(fits, fits_d, (size_t)iters * 8, cudaMemcpyDeviceToHost, s));
  CP_TRY(cudaMemcpyAsync(&nd, iters_done_d, sizeof(int), cudaMemcpyDeviceToHost, s));
  CP_TRY(cudaMemcpyAsync(&status, h->status_dev, 4, cudaMemcpyDeviceToHost, s));
  CP_TRY(cudaStreamSynchronize(s));
  if (iters_done) *iters_done = nd;
#undef CP_TRY
  if (status & kStatusNotSpd) {
    const uint32_t zero = 0;
    cudaMemcpyAsync(h->status_dev, &zero, 4, cudaMemcpyHostToDevice, s);
    cudaStreamSynchronize(s);
    return finish(fail(ALTO_ERR_NOT_SPD, "V of Alg. 1 is not positive definite"));
  }
  if (status & kStatusTimeout) return finish(fail(ALTO_ERR_TIMEOUT, "CP-ALS: a bounded wait expired"));
  return finish(ALTO_OK);
}

alto_status alto_autotune(alto_handle_t h, int R, const void *const *factors, alto_dtype fdtype,
                          float *out, int flags, void *stream, alto_tune_result *res) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (!rank_ok(R)) return fail(ALTO_ERR_UNSUPPORTED, "rank %d not in {4,8,16,32,64}", R);
  if (!factors || !out || !res) return fail(ALTO_ERR_INVALID_ARG, "factors/out/res NULL");
  if (fdtype != ALTO_F32 && fdtype != ALTO_BF16) return fail(ALTO_ERR_INVALID_ARG, "bad dtype");
  for (int m = 0; m < h->N; ++m)
    if (!factors[m] || !aligned16(factors[m]))
      return fail(ALTO_ERR_INVALID_ARG, "factors[%d] NULL or not 16-byte aligned", m);
  if (!aligned16(out)) return fail(ALTO_ERR_INVALID_ARG, "out not 16-byte aligned");
  *res = alto_tune_result{};
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  const int N = h->N;
  const bool bf16 = fdtype == ALTO_BF16;
  for (int n = 0; n < N; ++n) {
    alto_mode_plan auto_plan{ALTO_VARIANT_AUTO, 0, -1};
    h->plan[n] = auto_plan;
  }
  if (h->M == 0) {
    for (int n = 0; n < N; ++n) resolve_plan(h, n, R, &res->plan[n]);
    res->nparts = h->L;
    return ALTO_OK;
  }
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  CUDA_TRY(cudaEventCreate(&e0));
  CUDA_TRY(cudaEventCreate(&e1));
  auto done = [&](alto_status code) {
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return code;
  };
  // one warm-up run, then the faster of two timed runs
  auto time_plan = [&](int n, const alto_mode_plan &p, double *ms) -> alto_status {
    h->plan[n] = p;
    alto_status st2 = mttkrp_impl(h, n, factors, bf16, R, out, s);
    if (st2 != ALTO_OK) return st2;
    double best = 1e30;
    for (int r = 0; r < 2; ++r) {
      if (cudaEventRecord(e0, s) != cudaSuccess) return fail(ALTO_ERR_CUDA, "event");
      st2 = mttkrp_impl(h, n, factors, bf16, R, out, s);
      if (st2 != ALTO_OK) return st2;
      if (cudaEventRecord(e1, s) != cudaSuccess || cudaEventSynchronize(e1) != cudaSuccess)
        return fail(ALTO_ERR_CUDA, "event");
      float t = 0.f;
      cudaEventElapsedTime(&t, e0, e1);
      best = std::min(best, (double)t);
    }
    *ms = best;
    return ALTO_OK;
  };
  const uint64_t L0 = h->L;
  bool had_pos_out[kMaxModes] = {};
  for (int n = 0; n < N; ++n) had_pos_out[n] = h->pos_out[n] != nullptr;
  std::vector<uint64_t> Ls{L0};
  if (flags & ALTO_TUNE_SEGMENTS) {
    for (uint64_t seg : {4096ull, 16384ull, 65536ull}) {
      uint64_t L = std::max<uint64_t>(1, (h->M + seg - 1) / seg);
      if (std::find(Ls.begin(), Ls.end(), L) == Ls.end()) Ls.push_back(L);
    }
  }
  double best_total = 1e300;
  uint64_t best_L = L0;
  alto_mode_plan best_plan[kMaxModes];
  double best_ms[kMaxModes] = {};
  int timed = 0;
  for (uint64_t L : Ls) {
    if (L != h->L && (st = run_partition(h, L, s)) != ALTO_OK) return done(st);
    double total = 0.0;
    alto_mode_plan plan_L[kMaxModes];
    double ms_L[kMaxModes];
    for (int n = 0; n < N; ++n) {
      std::vector<alto_mode_plan> cands;
      const int cpls[2] = {4, 8};
      for (int c : cpls)
        if (R % c == 0 && c < R) cands.push_back(alto_mode_plan{ALTO_VARIANT_ATOMIC, c, -1});
      const size_t pull_smem = mttkrp_smem_bytes(true, R, 0, 0, h->max_interval[n]);
      if (pull_smem <= mttkrp_smem_limit())
        for (int c : cpls)
          if (R % c == 0 && c < R) cands.push_back(alto_mode_plan{ALTO_VARIANT_PULL, c, -1});
      if ((flags & ALTO_TUNE_OUTPUT) && L == L0)
        for (int c : cpls)
          if (R % c == 0 && (c == 4 || R >= 8)) cands.push_back(alto_mode_plan{ALTO_VARIANT_OUTPUT, c, 0});
      if (L == L0 && h->dims[n] <= 0x80000000ull)
        for (int v : {ALTO_VARIANT_TILED, ALTO_VARIANT_TILED_LINE})
          for (int c : cpls)
            if (R % c == 0 && (c == 4 || R >= 8)) cands.push_back(alto_mode_plan{v, c, -1});
      if (cands.empty()) cands.push_back(alto_mode_plan{ALTO_VARIANT_AUTO, 0, -1});
      double bms = 1e300;
      alto_mode_plan bp{};
      for (const alto_mode_plan &p : cands) {
        double ms = 0.0;
        if ((st = time_plan(n, p, &ms)) != ALTO_OK) return done(st);
        ++timed;
        if (ms < bms) {
          bms = ms;
          bp = p;
        }
      }
      if (L == L0) {
        double dms = 0.0;
        if ((st = time_plan(n, alto_mode_plan{ALTO_VARIANT_AUTO, 0, -1}, &dms)) != ALTO_OK)
          return done(st);
        res->default_ms[n] = dms;
      }
      plan_L[n] = bp;
      ms_L[n] = bms;
      total += bms;
    }
    if (total < best_total) {
      best_total = total;
      best_L = L;
      for (int n = 0; n < N; ++n) {
        best_plan[n] = plan_L[n];
        best_ms[n] = ms_L[n];
      }
    }
  }
  if (h->L != best_L && (st = run_partition(h, best_L, s)) != ALTO_OK) return done(st);
  for (int n = 0; n < N; ++n) {
    // an order the tuning built is kept only where OUTPUT won
    if (!had_pos_out[n] && best_plan[n].variant != ALTO_VARIANT_OUTPUT) free_pos_out(h, n, s);
    h->plan[n] = best_plan[n];
    resolve_plan(h, n, R, &res->plan[n]);
    res->ms[n] = best_ms[n];
  }
  res->nparts = best_L;
  res->candidates = timed;
  return done(ALTO_OK);
}

alto_status cpapr_run(alto_handle_t h, int R, const alto_apr_params *prm, float *const *factors,
                      double *lambda, double *objective, int *inner_steps, alto_apr_stats *stats,
                      void *stream) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (!rank_ok(R)) return fail(ALTO_ERR_UNSUPPORTED, "rank %d not in {4,8,16,32,64}", R);
  if (!prm || !factors || !lambda) return fail(ALTO_ERR_INVALID_ARG, "params/factors/lambda NULL");
  if (prm->k_max < 1 || prm->l_max < 1) return fail(ALTO_ERR_INVALID_ARG, "k_max and l_max must be >= 1");
  if (!(prm->tau > 0.0) || !(prm->kappa >= 0.0) || !(prm->kappa_tol >= 0.0) || !(prm->eps > 0.0))
    return fail(ALTO_ERR_INVALID_ARG, "tau and eps must be > 0, kappa and kappa_tol >= 0");
  if (prm->variant < 0 || prm->variant > 2) return fail(ALTO_ERR_INVALID_ARG, "variant %d", prm->variant);
  if (h->M == 0) return fail(ALTO_ERR_INVALID_ARG, "CP-APR needs nnz > 0");
  const int N = h->N;
  int ndev = 0;
  for (int m = 0; m < N; ++m) {
    if (!factors[m]) return fail(ALTO_ERR_INVALID_ARG, "factors[%d] is NULL", m);
    if (!aligned16(factors[m])) return fail(ALTO_ERR_INVALID_ARG, "factors[%d] not 16-byte aligned", m);
    ndev += is_device_ptr(factors[m]) ? 1 : 0;
  }
  if (ndev != 0 && ndev != N) return fail(ALTO_ERR_INVALID_ARG, "factors mix host and device memory");
  const bool host_factors = ndev == 0;
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  const int K = prm->k_max;
  uint64_t maxI = 0, sumI = 0;
  for (int m = 0; m < N; ++m) {
    maxI = std::max(maxI, h->dims[m]);
    sumI += h->dims[m];
  }
  // PRE (precomputed Pi) or OTF per mode, Section IV-C: precompute where the
  // mode's fiber reuse is limited and the other factors are much larger than
  // the fast memory (the L2 here); otherwise recompute on the fly.
  bool pre[kMaxModes] = {};
  bool any_pre = false;
  {
    int dev = 0, l2 = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&l2, cudaDevAttrL2CacheSize, dev);
    for (int n = 0; n < N; ++n) {
      const double reuse = (double)h->M / (double)std::max<uint64_t>(h->dims[n], 1);
      const uint64_t others = (sumI - h->dims[n]) * (uint64_t)R * 4;
      pre[n] = prm->variant == 2 || (prm->variant == 0 && reuse <= 4.0 && others > 4ull * (uint64_t)l2);
      any_pre |= pre[n];
    }
  }
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off += (bytes + 255) & ~(size_t)255;
    return o;
  };
  const size_t o_A = take(host_factors ? sumI * R * 4 : 0), o_B = take(maxI * R * 4),
               o_phi = take(sumI * R * 4), o_lam = take((size_t)R * 8), o_sum = take((size_t)R * 8),
               o_acc = take(8), o_flags = take(16), o_steps = take((size_t)K * N * 4);
  size_t o_pi = any_pre ? take(h->M * (uint64_t)R * 4) : 0;
  char *ws = static_cast<char *>(dalloc(h, off, s));
  if (!ws && any_pre) {  // Pi does not fit: recompute on the fly everywhere
    off = o_pi;
    any_pre = false;
    for (int n = 0; n < N; ++n) pre[n] = false;
    ws = static_cast<char *>(dalloc(h, off, s));
  }
  if (!ws) return fail(ALTO_ERR_OOM, "CP-APR workspace of %zu bytes", off);
  float *A[kMaxModes], *Phi[kMaxModes];
  {
    size_t fo = o_A, po = o_phi;
    for (int m = 0; m < N; ++m) {
      A[m] = host_factors ? reinterpret_cast<float *>(ws + fo) : factors[m];
      Phi[m] = reinterpret_cast<float *>(ws + po);
      fo += h->dims[m] * R * 4;
      po += h->dims[m] * R * 4;
    }
  }
  float *B = reinterpret_cast<float *>(ws + o_B);
  double *lam = reinterpret_cast<double *>(ws + o_lam);
  double *sums = reinterpret_cast<double *>(ws + o_sum);
  double *acc = reinterpret_cast<double *>(ws + o_acc);
  int *done = reinterpret_cast<int *>(ws + o_flags);
  int *stepped = done + 1;
  unsigned *kkt = reinterpret_cast<unsigned *>(done + 2);
  int *steps = reinterpret_cast<int *>(ws + o_steps);
  float *pim = any_pre ? reinterpret_cast<float *>(ws + o_pi) : nullptr;
  auto finish = [&](alto_status code) {
    dfree(h, ws, off, s);
    return code;
  };
#define AP_TRY(expr)                                                                          \
  do {                                                                                        \
    cudaError_t e_ = (expr);                                                                  \
    if (e_ != cudaSuccess) return finish(fail(ALTO_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_))); \
  } while (0)
#define AP_ST(expr)                                \
  do {                                             \
    alto_status s_ = (expr);                       \
    if (s_ != ALTO_OK) return finish(s_);          \
  } while (0)
  if (host_factors)
    for (int m = 0; m < N; ++m)
      AP_TRY(cudaMemcpyAsync(A[m], factors[m], h->dims[m] * R * 4, cudaMemcpyHostToDevice, s));
  {
    std::vector<double> ones((size_t)R, 1.0);
    AP_TRY(cudaMemcpyAsync(lam, ones.data(), (size_t)R * 8, cudaMemcpyHostToDevice, s));
  }
  AP_TRY(cudaMemsetAsync(steps, 0, (size_t)K * N * 4, s));
  AP_TRY(cudaMemsetAsync(ws + o_phi, 0, sumI * R * 4, s));
  // the initial guess as column-stochastic factors and lambda (same model)
  for (int m = 0; m < N; ++m) {
    AP_TRY(cudaMemsetAsync(sums, 0, (size_t)R * 8, s));
    AP_TRY(launch_colsum(A[m], h->dims[m], R, sums, h->num_sms, s));
    AP_TRY(launch_normalize(A[m], h->dims[m], R, sums, lam, h->num_sms, s));
  }
  FactorPtrs fp{};
  const float *Ac[kMaxModes];
  for (int m = 0; m < N; ++m) {
    fp.p[m] = A[m];
    Ac[m] = A[m];
  }
  const float eps = (float)prm->eps, tau = (float)prm->tau;
  const float kappa = (float)prm->kappa, kappa_tol = (float)prm->kappa_tol;
  int outer_done = 0;
  bool converged = false;
  std::vector<double> lam_h((size_t)R);
  for (int k = 0; k < K; ++k) {
    AP_TRY(cudaMemsetAsync(stepped, 0, sizeof(int), s));
    for (int n = 0; n < N; ++n) {
      const uint64_t I = h->dims[n];
      alto_mode_plan p;
      AP_ST(resolve_plan(h, n, R, &p));
      AP_TRY(launch_shift_scale(A[n], Phi[n], I, R, lam, k > 0 ? 1 : 0, kappa, kappa_tol, B,
                                h->num_sms, s));
      if (pre[n]) AP_TRY(launch_pi(h->dp, h->keys, h->M, n, fp, R, pim, h->num_sms, s));
      AP_TRY(cudaMemsetAsync(done, 0, sizeof(int), s));
      for (int l = 0; l < prm->l_max; ++l) {
        AP_TRY(launch_inner_begin(Phi[n], I, R, p.variant != ALTO_VARIANT_PULL, kkt, done,
                                  h->num_sms, s));
        {
          ProfScope ps(h, ALTO_PROF_MTTKRP, s);
          AP_ST(phi_impl(h, n, Ac, B, pre[n] ? pim : nullptr, eps, R, Phi[n], done, s));
        }
        AP_TRY(launch_kkt(B, Phi[n], I, R, kkt, done, h->num_sms, s));
        AP_TRY(launch_mu(B, Phi[n], I, R, kkt, tau, done, stepped, steps + k * N + n, h->num_sms, s));
      }
      // lambda = e^T B, A^(n) = B diag(lambda)^-1
      AP_TRY(cudaMemsetAsync(sums, 0, (size_t)R * 8, s));
      AP_TRY(launch_colsum(B, I, R, sums, h->num_sms, s));
      AP_TRY(cudaMemcpyAsync(A[n], B, I * R * 4, cudaMemcpyDeviceToDevice, s));
      AP_TRY(launch_normalize(A[n], I, R, sums, nullptr, h->num_sms, s));
      AP_TRY(cudaMemcpyAsync(lam, sums, (size_t)R * 8, cudaMemcpyDeviceToDevice, s));
    }
    outer_done = k + 1;
    if (objective) {
      AP_TRY(cudaMemsetAsync(acc, 0, 8, s));
      AP_TRY(launch_loglik(h->dp, h->keys, h->vals, h->M, fp, lam, R, acc, h->num_sms, s));
      double ll = 0.0;
      AP_TRY(cudaMemcpyAsync(&ll, acc, 8, cudaMemcpyDeviceToHost, s));
      AP_TRY(cudaMemcpyAsync(lam_h.data(), lam, (size_t)R * 8, cudaMemcpyDeviceToHost, s));
      AP_TRY(cudaStreamSynchronize(s));
      double total = 0.0;
      for (int r = 0; r < R; ++r) total += lam_h[r];
      objective[k] = total - ll;
    }
    int stp = 1;
    AP_TRY(cudaMemcpyAsync(&stp, stepped, sizeof(int), cudaMemcpyDeviceToHost, s));
    AP_TRY(cudaStreamSynchronize(s));
    if (stp == 0) {
      converged = true;
      break;
    }
  }
  if (host_factors)
    for (int m = 0; m < N; ++m)
      AP_TRY(cudaMemcpyAsync(factors[m], A[m], h->dims[m] * R * 4, cudaMemcpyDeviceToHost, s));
  AP_TRY(cudaMemcpyAsync(lambda, lam, (size_t)R * 8, cudaMemcpyDefault, s));
  std::vector<int> st_h((size_t)K * N);
  AP_TRY(cudaMemcpyAsync(st_h.data(), steps, (size_t)K * N * 4, cudaMemcpyDeviceToHost, s));
  AP_TRY(cudaStreamSynchronize(s));
  if (inner_steps) memcpy(inner_steps, st_h.data(), (size_t)K * N * 4);
  if (stats) {
    stats->outer_done = outer_done;
    stats->converged = converged ? 1 : 0;
    int tot = 0;
    for (int v : st_h) tot += v;
    stats->inner_steps_total = tot;
    int npre = 0;
    for (int n = 0; n < N; ++n) npre += pre[n] ? 1 : 0;
    stats->pre_modes = npre;
  }
#undef AP_TRY
#undef AP_ST
  return finish(ALTO_OK);
}

alto_status alto_phi(alto_handle_t h, int mode, const float *const *factors, const float *B, int R,
                     double eps, int pre, float *out, void *stream) {
  alto_status st = check_handle(h);
  if (st != ALTO_OK) return st;
  if (mode < 0 || mode >= h->N) return fail(ALTO_ERR_INVALID_ARG, "mode %d out of range", mode);
  if (!rank_ok(R)) return fail(ALTO_ERR_UNSUPPORTED, "rank %d not in {4,8,16,32,64}", R);
  if (!factors || !B || !out) return fail(ALTO_ERR_INVALID_ARG, "factors/B/out NULL");
  if (!(eps > 0.0)) return fail(ALTO_ERR_INVALID_ARG, "eps must be > 0");
  if (!aligned16(B) || !aligned16(out)) return fail(ALTO_ERR_INVALID_ARG, "B/out not 16-byte aligned");
  for (int m = 0; m < h->N; ++m) {
    if (m == mode) continue;
    if (!factors[m] || !aligned16(factors[m]))
      return fail(ALTO_ERR_INVALID_ARG, "factors[%d] NULL or not 16-byte aligned", m);
  }
  cudaStream_t s = (cudaStream_t)stream;
  h->stream = s;
  const uint64_t I = h->dims[mode];
  CUDA_TRY(cudaMemsetAsync(out, 0, I * R * sizeof(float), s));
  if (h->M == 0) return ALTO_OK;
  float *pim = nullptr;
  const size_t pbytes = h->M * (size_t)R * sizeof(float);
  if (pre) {
    pim = static_cast<float *>(dalloc(h, pbytes, s));
    if (!pim) return fail(ALTO_ERR_OOM, "Pi of %zu bytes", pbytes);
    FactorPtrs fp{};
    for (int m = 0; m < h->N; ++m) fp.p[m] = m == mode ? nullptr : factors[m];
    cudaError_t e = launch_pi(h->dp, h->keys, h->M, mode, fp, R, pim, h->num_sms, s);
    if (e != cudaSuccess) {
      dfree(h, pim, pbytes, s);
      return fail(ALTO_ERR_CUDA, "Pi: %s", cudaGetErrorString(e));
    }
  }
  st = phi_impl(h, mode, factors, B, pim, (float)eps, R, out, nullptr, s);
  if (pim) dfree(h, pim, pbytes, s);
  return st;
}

}  // extern "C"
