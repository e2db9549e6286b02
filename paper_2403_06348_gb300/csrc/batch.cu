// CP-ALS batch: many CP-ALS runs (Alg. 1) on different tensors advanced
// together. One step performs one mode update of every active run, as a
// CUDA graph of five launches:
//   batch_prepare_kernel  per run, fp64: V, Cholesky, W of its current mode
//                         (Alg. 1, solve); zeroes B^T B and the dot products
//   group_mttkrp_kernel   the segments of every run (group.cu)
//   batch_update_kernel   B_n = M_B W over the rows of every run, with the row
//                         tiles of all runs split evenly over the CTAs;
//                         B^T B and dot in the same pass; M_B zeroed once read
//   batch_finish_kernel   per run, fp64: lambda, s_n, G_n, the fit after the
//                         last mode, the stop test; then (iteration, mode)
//                         moves on
//   batch_renorm_kernel   rescales the factor a run just updated when its
//                         column norms left the range finish_body allows
// The runs' states (iteration, mode, stop) live on the device, so one captured
// graph replays step after step; the host uploads its tables only when runs
// join or leave, and reads the states back asynchronously.
#include <algorithm>
#include <climits>
#include <cstring>
#include <vector>

#include "cpals_body.cuh"
#include "group.cuh"
#include "handle.cuh"

namespace alto {

constexpr int kBatchMaxSlots = 4096;
constexpr uint64_t kBatchSegNnz = 4096;  // target nonzeros per segment of a run
constexpr int kReadbackRing = 4;

struct CpState {
  int it, n;        // iteration and mode of the next mode update
  int done_at;      // first iteration not run (INT_MAX while running)
  uint32_t status;  // kStatus* bits
  int iters_done;
  int stopped;      // 1 once the run has ended; every kernel skips it
  uint32_t gen;     // admission number of the run in this slot
  int renorm;       // this step's mode update asked to renormalise its factor
  int renorm_mode;  // that mode
  int pad;
};

struct CpProb {
  float *B[kMaxModes];  // factors B_m (A_m = B_m diag(s_m)) by mode
  float *M;             // MTTKRP output of the current mode, zero between steps
  double *G, *s, *Sn, *BtB, *dot;
  double *wcol, *rscale;  // column scales of W; renormalisation factors
  float *W;
  double *lambda, *fits;
  const double *norm_sq;
  uint64_t dims[kMaxModes];
  int N, R, iters, active;
  double tol;
};

__device__ __forceinline__ CpArgs make_args(const CpProb &q, CpState &st) {
  CpArgs a;
  a.G = q.G;
  a.s = q.s;
  a.Sn = q.Sn;
  a.BtB = q.BtB;
  a.dot = q.dot;
  a.W = q.W;
  a.wcol = q.wcol;
  a.rscale = q.rscale;
  a.renorm = &st.renorm;
  a.lambda = q.lambda;
  a.fits = q.fits;
  a.norm_sq = q.norm_sq;
  a.done_at = &st.done_at;
  a.iters_done = &st.iters_done;
  a.status = &st.status;
  a.N = q.N;
  a.n = st.n;
  a.R = q.R;
  a.it = st.it;
  a.last_mode = st.n == q.N - 1;
  a.tol = q.tol;
  return a;
}

__global__ void __launch_bounds__(kUpdThreads) batch_prepare_kernel(const CpProb *__restrict__ probs,
                                                                    CpState *st, int *tiles,
                                                                    const int *nslots) {
  extern __shared__ __align__(16) double sd[];
  const int P = *nslots;
  for (int p = blockIdx.x; p < P; p += gridDim.x) {
    __syncthreads();
    const CpProb &q = probs[p];
    CpState &s = st[p];
    if (threadIdx.x == 0) s.renorm = 0;  // set again by this step's finish if needed
    if (!q.active || s.stopped) {
      if (threadIdx.x == 0) tiles[p] = 0;
      continue;
    }
    const CpArgs a = make_args(q, s);
    prepare_body(a, sd);
    __syncthreads();
    if (s.done_at <= a.it) {  // V not positive definite: the run ends here
      if (threadIdx.x == 0) {
        s.stopped = 1;
        tiles[p] = 0;
      }
      continue;
    }
    const int R = q.R;
    for (int i = threadIdx.x; i < R * R; i += blockDim.x) q.BtB[i] = 0.0;
    for (int i = threadIdx.x; i < R; i += blockDim.x) q.dot[i] = 0.0;
    if (threadIdx.x == 0) {
      const uint64_t TR = 4096 / R;
      tiles[p] = (int)((q.dims[a.n] + TR - 1) / TR);
    }
  }
}

__global__ void __launch_bounds__(kUpdThreads, 2) batch_update_kernel(const CpProb *__restrict__ probs,
                                                                   const CpState *__restrict__ st,
                                                                   const int *__restrict__ tiles,
                                                                   const int *nslots) {
  extern __shared__ __align__(16) unsigned char smraw[];
  __shared__ int pre[kBatchMaxSlots + 1];
  __shared__ int wsum[kUpdThreads / 32];
  const int P = *nslots;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  // exclusive prefix of the tile counts: each thread a contiguous chunk
  const int per = (P + kUpdThreads - 1) / kUpdThreads;
  const int i0 = min(P, tid * per), i1 = min(P, i0 + per);
  int sum = 0;
  for (int i = i0; i < i1; ++i) sum += tiles[i];
  int incl = sum;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, incl, o);
    if (lane >= o) incl += y;
  }
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int woff = 0;
  for (int w = 0; w < warp; ++w) woff += wsum[w];
  int run = woff + incl - sum;
  for (int i = i0; i < i1; ++i) {
    pre[i] = run;
    run += tiles[i];
  }
  if (tid == kUpdThreads - 1) pre[P] = run;
  __syncthreads();
  const uint64_t T = (uint64_t)pre[P];
  const uint64_t b0 = T * blockIdx.x / gridDim.x, b1 = T * (blockIdx.x + 1) / gridDim.x;
  if (b0 >= b1) return;
  int lo = 0, hi = P;  // largest p with pre[p] <= b0
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if ((uint64_t)pre[mid] <= b0) lo = mid;
    else hi = mid;
  }
  int p = lo;
  uint64_t t = b0;
  while (t < b1) {
    while ((uint64_t)pre[p + 1] <= t) ++p;
    const uint64_t first = (uint64_t)pre[p];
    const uint64_t tend = min(b1, (uint64_t)pre[p + 1]);
    const CpProb &q = probs[p];
    const int n = st[p].n;
    update_body(q.M, q.W, q.B[n], q.dims[n], q.R, q.BtB, q.dot, t - first, 1, tend - first, true, smraw);
    t = tend;
  }
}

__global__ void __launch_bounds__(kUpdThreads) batch_finish_kernel(const CpProb *__restrict__ probs,
                                                                   CpState *st, const int *nslots) {
  const int P = *nslots;
  for (int p = blockIdx.x; p < P; p += gridDim.x) {
    __syncthreads();
    const CpProb &q = probs[p];
    CpState &s = st[p];
    if (!q.active || s.stopped) continue;
    const CpArgs a = make_args(q, s);
    finish_body(a);
    __syncthreads();
    if (threadIdx.x == 0) {
      s.renorm_mode = a.n;
      int n = a.n + 1, it = a.it;
      if (n == q.N) {
        n = 0;
        ++it;
      }
      s.n = n;
      s.it = it;
      if (it >= q.iters || s.done_at <= it) s.stopped = 1;
    }
  }
}

// Every CTA takes its share of the rows of each run whose finish asked for a
// renormalisation of the factor it just updated: B(:, r) *= rscale[r].
__global__ void __launch_bounds__(256) batch_renorm_kernel(const CpProb *__restrict__ probs,
                                                           const CpState *__restrict__ st, const int *nslots) {
  const int P = *nslots;
  for (int p = 0; p < P; ++p) {
    if (!st[p].renorm) continue;
    const CpProb &q = probs[p];
    const int n = st[p].renorm_mode, per_row = q.R / 4;
    const uint64_t total = q.dims[n] * (uint64_t)per_row;
    float4 *B4 = reinterpret_cast<float4 *>(q.B[n]);
    for (uint64_t t = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; t < total;
         t += (uint64_t)gridDim.x * blockDim.x) {
      const int c4 = (int)(t % per_row) * 4;
      float4 v = B4[t];
      v.x *= (float)q.rscale[c4];
      v.y *= (float)q.rscale[c4 + 1];
      v.z *= (float)q.rscale[c4 + 2];
      v.w *= (float)q.rscale[c4 + 3];
      B4[t] = v;
    }
  }
}

static size_t prepare_smem() { return (size_t)3 * ALTO_MAX_RANK * ALTO_MAX_RANK * sizeof(double); }

}  // namespace alto

using namespace alto;

namespace {

struct BatchSlot {
  bool used = false;
  alto_tensor *h = nullptr;
  int R = 0, iters = 0;
  uint32_t gen = 0;
  char *ws = nullptr;
  size_t ws_bytes = 0;
  CpProb cp{};
  GroupProb gp{};
  CpState last{};
  bool reported = false;
  cudaEvent_t result_ev = nullptr;  // recorded by alto_batch_result
};

struct Readback {
  CpState *host = nullptr;
  cudaEvent_t ev = nullptr;
  int P = 0;
};

}  // namespace

struct alto_batch {
  int max_slots = 0, num_sms = 1;
  cudaStream_t s = nullptr;
  bool own_stream = false;
  alto_allocator alloc{};
  bool user_alloc = false;
  std::vector<BatchSlot> slots;
  uint32_t next_gen = 1;
  int P = 0;  // slots in use: highest used index + 1
  // device tables
  char *tab = nullptr;
  size_t tab_bytes = 0;
  GroupProb *probs_dev = nullptr;
  CpProb *cp_dev = nullptr;
  CpState *st_dev = nullptr;
  int *tiles_dev = nullptr;
  int *nslots_dev = nullptr;
  unsigned *ctr_dev = nullptr;
  uint64_t *unit_off_dev = nullptr;
  uint32_t *unit_prob_dev = nullptr;
  size_t unit_cap = 0;
  bool dirty = true;
  cudaGraphExec_t exec = nullptr;
  // readbacks of the states, oldest first
  Readback rb[kReadbackRing];
  int rb_head = 0, rb_count = 0;
  cudaEvent_t order_ev = nullptr;
  std::vector<int> done_queue;
  uint64_t steps = 0, graph_launches = 0;
  size_t bytes_held = 0;
  // device time of the enqueued steps: event pairs around each alto_batch_step
  std::vector<std::pair<cudaEvent_t, cudaEvent_t>> timing;
  std::vector<cudaEvent_t> event_pool;
  double gpu_ms = 0.0;
};

namespace {

void *balloc(alto_batch *b, size_t bytes) {
  if (bytes == 0) bytes = 16;
  void *p = nullptr;
  if (b->user_alloc) {
    p = b->alloc.alloc(bytes, (void *)b->s, b->alloc.ctx);
  } else if (cudaMallocAsync(&p, bytes, b->s) != cudaSuccess) {
    cudaGetLastError();
    p = nullptr;
  }
  if (p) b->bytes_held += bytes;
  return p;
}

void bfree(alto_batch *b, void *p, size_t bytes) {
  if (!p) return;
  if (bytes == 0) bytes = 16;
  if (b->user_alloc)
    b->alloc.free(p, bytes, (void *)b->s, b->alloc.ctx);
  else
    cudaFreeAsync(p, b->s);
  b->bytes_held -= bytes;
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Units of the grouped MTTKRP, P and the problem tables, uploaded in stream
// order; the graph is captured again when a buffer it names is replaced.
alto_status upload_tables(alto_batch *b) {
  int P = 0;
  for (int i = 0; i < b->max_slots; ++i)
    if (b->slots[i].used) P = i + 1;
  b->P = P;
  std::vector<uint64_t> off(P + 1, 0);
  for (int i = 0; i < P; ++i) {
    const BatchSlot &sl = b->slots[i];
    off[i + 1] = off[i] + (sl.used ? sl.gp.L : 0);
  }
  const uint64_t U = off[P];
  if (U > 0xFFFFFFF0ull) return fail(ALTO_ERR_UNSUPPORTED, "%llu segments in one batch", (unsigned long long)U);
  if (U > b->unit_cap) {
    size_t cap = std::max<size_t>(U, 2 * b->unit_cap);
    bfree(b, b->unit_prob_dev, b->unit_cap * sizeof(uint32_t));
    b->unit_prob_dev = static_cast<uint32_t *>(balloc(b, cap * sizeof(uint32_t)));
    b->unit_cap = b->unit_prob_dev ? cap : 0;
    if (!b->unit_prob_dev) return fail(ALTO_ERR_OOM, "batch unit table of %zu entries", cap);
    if (b->exec) {
      cudaGraphExecDestroy(b->exec);
      b->exec = nullptr;
    }
  }
  std::vector<uint32_t> up(U);
  std::vector<GroupProb> gp(P);
  std::vector<CpProb> cp(P);
  for (int i = 0; i < P; ++i) {
    const BatchSlot &sl = b->slots[i];
    for (uint64_t u = off[i]; u < off[i + 1]; ++u) up[u] = (uint32_t)i;
    if (sl.used) {
      gp[i] = sl.gp;
      cp[i] = sl.cp;
    } else {
      gp[i] = GroupProb{};
      cp[i] = CpProb{};
    }
  }
  cudaStream_t s = b->s;
  if (P) {
    CUDA_TRY(cudaMemcpyAsync(b->probs_dev, gp.data(), P * sizeof(GroupProb), cudaMemcpyHostToDevice, s));
    CUDA_TRY(cudaMemcpyAsync(b->cp_dev, cp.data(), P * sizeof(CpProb), cudaMemcpyHostToDevice, s));
  }
  CUDA_TRY(cudaMemcpyAsync(b->unit_off_dev, off.data(), (P + 1) * sizeof(uint64_t), cudaMemcpyHostToDevice, s));
  if (U) CUDA_TRY(cudaMemcpyAsync(b->unit_prob_dev, up.data(), U * sizeof(uint32_t), cudaMemcpyHostToDevice, s));
  CUDA_TRY(cudaMemcpyAsync(b->nslots_dev, &P, sizeof(int), cudaMemcpyHostToDevice, s));
  b->dirty = false;
  return ALTO_OK;
}

int update_grid(alto_batch *b) {
  int per_sm = 1;
  cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, batch_update_kernel, kUpdThreads,
                                                update_smem(ALTO_MAX_RANK));
  return b->num_sms * std::max(per_sm, 1);
}

alto_status configure_kernels() {
  static bool done = false;
  if (done) return ALTO_OK;
  CUDA_TRY(cudaFuncSetAttribute(batch_prepare_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)prepare_smem()));
  CUDA_TRY(cudaFuncSetAttribute(batch_update_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                (int)update_smem(ALTO_MAX_RANK)));
  done = true;
  return ALTO_OK;
}

// One step: the five launches, recorded once into a graph.
cudaError_t enqueue_step(alto_batch *b) {
  cudaStream_t s = b->s;
  const int gp = std::min(b->max_slots, 2 * b->num_sms);
  batch_prepare_kernel<<<gp, kUpdThreads, prepare_smem(), s>>>(b->cp_dev, b->st_dev, b->tiles_dev,
                                                               b->nslots_dev);
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  e = launch_group_mttkrp(b->probs_dev, b->unit_off_dev, b->unit_prob_dev, b->nslots_dev, b->ctr_dev,
                          false, b->num_sms, s);
  if (e != cudaSuccess) return e;
  batch_update_kernel<<<update_grid(b), kUpdThreads, update_smem(ALTO_MAX_RANK), s>>>(
      b->cp_dev, b->st_dev, b->tiles_dev, b->nslots_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_finish_kernel<<<gp, kUpdThreads, 0, s>>>(b->cp_dev, b->st_dev, b->nslots_dev);
  e = cudaGetLastError();
  if (e != cudaSuccess) return e;
  batch_renorm_kernel<<<b->num_sms, 256, 0, s>>>(b->cp_dev, b->st_dev, b->nslots_dev);
  return cudaGetLastError();
}

alto_status capture_graph(alto_batch *b) {
  alto_status st = configure_kernels();
  if (st != ALTO_OK) return st;
  CUDA_TRY(configure_group_mttkrp());
  cudaGraph_t g = nullptr;
  CUDA_TRY(cudaStreamBeginCapture(b->s, cudaStreamCaptureModeThreadLocal));
  cudaError_t e = enqueue_step(b);
  cudaError_t e2 = cudaStreamEndCapture(b->s, &g);
  note_launches(-1);  // counted per graph launch instead
  if (e != cudaSuccess || e2 != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return fail(ALTO_ERR_CUDA, "batch step capture: %s",
                cudaGetErrorString(e != cudaSuccess ? e : e2));
  }
  e = cudaGraphInstantiate(&b->exec, g, 0);
  cudaGraphDestroy(g);
  if (e != cudaSuccess) {
    b->exec = nullptr;
    return fail(ALTO_ERR_CUDA, "batch graph instantiate: %s", cudaGetErrorString(e));
  }
  return ALTO_OK;
}

cudaEvent_t timing_event(alto_batch *b) {
  if (!b->event_pool.empty()) {
    cudaEvent_t e = b->event_pool.back();
    b->event_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) {
    cudaGetLastError();
    return nullptr;
  }
  return e;
}

// Adds the device time of every finished step bracket to gpu_ms.
void collect_timing(alto_batch *b) {
  size_t keep = 0;
  for (size_t i = 0; i < b->timing.size(); ++i) {
    auto &pr = b->timing[i];
    if (cudaEventQuery(pr.second) == cudaSuccess) {
      float ms = 0.f;
      if (cudaEventElapsedTime(&ms, pr.first, pr.second) == cudaSuccess) b->gpu_ms += ms;
      cudaGetLastError();
      b->event_pool.push_back(pr.first);
      b->event_pool.push_back(pr.second);
    } else {
      cudaGetLastError();
      b->timing[keep++] = pr;
    }
  }
  b->timing.resize(keep);
}

void process_readback(alto_batch *b, const Readback &r) {
  for (int i = 0; i < r.P && i < b->max_slots; ++i) {
    BatchSlot &sl = b->slots[i];
    if (!sl.used || r.host[i].gen != sl.gen) continue;
    sl.last = r.host[i];
    if (sl.last.stopped && !sl.reported) {
      sl.reported = true;
      b->done_queue.push_back(i);
    }
  }
}

// Consumes completed readbacks (oldest first); with wait, waits for the
// oldest one if none has completed.
alto_status drain_readbacks(alto_batch *b, bool wait) {
  while (b->rb_count > 0) {
    Readback &r = b->rb[b->rb_head];
    cudaError_t q = cudaEventQuery(r.ev);
    if (q == cudaErrorNotReady) {
      if (!wait) break;
      CUDA_TRY(cudaEventSynchronize(r.ev));
    } else if (q != cudaSuccess) {
      return fail(ALTO_ERR_CUDA, "batch readback: %s", cudaGetErrorString(q));
    }
    process_readback(b, r);
    b->rb_head = (b->rb_head + 1) % kReadbackRing;
    --b->rb_count;
    wait = false;
  }
  return ALTO_OK;
}

}  // namespace

extern "C" {

alto_status alto_batch_create(int max_slots, const alto_allocator *alloc, void *stream,
                              alto_batch_t *out) {
  if (!out) return fail(ALTO_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (max_slots < 1 || max_slots > kBatchMaxSlots)
    return fail(ALTO_ERR_INVALID_ARG, "max_slots %d not in 1..%d", max_slots, kBatchMaxSlots);
  if (alloc && (!alloc->alloc || !alloc->free)) return fail(ALTO_ERR_INVALID_ARG, "allocator incomplete");
  alto_batch *b = new alto_batch();
  b->max_slots = max_slots;
  b->slots.resize(max_slots);
  if (alloc) {
    b->alloc = *alloc;
    b->user_alloc = true;
  }
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    if (stream) {
      b->s = (cudaStream_t)stream;
    } else {
      e = cudaStreamCreateWithFlags(&b->s, cudaStreamNonBlocking);
      b->own_stream = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess) e = cudaEventCreateWithFlags(&b->order_ev, cudaEventDisableTiming);
  for (int i = 0; i < kReadbackRing && e == cudaSuccess; ++i) {
    e = cudaEventCreateWithFlags(&b->rb[i].ev, cudaEventDisableTiming);
    if (e == cudaSuccess)
      e = cudaMallocHost(reinterpret_cast<void **>(&b->rb[i].host), max_slots * sizeof(CpState));
  }
  if (e != cudaSuccess) {
    alto_batch_free(b);
    return fail(ALTO_ERR_CUDA, "batch set-up: %s", cudaGetErrorString(e));
  }
  // tables: probs | cp | states | tiles | unit_off | nslots + counters
  size_t o = 0;
  const size_t o_probs = o;
  o = align256(o + max_slots * sizeof(GroupProb));
  const size_t o_cp = o;
  o = align256(o + max_slots * sizeof(CpProb));
  const size_t o_st = o;
  o = align256(o + max_slots * sizeof(CpState));
  const size_t o_tiles = o;
  o = align256(o + max_slots * sizeof(int));
  const size_t o_off = o;
  o = align256(o + (max_slots + 1) * sizeof(uint64_t));
  const size_t o_int = o;
  o = align256(o + 16);
  b->tab_bytes = o;
  b->tab = static_cast<char *>(balloc(b, o));
  if (!b->tab) {
    alto_batch_free(b);
    return fail(ALTO_ERR_OOM, "batch tables of %zu bytes", o);
  }
  b->probs_dev = reinterpret_cast<GroupProb *>(b->tab + o_probs);
  b->cp_dev = reinterpret_cast<CpProb *>(b->tab + o_cp);
  b->st_dev = reinterpret_cast<CpState *>(b->tab + o_st);
  b->tiles_dev = reinterpret_cast<int *>(b->tab + o_tiles);
  b->unit_off_dev = reinterpret_cast<uint64_t *>(b->tab + o_off);
  b->nslots_dev = reinterpret_cast<int *>(b->tab + o_int);
  b->ctr_dev = reinterpret_cast<unsigned *>(b->tab + o_int + 4);
  e = cudaMemsetAsync(b->tab, 0, o, b->s);
  if (e == cudaSuccess) {
    b->unit_cap = 1024;
    b->unit_prob_dev = static_cast<uint32_t *>(balloc(b, b->unit_cap * sizeof(uint32_t)));
    if (!b->unit_prob_dev) {
      alto_batch_free(b);
      return fail(ALTO_ERR_OOM, "batch unit table");
    }
  } else {
    alto_batch_free(b);
    return fail(ALTO_ERR_CUDA, "batch set-up: %s", cudaGetErrorString(e));
  }
  *out = b;
  return ALTO_OK;
}

void alto_batch_free(alto_batch_t b) {
  if (!b) return;
  if (b->s) cudaStreamSynchronize(b->s);
  for (int i = 0; i < b->max_slots; ++i) {
    if (b->slots[i].used) bfree(b, b->slots[i].ws, b->slots[i].ws_bytes);
    if (b->slots[i].result_ev) cudaEventDestroy(b->slots[i].result_ev);
  }
  bfree(b, b->unit_prob_dev, b->unit_cap * sizeof(uint32_t));
  bfree(b, b->tab, b->tab_bytes);
  if (b->exec) cudaGraphExecDestroy(b->exec);
  for (auto &pr : b->timing) {
    cudaEventDestroy(pr.first);
    cudaEventDestroy(pr.second);
  }
  for (cudaEvent_t e : b->event_pool) cudaEventDestroy(e);
  for (int i = 0; i < kReadbackRing; ++i) {
    if (b->rb[i].ev) cudaEventDestroy(b->rb[i].ev);
    if (b->rb[i].host) cudaFreeHost(b->rb[i].host);
  }
  if (b->order_ev) cudaEventDestroy(b->order_ev);
  if (b->s) cudaStreamSynchronize(b->s);
  if (b->own_stream) cudaStreamDestroy(b->s);
  delete b;
}

alto_status alto_batch_prepare(alto_handle_t h, int R) {
  if (!h) return fail(ALTO_ERR_INVALID_ARG, "null handle");
  if (check_device(h) != ALTO_OK) return ALTO_ERR_INVALID_ARG;  // message set by check_device
  if (!(R == 4 || R == 8 || R == 16 || R == 32 || R == 64))
    return fail(ALTO_ERR_UNSUPPORTED, "rank %d not in {4,8,16,32,64}", R);
  cudaStream_t hs = h->stream;
  const uint64_t want_L = std::max<uint64_t>(1, (h->M + kBatchSegNnz - 1) / kBatchSegNnz);
  if (h->M > 0 && h->L > 2 * want_L) {
    alto_status st = repartition(h, want_L, hs);
    if (st != ALTO_OK) return st;
  }
  alto_status st = ensure_rank_runs(h, hs);
  if (st != ALTO_OK) return st;
  GroupProb gp{};
  return fill_group_prob(h, R, &gp, hs);
}

alto_status alto_batch_add(alto_batch_t b, alto_handle_t h, int R, int iters, double tol,
                           const float *const *factors, int *slot_out) {
  if (!b || !h) return fail(ALTO_ERR_INVALID_ARG, "null batch or handle");
  if (check_device(h) != ALTO_OK) return ALTO_ERR_INVALID_ARG;  // message set by check_device
  if (!(R == 4 || R == 8 || R == 16 || R == 32 || R == 64))
    return fail(ALTO_ERR_UNSUPPORTED, "rank %d not in {4,8,16,32,64}", R);
  if (iters < 1) return fail(ALTO_ERR_INVALID_ARG, "iters must be >= 1");
  if (!(tol >= 0.0)) return fail(ALTO_ERR_INVALID_ARG, "tol must be >= 0");
  if (h->M == 0) return fail(ALTO_ERR_INVALID_ARG, "CP-ALS needs nnz > 0");
  if (!factors) return fail(ALTO_ERR_INVALID_ARG, "factors NULL");
  const int N = h->N;
  for (int m = 0; m < N; ++m) {
    if (!factors[m]) return fail(ALTO_ERR_INVALID_ARG, "factors[%d] is NULL", m);
    if (((uintptr_t)factors[m] & 15u) != 0)
      return fail(ALTO_ERR_INVALID_ARG, "factors[%d] not 16-byte aligned", m);
  }
  int slot = -1;
  for (int i = 0; i < b->max_slots; ++i)
    if (!b->slots[i].used) {
      slot = i;
      break;
    }
  if (slot < 0) return fail(ALTO_ERR_UNSUPPORTED, "all %d batch slots are in use", b->max_slots);
  // on the handle's stream (free after alto_batch_prepare): segments of
  // about kBatchSegNnz nonzeros, rank runs, grouped hot-row tables
  cudaStream_t hs = h->stream;
  alto_status st = alto_batch_prepare(h, R);
  if (st != ALTO_OK) return st;
  GroupProb gp{};
  st = fill_group_prob(h, R, &gp, hs);
  if (st != ALTO_OK) return st;
  CUDA_TRY(cudaEventRecord(b->order_ev, hs));
  CUDA_TRY(cudaStreamWaitEvent(b->s, b->order_ev, 0));

  uint64_t maxI = 0, sumI = 0;
  for (int m = 0; m < N; ++m) {
    maxI = std::max(maxI, h->dims[m]);
    sumI += h->dims[m];
  }
  const size_t RR = (size_t)R * R;
  size_t off = 0;
  auto take = [&](size_t bytes) {
    const size_t o = off;
    off = align256(off + bytes);
    return o;
  };
  const size_t o_M = take(maxI * R * 4), o_G = take(N * RR * 8), o_s = take((size_t)N * R * 8),
               o_Sn = take((size_t)R * 8), o_BtB = take(RR * 8), o_dot = take((size_t)R * 8),
               o_W = take(2 * RR * 4), o_fits = take((size_t)iters * 8), o_lam = take((size_t)R * 8),
               o_wcol = take((size_t)R * 8), o_rscale = take((size_t)R * 8);
  size_t o_B[kMaxModes];
  for (int m = 0; m < N; ++m) o_B[m] = take(h->dims[m] * R * 4);
  char *ws = static_cast<char *>(balloc(b, off));
  if (!ws) return fail(ALTO_ERR_OOM, "CP-ALS run of %zu bytes", off);
  BatchSlot &sl = b->slots[slot];
  sl = BatchSlot();
  sl.ws = ws;
  sl.ws_bytes = off;
  sl.h = h;
  sl.R = R;
  sl.iters = iters;
  CpProb &cp = sl.cp;
  cp.M = reinterpret_cast<float *>(ws + o_M);
  cp.G = reinterpret_cast<double *>(ws + o_G);
  cp.s = reinterpret_cast<double *>(ws + o_s);
  cp.Sn = reinterpret_cast<double *>(ws + o_Sn);
  cp.BtB = reinterpret_cast<double *>(ws + o_BtB);
  cp.dot = reinterpret_cast<double *>(ws + o_dot);
  cp.W = reinterpret_cast<float *>(ws + o_W);
  cp.wcol = reinterpret_cast<double *>(ws + o_wcol);
  cp.rscale = reinterpret_cast<double *>(ws + o_rscale);
  cp.fits = reinterpret_cast<double *>(ws + o_fits);
  cp.lambda = reinterpret_cast<double *>(ws + o_lam);
  cp.norm_sq = h->norm_sq_dev;
  cp.N = N;
  cp.R = R;
  cp.iters = iters;
  cp.tol = tol;
  cp.active = 1;
  for (int m = 0; m < N; ++m) {
    cp.B[m] = reinterpret_cast<float *>(ws + o_B[m]);
    cp.dims[m] = h->dims[m];
  }
  cudaStream_t s = b->s;
  auto undo = [&](alto_status code) {
    bfree(b, ws, off);
    sl = BatchSlot();
    return code;
  };
#define BT_TRY(expr)                                                                             \
  do {                                                                                           \
    cudaError_t e_ = (expr);                                                                     \
    if (e_ != cudaSuccess) return undo(fail(ALTO_ERR_CUDA, "%s: %s", #expr, cudaGetErrorString(e_))); \
  } while (0)
  for (int m = 0; m < N; ++m)
    BT_TRY(cudaMemcpyAsync(cp.B[m], factors[m], h->dims[m] * R * 4, cudaMemcpyDefault, s));
  BT_TRY(cudaMemsetAsync(cp.M, 0, maxI * R * 4, s));
  BT_TRY(cudaMemsetAsync(cp.G, 0, N * RR * 8, s));
  BT_TRY(cudaMemsetAsync(cp.fits, 0, (size_t)iters * 8, s));
  BT_TRY(cudaMemsetAsync(cp.lambda, 0, (size_t)R * 8, s));
  {
    std::vector<double> ones((size_t)N * R, 1.0);
    BT_TRY(cudaMemcpyAsync(cp.s, ones.data(), ones.size() * 8, cudaMemcpyHostToDevice, s));
  }
  for (int m = 0; m < N; ++m) BT_TRY(launch_gram(cp.B[m], h->dims[m], R, cp.G + m * RR, b->num_sms, s));
  sl.gen = b->next_gen++;
  if (b->next_gen == 0) b->next_gen = 1;
  CpState init{};
  init.it = 0;
  init.n = 0;
  init.done_at = INT_MAX;
  init.gen = sl.gen;
  BT_TRY(cudaMemcpyAsync(b->st_dev + slot, &init, sizeof(init), cudaMemcpyHostToDevice, s));
  sl.gp = gp;
  sl.gp.out = cp.M;
  sl.gp.cur_mode = &b->st_dev[slot].n;
  sl.gp.done = &b->st_dev[slot].stopped;
  for (int q = 0; q < N; ++q) sl.gp.fac[q] = cp.B[h->mode_of[q]];
#undef BT_TRY
  sl.used = true;
  sl.last = init;
  b->dirty = true;
  if (slot_out) *slot_out = slot;
  return ALTO_OK;
}

alto_status alto_batch_step(alto_batch_t b, int nsteps) {
  if (!b) return fail(ALTO_ERR_INVALID_ARG, "null batch");
  if (nsteps < 0) return fail(ALTO_ERR_INVALID_ARG, "nsteps %d", nsteps);
  if (b->dirty) {
    alto_status st = upload_tables(b);
    if (st != ALTO_OK) return st;
  }
  if (b->P == 0 || nsteps == 0) return ALTO_OK;
  if (!b->exec) {
    alto_status st = capture_graph(b);
    if (st != ALTO_OK) return st;
  }
  cudaEvent_t t0 = timing_event(b), t1 = timing_event(b);
  if (t0 && t1) CUDA_TRY(cudaEventRecord(t0, b->s));
  for (int i = 0; i < nsteps; ++i) {
    CUDA_TRY(cudaGraphLaunch(b->exec, b->s));
    note_launches(5);
  }
  if (t0 && t1) {
    CUDA_TRY(cudaEventRecord(t1, b->s));
    b->timing.emplace_back(t0, t1);
  }
  collect_timing(b);
  b->steps += nsteps;
  b->graph_launches += nsteps;
  if (b->rb_count == kReadbackRing) {
    alto_status st = drain_readbacks(b, true);
    if (st != ALTO_OK) return st;
  }
  const int idx = (b->rb_head + b->rb_count) % kReadbackRing;
  Readback &r = b->rb[idx];
  r.P = b->P;
  CUDA_TRY(cudaMemcpyAsync(r.host, b->st_dev, b->P * sizeof(CpState), cudaMemcpyDeviceToHost, b->s));
  CUDA_TRY(cudaEventRecord(r.ev, b->s));
  ++b->rb_count;
  return ALTO_OK;
}

alto_status alto_batch_poll(alto_batch_t b, int wait, int *slots, int cap, int *ndone) {
  if (!b || !ndone) return fail(ALTO_ERR_INVALID_ARG, "null batch or ndone");
  if (cap > 0 && !slots) return fail(ALTO_ERR_INVALID_ARG, "slots NULL");
  *ndone = 0;
  alto_status st = drain_readbacks(b, false);
  if (st != ALTO_OK) return st;
  if (wait && b->done_queue.empty()) {
    st = drain_readbacks(b, true);
    if (st != ALTO_OK) return st;
  }
  int n = 0;
  while (n < cap && !b->done_queue.empty()) {
    slots[n++] = b->done_queue.front();
    b->done_queue.erase(b->done_queue.begin());
  }
  *ndone = n;
  return ALTO_OK;
}

alto_status alto_batch_result(alto_batch_t b, int slot, float *const *factors, double *lambda,
                              double *fits, int *iters_done, int *run_status) {
  if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].used)
    return fail(ALTO_ERR_INVALID_ARG, "slot %d is not in use", slot);
  BatchSlot &sl = b->slots[slot];
  if (!sl.reported) return fail(ALTO_ERR_INVALID_ARG, "slot %d has not been reported finished", slot);
  const CpProb &cp = sl.cp;
  const int N = cp.N, R = cp.R;
  cudaStream_t s = b->s;
  for (int m = 0; m < N; ++m) {
    CUDA_TRY(launch_scale(cp.B[m], cp.s + (size_t)m * R, cp.dims[m], R, b->num_sms, s));
    if (factors && factors[m])
      CUDA_TRY(cudaMemcpyAsync(factors[m], cp.B[m], cp.dims[m] * R * 4, cudaMemcpyDefault, s));
  }
  if (lambda) CUDA_TRY(cudaMemcpyAsync(lambda, cp.lambda, (size_t)R * 8, cudaMemcpyDefault, s));
  if (fits) CUDA_TRY(cudaMemcpyAsync(fits, cp.fits, (size_t)cp.iters * 8, cudaMemcpyDefault, s));
  if (!sl.result_ev) CUDA_TRY(cudaEventCreateWithFlags(&sl.result_ev, cudaEventDisableTiming));
  CUDA_TRY(cudaEventRecord(sl.result_ev, s));
  if (iters_done) *iters_done = sl.last.iters_done;
  if (run_status) *run_status = (sl.last.status & kStatusNotSpd) ? ALTO_ERR_NOT_SPD : ALTO_OK;
  return ALTO_OK;
}

alto_status alto_batch_copy_out(alto_batch_t b, int slot, float *const *factors, double *lambda,
                                double *fits, void *stream) {
  if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].used)
    return fail(ALTO_ERR_INVALID_ARG, "slot %d is not in use", slot);
  const BatchSlot &sl = b->slots[slot];
  if (!sl.result_ev) return fail(ALTO_ERR_INVALID_ARG, "slot %d: call alto_batch_result first", slot);
  const CpProb &cp = sl.cp;
  cudaStream_t s = (cudaStream_t)stream;
  CUDA_TRY(cudaStreamWaitEvent(s, sl.result_ev, 0));
  for (int m = 0; m < cp.N; ++m)
    if (factors && factors[m])
      CUDA_TRY(cudaMemcpyAsync(factors[m], cp.B[m], cp.dims[m] * cp.R * 4, cudaMemcpyDefault, s));
  if (lambda) CUDA_TRY(cudaMemcpyAsync(lambda, cp.lambda, (size_t)cp.R * 8, cudaMemcpyDefault, s));
  if (fits) CUDA_TRY(cudaMemcpyAsync(fits, cp.fits, (size_t)cp.iters * 8, cudaMemcpyDefault, s));
  CUDA_TRY(cudaStreamSynchronize(s));
  return ALTO_OK;
}

alto_status alto_batch_remove(alto_batch_t b, int slot) {
  if (!b || slot < 0 || slot >= b->max_slots || !b->slots[slot].used)
    return fail(ALTO_ERR_INVALID_ARG, "slot %d is not in use", slot);
  BatchSlot &sl = b->slots[slot];
  bfree(b, sl.ws, sl.ws_bytes);
  if (sl.result_ev) cudaEventDestroy(sl.result_ev);
  // the handle may be freed on its own stream once the batch is done with it
  CUDA_TRY(cudaEventRecord(b->order_ev, b->s));
  CUDA_TRY(cudaStreamWaitEvent(sl.h->stream, b->order_ev, 0));
  for (size_t i = 0; i < b->done_queue.size(); ++i)
    if (b->done_queue[i] == slot) {
      b->done_queue.erase(b->done_queue.begin() + i);
      break;
    }
  sl = BatchSlot();
  b->dirty = true;
  return ALTO_OK;
}

alto_status alto_batch_query(alto_batch_t b, alto_batch_info *info) {
  if (!b || !info) return fail(ALTO_ERR_INVALID_ARG, "null batch or info");
  int active = 0;
  for (int i = 0; i < b->max_slots; ++i) active += b->slots[i].used ? 1 : 0;
  info->active = active;
  info->slots_span = b->P;
  info->steps = b->steps;
  info->graph_launches = b->graph_launches;
  info->bytes_held = b->bytes_held;
  info->pending_readbacks = b->rb_count;
  collect_timing(b);
  info->gpu_ms = b->gpu_ms;
  return ALTO_OK;
}

alto_status alto_batch_sync(alto_batch_t b) {
  if (!b) return fail(ALTO_ERR_INVALID_ARG, "null batch");
  CUDA_TRY(cudaStreamSynchronize(b->s));
  return ALTO_OK;
}

alto_status alto_cpals_footprint(int nmodes, const uint64_t *dims, uint64_t nnz, int R, int iters,
                                 uint64_t *resident, uint64_t *peak) {
  if (nmodes < 1 || nmodes > kMaxModes || !dims) return fail(ALTO_ERR_INVALID_ARG, "bad modes/dims");
  int bits = 0;
  uint64_t maxI = 0, sumI = 0;
  for (int m = 0; m < nmodes; ++m) {
    uint64_t I = dims[m];
    int b = 0;
    while (b < 64 && (I - 1) >> b) ++b;
    bits += I <= 1 ? 0 : b;
    maxI = std::max(maxI, I);
    sumI += I;
  }
  const uint64_t kw = bits <= 64 ? 1 : 2;
  const uint64_t L = std::max<uint64_t>(1, (nnz + kBatchSegNnz - 1) / kBatchSegNnz);
  const uint64_t tensor = nnz * (8 * kw + 4) + L * nmodes * 8 + 4096;
  const uint64_t RR = (uint64_t)R * R;
  const uint64_t run = maxI * R * 4 + nmodes * RR * 8 + nmodes * (uint64_t)R * 8 + RR * 24 +
                       (uint64_t)R * 40 + (uint64_t)iters * 8 + sumI * R * 4 + 4096;
  // encode: the coordinates, the positions and values twice (sort buffers)
  const uint64_t encode = nnz * (4ull * nmodes + 2 * (8 * kw + 4));
  if (resident) *resident = tensor + run;
  if (peak) *peak = tensor + run + encode;
  return ALTO_OK;
}

}  // extern "C"
