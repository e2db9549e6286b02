/*
 * alto.h -- C ABI of the GB300 (sm_103a) ALTO sparse-tensor library.
 *
 * The library encodes a sparse tensor given in coordinate form into the ALTO
 * format (Adaptive Linearized Tensor Order, arXiv 2403.06348, Section III-A),
 * computes the mode-agnostic MTTKRP over that single encoded copy (Alg. 1
 * MTTKRP line, Alg. 3 and Alg. 4) and runs CP-ALS on top of it (Alg. 1).
 * Every step runs in the library's own CUDA kernels; there is no CPU
 * fallback.
 *
 * Conventions shared by every call:
 *  - Coordinates are 0-based. Mode n has length dims[n] (1 <= dims[n] < 2^32).
 *  - Dense matrices are row-major: A^(n) is dims[n] x R, element (i, r) at
 *    A[i * R + r]. They must be 16-byte aligned.
 *  - "stream" is a cudaStream_t passed as void* (NULL = legacy default
 *    stream). Calls enqueue work on that stream and return without waiting,
 *    unless the call says it synchronises.
 *  - A handle is used by one stream at a time; calls on one handle from two
 *    streams at once race.
 *  - Return values are alto_status codes. On failure alto_last_error() gives
 *    a message for the calling thread. Argument errors are detected before
 *    any work is enqueued and leave outputs untouched.
 *  - nnz < 2^32 in this version.
 */
#ifndef ALTO_H_
#define ALTO_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define ALTO_MAX_MODES 8
#define ALTO_MAX_RANK 64
#define ALTO_MAX_HOT 4096

typedef enum alto_status {
  ALTO_OK = 0,
  ALTO_ERR_INVALID_ARG = -1,   /* bad pointer, size, mode, rank or alignment   */
  ALTO_ERR_OOM = -2,           /* the allocator returned NULL                   */
  ALTO_ERR_CUDA = -3,          /* a CUDA runtime call failed                    */
  ALTO_ERR_UNSUPPORTED = -4,   /* > 128 index bits, rank not in {4,8,16,32,64}  */
  ALTO_ERR_COORD_RANGE = -5,   /* a coordinate >= dims[n] (detected on device)  */
  ALTO_ERR_NOT_SPD = -6,       /* CP-ALS: V of Alg. 1 not usable (non-finite)   */
  ALTO_ERR_TIMEOUT = -7        /* a bounded device wait gave up                 */
} alto_status;

/* Element type of factor matrices handed to alto_mttkrp. */
typedef enum alto_dtype { ALTO_F32 = 0, ALTO_BF16 = 1 } alto_dtype;

/* Output strategy of one mode's MTTKRP (Section IV-B, Alg. 4).
 *  ATOMIC: nonzeros are streamed in ALTO order; runs of equal output row are
 *          summed in registers; the most reused rows of the mode ("hot rows",
 *          picked at encode time) are staged in shared memory per line
 *          segment and flushed once per segment; all other rows are added to
 *          the output with vector atomics (the atomic updates of the
 *          output-oriented branch, without its stored order).
 *  PULL:   each line segment accumulates into a shared-memory Temp over its
 *          mode interval [T^s, T^e], writes it out as a partial, and a second
 *          kernel pulls, for each output row, the partials of the segments
 *          whose interval contains it (the recursive branch).
 *  OUTPUT: the output-oriented traversal through the stored order pos_out
 *          of the mode (alto_build_pos_out; built on first use with the
 *          current segment count when missing): nonzeros of one output row
 *          are consecutive in it, each group of threads walks a contiguous
 *          piece of it, sums each run of equal row in registers across the
 *          whole piece and adds the run to the output with one vector atomic.
 *          The stored order holds, per nonzero, its ordered position (4
 *          bytes), its line position (8 * key_words bytes) and its value (4
 *          bytes): pos_out and val_out of Alg. 4, read as one stream.
 *  TILED:  the output-oriented traversal done inside each tile of 1024
 *          consecutive nonzeros of the one ALTO copy, with no stored order:
 *          the tile arrives in shared memory by a bulk asynchronous copy, is
 *          decoded once, and its nonzeros are grouped by output row (one bin
 *          per hot row of the mode, one for the rest) before groups of
 *          threads walk contiguous pieces of it, summing runs of equal row in
 *          registers. Runs of the most frequent rows go to shared memory
 *          (flushed once per CTA), of the next most frequent rows to a few
 *          fp32 replicas that a second small kernel adds into the output,
 *          of all other rows straight to the output with vector atomics.
 *          Needs dims[mode] <= 2^31 (else ATOMIC). hot_rows resolves to the
 *          rows staged in shared memory.
 *  TILED_LINE: TILED without the grouping (each tile in line order).
 *  AUTO:   OUTPUT (measured faster on GB300 than PULL and ATOMIC for modes
 *          of any reuse); if the order cannot be allocated (or nnz is too
 *          large for it), the paper's rule: PULL when the fiber reuse
 *          nnz/dims[mode] exceeds 4 (the paper's cost of buffered
 *          accumulation) and the largest interval fits in shared memory,
 *          else ATOMIC. */
typedef enum alto_variant {
  ALTO_VARIANT_AUTO = 0,
  ALTO_VARIANT_ATOMIC = 1,
  ALTO_VARIANT_PULL = 2,
  ALTO_VARIANT_OUTPUT = 3,
  ALTO_VARIANT_TILED = 4,
  ALTO_VARIANT_TILED_LINE = 5
} alto_variant;

/* Optional device-memory allocator. alloc returns a device pointer aligned to
 * 256 bytes, or NULL on failure (the library then returns ALTO_ERR_OOM); free
 * releases it. Both are called from the host thread making the library call,
 * with that call's stream. NULL allocator = cudaMallocAsync/cudaFreeAsync. */
typedef struct alto_allocator {
  void *(*alloc)(size_t bytes, void *stream, void *ctx);
  void (*free)(void *ptr, size_t bytes, void *stream, void *ctx);
  void *ctx;
} alto_allocator;

typedef struct alto_tensor *alto_handle_t;

/* Read-only description of an encoded tensor (alto_query). */
typedef struct alto_info {
  int nmodes;
  int nbits;                          /* sum of bits over modes (Eq. 1 per nonzero) */
  int key_words;                      /* 64-bit words per position: 1 or 2          */
  int status;                         /* latched device-side status (alto_status)   */
  uint64_t nnz;
  uint64_t nparts;                    /* number of line segments L                  */
  uint64_t dims[ALTO_MAX_MODES];
  int bits[ALTO_MAX_MODES];           /* bits of each mode: bit_width(dims[n]-1)    */
  uint64_t mask_lo[ALTO_MAX_MODES];   /* ALTO bit mask of each mode, low 64 bits    */
  uint64_t mask_hi[ALTO_MAX_MODES];   /* high 64 bits                               */
  uint32_t max_interval[ALTO_MAX_MODES]; /* max over segments of T^e - T^s + 1       */
  uint32_t nhot[ALTO_MAX_MODES];      /* hot rows found per mode                    */
  double norm_sq;                     /* ||X||^2 = sum of squared values            */
  size_t device_bytes;                /* device memory held by the handle           */
  float encode_ms;                    /* device time of alto_encode's kernels, from
                                         the first (linearize) to the last (hot
                                         rows), CUDA events on the encode stream   */
  float sort_ms;                      /* of which the radix sort (digit counts and
                                         every pass; the one host read of the
                                         digit counts included)                    */
  int sort_passes;                    /* 8-bit radix passes launched: passes whose
                                         digit is the same for every nonzero are
                                         left out                                  */
} alto_info;

/* Per-mode MTTKRP plan (what the autotuner sets). */
typedef struct alto_mode_plan {
  int variant;        /* alto_variant                                             */
  int cols_per_lane;  /* factor columns per thread: 4, 8 or 16 (< R) split one
                         nonzero over R/cols_per_lane threads ("threads per
                         nonzero"); cols_per_lane == R (R >= 8) gives each
                         nonzero one thread, which walks its rows in 8-column
                         chunks; 0 = library default. OUTPUT, TILED and
                         TILED_LINE use 4 or 8 (larger requests and 0 take 8,
                         or 4 when R = 4)                                        */
  int hot_rows;       /* ATOMIC: staged hot rows, -1 = as many as fit; OUTPUT:
                         resolved to the hot rows its long runs may stage
                         (set by the library, up to 256); TILED, TILED_LINE:
                         at most this many hot rows staged in shared memory
                         (-1 = as many as fit two CTAs per SM), resolved to
                         the number staged                                      */
} alto_mode_plan;

/* ---------------------------------------------------------------------------
 * alto_encode -- Section III-A (linearization and ordering) and Section IV-A
 * (nnz-balanced line segments and their mode intervals).
 *
 *  coords  [nmodes][nnz] uint32, structure of arrays, 0-based; host or device
 *          memory (host memory is copied in; pin it for an asynchronous copy).
 *  vals    [nnz] float; host or device memory.
 *  dims    host array [nmodes] of mode lengths.
 *  nmodes  1..ALTO_MAX_MODES.
 *  nnz     number of nonzeros (0 allowed; duplicates are kept, and summed by
 *          every operation, as in COO).
 *  alloc   allocator for everything the handle owns, or NULL.
 *  stream  stream for all device work.
 *  out     receives the new handle.
 *
 * Steps: bits per mode = bit_width(dims[n]-1); bit groups from the least
 * significant bit, each group holding the modes that still have bits, shortest
 * mode at the lowest bit; position p = bit-level gather of the coordinates
 * (PDEP); stable sort of (p, value) by p (ties keep input order); L balanced
 * segments [floor(l*nnz/L), floor((l+1)*nnz/L)) with per-mode [min, max]
 * intervals; ||X||^2; the hot rows of every mode (sampled row counts).
 * The call synchronises the stream before returning (it reads back the
 * device status word and a few sizes). Coordinates >= dims[n] make it return
 * ALTO_ERR_COORD_RANGE and free everything. Errors: INVALID_ARG, OOM, CUDA,
 * UNSUPPORTED (more than 128 index bits), COORD_RANGE.
 * ------------------------------------------------------------------------- */
alto_status alto_encode(const uint32_t *coords, const float *vals, const uint64_t *dims,
                        int nmodes, uint64_t nnz, const alto_allocator *alloc, void *stream,
                        alto_handle_t *out);

/* Release the handle and everything it owns (freed on the stream of the last
 * call made with it; pending work on that stream is ordered before). NULL ok. */
void alto_free(alto_handle_t h);

/* Fill *info. Synchronises the handle's last stream to read the latched
 * device status. */
alto_status alto_query(alto_handle_t h, alto_info *info);

/* Re-partition into nparts line segments (Section IV-A) and recompute the
 * mode intervals. Synchronises. Drops cached pull plans. */
alto_status alto_set_partitions(alto_handle_t h, uint64_t nparts, void *stream);

/* Copy the partition to host memory: starts [nparts+1] (nonzero offsets) and
 * intervals [nparts][nmodes][2] (closed [T^s, T^e]; an empty segment has
 * (2^32-1, 0)). Either pointer may be NULL. Synchronises. */
alto_status alto_copy_partition(alto_handle_t h, uint64_t *starts, uint32_t *intervals);

/* Copy the ordered encoded tensor to device memory: keys [nnz][key_words]
 * uint64 (low word first) and vals [nnz] float. Either may be NULL. */
alto_status alto_copy_encoded(alto_handle_t h, uint64_t *keys, float *vals, void *stream);

/* De-linearize every position (EXTRACT with the mode masks, Alg. 3) into
 * coords [nmodes][nnz] (device) and copy the values in ALTO order to vals
 * (device, may be NULL). */
alto_status alto_decode(alto_handle_t h, uint32_t *coords, float *vals, void *stream);

/* Copy mode `mode`'s hot rows (most frequent first) to host memory; at most
 * cap rows; *count receives how many exist. Synchronises. */
alto_status alto_copy_hot_rows(alto_handle_t h, int mode, uint32_t *rows, uint32_t cap,
                               uint32_t *count);

/* Set / read the MTTKRP plan of one mode. alto_get_mode_plan resolves AUTO
 * for rank R into the concrete choice the next alto_mttkrp would make. */
alto_status alto_set_mode_plan(alto_handle_t h, int mode, const alto_mode_plan *plan);
alto_status alto_get_mode_plan(alto_handle_t h, int mode, int R, alto_mode_plan *plan);

/* ---------------------------------------------------------------------------
 * alto_build_pos_out -- the stored order of Alg. 4's output-oriented
 * traversal (pos_out) for one mode, or every mode with mode = -1: inside
 * every line segment l of nparts, [floor(l*nnz/nparts),
 * floor((l+1)*nnz/nparts)) as in Section IV-A, the segment's ordered
 * positions by increasing coordinate of the mode; equal coordinates keep line
 * order. Kept in the handle per mode, replacing an earlier order of that
 * mode, until alto_free_pos_out or alto_free: the nnz uint32 ordered
 * positions and, in that order, the line positions and values (Alg. 4's
 * pos_out and val_out), 4 + 8 * key_words + 4 bytes per nonzero per mode on
 * top of the one ALTO copy. The ALTO_VARIANT_OUTPUT plan streams it.
 *
 *  nparts  segments of the order; 0 = the handle's current segment count,
 *          raised where needed so that no segment holds more than 8192
 *          nonzeros; values above nnz count as nnz. Later
 *          alto_set_partitions calls do not change a stored order.
 * Built on the device: one CTA sorts each segment in shared memory when every
 * segment holds at most 8192 nonzeros (the default count does), else one
 * stable radix sort of (segment, coordinate) keys runs over the whole line
 * (scratch of about 28 bytes per nonzero). Asynchronous.
 * Errors: INVALID_ARG (mode), UNSUPPORTED (nnz > 2^32 - 4097), OOM, CUDA.
 * ------------------------------------------------------------------------- */
alto_status alto_build_pos_out(alto_handle_t h, int mode, uint64_t nparts, void *stream);

/* Copy the stored order of `mode` (nnz uint32 ordered positions) to dst, host
 * or device memory; synchronises the stream when dst is host memory.
 * *nparts (may be NULL) receives its segment count. Errors: INVALID_ARG
 * (mode, NULL dst, no order stored for the mode), CUDA. */
alto_status alto_copy_pos_out(alto_handle_t h, int mode, uint32_t *dst, uint64_t *nparts,
                              void *stream);

/* Release the stored order of `mode` (-1: every mode). Modes whose plan is
 * OUTPUT build it again on their next MTTKRP. */
alto_status alto_free_pos_out(alto_handle_t h, int mode);

/* ---------------------------------------------------------------------------
 * alto_mttkrp -- M = X_(mode) (A^(1) (.) ... A^(mode-1) (.) A^(mode+1) ... (.) A^(N))
 * (Alg. 1 MTTKRP line), computed nonzero by nonzero over the ALTO copy
 * (Alg. 3) with the conflict resolution of Alg. 4 chosen by the mode plan.
 *
 *  mode     0..nmodes-1, the output mode.
 *  factors  HOST array [nmodes] of DEVICE pointers to row-major dims[m] x R
 *           matrices of type fdtype; factors[mode] is not read (may be NULL).
 *  fdtype   ALTO_F32 or ALTO_BF16 (bf16 factors, fp32 arithmetic).
 *  R        rank: 4, 8, 16, 32 or 64.
 *  out      DEVICE dims[mode] x R float, overwritten (rows without nonzeros
 *           become 0).
 * The first call for a PULL mode builds that mode's row-to-segment lists on
 * the host (one synchronisation); later calls are asynchronous. fp32 results
 * differ from the exact sum by rounding only; the summation order of the
 * ATOMIC variant is not fixed, so bits may vary from run to run.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 * ------------------------------------------------------------------------- */
alto_status alto_mttkrp(alto_handle_t h, int mode, const void *const *factors,
                        alto_dtype fdtype, int R, float *out, void *stream);

/* ---------------------------------------------------------------------------
 * alto_mttkrp_noalloc -- the same MTTKRP as alto_mttkrp with the PULL
 * variant, for callers that cannot have the library allocate device memory
 * while they run (for example a service that reserved its whole device budget
 * at start-up, or a framework whose own allocator must see every device
 * allocation). The paper has no counterpart: it is an interface addition.
 *
 * It calls no cudaMalloc, cudaFree or other allocating routine. The segments'
 * partials live in one fixed device array of 8 Mi floats (32 MiB) inside the
 * library, which every GPU that loads the library holds until the process
 * exits. The first call on a device looks up that array's device address;
 * make that first call before any stream capture.
 *
 * Arguments are those of alto_mttkrp. Requirements, each checked:
 *  - the mode's row-to-segment lists must already exist: one earlier
 *    alto_mttkrp call on this mode with the PULL variant (alto_set_mode_plan)
 *    builds them, and that call may allocate;
 *  - the largest mode interval times R must fit shared memory;
 *  - sum over segments of (interval length) * R <= 8 Mi floats.
 * Errors: INVALID_ARG (bad arguments, lists not built), UNSUPPORTED (rank,
 * shared memory, or the fixed scratch too small, with the sizes in the
 * message), CUDA.
 * All calls share the one scratch array: calls that overlap on the GPU (two
 * streams, or two host threads) race and give wrong results. Nothing in the
 * array needs clearing between calls: every segment rewrites its whole part
 * before the reduction reads it.
 * ------------------------------------------------------------------------- */
alto_status alto_mttkrp_noalloc(alto_handle_t h, int mode, const void *const *factors,
                                alto_dtype fdtype, int R, float *out, void *stream);

/* ---------------------------------------------------------------------------
 * alto_mttkrp_grouped -- n MTTKRPs (Alg. 3 and 4) over n encoded tensors in
 * one persistent kernel launch. The tensors may differ in nnz, number of
 * modes, key width and rank.
 *
 * The units of work are the line segments of every handle (Section IV-A);
 * the GPU's CTAs take them in turn, so many small tensors share the device
 * without a launch each. Per segment, the output rows of the segment's mode
 * interval are staged in shared memory when they fit (interval x R x 4 bytes
 * <= about 220 KB) and flushed once with vector atomics; otherwise equal-row
 * runs go straight to the output with vector atomics. The hot-row tables and
 * the PULL partials of alto_mttkrp are not used. Work is balanced by segment,
 * so tensors whose segments hold very different numbers of nonzeros share it
 * less evenly (alto_set_partitions sets a handle's segment count).
 *
 *  n        number of problems (0 does nothing).
 *  hs       host [n] handles (a handle may appear more than once).
 *  modes    host [n] output mode of each problem.
 *  factors  host [n] arrays, each a host array [nmodes of that handle] of
 *           device pointers to I_m x R row-major matrices, 16-byte aligned;
 *           the output mode's entry is ignored.
 *  Rs       host [n] ranks (4, 8, 16, 32 or 64).
 *  fdtype   ALTO_F32 or ALTO_BF16, for every problem.
 *  outs     host [n] device pointers to I_mode x R floats, 16-byte aligned,
 *           overwritten (zeroed with cudaMemsetAsync, then accumulated).
 *  stream   all handles must be ready on this stream.
 * Allocates and frees (stream-ordered) one small table per call. Results are
 * rounded like alto_mttkrp's: fp32 sums in an order that varies run to run.
 * Errors: INVALID_ARG (which problem and why in alto_last_error), UNSUPPORTED,
 * CUDA.
 * ------------------------------------------------------------------------- */
alto_status alto_mttkrp_grouped(int n, const alto_handle_t *hs, const int *modes,
                                const void *const *const *factors, const int *Rs, alto_dtype fdtype,
                                float *const *outs, void *stream);

/* ---------------------------------------------------------------------------
 * alto_autotune -- picks, by measurement, each mode's MTTKRP plan (ATOMIC or
 * PULL, 4 or 8 columns per lane; hot rows as the library sizes them) and,
 * with ALTO_TUNE_SEGMENTS, the segment count among the current one and
 * segments of 4 Ki, 16 Ki and 64 Ki nonzeros. The paper chooses between its
 * two traversals by the per-mode fiber-reuse rule (Section IV-B); here that
 * rule is only the default, and the choice is the fastest measured plan.
 * Every candidate runs once untimed and twice timed (CUDA events, the faster
 * counts); the sum over modes decides the segment count. The winners stay set
 * on the handle (alto_get_mode_plan reads them).
 *
 *  factors  as in alto_mttkrp (all modes set; device, 16-byte aligned).
 *  out      device scratch of max_n I_n x R floats (overwritten).
 *  flags    0, or ALTO_TUNE_SEGMENTS and / or ALTO_TUNE_OUTPUT. With
 *           ALTO_TUNE_OUTPUT the OUTPUT plan (4 and 8 columns per lane) joins
 *           the candidates at the original segment count: each mode's order
 *           is built with that count; a mode keeps its order only if OUTPUT
 *           wins there.
 *  res      the chosen plan (resolved), its time and the default plan's time
 *           per mode, the segment count, and the number of timed candidates.
 * Synchronises the stream. Errors: those of alto_mttkrp.
 * ------------------------------------------------------------------------- */
#define ALTO_TUNE_SEGMENTS 1
#define ALTO_TUNE_OUTPUT 2

typedef struct alto_tune_result {
  alto_mode_plan plan[ALTO_MAX_MODES];
  double ms[ALTO_MAX_MODES];          /* chosen plan, ms per MTTKRP          */
  double default_ms[ALTO_MAX_MODES];  /* library default at the original L  */
  uint64_t nparts;
  int candidates;
} alto_tune_result;

alto_status alto_autotune(alto_handle_t h, int R, const void *const *factors, alto_dtype fdtype,
                          float *out, int flags, void *stream, alto_tune_result *res);

/* ---------------------------------------------------------------------------
 * cpals_run -- CP-ALS, Alg. 1: for each iteration and each mode n:
 * V = Hadamard product of the Grams G_m = A^(m)T A^(m), m != n (fp64);
 * M = MTTKRP (alto_mttkrp); A^(n) = M V^-1 through a Cholesky factorisation of
 * V (fp64); lambda = column 2-norms of A^(n); A^(n) /= lambda; after the last
 * mode the fit 1 - ||X - X_hat|| / ||X|| (fp64).
 *
 *  R        rank (4, 8, 16, 32 or 64).
 *  iters    maximum number of iterations (>= 1).
 *  factors  HOST array [nmodes] of pointers to dims[m] x R float matrices:
 *           the initial guess on entry, the normalised result on return.
 *           All device pointers or all host pointers (host ones are copied
 *           in and out; pin them for asynchronous copies).
 *  lambda   [R] double (host or device), the column norms of the last update.
 *  fits     host [iters] double, the fit after each iteration, or NULL.
 *  tol      0 runs exactly iters iterations; > 0 stops after the first
 *           iteration whose fit changed by less than tol.
 *  iters_done  host int, iterations run, or NULL.
 * Synchronises when fits, iters_done or host factors are given, and always
 * reads back the device status at the end. Requires nnz > 0.
 * A V that is not positive definite (the Cholesky factorisation meets a pivot
 * <= 0) is inverted through its eigendecomposition instead (fp64 Jacobi,
 * eigenvalues below 1e-15 of the largest dropped): the pseudo-inverse Alg. 1
 * names. Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA, NOT_SPD (V has a
 * non-finite entry: the factors are left at the last completed update).
 * ------------------------------------------------------------------------- */
alto_status cpals_run(alto_handle_t h, int R, int iters, float *const *factors, double *lambda,
                      double *fits, double tol, int *iters_done, void *stream);

/* ---------------------------------------------------------------------------
 * cpapr_run -- CP-APR with multiplicative updates (Alg. 2) for count data:
 * for each outer iteration and each mode n: S shifts inadmissible zeros
 * (kappa where A(i,r) < kappa_tol and the previous Phi(i,r) > 1), B = (A^(n)
 * + S) diag(lambda); then at most l_max times: Phi = (X_(n) ./ max(B Pi,
 * eps)) Pi^T (the Phi kernel of Alg. 5 on the ALTO tensor, with the MTTKRP's
 * per-mode conflict resolution), stop when max |min(B, 1 - Phi)| < tau, else
 * B = B .* Phi; then lambda = e^T B and A^(n) = B diag(lambda)^-1. The whole
 * run stops after an outer iteration in which no mode took a step.
 * Pi's rows are recomputed from the factors for every nonzero (OTF) or, for a
 * mode whose fiber reuse is at most 4 while the other factors are more than
 * four times the L2 size, precomputed once per mode and outer iteration
 * (PRE, nnz x R floats; OTF everywhere if that does not fit), Section IV-C.
 *
 *  factors  HOST array [nmodes] of pointers to dims[m] x R floats, all device
 *           or all host: the initial guess (positive) on entry, the
 *           column-stochastic result on return.
 *  lambda   [R] double, host or device: the column weights of the result.
 *  objective  host [k_max] double or NULL: after every outer iteration,
 *           sum(lambda) - sum over nonzeros of x log M(x) (the negative
 *           Poisson log-likelihood up to a constant). Costs one sync each.
 *  inner_steps  host [k_max * nmodes] int or NULL: update steps per outer
 *           iteration and mode.
 *  stats    outer iterations run, whether it converged, total update steps,
 *           modes run with PRE.
 * Factors and Phi are fp32, lambda and the objective fp64. Synchronises once
 * per outer iteration. Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA.
 * ------------------------------------------------------------------------- */
/* alto_phi -- the Phi kernel of Alg. 5 alone (a test aid and a building
 * block): out = (X_(mode) ./ max(B Pi, eps)) Pi^T, i.e. every nonzero adds
 * v / max(B(i_mode,:) . krp, eps) * krp to row i_mode, krp the Hadamard
 * product of the other factors' rows. factors: host array [nmodes] of device
 * I_m x R fp32 matrices (factors[mode] ignored); B: device I_mode x R fp32;
 * out: device I_mode x R fp32, overwritten. pre != 0 precomputes Pi (nnz x R
 * floats, allocated and freed on the stream) instead of gathering on the fly.
 * Errors: INVALID_ARG, UNSUPPORTED, OOM, CUDA. */
alto_status alto_phi(alto_handle_t h, int mode, const float *const *factors, const float *B, int R,
                     double eps, int pre, float *out, void *stream);

typedef struct alto_apr_params {
  int k_max;          /* outer iterations (>= 1)                               */
  int l_max;          /* inner iterations per mode (>= 1); the paper uses 10   */
  double tau;         /* KKT tolerance (> 0)                                    */
  double kappa;       /* inadmissible-zero shift (>= 0)                        */
  double kappa_tol;   /* entries below this may be shifted (>= 0)              */
  double eps;         /* smallest divisor (> 0)                                 */
  int variant;        /* 0 = PRE/OTF per mode by the rule above, 1 = OTF, 2 = PRE */
} alto_apr_params;

typedef struct alto_apr_stats {
  int outer_done;
  int converged;
  int inner_steps_total;
  int pre_modes;
} alto_apr_stats;

alto_status cpapr_run(alto_handle_t h, int R, const alto_apr_params *params, float *const *factors,
                      double *lambda, double *objective, int *inner_steps, alto_apr_stats *stats,
                      void *stream);

/* ---------------------------------------------------------------------------
 * CP-ALS batch -- many CP-ALS runs (Alg. 1) on different tensors advanced
 * together on one stream: a step performs one mode update of every active run
 * (prepare, grouped MTTKRP, update, finish: the same arithmetic as cpals_run),
 * replayed from one CUDA graph. Runs join and leave between steps; each run
 * keeps its own iteration, mode and stop rule on the device. No counterpart in
 * the paper: it batches the paper's per-tensor loop.
 *
 * alto_batch_create  max_slots 1..4096 concurrent runs; alloc as in
 *                    alto_encode (NULL = cudaMallocAsync); stream NULL = a new
 *                    non-blocking stream owned by the batch. Every call below
 *                    is ordered on that stream.
 * alto_batch_add     admits a run of CP-ALS on handle h: rank R, at most iters
 *                    iterations, tol as in cpals_run, initial factors
 *                    (host array [nmodes] of host or device pointers, copied
 *                    in). The batch orders itself after the handle's stream,
 *                    may re-partition the handle into segments of about 4096
 *                    nonzeros, and reads h until alto_batch_remove. *slot
 *                    receives the run's slot. Errors: INVALID_ARG,
 *                    UNSUPPORTED (rank, no free slot), OOM, CUDA.
 * alto_batch_prepare  the per-handle set-up alto_batch_add needs (segments of
 *                    about 4096 nonzeros, rank-ordered decode runs, hot-row
 *                    tables for rank R), done on the handle's stream and
 *                    waited for; call it where waiting is cheap (e.g. right
 *                    after alto_encode) and alto_batch_add then finds it done.
 * alto_batch_step    enqueues nsteps steps and one asynchronous read-back of
 *                    the runs' states; returns without waiting (it waits only
 *                    when four read-backs are still outstanding).
 * alto_batch_poll    writes up to cap slots whose runs have ended, as seen by
 *                    the completed read-backs, to slots[]; wait != 0 waits for
 *                    the oldest outstanding read-back when none has ended yet.
 * alto_batch_result  for a slot reported by alto_batch_poll: enqueues the
 *                    normalised factors (A_m = B_m diag(s_m)) into factors[m]
 *                    (host or device; NULL entries skipped), lambda [R] and
 *                    fits [iters] (host or device, nullable) on the batch
 *                    stream; host destinations are valid after
 *                    alto_batch_sync (pin them for asynchronous copies).
 *                    *iters_done and *run_status (ALTO_OK or
 *                    ALTO_ERR_NOT_SPD) come from the read-back.
 * alto_batch_copy_out  after alto_batch_result (which may pass NULL
 *                    destinations and then only normalises in place): copies
 *                    the slot's factors, lambda and fits into host or device
 *                    buffers on `stream` and waits for them. It reads only
 *                    that slot, so another host thread may call it while the
 *                    batch goes on, until the slot is removed.
 * alto_batch_remove  frees the slot (stream-ordered) and orders the handle's
 *                    stream after the batch, so the handle may then be freed.
 * alto_batch_sync    waits for everything enqueued on the batch stream.
 * alto_cpals_footprint  device bytes one run holds while resident (encoded
 *                    tensor + CP-ALS state) and at its peak (plus the encode's
 *                    transient buffers), for admission by memory budget.
 * ------------------------------------------------------------------------- */
typedef struct alto_batch *alto_batch_t;

typedef struct alto_batch_info {
  int active;                /* runs admitted and not removed                   */
  int slots_span;            /* highest slot in use + 1 (as of the last step)   */
  uint64_t steps;            /* steps enqueued                                   */
  uint64_t graph_launches;   /* graph launches enqueued                          */
  uint64_t bytes_held;       /* device bytes held by the batch                   */
  int pending_readbacks;
  double gpu_ms;             /* device time of the finished steps (CUDA events)  */
} alto_batch_info;

alto_status alto_batch_create(int max_slots, const alto_allocator *alloc, void *stream,
                              alto_batch_t *out);
void alto_batch_free(alto_batch_t b);
alto_status alto_batch_add(alto_batch_t b, alto_handle_t h, int R, int iters, double tol,
                           const float *const *factors, int *slot);
alto_status alto_batch_prepare(alto_handle_t h, int R);
alto_status alto_batch_step(alto_batch_t b, int nsteps);
alto_status alto_batch_poll(alto_batch_t b, int wait, int *slots, int cap, int *ndone);
alto_status alto_batch_result(alto_batch_t b, int slot, float *const *factors, double *lambda,
                              double *fits, int *iters_done, int *run_status);
alto_status alto_batch_copy_out(alto_batch_t b, int slot, float *const *factors, double *lambda,
                                double *fits, void *stream);
alto_status alto_batch_remove(alto_batch_t b, int slot);
alto_status alto_batch_query(alto_batch_t b, alto_batch_info *info);
alto_status alto_batch_sync(alto_batch_t b);
alto_status alto_cpals_footprint(int nmodes, const uint64_t *dims, uint64_t nnz, int R, int iters,
                                 uint64_t *resident, uint64_t *peak);

/* ---------------------------------------------------------------------------
 * alto_fill_uniform -- n floats of dst (device) set to seeded uniform values
 * in [0, 1): element i is (SplitMix64(seed * 2^32 + i) >> 40) * 2^-24, where
 * SplitMix64(x) = mix(x + 0x9E3779B97F4A7C15) with the published finaliser
 * (Steele, Lea and Flood, 2014). For initial CP-ALS factors drawn on the GPU;
 * the paper leaves the initialisation to the caller. seed < 2^32, n <= 2^32.
 * Asynchronous on stream. Errors: INVALID_ARG, CUDA.
 * ------------------------------------------------------------------------- */
alto_status alto_fill_uniform(float *dst, uint64_t n, uint64_t seed, void *stream);

/* ---------------------------------------------------------------------------
 * Instrumentation (no counterpart in the paper; used to report kernel time
 * against the memory roofline).
 *
 * alto_profile_enable: when on, every kernel the handle launches from
 * alto_mttkrp and cpals_run is bracketed by a pair of CUDA events recorded on
 * the launching stream; alto_profile_read synchronises those events and
 * returns, per kernel kind, the number of launches and their summed device
 * time in milliseconds (reset != 0 clears the totals afterwards).
 * alto_kernel_launches: process-wide count of kernels this library has
 * launched (all handles, all kinds; memsets and copies are not counted).
 * ------------------------------------------------------------------------- */
typedef enum alto_prof_kind {
  ALTO_PROF_MTTKRP = 0,       /* the segment kernel of Alg. 3/4             */
  ALTO_PROF_PULL_REDUCE = 1,  /* the pull-based reduction of Alg. 4         */
  ALTO_PROF_ZERO = 2,         /* zeroing of the output (ATOMIC, OUTPUT)      */
  ALTO_PROF_GRAM = 3,         /* A^T A of the initial factors                */
  ALTO_PROF_SOLVE = 4,        /* fp64 Hadamard / Cholesky / lambda / fit    */
  ALTO_PROF_RMUL = 5,         /* A^(n) = M V^-1 with its Gram (one pass) and
                                 the final column normalisation             */
  ALTO_PROF_POS_OUT = 6,      /* building a stored output-oriented order     */
  ALTO_PROF_KINDS = 7
} alto_prof_kind;

typedef struct alto_profile {
  uint64_t launches[ALTO_PROF_KINDS];
  double ms[ALTO_PROF_KINDS];
} alto_profile;

alto_status alto_profile_enable(alto_handle_t h, int on);
alto_status alto_profile_read(alto_handle_t h, alto_profile *out, int reset);
uint64_t alto_kernel_launches(void);

/* Message describing the calling thread's last error ("" if none). */
const char *alto_last_error(void);

/* Library version, major*10000 + minor*100 + patch. */
int alto_version(void);

#ifdef __cplusplus
}
#endif

#endif /* ALTO_H_ */
