/*
 * Plain C fp64 oracle for COO MTTKRP and ALTO linearization.
 * Test infrastructure only: used by tests/, __graft_entry__.smoke() and the
 * CPU-baseline legs of bench.py; never by the product library.
 *
 * MTTKRP follows its definition (Alg. 1, MTTKRP line; Alg. 3):
 *   M(i,:) = sum over nonzeros x with i_mode(x) = i of
 *            v_x * prod_{m != mode} A_m(i_m(x), :)
 * evaluated in double precision, every row summed in input order. The
 * multi-threaded form first lists, for every output row, the nonzeros that
 * land in it (in input order) and then sums each row on one thread, so its
 * result is bit-identical to the single-threaded scatter.
 *
 * Linearization follows Section III-A: bit g of mode n is copied to key
 * position pos[n][g] (a bit-level gather); positions come from the caller's
 * bit plan.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

static double term(int nmodes, uint64_t x, uint64_t M, const uint32_t *coords,
                   const float *vals, const float *const *factors, int R, int mode,
                   int r) {
    double t = (double)vals[x];
    for (int m = 0; m < nmodes; ++m) {
        if (m == mode) continue;
        uint64_t row = coords[(uint64_t)m * M + x];
        t *= (double)factors[m][row * (uint64_t)R + (uint64_t)r];
    }
    return t;
}

/* out: I_mode x R doubles, overwritten. Returns 0, or -1 on allocation failure. */
int oracle_mttkrp_f64(int nmodes, uint64_t M, const uint32_t *coords, const float *vals,
                      const uint64_t *dims, const float *const *factors, int R, int mode,
                      double *out, int nthreads) {
    uint64_t I = dims[mode];
    memset(out, 0, sizeof(double) * I * (uint64_t)R);
    if (nthreads <= 1) {
        for (uint64_t x = 0; x < M; ++x) {
            uint64_t i = coords[(uint64_t)mode * M + x];
            for (int r = 0; r < R; ++r)
                out[i * R + r] += term(nmodes, x, M, coords, vals, factors, R, mode, r);
        }
        return 0;
    }
    /* list the nonzeros of every output row, keeping input order */
    uint64_t *ptr = (uint64_t *)calloc(I + 1, sizeof(uint64_t));
    uint64_t *lst = (uint64_t *)malloc(sizeof(uint64_t) * (M ? M : 1));
    if (!ptr || !lst) { free(ptr); free(lst); return -1; }
    const uint32_t *ci = coords + (uint64_t)mode * M;
    for (uint64_t x = 0; x < M; ++x) ptr[ci[x] + 1]++;
    for (uint64_t i = 0; i < I; ++i) ptr[i + 1] += ptr[i];
    uint64_t *fill = (uint64_t *)malloc(sizeof(uint64_t) * (I ? I : 1));
    if (!fill) { free(ptr); free(lst); return -1; }
    memcpy(fill, ptr, sizeof(uint64_t) * I);
    for (uint64_t x = 0; x < M; ++x) lst[fill[ci[x]]++] = x;
    free(fill);
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 1024) num_threads(nthreads)
#endif
    for (int64_t i = 0; i < (int64_t)I; ++i) {
        for (uint64_t k = ptr[i]; k < ptr[i + 1]; ++k) {
            uint64_t x = lst[k];
            for (int r = 0; r < R; ++r)
                out[(uint64_t)i * R + r] += term(nmodes, x, M, coords, vals, factors, R, mode, r);
        }
    }
    free(ptr);
    free(lst);
    return 0;
}

/* Only the rows listed in `rows` (nrows of them, distinct): out is nrows x R.
 * One pass over the nonzeros in input order. */
int oracle_mttkrp_rows_f64(int nmodes, uint64_t M, const uint32_t *coords, const float *vals,
                           const uint64_t *dims, const float *const *factors, int R, int mode,
                           const uint32_t *rows, int64_t nrows, double *out) {
    uint64_t I = dims[mode];
    int64_t *slot = (int64_t *)malloc(sizeof(int64_t) * (I ? I : 1));
    if (!slot) return -1;
    for (uint64_t i = 0; i < I; ++i) slot[i] = -1;
    for (int64_t k = 0; k < nrows; ++k) slot[rows[k]] = k;
    memset(out, 0, sizeof(double) * (uint64_t)nrows * (uint64_t)R);
    const uint32_t *ci = coords + (uint64_t)mode * M;
    for (uint64_t x = 0; x < M; ++x) {
        int64_t s = slot[ci[x]];
        if (s < 0) continue;
        for (int r = 0; r < R; ++r)
            out[(uint64_t)s * R + r] += term(nmodes, x, M, coords, vals, factors, R, mode, r);
    }
    free(slot);
    return 0;
}

/* pos: nmodes x 32 key positions (pos[n*32+g] for g < bits[n]).
 * keys: M x kw words (kw = 1 or 2), word 0 = low 64 bits. */
void oracle_linearize(int nmodes, uint64_t M, const uint32_t *coords, const int *bits,
                      const int *pos, int kw, uint64_t *keys) {
    for (uint64_t x = 0; x < M; ++x) {
        uint64_t w[2] = {0, 0};
        for (int n = 0; n < nmodes; ++n) {
            uint32_t c = coords[(uint64_t)n * M + x];
            for (int g = 0; g < bits[n]; ++g) {
                int q = pos[n * 32 + g];
                uint64_t b = (uint64_t)((c >> g) & 1u);
                w[q >> 6] |= b << (q & 63);
            }
        }
        keys[x * (uint64_t)kw] = w[0];
        if (kw == 2) keys[x * 2 + 1] = w[1];
    }
}

int oracle_max_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}
