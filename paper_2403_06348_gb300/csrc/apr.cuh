// CP-APR with multiplicative updates (Alg. 2): the element-wise and
// reduction kernels around the Phi kernel (apr.cu). Factors, B and Phi are
// fp32 I x R row-major; lambda and column sums are fp64.
#pragma once

#include "alto_internal.cuh"

namespace alto {

struct FactorPtrs {
  const float *p[kMaxModes];
};

// sums[r] += sum_i A(i, r) (sums zeroed by the caller).
cudaError_t launch_colsum(const float *A, uint64_t I, int R, double *sums, int num_sms,
                          cudaStream_t s);

// A(:, r) /= sums[r] where sums[r] > 0; with lam, lam[r] *= sums[r] (lam may
// be null). Launched once, after launch_colsum.
cudaError_t launch_normalize(float *A, uint64_t I, int R, const double *sums, double *lam,
                             int num_sms, cudaStream_t s);

// B = (A + S) diag(lam), S(i,r) = kappa where shift && A(i,r) < kappa_tol &&
// Phi_prev(i,r) > 1 (Alg. 2, the inadmissible-zero adjustment).
cudaError_t launch_shift_scale(const float *A, const float *phi_prev, uint64_t I, int R,
                               const double *lam, int shift, float kappa, float kappa_tol, float *B,
                               int num_sms, cudaStream_t s);

// Start of an inner iteration unless *done: zero Phi (when zero_phi) and the
// KKT maximum.
cudaError_t launch_inner_begin(float *phi, uint64_t I, int R, bool zero_phi, unsigned *kkt_bits,
                               const int *done, int num_sms, cudaStream_t s);

// Unless *done: *kkt = max over (i, r) of |min(B, 1 - Phi)| (as float bits).
cudaError_t launch_kkt(const float *B, const float *phi, uint64_t I, int R, unsigned *kkt_bits,
                       const int *done, int num_sms, cudaStream_t s);

// Unless *done: if *kkt < tau the inner loop ends (*done = 1); else
// B *= Phi element-wise, *stepped = 1 and ++*steps.
cudaError_t launch_mu(float *B, const float *phi, uint64_t I, int R, const unsigned *kkt_bits,
                      float tau, int *done, int *stepped, int *steps, int num_sms, cudaStream_t s);

// Pi(x, :) = *_{m != n} A^(m)(i_m(x), :) for every ordered nonzero x (PRE).
cudaError_t launch_pi(const DecodePlan &dp, const uint64_t *keys, uint64_t nnz, int mode,
                      const FactorPtrs &factors, int R, float *pi, int num_sms, cudaStream_t s);

// *acc += sum over nonzeros of v log(max(M(x), tiny)), M(x) = sum_r lam_r
// prod_m A^(m)(i_m(x), r): the data term of the Poisson objective.
cudaError_t launch_loglik(const DecodePlan &dp, const uint64_t *keys, const float *vals, uint64_t nnz,
                          const FactorPtrs &factors, const double *lam, int R, double *acc,
                          int num_sms, cudaStream_t s);

}  // namespace alto
