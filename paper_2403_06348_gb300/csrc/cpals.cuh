// CP-ALS glue kernels (Alg. 1) and their launchers (cpals.cu).
#pragma once

#include "alto_internal.cuh"

namespace alto {

// Factors are kept internally as B_m with A_m = B_m diag(s_m): the column
// normalisation of Alg. 1 is carried as the scale vector s_m and folded into
// the next solve, because MTTKRP commutes with column scaling.
struct CpArgs {
  double *G;              // [N][R][R] Grams of the normalised factors A_m
  double *s;              // [N][R] column scales s_m
  double *Sn;             // [R] prod_{m != n} s_m of the current mode (kept for the fit)
  const double *BtB;      // [R][R] B_n^T B_n of the new (unnormalised) update
  const double *dot;      // [R] sum_i M_B(i, r) B_n(i, r)
  float *W;               // [2][R][R] W1 then W2 (fp32): W1 W2 = diag(Sn) V^-1 diag(1 / wcol),
                          // W1 = diag(Sn) F, W2 = G for the factors F G of V^-1 (or V^+)
  double *wcol;           // [R] power-of-two column scales of W2 (the fp32 W stays in range)
  double *rscale;         // [R] renormalisation factors of B_n (renorm_kernel)
  int *renorm;            // nonzero: B_n is to be renormalised (s_n already set to 1)
  double *lambda;         // [R] column norms of the last update
  double *fits;           // [iters]
  const double *norm_sq;  // ||X||^2
  int *done_at;           // first iteration to skip (INT_MAX: none)
  int *iters_done;
  uint32_t *status;
  int N, n, R, it;
  int last_mode;
  double tol;
};

cudaError_t launch_gram(const float *A, uint64_t I, int R, double *G, int num_sms, cudaStream_t s);
cudaError_t launch_prepare(const CpArgs &a, cudaStream_t s);
// B = (M W1) W2 into B (W = W1 then W2, each R x R) with BtB += B^T B and
// dot += diag(M^T B) (both zeroed by the caller); one pass over M.
cudaError_t launch_update(const float *M, const float *W, float *B, uint64_t I, int R, double *BtB,
                          double *dot, const int *done_at, int it, int num_sms, cudaStream_t s);
// The same on the tensor cores (TF32 with an error-compensating split,
// update_tc.cu) for the ranks update_tc_supported accepts; a bounded wait that
// expires sets kStatusTimeout in *status.
bool update_tc_supported(int R);
cudaError_t launch_update_tc(const float *M, const float *W, float *B, uint64_t I, int R, double *BtB,
                             double *dot, const int *done_at, int it, uint32_t *status, int num_sms,
                             cudaStream_t s);
cudaError_t launch_finish(const CpArgs &a, cudaStream_t s);
// B(:, r) *= rscale[r] when *renorm is set (finish decided it); else nothing.
cudaError_t launch_renorm(float *B, const double *rscale, const int *renorm, uint64_t I, int R, int num_sms,
                          cudaStream_t s);
cudaError_t launch_scale(float *B, const double *s_m, uint64_t I, int R, int num_sms, cudaStream_t s);

}  // namespace alto
