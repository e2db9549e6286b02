// CP-ALS glue kernels (Alg. 1) and their launchers (cpals.cu).
#pragma once

#include "alto_internal.cuh"

namespace alto {

struct SolveArgs {
  const double *G;       // [N][R][R] Grams of the current (normalised) factors
  double *G_out;         // G + n*R*R: overwritten with the new mode-n Gram
  const double *MtM;     // [R][R] M^T M of this mode's MTTKRP
  float *W;              // [R][R] out: V^-1 diag(1/lambda), fp32
  double *lambda;        // [R] out
  double *fits;          // [iters] fit after each iteration
  const double *norm_sq; // ||X||^2
  int *done_at;          // first iteration to skip (early stop); INT_MAX = none
  int *iters_done;
  uint32_t *status;
  int N, n, R, it;
  int last_mode;         // n == N-1: evaluate the fit
  double tol;
};

cudaError_t launch_gram(const float *A, uint64_t I, int R, double *G, const int *done_at, int it,
                        int num_sms, cudaStream_t s);
cudaError_t launch_solve(const SolveArgs &a, cudaStream_t s);
cudaError_t launch_rmul(const float *M, const float *W, float *A, uint64_t I, int R,
                        const int *done_at, int it, int num_sms, cudaStream_t s);

}  // namespace alto
