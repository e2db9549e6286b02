// Device bodies of the CP-ALS glue kernels (Alg. 1), shared by the
// one-tensor kernels (cpals.cu) and the CP-ALS batch (batch.cu). Every body
// is run by all threads of one CTA of kUpdThreads (256) threads.
#pragma once

#include "cpals.cuh"

namespace alto {

constexpr int kUpdThreads = 256;

// Shared memory of update_body at rank R.
inline size_t update_smem(int R) {
  const int TR = 4096 / R;
  return (size_t)(R * R + R) * sizeof(double) +
         (size_t)(2 * R * R + R * (TR + 4) + TR * (R + 4)) * sizeof(float);
}

// Pseudo-inverse of the symmetric R x R matrix A (destroyed) into Y, with Q
// as work space: cyclic Jacobi rotations in the round-robin order (R/2
// disjoint pairs per step, R - 1 steps per sweep; Golub and Van Loan,
// "parallel Jacobi") until the off-diagonal mass is below 1e-15 of the
// total. Then A^+ = Q diag(1/lambda) Q^T over the eigenvalues with |lambda| >
// 1e-15 max |lambda| (the cut numpy's pinv makes) leaves as two factors,
// A^+ = F G: F = Q |Lambda|^-1/2 into Y and G = sign(Lambda) |Lambda|^-1/2 Q^T
// into A (columns of F and rows of G under the cut are 0). Returns false if
// A has a non-finite entry. Called by all threads of the CTA.
__device__ __forceinline__ bool pinv_body(double *A, double *Q, double *Y, int R, int lgR) {
  const int tid = threadIdx.x, nt = blockDim.x, RR = R * R, half = R / 2;
  __shared__ double c_s[ALTO_MAX_RANK / 2], s_s[ALTO_MAX_RANK / 2], red[2][32];
  __shared__ int p_s[ALTO_MAX_RANK / 2], q_s[ALTO_MAX_RANK / 2];
  const int lane = tid & 31, warp = tid >> 5, nw = (nt + 31) >> 5;
  bool finite = true;
  for (int e = tid; e < RR; e += nt) {
    Q[e] = ((e >> lgR) == (e & (R - 1))) ? 1.0 : 0.0;
    finite = finite && isfinite(A[e]);
  }
  if (!__syncthreads_and(finite)) return false;
  for (int sweep = 0; sweep < 30; ++sweep) {
    double off = 0.0, tot = 0.0;
    for (int e = tid; e < RR; e += nt) {
      const double v = A[e] * A[e];
      tot += v;
      if ((e >> lgR) != (e & (R - 1))) off += v;
    }
    for (int o = 16; o > 0; o >>= 1) {
      off += __shfl_xor_sync(0xffffffffu, off, o);
      tot += __shfl_xor_sync(0xffffffffu, tot, o);
    }
    if (lane == 0) {
      red[0][warp] = off;
      red[1][warp] = tot;
    }
    __syncthreads();
    off = tot = 0.0;
    for (int w = 0; w < nw; ++w) {
      off += red[0][w];
      tot += red[1][w];
    }
    __syncthreads();
    if (!(off > 1e-30 * tot)) break;  // the same sums in every thread
    for (int step = 0; step < R - 1; ++step) {
      if (tid < half) {
        int p, q;
        if (tid == 0) {
          p = step;
          q = R - 1;
        } else {
          p = (step + tid) % (R - 1);
          q = (step - tid + R - 1) % (R - 1);
        }
        const double apq = A[p * R + q];
        double c = 1.0, sn = 0.0;
        if (apq != 0.0) {
          const double tau = (A[q * R + q] - A[p * R + p]) / (2.0 * apq);
          const double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
          c = 1.0 / sqrt(1.0 + t * t);
          sn = t * c;
        }
        p_s[tid] = p;
        q_s[tid] = q;
        c_s[tid] = c;
        s_s[tid] = sn;
      }
      __syncthreads();
      for (int w = tid; w < half * R; w += nt) {  // rows p, q of every pair
        const int k = w >> lgR, j = w & (R - 1);
        const int p = p_s[k], q = q_s[k];
        const double c = c_s[k], sn = s_s[k];
        const double ap = A[p * R + j], aq = A[q * R + j];
        A[p * R + j] = c * ap - sn * aq;
        A[q * R + j] = sn * ap + c * aq;
      }
      __syncthreads();
      for (int w = tid; w < half * R; w += nt) {  // columns p, q; Q accumulates J
        const int k = w >> lgR, i = w & (R - 1);
        const int p = p_s[k], q = q_s[k];
        const double c = c_s[k], sn = s_s[k];
        const double ap = A[i * R + p], aq = A[i * R + q];
        A[i * R + p] = c * ap - sn * aq;
        A[i * R + q] = sn * ap + c * aq;
        const double qp = Q[i * R + p], qq = Q[i * R + q];
        Q[i * R + p] = c * qp - sn * qq;
        Q[i * R + q] = sn * qp + c * qq;
      }
      __syncthreads();
    }
  }
  // eigenvalues on the diagonal; the cut relative to the largest
  __shared__ double ev[ALTO_MAX_RANK];
  double mx = 0.0;
  for (int k = 0; k < R; ++k) mx = fmax(mx, fabs(A[k * R + k]));
  const double cut = 1e-15 * mx;
  for (int k = tid; k < R; k += nt) ev[k] = A[k * R + k];
  __syncthreads();
  for (int e = tid; e < RR; e += nt) {
    const int i = e >> lgR, k = e & (R - 1);
    const double lk = ev[k];
    Y[e] = fabs(lk) > cut ? Q[i * R + k] / sqrt(fabs(lk)) : 0.0;            // F[i][k]
    const double li = ev[i];
    A[e] = fabs(li) > cut ? copysign(1.0 / sqrt(fabs(li)), li) * Q[k * R + i] : 0.0;  // G[i][k]
  }
  __syncthreads();
  return true;
}

// V = Hadamard product of the other modes' Grams, its Cholesky factor L
// (V = L L^T), X = L^-1 and the solve factors W1 = diag(Sn) X^T, W2 = X
// (V^-1 = X^T X, never formed), all in fp64
// inside one CTA. Every elimination step is one pass over the R x R square
// followed by one barrier: a thread recomputes the pivot quantities it needs
// from values that are final before the step, and each step writes only
// entries that no thread reads in that step.
// sd: 3 R^2 doubles of shared memory.
__device__ __forceinline__ void prepare_body(const CpArgs &a, double *sd) {
  if (*a.done_at <= a.it) return;
  const int R = a.R, RR = R * R, tid = threadIdx.x, nt = blockDim.x;
  const int lgR = __ffs(R) - 1;
  double *V = sd;       // V; after the factorisation, X = L^-1
  double *L = V + RR;   // Cholesky factor (lower)
  double *Y = L + RR;   // forward-substitution work; then V^-1
  // 1/d_k and 1/sqrt(d_k) of each pivot, computed once by the thread that
  // finalises d_k (fp64 division is slow; every other thread reads them)
  __shared__ double s_inv[ALTO_MAX_RANK], s_rs[ALTO_MAX_RANK];
  for (int e = tid; e < RR; e += nt) {
    double v = 1.0;
    for (int m = 0; m < a.N; ++m)
      if (m != a.n) v *= a.G[(size_t)m * RR + e];
    V[e] = v;
    Y[e] = ((e >> lgR) == (e & (R - 1))) ? 1.0 : 0.0;
    if (e == 0 && v > 0.0) {
      s_inv[0] = 1.0 / v;
      s_rs[0] = rsqrt(v);
    }
  }
  __syncthreads();
  // Cholesky, right-looking: step k writes column k of L and updates the
  // trailing lower triangle (i >= j > k) of V from column k of V.
  bool spd = true;
  for (int k = 0; k < R; ++k) {
    const double d = V[k * R + k];
    if (!(d > 0.0) || !isfinite(d)) {  // the same d in every thread
      spd = false;
      break;
    }
    const double inv_d = s_inv[k], rs = s_rs[k];
    for (int e = tid; e < RR; e += nt) {
      const int i = e >> lgR, j = e & (R - 1);
      if (j == k) {
        if (i >= k) L[e] = V[e] * rs;
      } else if (j > k && j <= i) {
        const double v = V[e] - V[i * R + k] * V[j * R + k] * inv_d;
        V[e] = v;
        if (i == k + 1 && j == k + 1 && v > 0.0) {  // the next pivot
          s_inv[k + 1] = 1.0 / v;
          s_rs[k + 1] = rsqrt(v);
        }
      }
    }
    __syncthreads();
  }
  // The solve leaves as two factors F G = V^-1 (or V^+), never as the
  // explicit inverse: B_n = (M F) G keeps the error of each fp32 product near
  // sqrt(cond V) times the rounding instead of cond V (on the 1e8-nonzero
  // Zipf tensor, iteration 1's last V has cond 1.4e6, and M V^-1 formed in
  // fp32 moved the fit by 8e-4; the two factors by 2e-7).
  //   Cholesky V = L L^T: F = X^T, G = X with X = L^-1;
  //   otherwise (the pseudo-inverse, as Alg. 1 states it): F and G from the
  //   eigendecomposition of V (fp64 Jacobi).
  // F goes to Y, G to V; only a V with a non-finite entry ends the run.
  if (!spd) {
    for (int e = tid; e < RR; e += nt) {
      double v = 1.0;
      for (int m = 0; m < a.N; ++m)
        if (m != a.n) v *= a.G[(size_t)m * RR + e];
      V[e] = v;
    }
    __syncthreads();
    if (!pinv_body(V, L, Y, R, lgR)) {
      if (tid == 0) {
        atomicOr(a.status, kStatusNotSpd);
        *a.done_at = a.it;
      }
      return;
    }
    if (tid == 0) atomicOr(a.status, kStatusPinv);
  } else {
    // X = L^-1 by forward substitution on Y = I: step k finalises row k of X
    // (into V) and removes column k of L from the rows below.
    for (int k = 0; k < R; ++k) {
      const double inv = s_rs[k];  // 1 / L[k][k] = 1 / sqrt(d_k)
      for (int e = tid; e < RR; e += nt) {
        const int i = e >> lgR, c = e & (R - 1);
        if (c > k || i < k) continue;
        const double xk = Y[k * R + c] * inv;
        if (i == k) V[e] = xk;
        else Y[e] -= L[i * R + k] * xk;
      }
      __syncthreads();
    }
    // X is lower triangular: zero above the diagonal, F = X^T
    for (int e = tid; e < RR; e += nt) {
      const int i = e >> lgR, c = e & (R - 1);
      if (c > i) V[e] = 0.0;
    }
    __syncthreads();
    for (int e = tid; e < RR; e += nt) {
      const int i = e >> lgR, c = e & (R - 1);
      Y[e] = V[c * R + i];
    }
  }
  for (int r = tid; r < R; r += nt) {
    double p = 1.0;
    for (int m = 0; m < a.N; ++m)
      if (m != a.n) p *= a.s[(size_t)m * R + r];
    a.Sn[r] = p;
  }
  __syncthreads();
  // W1 = diag(Sn) F and W2 = G, stored in fp32 (W1 then W2). Sn multiplies
  // the other modes' deferred scales and can leave the fp32 range although
  // the solve is well defined: a column of W1 whose largest entry is outside
  // [2^-60, 2^60] is divided by a power of two near it (the same power
  // multiplies the matching row of W2), and so is a column of W2 (undone in
  // fp64 by finish_body through wcol). Other columns keep scale 1, so that
  // B_n = M W1 W2 keeps its natural magnitude (the column norms lambda).
  for (int e = tid; e < RR; e += nt) Y[e] *= a.Sn[e >> lgR];
  __syncthreads();
  __shared__ int bad;
  __shared__ double ycol[ALTO_MAX_RANK];
  if (tid == 0) bad = 0;
  __syncthreads();
  for (int c = tid; c < R; c += nt) {
    double mx = 0.0;
    for (int k = 0; k < R; ++k) mx = fmax(mx, fabs(Y[k * R + c]));
    if (!isfinite(mx)) bad = 1;
    ycol[c] = (mx > 0.0 && isfinite(mx) && (mx > 0x1p60 || mx < 0x1p-60)) ? ldexp(1.0, ilogb(mx)) : 1.0;
  }
  __syncthreads();
  for (int e = tid; e < RR; e += nt) V[e] *= ycol[e >> lgR];
  __syncthreads();
  for (int c = tid; c < R; c += nt) {
    double mx = 0.0;
    for (int k = 0; k < R; ++k) mx = fmax(mx, fabs(V[k * R + c]));
    if (!isfinite(mx)) bad = 1;
    a.wcol[c] = (mx > 0.0 && isfinite(mx) && (mx > 0x1p60 || mx < 0x1p-60)) ? ldexp(1.0, ilogb(mx)) : 1.0;
  }
  __syncthreads();
  if (bad) {
    if (tid == 0) {
      atomicOr(a.status, kStatusNotSpd);
      *a.done_at = a.it;
    }
    return;
  }
  for (int e = tid; e < RR; e += nt) {
    a.W[e] = (float)(Y[e] / ycol[e & (R - 1)]);
    a.W[RR + e] = (float)(V[e] / a.wcol[e & (R - 1)]);
  }
}

// B = (M W1) W2 with B^T B and the column dot products of M and B, one pass.
// A tile of TR = 4096 / R rows: every thread computes a 4-row x 4-column block
// of Y = M W1 from the transposed M tile (two 16-byte shared loads per 16
// FMAs), puts it in shared memory, computes its block of B = Y W2 the same
// way, adds its block's column products M(r,c) B(r,c), stores B, and then
// accumulates a 4 x 4 block of B^T B over its share of the tile's rows.
// fp32 partial sums cover at most 32 tiles per thread before they move to
// fp64. The CTA walks tiles t0, t0 + tstep, ... < t1 (TR rows each); with
// clear_m it also zeroes the M rows it has read.

// o = the 4 x 4 block (rows 4 rb.., columns 4 cb..) of T W, T given
// transposed in shared memory (column k of T at t + k * ld), W row-major R x R
__device__ __forceinline__ void block_product(const float *t, int ld, const float *w, int R, int rb, int cb,
                                              float (&o)[4][4]) {
#pragma unroll
  for (int x = 0; x < 4; ++x)
#pragma unroll
    for (int y = 0; y < 4; ++y) o[x][y] = 0.f;
  for (int k = 0; k < R; ++k) {
    const float4 tk = *reinterpret_cast<const float4 *>(t + k * ld + 4 * rb);
    const float4 wk = *reinterpret_cast<const float4 *>(w + k * R + 4 * cb);
    const float ta[4] = {tk.x, tk.y, tk.z, tk.w}, wa[4] = {wk.x, wk.y, wk.z, wk.w};
#pragma unroll
    for (int x = 0; x < 4; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) o[x][y] = fmaf(ta[x], wa[y], o[x][y]);
  }
}

// SYM: the Gram pass forms only the blocks of B^T B on and above the diagonal
// (B4 (B4 + 1) / 2 of the B4^2 4 x 4 blocks) and mirrors them at the end;
// worth it where one call covers many tiles (the single-tensor update). The
// batch update, which calls this once per short tile range, keeps all blocks
// and its cheap warp pre-reduction.
template <bool SYM = false>
__device__ __forceinline__ void update_body(float *M, const float *__restrict__ W,
                                            float *__restrict__ Bout, uint64_t I, int R,
                                            double *__restrict__ BtB, double *__restrict__ dot,
                                            uint64_t t0, uint64_t tstep, uint64_t t1, bool clear_m,
                                            unsigned char *smraw) {
  __syncthreads();  // shared memory may still be read by a previous call
  const int TR = 4096 / R;       // rows per tile
  const int TRP = TR + 4;        // padded row count of the transposed tile
  const int RP = R + 4;          // padded row length of the B tile
  double *red = reinterpret_cast<double *>(smraw);       // R*R + R
  float *w = reinterpret_cast<float *>(red + R * R + R);  // 2 R*R: W1, W2
  float *mt = w + 2 * R * R;                              // R * TRP (M tile, transposed)
  float *bt = mt + R * TRP;                               // TR * RP (B tile; first M W1, transposed)
  const int tid = threadIdx.x;
  const int B4 = R / 4;                      // column blocks
  const int cb = tid % B4, rb = tid / B4;    // phase 1: rows 4*rb .. 4*rb+3, cols 4*cb ..
  const int BB = SYM ? B4 * (B4 + 1) / 2 : B4 * B4, RG = kUpdThreads / BB;
  const int tb = tid % BB, rg = tid / BB;
  int bi = tb / B4, bj = tb % B4;
  if (SYM) {  // tb-th block of the upper triangle, row by row
    int rem = tb;
    bi = 0;
    while (rem >= B4 - bi) {
      rem -= B4 - bi;
      ++bi;
    }
    bj = bi + rem;
  }
  const bool gram = rg < RG;  // SYM leaves kUpdThreads mod BB threads out
  for (int i = tid; i < R * R + R; i += kUpdThreads) red[i] = 0.0;
  for (int i = tid; i < 2 * R * R; i += kUpdThreads) w[i] = W[i];
  float g[4][4], dp[4];
  double dg[4][4], ddp[4];
#pragma unroll
  for (int x = 0; x < 4; ++x) {
    dp[x] = 0.f;
    ddp[x] = 0.0;
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      g[x][y] = 0.f;
      dg[x][y] = 0.0;
    }
  }
  int tiles = 0;
  float4 *M4 = reinterpret_cast<float4 *>(M);
  // A tile is TR x R = 4096 floats: kPer 16-byte vectors per thread. The next
  // tile's vectors are loaded into registers while the current one is used.
  constexpr int kPer = 4096 / 4 / kUpdThreads;
  float4 nxt[kPer];
  auto load_tile = [&](uint64_t tt) {
    const uint64_t rr0 = tt * (uint64_t)TR;
    const int nr = (I - rr0) < (uint64_t)TR ? (int)(I - rr0) : TR;
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int i = tid + j * kUpdThreads, r = i / B4;
      nxt[j] = r < nr ? M4[(rr0 + r) * B4 + (i - r * B4)] : make_float4(0.f, 0.f, 0.f, 0.f);
    }
  };
  if (t0 < t1) load_tile(t0);
  for (uint64_t t = t0; t < t1; t += tstep) {
    const uint64_t r0 = t * (uint64_t)TR;
    const int nrows = (I - r0) < (uint64_t)TR ? (int)(I - r0) : TR;
    __syncthreads();
    // transpose the M tile into shared memory (rows beyond nrows are zero)
#pragma unroll
    for (int j = 0; j < kPer; ++j) {
      const int i = tid + j * kUpdThreads;
      const int r = i / B4, c = (i - r * B4) * 4;
      const float4 m = nxt[j];
      if (clear_m && r < nrows) M4[(r0 + r) * B4 + (i - r * B4)] = make_float4(0.f, 0.f, 0.f, 0.f);
      mt[(c + 0) * TRP + r] = m.x;
      mt[(c + 1) * TRP + r] = m.y;
      mt[(c + 2) * TRP + r] = m.z;
      mt[(c + 3) * TRP + r] = m.w;
    }
    if (t + tstep < t1) load_tile(t + tstep);
    __syncthreads();
    float o[4][4];
    // Y = M W1 (its block goes to shared memory, transposed like M), then
    // B = Y W2
    block_product(mt, TRP, w, R, rb, cb, o);
#pragma unroll
    for (int y = 0; y < 4; ++y)
      *reinterpret_cast<float4 *>(bt + (4 * cb + y) * TRP + 4 * rb) = make_float4(o[0][y], o[1][y], o[2][y], o[3][y]);
    __syncthreads();
    block_product(bt, TRP, w + R * R, R, rb, cb, o);
    __syncthreads();  // every read of Y is done before B overwrites it
    // column products with M, store B (global and shared)
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      const float4 mc = *reinterpret_cast<const float4 *>(mt + (4 * cb + y) * TRP + 4 * rb);
      const float ma[4] = {mc.x, mc.y, mc.z, mc.w};
#pragma unroll
      for (int x = 0; x < 4; ++x) dp[y] = fmaf(ma[x], o[x][y], dp[y]);
    }
#pragma unroll
    for (int x = 0; x < 4; ++x) {
      const int r = 4 * rb + x;
      const float4 ov = make_float4(o[x][0], o[x][1], o[x][2], o[x][3]);
      *reinterpret_cast<float4 *>(bt + r * RP + 4 * cb) = ov;
      if (r < nrows) *reinterpret_cast<float4 *>(Bout + (r0 + r) * (uint64_t)R + 4 * cb) = ov;
    }
    __syncthreads();
    for (int r = gram ? rg : nrows; r < nrows; r += RG) {
      const float4 xv = *reinterpret_cast<const float4 *>(bt + r * RP + 4 * bi);
      const float4 yv = *reinterpret_cast<const float4 *>(bt + r * RP + 4 * bj);
      const float xa[4] = {xv.x, xv.y, xv.z, xv.w}, ya[4] = {yv.x, yv.y, yv.z, yv.w};
#pragma unroll
      for (int x = 0; x < 4; ++x)
#pragma unroll
        for (int y = 0; y < 4; ++y) g[x][y] = fmaf(xa[x], ya[y], g[x][y]);
    }
    if (++tiles == 32) {
#pragma unroll
      for (int x = 0; x < 4; ++x) {
        ddp[x] += (double)dp[x];
        dp[x] = 0.f;
#pragma unroll
        for (int y = 0; y < 4; ++y) {
          dg[x][y] += (double)g[x][y];
          g[x][y] = 0.f;
        }
      }
      tiles = 0;
    }
  }
  __syncthreads();
  // Threads holding the same block of B^T B (the same tb) or the same columns
  // of the dot products (the same cb) are first summed inside the warp (lanes
  // equal modulo BB or B4), so at most one shared atomic per warp and address.
  const unsigned full = 0xffffffffu;
  const int lane = tid & 31;
#pragma unroll
  for (int x = 0; x < 4; ++x) {
#pragma unroll
    for (int y = 0; y < 4; ++y) {
      double v = dg[x][y] + (double)g[x][y];
      if (SYM) {
        if (gram) {
          atomicAdd(&red[(4 * bi + x) * R + 4 * bj + y], v);
          if (bi != bj) atomicAdd(&red[(4 * bj + y) * R + 4 * bi + x], v);
        }
        continue;
      }
      for (int o = 16; o >= BB; o >>= 1) v += __shfl_xor_sync(full, v, o);
      if (BB >= 32 || lane < BB) atomicAdd(&red[(4 * bi + x) * R + 4 * bj + y], v);
    }
    double v = ddp[x] + (double)dp[x];
    for (int o = 16; o >= B4; o >>= 1) v += __shfl_xor_sync(full, v, o);
    if (B4 >= 32 || lane < B4) atomicAdd(&red[R * R + 4 * cb + x], v);
  }
  __syncthreads();
  for (int i = tid; i < R * R; i += kUpdThreads)
    if (red[i] != 0.0) atomicAdd(&BtB[i], red[i]);
  for (int i = tid; i < R; i += kUpdThreads)
    if (red[R * R + i] != 0.0) atomicAdd(&dot[i], red[R * R + i]);
}

__device__ __forceinline__ void finish_body(const CpArgs &a) {
  if (*a.done_at <= a.it) return;
  const int R = a.R, RR = R * R, tid = threadIdx.x;
  __shared__ double lam[ALTO_MAX_RANK], sn[ALTO_MAX_RANK];
  __shared__ double part[2][256];
  double *sv = a.s + (size_t)a.n * R;
  double *Gn = a.G + (size_t)a.n * RR;
  // the stored B_n is the solution with column r divided by wcol[r]:
  // lambda_r = wcol[r] ||B_n(:, r)||, and A_n(:, r) = B_n(:, r) / ||B_n(:, r)||
  __shared__ double bn[ALTO_MAX_RANK];
  __shared__ int flags;  // bit 0: non-finite update, bit 1: renormalise B_n
  if (tid == 0) flags = 0;
  __syncthreads();
  for (int r = tid; r < R; r += blockDim.x) {
    const double g = a.BtB[r * R + r];
    if (!isfinite(g)) atomicOr(&flags, 1);
    bn[r] = g > 0.0 ? sqrt(g) : 0.0;
    lam[r] = bn[r] * a.wcol[r];
  }
  __syncthreads();
  if (flags & 1) {  // the update left the fp32 range: the run ends here
    if (tid == 0) {
      atomicOr(a.status, kStatusNotSpd);
      *a.done_at = a.it;
    }
    return;
  }
  // a column of rounding noise (norm at most 1e-12 of the largest, left by a
  // pseudo-inverse solve) is a zero column: lambda_r = 0 and s_r = 0
  double lmax = 0.0;
  for (int r = 0; r < R; ++r) lmax = fmax(lmax, lam[r]);
  __syncthreads();
  // Column norms of B_n far from 1 would let the deferred normalisation
  // drift out of the fp32 range over the iterations (the MTTKRP multiplies
  // the other N - 1 factors' entries): outside [2^-e, 2^e], with
  // e = min(60, 90 / (N - 1)), B_n is renormalised (renorm_kernel).
  const double elim = a.N > 1 ? fmin(60.0, floor(90.0 / (a.N - 1))) : 60.0;
  const double hi = ldexp(1.0, (int)elim), lo = ldexp(1.0, -(int)elim);
  for (int r = tid; r < R; r += blockDim.x) {
    double l = lam[r];
    if (!(l > 1e-12 * lmax)) l = 0.0;
    lam[r] = l;
    sn[r] = l > 0.0 ? 1.0 / bn[r] : 0.0;
    a.lambda[r] = l;
    if (sn[r] != 0.0 && (sn[r] > hi || sn[r] < lo)) atomicOr(&flags, 2);
  }
  __syncthreads();
  for (int e = tid; e < RR; e += blockDim.x) Gn[e] = a.BtB[e] * sn[e / R] * sn[e % R];
  const bool renorm = (flags & 2) != 0 && a.rscale != nullptr;
  for (int r = tid; r < R; r += blockDim.x) {
    if (renorm) a.rscale[r] = sn[r];
    sv[r] = renorm ? (sn[r] != 0.0 ? 1.0 : 0.0) : sn[r];
  }
  if (tid == 0 && a.renorm) *a.renorm = renorm ? 1 : 0;
  __syncthreads();
  if (!a.last_mode) return;
  // fit = 1 - sqrt(max(0, ||X||^2 + lam^T (*_m G_m) lam - 2 <X, X_hat>)) / ||X||,
  // <X, X_hat> = sum_r lam_r sum_i M(i,r) A_n(i,r) = sum_r Sn_r sum_i M_B(i,r) B_n(i,r)
  double s1 = 0.0, s2 = 0.0;
  for (int e = tid; e < RR; e += blockDim.x) {
    double h = 1.0;
    for (int m = 0; m < a.N; ++m) h *= a.G[(size_t)m * RR + e];
    s1 += lam[e / R] * lam[e % R] * h;
  }
  for (int r = tid; r < R; r += blockDim.x) s2 += a.Sn[r] * a.wcol[r] * a.dot[r];
  part[0][tid] = s1;
  part[1][tid] = s2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (tid < o) {
      part[0][tid] += part[0][tid + o];
      part[1][tid] += part[1][tid + o];
    }
    __syncthreads();
  }
  if (tid == 0) {
    const double nx = *a.norm_sq;
    const double resid = nx + part[0][0] - 2.0 * part[1][0];
    const double fit = nx > 0.0 ? 1.0 - sqrt(resid > 0.0 ? resid : 0.0) / sqrt(nx) : 0.0;
    a.fits[a.it] = fit;
    *a.iters_done = a.it + 1;
    if (a.tol > 0.0 && a.it > 0 && fabs(fit - a.fits[a.it - 1]) < a.tol) *a.done_at = a.it + 1;
  }
}

}  // namespace alto
