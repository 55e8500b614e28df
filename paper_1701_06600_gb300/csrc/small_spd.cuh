// Small symmetric positive definite R x R systems in shared memory (the Gram matrix of the sampled
// least-squares problem, Alg. 3), shared by the two thread-block-cluster loop kernels.
//
// Every routine is deterministic (fixed operation order, no data-dependent thread counts), so the
// CTAs of a cluster that run it on identical inputs get bit-identical results and take the same
// singularity decision.
#pragma once

#include <math.h>

namespace cpr {

// 1/sqrt(d) for d > 0 in FP64: FP32 seed, two Newton steps (2^-23 -> 2^-46 -> FP64 rounding).
__device__ __forceinline__ double rsqrt64(double d) {
  double y = (double)rsqrtf((float)d);
  y = y * fma(-0.5 * d * y, y, 1.5);
  y = y * fma(-0.5 * d * y, y, 1.5);
  return y;
}

// 1/d for d > 0 in FP64: FP32 seed, two Newton steps.
__device__ __forceinline__ double recip64(double d) {
  double x = (double)__frcp_rn((float)d);
  x = x * fma(-d, x, 2.0);
  x = x * fma(-d, x, 2.0);
  return x;
}

// Cholesky G = L L^T in shared memory (lower triangle; the diagonal gets L_kk and dinv[k] = 1/L_kk).
// A pivot that is not positive relative to the largest diagonal entry (or not finite) sets *s_bad.
__device__ inline void cholesky_smem(double* G, double* dinv, int R, int* s_bad) {
  const int tid = threadIdx.x, lane = tid & 31;
  if (R <= 32) {
    if (tid < 32) {                       // one warp; lane i owns row i
      double md = lane < R ? G[lane * R + lane] : 0.0;
      for (int o = 16; o > 0; o >>= 1) md = fmax(md, __shfl_xor_sync(0xffffffffu, md, o));
      for (int k = 0; k < R; ++k) {
        double d = G[k * R + k];
        const bool bad = !(d > 1e-26 * md) || !isfinite(d);
        if (bad) d = 1.0;
        const double y = rsqrt64(d);
        if (lane == 0) {
          G[k * R + k] = d * y;
          dinv[k] = y;
          if (bad) *s_bad = 1;
        }
        __syncwarp();
        if (lane > k && lane < R) G[lane * R + k] *= y;
        __syncwarp();
        if (lane > k && lane < R) {
          const double lik = G[lane * R + k];
          for (int c = k + 1; c <= lane; ++c) G[lane * R + c] = fma(-lik, G[c * R + k], G[lane * R + c]);
        }
        __syncwarp();
      }
    }
    __syncthreads();
    return;
  }
  __shared__ double maxdiag;
  if (tid == 0) {
    double m = 0.0;
    for (int k = 0; k < R; ++k) m = fmax(m, G[k * R + k]);
    maxdiag = m;
  }
  __syncthreads();
  for (int k = 0; k < R; ++k) {
    if (tid == 0) {
      double d = G[k * R + k];
      if (!(d > 1e-26 * maxdiag) || !isfinite(d)) {
        *s_bad = 1;
        d = 1.0;
      }
      const double y = rsqrt64(d);
      G[k * R + k] = d * y;
      dinv[k] = y;
    }
    __syncthreads();
    const double inv = dinv[k];
    for (int i = k + 1 + tid; i < R; i += blockDim.x) G[i * R + k] *= inv;
    __syncthreads();
    const int rem = R - k - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      const int i = k + 1 + e / rem, c = k + 1 + e % rem;
      if (c <= i) G[i * R + c] = fma(-G[i * R + k], G[c * R + k], G[i * R + c]);
    }
    __syncthreads();
  }
}

// X = G^-1 in FP64 by the whole block: Cholesky of a copy Lw of G, the triangular inverse
// Tm = L^-1 (one column per thread), X = L^-T L^-1.  Lw, Tm: R x R scratch; dinv: R.
__device__ inline void spd_inverse_fp64(const double* G, double* X, double* Lw, double* Tm, double* dinv, int R,
                                        int* s_bad) {
  const int tid = threadIdx.x;
  for (int e = tid; e < R * R; e += blockDim.x) Lw[e] = G[e];
  __syncthreads();
  cholesky_smem(Lw, dinv, R, s_bad);
  if (tid < R) {
    const int c = tid;
    for (int r = 0; r < c; ++r) Tm[r * R + c] = 0.0;
    Tm[c * R + c] = dinv[c];
    for (int r = c + 1; r < R; ++r) {
      double s0 = 0.0, s1 = 0.0;
      int l = c;
      for (; l + 1 < r; l += 2) {
        s0 = fma(Lw[r * R + l], Tm[l * R + c], s0);
        s1 = fma(Lw[r * R + l + 1], Tm[(l + 1) * R + c], s1);
      }
      if (l < r) s0 = fma(Lw[r * R + l], Tm[l * R + c], s0);
      Tm[r * R + c] = -(s0 + s1) * dinv[r];
    }
  }
  __syncthreads();
  for (int e = tid; e < R * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    double a0 = 0.0, a1 = 0.0;
    int l = max(r, c);
    for (; l + 1 < R; l += 2) {
      a0 = fma(Tm[l * R + r], Tm[l * R + c], a0);
      a1 = fma(Tm[(l + 1) * R + r], Tm[(l + 1) * R + c], a1);
    }
    if (l < R) a0 = fma(Tm[l * R + r], Tm[l * R + c], a0);
    X[e] = a0 + a1;
  }
  __syncthreads();
}

}  // namespace cpr
