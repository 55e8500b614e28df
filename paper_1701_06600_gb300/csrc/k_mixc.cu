// CPRAND-MIX in its complex form (Alg. 4): the kernels of one mode update and of the sampled fit.
//
// The mixing operator of mode n is W_n = F_n D_n with F_n the unitary DFT; the mixed tensor is
// complex (interleaved FP32 pairs).  The factors A^(m) stay real (FP64) and their mixed copies
// A^^(m) = W_m A^(m) are complex FP32.  A mode-n update:
//   1. the sampled fibers of the mixed tensor (contiguous in its mode-n unfolding copy) are unmixed
//      in mode n, X_S = W_n^H X^_S, and stored as the stacked real matrix [Re X_S, Im X_S] (I_n x 2S);
//   2. the rows of the mixed Khatri-Rao product, Z^_S(j, :) = prod_{m != n} A^^(m)(i_m, :), stacked
//      as [Re Z^_S; Im Z^_S] (2S x R, FP64);
//   3. the normal equations of the real least squares of eq. (rcLS): G = Z_r^T Z_r, M = X_r Z_r;
//   4. A = M G^-1 (FP64 Cholesky inverse), column norms, normalization;
//   5. the new mixed copy A^^(n) = W_n A^(n).
// The stopping test is the sampled fit of §3.4 on the original real tensor with the real factors.
#include <math.h>

#include "internal.cuh"
#include "small_spd.cuh"

namespace cpr {
namespace {

constexpr int kSB = 16;   // sampled fibers per block of the unmixing kernel

__device__ __forceinline__ double2 cmul64(double2 a, double2 b) {
  return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

// W = F D (I x I, row k, column i): exp(-2 pi i k i / I) d_i / sqrt(I), from FP64, rounded once
__global__ void k_cf_ops(int I, const double* __restrict__ signs, float2* __restrict__ W) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)I * I) return;
  const int64_t k = e / I, i = e - k * I;
  const int64_t q = (k * i) % I;
  double s, c;
  sincospi(2.0 * (double)q / (double)I, &s, &c);
  const double f = signs[i] / sqrt((double)I);
  W[e] = make_float2((float)(c * f), (float)(-s * f));
}

// Random initial factor of mode m (the init stream, as CPRAND) and its mixed copy is made by
// k_cf_mix_factor afterwards.
__global__ void k_cf_init(int I, int R, int m, uint64_t seed, uint32_t b, double* __restrict__ A) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)I * R) return;
  const uint32_t i = (uint32_t)(e / R), r = (uint32_t)(e % R);
  const uint4 w = philox10(make_uint4(i, counter_word1(kStreamInit, 0, m), r / 4, b), (uint32_t)seed,
                           (uint32_t)(seed >> 32));
  A[e] = (double)(word_of(w, r % 4) >> 8) * (1.0 / 16777216.0);
}

// A^^ = W A (I x R complex, FP32 products accumulated in FP32 per 32-term chunk, chunks in FP64)
__global__ void k_cf_mix_factor(int I, int R, const float2* __restrict__ W, const double* __restrict__ A,
                                float2* __restrict__ Ah) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)I * R) return;
  const int k = (int)(e / R), r = (int)(e - (int64_t)(e / R) * R);
  const float2* w = W + (int64_t)k * I;
  double re = 0.0, im = 0.0;
  for (int i0 = 0; i0 < I; i0 += 32) {
    float pr = 0.f, pi = 0.f;
    for (int i = i0; i < min(I, i0 + 32); ++i) {
      const float a = (float)A[(int64_t)i * R + r];
      pr = fmaf(w[i].x, a, pr);
      pi = fmaf(w[i].y, a, pi);
    }
    re += pr;
    im += pi;
  }
  Ah[e] = make_float2((float)re, (float)im);
}

struct CfArgs {
  const float2* Xn;        // the mixed tensor's mode-n unfolding copy (fibers of I_n complex values)
  const uint32_t* idx;     // S x N sampled multi-indices
  const float2* W;         // W_n, I_n x I_n
  const float2* Ah[kMaxOrder];   // mixed factors, I_m x R
  int64_t dims[kMaxOrder];
  int N, n, S, R;
};

// 1. X_r = [Re, Im](W_n^H X^_S): a block unmixes kSB sampled fibers (staged in shared memory) for a
// range of rows i; each thread accumulates kSB complex outputs over k (FP32 per 32-term chunk).
__global__ void k_cf_unmix_fibers(CfArgs a, float* __restrict__ Xr) {
  extern __shared__ float2 xs[];   // kSB x I
  __shared__ int64_t col[kSB];
  const int I = (int)a.dims[a.n], S = a.S;
  const int j0 = blockIdx.x * kSB, nj = min(kSB, S - j0);
  if (threadIdx.x < nj) {   // column of the mode-n unfolding holding fiber j0 + t (index map of §2.1)
    const uint32_t* id = a.idx + (int64_t)(j0 + threadIdx.x) * a.N;
    int64_t c = 0, J = 1;
    for (int m = 0; m < a.N; ++m) {
      if (m == a.n) continue;
      c += (int64_t)id[m] * J;
      J *= a.dims[m];
    }
    col[threadIdx.x] = c;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < nj * I; e += blockDim.x) {
    const int jj = e / I, k = e - jj * I;
    xs[e] = a.Xn[col[jj] * I + k];
  }
  __syncthreads();
  for (int i = blockIdx.y * blockDim.x + threadIdx.x; i < I; i += gridDim.y * blockDim.x) {
    double re[kSB], im[kSB];
#pragma unroll
    for (int jj = 0; jj < kSB; ++jj) re[jj] = im[jj] = 0.0;
    for (int k0 = 0; k0 < I; k0 += 32) {
      float pr[kSB], pi[kSB];
#pragma unroll
      for (int jj = 0; jj < kSB; ++jj) pr[jj] = pi[jj] = 0.f;
      for (int k = k0; k < min(I, k0 + 32); ++k) {
        const float2 w = a.W[(int64_t)k * I + i];   // conj(W[k][i]) = (w.x, -w.y)
#pragma unroll
        for (int jj = 0; jj < kSB; ++jj) {
          const float2 x = xs[jj * I + k];
          pr[jj] = fmaf(w.x, x.x, fmaf(w.y, x.y, pr[jj]));
          pi[jj] = fmaf(w.x, x.y, fmaf(-w.y, x.x, pi[jj]));
        }
      }
#pragma unroll
      for (int jj = 0; jj < kSB; ++jj) {
        re[jj] += pr[jj];
        im[jj] += pi[jj];
      }
    }
    float* row = Xr + (int64_t)i * 2 * S;
#pragma unroll
    for (int jj = 0; jj < kSB; ++jj)
      if (jj < nj) {
        row[j0 + jj] = (float)re[jj];
        row[S + j0 + jj] = (float)im[jj];
      }
  }
}

// 2. Z_r = [Re; Im] of the sampled rows of the mixed Khatri-Rao product (FP64 products)
__global__ void k_cf_skr(CfArgs a, double* __restrict__ Zr) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int S = a.S, R = a.R;
  if (e >= (int64_t)S * R) return;
  const int j = (int)(e / R), r = (int)(e - (int64_t)j * R);
  double2 z = make_double2(1.0, 0.0);
  for (int m = 0; m < a.N; ++m) {
    if (m == a.n) continue;
    const float2 v = a.Ah[m][(int64_t)a.idx[(int64_t)j * a.N + m] * R + r];
    z = cmul64(z, make_double2((double)v.x, (double)v.y));
  }
  Zr[(int64_t)j * R + r] = z.x;
  Zr[(int64_t)(S + j) * R + r] = z.y;
}

// 3a. G = Z_r^T Z_r (R x R, FP64): one thread per entry of the upper triangle, mirrored
__global__ void k_cf_gram(const double* __restrict__ Zr, int rows, int R, double* __restrict__ G) {
  for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < R * R; e += gridDim.x * blockDim.x) {
    const int r = e / R, c = e - r * R;
    if (c < r) continue;
    double s0 = 0.0, s1 = 0.0;
    int j = 0;
    for (; j + 1 < rows; j += 2) {
      s0 = fma(Zr[(int64_t)j * R + r], Zr[(int64_t)j * R + c], s0);
      s1 = fma(Zr[(int64_t)(j + 1) * R + r], Zr[(int64_t)(j + 1) * R + c], s1);
    }
    if (j < rows) s0 = fma(Zr[(int64_t)j * R + r], Zr[(int64_t)j * R + c], s0);
    G[r * R + c] = s0 + s1;
    G[c * R + r] = s0 + s1;
  }
}

// 3b. M = X_r Z_r (I x R, FP64 accumulation): one thread per entry
__global__ void k_cf_contract(const float* __restrict__ Xr, const double* __restrict__ Zr, int I, int cols, int R,
                              double* __restrict__ M) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)I * R) return;
  const int i = (int)(e / R), r = (int)(e - (int64_t)i * R);
  const float* x = Xr + (int64_t)i * cols;
  double s0 = 0.0, s1 = 0.0;
  int j = 0;
  for (; j + 1 < cols; j += 2) {
    s0 = fma((double)x[j], Zr[(int64_t)j * R + r], s0);
    s1 = fma((double)x[j + 1], Zr[(int64_t)(j + 1) * R + r], s1);
  }
  if (j < cols) s0 = fma((double)x[j], Zr[(int64_t)j * R + r], s0);
  M[e] = s0 + s1;
}

// 4a. G^-1 (FP64 Cholesky inverse, one block); a singular Gram sets *bad
__global__ void k_cf_inverse(const double* __restrict__ Gg, int R, double* __restrict__ Xg, int* bad) {
  extern __shared__ double sh[];
  double* G = sh;
  double* X = G + R * R;
  double* Lw = X + R * R;
  double* Tm = Lw + R * R;
  double* dinv = Tm + R * R;
  __shared__ int s_bad;
  if (threadIdx.x == 0) s_bad = 0;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) G[e] = Gg[e];
  __syncthreads();
  spd_inverse_fp64(G, X, Lw, Tm, dinv, R, &s_bad);
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) Xg[e] = X[e];
  if (threadIdx.x == 0 && s_bad) atomicExch(bad, 1);
}

// 4b. A = M G^-1 (FP64), one thread per entry; per-block column sums of squares
__global__ void k_cf_apply(const double* __restrict__ M, const double* __restrict__ Gi, int I, int R,
                           double* __restrict__ A) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)I * R) return;
  const int i = (int)(e / R), r = (int)(e - (int64_t)i * R);
  const double* m = M + (int64_t)i * R;
  double s0 = 0.0, s1 = 0.0;
  int l = 0;
  for (; l + 1 < R; l += 2) {
    s0 = fma(m[l], Gi[l * R + r], s0);
    s1 = fma(m[l + 1], Gi[(l + 1) * R + r], s1);
  }
  if (l < R) s0 = fma(m[l], Gi[l * R + r], s0);
  A[e] = s0 + s1;
}

// 4c. column norms (fixed order over rows, one thread per column) and normalization: lam_r = ||a_r||,
// a zero column keeps weight 0 and stays as it is
__global__ void k_cf_normalize(double* __restrict__ A, int I, int R, double* __restrict__ lam) {
  __shared__ double s_inv[64];
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double s = 0.0;
    for (int i = 0; i < I; ++i) s = fma(A[(int64_t)i * R + r], A[(int64_t)i * R + r], s);
    const double nrm = sqrt(s);
    lam[r] = nrm;
    s_inv[r] = nrm > 0.0 ? 1.0 / nrm : 1.0;
  }
  __syncthreads();
  for (int64_t e = threadIdx.x; e < (int64_t)I * R; e += blockDim.x) A[e] *= s_inv[e % R];
}

struct CfFit {
  const double* A[kMaxOrder];   // real factors, I_m x R
  const double* lam;
  const uint32_t* idx;          // P_hat x N
  const double* x;              // P_hat values of the tensor
  int64_t dims[kMaxOrder];
  int N, R, P_hat;
};

// the fixed fit entries (the fit stream, as CPRAND) and their values in the real tensor
__global__ void k_cf_fit_setup(const float* __restrict__ X, CfFit f, uint64_t seed, uint32_t b, uint32_t* idx,
                               double* xv) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= f.P_hat) return;
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint4 w0 = philox10(make_uint4((uint32_t)j, counter_word1(kStreamFit, 0, 0), 0u, b), k0, k1);
  uint4 w1 = make_uint4(0u, 0u, 0u, 0u);
  if (f.N > 4) w1 = philox10(make_uint4((uint32_t)j, counter_word1(kStreamFit, 1, 0), 0u, b), k0, k1);
  int64_t off = 0, st = 1;
  for (int m = 0; m < f.N; ++m) {
    const uint32_t w = m < 4 ? word_of(w0, m) : word_of(w1, m - 4);
    const uint32_t im = scale_index(w, (uint32_t)f.dims[m]);
    idx[j * f.N + m] = im;
    off += (int64_t)im * st;
    st *= f.dims[m];
  }
  xv[j] = (double)X[off];
}

// squared model errors at the fit entries, one FP64 partial sum per block (fixed order)
__global__ void k_cf_fit(CfFit f, double* __restrict__ part) {
  __shared__ double red[256];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  double e2 = 0.0;
  if (j < f.P_hat) {
    double model = 0.0;
    for (int r = 0; r < f.R; ++r) {
      double t = f.lam[r];
      for (int m = 0; m < f.N; ++m) t *= f.A[m][(int64_t)f.idx[j * f.N + m] * f.R + r];
      model += t;
    }
    const double e = f.x[j] - model;
    e2 = e * e;
  }
  red[threadIdx.x] = e2;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

}  // namespace

cudaError_t launch_cf_ops(int I, const double* signs, float2* W, cudaStream_t s) {
  const int64_t n = (int64_t)I * I;
  k_cf_ops<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(I, signs, W);
  return cudaGetLastError();
}

cudaError_t launch_cf_init(int I, int R, int m, uint64_t seed, uint32_t b, double* A, cudaStream_t s) {
  const int64_t n = (int64_t)I * R;
  k_cf_init<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(I, R, m, seed, b, A);
  return cudaGetLastError();
}

cudaError_t launch_cf_mix_factor(int I, int R, const float2* W, const double* A, float2* Ah, cudaStream_t s) {
  const int64_t n = (int64_t)I * R;
  k_cf_mix_factor<<<(unsigned)((n + 127) / 128), 128, 0, s>>>(I, R, W, A, Ah);
  return cudaGetLastError();
}

// one mode-n update: A (I_n x R, FP64) and lam come out normalized, Ah[n] is not updated here
cudaError_t launch_cf_update(const float2* Xn, const uint32_t* idx, const float2* W, const float2* const* Ah,
                             int N, const int64_t* dims, int n, int S, int R, float* Xr, double* Zr, double* G,
                             double* Gi, double* M, double* A, double* lam, int* bad, cudaStream_t s) {
  CfArgs a;
  a.Xn = Xn;
  a.idx = idx;
  a.W = W;
  for (int m = 0; m < kMaxOrder; ++m) {
    a.Ah[m] = m < N ? Ah[m] : nullptr;
    a.dims[m] = m < N ? dims[m] : 1;
  }
  a.N = N;
  a.n = n;
  a.S = S;
  a.R = R;
  const int I = (int)dims[n];
  const size_t xs_bytes = (size_t)kSB * I * sizeof(float2);
  if (xs_bytes > 200 * 1024) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_cf_unmix_fibers, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  const unsigned gy = (unsigned)((I + 127) / 128);
  k_cf_unmix_fibers<<<dim3((unsigned)((S + kSB - 1) / kSB), gy), 128, xs_bytes, s>>>(a, Xr);
  k_cf_skr<<<(unsigned)(((int64_t)S * R + 255) / 256), 256, 0, s>>>(a, Zr);
  k_cf_gram<<<(unsigned)((R * R + 127) / 128), 128, 0, s>>>(Zr, 2 * S, R, G);
  k_cf_contract<<<(unsigned)(((int64_t)I * R + 127) / 128), 128, 0, s>>>(Xr, Zr, I, 2 * S, R, M);
  const size_t inv_bytes = (size_t)(4 * R * R + R) * sizeof(double);
  static bool attr2 = false;
  if (!attr2) {
    cudaError_t e = cudaFuncSetAttribute(k_cf_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr2 = true;
  }
  k_cf_inverse<<<1, 256, inv_bytes, s>>>(G, R, Gi, bad);
  k_cf_apply<<<(unsigned)(((int64_t)I * R + 127) / 128), 128, 0, s>>>(M, Gi, I, R, A);
  k_cf_normalize<<<1, 256, 0, s>>>(A, I, R, lam);
  return cudaGetLastError();
}

cudaError_t launch_cf_fit_setup(const float* X, int N, const int64_t* dims, int R, int P_hat, uint64_t seed,
                                uint32_t b, uint32_t* idx, double* xv, cudaStream_t s) {
  CfFit f{};
  for (int m = 0; m < kMaxOrder; ++m) f.dims[m] = m < N ? dims[m] : 1;
  f.N = N;
  f.R = R;
  f.P_hat = P_hat;
  k_cf_fit_setup<<<(unsigned)((P_hat + 255) / 256), 256, 0, s>>>(X, f, seed, b, idx, xv);
  return cudaGetLastError();
}

int cf_fit_blocks(int P_hat) { return (P_hat + 255) / 256; }

cudaError_t launch_cf_fit(const double* const* A, const double* lam, int N, const int64_t* dims, int R, int P_hat,
                          const uint32_t* idx, const double* xv, double* part, cudaStream_t s) {
  CfFit f{};
  for (int m = 0; m < kMaxOrder; ++m) {
    f.A[m] = m < N ? A[m] : nullptr;
    f.dims[m] = m < N ? dims[m] : 1;
  }
  f.lam = lam;
  f.idx = idx;
  f.x = xv;
  f.N = N;
  f.R = R;
  f.P_hat = P_hat;
  k_cf_fit<<<(unsigned)cf_fit_blocks(P_hat), 256, 0, s>>>(f, part);
  return cudaGetLastError();
}

}  // namespace cpr
