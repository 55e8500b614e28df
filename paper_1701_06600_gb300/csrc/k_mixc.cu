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

constexpr int kSB = 4;    // sampled fibers per block of the unmixing kernel

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

// A^^ = W A (I x R complex): one warp per entry, the lanes split the sum over i (FP32 products and
// per-lane sums, a fixed-order shuffle tree in FP64)
__global__ void k_cf_mix_factor(int I, int R, const float2* __restrict__ W, const double* __restrict__ A,
                                float2* __restrict__ Ah) {
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= (int64_t)I * R) return;   // whole warps
  const int k = (int)(e / R), r = (int)(e - (int64_t)k * R);
  const float2* w = W + (int64_t)k * I;
  float pr = 0.f, pi = 0.f;
  for (int i = lane; i < I; i += 32) {
    const float av = (float)A[(int64_t)i * R + r];
    pr = fmaf(w[i].x, av, pr);
    pi = fmaf(w[i].y, av, pi);
  }
  double re = pr, im = pi;
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) Ah[e] = make_float2((float)re, (float)im);
}

struct CfArgs {
  const float2* Xn;        // the mixed tensor's mode-n unfolding copy (fibers of I_n complex values)
  const uint32_t* idx;     // S x N sampled multi-indices
  const float2* W;         // W_n, I_n x I_n
  const float2* Ah[kMaxOrder];   // mixed factors, I_m x R
  int64_t dims[kMaxOrder];
  int N, n, S, R;
};

// 1. X_r = [Re, Im](W_n^H X^_S): a block of 32 x kSB threads unmixes kSB sampled fibers (staged in
// shared memory) for 32 consecutive rows i, one output per thread (FP32 products over 32-term chunks,
// the chunks summed in FP64)
__global__ void k_cf_unmix_fibers(CfArgs a, float* __restrict__ Xr) {
  extern __shared__ float2 xs[];   // kSB x I
  __shared__ int64_t col[kSB];
  const int I = (int)a.dims[a.n], S = a.S;
  const int j0 = blockIdx.x * kSB, nj = min(kSB, S - j0);
  const int t = threadIdx.y * 32 + threadIdx.x, nt = 32 * kSB;
  if (t < nj) {   // column of the mode-n unfolding holding fiber j0 + t (index map of §2.1)
    const uint32_t* id = a.idx + (int64_t)(j0 + t) * a.N;
    int64_t c = 0, J = 1;
    for (int m = 0; m < a.N; ++m) {
      if (m == a.n) continue;
      c += (int64_t)id[m] * J;
      J *= a.dims[m];
    }
    col[t] = c;
  }
  __syncthreads();
  for (int e = t; e < nj * I; e += nt) {
    const int jj = e / I, k = e - jj * I;
    xs[e] = a.Xn[col[jj] * I + k];
  }
  __syncthreads();
  const int i = blockIdx.y * 32 + threadIdx.x, jj = threadIdx.y;
  if (i >= I || jj >= nj) return;
  const float2* x = xs + jj * I;
  double re = 0.0, im = 0.0;
  for (int k0 = 0; k0 < I; k0 += 32) {
    float pr = 0.f, pi = 0.f;
    for (int k = k0; k < min(I, k0 + 32); ++k) {
      const float2 w = a.W[(int64_t)k * I + i];   // conj(W[k][i]) = (w.x, -w.y)
      const float2 v = x[k];
      pr = fmaf(w.x, v.x, fmaf(w.y, v.y, pr));
      pi = fmaf(w.x, v.y, fmaf(-w.y, v.x, pi));
    }
    re += pr;
    im += pi;
  }
  float* row = Xr + (int64_t)i * 2 * S;
  row[j0 + jj] = (float)re;
  row[S + j0 + jj] = (float)im;
}

// 2. Z_r = [Re; Im] of the sampled rows of the mixed Khatri-Rao product (FP64 products; an FP32 copy
// for the contraction)
__global__ void k_cf_skr(CfArgs a, double* __restrict__ Zr, float* __restrict__ Zf) {
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
  Zf[(int64_t)j * R + r] = (float)z.x;
  Zf[(int64_t)(S + j) * R + r] = (float)z.y;
}

// 3a. G = Z_r^T Z_r (R x R, FP64): one block per entry of the upper triangle (its 2S products split
// over the threads, then a fixed-order tree), mirrored
__global__ void k_cf_gram(const double* __restrict__ Zr, int rows, int R, double* __restrict__ G) {
  __shared__ double red[128];
  const int e = blockIdx.x, r = e / R, c = e - r * R;
  if (c < r) return;
  double a = 0.0;
  for (int j = threadIdx.x; j < rows; j += blockDim.x) a = fma(Zr[(int64_t)j * R + r], Zr[(int64_t)j * R + c], a);
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = 64; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    G[r * R + c] = red[0];
    G[c * R + r] = red[0];
  }
}

// 3b. M = X_r Z_r (I x R): one warp per entry, the lanes split the sum over the 2S rows (FP32
// products and per-lane sums, the contraction's accumulation type as in the real form; a fixed-order
// shuffle tree in FP64)
__global__ void k_cf_contract(const float* __restrict__ Xr, const float* __restrict__ Zf, int I, int cols, int R,
                              double* __restrict__ M) {
  const int64_t e = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int lane = threadIdx.x & 31;
  if (e >= (int64_t)I * R) return;   // whole warps
  const int i = (int)(e / R), r = (int)(e - (int64_t)i * R);
  const float* x = Xr + (int64_t)i * cols;
  float s0 = 0.f;
  for (int j = lane; j < cols; j += 32) s0 = fmaf(x[j], Zf[(int64_t)j * R + r], s0);
  double a = s0;
  for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
  if (lane == 0) M[e] = a;
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

// 4c. column norms and normalization, one block per column (fixed-order tree over the rows):
// lam_r = ||a_r||; a zero column keeps weight 0 and stays as it is
__global__ void k_cf_normalize(double* __restrict__ A, int I, int R, double* __restrict__ lam) {
  __shared__ double red[256];
  const int r = blockIdx.x;
  double a = 0.0;
  for (int i = threadIdx.x; i < I; i += blockDim.x) a = fma(A[(int64_t)i * R + r], A[(int64_t)i * R + r], a);
  red[threadIdx.x] = a;
  __syncthreads();
  for (int o = 128; o > 0; o >>= 1) {
    if (threadIdx.x < o) red[threadIdx.x] += red[threadIdx.x + o];
    __syncthreads();
  }
  const double nrm = sqrt(red[0]);
  if (threadIdx.x == 0) lam[r] = nrm;
  const double inv = nrm > 0.0 ? 1.0 / nrm : 1.0;
  for (int i = threadIdx.x; i < I; i += blockDim.x) A[(int64_t)i * R + r] *= inv;
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
  k_cf_mix_factor<<<(unsigned)((n * 32 + 255) / 256), 256, 0, s>>>(I, R, W, A, Ah);
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
  k_cf_unmix_fibers<<<dim3((unsigned)((S + kSB - 1) / kSB), (unsigned)((I + 31) / 32)), dim3(32, kSB), xs_bytes, s>>>(
      a, Xr);
  float* Zf = reinterpret_cast<float*>(Zr + (int64_t)2 * S * R);   // the FP32 copy after the FP64 one
  k_cf_skr<<<(unsigned)(((int64_t)S * R + 255) / 256), 256, 0, s>>>(a, Zr, Zf);
  k_cf_gram<<<(unsigned)(R * R), 128, 0, s>>>(Zr, 2 * S, R, G);
  k_cf_contract<<<(unsigned)(((int64_t)I * R * 32 + 255) / 256), 256, 0, s>>>(Xr, Zf, I, 2 * S, R, M);
  const size_t inv_bytes = (size_t)(4 * R * R + R) * sizeof(double);
  static bool attr2 = false;
  if (!attr2) {
    cudaError_t e = cudaFuncSetAttribute(k_cf_inverse, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024);
    if (e != cudaSuccess) return e;
    attr2 = true;
  }
  k_cf_inverse<<<1, 256, inv_bytes, s>>>(G, R, Gi, bad);
  k_cf_apply<<<(unsigned)(((int64_t)I * R + 127) / 128), 128, 0, s>>>(M, Gi, I, R, A);
  k_cf_normalize<<<(unsigned)R, 256, 0, s>>>(A, I, R, lam);
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
