// Mixing preprocess and unmixing of CPRAND-MIX in its real-transform form (Alg. 5).
//
// Mode-n operator W_n = F_n D_n: D_n = diag of Philox signs (stream 3), F_n = orthonormal DCT-II,
//   F_n[i][k] = c_i cos(pi (2k+1) i / (2 I_n)), c_0 = sqrt(1/I_n), c_i = sqrt(2/I_n).
// The cosine argument is reduced exactly in integers ((2k+1) i mod 4 I_n) before cospi.
//
// Mode-n product Y = X x_n W_n on the column-major tensor, viewed as [L][I_n][Rr] with
// L = prod_{m<n} I_m (contiguous) and Rr = prod_{m>n} I_m:
//   mode 1 (L = 1):  Y[:, r] = W X[:, r]          -> rows of the GEMM are the Rr fibers (k contiguous)
//   mode n > 1:      Y_r[l][i] = sum_k X_r[l][k] W[i][k]  (batched over r, l contiguous)
// Both are one register-tiled SIMT GEMM (128 x 64 output tile, 8 x 4 per thread, FP32
// accumulation; FP64 for FP64 tensors).  Unmixing A = D_n F_n^T A^ runs in FP64.
#include <math.h>

#include "internal.cuh"

namespace cpr {

// cos(pi q / (2 I)) for q in [0, 4I): every entry of F_n is c_i times one of these, with
// q = (2k+1) i mod 4I (exact integer reduction).  FP64 cospi is called 4I times per mode, not I^2.
__global__ void k_cos_table(int I, double* table) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q < 4 * I) table[q] = cospi((double)q / (2.0 * I));
}

// fft_tab (5 I floats, or null): the tables of the factored transform, from the same cosine table:
// twiddles exp(-2 pi i t / I) = (cos, -sin)(2 pi t / I), post-scales c_k (cos, sin)(pi k / (2I)) / 2,
// the signs; sin(pi x / (2I)) is read as cos(pi (I - x) / (2I)) (cosine even for negative I - x)
__global__ void k_build_mix_ops(int I, uint64_t seed, uint32_t b, int n, const double* __restrict__ table,
                                float* W32, double* W64, double* F64, double* signs, float* fft_tab) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= (int64_t)I * I) return;
  const int i = (int)(e / I), k = (int)(e % I);
  const uint32_t k0 = (uint32_t)seed, k1 = (uint32_t)(seed >> 32);
  const uint4 w = philox10(make_uint4((uint32_t)k, counter_word1(kStreamSigns, 0, n), 0u, b), k0, k1);
  const double d = (w.x & 1u) ? -1.0 : 1.0;
  const int64_t q = ((int64_t)(2 * k + 1) * i) % (4 * (int64_t)I);
  const double c = (i == 0) ? sqrt(1.0 / I) : sqrt(2.0 / I);
  const double f = c * table[q];
  if (F64) F64[e] = f;
  if (W64) W64[e] = f * d;
  if (W32) W32[e] = (float)(f * d);
  if (signs && i == 0) signs[k] = d;
  if (fft_tab && i == 0) {   // entry t = k of the tables
    const int t = k;
    fft_tab[2 * t] = (float)table[4 * t];
    fft_tab[2 * t + 1] = (float)(-table[abs(I - 4 * t)]);
    const double ck = t == 0 ? sqrt(1.0 / I) : sqrt(2.0 / I);
    fft_tab[2 * I + 2 * t] = (float)(0.5 * ck * table[t]);
    fft_tab[2 * I + 2 * t + 1] = (float)(0.5 * ck * table[I - t]);
    fft_tab[4 * I + t] = (float)d;
  }
}

cudaError_t launch_build_mix_ops(int I, uint64_t seed, uint32_t b, int n, double* table, float* W32, double* W64,
                                 double* F64, double* signs, cudaStream_t s, float* fft_tab) {
  k_cos_table<<<(4 * I + 255) / 256, 256, 0, s>>>(I, table);
  const int64_t total = (int64_t)I * I;
  k_build_mix_ops<<<(unsigned)((total + 255) / 256), 256, 0, s>>>(I, seed, b, n, table, W32, W64, F64, signs, fft_tab);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess && fft_tab) e = launch_build_bs_tables(I, fft_tab, s);
  return e;
}

template <typename T> struct Conv;
template <> struct Conv<double> {
  static __device__ __forceinline__ double in(double v) { return v; }
  static __device__ __forceinline__ double out(double v) { return v; }
};
template <> struct Conv<float> {
  static __device__ __forceinline__ float in(float v) { return v; }
  static __device__ __forceinline__ float out(float v) { return v; }
};
template <> struct Conv<__nv_bfloat16> {
  static __device__ __forceinline__ float in(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ __nv_bfloat16 out(float v) { return __float2bfloat16(v); }
};

template <typename T, typename ACC, bool KC>
__global__ void __launch_bounds__(256) k_mix_mode(const T* __restrict__ X, T* __restrict__ Y,
                                                  const ACC* __restrict__ W, int64_t Mdim, int I, int64_t L,
                                                  int64_t nbatch) {
  constexpr int BM = 128, BC = 64, BK = 16;
  __shared__ ACC As[BK][BM + 4];
  __shared__ ACC Ws[BK][BC + 4];
  const int tid = threadIdx.x, tm = tid & 15, tc = tid >> 4;
  const int64_t m0 = (int64_t)blockIdx.x * BM;
  const int c0 = blockIdx.y * BC;
  for (int64_t bz = blockIdx.z; bz < nbatch; bz += gridDim.z) {
    const int64_t base = KC ? 0 : bz * L * I;
    ACC acc[8][4];
#pragma unroll
    for (int x = 0; x < 8; ++x)
#pragma unroll
      for (int y = 0; y < 4; ++y) acc[x][y] = ACC(0);
    for (int k0 = 0; k0 < I; k0 += BK) {
      if (KC) {
        const int kk = tid & 15;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int mm = (tid >> 4) + 16 * q;
          const int64_t m = m0 + mm;
          const int k = k0 + kk;
          As[kk][mm] = (m < Mdim && k < I) ? (ACC)Conv<T>::in(X[m * I + k]) : ACC(0);
        }
      } else {
        const int mm = tid & 127;
#pragma unroll
        for (int q = 0; q < 8; ++q) {
          const int kk = (tid >> 7) + 2 * q;
          const int64_t m = m0 + mm;
          const int k = k0 + kk;
          As[kk][mm] = (m < Mdim && k < I) ? (ACC)Conv<T>::in(X[base + m + (int64_t)k * L]) : ACC(0);
        }
      }
      {
        const int kk = tid & 15;
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int cc = (tid >> 4) + 16 * q;
          const int c = c0 + cc, k = k0 + kk;
          Ws[kk][cc] = (c < I && k < I) ? W[(int64_t)c * I + k] : ACC(0);
        }
      }
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < BK; ++kk) {
        ACC a[8], w[4];
#pragma unroll
        for (int x = 0; x < 8; ++x) a[x] = As[kk][tm * 8 + x];
#pragma unroll
        for (int y = 0; y < 4; ++y) w[y] = Ws[kk][tc * 4 + y];
#pragma unroll
        for (int x = 0; x < 8; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) acc[x][y] = fma(a[x], w[y], acc[x][y]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int x = 0; x < 8; ++x) {
      const int64_t m = m0 + tm * 8 + x;
      if (m >= Mdim) continue;
#pragma unroll
      for (int y = 0; y < 4; ++y) {
        const int c = c0 + tc * 4 + y;
        if (c >= I) continue;
        if (KC) Y[m * I + c] = Conv<T>::out(acc[x][y]);
        else Y[base + m + (int64_t)c * L] = Conv<T>::out(acc[x][y]);
      }
    }
  }
}

template <typename T, typename ACC>
static cudaError_t mix_dispatch(const void* X, void* Y, const ACC* W, int N, const int64_t* dims, int n,
                                cudaStream_t s) {
  int64_t L = 1, Rr = 1;
  for (int m = 0; m < n; ++m) L *= dims[m];
  for (int m = n + 1; m < N; ++m) Rr *= dims[m];
  const int I = (int)dims[n];
  const int cblocks = (I + 63) / 64;
  if (n == 0) {
    const int64_t Mdim = Rr;
    const dim3 grid((unsigned)((Mdim + 127) / 128), cblocks, 1);
    k_mix_mode<T, ACC, true><<<grid, 256, 0, s>>>((const T*)X, (T*)Y, W, Mdim, I, 1, 1);
  } else {
    const int64_t nz = Rr < 65535 ? Rr : 65535;
    const dim3 grid((unsigned)((L + 127) / 128), cblocks, (unsigned)nz);
    k_mix_mode<T, ACC, false><<<grid, 256, 0, s>>>((const T*)X, (T*)Y, W, L, I, L, Rr);
  }
  return cudaGetLastError();
}

cudaError_t launch_mix_mode(const void* X, void* Y, int dtype, int N, const int64_t* dims, int n, const float* W32,
                            const double* W64, cudaStream_t s) {
  switch (dtype) {
    case CPR_F64: return mix_dispatch<double, double>(X, Y, W64, N, dims, n, s);
    case CPR_F32: return mix_dispatch<float, float>(X, Y, W32, N, dims, n, s);
    default: return mix_dispatch<__nv_bfloat16, float>(X, Y, W32, N, dims, n, s);
  }
}

// Mode-n unfolding X_(n) stored column-major: with X viewed as [L][I_n][Rr] (L = prod_{m<n} I_m
// fastest), Y[i + I_n (l + L r)] = X[l + L (i + I_n r)].  Column j = l + L r of X_(n) is the mode-n
// fiber with unfolding index j (the index map of Sec. 2.1), contiguous in Y.  64 x 64 tiles through
// shared memory, 256 threads: every thread issues its 16 loads (coalesced along l) before its first
// store (coalesced along i), so a block keeps 16 KB of reads in flight.
template <typename T>
__global__ void __launch_bounds__(256, 4) k_unfold_copy(const T* __restrict__ X, T* __restrict__ Y, int64_t L,
                                                        int64_t I, int64_t Rr) {
  __shared__ T tile[64][65];
  const int lane = threadIdx.x & 31, wy = threadIdx.x >> 5;   // 32 lanes x 8 warps
  const int64_t l0 = (int64_t)blockIdx.x * 64, i0 = (int64_t)blockIdx.y * 64;
  const int nl = (int)(L - l0 < 64 ? L - l0 : 64), ni = (int)(I - i0 < 64 ? I - i0 : 64);   // tile extents
  for (int64_t r = blockIdx.z; r < Rr; r += gridDim.z) {
    const T* src = X + r * L * I + l0 + i0 * L;   // tile origin in X (l fastest)
    T* dst = Y + r * L * I + i0 + l0 * I;         // tile origin in Y (i fastest)
    T v[16];
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int i = wy + 8 * k;
      const T* row = src + (int64_t)i * L;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int l = lane + 32 * h;
        v[2 * k + h] = (l < nl && i < ni) ? row[l] : T(0);
      }
    }
#pragma unroll
    for (int k = 0; k < 8; ++k)
#pragma unroll
      for (int h = 0; h < 2; ++h) tile[wy + 8 * k][lane + 32 * h] = v[2 * k + h];
    __syncthreads();
#pragma unroll
    for (int k = 0; k < 8; ++k) {
      const int l = wy + 8 * k;
      T* col = dst + (int64_t)l * I;
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int i = lane + 32 * h;
        if (l < nl && i < ni) col[i] = tile[i][l];
      }
    }
    __syncthreads();
  }
}

cudaError_t launch_unfold_copy(const void* X, void* Y, int dtype, int N, const int64_t* dims, int n, cudaStream_t s) {
  int64_t L = 1, Rr = 1;
  for (int m = 0; m < n; ++m) L *= dims[m];
  for (int m = n + 1; m < N; ++m) Rr *= dims[m];
  const int64_t I = dims[n];
  const dim3 grid((unsigned)((L + 63) / 64), (unsigned)((I + 63) / 64), (unsigned)(Rr < 65535 ? Rr : 65535));
  switch (dtype) {
    case CPR_F64: k_unfold_copy<double><<<grid, 256, 0, s>>>((const double*)X, (double*)Y, L, I, Rr); break;
    case CPR_F32: k_unfold_copy<float><<<grid, 256, 0, s>>>((const float*)X, (float*)Y, L, I, Rr); break;
    default:
      k_unfold_copy<unsigned short><<<grid, 256, 0, s>>>((const unsigned short*)X, (unsigned short*)Y, L, I, Rr);
  }
  return cudaGetLastError();
}

// A = D F^T A^ in FP64 (Alg. 5, unmixing) for every mode in one launch.  FP64 arithmetic bounds it,
// so the work is spread over the whole GPU: a block computes 8 rows i of one mode's A (8R outputs);
// chunks of 32 k of F (8 consecutive entries of each row k: 64 contiguous bytes) and of A^ (R
// contiguous entries per row) are staged in shared memory; each output's sum over k is split over
// ks threads (a power of two) whose partials are combined by a fixed butterfly of shuffles.
constexpr int kUnmixRows = 8, kUnmixK = 32;
__global__ void __launch_bounds__(256) k_unmix(UnmixArgs u) {
  __shared__ double Fc[kUnmixK][kUnmixRows];
  __shared__ double Ac[kUnmixK][kMaxRank];
  int n = 0;
  while (n + 1 < u.N && (int)blockIdx.x >= u.first_block[n + 1]) ++n;
  const int I = u.I[n], R = u.R;
  const int i0 = ((int)blockIdx.x - u.first_block[n]) * kUnmixRows;
  const double* __restrict__ F = u.F[n];
  const double* __restrict__ Ah = u.Ahat[n];
  const int nout = kUnmixRows * R;   // up to 512: two output groups of blockDim.x / ks
  int ks = 1;
  while (ks < 32 && ks * 2 * nout <= (int)blockDim.x) ks *= 2;
  const int t = threadIdx.x, s = t % ks, og = (int)blockDim.x / ks;
  double a0[2] = {0.0, 0.0}, a1[2] = {0.0, 0.0};
  for (int k0 = 0; k0 < I; k0 += kUnmixK) {
    const int kc = min(kUnmixK, I - k0);
    for (int e = t; e < kUnmixK * kUnmixRows; e += blockDim.x) {
      const int kk = e / kUnmixRows, q = e - kk * kUnmixRows;
      Fc[kk][q] = (kk < kc && i0 + q < I) ? F[(int64_t)(k0 + kk) * I + i0 + q] : 0.0;
    }
    for (int e = t; e < kc * R; e += blockDim.x) {
      const int kk = e / R, c = e - kk * R;
      Ac[kk][c] = Ah[(int64_t)(k0 + kk) * R + c];
    }
    __syncthreads();
#pragma unroll
    for (int g = 0; g < 2; ++g) {
      const int o = t / ks + g * og;
      if (o < nout) {
        const int ii = o / R, r = o - ii * R;
        int kk = s;
        for (; kk + ks < kc; kk += 2 * ks) {
          a0[g] = fma(Fc[kk][ii], Ac[kk][r], a0[g]);
          a1[g] = fma(Fc[kk + ks][ii], Ac[kk + ks][r], a1[g]);
        }
        if (kk < kc) a0[g] = fma(Fc[kk][ii], Ac[kk][r], a0[g]);
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int g = 0; g < 2; ++g) {
    const int o = t / ks + g * og;
    double acc = a0[g] + a1[g];
    for (int w = 1; w < ks; w <<= 1) acc += __shfl_xor_sync(0xffffffffu, acc, w);
    if (o < nout && s == 0) {
      const int ii = o / R, r = o - ii * R, i = i0 + ii;
      if (i < I) u.A[n][(int64_t)i * R + r] = u.sg[n][i] * acc;
    }
  }
}

cudaError_t launch_unmix_all(const UnmixArgs& u_in, cudaStream_t s) {
  UnmixArgs u = u_in;
  int blocks = 0;
  for (int n = 0; n < u.N; ++n) {
    u.first_block[n] = blocks;
    blocks += (u.I[n] + kUnmixRows - 1) / kUnmixRows;
  }
  if (blocks <= 0) return cudaSuccess;
  k_unmix<<<blocks, 256, 0, s>>>(u);
  return cudaGetLastError();
}

cudaError_t launch_unmix(const double* Ahat, double* A, const double* F64, const double* signs, int I, int R,
                         cudaStream_t s) {
  UnmixArgs u{};
  u.N = 1;
  u.R = R;
  u.Ahat[0] = Ahat;
  u.A[0] = A;
  u.F[0] = F64;
  u.sg[0] = signs;
  u.I[0] = I;
  return launch_unmix_all(u, s);
}

}  // namespace cpr
