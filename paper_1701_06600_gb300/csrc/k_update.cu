// Kernels of one mode-n update of CPRAND (Alg. 3, with Alg. 2 for the sampled Khatri-Rao rows).
//
// Per mode n, for every problem of the batch:
//   k_sample_skr_gram   draw S multi-indices (Philox), fiber base offsets, Z_S rows (Alg. 2) and a
//                       partial FP64 Gram Z_S^T Z_S over a chunk of kGramChunk samples
//   k_gather_contract   M = X_S Z_S: each thread owns one fiber row i_n and streams the sampled
//                       fibers of its split, FP32 accumulation (FP64 for FP64 tensors)
//   k_gram_chol         sum the partial Grams (fixed order) and Cholesky-factor G = L L^T in FP64
//   k_solve_rows        sum the partial M rows, solve a G = m per row with L (FP64), column sums of
//                       squares for the normalization
//   k_normalize         lambda_r = column 2-norm, columns scaled to unit length (FP64 + FP32 copy)
// All reductions run in a fixed order, so a run is bitwise reproducible.
#include <math.h>

#include "internal.cuh"

namespace cpr {

__global__ void k_init_state(const Prob* probs, int B) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  State* s = probs[b].state;
  s->iter = 0;
  s->done = 0;
  s->status = CPR_OK;
  s->stall = 0;
  s->best = -INFINITY;
  s->last_fit = NAN;
}

cudaError_t launch_init_state(const Prob* probs, int B, cudaStream_t s) {
  k_init_state<<<(B + 127) / 128, 128, 0, s>>>(probs, B);
  return cudaGetLastError();
}

// Random initial factors (Philox stream 2, U[0,1)) for modes 2..N, lambda = 1; or, with from_a64,
// the FP32 working copy of caller-given FP64 factors of every mode.
__global__ void k_init_factors(const Prob* probs, int from_a64) {
  const Prob& p = probs[blockIdx.y];
  const int R = p.R;
  const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  for (int n = 0; n < p.N; ++n) {
    if (!from_a64 && n == 0) continue;
    const int64_t cnt = p.dims[n] * R;
    for (int64_t e = tid; e < cnt; e += stride) {
      double v;
      if (from_a64) {
        v = p.A64[n][e];
      } else {
        const uint32_t i = (uint32_t)(e / R), r = (uint32_t)(e % R);
        const uint4 w = philox10(make_uint4(i, counter_word1(kStreamInit, 0, n), r / 4, p.b), k0, k1);
        v = (double)(word_of(w, r % 4) >> 8) * (1.0 / 16777216.0);
        p.A64[n][e] = v;
      }
      p.A32[n][e] = (float)v;
    }
  }
  if (!from_a64 && blockIdx.x == 0)
    for (int r = threadIdx.x; r < R; r += blockDim.x) p.lambda[r] = 1.0;
}

cudaError_t launch_init_factors(const Prob* probs, const GridInfo& g, int from_a64, cudaStream_t s) {
  int64_t most = 0;
  for (int n = 0; n < kMaxOrder; ++n) most = most > g.max_I[n] ? most : g.max_I[n];
  int64_t blocks = (most * g.max_R + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 1024) blocks = 1024;
  k_init_factors<<<dim3((unsigned)blocks, g.B), 256, 0, s>>>(probs, from_a64);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Sampling + SKR + partial Gram.  One block = kGramChunk samples of one problem.
// Sample j of mode n in outer iteration t: counter (j, (0<<8)|(blk<<4)|n, t, b); the k-th mode
// other than n takes word k%4 of block k/4; i_m = floor(w * I_m / 2^32).
// ------------------------------------------------------------------------------------------------
template <bool F64>
__global__ void __launch_bounds__(128) k_sample_skr_gram(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.y];
  if (n >= p.N || is_done(p)) return;
  const int S = p.S, R = p.R, N = p.N;
  const int j0 = blockIdx.x * kGramChunk;
  if (j0 >= S) return;
  const int cnt = min(kGramChunk, S - j0);
  __shared__ uint32_t ids[kGramChunk][kMaxOrder];
  extern __shared__ double Zs[];  // cnt x R
  const uint32_t t = p.t0 + (uint32_t)p.state->iter;
  const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
  const int tid = threadIdx.x;
  if (tid < cnt) {
    const uint32_t j = (uint32_t)(j0 + tid);
    const uint4 w0 = philox10(make_uint4(j, counter_word1(kStreamSamples, 0, n), t, p.b), k0, k1);
    uint4 w1 = make_uint4(0u, 0u, 0u, 0u);
    if (N - 1 > 4) w1 = philox10(make_uint4(j, counter_word1(kStreamSamples, 1, n), t, p.b), k0, k1);
    int64_t off = 0;
    int k = 0;
    for (int m = 0; m < N; ++m) {
      uint32_t im = 0;
      if (m != n) {
        const uint32_t w = k < 4 ? word_of(w0, k) : word_of(w1, k - 4);
        im = scale_index(w, (uint32_t)p.dims[m]);
        off += (int64_t)im * p.st[m];
        ++k;
      }
      ids[tid][m] = im;
      p.idx[(int64_t)j * N + m] = im;
    }
    p.off[j] = off;
  }
  __syncthreads();
  for (int e = tid; e < cnt * R; e += blockDim.x) {
    const int jj = e / R, r = e - jj * R;
    double z = 1.0;
    for (int m = 0; m < N; ++m) {
      if (m == n) continue;
      const int64_t a = (int64_t)ids[jj][m] * R + r;
      z *= F64 ? p.A64[m][a] : (double)p.A32[m][a];
    }
    Zs[e] = z;
    const int64_t gidx = (int64_t)j0 * R + e;
    if (F64) p.Z64[gidx] = z; else p.Z32[gidx] = (float)z;
  }
  __syncthreads();
  double* Gp = p.Gpart + (int64_t)blockIdx.x * R * R;
  for (int e = tid; e < R * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    if (c < r) continue;
    double acc = 0.0;
    for (int jj = 0; jj < cnt; ++jj) acc = fma(Zs[jj * R + r], Zs[jj * R + c], acc);
    Gp[e] = acc;
  }
}

cudaError_t launch_sample_skr_gram(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  const size_t smem = (size_t)kGramChunk * g.max_R * sizeof(double);
  if (g.any_f64)
    k_sample_skr_gram<true><<<dim3(g.max_ng, g.B), 128, smem, s>>>(probs, n);
  else
    k_sample_skr_gram<false><<<dim3(g.max_ng, g.B), 128, smem, s>>>(probs, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Fiber gather fused with the contraction M = X_S Z_S (Sec. 3.2; Alg. 3 lines building Z_S and
// X_S^T, cost Sec. 3.2.1).  Block = kContractRows consecutive rows i_n of one sample split; each
// thread keeps its row of R accumulators in registers; Z rows and offsets of the split sit in
// shared memory and are read as broadcasts.  Mode 1 fibers are contiguous (coalesced); other modes
// read one element per sector.
// ------------------------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ float to_acc_f(T v);
template <> __device__ __forceinline__ float to_acc_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_acc_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename T, typename ACC, int MAXR>
__global__ void __launch_bounds__(kContractRows) k_gather_contract(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.y];
  if (n >= p.N || is_done(p)) return;
  const int R = p.R, S = p.S;
  const int64_t I = p.dims[n];
  const int ntile = (int)((I + kContractRows - 1) / kContractRows);
  const int tile = blockIdx.x % ntile, split = blockIdx.x / ntile;
  if (split >= p.nsplit) return;
  const int js = split * p.spl;
  const int cnt = min(p.spl, S - js);
  if (cnt <= 0) return;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  int64_t* offs = reinterpret_cast<int64_t*>(smem_raw);
  ACC* Zs = reinterpret_cast<ACC*>(smem_raw + (((size_t)p.spl * sizeof(int64_t) + 15) & ~(size_t)15));
  for (int e = threadIdx.x; e < cnt; e += blockDim.x) offs[e] = p.off[js + e];
  for (int e = threadIdx.x; e < cnt * R; e += blockDim.x) {
    if constexpr (sizeof(ACC) == 8) Zs[e] = p.Z64[(int64_t)js * R + e];
    else Zs[e] = p.Z32[(int64_t)js * R + e];
  }
  __syncthreads();
  const int64_t i = (int64_t)tile * kContractRows + threadIdx.x;
  if (i >= I) return;
  const T* __restrict__ X = reinterpret_cast<const T*>(p.X);
  const int64_t sti = i * p.st[n];
  ACC acc[MAXR];
#pragma unroll
  for (int r = 0; r < MAXR; ++r) acc[r] = ACC(0);
  int j = 0;
  for (; j + 8 <= cnt; j += 8) {
    ACC x[8];
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      if constexpr (sizeof(ACC) == 8) x[q] = (ACC)__ldg(&X[offs[j + q] + sti]);
      else x[q] = to_acc_f<T>(X[offs[j + q] + sti]);
    }
#pragma unroll
    for (int q = 0; q < 8; ++q) {
      const ACC* z = Zs + (j + q) * R;
#pragma unroll
      for (int r = 0; r < MAXR; ++r)
        if (r < R) acc[r] = fma(x[q], z[r], acc[r]);
    }
  }
  for (; j < cnt; ++j) {
    ACC x;
    if constexpr (sizeof(ACC) == 8) x = (ACC)__ldg(&X[offs[j] + sti]);
    else x = to_acc_f<T>(X[offs[j] + sti]);
    const ACC* z = Zs + j * R;
#pragma unroll
    for (int r = 0; r < MAXR; ++r)
      if (r < R) acc[r] = fma(x, z[r], acc[r]);
  }
  ACC* M = reinterpret_cast<ACC*>(p.Mpart) + ((int64_t)split * p.imax + i) * R;
#pragma unroll
  for (int r = 0; r < MAXR; ++r)
    if (r < R) M[r] = acc[r];
}

template <typename T, typename ACC>
static cudaError_t dispatch_contract(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  const size_t smem = (((size_t)g.max_spl * sizeof(int64_t) + 15) & ~(size_t)15) +
                      (size_t)g.max_spl * g.max_R * sizeof(ACC);
  const dim3 grid(g.max_tiles_x_split[n], g.B);
  if (g.max_R <= 8) k_gather_contract<T, ACC, 8><<<grid, kContractRows, smem, s>>>(probs, n);
  else if (g.max_R <= 16) k_gather_contract<T, ACC, 16><<<grid, kContractRows, smem, s>>>(probs, n);
  else if (g.max_R <= 32) k_gather_contract<T, ACC, 32><<<grid, kContractRows, smem, s>>>(probs, n);
  else k_gather_contract<T, ACC, 64><<<grid, kContractRows, smem, s>>>(probs, n);
  return cudaGetLastError();
}

cudaError_t launch_gather_contract(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  if (g.max_tiles_x_split[n] <= 0) return cudaSuccess;
  switch (g.dtype) {
    case CPR_F64: return dispatch_contract<double, double>(probs, g, n, s);
    case CPR_F32: return dispatch_contract<float, float>(probs, g, n, s);
    default: return dispatch_contract<__nv_bfloat16, float>(probs, g, n, s);
  }
}

// ------------------------------------------------------------------------------------------------
// G = sum of partial Grams (fixed order), then Cholesky G = L L^T in FP64 (right-looking, in
// shared memory).  A pivot that is not positive (relative to the largest diagonal) marks the
// problem CPR_ESINGULAR and stops it.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(256) k_gram_chol(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.x];
  if (n >= p.N || is_done(p)) return;
  const int R = p.R;
  const int ng = (p.S + kGramChunk - 1) / kGramChunk;
  extern __shared__ double G[];  // R x R
  __shared__ int bad;
  __shared__ double maxdiag;
  const int tid = threadIdx.x;
  if (tid == 0) bad = 0;
  for (int e = tid; e < R * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    if (c < r) continue;
    double acc = 0.0;
    for (int q = 0; q < ng; ++q) acc += p.Gpart[(int64_t)q * R * R + e];
    G[r * R + c] = acc;
    G[c * R + r] = acc;
  }
  __syncthreads();
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
        bad = 1;
        d = 1.0;
      }
      G[k * R + k] = sqrt(d);
    }
    __syncthreads();
    const double dk = G[k * R + k];
    for (int i = k + 1 + tid; i < R; i += blockDim.x) G[i * R + k] /= dk;
    __syncthreads();
    const int rem = R - k - 1;
    for (int e = tid; e < rem * rem; e += blockDim.x) {
      const int i = k + 1 + e / rem, c = k + 1 + e % rem;
      if (c <= i) G[i * R + c] -= G[i * R + k] * G[c * R + k];
    }
    __syncthreads();
  }
  for (int e = tid; e < R * R; e += blockDim.x) p.L[e] = G[e];
  if (tid == 0 && bad) {
    p.state->status = CPR_ESINGULAR;
    p.state->done = 1;
  }
}

cudaError_t launch_gram_chol(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  k_gram_chol<<<g.B, 256, (size_t)g.max_R * g.max_R * sizeof(double), s>>>(probs, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Row solves: for each row i of the new factor, m_i = sum over splits of M rows, then
// a_i (L L^T) = m_i by a forward and a backward substitution in FP64.  Writes the unnormalized
// rows to A64[n] and this block's column sums of squares to Npart.
// ------------------------------------------------------------------------------------------------
template <typename ACC>
__global__ void __launch_bounds__(kSolveRows) k_solve_rows(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.y];
  if (n >= p.N || is_done(p)) return;
  const int R = p.R, R1 = R + 1;
  const int64_t I = p.dims[n];
  const int64_t i0 = (int64_t)blockIdx.x * kSolveRows;
  if (i0 >= I) return;
  const int rows = (int)min((int64_t)kSolveRows, I - i0);
  extern __shared__ double sm[];
  double* Ls = sm;             // R x (R+1)
  double* V = sm + R * R1;     // kSolveRows x (R+1)
  const int tid = threadIdx.x;
  for (int e = tid; e < R * R; e += blockDim.x) Ls[(e / R) * R1 + e % R] = p.L[e];
  const ACC* Mp = reinterpret_cast<const ACC*>(p.Mpart);
  for (int e = tid; e < rows * R; e += blockDim.x) {
    const int li = e / R, r = e - li * R;
    double acc = 0.0;
    for (int q = 0; q < p.nsplit; ++q) acc += (double)Mp[((int64_t)q * p.imax + i0 + li) * R + r];
    V[li * R1 + r] = acc;
  }
  __syncthreads();
  if (tid < rows) {
    double* v = V + tid * R1;
    for (int k = 0; k < R; ++k) {
      double s = v[k];
      for (int l = 0; l < k; ++l) s -= Ls[k * R1 + l] * v[l];
      v[k] = s / Ls[k * R1 + k];
    }
    for (int k = R - 1; k >= 0; --k) {
      double s = v[k];
      for (int l = k + 1; l < R; ++l) s -= Ls[l * R1 + k] * v[l];
      v[k] = s / Ls[k * R1 + k];
    }
  }
  __syncthreads();
  double* A = p.A64[n] + i0 * R;
  for (int e = tid; e < rows * R; e += blockDim.x) A[e] = V[(e / R) * R1 + e % R];
  for (int r = tid; r < R; r += blockDim.x) {
    double s = 0.0;
    for (int li = 0; li < rows; ++li) {
      const double v = V[li * R1 + r];
      s += v * v;
    }
    p.Npart[(int64_t)blockIdx.x * R + r] = s;
  }
}

cudaError_t launch_solve_rows(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  const size_t smem = ((size_t)g.max_R * (g.max_R + 1) + (size_t)kSolveRows * (g.max_R + 1)) * sizeof(double);
  const dim3 grid((g.max_I[n] + kSolveRows - 1) / kSolveRows, g.B);
  if (g.dtype == CPR_F64) {
    cudaFuncSetAttribute(k_solve_rows<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_solve_rows<double><<<grid, kSolveRows, smem, s>>>(probs, n);
  } else {
    cudaFuncSetAttribute(k_solve_rows<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_solve_rows<float><<<grid, kSolveRows, smem, s>>>(probs, n);
  }
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Normalization (Alg. 3 last step): lambda_r = ||a_r||_2 (FP64), columns scaled to unit length;
// a zero column keeps lambda_r = 0 and is left unchanged.
// ------------------------------------------------------------------------------------------------
__global__ void __launch_bounds__(kNormRows) k_normalize(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.y];
  if (n >= p.N || is_done(p)) return;
  const int R = p.R;
  const int64_t I = p.dims[n];
  const int64_t i0 = (int64_t)blockIdx.x * kNormRows;
  if (i0 >= I) return;
  const int nrb = (int)((I + kSolveRows - 1) / kSolveRows);
  __shared__ double lam[kMaxRank];
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double s = 0.0;
    for (int q = 0; q < nrb; ++q) s += p.Npart[(int64_t)q * R + r];
    lam[r] = sqrt(s);
  }
  __syncthreads();
  if (blockIdx.x == 0)
    for (int r = threadIdx.x; r < R; r += blockDim.x) p.lambda[r] = lam[r];
  const int64_t i1 = min(I, i0 + kNormRows);
  double* A = p.A64[n];
  float* A32 = p.A32[n];
  for (int64_t e = i0 * R + threadIdx.x; e < i1 * R; e += blockDim.x) {
    const double l = lam[e % R];
    double a = A[e];
    if (l > 0.0) a = a / l;
    A[e] = a;
    A32[e] = (float)a;
  }
}

cudaError_t launch_normalize(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  const dim3 grid((g.max_I[n] + kNormRows - 1) / kNormRows, g.B);
  k_normalize<<<grid, kNormRows, 0, s>>>(probs, n);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// Step hooks without a Prob table: the sampler alone and the fiber gather alone.
// ------------------------------------------------------------------------------------------------
struct SampleArgs {
  int64_t dims[kMaxOrder];
  int64_t st[kMaxOrder];
  int N, n;
  int64_t S;
  uint64_t seed;
  uint32_t b, t;
};

__global__ void k_sample_only(SampleArgs a, uint32_t* idx, int64_t* off) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= a.S) return;
  const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
  const uint4 w0 = philox10(make_uint4((uint32_t)j, counter_word1(kStreamSamples, 0, a.n), a.t, a.b), k0, k1);
  uint4 w1 = make_uint4(0u, 0u, 0u, 0u);
  if (a.N - 1 > 4) w1 = philox10(make_uint4((uint32_t)j, counter_word1(kStreamSamples, 1, a.n), a.t, a.b), k0, k1);
  int64_t o = 0;
  int k = 0;
  for (int m = 0; m < a.N; ++m) {
    uint32_t im = 0;
    if (m != a.n) {
      const uint32_t w = k < 4 ? word_of(w0, k) : word_of(w1, k - 4);
      im = scale_index(w, (uint32_t)a.dims[m]);
      o += (int64_t)im * a.st[m];
      ++k;
    }
    if (idx) idx[j * a.N + m] = im;
  }
  if (off) off[j] = o;
}

cudaError_t launch_sample_only(const void*, int N, const int64_t* dims, int n, int64_t S, uint64_t seed,
                               uint32_t b, uint32_t t, uint32_t* idx, int64_t* off, cudaStream_t s) {
  SampleArgs a{};
  int64_t st = 1;
  for (int m = 0; m < N; ++m) {
    a.dims[m] = dims[m];
    a.st[m] = st;
    st *= dims[m];
  }
  a.N = N;
  a.n = n;
  a.S = S;
  a.seed = seed;
  a.b = b;
  a.t = t;
  if (S <= 0) return cudaSuccess;
  k_sample_only<<<(unsigned)((S + 255) / 256), 256, 0, s>>>(a, idx, off);
  return cudaGetLastError();
}

template <typename T>
__global__ void k_gather_only(const T* X, int64_t I, int64_t st, int64_t S, const int64_t* off, T* out) {
  const int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= I * S) return;
  const int64_t j = e / I, i = e - j * I;
  out[e] = X[off[j] + i * st];
}

cudaError_t launch_gather_only(const void* X, int dtype, int64_t I, int64_t st, int64_t S, const int64_t* off,
                               void* out, cudaStream_t s) {
  const int64_t total = I * S;
  if (total <= 0) return cudaSuccess;
  const unsigned blocks = (unsigned)((total + 255) / 256);
  switch (dtype) {
    case CPR_F64: k_gather_only<double><<<blocks, 256, 0, s>>>((const double*)X, I, st, S, off, (double*)out); break;
    case CPR_F32: k_gather_only<float><<<blocks, 256, 0, s>>>((const float*)X, I, st, S, off, (float*)out); break;
    default:
      k_gather_only<unsigned short><<<blocks, 256, 0, s>>>((const unsigned short*)X, I, st, S, off, (unsigned short*)out);
  }
  return cudaGetLastError();
}

}  // namespace cpr
