// Kernels of one mode-n update of CPRAND (Alg. 3, with Alg. 2 for the sampled Khatri-Rao rows).
//
// Two launches per mode n, each serving every problem of the batch:
//   k_sample_contract   sampling + SKR + fiber gather fused with M = X_S Z_S (FP32 accumulation),
//                       partial FP64 Grams; the last block sums the Grams and factors G = L L^T
//   k_solve             partial-M reduction, FP64 row solves with L, column norms; the last block
//                       writes lambda and the lazy column scales
// Columns are normalized lazily: a factor is stored unnormalized with a per-column scale that its
// consumers (the next SKR, the fit) multiply in; k_finalize folds the scales in at the end.
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
  s->counter = 0;
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
  if (blockIdx.x == 0) {
    for (int e = threadIdx.x; e < p.N * R; e += blockDim.x) p.scale[e / R][e % R] = 1.0;
    if (!from_a64)
      for (int r = threadIdx.x; r < R; r += blockDim.x) p.lambda[r] = 1.0;
  }
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
// Phase 1 of a mode-n update: sampling + SKR + fiber gather + contraction + Gram slice.
//
// Block (tile, split) of a problem owns kP1Rows fiber rows i_n and the samples [js, js + spl).
// Its first threads draw the split's multi-indices (Philox stream 0, counter (j, n, t, b); the
// k-th mode other than n takes word k%4 of block k/4; i_m = floor(w I_m / 2^32)), every thread
// then builds Z_S rows from the factor rows times their lazy column scales (Alg. 2), and each
// thread streams its fiber row of the split's sampled fibers against those rows (M = X_S Z_S,
// FP32 accumulation; FP64 for FP64 tensors).  The ntile blocks of a split share out the R x R
// entries of that split's FP64 Gram.  The last block of the problem to finish sums the partial
// Grams in a fixed order and Cholesky-factors G = L L^T in FP64; a pivot that is not positive
// (relative to the largest diagonal entry) marks the problem CPR_ESINGULAR and stops it.
// ------------------------------------------------------------------------------------------------
template <typename T> __device__ __forceinline__ float to_acc_f(T v);
template <> __device__ __forceinline__ float to_acc_f<float>(float v) { return v; }
template <> __device__ __forceinline__ float to_acc_f<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename ACC, typename T>
__device__ __forceinline__ ACC load_x(const T* __restrict__ X, int64_t i) {
  if constexpr (sizeof(ACC) == 8) return (ACC)__ldg(&X[i]);
  else return to_acc_f<T>(X[i]);
}

__host__ __device__ inline size_t p1_smem_bytes(int spl, int R, int acc_bytes) {
  const int zd = (spl > R ? spl : R) * R;
  return (size_t)kMaxSplit * 8 + (size_t)kMaxSplit * kMaxOrder * 4 + (size_t)zd * 8 + (size_t)spl * R * acc_bytes;
}

template <typename T, typename ACC, int MAXR>
__global__ void __launch_bounds__(kP1Rows) k_sample_contract(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.y];
  if (n >= p.N || is_done(p)) return;
  const int R = p.R, S = p.S, N = p.N;
  const int64_t I = p.dims[n];
  const int ntile = (int)((I + kP1Rows - 1) / kP1Rows);
  const int tile = blockIdx.x % ntile, split = blockIdx.x / ntile;
  if (split >= p.nsplit) return;
  const int js = split * p.spl;
  const int cnt = min(p.spl, S - js);
  extern __shared__ __align__(16) unsigned char smem[];
  int64_t* offs = reinterpret_cast<int64_t*>(smem);
  uint32_t* ids = reinterpret_cast<uint32_t*>(smem + kMaxSplit * 8);
  double* Zd = reinterpret_cast<double*>(smem + kMaxSplit * 8 + kMaxSplit * kMaxOrder * 4);
  ACC* Zs = reinterpret_cast<ACC*>(Zd + (p.spl > R ? p.spl : R) * R);
  const int tid = threadIdx.x;
  const uint32_t t = p.t0 + (uint32_t)p.state->iter;
  if (tid < cnt && p.user_idx) {   // caller-given multi-indices (test hook)
    const uint32_t* u = p.user_idx + ((int64_t)n * S + js + tid) * N;
    for (int m = 0; m < N; ++m) ids[tid * kMaxOrder + m] = m == n ? 0u : u[m];
    int64_t stride;
    offs[tid] = fiber_offset(p, n, ids + tid * kMaxOrder, &stride);
  } else if (tid < cnt) {
    const uint32_t j = (uint32_t)(js + tid);
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
    const uint4 w0 = philox10(make_uint4(j, counter_word1(kStreamSamples, 0, n), t, p.b), k0, k1);
    uint4 w1 = make_uint4(0u, 0u, 0u, 0u);
    if (N - 1 > 4) w1 = philox10(make_uint4(j, counter_word1(kStreamSamples, 1, n), t, p.b), k0, k1);
    int k = 0;
    for (int m = 0; m < N; ++m) {
      uint32_t im = 0;
      if (m != n) {
        const uint32_t w = k < 4 ? word_of(w0, k) : word_of(w1, k - 4);
        im = scale_index(w, (uint32_t)p.dims[m]);
        ++k;
      }
      ids[tid * kMaxOrder + m] = im;
    }
    int64_t stride;
    offs[tid] = fiber_offset(p, n, ids + tid * kMaxOrder, &stride);
  }
  __syncthreads();
  for (int e = tid; e < cnt * R; e += blockDim.x) {
    const int jj = e / R, r = e - jj * R;
    double z = 1.0;
    for (int m = 0; m < N; ++m) {
      if (m == n) continue;
      const int64_t a = (int64_t)ids[jj * kMaxOrder + m] * R + r;
      const double v = (sizeof(ACC) == 8) ? p.A64[m][a] : (double)p.A32[m][a];
      z *= v * p.scale[m][r];
    }
    Zd[e] = z;
    Zs[e] = (ACC)z;
  }
  __syncthreads();
  const int64_t i = (int64_t)tile * kP1Rows + tid;
  if (i < I) {
    const T* __restrict__ X = reinterpret_cast<const T*>(p.Xrep[n]);
    const int64_t sti = i * (p.use_rep ? 1 : p.st[n]);
    ACC acc[MAXR];
#pragma unroll
    for (int r = 0; r < MAXR; ++r) acc[r] = ACC(0);
    int j = 0;
    for (; j + 8 <= cnt; j += 8) {
      ACC x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) x[q] = load_x<ACC>(X, offs[j + q] + sti);
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const ACC* z = Zs + (j + q) * R;
#pragma unroll
        for (int r = 0; r < MAXR; ++r)
          if (r < R) acc[r] = fma(x[q], z[r], acc[r]);
      }
    }
    for (; j < cnt; ++j) {
      const ACC x = load_x<ACC>(X, offs[j] + sti);
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
  // this tile's share of the split's Gram entries (upper triangle)
  double* Gp = p.Gpart + (int64_t)split * R * R;
  for (int e = tile + ntile * tid; e < R * R; e += ntile * blockDim.x) {
    const int r = e / R, c = e - r * R;
    if (c < r) continue;
    double a = 0.0;
    for (int jj = 0; jj < cnt; ++jj) a = fma(Zd[jj * R + r], Zd[jj * R + c], a);
    Gp[e] = a;
  }
  if (!arrive_last(p.state, (uint32_t)(ntile * p.nsplit))) return;
  double* G = Zd;  // reuse: holds at least R*R doubles
  const int ns = p.nsplit;
  for (int e = tid; e < R * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    if (c < r) continue;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int q = 0;
    for (; q + 4 <= ns; q += 4) {
      a0 += __ldcg(&p.Gpart[(int64_t)(q + 0) * R * R + e]);
      a1 += __ldcg(&p.Gpart[(int64_t)(q + 1) * R * R + e]);
      a2 += __ldcg(&p.Gpart[(int64_t)(q + 2) * R * R + e]);
      a3 += __ldcg(&p.Gpart[(int64_t)(q + 3) * R * R + e]);
    }
    for (; q < ns; ++q) a0 += __ldcg(&p.Gpart[(int64_t)q * R * R + e]);
    const double g = (a0 + a1) + (a2 + a3);
    G[r * R + c] = g;
    G[c * R + r] = g;
  }
  __syncthreads();
  const bool ok = block_cholesky(G, R);
  for (int e = tid; e < R * R; e += blockDim.x) p.L[e] = G[e];
  if (tid == 0 && !ok) {
    p.state->status = CPR_ESINGULAR;
    p.state->done = 1;
  }
}

template <typename T, typename ACC, int MAXR>
static cudaError_t p1_attr() {
  const size_t most = p1_smem_bytes(kMaxSplit, kMaxRank, (int)sizeof(ACC));
  return cudaFuncSetAttribute(k_sample_contract<T, ACC, MAXR>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)most);
}

template <typename T, typename ACC, int MAXR>
static cudaError_t p1_launch(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  const size_t smem = p1_smem_bytes(g.max_spl, g.max_R, (int)sizeof(ACC));
  k_sample_contract<T, ACC, MAXR><<<dim3(g.max_tiles_x_split[n], g.B), kP1Rows, smem, s>>>(probs, n);
  return cudaGetLastError();
}

template <typename T, typename ACC>
static cudaError_t p1_dispatch(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  if (g.max_R <= 8) return p1_launch<T, ACC, 8>(probs, g, n, s);
  if (g.max_R <= 16) return p1_launch<T, ACC, 16>(probs, g, n, s);
  if (g.max_R <= 32) return p1_launch<T, ACC, 32>(probs, g, n, s);
  return p1_launch<T, ACC, 64>(probs, g, n, s);
}

cudaError_t launch_sample_contract(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  if (g.max_tiles_x_split[n] <= 0) return cudaSuccess;
  switch (g.dtype) {
    case CPR_F64: return p1_dispatch<double, double>(probs, g, n, s);
    case CPR_F32: return p1_dispatch<float, float>(probs, g, n, s);
    default: return p1_dispatch<__nv_bfloat16, float>(probs, g, n, s);
  }
}

// ------------------------------------------------------------------------------------------------
// Phase 2 of a mode-n update: for the block's kP2Rows rows of the new factor, m_i = sum over
// splits of the partial M rows, then a_i (L L^T) = m_i by forward and backward substitution in
// FP64 (Alg. 3 least-squares step through the normal equations).  The rows are stored
// unnormalized (FP64 and FP32); the last block of the problem sums the column sums of squares
// and writes lambda_r = ||a_r|| and the lazy scales 1 / ||a_r|| (1 for a zero column) (Alg. 3
// normalization step).
// ------------------------------------------------------------------------------------------------
template <typename ACC>
__global__ void __launch_bounds__(kP2Threads) k_solve(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.y];
  if (n >= p.N || is_done(p)) return;
  const int R = p.R, R1 = R + 1;
  const int64_t I = p.dims[n];
  const int64_t i0 = (int64_t)blockIdx.x * kP2Rows;
  if (i0 >= I) return;
  const int nrb = (int)((I + kP2Rows - 1) / kP2Rows);
  const int rows = (int)min((int64_t)kP2Rows, I - i0);
  extern __shared__ double sm[];
  double* Ls = sm;             // R x (R+1)
  double* V = sm + R * R1;     // kP2Rows x (R+1)
  const int tid = threadIdx.x;
  for (int e = tid; e < R * R; e += blockDim.x) Ls[(e / R) * R1 + e % R] = p.L[e];
  const ACC* Mp = reinterpret_cast<const ACC*>(p.Mpart);
  const int ns = p.nsplit;
  const int64_t stride = (int64_t)p.imax * R;
  for (int e = tid; e < rows * R; e += blockDim.x) {
    const int li = e / R, r = e - li * R;
    const ACC* src = Mp + (i0 + li) * R + r;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int q = 0;
    for (; q + 4 <= ns; q += 4) {
      a0 += (double)src[(q + 0) * stride];
      a1 += (double)src[(q + 1) * stride];
      a2 += (double)src[(q + 2) * stride];
      a3 += (double)src[(q + 3) * stride];
    }
    for (; q < ns; ++q) a0 += (double)src[q * stride];
    V[li * R1 + r] = (a0 + a1) + (a2 + a3);
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
  float* A32 = p.A32[n] + i0 * R;
  for (int e = tid; e < rows * R; e += blockDim.x) {
    const double v = V[(e / R) * R1 + e % R];
    A[e] = v;
    A32[e] = (float)v;
  }
  for (int r = tid; r < R; r += blockDim.x) {
    double s = 0.0;
    for (int li = 0; li < rows; ++li) {
      const double v = V[li * R1 + r];
      s = fma(v, v, s);
    }
    p.Npart[(int64_t)blockIdx.x * R + r] = s;
  }
  if (!arrive_last(p.state, (uint32_t)nrb)) return;
  for (int r = tid; r < R; r += blockDim.x) {
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int q = 0;
    for (; q + 4 <= nrb; q += 4) {
      a0 += __ldcg(&p.Npart[(int64_t)(q + 0) * R + r]);
      a1 += __ldcg(&p.Npart[(int64_t)(q + 1) * R + r]);
      a2 += __ldcg(&p.Npart[(int64_t)(q + 2) * R + r]);
      a3 += __ldcg(&p.Npart[(int64_t)(q + 3) * R + r]);
    }
    for (; q < nrb; ++q) a0 += __ldcg(&p.Npart[(int64_t)q * R + r]);
    const double nrm = sqrt((a0 + a1) + (a2 + a3));
    p.lambda[r] = nrm;
    p.scale[n][r] = nrm > 0.0 ? 1.0 / nrm : 1.0;
  }
}

template <typename ACC>
static cudaError_t p2_attr() {
  const size_t most = ((size_t)kMaxRank * (kMaxRank + 1) + (size_t)kP2Rows * (kMaxRank + 1)) * sizeof(double);
  return cudaFuncSetAttribute(k_solve<ACC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)most);
}

// Opt every kernel that may need more than 48 KB of dynamic shared memory into its maximum, once
// per device, before any launch (and before any stream capture).
cudaError_t prepare_kernel_attributes() {
  static int done_mask = 0;
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return e;
  if (dev < 32 && (done_mask >> dev) & 1) return cudaSuccess;
  cudaError_t (*fns[])() = {
      p1_attr<double, double, 8>, p1_attr<double, double, 16>, p1_attr<double, double, 32>, p1_attr<double, double, 64>,
      p1_attr<float, float, 8>, p1_attr<float, float, 16>, p1_attr<float, float, 32>, p1_attr<float, float, 64>,
      p1_attr<__nv_bfloat16, float, 8>, p1_attr<__nv_bfloat16, float, 16>, p1_attr<__nv_bfloat16, float, 32>,
      p1_attr<__nv_bfloat16, float, 64>, p2_attr<double>, p2_attr<float>};
  for (auto f : fns)
    if ((e = f()) != cudaSuccess) return e;
  if ((e = prepare_als_attributes()) != cudaSuccess) return e;
  if (dev < 32) done_mask |= 1 << dev;
  return cudaSuccess;
}

template <typename ACC>
static cudaError_t p2_launch(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  const size_t smem = ((size_t)g.max_R * (g.max_R + 1) + (size_t)kP2Rows * (g.max_R + 1)) * sizeof(double);
  const dim3 grid((g.max_I[n] + kP2Rows - 1) / kP2Rows, g.B);
  k_solve<ACC><<<grid, kP2Threads, smem, s>>>(probs, n);
  return cudaGetLastError();
}

cudaError_t launch_solve(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  return g.dtype == CPR_F64 ? p2_launch<double>(probs, g, n, s) : p2_launch<float>(probs, g, n, s);
}

// ------------------------------------------------------------------------------------------------
// End of a run: fold the lazy column scales into the FP64 factor of mode n (unit columns).
// ------------------------------------------------------------------------------------------------
__global__ void k_finalize(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.y];
  if (n >= p.N) return;
  const int R = p.R;
  const int64_t cnt = p.dims[n] * R;
  for (int64_t e = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; e < cnt; e += (int64_t)gridDim.x * blockDim.x)
    p.A64[n][e] *= p.scale[n][e % R];
}

cudaError_t launch_finalize(const Prob* probs, const GridInfo& g, int n, cudaStream_t s) {
  int64_t blocks = ((int64_t)g.max_I[n] * g.max_R + 255) / 256;
  if (blocks < 1) blocks = 1;
  if (blocks > 1024) blocks = 1024;
  k_finalize<<<dim3((unsigned)blocks, g.B), 256, 0, s>>>(probs, n);
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

// Contiguous fibers (stride 1, the first mode or a column-major unfolding copy): one warp per
// fiber, grid-stride over the fibers, the next fiber's offset loaded ahead; a fiber whose start and
// destination are 16-byte aligned and whose length is a multiple of the vector moves as 16-byte
// vectors with all of a lane's loads (up to 4 per 128 vectors) issued before its stores, else
// element by element.
template <typename T>
__global__ void __launch_bounds__(256) k_gather_contig(const T* __restrict__ X, int64_t I, int64_t S,
                                                       const int64_t* __restrict__ off, T* __restrict__ out) {
  constexpr int E = 16 / (int)sizeof(T);
  const int lane = threadIdx.x & 31;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  int64_t j = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int64_t oj = j < S ? __ldg(off + j) : 0;
  for (; j < S; j += nw) {
    const int64_t jn = j + nw;
    const int64_t on = jn < S ? __ldg(off + jn) : 0;   // next fiber's offset, in flight meanwhile
    const T* src = X + oj;
    T* dst = out + j * I;
    const bool vec = I % E == 0 && (reinterpret_cast<uintptr_t>(src) & 15) == 0 &&
                     (reinterpret_cast<uintptr_t>(dst) & 15) == 0;
    if (vec) {
      const uint4* s4 = reinterpret_cast<const uint4*>(src);
      uint4* d4 = reinterpret_cast<uint4*>(dst);
      const int64_t nv = I / E;
      for (int64_t v0 = 0; v0 < nv; v0 += 128) {
        uint4 a[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t v = v0 + lane + 32 * q;
          if (v < nv) a[q] = __ldg(s4 + v);
        }
#pragma unroll
        for (int q = 0; q < 4; ++q) {
          const int64_t v = v0 + lane + 32 * q;
          if (v < nv) d4[v] = a[q];
        }
      }
    } else {
      for (int64_t i = lane; i < I; i += 32) dst[i] = src[i];
    }
    oj = on;
  }
}

template <typename T>
static void gather_dispatch(const T* X, int64_t I, int64_t st, int64_t S, const int64_t* off, T* out, cudaStream_t s) {
  if (st == 1) {
    int dev = 0, sms = 148;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int64_t want = (S + 7) / 8;                 // 8 warps (fibers) per block
    const int64_t blocks = want < (int64_t)sms * 8 ? want : (int64_t)sms * 8;
    k_gather_contig<T><<<(unsigned)blocks, 256, 0, s>>>(X, I, S, off, out);
  } else {
    const int64_t total = I * S;
    k_gather_only<T><<<(unsigned)((total + 255) / 256), 256, 0, s>>>(X, I, st, S, off, out);
  }
}

cudaError_t launch_gather_only(const void* X, int dtype, int64_t I, int64_t st, int64_t S, const int64_t* off,
                               void* out, cudaStream_t s) {
  const int64_t total = I * S;
  if (total <= 0) return cudaSuccess;
  switch (dtype) {
    case CPR_F64: gather_dispatch<double>((const double*)X, I, st, S, off, (double*)out, s); break;
    case CPR_F32: gather_dispatch<float>((const float*)X, I, st, S, off, (float*)out, s); break;
    default:
      gather_dispatch<unsigned short>((const unsigned short*)X, I, st, S, off, (unsigned short*)out, s);
  }
  return cudaGetLastError();
}

}  // namespace cpr
