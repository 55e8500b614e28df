// Sampled fit estimate and stopping test (Sec. 3.4, Sec. 4.2), and the ||X|| reduction.
//
//   k_fit_setup    once per run: the fixed set of P_hat entries (Philox stream 1, i.i.d. uniform)
//                  and their tensor values, gathered once
//   k_fit          every outer iteration: e_i = x_i - sum_r lambda_r prod_n A^(n)(i_n, r), block
//                  sums of e_i^2 in FP64; the last block forms F^ = 1 - sqrt(P mean e^2) / ||X||,
//                  records it and applies the stopping rules (device-side done flag)
//   k_loop_cond    sets the while-condition of a captured iteration graph
//   k_sumsq        ||X||^2: 16-byte vector loads, FP32 sums per vector folded into FP64
#include <math.h>

#include "internal.cuh"

namespace cpr {

template <typename T>
__global__ void k_fit_setup(const Prob* probs) {
  const Prob& p = probs[blockIdx.y];
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= p.P_hat) return;
  const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
  const int N = p.N;
  const uint4 w0 = philox10(make_uint4((uint32_t)j, counter_word1(kStreamFit, 0, 0), 0u, p.b), k0, k1);
  uint4 w1 = make_uint4(0u, 0u, 0u, 0u);
  if (N > 4) w1 = philox10(make_uint4((uint32_t)j, counter_word1(kStreamFit, 1, 0), 0u, p.b), k0, k1);
  int64_t off = 0;
  for (int m = 0; m < N; ++m) {
    const uint32_t w = m < 4 ? word_of(w0, m) : word_of(w1, m - 4);
    const uint32_t im = scale_index(w, (uint32_t)p.dims[m]);
    p.fit_idx[j * N + m] = im;
    off += (int64_t)im * p.st[m];
  }
  p.fit_x[j] = load_as_double<T>(reinterpret_cast<const T*>(p.X), off);
}

cudaError_t launch_fit_setup(const Prob* probs, const GridInfo& g, cudaStream_t s) {
  const dim3 grid((g.max_Phat + 255) / 256, g.B);
  switch (g.dtype) {
    case CPR_F64: k_fit_setup<double><<<grid, 256, 0, s>>>(probs); break;
    case CPR_F32: k_fit_setup<float><<<grid, 256, 0, s>>>(probs); break;
    default: k_fit_setup<__nv_bfloat16><<<grid, 256, 0, s>>>(probs);
  }
  return cudaGetLastError();
}

__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t += red[q];
  return t;  // valid in thread 0
}

// Partial sums of e_i^2 over the block's fit entries; the model entry is
// sum_r w_r prod_n A^(n)(i_n, r) with w_r = lambda_r prod_n scale_n[r] (the lazy column scales).
// The last block of the problem sums the partials (fixed order), forms the fit and applies the
// stopping rules.
template <bool F64>
__global__ void __launch_bounds__(kFitThreads) k_fit(const Prob* probs) {
  const Prob& p = probs[blockIdx.y];
  if (is_done(p)) return;
  if ((int64_t)blockIdx.x * kFitThreads >= p.P_hat) return;
  __shared__ double red[kFitThreads / 32];
  __shared__ double wr[kMaxRank];
  const int R = p.R, N = p.N;
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    double w = p.lambda[r];
    for (int m = 0; m < N; ++m) w *= p.scale[m][r];
    wr[r] = w;
  }
  __syncthreads();
  const int64_t j = (int64_t)blockIdx.x * kFitThreads + threadIdx.x;
  double e2 = 0.0;
  if (j < p.P_hat) {
    const uint32_t* id = p.fit_idx + j * N;
    double model;
    if (F64) {
      double acc = 0.0;
      for (int r = 0; r < R; ++r) {
        double t = wr[r];
        for (int m = 0; m < N; ++m) t *= p.A64[m][(int64_t)id[m] * R + r];
        acc += t;
      }
      model = acc;
    } else {
      float acc = 0.0f;
      for (int r = 0; r < R; ++r) {
        float t = (float)wr[r];
        for (int m = 0; m < N; ++m) t *= p.A32[m][(int64_t)id[m] * R + r];
        acc += t;
      }
      model = (double)acc;
    }
    const double e = p.fit_x[j] - model;
    e2 = e * e;
  }
  const double t = block_sum(e2, red);
  if (threadIdx.x == 0) p.fit_part[blockIdx.x] = t;
  if (!arrive_last(p.state, (uint32_t)p.nfb)) return;
  if (threadIdx.x < 32) {
    double s = 0.0;
    for (int q = threadIdx.x; q < p.nfb; q += 32) s += __ldcg(&p.fit_part[q]);
    for (int o = 16; o > 0; o >>= 1) s += __shfl_down_sync(0xffffffffu, s, o);
    if (threadIdx.x == 0) {
      State* st = p.state;
      const double fit = 1.0 - sqrt((double)p.P * (s / (double)p.P_hat)) / st->norm_x;
      apply_stop_rules(p, st, fit);
    }
  }
}

cudaError_t launch_fit(const Prob* probs, const GridInfo& g, cudaStream_t s) {
  const dim3 grid(g.max_nfb, g.B);
  if (g.any_f64) k_fit<true><<<grid, kFitThreads, 0, s>>>(probs);
  else k_fit<false><<<grid, kFitThreads, 0, s>>>(probs);
  return cudaGetLastError();
}

// Sets the while-condition of a captured iteration graph: keep looping while any problem of the
// batch is still running and fewer than `cap` iterations have run (the cap bounds the loop even if
// a stop flag were never set).
__global__ void k_loop_cond(const Prob* probs, int B, int* loop_iter, int cap, cudaGraphConditionalHandle h) {
  __shared__ int active;
  if (threadIdx.x == 0) active = 0;
  __syncthreads();
  for (int b = threadIdx.x; b < B; b += blockDim.x)
    if (*((volatile int32_t*)&probs[b].state->done) == 0) atomicAdd(&active, 1);
  __syncthreads();
  if (threadIdx.x == 0) {
    const int it = *loop_iter + 1;
    *loop_iter = it;
    cudaGraphSetConditional(h, (active > 0 && it < cap) ? 1u : 0u);
  }
}

cudaError_t launch_loop_cond(const Prob* probs, int B, int* loop_iter, int cap, unsigned long long cond_handle,
                             cudaStream_t s) {
  k_loop_cond<<<1, 128, 0, s>>>(probs, B, loop_iter, cap, (cudaGraphConditionalHandle)cond_handle);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// ||X||^2 (used by the fit, Sec. 3.4).
// ------------------------------------------------------------------------------------------------
int sumsq_blocks(int64_t P) {
  int64_t b = (P + 256 * 64 - 1) / (256 * 64);
  if (b < 1) b = 1;
  if (b > kSumsqMaxBlocks) b = kSumsqMaxBlocks;
  return (int)b;
}

// Each thread keeps 8 independent loads in flight (16-byte vectors where the data allows); squares
// are summed in FP32 within a vector and folded into an FP64 accumulator.  When amax is given, the
// largest |x| is also recorded there (as the bit pattern of a non-negative float, for atomicMax).
template <typename T>
__global__ void __launch_bounds__(256) k_sumsq(const T* __restrict__ X, int64_t P, double* part, unsigned* amax) {
  __shared__ double red[8];
  double acc = 0.0;
  float mx = 0.f;
  const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t nthr = (int64_t)gridDim.x * blockDim.x;
  constexpr int VEC = 16 / sizeof(T);   // elements per 16-byte vector
  const bool aligned = (reinterpret_cast<uintptr_t>(X) & 15) == 0;
  const int64_t nvec = aligned ? P / VEC : 0;
  const uint4* Xv = reinterpret_cast<const uint4*>(X);
  int64_t v = tid;
  for (; v + 7 * nthr < nvec; v += 8 * nthr) {
    uint4 q[8];
#pragma unroll
    for (int u = 0; u < 8; ++u) q[u] = __ldcs(&Xv[v + u * nthr]);
    // FP32 tensors: the eight per-vector FP32 sums are added with Kahan compensation in FP32 and folded
    // into FP64 once (two FP64 additions per 8 vectors, not one per vector: the FP64 pipe bounded this)
    float ks = 0.f, kc = 0.f;
#pragma unroll
    for (int u = 0; u < 8; ++u) {
      const T* e = reinterpret_cast<const T*>(&q[u]);
      if constexpr (sizeof(T) == 8) {
        acc = fma((double)e[0], (double)e[0], acc);
        acc = fma((double)e[1], (double)e[1], acc);
        mx = fmaxf(mx, fmaxf(fabsf((float)e[0]), fabsf((float)e[1])));
      } else {
        float f = 0.0f;
#pragma unroll
        for (int w = 0; w < VEC; ++w) {
          float x;
          if constexpr (sizeof(T) == 4) x = e[w];
          else x = __bfloat162float(e[w]);
          f = fmaf(x, x, f);
          mx = fmaxf(mx, fabsf(x));
        }
        const float y = f - kc;
        const float t = ks + y;
        kc = (t - ks) - y;
        ks = t;
      }
    }
    if constexpr (sizeof(T) != 8) acc += (double)ks - (double)kc;
  }
  for (; v < nvec; v += nthr) {
    const uint4 q = __ldcs(&Xv[v]);
    const T* e = reinterpret_cast<const T*>(&q);
    for (int w = 0; w < VEC; ++w) {
      double x;
      if constexpr (sizeof(T) == 2) x = (double)__bfloat162float(e[w]);
      else x = (double)e[w];
      acc = fma(x, x, acc);
      mx = fmaxf(mx, fabsf((float)x));
    }
  }
  for (int64_t i = nvec * VEC + tid; i < P; i += nthr) {   // tail (or everything if unaligned)
    double x;
    if constexpr (sizeof(T) == 2) x = (double)__bfloat162float(X[i]);
    else x = (double)X[i];
    acc = fma(x, x, acc);
    mx = fmaxf(mx, fabsf((float)x));
  }
  if (amax) {
    const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(mx));
    if ((threadIdx.x & 31) == 0 && m) atomicMax(amax, m);
  }
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

cudaError_t launch_sumsq(const void* X, int dtype, int64_t P, double* part, int nblk, cudaStream_t s,
                         unsigned* amax) {
  switch (dtype) {
    case CPR_F64: k_sumsq<double><<<nblk, 256, 0, s>>>((const double*)X, P, part, amax); break;
    case CPR_F32: k_sumsq<float><<<nblk, 256, 0, s>>>((const float*)X, P, part, amax); break;
    default: k_sumsq<__nv_bfloat16><<<nblk, 256, 0, s>>>((const __nv_bfloat16*)X, P, part, amax);
  }
  return cudaGetLastError();
}

// First level for many partials (one per CTA of a mixing pass): CTA b sums part[4096 b ..
// 4096 b + 4095] in a fixed order (16 loads in flight per thread) into out[b].
constexpr int kPartChunk = 4096;
__global__ void __launch_bounds__(256) k_sumsq_partials(const double* __restrict__ part, int64_t nblk, double* out) {
  __shared__ double red[8];
  const int64_t base = (int64_t)blockIdx.x * kPartChunk;
  double v[kPartChunk / 256];
#pragma unroll
  for (int u = 0; u < kPartChunk / 256; ++u) {
    const int64_t q = base + u * 256 + threadIdx.x;
    v[u] = q < nblk ? part[q] : 0.0;
  }
  double a = 0.0;
#pragma unroll
  for (int u = 0; u < kPartChunk / 256; ++u) a += v[u];
  const double t = block_sum(a, red);
  if (threadIdx.x == 0) out[blockIdx.x] = t;
}

int64_t sumsq_partials_blocks(int64_t nblk) { return (nblk + kPartChunk - 1) / kPartChunk; }

cudaError_t launch_sumsq_partials(const double* part, int64_t nblk, double* out, cudaStream_t s) {
  const int64_t nb = sumsq_partials_blocks(nblk);
  if (nb < 1 || nb > INT32_MAX) return cudaErrorInvalidValue;
  k_sumsq_partials<<<(unsigned)nb, 256, 0, s>>>(part, nblk, out);
  return cudaGetLastError();
}

__global__ void __launch_bounds__(256) k_sumsq_finish(const double* part, int nblk, double* out_norm, State* st,
                                                      int nstates) {
  __shared__ double red[8];
  double a = 0.0;
  for (int q = threadIdx.x; q < nblk; q += blockDim.x) a += part[q];
  const double t = block_sum(a, red);
  if (threadIdx.x == 0) {
    const double nrm = sqrt(t);
    if (out_norm) *out_norm = nrm;
    for (int q = 0; q < nstates; ++q) {
      st[q].norm_x = nrm;
      if (!isfinite(nrm)) {   // a NaN or Inf in X: no fit can be formed, the run does not start
        st[q].status = CPR_ENONFINITE;
        st[q].done = 1;
      }
    }
  }
}

cudaError_t launch_sumsq_finish(const double* part, int nblk, double* out_norm, State* st, int nstates,
                                cudaStream_t s) {
  k_sumsq_finish<<<1, 256, 0, s>>>(part, nblk, out_norm, st, nstates);
  return cudaGetLastError();
}

}  // namespace cpr
