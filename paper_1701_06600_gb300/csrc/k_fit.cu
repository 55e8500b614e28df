// Sampled fit estimate and stopping test (Sec. 3.4, Sec. 4.2), and the ||X|| reduction.
//
//   k_fit_setup    once per run: the fixed set of P_hat entries (Philox stream 1, i.i.d. uniform)
//                  and their tensor values, gathered once
//   k_fit_partial  every outer iteration: e_i = x_i - sum_r lambda_r prod_n A^(n)(i_n, r), block
//                  sums of e_i^2 in FP64
//   k_fit_finish   F^ = 1 - sqrt(P * mean e^2) / ||X||, trace, stopping rules, done flag; with a
//                  graph while-loop, the last block sets the loop condition (any problem active)
//   k_sumsq        ||X||^2: FP32 sums of 16 squares folded into an FP64 accumulator per thread
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

template <bool F64>
__global__ void __launch_bounds__(kFitThreads) k_fit_partial(const Prob* probs) {
  const Prob& p = probs[blockIdx.y];
  if (is_done(p)) return;
  if ((int64_t)blockIdx.x * kFitThreads >= p.P_hat) return;
  __shared__ double red[kFitThreads / 32];
  const int64_t j = (int64_t)blockIdx.x * kFitThreads + threadIdx.x;
  const int R = p.R, N = p.N;
  double e2 = 0.0;
  if (j < p.P_hat) {
    const uint32_t* id = p.fit_idx + j * N;
    double model;
    if (F64) {
      double acc = 0.0;
      for (int r = 0; r < R; ++r) {
        double t = p.lambda[r];
        for (int m = 0; m < N; ++m) t *= p.A64[m][(int64_t)id[m] * R + r];
        acc += t;
      }
      model = acc;
    } else {
      float acc = 0.0f;
      for (int r = 0; r < R; ++r) {
        float t = (float)p.lambda[r];
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
}

cudaError_t launch_fit_partial(const Prob* probs, const GridInfo& g, cudaStream_t s) {
  const dim3 grid(g.max_nfb, g.B);
  if (g.any_f64) k_fit_partial<true><<<grid, kFitThreads, 0, s>>>(probs);
  else k_fit_partial<false><<<grid, kFitThreads, 0, s>>>(probs);
  return cudaGetLastError();
}

__global__ void k_fit_finish(const Prob* probs, int B, int* counter, cudaGraphConditionalHandle h,
                             int use_cond) {
  const Prob& p = probs[blockIdx.x];
  State* st = p.state;
  if (threadIdx.x == 0 && !is_done(p)) {
    double sum = 0.0;
    for (int q = 0; q < p.nfb; ++q) sum += p.fit_part[q];
    const double fit = 1.0 - sqrt((double)p.P * (sum / (double)p.P_hat)) / st->norm_x;
    const int it = st->iter;
    if (p.trace) p.trace[it] = fit;
    const int t1 = it + 1;
    bool stop = false;
    if (!isfinite(fit)) {
      st->status = CPR_ENONFINITE;
      stop = true;
    } else if (p.fixed_iters > 0) {
      stop = t1 >= p.fixed_iters;
    } else {
      if (fit > st->best) {
        st->best = fit;
        st->stall = 0;
      } else {
        st->stall += 1;
      }
      if (t1 >= p.max_iters) stop = true;
      if (t1 >= 2 && fabs(fit - st->last_fit) <= p.tol) stop = true;
      if (p.eta >= 0.0 && fit >= 1.0 - 1.2 * p.eta) stop = true;
      if (p.stall_iters > 0 && st->stall >= p.stall_iters) stop = true;
    }
    st->last_fit = fit;
    st->iter = t1;
    if (stop) st->done = 1;
  }
  if (use_cond && threadIdx.x == 0) {
    __threadfence();
    const int prev = atomicAdd(counter, 1);
    if (prev == B - 1) {  // last block: every problem's flag for this iteration is final
      __threadfence();
      int active = 0;
      for (int q = 0; q < B; ++q) active += (*((volatile int32_t*)&probs[q].state->done) == 0);
      *counter = 0;
      cudaGraphSetConditional(h, active > 0 ? 1u : 0u);
    }
  }
}

cudaError_t launch_fit_finish(const Prob* probs, const GridInfo& g, int* counter, unsigned long long cond_handle,
                              int use_cond, cudaStream_t s) {
  k_fit_finish<<<g.B, 32, 0, s>>>(probs, g.B, counter, (cudaGraphConditionalHandle)cond_handle, use_cond);
  return cudaGetLastError();
}

// ------------------------------------------------------------------------------------------------
// ||X||^2 (used by the fit, Sec. 3.4).
// ------------------------------------------------------------------------------------------------
int sumsq_blocks(int64_t P) {
  int64_t b = (P + 256 * 16 - 1) / (256 * 16);
  if (b < 1) b = 1;
  if (b > 152 * 8) b = 152 * 8;
  return (int)b;
}

template <typename T>
__global__ void __launch_bounds__(256) k_sumsq(const T* __restrict__ X, int64_t P, double* part) {
  __shared__ double red[8];
  const int64_t stride = (int64_t)gridDim.x * blockDim.x;
  double acc = 0.0;
  float f = 0.0f;
  int c = 0;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += stride) {
    if constexpr (sizeof(T) == 8) {
      const double v = X[i];
      acc = fma(v, v, acc);
    } else {
      float v;
      if constexpr (sizeof(T) == 4) v = X[i];
      else v = __bfloat162float(X[i]);
      f = fmaf(v, v, f);
      if (++c == 16) {
        acc += (double)f;
        f = 0.0f;
        c = 0;
      }
    }
  }
  acc += (double)f;
  const double t = block_sum(acc, red);
  if (threadIdx.x == 0) part[blockIdx.x] = t;
}

cudaError_t launch_sumsq(const void* X, int dtype, int64_t P, double* part, int nblk, cudaStream_t s) {
  switch (dtype) {
    case CPR_F64: k_sumsq<double><<<nblk, 256, 0, s>>>((const double*)X, P, part); break;
    case CPR_F32: k_sumsq<float><<<nblk, 256, 0, s>>>((const float*)X, P, part); break;
    default: k_sumsq<__nv_bfloat16><<<nblk, 256, 0, s>>>((const __nv_bfloat16*)X, P, part);
  }
  return cudaGetLastError();
}

__global__ void k_sumsq_finish(const double* part, int nblk, double* out_norm, State* st, int nstates) {
  if (threadIdx.x != 0) return;
  double s = 0.0;
  for (int q = 0; q < nblk; ++q) s += part[q];
  const double nrm = sqrt(s);
  if (out_norm) *out_norm = nrm;
  for (int q = 0; q < nstates; ++q) st[q].norm_x = nrm;
}

cudaError_t launch_sumsq_finish(const double* part, int nblk, double* out_norm, State* st, int nstates,
                                cudaStream_t s) {
  k_sumsq_finish<<<1, 32, 0, s>>>(part, nblk, out_norm, st, nstates);
  return cudaGetLastError();
}

}  // namespace cpr
