// Sampled fit estimate that needs no caller workspace and allocates nothing.
//
// Who this is for: code that must not allocate device memory at the moment it asks for a fit --
// for example a plugin that may only use memory its host application handed out, a process whose
// whole device memory is owned by another allocator, or a caller on a latency-critical path where
// an allocation (and the synchronization it can imply) is not acceptable.  Such callers pass only
// the tensor and the model; the scratch this computation needs lives in one fixed-size array in
// device memory that the library declares at file scope.  Every device that loads the library
// holds that array (about 42 KB) until the process exits.
//
// The array is shared by every call on a device and keeps whatever the previous call left in it.
// Each call first clears the counter that must start at zero.  Two calls whose kernels overlap on
// the GPU (for instance on two streams with no ordering between them) race on the array and give
// undefined results: order such calls on one stream or with events.
//
// The host needs the array's device address: on the first call on each device (with that device
// current) the library looks it up with cudaGetSymbolAddress and caches it; make that first call
// outside any stream capture.
#include <math.h>
#include <string.h>

#include <mutex>

#include "internal.cuh"

namespace cpr {
namespace {

constexpr int kNaThreads = 256;
constexpr int64_t kNaMaxFit = CPR_NOALLOC_MAX_FIT_SAMPLES;
constexpr int kNaMaxFitBlocks = (int)(kNaMaxFit / kNaThreads);
constexpr int kNaNormBlocks = kSumsqMaxBlocks;  // the most blocks the ||X|| reduction uses
// scratch layout, in doubles
constexpr int kNaFitPart = 0;
constexpr int kNaNormPart = kNaFitPart + kNaMaxFitBlocks;
constexpr int kNaNorm = kNaNormPart + kNaNormBlocks;
constexpr int kNaFit = kNaNorm + 1;
constexpr int kNaCounter = kNaFit + 1;   // an unsigned int stored in this slot
constexpr int kNaScratchDoubles = kNaCounter + 6;

}  // namespace
}  // namespace cpr

static __device__ __align__(256) double g_noalloc_scratch[cpr::kNaScratchDoubles];

namespace cpr {
namespace {

struct NaArgs {
  int64_t dims[kMaxOrder];
  int64_t st[kMaxOrder];
  const double* factors[kMaxOrder];
  const double* lambda;
  int N, R;
  int64_t P_hat;
  double P;
  uint64_t seed;
  uint32_t b;
  int use_scratch_norm;
  double norm_x;
};

// The device address of the scratch array on the current device, looked up once per device.
double* scratch_for_current_device(cudaError_t* err) {
  static std::mutex mu;
  static double* ptrs[64] = {};
  int dev = 0;
  *err = cudaGetDevice(&dev);
  if (*err != cudaSuccess) return nullptr;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  std::lock_guard<std::mutex> lk(mu);
  if (!ptrs[dev]) {
    void* p = nullptr;
    *err = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (*err != cudaSuccess) return nullptr;
    ptrs[dev] = static_cast<double*>(p);
  }
  return ptrs[dev];
}

__device__ __forceinline__ double na_block_sum(double v) {
  __shared__ double red[kNaThreads / 32];
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  if (threadIdx.x == 0)
    for (int q = 0; q < kNaThreads / 32; ++q) t += red[q];
  return t;
}

// Same draws as the library's fit set (Philox stream 1, counter (j, (1<<8)|(blk<<4), 0, b)); the
// model entry is evaluated in FP64 from the caller's FP64 factors; the last block forms the fit.
template <typename T>
__global__ void __launch_bounds__(kNaThreads) k_fit_noalloc(const T* __restrict__ X, NaArgs a, double* scratch) {
  const int64_t j = (int64_t)blockIdx.x * kNaThreads + threadIdx.x;
  double e2 = 0.0;
  if (j < a.P_hat) {
    const uint32_t k0 = (uint32_t)a.seed, k1 = (uint32_t)(a.seed >> 32);
    const uint4 w0 = philox10(make_uint4((uint32_t)j, counter_word1(kStreamFit, 0, 0), 0u, a.b), k0, k1);
    uint4 w1 = make_uint4(0u, 0u, 0u, 0u);
    if (a.N > 4) w1 = philox10(make_uint4((uint32_t)j, counter_word1(kStreamFit, 1, 0), 0u, a.b), k0, k1);
    uint32_t id[kMaxOrder];
    int64_t off = 0;
    for (int m = 0; m < a.N; ++m) {
      const uint32_t w = m < 4 ? word_of(w0, m) : word_of(w1, m - 4);
      id[m] = scale_index(w, (uint32_t)a.dims[m]);
      off += (int64_t)id[m] * a.st[m];
    }
    double model = 0.0;
    for (int r = 0; r < a.R; ++r) {
      double t = a.lambda[r];
      for (int m = 0; m < a.N; ++m) t *= a.factors[m][(int64_t)id[m] * a.R + r];
      model += t;
    }
    const double e = load_as_double<T>(X, off) - model;
    e2 = e * e;
  }
  const double t = na_block_sum(e2);
  if (threadIdx.x == 0) scratch[kNaFitPart + blockIdx.x] = t;
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned int* counter = reinterpret_cast<unsigned int*>(scratch + kNaCounter);
    last = (atomicAdd(counter, 1u) == gridDim.x - 1);
  }
  __syncthreads();
  if (!last) return;
  __threadfence();
  double s = 0.0;
  for (int q = threadIdx.x; q < (int)gridDim.x; q += kNaThreads) s += __ldcg(&scratch[kNaFitPart + q]);
  const double total = na_block_sum(s);
  if (threadIdx.x == 0) {
    const double nrm = a.use_scratch_norm ? __ldcg(&scratch[kNaNorm]) : a.norm_x;
    scratch[kNaFit] = 1.0 - sqrt(a.P * (total / (double)a.P_hat)) / nrm;
    *reinterpret_cast<unsigned int*>(scratch + kNaCounter) = 0u;
  }
}

}  // namespace
}  // namespace cpr

using namespace cpr;

extern "C" int cpr_fit_estimate_noalloc(const cpr_tensor* X, const cpr_ktensor* K, int64_t P_hat, uint64_t seed,
                                        uint32_t b, double norm_x, double* fit_host, void* stream) {
  // argument checks (nothing is enqueued when one fails)
  if (!X || !K || !fit_host || !X->data) return CPR_EINVAL;
  if (X->order < 2 || X->order > CPR_MAX_ORDER || X->dtype < CPR_F64 || X->dtype > CPR_BF16) return CPR_EINVAL;
  if (K->order != X->order || K->rank < 1 || K->rank > CPR_MAX_RANK || !K->lambda) return CPR_EINVAL;
  if (P_hat < 1 || P_hat > kNaMaxFit) return CPR_EINVAL;   // beyond the fixed scratch: rejected
  NaArgs a;
  memset(&a, 0, sizeof(a));
  int64_t st = 1;
  double P = 1.0;
  double Pd = 1.0;
  for (int n = 0; n < X->order; ++n) Pd *= (double)X->dims[n];
  if (Pd > 4.0e18) return CPR_EINVAL;   // the same bound on the entry count as cpr_fit_estimate
  for (int n = 0; n < X->order; ++n) {
    if (X->dims[n] < 1 || X->dims[n] >= (int64_t(1) << 31) || K->dims[n] != X->dims[n] || !K->factors[n])
      return CPR_EINVAL;
    a.dims[n] = X->dims[n];
    a.st[n] = st;
    a.factors[n] = K->factors[n];
    st *= X->dims[n];
    P *= (double)X->dims[n];
  }
  a.lambda = K->lambda;
  a.N = X->order;
  a.R = K->rank;
  a.P_hat = P_hat;
  a.P = P;
  a.seed = seed;
  a.b = b;
  a.use_scratch_norm = norm_x < 0.0;
  a.norm_x = norm_x;
  cudaError_t err = cudaSuccess;
  double* scratch = scratch_for_current_device(&err);
  if (!scratch) return CPR_ECUDA;
  cudaStream_t s = (cudaStream_t)stream;
  // the call ends with a synchronization and a copy into pageable host memory, which a captured
  // stream cannot take: refuse before anything is enqueued
  cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cst) != cudaSuccess) return CPR_ECUDA;
  if (cst != cudaStreamCaptureStatusNone) return CPR_EINVAL;
  const int nblk = a.use_scratch_norm ? sumsq_blocks(st) : 0;
  if (nblk > kNaNormBlocks) return CPR_EINVAL;   // cannot happen while both use kSumsqMaxBlocks
  if (cudaMemsetAsync(scratch + kNaCounter, 0, sizeof(double), s) != cudaSuccess) return CPR_ECUDA;
  if (a.use_scratch_norm) {
    if (launch_sumsq(X->data, X->dtype, st, scratch + kNaNormPart, nblk, s) != cudaSuccess) return CPR_ECUDA;
    if (launch_sumsq_finish(scratch + kNaNormPart, nblk, scratch + kNaNorm, nullptr, 0, s) != cudaSuccess)
      return CPR_ECUDA;
  }
  const unsigned blocks = (unsigned)((P_hat + kNaThreads - 1) / kNaThreads);
  switch (X->dtype) {
    case CPR_F64: k_fit_noalloc<double><<<blocks, kNaThreads, 0, s>>>((const double*)X->data, a, scratch); break;
    case CPR_F32: k_fit_noalloc<float><<<blocks, kNaThreads, 0, s>>>((const float*)X->data, a, scratch); break;
    default: k_fit_noalloc<__nv_bfloat16><<<blocks, kNaThreads, 0, s>>>((const __nv_bfloat16*)X->data, a, scratch);
  }
  if (cudaGetLastError() != cudaSuccess) return CPR_ECUDA;
  if (cudaMemcpyAsync(fit_host, scratch + kNaFit, sizeof(double), cudaMemcpyDeviceToHost, s) != cudaSuccess)
    return CPR_ECUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return CPR_ECUDA;
  return CPR_OK;
}
