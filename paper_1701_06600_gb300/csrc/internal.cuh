// Internal declarations shared by the CUDA translation units of libcprand.
//
// Device-side design (GB300, sm_103a):
//  * Every kernel serves a BATCH of independent problems (blockIdx.y = problem).  A single
//    decomposition is a batch of one, so the batched multi-start path and the single path are the
//    same kernels.
//  * Everything a kernel needs about a problem is in a Prob descriptor in device memory, and every
//    per-iteration quantity (the outer-iteration counter t, the stop flag) is read from the
//    problem's State in device memory.  Kernel arguments therefore never change between outer
//    iterations, which is what lets one iteration be captured once in a CUDA graph and replayed
//    under a device-evaluated while-condition.
//  * A problem whose stopping rule fired (State::done) makes every later kernel return at once.
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include "../../include/cprand.h"

namespace cpr {

constexpr int kMaxOrder = CPR_MAX_ORDER;
constexpr int kMaxRank = CPR_MAX_RANK;

// Tiling constants (block shapes sized so small problems still spread over the 152 SMs).
constexpr int kP1Rows = 128;       // fiber rows (= threads) per block of the sample/contract kernel
constexpr int kMaxSplit = 64;      // most samples per block of the sample/contract kernel
constexpr int kP2Rows = 32;        // factor rows per block of the solve kernel
constexpr int kP2Threads = 128;    // threads per block of the solve kernel
constexpr int kFitThreads = 256;   // fit entries per block in the fit kernel

struct State {
  int32_t iter;      // outer iterations completed in this run
  int32_t done;      // stopping rule fired (or an error occurred)
  int32_t status;    // CPR_OK or a device-detected CPR_E*
  int32_t stall;     // iterations since the best fit last improved
  double best;       // best sampled fit so far
  double last_fit;   // sampled fit of the last completed iteration
  double norm_x;     // ||X||
  uint32_t counter;  // blocks of the current phase that have finished (last-block detection)
  uint32_t pad;
};

struct Prob {
  int32_t N, R, S, dtype;
  int64_t dims[kMaxOrder];
  int64_t st[kMaxOrder];   // column-major strides: st[n] = prod_{m<n} dims[m]
  int64_t P;               // prod dims
  const void* X;           // tensor being decomposed (the mixed tensor for CPRAND-MIX)
  const void* Xrep[kMaxOrder];  // mode-n gathers read Xrep[n]: X itself (mode 1, or no copies) or
                                // X_(n) stored column-major (every sampled fiber contiguous)
  int32_t use_rep;         // Xrep[n] for n >= 1 are the column-major unfoldings
  int32_t pad_rep;

  float* A32[kMaxOrder];   // FP32 working copy of each factor (I_n x R row-major), unnormalized
  double* A64[kMaxOrder];  // FP64 factors (I_n x R row-major), unnormalized during a run
  double* scale[kMaxOrder];// per mode, R inverse column norms (1 where the norm is 0): the
                           // normalized factor is A * scale, applied lazily by its consumers
  double* lambda;          // R: column norms of the mode updated last
  void* Apad[kMaxOrder];   // cluster loop: factor rows padded to Rp = 4 ceil(R/4) elements (FP32,
                           // FP64 for FP64 tensors) for 16-byte vector reads by the fit

  // scratch of one mode update
  double* Gpart;           // nsplit x R x R partial Grams (upper triangle used)
  double* L;               // R x R Cholesky factor (lower)
  void* Mpart;             // nsplit x Imax x R partial X_S Z_S (float, or double for FP64)
  double* Npart;           // ceil(Imax / kP2Rows) x R partial column sums of squares
  int32_t spl, nsplit;     // samples per block split, number of splits
  int32_t imax;            // max dims (row stride of Mpart)
  int32_t pad1;

  // sampled fit (Sec. 3.4)
  int32_t P_hat, nfb;
  uint32_t* fit_idx;       // P_hat x N
  double* fit_x;           // P_hat tensor values
  double* fit_part;        // nfb partial sums of e^2
  double* trace;           // may be null

  // stopping rules (Sec. 4.2)
  int32_t max_iters, fixed_iters, stall_iters, pad0;
  double tol, eta;

  // random streams
  uint64_t seed;
  uint32_t b, t0;

  State* state;

  // CP-ALS (Alg. 1): exact MTTKRP over the unfolding copies, Grams of the normalized factors
  double* gram[kMaxOrder]; // per mode, R x R Gram A^T A of the normalized factor
  double* V;               // R x R Hadamard product of the other modes' Grams (mode updated last)
  double* Mfold;           // imax x R: the MTTKRP of the mode being updated (split partials summed)
  int64_t jsplit[kMaxOrder];  // MTTKRP: unfolding columns per split, per mode
  int32_t als_nsplit[kMaxOrder];  // MTTKRP: splits per mode
  int32_t als_rg;          // MTTKRP: rank groups of 8 columns per thread tile (1, 2, 4 or 8)
  int32_t pad2;

  // caller-given sample multi-indices (test hook): N x S x N uint32, entry ((n S + j) N + m) is
  // i_m of sample j of every mode-n update (the mode-n slot is ignored); null: Philox draws
  const uint32_t* user_idx;
  int32_t grid_min_split;  // whole-GPU loop: fewest samples per contraction split (0: 16)
  int32_t pad3;
};

// Global scratch and barrier words of the whole-GPU loop (k_grid.cu), carved from the workspace.
constexpr int kGridMaxCTAs = 256;  // CTAs the scratch is sized for (one per SM)
constexpr int kGridMaxRows = 32;   // factor rows a CTA solves per mode update (I_n <= 32 G)
constexpr int kGridTileRows = 128; // most fiber rows of a contraction tile (sizes the partial M)
constexpr uint32_t kDefaultWaitPolls = 1u << 22;   // polls of a bounded wait unless opts say otherwise
struct GridScratch {
  float2* Gpart;     // G x NE partial Grams (packed upper triangle; FP32 pairs hi + lo)
  float2* Gfull;     // NE (pairs)
  float* Mpart;      // nsplit x R x I_n partial M (column-major per split)
  float2* Npart;     // G x R column sums of squares (pairs)
  double* fitpart;   // G partial fit sums
  unsigned* bar;     // [0] arrivals, [1] generation (zeroed before each launch)
  int* err;          // set when a barrier wait ran out
  uint32_t wait_limit;  // polls per barrier wait
  int32_t use_tc;       // contraction on the tensor cores (1) or by FP32 FMA (0)
};

// ------------------------------------------------------------------------------------------------
// Philox4x32-10 (Salmon et al., SC'11): 10 rounds of two 32x32->64 multiplies with key bumps.
// ------------------------------------------------------------------------------------------------
__device__ __forceinline__ uint4 philox10(uint4 c, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int rnd = 0; rnd < 10; ++rnd) {
    if (rnd) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t lo0 = 0xD2511F53u * c.x, hi0 = __umulhi(0xD2511F53u, c.x);
    const uint32_t lo1 = 0xCD9E8D57u * c.z, hi1 = __umulhi(0xCD9E8D57u, c.z);
    c = make_uint4(hi1 ^ c.y ^ k0, lo1, hi0 ^ c.w ^ k1, lo0);
  }
  return c;
}

__device__ __forceinline__ uint32_t word_of(const uint4& w, int q) {
  return q == 0 ? w.x : (q == 1 ? w.y : (q == 2 ? w.z : w.w));
}

// index in [0, extent): high word of the 64-bit product
__device__ __forceinline__ uint32_t scale_index(uint32_t w, uint32_t extent) {
  return __umulhi(w, extent);
}

__device__ __forceinline__ uint32_t counter_word1(uint32_t stream, uint32_t block, uint32_t mode) {
  return (stream << 8) | (block << 4) | mode;
}

constexpr uint32_t kStreamSamples = 0, kStreamFit = 1, kStreamInit = 2, kStreamSigns = 3;

template <typename T> __device__ __forceinline__ double load_as_double(const T* p, int64_t i);
template <> __device__ __forceinline__ double load_as_double<double>(const double* p, int64_t i) { return p[i]; }
template <> __device__ __forceinline__ double load_as_double<float>(const float* p, int64_t i) { return (double)p[i]; }
template <> __device__ __forceinline__ double load_as_double<__nv_bfloat16>(const __nv_bfloat16* p, int64_t i) {
  return (double)__bfloat162float(p[i]);
}

__device__ __forceinline__ bool is_done(const Prob& p) {
  return *((volatile int32_t*)&p.state->done) != 0;
}

// Every block of a problem calls this after writing its partial results; it returns true in
// exactly one block (the last to arrive), which may then read every block's partials.  The
// counter is reset by that block for the next phase (phases of one problem run in stream order).
__device__ __forceinline__ bool arrive_last(State* st, uint32_t nblocks) {
  __shared__ int last;
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) {
    const uint32_t prev = atomicAdd(&st->counter, 1u);
    last = (prev == nblocks - 1);
    if (last) st->counter = 0;
  }
  __syncthreads();
  if (last) __threadfence();
  return last != 0;
}

// Stopping rules of Sec. 4.2 for one problem after its fit (one thread): record the trace entry,
// update the best fit and stall count, advance the iteration counter, set done when a rule fires.
__device__ __forceinline__ void apply_stop_rules(const Prob& p, State* st, double fit) {
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

// Cholesky G = L L^T in place (lower triangle), R x R in shared memory, by the whole block.
// Returns false (on every thread) if a pivot is not positive relative to the largest diagonal.
__device__ __forceinline__ bool block_cholesky(double* G, int R) {
  __shared__ int bad;
  __shared__ double maxdiag;
  const int tid = threadIdx.x;
  if (tid == 0) {
    double m = 0.0;
    for (int k = 0; k < R; ++k) m = fmax(m, G[k * R + k]);
    maxdiag = m;
    bad = 0;
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
  return bad == 0;
}

// ------------------------------------------------------------------------------------------------
// Launch wrappers (defined in the .cu files).  `probs` is the device descriptor array, B the batch
// size, bmax_* the per-batch maxima used to size grids.
// ------------------------------------------------------------------------------------------------
struct GridInfo {
  int B;
  int max_S;        // max S over problems
  int max_spl;      // max samples per split
  int max_nfb;      // max fit blocks
  int max_I[kMaxOrder];  // max dims[n] over problems
  int max_tiles_x_split[kMaxOrder];  // max over problems of ceil(I_n/kP1Rows)*nsplit
  int max_R;
  int max_Phat;
  int any_f64;      // tensors are FP64
  int dtype;
  int64_t max_P;
};

cudaError_t launch_init_state(const Prob* probs, int B, cudaStream_t s);
cudaError_t launch_init_factors(const Prob* probs, const GridInfo& g, int from_a64, cudaStream_t s);
cudaError_t launch_sample_contract(const Prob* probs, const GridInfo& g, int n, cudaStream_t s);
cudaError_t launch_solve(const Prob* probs, const GridInfo& g, int n, cudaStream_t s);
cudaError_t launch_finalize(const Prob* probs, const GridInfo& g, int n, cudaStream_t s);
cudaError_t launch_fit_setup(const Prob* probs, const GridInfo& g, cudaStream_t s);
cudaError_t launch_fit(const Prob* probs, const GridInfo& g, cudaStream_t s);
cudaError_t launch_loop_cond(const Prob* probs, int B, int* loop_iter, int cap, unsigned long long cond_handle,
                             cudaStream_t s);
cudaError_t prepare_kernel_attributes();
// the whole iteration loop in thread-block clusters (small problems)
int cluster_smem_bytes(const Prob* probs_host, int B, int C);
int cluster_capacity(int dtype, int C, int smem, int maxR);
cudaError_t launch_cluster_run(const Prob* probs, int B, int* queue, int dtype, int C, int smem, int nclusters,
                               int maxR, cudaStream_t s);
// the whole iteration loop over the whole GPU (cooperative launch, grid barriers), one problem at
// a time: large FP32 / BF16 problems
int grid_capacity(int dtype, int maxR);
bool grid_fits(const Prob& p, int G);
cudaError_t launch_grid_run(const Prob* probs, int B, const GridScratch& gs, int dtype, int maxR, int G,
                            cudaStream_t s);
// the whole iteration loop in 16-CTA clusters with every factor replicated in each CTA (the first
// choice when every problem of the call fits)
int loop_rep_smem_bytes(const Prob* probs_host, int B);
int loop_rep_capacity(int dtype, int smem, int maxR);
cudaError_t launch_loop_rep(const Prob* probs, int B, int* queue, int dtype, int smem, int nclusters, int maxR,
                            cudaStream_t s);
cudaError_t launch_sumsq(const void* X, int dtype, int64_t P, double* part, int nblk, cudaStream_t s,
                         unsigned* amax = nullptr);
cudaError_t launch_sumsq_finish(const double* part, int nblk, double* out_norm, State* st,
                                int nstates, cudaStream_t s);
// ||X|| reduction: at most kSumsqMaxBlocks partial sums.  A fixed cap (not the device's SM count)
// keeps the summation order, and so the result, the same on every device.
constexpr int kSumsqMaxBlocks = 1216;
int sumsq_blocks(int64_t P);
// a first level for many sum-of-squares partials: part[0 .. nblk) into sumsq_partials_blocks(nblk)
// sums (fixed order), for launch_sumsq_finish
int64_t sumsq_partials_blocks(int64_t nblk);
cudaError_t launch_sumsq_partials(const double* part, int64_t nblk, double* out, cudaStream_t s);

// step hooks
cudaError_t launch_sample_only(const void* X, int N, const int64_t* dims, int n, int64_t S,
                               uint64_t seed, uint32_t b, uint32_t t, uint32_t* idx, int64_t* off,
                               cudaStream_t s);
cudaError_t launch_gather_only(const void* X, int dtype, int64_t I, int64_t st, int64_t S,
                               const int64_t* off, void* out, cudaStream_t s);

// mode-n unfolding X_(n) stored column-major (a batched transpose)
cudaError_t launch_unfold_copy(const void* X, void* Y, int dtype, int N, const int64_t* dims, int n, cudaStream_t s);

// Storage offset of the first entry of the mode-n fiber with multi-index idx (mode-n slot ignored),
// and the stride between its entries, in the copy a mode-n gather reads.
__device__ __forceinline__ int64_t fiber_offset(const Prob& p, int n, const uint32_t* idx_by_mode, int64_t* stride) {
  int64_t off = 0;
  const int64_t In = p.dims[n];
  for (int m = 0; m < p.N; ++m) {
    if (m == n) continue;
    const int64_t w = (p.use_rep && m < n) ? p.st[m] * In : p.st[m];
    off += (int64_t)idx_by_mode[m] * w;
  }
  *stride = p.use_rep ? 1 : p.st[n];
  return off;
}

// CP-ALS (Alg. 1); every launch serves problem 0 of the table (CP-ALS runs one problem per call)
int mttkrp_rank_groups(int R);
int mttkrp_tile_rows(int rg, int dtype);
int mttkrp_tile_cols(int rg, int dtype);
cudaError_t launch_als_gram(const Prob* probs, const Prob& hp, int n, cudaStream_t s);
cudaError_t launch_als_prep(const Prob* probs, const Prob& hp, int n, cudaStream_t s);
cudaError_t launch_mttkrp(const Prob* probs, const Prob& hp, int n, cudaStream_t s);
cudaError_t launch_als_solve(const Prob* probs, const Prob& hp, int n, cudaStream_t s);
// M == nullptr: into the problem's Mfold buffer
cudaError_t launch_mttkrp_fold(const Prob* probs, const Prob& hp, int n, double* M, cudaStream_t s);
cudaError_t prepare_als_attributes();
constexpr int kAlsRows = 32;       // factor rows per block of the CP-ALS solve and Gram kernels

// mixing on the tensor cores (FP32 tensors, I_n a multiple of 4)
bool mix_tc_supported(int dtype, int I);
cudaError_t launch_split_tf32(const float* w, float* hi, float* lo, int64_t n, cudaStream_t s);
cudaError_t launch_mix_tc(const float* U, float* ystd, float* yunf, float* ynext, const float* Whi, const float* Wlo,
                          int N, const int64_t* dims, int n, int three_x, int* err, cudaStream_t s);

// mixing with FP16 operand halves (FP32 tensors, every I_n a multiple of 8)
bool mix_tc16_supported(int dtype, int I);
cudaError_t launch_split_f16(const float* w, void* out16, int64_t n, cudaStream_t s);
cudaError_t launch_absmax(const void* X, int dtype, int64_t P, unsigned* out, cudaStream_t s);
cudaError_t launch_mix_tc16(const float* U, float* ystd, float* yunf, float* ynext, const void* W16, int N,
                            const int64_t* dims, int n, const unsigned* amax_in, unsigned* amax_out, int* err,
                            cudaStream_t s);

// mixing by the factored DCT-II (FP32 / BF16 tensors whose every I_n factors into 2, 3, 5, 7):
// pass n reads the mode-n unfolding and writes the mode-(n+1 mod N) unfolding (the last pass: the
// standard layout, and its own layout into ysame when given); tab = 5 I floats (twiddles,
// post-scales, signs) from launch_build_mix_ops
bool mix_fft_supported(int dtype, int N, const int64_t* dims);
// the Bluestein tables of a length with a prime factor above 7 (7 I + 4 M floats from fft_tab on,
// after the 5 I DCT floats); nothing for a 7-smooth length
cudaError_t launch_build_bs_tables(int I, float* fft_tab, cudaStream_t s);
// whether the first pass's per-CTA sums of squares and their first-level sums (8 bytes each) fit
// in one tensor-sized buffer of this dtype
bool mix_fft_norm_fits(int dtype, int N, const int64_t* dims);
// normpart: when given, one FP64 sum of squares of the pass's input per CTA (nblocks of them, the
// count returned through nblocks), for launch_sumsq_finish
cudaError_t launch_mix_fft(const void* U, void* yv, void* ysame, const float* tab, int dtype, int N,
                           const int64_t* dims, int n, int* err, cudaStream_t s, double* normpart = nullptr,
                           int64_t* nblocks = nullptr);
int mix_engine();   // CPR_MIX_* (process-wide, cpr_set_mix_engine)
// the unitary DFT passes of the complex form (Alg. 4): complex (float2) output; the first pass reads
// the real FP32 tensor (real_in), later passes complex input; tab as for launch_mix_fft
bool mix_cfft_supported(int N, const int64_t* dims);
cudaError_t launch_mix_cfft(const void* U, bool real_in, void* yv, void* ysame, const float* tab, int N,
                            const int64_t* dims, int n, int* err, cudaStream_t s);

// CPRAND-MIX in its complex form (Alg. 4), k_mixc.cu
cudaError_t launch_cf_ops(int I, const double* signs, float2* W, cudaStream_t s);
cudaError_t launch_cf_init(int I, int R, int m, uint64_t seed, uint32_t b, double* A, cudaStream_t s);
cudaError_t launch_cf_mix_factor(int I, int R, const float2* W, const double* A, float2* Ah, cudaStream_t s);
cudaError_t launch_cf_update(const float2* Xn, const uint32_t* idx, const float2* W, const float2* const* Ah,
                             int N, const int64_t* dims, int n, int S, int R, float* Xr, double* Zr, double* G,
                             double* Gi, double* M, double* A, double* lam, int* bad, cudaStream_t s);
cudaError_t launch_cf_fit_setup(const float* X, int N, const int64_t* dims, int R, int P_hat, uint64_t seed,
                                uint32_t b, uint32_t* idx, double* xv, cudaStream_t s);
int cf_fit_blocks(int P_hat);
cudaError_t launch_cf_fit(const double* const* A, const double* lam, int N, const int64_t* dims, int R, int P_hat,
                          const uint32_t* idx, const double* xv, double* part, cudaStream_t s);

// mixing (Alg. 5)
cudaError_t launch_build_mix_ops(int I, uint64_t seed, uint32_t b, int n, double* table, float* W32,
                                 double* W64, double* F64, double* signs, cudaStream_t s, float* fft_tab = nullptr);
cudaError_t launch_mix_mode(const void* X, void* Y, int dtype, int N, const int64_t* dims, int n,
                            const float* W32, const double* W64, cudaStream_t s);
cudaError_t launch_unmix(const double* Ahat, double* A, const double* F64, const double* signs,
                         int I, int R, cudaStream_t s);
struct UnmixArgs {        // every mode of one problem: A[n] = D_n F_n^T Ahat[n]
  const double* Ahat[kMaxOrder];
  double* A[kMaxOrder];
  const double* F[kMaxOrder];
  const double* sg[kMaxOrder];
  int I[kMaxOrder];
  int first_block[kMaxOrder];   // filled by the launcher
  int N, R;
};
cudaError_t launch_unmix_all(const UnmixArgs& u, cudaStream_t s);

}  // namespace cpr
