/*
 * cprand.h -- C ABI of the GB300 (sm_103a) CPRAND / CPRAND-MIX library.
 *
 * Randomized CP tensor decomposition after Battaglino, Ballard and Kolda, "A Practical
 * Randomized CP Tensor Decomposition" (SIAM J. Matrix Anal. Appl., 2018; arXiv 1701.06600).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 *  - A dense order-N tensor is stored column-major: entry (i_1, ..., i_N) (0-based) lives at
 *    offset sum_n i_n * st_n with st_n = prod_{m<n} I_m, i.e. i_1 varies fastest.  This is the
 *    order the mode-n unfolding of Sec. 2.1 assumes.  Offsets are 64-bit.
 *  - Modes are 0-based in this API (mode n here is mode n+1 in the paper).
 *  - Factor matrices A^(n) are I_n x R, row-major (the R entries of a row are contiguous), FP64.
 *    lambda holds the R component weights of the normalized model (Sec. 2.1, eq. cpform+lambda).
 *  - Every pointer inside cpr_tensor / cpr_ktensor and every buffer argument named *_dev or ws is
 *    DEVICE memory owned by the caller.  The library allocates no device memory: scratch space is
 *    the caller's workspace `ws` of at least cpr_workspace_size(...) bytes (256-byte aligned).
 *  - All device work is enqueued on the caller's `stream` (a cudaStream_t passed as void*; NULL
 *    means the legacy default stream).  Step entry points return right after enqueueing.  The
 *    whole-algorithm entry points (cpr_cp_als, cpr_cprand, cpr_cprand_mix, cpr_cprand_batched) synchronize
 *    the stream once at the end to fill cpr_result.
 *  - Return value: CPR_OK (0) or a CPR_E* status.  Arguments are checked on the host before any
 *    work is enqueued; a failed check enqueues nothing.  Device-detected conditions (a
 *    non-positive-definite Gram matrix, a non-finite fit) are reported through cpr_result.status.
 *    Nothing on the device traps.
 *  - Random quantities are Philox4x32-10 draws keyed by the 64-bit seed; counter words are
 *    (item, (stream << 8) | (block << 4) | mode, iteration or column group, batch index), with
 *    stream 0 = least-squares samples, 1 = fit entries, 2 = initial factors, 3 = mixing signs.
 *    An index in [0, I) is floor(w * I / 2^32); a uniform value is (w >> 8) * 2^-24; a sign is
 *    +1 when the low bit of w is 0.
 */
#ifndef CPRAND_H
#define CPRAND_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#if defined(__GNUC__)
#define CPR_API __attribute__((visibility("default")))
#else
#define CPR_API
#endif

#define CPR_MAX_ORDER 8
#define CPR_MAX_RANK 64

typedef enum { CPR_F64 = 0, CPR_F32 = 1, CPR_BF16 = 2 } cpr_dtype;

enum {
  CPR_OK = 0,
  CPR_EINVAL = 1,      /* bad argument: order, rank, S < R, dims, dtype, null pointer, ... */
  CPR_EWORKSPACE = 2,  /* ws_bytes smaller than cpr_workspace_size() or ws misaligned */
  CPR_ESINGULAR = 3,   /* Gram matrix (Z_S^T Z_S, or Z^T Z for CP-ALS) not positive definite */
  CPR_ENONFINITE = 4,  /* a NaN or Inf reached the fit estimate */
  CPR_ETIMEOUT = 5,    /* a bounded device-side wait expired */
  CPR_ECUDA = 6        /* a CUDA runtime call failed */
};

/* Methods for cpr_workspace_size. */
enum {
  CPR_METHOD_CPRAND = 0,
  CPR_METHOD_CPRAND_MIX = 1,
  CPR_METHOD_UPDATE = 2,   /* cpr_sampled_update */
  CPR_METHOD_FIT = 3,      /* cpr_fit_estimate */
  CPR_METHOD_NORM = 4,     /* cpr_tensor_norm */
  CPR_METHOD_CP_ALS = 5,   /* cpr_cp_als (S ignored) */
  CPR_METHOD_MTTKRP = 6    /* cpr_mttkrp (S ignored; the size does not depend on the mode) */
};

typedef struct {
  const void* data;              /* device, column-major */
  int32_t dtype;                 /* cpr_dtype */
  int32_t order;                 /* N, 2 .. CPR_MAX_ORDER */
  int64_t dims[CPR_MAX_ORDER];   /* I_1 .. I_N, each >= 1 and < 2^31 */
} cpr_tensor;

typedef struct {
  int32_t order;
  int32_t rank;                  /* R, 1 .. CPR_MAX_RANK */
  int64_t dims[CPR_MAX_ORDER];
  double* lambda;                /* device, R */
  double* factors[CPR_MAX_ORDER];/* device, factor n is I_n x R row-major */
} cpr_ktensor;

typedef struct {
  int32_t max_iters;     /* outer-iteration cap (Sec. 4.2: 200) */
  int32_t fixed_iters;   /* > 0: run exactly this many outer iterations, no other rule */
  double fit_tol;        /* stop when |F_t - F_{t-1}| <= fit_tol, from the 2nd iteration (1e-4) */
  double noise_eta;      /* >= 0: stop when F_t >= 1 - 1.2 eta (Sec. 4.2); < 0: rule off */
  int32_t stall_iters;   /* > 0: stop when the best fit has not improved for this many iters */
  int32_t init_from_out; /* 1: the initial factors of modes 2..N are read from out->factors
                            (mixed basis for cpr_cprand_mix); 0: Philox U[0,1) */
  int64_t fit_samples;   /* P_hat, entries of the sampled fit (Sec. 3.4: 2^14) */
  uint64_t seed;         /* Philox key */
  uint32_t batch_index;  /* counter word 3 (decomposition index inside a batch) */
  uint32_t first_iter;   /* counter word 2 of the first outer iteration (resume) */
  double* fit_trace_dev; /* device, >= max(max_iters, fixed_iters) doubles, or NULL */
  int32_t loop_path;     /* how the outer iterations are launched: 0 automatic (a thread-block
                            cluster per problem when every problem of the call fits one with its
                            factors replicated in each CTA, or, for a single problem, with them
                            distributed over the CTAs; else the captured graph); 1 clusters (every factor replicated in each CTA's
                            shared memory when every problem fits that layout, else each factor's
                            rows distributed over the CTAs; CPR_EINVAL if a problem fits neither);
                            2 captured graph; 3 plain stream launches; 4 clusters with distributed
                            factor rows only; 5 the whole GPU (one cooperative launch of one CTA per
                            SM, grid-wide barriers between the phases of a mode update; single
                            FP32 / BF16 problems with every I_n <= 32 x the SM count, CPR_EINVAL
                            otherwise).  Automatic choice for a single problem that does not fit
                            the replicated-factor cluster: the whole GPU when it fits, else the
                            distributed-factor cluster, else the graph.  Read from the first
                            problem's options in a batched call. */
  int32_t layout;        /* 0: before iterating, also store every mode-n unfolding X_(n) as its own
                            column-major copy (N-1 extra copies of the tensor in the workspace) so
                            that every sampled fiber is read contiguously; 1: gather every mode
                            from the single tensor (fibers of modes 2..N are strided) */
  const uint32_t* user_samples; /* test hook, device, or NULL: the sample multi-indices to use in
                            place of the Philox draws, N x user_S x N uint32 (entry
                            (n * user_S + j) * N + m is i_m of sample j of every mode-n update;
                            the mode-n slot is ignored; every index must be below I_m).  Requires
                            S == user_S; the iterations run on the captured graph (loop_path 0 or
                            2; 3 and 5 are also accepted).  With every multi-index of the other
                            modes listed once, the update is the exact ALS update of Alg. 1. */
  int64_t user_S;
  int64_t wait_budget;   /* polls of each wait at a grid-wide barrier of the whole-GPU loop
                            (loop_path 5; a poll is one acquire load and a 32 ns sleep); 0: the
                            library default (2^22 polls, on the order of a second).  A wait that
                            runs out makes every CTA leave at its next barrier and the call return
                            CPR_ETIMEOUT (that kernel issues no asynchronous copies).  The waits on
                            TMA copies (cluster loops, mixing kernels) keep the library's fixed
                            limits; after one runs out the kernel waits again, bounded, for its own
                            copies before it returns, and the call reports CPR_ETIMEOUT. */
} cpr_opts;

typedef struct {
  int32_t iters;         /* outer iterations run */
  int32_t status;        /* CPR_OK or a device-detected CPR_E* */
  double fit_est;        /* last sampled fit estimate */
  double norm_x;         /* ||X|| (Frobenius) */
  int64_t kernel_launches; /* kernels this call put on the GPU */
  double ms_setup;       /* device time of ||X||, mixing, initial factors and fit-set setup */
  double ms_iterate;     /* device time of the outer iterations (wall time between two events) */
  double ms_finish;      /* device time of unmixing and output copies */
} cpr_result;

/* Contraction engine of the whole-GPU loop (loop_path 5; process-wide, applies to calls enqueued
 * afterwards): CPR_CONTRACT_AUTO and CPR_CONTRACT_TC compute M = X_S Z_S (Alg. 3) on the tensor cores
 * (tcgen05, kind::tf32, each FP32 operand split into two TF32 values rounded to nearest,
 * hi = tf32(x) and lo = tf32(x - hi): hi*hi + hi*lo + lo*hi accumulated in FP32 in TMEM, about
 * 3 * 2^-22 relative per product; BF16 tensor values are exact TF32 values, so their lo*hi term is
 * zero and is skipped); CPR_CONTRACT_FMA by FP32 FMA.  Returns the previous
 * engine, or -1 (nothing changed) for an unknown value. */
enum { CPR_CONTRACT_AUTO = 0, CPR_CONTRACT_TC = 1, CPR_CONTRACT_FMA = 2 };
CPR_API int cpr_set_contract_engine(int engine);

/* A schedule of the iteration loop, as chosen by the autotuner. */
typedef struct {
  int32_t loop_path;      /* cpr_opts.loop_path value of the chosen engine (1, 2, 4 or 5) */
  int32_t split_per_sm;   /* graph engine: (fiber tile, sample split) blocks per SM per mode update */
  int32_t grid_min_split; /* whole-GPU engine: fewest samples per contraction split */
  int32_t pad;
  double ms_per_iter;     /* device time per outer iteration when it was tuned */
} cpr_schedule;

/* Kernel classes of the profiler. */
enum {
  CPR_KERNEL_MIX = 0,        /* mode-n mixing product (Alg. 5 mixing step) */
  CPR_KERNEL_SAMPLE_SKR = 1, /* sampler + sampled Khatri-Rao rows + partial Grams */
  CPR_KERNEL_CONTRACT = 2,   /* fiber gather fused with X_S Z_S */
  CPR_KERNEL_CHOL = 3,       /* Gram reduction + Cholesky */
  CPR_KERNEL_SOLVE = 4,      /* row solves */
  CPR_KERNEL_NORMALIZE = 5,  /* column normalization */
  CPR_KERNEL_FIT = 6,        /* sampled fit + stopping test */
  CPR_KERNEL_OTHER = 7,      /* setup, norm, unmixing */
  CPR_KERNEL_LOOP = 8,       /* whole iteration loop in one thread-block cluster per problem */
  CPR_KERNEL_CLASSES = 9
};

/* Fill *opts with the paper's defaults (Sec. 4.2): max_iters 200, fit_tol 1e-4, noise rule off,
 * no stall rule, P_hat = 2^14, seed 0, random initial factors. */
CPR_API void cpr_default_opts(cpr_opts* opts);

/* Text for a status code; never NULL. */
CPR_API const char* cpr_status_string(int status);

/* S = 10 R ln R rounded to nearest (Sec. 3.2; Sec. 4.2 prints S = 80 for R = 5, 108 for R = 6). */
CPR_API int64_t cpr_sample_size(int R);

/* Bytes of workspace the given method needs for tensor X, rank R and S samples; 0 on a bad
 * argument.  For CPR_METHOD_FIT, S is ignored and opts->fit_samples sizes the fit set. */
CPR_API size_t cpr_workspace_size(int method, const cpr_tensor* X, int R, int64_t S, const cpr_opts* opts);

/* ---------------------------------------------------------------------------------------------
 * Whole algorithms
 * ------------------------------------------------------------------------------------------- */

/* CP-ALS (Alg. 1): the exact alternating least squares the randomized methods approximate.  Each
 * outer iteration updates modes 1..N in turn: M = X_(n) Z^(n) (the exact MTTKRP over every entry of
 * X, with Z^(n) the Khatri-Rao product of the other factors, built tile by tile and never stored),
 * V = Hadamard product of the other factors' Grams A^(m)T A^(m) (Sec. 2.1), A^(n) = M V^-1 by an FP64
 * Cholesky of V (Alg. 1 writes the pseudoinverse; a V that is not positive definite stops the run
 * with CPR_ESINGULAR in result->status), then column normalization into lambda.  After each outer
 * iteration the exact fit 1 - ||X - X~|| / ||X|| (Sec. 4.2) is formed from the last MTTKRP and the
 * Grams, ||X - X~||^2 = ||X||^2 - 2 <X, X~> + ||X~||^2, without another pass over X, and drives the
 * stopping rules (opts->fit_tol, max_iters, fixed_iters, noise_eta, stall_iters) on the device;
 * result->fit_est holds that exact fit.  The MTTKRP multiplies in FP32 and sums in FP32 over at most
 * 256 columns of X_(n) before folding into FP64 (FP64 throughout for an FP64 tensor); the Grams,
 * solve, normalization and fit are FP64.  Before iterating, the call stores the mode-n unfoldings
 * X_(n), n >= 2, as column-major copies in the workspace (N-1 extra copies of the tensor).  Initial
 * factors of modes 2..N: Philox U[0,1) (stream 2, as cpr_cprand) or out->factors with
 * opts->init_from_out.  opts->S-related fields and fit_samples are ignored; loop_path 3 launches
 * every kernel from the host, any other value runs the iterations as one captured graph. */
CPR_API int cpr_cp_als(const cpr_tensor* X, int R, const cpr_opts* opts, cpr_ktensor* out,
                       cpr_result* result, void* ws, size_t ws_bytes, void* stream);

/* CPRAND (Alg. 3): randomized ALS.  Each outer iteration updates modes 1..N in turn; the mode-n
 * update draws S fresh multi-indices, builds the sampled Khatri-Rao rows Z_S (Alg. 2), gathers
 * the matching mode-n fibers X_S, solves min ||Z_S A^T - X_S^T|| through the R x R normal
 * equations (FP64 Gram and Cholesky; the contraction X_S Z_S accumulates in FP32, or FP64 for an
 * FP64 tensor) and normalizes the columns into lambda.  After each outer iteration the sampled
 * fit of Sec. 3.4 (fixed P_hat entries) drives the stopping rules of Sec. 4.2 on the device.
 * Output: out->lambda and out->factors (normalized columns).  out->order/rank/dims must match X
 * and R.  S >= R. */
CPR_API int cpr_cprand(const cpr_tensor* X, int R, int64_t S, const cpr_opts* opts, cpr_ktensor* out,
               cpr_result* result, void* ws, size_t ws_bytes, void* stream);

/* CPRAND-MIX in its real-transform form (Alg. 5, "CPRAND-PREMIX"): mix every mode with F_n D_n
 * (D_n Philox signs, F_n the orthonormal DCT-II), run CPRAND on the mixed tensor (held in the
 * workspace; X itself is not modified), then unmix A^(n) = D_n F_n^T A^^(n).  The stopping test
 * runs on the mixed tensor, whose norm equals ||X||. */
CPR_API int cpr_cprand_mix(const cpr_tensor* X, int R, int64_t S, const cpr_opts* opts, cpr_ktensor* out,
                   cpr_result* result, void* ws, size_t ws_bytes, void* stream);

/* Many independent decompositions at once (the paper's multiple random starts, Sec. 4.2): B
 * problems of any shapes and ranks (all of the same order and dtype) advance together, every
 * kernel launch serving all of them; each stops on its own rule.  opts[b].batch_index should be
 * b.  mix != 0 runs CPRAND-MIX for every problem.  Workspace from cpr_batched_workspace_size. */
CPR_API size_t cpr_batched_workspace_size(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss,
                                  const cpr_opts* opts, int mix);
CPR_API int cpr_cprand_batched(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss,
                       const cpr_opts* opts, int mix, cpr_ktensor* outs, cpr_result* results,
                       void* ws, size_t ws_bytes, void* stream);
/* cpr_cprand_batched with mix = 1: B independent CPRAND-MIX decompositions (Alg. 5) at once. */
CPR_API int cpr_cprand_mix_batched(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss,
                                   const cpr_opts* opts, cpr_ktensor* outs, cpr_result* results, void* ws,
                                   size_t ws_bytes, void* stream);

/* ---------------------------------------------------------------------------------------------
 * Steps of the hot path (each is also a parity-test hook)
 * ------------------------------------------------------------------------------------------- */

/* Sampled multi-indices of one mode update (Alg. 3, "define sampling operator"): for samples
 * j < S, idx_dev[j*N + m] = i_m^(j) for m != mode (idx_dev[j*N + mode] = 0), drawn from Philox
 * stream 0 with counter (j, mode, t, b); off_dev[j] = sum_{m != mode} i_m st_m, the storage
 * offset of the first entry of the sampled fiber (Sec. 2.1 index map).  Either output may be
 * NULL.  idx_dev: S*N uint32; off_dev: S int64. */
CPR_API int cpr_sample_indices(const cpr_tensor* X, int mode, int64_t S, uint64_t seed, uint32_t b,
                       uint32_t t, uint32_t* idx_dev, int64_t* off_dev, void* stream);

/* Fiber gather X_S = (S X_(n)^T)^T (Sec. 3.2): xs_dev[i + I_n * j] = X[off_dev[j] + i * st_mode]
 * for i < I_n, j < S, a bit copy in X's dtype (I_n x S, column-major).  Fibers of stride 1 (mode 0,
 * which also covers a mode-n unfolding stored column-major and described with mode n's extent
 * first) are copied one warp per fiber with 16-byte vectors where the fiber's start, its
 * destination and its length allow it; strided fibers element by element. */
CPR_API int cpr_gather_fibers(const cpr_tensor* X, int mode, int64_t S, const int64_t* off_dev,
                      void* xs_dev, void* stream);

/* One mode-n update of Alg. 3: sample (seed, b, t), SKR, gather, contract, FP64 Gram +
 * Cholesky solve, normalize.  Reads K->factors[m] for m != mode (FP64; rounded to FP32 for the
 * contraction unless X is FP64), writes K->factors[mode] and K->lambda.  result may be NULL;
 * when given, this call synchronizes the stream and reports a singular Gram in result->status. */
CPR_API int cpr_sampled_update(const cpr_tensor* X, cpr_ktensor* K, int mode, int64_t S, uint64_t seed,
                       uint32_t b, uint32_t t, cpr_result* result, void* ws, size_t ws_bytes,
                       void* stream);

/* Exact MTTKRP (Alg. 1, the right-hand side of the mode-n update): M_dev (I_mode x R, row-major FP64)
 * = X_(mode) Z^(mode) with Z^(mode) = A^(N) (.) ... (.) A^(mode+1) (.) A^(mode-1) (.) ... (.) A^(1)
 * over K->factors as given (lambda is not applied).  FP32 products and FP32 sums over at most 256
 * columns of X_(mode), folded into FP64 (FP64 throughout for an FP64 tensor).  For mode >= 1 the
 * call first stores X_(mode) column-major in the workspace. */
CPR_API int cpr_mttkrp(const cpr_tensor* X, const cpr_ktensor* K, int mode, double* M_dev, void* ws,
                       size_t ws_bytes, void* stream);

/* Sampled fit estimate (Sec. 3.4): F^ = 1 - sqrt(P * mean_i e_i^2) / ||X|| over P_hat entries
 * drawn from Philox stream 1 (seed, b), e_i = x_i - sum_r lambda_r prod_n A^(n)(i_n, r).  norm_x
 * < 0 computes ||X|| first.  Writes the estimate to *fit_host (synchronizes the stream). */
CPR_API int cpr_fit_estimate(const cpr_tensor* X, const cpr_ktensor* K, int64_t P_hat, uint64_t seed,
                     uint32_t b, double norm_x, double* fit_host, void* ws, size_t ws_bytes,
                     void* stream);

/* Mixing preprocess (Alg. 5, mixing step): out_dev = X x_1 F_1 D_1 ... x_N F_N D_N, mode 1
 * first, in X's dtype and layout.  FP32 and BF16 tensors whose every I_n (>= 5) factors into 2, 3,
 * 5 and 7: each mode product is a factored DCT-II (a mixed-radix FFT of the reordered fiber in
 * shared memory, FP32 arithmetic, twiddles rounded from FP64 values, or products of two such values;
 * about 1e-7 relative; stage plans compiled in for I_n = 100, 400 and 1500).  Other
 * FP32 tensors: tensor-core dense products with both operands split into two halves (FP16 halves
 * scaled by powers of two when every I_n is a multiple of 8, else TF32 halves; about 2^-21 relative
 * per product) accumulated in FP32; other BF16 tensors: FP32 SIMT products; FP64 tensors: FP64.
 * BF16 results are rounded to BF16 after every mode product.  out_dev must not overlap X.  ws from
 * cpr_workspace_size(CPR_METHOD_CPRAND_MIX, ...) is enough. */
CPR_API int cpr_mix_tensor(const cpr_tensor* X, void* out_dev, uint64_t seed, uint32_t b, void* ws,
                   size_t ws_bytes, void* stream);

/* Unmixing (Alg. 5, last step): out->factors[n] = D_n F_n^T Khat->factors[n] (FP64), lambda
 * copied.  Khat and out may not share factor buffers. */
CPR_API int cpr_unmix_factors(const cpr_ktensor* Khat, cpr_ktensor* out, uint64_t seed, uint32_t b,
                      void* ws, size_t ws_bytes, void* stream);

/* CPRAND-MIX in its complex form (Alg. 4), the paper's experimental variant: every mode is mixed with
 * F_n D_n, F_n the unitary DFT (D_n the Philox signs of cpr_cprand_mix), so the mixed tensor is
 * complex; the factors stay real.  A mode-n update unmixes the S sampled fibers of the mixed tensor
 * in mode n (D_n F_n^* per fiber), forms the sampled rows of the Khatri-Rao product of the mixed
 * factors F_m D_m A^(m), and solves the least squares over real A^(n) by stacking real and imaginary
 * parts (eq. (rcLS)); then normalizes and mixes the new factor.  Samples, initial factors and fit
 * entries use the Philox streams of cpr_cprand_mix; the stopping rules of Sec. 4.2 are checked on the
 * host after each outer iteration (the sampled fit on X with the real factors).
 *   X: FP32, every I_n in [5, 6000] a product of 2, 3, 5 and 7; R <= CPR_MAX_RANK; S >= R.
 *   out: caller-owned real factors (I_n x R, FP64) and lambda, returned normalized in the original
 *   basis (no unmixing step).  opts->init_from_out must be 0.  ws: at least
 *   cpr_cprand_mix_fft_workspace_size(...) bytes (about (N + 1) complex copies of the tensor).
 * Returns CPR_EINVAL for unsupported shapes or types; device-detected conditions (singular Gram,
 * non-finite fit) in result->status.  Synchronizes the stream once per outer iteration. */
CPR_API size_t cpr_cprand_mix_fft_workspace_size(const cpr_tensor* X, int R, int64_t S, const cpr_opts* opts);
CPR_API int cpr_cprand_mix_fft(const cpr_tensor* X, int R, int64_t S, const cpr_opts* opts, cpr_ktensor* out,
                               cpr_result* result, void* ws, size_t ws_bytes, void* stream);

/* Mixing engine (process-wide; applies to cpr_mix_tensor and to every CPRAND-MIX call enqueued
 * afterwards): CPR_MIX_AUTO takes the factored DCT where it applies (see cpr_mix_tensor), else the
 * dense products; CPR_MIX_DENSE always takes the dense products (the tensor-core kernels for FP32);
 * CPR_MIX_FFT is AUTO (the factored transform is used only where it applies).  Returns the previous
 * engine, or -1 (nothing changed) for an unknown value.  Both engines compute the same operator
 * F_n D_n; they differ in rounding only. */
enum { CPR_MIX_AUTO = 0, CPR_MIX_FFT = 1, CPR_MIX_DENSE = 2 };
CPR_API int cpr_set_mix_engine(int engine);

/* Kernel profiler (process-wide, host-side bookkeeping only).  After cpr_profile_begin(mask),
 * every launch of a kernel class whose bit is set in mask is bracketed by a pair of CUDA events
 * recorded on the launching stream; cpr_profile_end synchronizes those events and returns, per
 * class c, the summed device time ms[c] and the launch count launches[c] (arrays of
 * CPR_KERNEL_CLASSES entries, either may be NULL), then stops recording.  Events are created by
 * the profiler; no device memory is allocated.  Launch counts are kept for every class whether or
 * not its bit is set.  Not thread-safe against concurrent begin/end. */
CPR_API int cpr_profile_begin(unsigned mask);
CPR_API int cpr_profile_end(double* ms, int64_t* launches);

/* Sampled fit estimate for callers that cannot allocate device memory when they need it (a plugin
 * restricted to memory its host application owns, a process whose device memory belongs to another
 * allocator, a latency-critical path).  The paper has no counterpart: this is the computation of
 * cpr_fit_estimate (same Philox fit entries; the model is evaluated in FP64 from the FP64 factors)
 * with its scratch in one fixed array of device memory declared by the library (about 42 KB per
 * device, held until the process exits) instead of a caller workspace.  It allocates nothing.
 * P_hat must be in [1, CPR_NOALLOC_MAX_FIT_SAMPLES]; a larger P_hat is rejected with CPR_EINVAL
 * before anything is enqueued.  norm_x < 0 computes ||X|| in the same array.  Every call on a
 * device shares the array (each call clears what must start at zero): calls whose work overlaps on
 * the GPU race and must be ordered by the caller.  The first call on each device looks up the
 * array's device address (cudaGetSymbolAddress) with that device current.  Every call synchronizes
 * the stream and copies the estimate into *fit_host, so it cannot be recorded into a graph: on a
 * stream that is being captured it returns CPR_EINVAL and enqueues nothing.  Its launches are not
 * counted or timed by the kernel profiler (cpr_profile_begin / cpr_profile_end). */
#define CPR_NOALLOC_MAX_FIT_SAMPLES (1 << 20)
CPR_API int cpr_fit_estimate_noalloc(const cpr_tensor* X, const cpr_ktensor* K, int64_t P_hat, uint64_t seed,
                                     uint32_t b, double norm_x, double* fit_host, void* stream);

/* Schedule autotuner (no counterpart in the paper; an implementation aid for the batched starts of
 * Sec. 4.2 and the large single problems).  cpr_autotune runs the given batch (arguments as for
 * cpr_cprand_batched, every problem with fixed_iters = trial_iters, no trace, no caller samples) once
 * with the default schedule (warm-up) and once per candidate: the replicated- and distributed-factor
 * clusters, the whole-GPU loop with 16, 32 and 64 samples at least per contraction split, and the
 * captured graph with 1, 2 and 4 blocks per SM per mode update; candidates that do not apply to the
 * batch are skipped.  The schedule with the least device time per outer iteration is recorded for the
 * batch's bucket -- dtype, order, batch size, mixing, and per mode the largest extent, the rank and
 * the sample count, each rounded (extents and S to the next power of two, R to the next multiple
 * of 8) -- and returned in *best.  Every later call in this process whose loop_path is 0 and whose
 * batch falls in a recorded bucket runs with the recorded schedule.  The outputs and the workspace
 * are those of cpr_cprand_batched (they hold the last candidate's result afterwards).  Synchronizes
 * the stream after every candidate.
 * cpr_tune_lookup: the recorded schedule of a batch's bucket (CPR_EINVAL when there is none).
 * cpr_tune_save / cpr_tune_load: write the table to a text file (one bucket per line) / add a file's
 * buckets to it; the file named by the environment variable CPRAND_TUNE_CACHE is loaded on the
 * first lookup.  cpr_tune_clear: empty the table.  Host-side only; not thread-safe against
 * concurrent tuning of the same bucket. */
CPR_API int cpr_autotune(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss, const cpr_opts* opts, int mix,
                         cpr_ktensor* outs, void* ws, size_t ws_bytes, void* stream, int trial_iters,
                         cpr_schedule* best);
CPR_API int cpr_tune_lookup(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss, int mix, cpr_schedule* out);
CPR_API int cpr_tune_save(const char* path);
CPR_API int cpr_tune_load(const char* path);
CPR_API void cpr_tune_clear(void);

/* ||X||_F (FP64 accumulation) written to *norm_host (synchronizes the stream). */
CPR_API int cpr_tensor_norm(const cpr_tensor* X, double* norm_host, void* ws, size_t ws_bytes,
                    void* stream);

#ifdef __cplusplus
}
#endif

#endif /* CPRAND_H */
