// C-ABI entry points of libcprand (declared in include/cprand.h): argument checks, workspace
// layout, and the order of kernel launches.  No device memory is allocated here; every buffer is
// carved out of the caller's workspace.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <atomic>
#include <map>
#include <mutex>
#include <string>
#include <vector>

#include "internal.cuh"

using namespace cpr;

namespace {
std::atomic<int> g_mix_engine{CPR_MIX_AUTO};
std::atomic<int> g_contract_engine{CPR_CONTRACT_AUTO};
}
int cpr::mix_engine() { return g_mix_engine.load(); }

namespace {

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

// Carves typed sub-buffers out of the workspace; with a null base it only measures.
struct Carver {
  char* base;
  size_t off = 0;
  explicit Carver(void* b) : base(static_cast<char*>(b)) {}
  template <class T> T* take(size_t count) {
    off = align256(off);
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += count * sizeof(T);
    return p;
  }
};

int elem_size(int dtype) { return dtype == CPR_F64 ? 8 : (dtype == CPR_F32 ? 4 : 2); }

int check_tensor(const cpr_tensor* X, bool need_data) {
  if (!X) return CPR_EINVAL;
  if (X->order < 2 || X->order > CPR_MAX_ORDER) return CPR_EINVAL;
  if (X->dtype < CPR_F64 || X->dtype > CPR_BF16) return CPR_EINVAL;
  if (need_data && !X->data) return CPR_EINVAL;
  double P = 1.0;
  for (int n = 0; n < X->order; ++n) {
    if (X->dims[n] < 1 || X->dims[n] >= (int64_t(1) << 31)) return CPR_EINVAL;
    P *= (double)X->dims[n];
  }
  if (P > 4.0e18) return CPR_EINVAL;
  return CPR_OK;
}

int64_t prod_dims(const cpr_tensor* X) {
  int64_t P = 1;
  for (int n = 0; n < X->order; ++n) P *= X->dims[n];
  return P;
}

int check_rank_samples(int R, int64_t S) {
  if (R < 1 || R > CPR_MAX_RANK) return CPR_EINVAL;
  if (S < R || S > INT32_MAX) return CPR_EINVAL;
  return CPR_OK;
}

int check_ktensor(const cpr_ktensor* K, const cpr_tensor* X, int R) {
  if (!K || K->order != X->order || K->rank != R || !K->lambda) return CPR_EINVAL;
  for (int n = 0; n < X->order; ++n)
    if (K->dims[n] != X->dims[n] || !K->factors[n]) return CPR_EINVAL;
  return CPR_OK;
}

int check_ws(void* ws, size_t ws_bytes, size_t need) {
  if (need > 0 && !ws) return CPR_EWORKSPACE;
  if (reinterpret_cast<uintptr_t>(ws) % 256 != 0) return CPR_EWORKSPACE;
  if (ws_bytes < need) return CPR_EWORKSPACE;
  return CPR_OK;
}

#define CPR_CUDA(call)                 \
  do {                                 \
    cudaError_t e_ = (call);           \
    if (e_ != cudaSuccess) return CPR_ECUDA; \
  } while (0)

// ------------------------------------------------------------------------------------------------
// Kernel profiler and phase events.  Events come from a process-wide pool (created once, reused).
// ------------------------------------------------------------------------------------------------
struct ProfRec {
  int cls;
  cudaEvent_t a, b;
};

struct Profiler {
  std::mutex mu;
  bool on = false;
  unsigned mask = 0;
  std::vector<ProfRec> recs;
  int64_t counts[CPR_KERNEL_CLASSES] = {};
  std::vector<cudaEvent_t> pool;
};

Profiler& prof() {
  static Profiler p;
  return p;
}

cudaEvent_t take_event() {
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  if (!p.pool.empty()) {
    cudaEvent_t e = p.pool.back();
    p.pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  if (cudaEventCreate(&e) != cudaSuccess) return nullptr;
  return e;
}

void give_event(cudaEvent_t e) {
  if (!e) return;
  Profiler& p = prof();
  std::lock_guard<std::mutex> lk(p.mu);
  p.pool.push_back(e);
}

// Enqueue one kernel launch (a callable returning cudaError_t) of class cls; brackets it with
// profiler events when that class is being recorded.
template <class F>
int launch(int cls, cudaStream_t s, int64_t* launches, F&& f) {
  Profiler& p = prof();
  bool rec = p.on && ((p.mask >> cls) & 1u);
  if (rec) {
    // a launch recorded into a graph body runs later, many times: it cannot be timed with events
    cudaStreamCaptureStatus cst = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cst) != cudaSuccess) return CPR_ECUDA;
    rec = cst == cudaStreamCaptureStatusNone;
  }
  cudaEvent_t a = nullptr, b = nullptr;
  if (rec) {
    a = take_event();
    if (!a || cudaEventRecord(a, s) != cudaSuccess) return CPR_ECUDA;
  }
  if (f() != cudaSuccess) return CPR_ECUDA;
  if (rec) {
    b = take_event();
    if (!b || cudaEventRecord(b, s) != cudaSuccess) return CPR_ECUDA;
    std::lock_guard<std::mutex> lk(p.mu);
    p.recs.push_back(ProfRec{cls, a, b});
  }
  if (p.on) {
    std::lock_guard<std::mutex> lk(p.mu);
    p.counts[cls] += 1;
  }
  if (launches) *launches += 1;
  return CPR_OK;
}

#define CPR_LAUNCH(cls, expr)                                                  \
  do {                                                                         \
    int st_ = launch((cls), s, &launches, [&]() -> cudaError_t { return (expr); }); \
    if (st_) return st_;                                                       \
  } while (0)

// Four events bracketing the phases of a whole-algorithm call.
struct PhaseEvents {
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  PhaseEvents() {
    for (auto& x : e) x = take_event();
  }
  ~PhaseEvents() {
    for (auto& x : e) give_event(x);
  }
  int mark(int i, cudaStream_t s) { return (e[i] && cudaEventRecord(e[i], s) == cudaSuccess) ? CPR_OK : CPR_ECUDA; }
  double ms(int i, int j) const {
    float v = 0.f;
    if (!e[i] || !e[j] || cudaEventElapsedTime(&v, e[i], e[j]) != cudaSuccess) return NAN;
    return (double)v;
  }
};

// Mixing buffers of one problem.
struct MixBufs {
  float* W32[kMaxOrder] = {};
  float* Wlo[kMaxOrder] = {};   // tensor-core path: low tf32 halves (W32 then holds the high halves)
  double* W64[kMaxOrder] = {};
  double* F64[kMaxOrder] = {};
  double* sg[kMaxOrder] = {};
  double* table = nullptr; // cos(pi q / (2 I)), q < 4 I, reused mode after mode
  void* xhat = nullptr;   // mixed tensor
};

// A batch of problems laid out in the workspace.
struct Plan {
  int B = 0, mix = 0, dtype = 0;
  GridInfo g{};
  std::vector<Prob> probs;
  std::vector<MixBufs> mixb;
  Prob* d_probs = nullptr;
  State* d_states = nullptr;
  int* d_counter = nullptr;
  double* d_normpart = nullptr;
  void* d_tmp = nullptr;     // shared ping-pong buffer of the mixing passes
  void* d_tmp2 = nullptr;    // second pass buffer (tensor-core mixing reads unfoldings)
  int normblk = 0;
  GridScratch gscr{};        // whole-GPU loop (single FP32 / BF16 problems)
  bool has_grid = false;
  size_t bytes = 0;
};

struct ProbSpec {
  const cpr_tensor* X;
  int R;
  int64_t S;
  int64_t P_hat;
  const cpr_opts* opts;
  double* const* user_A64;   // non-null: factors live in caller buffers (step entry points)
  double* user_lambda;
};

// SMs of the current device (queried once per device).
int device_sms() {
  static int cache[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return 148;
  if (!cache[dev]) {
    int v = 0;
    if (cudaDeviceGetAttribute(&v, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || v < 1) v = 148;
    cache[dev] = v;
  }
  return cache[dev];
}

// A schedule: how the iteration loop is launched and the tile parameters the autotuner chooses.
struct Schedule {
  int loop_path = 0;        // cpr_opts.loop_path values; 0: the automatic rule
  int split_per_sm = 2;     // graph path: (tile, split) blocks per SM per mode update across the batch
  int grid_min_split = 16;  // whole-GPU loop: fewest samples per contraction split
};
constexpr int kMaxSplitPerSM = 4;   // the workspace is sized for the finest split a schedule may use

// Pick the sample split: enough (tile, split) blocks per mode update to give the GPU about per_sm
// blocks per SM across the batch, between 16 and kMaxSplit samples per block.
void choose_split(int B, int64_t imax_mean, int S, int per_sm, int* spl, int* nsplit) {
  const int64_t target = std::max<int64_t>(1, ((int64_t)per_sm * device_sms()) / std::max(1, B));
  const int64_t ntile = std::max<int64_t>(1, (imax_mean + kP1Rows - 1) / kP1Rows);
  const int64_t ns0 = (target + ntile - 1) / ntile;
  int64_t sp = (S + ns0 - 1) / ns0;
  sp = std::max<int64_t>(sp, std::min<int64_t>(16, S));
  sp = std::min<int64_t>(sp, kMaxSplit);
  *spl = (int)sp;
  *nsplit = (int)((S + sp - 1) / sp);
}

// CP-ALS column split of the mode-n MTTKRP: about 8 CTAs per SM across the row tiles, at least 8
// column tiles per split, splits a whole number of column tiles.
void choose_als_split(Prob& p, int n) {
  const int TI = mttkrp_tile_rows(p.als_rg, p.dtype), JT = mttkrp_tile_cols(p.als_rg, p.dtype);
  const int64_t I = p.dims[n], J = p.P / I;
  const int64_t rowtiles = (I + TI - 1) / TI;
  int64_t ns = ((int64_t)device_sms() * 8 + rowtiles - 1) / rowtiles;
  const int64_t tiles = (J + JT - 1) / JT;
  ns = std::max<int64_t>(1, std::min(ns, tiles / 8));
  int64_t js = (J + ns - 1) / ns;
  js = (js + JT - 1) / JT * JT;
  p.jsplit[n] = js;
  p.als_nsplit[n] = (int)((J + js - 1) / js);
}

// Lays out (ws == nullptr: measures) the buffers of B problems.  mix: also the mixing buffers.
// als: CP-ALS buffers (Grams, MTTKRP partials, unfolding copies of every mode when als_mode < 0,
// else one copy buffer used for mode als_mode).
Plan make_plan(int B, const ProbSpec* specs, int mix, void* ws, int als = 0, int als_mode = -1,
               const Schedule* sch = nullptr) {
  const Schedule dflt;
  if (!sch) sch = &dflt;
  Plan pl;
  pl.B = B;
  pl.mix = mix;
  pl.dtype = specs[0].X->dtype;
  Carver cv(ws);
  pl.d_probs = cv.take<Prob>(B);
  pl.d_states = cv.take<State>(B);
  pl.d_counter = cv.take<int>(16);   // [0] iterations, [1] cluster queue, [2] device error, [4..] mixing maxima
  int64_t maxP = 0;
  for (int b = 0; b < B; ++b) maxP = std::max(maxP, prod_dims(specs[b].X));
  pl.normblk = sumsq_blocks(maxP);
  pl.d_normpart = cv.take<double>(pl.normblk);
  if (B == 1 && specs[0].S > 0 && specs[0].X->dtype != CPR_F64 && !als) {
    const int R = specs[0].R;
    const int NE = R * (R + 1) / 2;
    int64_t imax = 1;
    for (int n = 0; n < specs[0].X->order; ++n) imax = std::max<int64_t>(imax, specs[0].X->dims[n]);
    GridScratch& g = pl.gscr;
    g.Gpart = cv.take<float2>((size_t)kGridMaxCTAs * NE);
    g.Gfull = cv.take<float2>((size_t)NE);
    g.Mpart = cv.take<float>((size_t)std::max<int64_t>((int64_t)kGridMaxCTAs * kGridTileRows, imax) * R);
    g.Npart = cv.take<float2>((size_t)kGridMaxCTAs * R);
    g.fitpart = cv.take<double>((size_t)kGridMaxCTAs);
    g.bar = cv.take<unsigned>(4);
    g.err = reinterpret_cast<int*>(g.bar + 2);
    pl.has_grid = true;
  }
  if (mix) {
    pl.d_tmp = cv.take<unsigned char>((size_t)maxP * elem_size(pl.dtype));
    if (pl.dtype == CPR_F32) pl.d_tmp2 = cv.take<unsigned char>((size_t)maxP * elem_size(pl.dtype));
  }
  GridInfo& g = pl.g;
  memset(&g, 0, sizeof(g));
  g.B = B;
  g.dtype = pl.dtype;
  g.any_f64 = pl.dtype == CPR_F64;
  g.max_P = maxP;
  pl.probs.resize(B);
  pl.mixb.resize(B);
  const bool f64 = pl.dtype == CPR_F64;
  for (int b = 0; b < B; ++b) {
    const ProbSpec& sp = specs[b];
    const cpr_tensor* X = sp.X;
    Prob& p = pl.probs[b];
    memset(&p, 0, sizeof(p));
    p.N = X->order;
    p.R = sp.R;
    p.S = (int)sp.S;
    p.dtype = X->dtype;
    int64_t st = 1, imax = 0, isum = 0;
    for (int n = 0; n < p.N; ++n) {
      p.dims[n] = X->dims[n];
      p.st[n] = st;
      st *= X->dims[n];
      imax = std::max(imax, X->dims[n]);
      isum += X->dims[n];
    }
    p.P = st;
    p.X = X->data;
    p.imax = (int)imax;
    const int R = p.R, N = p.N, S = p.S;
    const int Rp = (R + 3) / 4 * 4;
    for (int n = 0; n < N; ++n) {
      p.A32[n] = cv.take<float>((size_t)p.dims[n] * R);
      p.A64[n] = sp.user_A64 ? sp.user_A64[n] : cv.take<double>((size_t)p.dims[n] * R);
      p.scale[n] = cv.take<double>(R);
      p.Apad[n] = (S > 0) ? (void*)cv.take<unsigned char>((size_t)p.dims[n] * Rp * (f64 ? 8 : 4)) : nullptr;
    }
    p.lambda = sp.user_lambda ? sp.user_lambda : cv.take<double>(R);
    if (S > 0) {
      choose_split(B, isum / N, S, sch->split_per_sm, &p.spl, &p.nsplit);
      int spl_most = 0, ns_most = 0;   // the finest split any schedule may pick sizes the buffers
      choose_split(B, isum / N, S, kMaxSplitPerSM, &spl_most, &ns_most);
      ns_most = std::max(ns_most, p.nsplit);
      p.grid_min_split = sch->grid_min_split;
      p.Gpart = cv.take<double>((size_t)ns_most * R * R);
      p.L = cv.take<double>((size_t)R * R);
      p.Mpart = cv.take<unsigned char>((size_t)ns_most * imax * R * (f64 ? 8 : 4));
      p.Npart = cv.take<double>((size_t)((imax + kP2Rows - 1) / kP2Rows) * R);
    }
    if (als) {
      p.als_rg = mttkrp_rank_groups(R);
      int64_t most = 1;
      for (int n = 0; n < N; ++n) {
        choose_als_split(p, n);
        most = std::max<int64_t>(most, p.als_nsplit[n]);
      }
      const int64_t nrb = (imax + kAlsRows - 1) / kAlsRows;
      for (int n = 0; n < N; ++n) p.gram[n] = cv.take<double>((size_t)R * R);
      p.V = cv.take<double>((size_t)R * R);
      p.L = cv.take<double>((size_t)R * R);
      p.Gpart = cv.take<double>((size_t)nrb * R * R);
      p.Npart = cv.take<double>((size_t)nrb);
      p.Mpart = cv.take<double>((size_t)most * imax * R);
      p.Mfold = cv.take<double>((size_t)imax * R);
    }
    p.P_hat = (int)sp.P_hat;
    if (p.P_hat > 0) {
      p.nfb = (p.P_hat + kFitThreads - 1) / kFitThreads;
      p.fit_idx = cv.take<uint32_t>((size_t)p.P_hat * N);
      p.fit_x = cv.take<double>(p.P_hat);
      p.fit_part = cv.take<double>(p.nfb);
    }
    const cpr_opts* o = sp.opts;
    if (o) {
      p.max_iters = o->max_iters;
      p.fixed_iters = o->fixed_iters;
      p.stall_iters = o->stall_iters;
      p.tol = o->fit_tol;
      p.eta = o->noise_eta;
      p.seed = o->seed;
      p.b = o->batch_index;
      p.t0 = o->first_iter;
      p.trace = o->fit_trace_dev;
      p.user_idx = o->user_samples;
    }
    p.state = pl.d_states + b;   // pointer arithmetic on a null base only measures
    if (mix) {
      MixBufs& mb = pl.mixb[b];
      for (int n = 0; n < N; ++n) {
        const size_t I = (size_t)p.dims[n];
        if (f64) mb.W64[n] = cv.take<double>(I * I);
        else mb.W32[n] = cv.take<float>(I * I);
        if (pl.dtype == CPR_F32) mb.Wlo[n] = cv.take<float>(I * I);
        mb.F64[n] = cv.take<double>(I * I);
        mb.sg[n] = cv.take<double>(I);
      }
      mb.table = cv.take<double>((size_t)4 * imax);
      mb.xhat = cv.take<unsigned char>((size_t)p.P * elem_size(pl.dtype));
      p.X = mb.xhat;
    }
    // the copies each mode-n gather reads
    p.use_rep = ((S > 0 && o && o->layout == 0) || als) ? 1 : 0;
    p.Xrep[0] = p.X;
    if (als && als_mode >= 0) {
      void* one = cv.take<unsigned char>((size_t)p.P * elem_size(pl.dtype));
      for (int n = 1; n < N; ++n) p.Xrep[n] = n == als_mode ? one : nullptr;
    } else {
      for (int n = 1; n < N; ++n)
        p.Xrep[n] = p.use_rep ? (const void*)cv.take<unsigned char>((size_t)p.P * elem_size(pl.dtype)) : p.X;
    }
    // grid maxima
    g.max_S = std::max(g.max_S, S);
    g.max_spl = std::max(g.max_spl, p.spl);
    g.max_nfb = std::max(g.max_nfb, p.nfb);
    g.max_R = std::max(g.max_R, R);
    g.max_Phat = std::max(g.max_Phat, p.P_hat);
    for (int n = 0; n < N; ++n) {
      g.max_I[n] = std::max<int>(g.max_I[n], (int)p.dims[n]);
      const int ntile = (int)((p.dims[n] + kP1Rows - 1) / kP1Rows);
      g.max_tiles_x_split[n] = std::max(g.max_tiles_x_split[n], ntile * std::max(1, p.nsplit));
    }
  }
  pl.bytes = align256(cv.off);
  return pl;
}

cpr_opts defaults() {
  cpr_opts o;
  cpr_default_opts(&o);
  return o;
}

// Enqueue the mode loop and the fit/stop test of one outer iteration for the whole batch.
// The N mixing passes X -> final (standard layout), Alg. 5 mixing step.  On the tensor cores when
// every mode allows it (FP32, I_n a multiple of 4): pass 0 reads X directly, pass n >= 1 reads the
// mode-n unfolding of the previous result (t2), results alternate through t1 and the last lands in
// `final`; the last pass also writes its unfolding into rep_last when given (*wrote_rep_last).
// Otherwise SIMT passes ping-pong between final and t1 so that the last lands in final.
// the factored transform mixes this tensor (its tables are then built with the operators, in the
// buffer of the dense FP32 operator, which is not needed)
bool fft_mixing(int dtype, int N, const int64_t* dims) {
  return mix_engine() != CPR_MIX_DENSE && mix_fft_supported(dtype, N, dims);
}

// Whether enqueue_mixing takes the factored DCT passes for these buffers and tables.
bool mixing_uses_fft(const void* t1, int dtype, int N, const int64_t* dims, float* const* W32, double* const* SG) {
  bool fft = t1 != nullptr && fft_mixing(dtype, N, dims);
  for (int n = 0; n < N && fft; ++n) fft = W32[n] != nullptr && SG[n] != nullptr;
  return fft;
}

int enqueue_mixing(const void* src, void* final, void* t1, void* t2, void* rep_last, int dtype, int N,
                   const int64_t* dims, float* const* W32, float* const* Wlo, double* const* W64,
                   double* const* SG, int* err, unsigned* amax, bool amax0_ready, cudaStream_t s, int64_t& launches,
                   bool* wrote_rep_last, State* norm_state) {
  *wrote_rep_last = false;
  if (mixing_uses_fft(t1, dtype, N, dims, W32, SG)) {
    // factored DCT passes (the tables are in the dense operator's buffer, 5 I <= I^2 floats, built
    // with the operators); pass n writes the layout pass n + 1 reads, the outputs alternate between
    // final and t1 so that the last pass writes final.  With norm_state, the first pass (which reads
    // the caller's tensor) also leaves one sum of squares per CTA in the buffer it does not write,
    // summed into norm_state->norm_x before the second pass overwrites that buffer.
    void* bufs[2] = {final, t1};
    const void* U = src;
    for (int n = 0; n < N; ++n) {
      void* y = bufs[(N - 1 - n) & 1];
      void* ys = (n == N - 1 && rep_last) ? rep_last : nullptr;
      double* part = (n == 0 && norm_state) ? static_cast<double*>(bufs[N & 1]) : nullptr;
      int64_t nblk = 0;
      CPR_LAUNCH(CPR_KERNEL_MIX, launch_mix_fft(U, y, ys, W32[n], dtype, N, dims, n, err, s, part, &nblk));
      if (part) {   // one partial per CTA: a first level of 4096-partial sums, then the finish
        if (nblk <= 0) return CPR_EINVAL;
        double* part2 = part + nblk;
        const int64_t nb2 = sumsq_partials_blocks(nblk);
        if (nb2 > INT32_MAX) return CPR_EINVAL;
        CPR_LAUNCH(CPR_KERNEL_OTHER, launch_sumsq_partials(part, nblk, part2, s));
        CPR_LAUNCH(CPR_KERNEL_OTHER, launch_sumsq_finish(part2, (int)nb2, nullptr, norm_state, 1, s));
      }
      if (ys) *wrote_rep_last = true;
      U = y;
    }
    return CPR_OK;
  }
  if (norm_state) return CPR_EINVAL;   // the caller reduces ||X|| itself on the other paths
  bool tc = dtype == CPR_F32 && t2 != nullptr;
  for (int n = 0; n < N && tc; ++n) tc = Wlo[n] != nullptr && mix_tc_supported(dtype, (int)dims[n]);
  bool tc16 = tc && amax != nullptr;
  for (int n = 0; n < N && tc16; ++n) tc16 = mix_tc16_supported(dtype, (int)dims[n]);
  if (tc16) {
    // FP16-split tensor-core passes: W's FP16 halves go into the Wlo buffer (2 I^2 halves = I^2
    // floats); amax[n] = largest |entry| of pass n's input (the input tensor's from a max pass)
    int64_t P = 1;
    for (int n = 0; n < N; ++n) P *= dims[n];
    if (!amax0_ready) {   // else the norm pass already recorded amax[0] (and cleared the rest)
      CPR_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned) * (size_t)(N + 1), s));
      CPR_LAUNCH(CPR_KERNEL_OTHER, launch_absmax(src, dtype, P, amax, s));
    }
    for (int n = 0; n < N; ++n)
      CPR_LAUNCH(CPR_KERNEL_OTHER, launch_split_f16(W32[n], Wlo[n], dims[n] * dims[n], s));
    const float* U = static_cast<const float*>(src);
    for (int n = 0; n < N; ++n) {
      if (n > 1) CPR_LAUNCH(CPR_KERNEL_OTHER, launch_unfold_copy(t1, t2, dtype, N, dims, n, s));
      if (n > 0) U = static_cast<const float*>(t2);
      const bool last = n == N - 1;
      float* ystd = last ? static_cast<float*>(final) : (n == 0 ? nullptr : static_cast<float*>(t1));
      float* ynext = (n == 0 && !last) ? static_cast<float*>(t2) : nullptr;
      float* yunf = (last && rep_last && n > 0) ? static_cast<float*>(rep_last) : nullptr;
      CPR_LAUNCH(CPR_KERNEL_MIX, launch_mix_tc16(U, ystd, yunf, ynext, Wlo[n], N, dims, n, amax + n,
                                                 last ? nullptr : amax + n + 1, err, s));
      if (yunf) *wrote_rep_last = true;
    }
    return CPR_OK;
  }
  if (tc) {
    for (int n = 0; n < N; ++n)
      CPR_LAUNCH(CPR_KERNEL_OTHER, launch_split_tf32(W32[n], W32[n], Wlo[n], dims[n] * dims[n], s));
    // pass n reads the mode-n unfolding of the previous result: the first pass writes the mode-2
    // unfolding directly; later passes write the standard layout, transposed by an unfolding copy
    const float* U = static_cast<const float*>(src);
    for (int n = 0; n < N; ++n) {
      if (n > 1) CPR_LAUNCH(CPR_KERNEL_OTHER, launch_unfold_copy(t1, t2, dtype, N, dims, n, s));
      if (n > 0) U = static_cast<const float*>(t2);
      const bool last = n == N - 1;
      float* ystd = last ? static_cast<float*>(final) : (n == 0 ? nullptr : static_cast<float*>(t1));
      float* ynext = (n == 0 && !last) ? static_cast<float*>(t2) : nullptr;
      float* yunf = (last && rep_last && n > 0) ? static_cast<float*>(rep_last) : nullptr;
      CPR_LAUNCH(CPR_KERNEL_MIX, launch_mix_tc(U, ystd, yunf, ynext, W32[n], Wlo[n], N, dims, n, 1, err, s));
      if (yunf) *wrote_rep_last = true;
    }
    return CPR_OK;
  }
  const void* cur_src = src;
  void* bufs[2] = {final, t1};
  int cur = (N % 2 == 1) ? 0 : 1;
  for (int n = 0; n < N; ++n) {
    CPR_LAUNCH(CPR_KERNEL_MIX, launch_mix_mode(cur_src, bufs[cur], dtype, N, dims, n, W32[n], W64[n], s));
    cur_src = bufs[cur];
    cur ^= 1;
  }
  return CPR_OK;
}

int enqueue_mode_update(const Plan& pl, int n, cudaStream_t s, int64_t& launches) {
  CPR_LAUNCH(CPR_KERNEL_CONTRACT, launch_sample_contract(pl.d_probs, pl.g, n, s));
  CPR_LAUNCH(CPR_KERNEL_SOLVE, launch_solve(pl.d_probs, pl.g, n, s));
  return CPR_OK;
}

int enqueue_iteration(const Plan& pl, int maxN, int cap, int use_cond, unsigned long long cond, cudaStream_t s,
                      int64_t& launches) {
  for (int n = 0; n < maxN; ++n)
    if (int st = enqueue_mode_update(pl, n, s, launches)) return st;
  CPR_LAUNCH(CPR_KERNEL_FIT, launch_fit(pl.d_probs, pl.g, s));
  if (use_cond) CPR_LAUNCH(CPR_KERNEL_OTHER, launch_loop_cond(pl.d_probs, pl.B, pl.d_counter, cap, cond, s));
  return CPR_OK;
}

// All outer iterations as ONE graph launch: the body (the mode updates and the fit of one
// iteration) is captured once into a while-conditional node whose condition the last kernel of
// the body sets on the device.  No host round trip between iterations.  *body_kernels receives the
// number of kernels in the body; the device counter pl.d_counter[0] counts executed iterations.
// A non-blocking stream per device used only to record graph bodies (the caller's stream may be the
// legacy default stream, which cannot be captured).  Nothing runs on it.
cudaStream_t capture_stream() {
  static std::mutex mu;
  static cudaStream_t streams[64] = {};
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return nullptr;
  std::lock_guard<std::mutex> lk(mu);
  if (!streams[dev] && cudaStreamCreateWithFlags(&streams[dev], cudaStreamNonBlocking) != cudaSuccess)
    streams[dev] = nullptr;
  return streams[dev];
}

// enqueue_body(capture_stream, condition_handle, kernel_count) enqueues one iteration and the kernel that
// sets the condition.
template <class Body>
int run_graph_loop(Body&& enqueue_body, cudaStream_t s, int64_t* body_kernels) {
  cudaStream_t cs = capture_stream();
  if (!cs) return CPR_ECUDA;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  int st = CPR_OK;
  cudaGraphConditionalHandle h = 0;
  cudaGraphNodeParams np = {};
  cudaGraphNode_t node = nullptr;
  if (cudaGraphCreate(&graph, 0) != cudaSuccess) return CPR_ECUDA;
  do {
    if (cudaGraphConditionalHandleCreate(&h, graph, 1u, cudaGraphCondAssignDefault) != cudaSuccess) {
      st = CPR_ECUDA;
      break;
    }
    np.type = cudaGraphNodeTypeConditional;
    np.conditional.handle = h;
    np.conditional.type = cudaGraphCondTypeWhile;
    np.conditional.size = 1;
    if (cudaGraphAddNode(&node, graph, nullptr, nullptr, 0, &np) != cudaSuccess) {
      st = CPR_ECUDA;
      break;
    }
    cudaGraph_t body = np.conditional.phGraph_out[0];
    if (cudaStreamBeginCaptureToGraph(cs, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
      st = CPR_ECUDA;
      break;
    }
    int64_t n_body = 0;
    const int cst = enqueue_body(cs, (unsigned long long)h, n_body);
    cudaGraph_t captured = nullptr;
    const cudaError_t ce = cudaStreamEndCapture(cs, &captured);
    if (cst != CPR_OK || ce != cudaSuccess) {
      st = cst != CPR_OK ? cst : CPR_ECUDA;
      break;
    }
    *body_kernels = n_body;
    if (cudaGraphInstantiate(&exec, graph, 0) != cudaSuccess) {
      st = CPR_ECUDA;
      break;
    }
    if (cudaGraphLaunch(exec, s) != cudaSuccess) st = CPR_ECUDA;
  } while (0);
  if (exec) cudaGraphExecDestroy(exec);   // safe while the launch is in flight
  cudaGraphDestroy(graph);
  return st;
}

int enqueue_finalize(const Plan& pl, int maxN, cudaStream_t s, int64_t& launches) {
  for (int n = 0; n < maxN; ++n) CPR_LAUNCH(CPR_KERNEL_OTHER, launch_finalize(pl.d_probs, pl.g, n, s));
  return CPR_OK;
}

// ------------------------------------------------------------------------------------------------
// Schedule autotuner: the tuned schedule of a problem bucket (dtype, order, batch size, mixing, and
// per mode the largest extent, the largest rank and sample count of the batch, each bucketed) is
// kept in a process-wide table, applied by every call with loop_path 0, and can be saved to and
// loaded from a text file (one line per bucket: key, loop path, split per SM, grid minimum split,
// milliseconds per outer iteration when it was tuned).  The environment variable CPRAND_TUNE_CACHE
// names a file loaded on the first lookup.
// ------------------------------------------------------------------------------------------------
int ceil_log2(int64_t v) {
  int k = 0;
  while (((int64_t)1 << k) < v) ++k;
  return k;
}

std::string tune_key(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss, int mix) {
  int64_t mx[CPR_MAX_ORDER] = {};
  int R = 0;
  int64_t S = 0;
  for (int b = 0; b < B; ++b) {
    for (int n = 0; n < Xs[b].order; ++n) mx[n] = std::max(mx[n], Xs[b].dims[n]);
    R = std::max(R, Rs[b]);
    S = std::max(S, Ss[b]);
  }
  std::string k = "d" + std::to_string(Xs[0].dtype) + ":N" + std::to_string(Xs[0].order) + ":B" +
                  std::to_string(ceil_log2(B)) + ":m" + std::to_string(mix ? 1 : 0) + ":I";
  for (int n = 0; n < Xs[0].order; ++n) k += (n ? "," : "") + std::to_string(ceil_log2(mx[n]));
  k += ":R" + std::to_string((R + 7) / 8) + ":S" + std::to_string(ceil_log2(S));
  return k;
}

struct TuneEntry {
  Schedule sch;
  double ms_per_iter;
};

struct TuneTable {
  std::mutex mu;
  std::map<std::string, TuneEntry> map;
  bool env_loaded = false;
};

TuneTable& tune_table() {
  static TuneTable t;
  return t;
}

int tune_load_locked(TuneTable& t, const char* path) {
  FILE* f = fopen(path, "r");
  if (!f) return CPR_EINVAL;
  char key[512];
  int lp, sp, gm;
  double ms;
  while (fscanf(f, "%511s %d %d %d %lf", key, &lp, &sp, &gm, &ms) == 5) {
    if (lp < 0 || lp > 5 || sp < 1 || sp > kMaxSplitPerSM || gm < 1 || gm > 1024) continue;
    Schedule sc;
    sc.loop_path = lp;
    sc.split_per_sm = sp;
    sc.grid_min_split = gm;
    t.map[key] = TuneEntry{sc, ms};
  }
  fclose(f);
  return CPR_OK;
}

bool tune_lookup(const std::string& key, Schedule* out, double* ms = nullptr) {
  TuneTable& t = tune_table();
  std::lock_guard<std::mutex> lk(t.mu);
  if (!t.env_loaded) {
    t.env_loaded = true;
    const char* path = getenv("CPRAND_TUNE_CACHE");
    if (path && *path) tune_load_locked(t, path);
  }
  auto it = t.map.find(key);
  if (it == t.map.end()) return false;
  *out = it->second.sch;
  if (ms) *ms = it->second.ms_per_iter;
  return true;
}

int run_batched(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss, const cpr_opts* opts, int mix,
                cpr_ktensor* outs, cpr_result* results, void* ws, size_t ws_bytes, cudaStream_t s,
                const Schedule* forced = nullptr) {
  if (B < 1 || !Xs || !Rs || !Ss || !outs) return CPR_EINVAL;
  std::vector<cpr_opts> op(B);
  std::vector<ProbSpec> specs(B);
  int maxN = 0;
  for (int b = 0; b < B; ++b) {
    if (int st = check_tensor(&Xs[b], true)) return st;
    if (Xs[b].dtype != Xs[0].dtype) return CPR_EINVAL;
    if (int st = check_rank_samples(Rs[b], Ss[b])) return st;
    if (int st = check_ktensor(&outs[b], &Xs[b], Rs[b])) return st;
    op[b] = opts ? opts[b] : defaults();
    if (!opts) op[b].batch_index = (uint32_t)b;
    if (op[b].fit_samples < 1 || op[b].fit_samples > INT32_MAX) return CPR_EINVAL;
    if (op[b].max_iters < 1 && op[b].fixed_iters < 1) return CPR_EINVAL;
    if (op[b].init_from_out != op[0].init_from_out) return CPR_EINVAL;
    if (op[b].user_samples && op[b].user_S != Ss[b]) return CPR_EINVAL;
    if (op[b].wait_budget < 0) return CPR_EINVAL;
    specs[b] = ProbSpec{&Xs[b], Rs[b], Ss[b], op[b].fit_samples, &op[b], nullptr, nullptr};
    maxN = std::max(maxN, (int)Xs[b].order);
  }
  // the schedule: forced (autotuner trials), tuned for this bucket (loop_path 0), or the defaults
  bool any_user = false;
  for (int b = 0; b < B; ++b) any_user = any_user || op[b].user_samples != nullptr;
  Schedule sch;
  if (forced) sch = *forced;
  else if (op[0].loop_path == 0 && !any_user && tune_lookup(tune_key(B, Xs, Rs, Ss, mix), &sch)) {}
  else sch = Schedule{};
  const Plan measure = make_plan(B, specs.data(), mix, nullptr, 0, -1, &sch);
  if (int st = check_ws(ws, ws_bytes, measure.bytes)) return st;
  Plan pl = make_plan(B, specs.data(), mix, ws, 0, -1, &sch);
  CPR_CUDA(prepare_kernel_attributes());
  int64_t launches = 0;
  PhaseEvents ph;
  if (int st = ph.mark(0, s)) return st;
  CPR_CUDA(cudaMemcpyAsync(pl.d_probs, pl.probs.data(), sizeof(Prob) * B, cudaMemcpyHostToDevice, s));
  CPR_CUDA(cudaMemsetAsync(pl.d_counter, 0, 4 * sizeof(int), s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_init_state(pl.d_probs, B, s));
  const bool from_out = op[0].init_from_out != 0;
  for (int b = 0; b < B; ++b) {
    const Prob& p = pl.probs[b];
    bool rep_last_done = false;
    // ||X|| on the caller's tensor (equal to the mixed tensor's norm, Alg. 5); for CPRAND-MIX the same
    // pass records the largest |x| (the scale of the first FP16-split mixing pass)
    // (with the factored DCT passes, the first pass reduces ||X|| from the fibers it has loaded)
    unsigned* amax = mix ? reinterpret_cast<unsigned*>(pl.d_counter + 4) : nullptr;
    const bool norm_in_mix = mix && mixing_uses_fft(pl.d_tmp, p.dtype, p.N, p.dims, pl.mixb[b].W32, pl.mixb[b].sg) &&
                             mix_fft_norm_fits(p.dtype, p.N, p.dims);
    if (!norm_in_mix) {
      if (amax) CPR_CUDA(cudaMemsetAsync(amax, 0, sizeof(unsigned) * (size_t)(p.N + 1), s));
      CPR_LAUNCH(CPR_KERNEL_OTHER, launch_sumsq(Xs[b].data, p.dtype, p.P, pl.d_normpart, pl.normblk, s, amax));
      CPR_LAUNCH(CPR_KERNEL_OTHER, launch_sumsq_finish(pl.d_normpart, pl.normblk, nullptr, pl.d_states + b, 1, s));
    }
    if (mix) {
      const MixBufs& mb = pl.mixb[b];
      const bool fftm = pl.d_tmp != nullptr && fft_mixing(p.dtype, p.N, p.dims) && mb.W32[0] != nullptr;
      for (int n = 0; n < p.N; ++n)
        CPR_LAUNCH(CPR_KERNEL_OTHER,
                   launch_build_mix_ops((int)p.dims[n], p.seed, p.b, n, mb.table, fftm ? nullptr : mb.W32[n], mb.W64[n],
                                        mb.F64[n], mb.sg[n], s, fftm ? mb.W32[n] : nullptr));
      if (int st = enqueue_mixing(Xs[b].data, mb.xhat, pl.d_tmp, pl.d_tmp2,
                                  p.use_rep ? const_cast<void*>(p.Xrep[p.N - 1]) : nullptr, p.dtype, p.N, p.dims,
                                  mb.W32, mb.Wlo, mb.W64, mb.sg, pl.d_counter + 2, amax, true, s, launches,
                                  &rep_last_done, norm_in_mix ? pl.d_states + b : nullptr))
        return st;
    }
    if (p.use_rep)
      for (int n = 1; n < p.N - (rep_last_done ? 1 : 0); ++n)
        CPR_LAUNCH(CPR_KERNEL_OTHER, launch_unfold_copy(p.X, const_cast<void*>(p.Xrep[n]), p.dtype, p.N, p.dims, n, s));
    if (from_out) {
      for (int n = 1; n < p.N; ++n)
        CPR_CUDA(cudaMemcpyAsync(p.A64[n], outs[b].factors[n], sizeof(double) * p.dims[n] * p.R,
                                 cudaMemcpyDeviceToDevice, s));
      static const double ones[CPR_MAX_RANK] = {1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,
                                                1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1,
                                                1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1, 1};
      CPR_CUDA(cudaMemcpyAsync(p.lambda, ones, sizeof(double) * p.R, cudaMemcpyHostToDevice, s));
    }
  }
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_init_factors(pl.d_probs, pl.g, from_out ? 1 : 0, s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_fit_setup(pl.d_probs, pl.g, s));
  if (int st = ph.mark(1, s)) return st;
  // outer iterations; every problem stops on its own rule, the loop ends when all have
  int cap = 0;
  for (int b = 0; b < B; ++b) cap = std::max(cap, op[b].fixed_iters > 0 ? op[b].fixed_iters : op[b].max_iters);
  std::vector<State> hs(B);
  int64_t body_kernels = 0;
  // the iteration loop runs as one graph launch unless the profiler records a kernel class that
  // lives inside the loop (events need plain stream launches)
  const unsigned loop_classes = (1u << CPR_KERNEL_SAMPLE_SKR) | (1u << CPR_KERNEL_CONTRACT) | (1u << CPR_KERNEL_CHOL) |
                                (1u << CPR_KERNEL_SOLVE) | (1u << CPR_KERNEL_NORMALIZE) | (1u << CPR_KERNEL_FIT);
  if (op[0].loop_path < 0 || op[0].loop_path > 5) return CPR_EINVAL;
  const int path = (forced || op[0].loop_path == 0) ? sch.loop_path : op[0].loop_path;
  bool user_samples = false;
  for (int b = 0; b < B; ++b) user_samples = user_samples || op[b].user_samples != nullptr;
  // caller-given samples: the graph kernels, the plain stream launches and the whole-GPU loop read them
  if (user_samples && (path == 1 || path == 4)) return CPR_EINVAL;
  const bool stream_only = path == 3 || (prof().on && (prof().mask & loop_classes));
  // the whole GPU for one large FP32 / BF16 problem (explicitly, or automatically when the
  // replicated-factor cluster cannot hold it)
  int grid_G = 0;
  bool use_grid = false;
  if (!stream_only && pl.has_grid && (path == 5 || path == 0)) {
    int maxR = pl.probs[0].R;
    grid_G = grid_capacity(pl.dtype, maxR);
    const bool fits = grid_G > 0 && grid_fits(pl.probs[0], grid_G);
    if (path == 5) {
      if (!fits) return CPR_EINVAL;
      use_grid = true;
    } else if (fits && !user_samples) {
      const int rs = loop_rep_smem_bytes(pl.probs.data(), B);
      use_grid = !(rs > 0 && loop_rep_capacity(pl.dtype, rs, maxR) > 0);
    }
  } else if (path == 5) {
    return CPR_EINVAL;
  }
  // small problems: the whole loop in thread-block clusters (one cluster per problem at a time);
  // first choice: every factor replicated in each CTA of the cluster; else factor rows
  // distributed over the CTAs
  int C = 16, csmem = -1, ncl = 0;
  bool rep = false;
  if (use_grid) {
    GridScratch gsc = pl.gscr;
    gsc.wait_limit = op[0].wait_budget > 0 ? (uint32_t)std::min<int64_t>(op[0].wait_budget, UINT32_MAX)
                                           : kDefaultWaitPolls;
    gsc.use_tc = g_contract_engine.load() == CPR_CONTRACT_FMA ? 0 : 1;
    CPR_CUDA(cudaMemsetAsync(gsc.bar, 0, 4 * sizeof(unsigned), s));
    CPR_LAUNCH(CPR_KERNEL_LOOP, launch_grid_run(pl.d_probs, B, gsc, pl.dtype, pl.probs[0].R, grid_G, s));
    ncl = 1;   // the loop has run
  } else if (!stream_only && path != 2 && !user_samples) {
    int maxR = 0;
    for (int b = 0; b < B; ++b) maxR = std::max(maxR, pl.probs[b].R);
    if (path != 4) {
      const int rs = loop_rep_smem_bytes(pl.probs.data(), B);
      if (rs > 0) {
        const int cap = loop_rep_capacity(pl.dtype, rs, maxR);
        if (cap > 0) {
          rep = true;
          csmem = rs;
          ncl = cap;
        }
      }
    }
    // a batch of several problems whose factors cannot be replicated runs faster as the graph
    // (every problem's mode update in the same launches: 77 vs 106 ms for 64 problems of dims up to
    // 511 and ranks up to 32) than queued on distributed-factor clusters; a single problem, or an
    // explicit cluster path, still takes the clusters
    const bool batch_graph = !rep && path == 0 && B > 1;
    if (!rep && !batch_graph) {
      for (int c : {16, 8}) {
        C = c;
        csmem = cluster_smem_bytes(pl.probs.data(), B, C);
        if (csmem < 0) continue;
        ncl = cluster_capacity(pl.dtype, C, csmem, maxR);
        if (ncl > 0) break;
      }
    }
    if ((path == 1 || path == 4) && ncl <= 0) return CPR_EINVAL;
    if (ncl > 0) {
      ncl = std::min(ncl, B);
      CPR_CUDA(cudaMemsetAsync(pl.d_counter + 1, 0, sizeof(int), s));
      if (rep)
        CPR_LAUNCH(CPR_KERNEL_LOOP, launch_loop_rep(pl.d_probs, B, pl.d_counter + 1, pl.dtype, csmem, ncl, maxR, s));
      else
        CPR_LAUNCH(CPR_KERNEL_LOOP,
                   launch_cluster_run(pl.d_probs, B, pl.d_counter + 1, pl.dtype, C, csmem, ncl, maxR, s));
    }
  }
  const bool use_graph = !stream_only && ncl <= 0;
  if (ncl > 0) {
    // the cluster kernel ran the whole loop
  } else if (use_graph) {
    auto body = [&](cudaStream_t cs, unsigned long long h, int64_t& nb) {
      return enqueue_iteration(pl, maxN, cap, 1, h, cs, nb);
    };
    if (int st = run_graph_loop(body, s, &body_kernels)) return st;
  } else {
    // profiling: plain stream launches (events around single kernels), stop flag polled per chunk
    int ran = 0, chunk = 4;
    while (ran < cap) {
      const int todo = std::min(chunk, cap - ran);
      for (int c = 0; c < todo; ++c)
        if (int st = enqueue_iteration(pl, maxN, cap, 0, 0ull, s, launches)) return st;
      ran += todo;
      CPR_CUDA(cudaMemcpyAsync(hs.data(), pl.d_states, sizeof(State) * B, cudaMemcpyDeviceToHost, s));
      CPR_CUDA(cudaStreamSynchronize(s));
      bool all = true;
      for (int b = 0; b < B; ++b) all = all && hs[b].done;
      if (all) break;
      chunk = std::min(chunk * 2, 16);
    }
  }
  if (int st = ph.mark(2, s)) return st;
  if (int st = enqueue_finalize(pl, maxN, s, launches)) return st;
  // outputs (unmixed for CPRAND-MIX)
  for (int b = 0; b < B; ++b) {
    const Prob& p = pl.probs[b];
    if (mix) {
      UnmixArgs u{};
      u.N = p.N;
      u.R = p.R;
      for (int n = 0; n < p.N; ++n) {
        u.Ahat[n] = p.A64[n];
        u.A[n] = outs[b].factors[n];
        u.F[n] = pl.mixb[b].F64[n];
        u.sg[n] = pl.mixb[b].sg[n];
        u.I[n] = (int)p.dims[n];
      }
      CPR_LAUNCH(CPR_KERNEL_OTHER, launch_unmix_all(u, s));
    } else {
      for (int n = 0; n < p.N; ++n)
        CPR_CUDA(cudaMemcpyAsync(outs[b].factors[n], p.A64[n], sizeof(double) * p.dims[n] * p.R,
                                 cudaMemcpyDeviceToDevice, s));
    }
    CPR_CUDA(cudaMemcpyAsync(outs[b].lambda, p.lambda, sizeof(double) * p.R, cudaMemcpyDeviceToDevice, s));
  }
  CPR_CUDA(cudaMemcpyAsync(hs.data(), pl.d_states, sizeof(State) * B, cudaMemcpyDeviceToHost, s));
  int loop_iters = 0;
  CPR_CUDA(cudaMemcpyAsync(&loop_iters, pl.d_counter, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (int st = ph.mark(3, s)) return st;
  int dev_err = 0, grid_err = 0;
  CPR_CUDA(cudaMemcpyAsync(&dev_err, pl.d_counter + 2, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (use_grid) CPR_CUDA(cudaMemcpyAsync(&grid_err, pl.gscr.err, sizeof(int), cudaMemcpyDeviceToHost, s));
  CPR_CUDA(cudaStreamSynchronize(s));
  if (dev_err || grid_err) return CPR_ETIMEOUT;
  launches += (int64_t)loop_iters * body_kernels;
  if (results) {
    for (int b = 0; b < B; ++b) {
      results[b].iters = hs[b].iter;
      results[b].status = hs[b].status;
      results[b].fit_est = hs[b].last_fit;
      results[b].norm_x = hs[b].norm_x;
      results[b].kernel_launches = launches;
      results[b].ms_setup = ph.ms(0, 1);
      results[b].ms_iterate = ph.ms(1, 2);
      results[b].ms_finish = ph.ms(2, 3);
    }
  }
  return CPR_OK;
}

// One outer iteration of CP-ALS (Alg. 1): per mode the Gram Hadamard product and its Cholesky
// factor, the exact MTTKRP, the row solves (the last mode's solve also forms the exact fit and
// applies the stopping rules); then the graph condition.
int enqueue_als_iteration(const Plan& pl, int cap, int use_cond, unsigned long long cond, cudaStream_t s,
                          int64_t& launches) {
  const Prob& p = pl.probs[0];
  for (int n = 0; n < p.N; ++n) {
    CPR_LAUNCH(CPR_KERNEL_CHOL, launch_als_prep(pl.d_probs, p, n, s));
    CPR_LAUNCH(CPR_KERNEL_CONTRACT, launch_mttkrp(pl.d_probs, p, n, s));
    CPR_LAUNCH(CPR_KERNEL_CONTRACT, launch_mttkrp_fold(pl.d_probs, p, n, nullptr, s));
    CPR_LAUNCH(CPR_KERNEL_SOLVE, launch_als_solve(pl.d_probs, p, n, s));
  }
  if (use_cond) CPR_LAUNCH(CPR_KERNEL_OTHER, launch_loop_cond(pl.d_probs, 1, pl.d_counter, cap, cond, s));
  return CPR_OK;
}

int run_cp_als(const cpr_tensor* X, int R, const cpr_opts* opts, cpr_ktensor* out, cpr_result* result, void* ws,
               size_t ws_bytes, cudaStream_t s) {
  if (int st = check_tensor(X, true)) return st;
  if (R < 1 || R > CPR_MAX_RANK) return CPR_EINVAL;
  if (int st = check_ktensor(out, X, R)) return st;
  cpr_opts o = opts ? *opts : defaults();
  if (o.max_iters < 1 && o.fixed_iters < 1) return CPR_EINVAL;
  if (o.loop_path < 0 || o.loop_path > 4) return CPR_EINVAL;
  ProbSpec sp{X, R, 0, 0, &o, nullptr, nullptr};
  const Plan measure = make_plan(1, &sp, 0, nullptr, 1, -1);
  if (int st = check_ws(ws, ws_bytes, measure.bytes)) return st;
  Plan pl = make_plan(1, &sp, 0, ws, 1, -1);
  CPR_CUDA(prepare_kernel_attributes());
  const Prob& p = pl.probs[0];
  int64_t launches = 0;
  PhaseEvents ph;
  if (int st = ph.mark(0, s)) return st;
  CPR_CUDA(cudaMemcpyAsync(pl.d_probs, pl.probs.data(), sizeof(Prob), cudaMemcpyHostToDevice, s));
  CPR_CUDA(cudaMemsetAsync(pl.d_counter, 0, 4 * sizeof(int), s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_init_state(pl.d_probs, 1, s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_sumsq(X->data, p.dtype, p.P, pl.d_normpart, pl.normblk, s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_sumsq_finish(pl.d_normpart, pl.normblk, nullptr, pl.d_states, 1, s));
  for (int n = 1; n < p.N; ++n)
    CPR_LAUNCH(CPR_KERNEL_OTHER, launch_unfold_copy(p.X, const_cast<void*>(p.Xrep[n]), p.dtype, p.N, p.dims, n, s));
  const bool from_out = o.init_from_out != 0;
  if (from_out)
    for (int n = 1; n < p.N; ++n)
      CPR_CUDA(cudaMemcpyAsync(p.A64[n], out->factors[n], sizeof(double) * p.dims[n] * p.R, cudaMemcpyDeviceToDevice,
                               s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_init_factors(pl.d_probs, pl.g, from_out ? 1 : 0, s));
  for (int n = 1; n < p.N; ++n) CPR_LAUNCH(CPR_KERNEL_OTHER, launch_als_gram(pl.d_probs, p, n, s));
  if (int st = ph.mark(1, s)) return st;
  const int cap = o.fixed_iters > 0 ? o.fixed_iters : o.max_iters;
  const unsigned loop_classes = (1u << CPR_KERNEL_CONTRACT) | (1u << CPR_KERNEL_CHOL) | (1u << CPR_KERNEL_SOLVE);
  const bool stream_only = o.loop_path == 3 || (prof().on && (prof().mask & loop_classes));
  int64_t body_kernels = 0;
  if (!stream_only) {
    auto body = [&](cudaStream_t cs, unsigned long long h, int64_t& nb) {
      return enqueue_als_iteration(pl, cap, 1, h, cs, nb);
    };
    if (int st = run_graph_loop(body, s, &body_kernels)) return st;
  } else {
    State hs;
    int ran = 0, chunk = 4;
    while (ran < cap) {
      const int todo = std::min(chunk, cap - ran);
      for (int c = 0; c < todo; ++c)
        if (int st = enqueue_als_iteration(pl, cap, 0, 0ull, s, launches)) return st;
      ran += todo;
      CPR_CUDA(cudaMemcpyAsync(&hs, pl.d_states, sizeof(State), cudaMemcpyDeviceToHost, s));
      CPR_CUDA(cudaStreamSynchronize(s));
      if (hs.done) break;
      chunk = std::min(chunk * 2, 16);
    }
  }
  if (int st = ph.mark(2, s)) return st;
  for (int n = 0; n < p.N; ++n) {
    CPR_LAUNCH(CPR_KERNEL_OTHER, launch_finalize(pl.d_probs, pl.g, n, s));
    CPR_CUDA(cudaMemcpyAsync(out->factors[n], p.A64[n], sizeof(double) * p.dims[n] * p.R, cudaMemcpyDeviceToDevice,
                             s));
  }
  CPR_CUDA(cudaMemcpyAsync(out->lambda, p.lambda, sizeof(double) * p.R, cudaMemcpyDeviceToDevice, s));
  State h;
  int loop_iters = 0;
  CPR_CUDA(cudaMemcpyAsync(&h, pl.d_states, sizeof(State), cudaMemcpyDeviceToHost, s));
  CPR_CUDA(cudaMemcpyAsync(&loop_iters, pl.d_counter, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (int st = ph.mark(3, s)) return st;
  CPR_CUDA(cudaStreamSynchronize(s));
  launches += (int64_t)loop_iters * body_kernels;
  if (result) {
    result->iters = h.iter;
    result->status = h.status;
    result->fit_est = h.last_fit;
    result->norm_x = h.norm_x;
    result->kernel_launches = launches;
    result->ms_setup = ph.ms(0, 1);
    result->ms_iterate = ph.ms(1, 2);
    result->ms_finish = ph.ms(2, 3);
  }
  return CPR_OK;
}

}  // namespace

extern "C" {

void cpr_default_opts(cpr_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->max_iters = 200;
  o->fixed_iters = 0;
  o->fit_tol = 1e-4;
  o->noise_eta = -1.0;
  o->stall_iters = 0;
  o->init_from_out = 0;
  o->fit_samples = 16384;
  o->seed = 0;
  o->batch_index = 0;
  o->first_iter = 0;
  o->fit_trace_dev = nullptr;
  o->loop_path = 0;
  o->layout = 0;
}

const char* cpr_status_string(int status) {
  switch (status) {
    case CPR_OK: return "ok";
    case CPR_EINVAL: return "invalid argument";
    case CPR_EWORKSPACE: return "workspace too small or misaligned";
    case CPR_ESINGULAR: return "Gram matrix is not positive definite";
    case CPR_ENONFINITE: return "non-finite value in the fit estimate";
    case CPR_ETIMEOUT: return "bounded device wait expired";
    case CPR_ECUDA: return "CUDA runtime error";
    default: return "unknown status";
  }
}

int64_t cpr_sample_size(int R) {
  if (R < 1) return 0;
  return (int64_t)floor(10.0 * R * log((double)R) + 0.5);
}

size_t cpr_workspace_size(int method, const cpr_tensor* X, int R, int64_t S, const cpr_opts* opts) {
  if (check_tensor(X, false)) return 0;
  cpr_opts o = opts ? *opts : defaults();
  switch (method) {
    case CPR_METHOD_CPRAND:
    case CPR_METHOD_CPRAND_MIX: {
      if (check_rank_samples(R, S)) return 0;
      ProbSpec sp{X, R, S, o.fit_samples, &o, nullptr, nullptr};
      return make_plan(1, &sp, method == CPR_METHOD_CPRAND_MIX, nullptr).bytes;
    }
    case CPR_METHOD_UPDATE: {
      if (check_rank_samples(R, S)) return 0;
      o.layout = 1;
      static double* dummy[CPR_MAX_ORDER] = {};
      ProbSpec sp{X, R, S, 0, &o, dummy, (double*)nullptr};
      // caller-owned factors and lambda take no workspace
      Plan pl = make_plan(1, &sp, 0, nullptr);
      return pl.bytes;
    }
    case CPR_METHOD_FIT: {
      if (R < 1 || R > CPR_MAX_RANK || o.fit_samples < 1 || o.fit_samples > INT32_MAX) return 0;
      static double* dummy[CPR_MAX_ORDER] = {};
      ProbSpec sp{X, R, 0, o.fit_samples, &o, dummy, nullptr};
      return make_plan(1, &sp, 0, nullptr).bytes;
    }
    case CPR_METHOD_NORM:
      return align256(sizeof(double) * (sumsq_blocks(prod_dims(X)) + 1)) + 256;
    case CPR_METHOD_CP_ALS: {
      if (R < 1 || R > CPR_MAX_RANK) return 0;
      ProbSpec sp{X, R, 0, 0, &o, nullptr, nullptr};
      return make_plan(1, &sp, 0, nullptr, 1, -1).bytes;
    }
    case CPR_METHOD_MTTKRP: {
      if (R < 1 || R > CPR_MAX_RANK) return 0;
      static double* dummy[CPR_MAX_ORDER] = {};
      ProbSpec sp{X, R, 0, 0, &o, dummy, (double*)nullptr};
      return make_plan(1, &sp, 0, nullptr, 1, 0).bytes;
    }
    default:
      return 0;
  }
}

int cpr_cprand(const cpr_tensor* X, int R, int64_t S, const cpr_opts* opts, cpr_ktensor* out, cpr_result* result,
               void* ws, size_t ws_bytes, void* stream) {
  if (!X) return CPR_EINVAL;
  return run_batched(1, X, &R, &S, opts, 0, out, result, ws, ws_bytes, (cudaStream_t)stream);
}

int cpr_cprand_mix(const cpr_tensor* X, int R, int64_t S, const cpr_opts* opts, cpr_ktensor* out,
                   cpr_result* result, void* ws, size_t ws_bytes, void* stream) {
  if (!X) return CPR_EINVAL;
  return run_batched(1, X, &R, &S, opts, 1, out, result, ws, ws_bytes, (cudaStream_t)stream);
}

size_t cpr_batched_workspace_size(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss,
                                  const cpr_opts* opts, int mix) {
  if (B < 1 || !Xs || !Rs || !Ss) return 0;
  std::vector<cpr_opts> op(B);
  std::vector<ProbSpec> specs(B);
  for (int b = 0; b < B; ++b) {
    if (check_tensor(&Xs[b], false) || check_rank_samples(Rs[b], Ss[b])) return 0;
    if (Xs[b].dtype != Xs[0].dtype) return 0;
    op[b] = opts ? opts[b] : defaults();
    specs[b] = ProbSpec{&Xs[b], Rs[b], Ss[b], op[b].fit_samples, &op[b], nullptr, nullptr};
  }
  return make_plan(B, specs.data(), mix, nullptr).bytes;
}

int cpr_cprand_batched(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss, const cpr_opts* opts, int mix,
                       cpr_ktensor* outs, cpr_result* results, void* ws, size_t ws_bytes, void* stream) {
  return run_batched(B, Xs, Rs, Ss, opts, mix ? 1 : 0, outs, results, ws, ws_bytes, (cudaStream_t)stream);
}

// ---- CPRAND-MIX in its complex form (Alg. 4): unitary-DFT mixing, real factors, host-driven loop ----
namespace {
struct CfLayout {
  double* signs[kMaxOrder];
  double* table;
  float* tab[kMaxOrder];
  float2* W[kMaxOrder];
  float2* Xh;                // the mixed tensor, standard layout (complex)
  float2* tmp;               // the other buffer of the pass chain
  float2* rep[kMaxOrder];    // mode-n unfolding copies, n >= 1
  float2* Ah[kMaxOrder];     // mixed factors
  uint32_t* idx;             // S x N
  float* Xr;                 // Imax x 2S
  double* Zr;                // 2S x R
  double* G;
  double* Gi;
  double* M;                 // Imax x R
  uint32_t* fidx;            // P_hat x N
  double* fx;                // P_hat
  double* fpart;             // fit partial sums
  double* npart;             // norm partial sums
  int* err;                  // [0] wait expired, [1] singular Gram
};

size_t cf_layout(Carver& c, const cpr_tensor* X, int R, int64_t S, int64_t P_hat, CfLayout& L) {
  const int N = X->order;
  const int64_t P = prod_dims(X);
  int64_t imax = 0;
  for (int n = 0; n < N; ++n) imax = std::max(imax, X->dims[n]);
  for (int n = 0; n < N; ++n) {
    const size_t I = (size_t)X->dims[n];
    L.signs[n] = c.take<double>(I);
    L.tab[n] = c.take<float>(5 * I);
    L.W[n] = c.take<float2>(I * I);
    L.Ah[n] = c.take<float2>(I * (size_t)R);
  }
  L.table = c.take<double>((size_t)4 * imax);
  L.Xh = c.take<float2>((size_t)P);
  L.tmp = c.take<float2>((size_t)P);
  L.rep[0] = L.Xh;
  for (int n = 1; n < N; ++n) L.rep[n] = c.take<float2>((size_t)P);
  L.idx = c.take<uint32_t>((size_t)S * N);
  L.Xr = c.take<float>((size_t)imax * 2 * S);
  L.Zr = c.take<double>((size_t)3 * S * R);   // FP64 rows (2S x R), then their FP32 copy
  L.G = c.take<double>((size_t)R * R);
  L.Gi = c.take<double>((size_t)R * R);
  L.M = c.take<double>((size_t)imax * R);
  L.fidx = c.take<uint32_t>((size_t)P_hat * N);
  L.fx = c.take<double>((size_t)P_hat);
  L.fpart = c.take<double>((size_t)cf_fit_blocks((int)P_hat));
  L.npart = c.take<double>((size_t)sumsq_blocks(P));
  L.err = c.take<int>(4);
  return align256(c.off) + 256;
}

int cf_check(const cpr_tensor* X, int R, int64_t S, const cpr_opts& o) {
  if (int st = check_tensor(X, false)) return st;
  if (X->dtype != CPR_F32 || check_rank_samples(R, S)) return CPR_EINVAL;
  if (!mix_cfft_supported(X->order, X->dims)) return CPR_EINVAL;
  for (int n = 0; n < X->order; ++n)
    if (X->dims[n] > 6000) return CPR_EINVAL;   // the unmixing kernel stages 4 fibers in shared memory
  if (o.fit_samples < 1 || o.fit_samples > INT32_MAX || S > INT32_MAX / 2) return CPR_EINVAL;
  return CPR_OK;
}
}  // namespace

size_t cpr_cprand_mix_fft_workspace_size(const cpr_tensor* X, int R, int64_t S, const cpr_opts* opts) {
  const cpr_opts o = opts ? *opts : defaults();
  if (cf_check(X, R, S, o)) return 0;
  Carver c(nullptr);
  CfLayout L;
  return cf_layout(c, X, R, S, o.fit_samples, L);
}

int cpr_cprand_mix_fft(const cpr_tensor* X, int R, int64_t S, const cpr_opts* opts, cpr_ktensor* out,
                       cpr_result* result, void* ws, size_t ws_bytes, void* stream) {
  const cpr_opts o = opts ? *opts : defaults();
  if (!X || !X->data) return CPR_EINVAL;
  if (int st = cf_check(X, R, S, o)) return st;
  if (int st = check_ktensor(out, X, R)) return st;
  if (o.init_from_out) return CPR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int N = X->order;
  const int64_t P = prod_dims(X);
  const int Ph = (int)o.fit_samples;
  Carver cm(nullptr);
  CfLayout L;
  if (int st = check_ws(ws, ws_bytes, cf_layout(cm, X, R, S, Ph, L))) return st;
  Carver cw(ws);
  cf_layout(cw, X, R, S, Ph, L);
  int64_t launches = 0;
  PhaseEvents ph;
  if (int st = ph.mark(0, s)) return st;
  CPR_CUDA(cudaMemsetAsync(L.err, 0, 4 * sizeof(int), s));
  // ||X|| (FP64 partial sums, summed on the host in a fixed order)
  const int nblk = sumsq_blocks(P);
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_sumsq(X->data, X->dtype, P, L.npart, nblk, s));
  // operators: signs (Philox), FFT tables, W = F D; the mixed tensor by N unitary-DFT passes
  for (int n = 0; n < N; ++n) {
    const int I = (int)X->dims[n];
    CPR_LAUNCH(CPR_KERNEL_OTHER, launch_build_mix_ops(I, o.seed, o.batch_index, n, L.table, nullptr, nullptr, nullptr,
                                                      L.signs[n], s, L.tab[n]));
    CPR_LAUNCH(CPR_KERNEL_OTHER, launch_cf_ops(I, L.signs[n], L.W[n], s));
  }
  {
    void* bufs[2] = {L.Xh, L.tmp};
    const void* U = X->data;
    for (int n = 0; n < N; ++n) {
      void* y = bufs[(N - 1 - n) & 1];
      void* ys = n == N - 1 ? static_cast<void*>(L.rep[N - 1]) : nullptr;
      CPR_LAUNCH(CPR_KERNEL_MIX, launch_mix_cfft(U, n == 0, y, ys, L.tab[n], N, X->dims, n, L.err, s));
      U = y;
    }
    for (int n = 1; n < N - 1; ++n)   // 8-byte entries: the unfolding copy moves them as FP64 words
      CPR_LAUNCH(CPR_KERNEL_OTHER, launch_unfold_copy(L.Xh, L.rep[n], CPR_F64, N, X->dims, n, s));
  }
  // initial factors (the init stream, as CPRAND) and their mixed copies; the fit entries
  for (int m = 1; m < N; ++m) {
    const int I = (int)X->dims[m];
    CPR_LAUNCH(CPR_KERNEL_OTHER, launch_cf_init(I, R, m, o.seed, o.batch_index, out->factors[m], s));
    CPR_LAUNCH(CPR_KERNEL_OTHER, launch_cf_mix_factor(I, R, L.W[m], out->factors[m], L.Ah[m], s));
  }
  CPR_LAUNCH(CPR_KERNEL_OTHER,
             launch_cf_fit_setup(static_cast<const float*>(X->data), N, X->dims, R, Ph, o.seed, o.batch_index, L.fidx,
                                 L.fx, s));
  std::vector<double> npart(nblk);
  CPR_CUDA(cudaMemcpyAsync(npart.data(), L.npart, sizeof(double) * nblk, cudaMemcpyDeviceToHost, s));
  CPR_CUDA(cudaStreamSynchronize(s));
  double nx2 = 0.0;
  for (double v : npart) nx2 += v;
  const double normx = sqrt(nx2);
  if (int st = ph.mark(1, s)) return st;
  // outer iterations; the stopping rules of Sec. 4.2 on the host after every iteration
  const int cap = o.fixed_iters > 0 ? o.fixed_iters : o.max_iters;
  const int fb = cf_fit_blocks(Ph);
  std::vector<double> fpart(fb);
  int errs[4] = {0, 0, 0, 0};
  double best = -1e300, last = 0.0, fit = 0.0;
  int iters = 0, stall = 0, status = CPR_OK;
  const float2* Ahc[kMaxOrder];
  const double* Ac[kMaxOrder];
  for (int m = 0; m < N; ++m) {
    Ahc[m] = L.Ah[m];
    Ac[m] = out->factors[m];
  }
  while (iters < cap) {
    const uint32_t t = o.first_iter + (uint32_t)iters;
    for (int n = 0; n < N; ++n) {
      CPR_LAUNCH(CPR_KERNEL_SAMPLE_SKR,
                 launch_sample_only(X->data, N, X->dims, n, S, o.seed, o.batch_index, t, L.idx, nullptr, s));
      CPR_LAUNCH(CPR_KERNEL_SOLVE, launch_cf_update(L.rep[n], L.idx, L.W[n], Ahc, N, X->dims, n, (int)S, R, L.Xr,
                                                    L.Zr, L.G, L.Gi, L.M, out->factors[n], out->lambda, L.err + 1, s));
      CPR_LAUNCH(CPR_KERNEL_SOLVE, launch_cf_mix_factor((int)X->dims[n], R, L.W[n], out->factors[n], L.Ah[n], s));
    }
    CPR_LAUNCH(CPR_KERNEL_FIT, launch_cf_fit(Ac, out->lambda, N, X->dims, R, Ph, L.fidx, L.fx, L.fpart, s));
    CPR_CUDA(cudaMemcpyAsync(fpart.data(), L.fpart, sizeof(double) * fb, cudaMemcpyDeviceToHost, s));
    CPR_CUDA(cudaMemcpyAsync(errs, L.err, sizeof(errs), cudaMemcpyDeviceToHost, s));
    CPR_CUDA(cudaStreamSynchronize(s));
    double e2 = 0.0;
    for (double v : fpart) e2 += v;
    const double v = (double)P / (double)Ph * e2;
    fit = 1.0 - sqrt(v) / normx;
    if (o.fit_trace_dev) CPR_CUDA(cudaMemcpyAsync(o.fit_trace_dev + iters, &fit, sizeof(double), cudaMemcpyHostToDevice, s));
    ++iters;
    bool stop = false;
    if (errs[0]) {
      status = CPR_ETIMEOUT;
      stop = true;
    } else if (errs[1]) {
      status = CPR_ESINGULAR;
      stop = true;
    } else if (!std::isfinite(fit)) {
      status = CPR_ENONFINITE;
      stop = true;
    } else if (o.fixed_iters > 0) {
      stop = iters >= o.fixed_iters;
    } else {
      if (fit > best) {
        best = fit;
        stall = 0;
      } else {
        ++stall;
      }
      if (iters >= o.max_iters) stop = true;
      if (iters >= 2 && fabs(fit - last) <= o.fit_tol) stop = true;
      if (o.noise_eta >= 0.0 && fit >= 1.0 - 1.2 * o.noise_eta) stop = true;
      if (o.stall_iters > 0 && stall >= o.stall_iters) stop = true;
    }
    last = fit;
    if (stop) break;
  }
  if (int st = ph.mark(2, s)) return st;
  if (int st = ph.mark(3, s)) return st;
  CPR_CUDA(cudaStreamSynchronize(s));
  if (result) {
    result->iters = iters;
    result->status = status;
    result->fit_est = fit;
    result->norm_x = normx;
    result->kernel_launches = launches;
    result->ms_setup = ph.ms(0, 1);
    result->ms_iterate = ph.ms(1, 2);
    result->ms_finish = ph.ms(2, 3);
  }
  return CPR_OK;
}

int cpr_cp_als(const cpr_tensor* X, int R, const cpr_opts* opts, cpr_ktensor* out, cpr_result* result, void* ws,
               size_t ws_bytes, void* stream) {
  return run_cp_als(X, R, opts, out, result, ws, ws_bytes, (cudaStream_t)stream);
}

int cpr_mttkrp(const cpr_tensor* X, const cpr_ktensor* K, int mode, double* M_dev, void* ws, size_t ws_bytes,
               void* stream) {
  if (int st = check_tensor(X, true)) return st;
  if (!K || !M_dev) return CPR_EINVAL;
  const int R = K->rank;
  if (R < 1 || R > CPR_MAX_RANK) return CPR_EINVAL;
  if (K->order != X->order) return CPR_EINVAL;
  for (int n = 0; n < X->order; ++n)
    if (K->dims[n] != X->dims[n] || !K->factors[n]) return CPR_EINVAL;
  if (mode < 0 || mode >= X->order) return CPR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cpr_opts o = defaults();
  ProbSpec sp{X, R, 0, 0, &o, K->factors, K->lambda};
  const Plan measure = make_plan(1, &sp, 0, nullptr, 1, 0);
  if (int st = check_ws(ws, ws_bytes, measure.bytes)) return st;
  Plan pl = make_plan(1, &sp, 0, ws, 1, mode);
  CPR_CUDA(prepare_kernel_attributes());
  const Prob& p = pl.probs[0];
  int64_t launches = 0;
  CPR_CUDA(cudaMemcpyAsync(pl.d_probs, pl.probs.data(), sizeof(Prob), cudaMemcpyHostToDevice, s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_init_state(pl.d_probs, 1, s));
  if (mode > 0)
    CPR_LAUNCH(CPR_KERNEL_OTHER,
               launch_unfold_copy(p.X, const_cast<void*>(p.Xrep[mode]), p.dtype, p.N, p.dims, mode, s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_init_factors(pl.d_probs, pl.g, 1, s));
  CPR_LAUNCH(CPR_KERNEL_CONTRACT, launch_mttkrp(pl.d_probs, p, mode, s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_mttkrp_fold(pl.d_probs, p, mode, M_dev, s));
  return CPR_OK;
}

int cpr_sample_indices(const cpr_tensor* X, int mode, int64_t S, uint64_t seed, uint32_t b, uint32_t t,
                       uint32_t* idx_dev, int64_t* off_dev, void* stream) {
  if (int st = check_tensor(X, false)) return st;
  if (mode < 0 || mode >= X->order || S < 0 || S > INT32_MAX) return CPR_EINVAL;
  if (S > 0 && !idx_dev && !off_dev) return CPR_EINVAL;
  CPR_CUDA(launch_sample_only(X->data, X->order, X->dims, mode, S, seed, b, t, idx_dev, off_dev,
                              (cudaStream_t)stream));
  return CPR_OK;
}

int cpr_gather_fibers(const cpr_tensor* X, int mode, int64_t S, const int64_t* off_dev, void* xs_dev, void* stream) {
  if (int st = check_tensor(X, true)) return st;
  if (mode < 0 || mode >= X->order || S < 0 || S > INT32_MAX) return CPR_EINVAL;
  if (S > 0 && (!off_dev || !xs_dev)) return CPR_EINVAL;
  int64_t st = 1;
  for (int m = 0; m < mode; ++m) st *= X->dims[m];
  CPR_CUDA(launch_gather_only(X->data, X->dtype, X->dims[mode], st, S, off_dev, xs_dev, (cudaStream_t)stream));
  return CPR_OK;
}

int cpr_sampled_update(const cpr_tensor* X, cpr_ktensor* K, int mode, int64_t S, uint64_t seed, uint32_t b,
                       uint32_t t, cpr_result* result, void* ws, size_t ws_bytes, void* stream) {
  if (int st = check_tensor(X, true)) return st;
  if (!K) return CPR_EINVAL;
  const int R = K->rank;
  if (int st = check_rank_samples(R, S)) return st;
  if (int st = check_ktensor(K, X, R)) return st;
  if (mode < 0 || mode >= X->order) return CPR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cpr_opts o = defaults();
  o.seed = seed;
  o.batch_index = b;
  o.first_iter = t;
  o.fixed_iters = 1;
  o.layout = 1;
  ProbSpec sp{X, R, S, 0, &o, K->factors, K->lambda};
  const Plan measure = make_plan(1, &sp, 0, nullptr);
  if (int st = check_ws(ws, ws_bytes, measure.bytes)) return st;
  Plan pl = make_plan(1, &sp, 0, ws);
  CPR_CUDA(prepare_kernel_attributes());
  int64_t launches = 0;
  CPR_CUDA(cudaMemcpyAsync(pl.d_probs, pl.probs.data(), sizeof(Prob), cudaMemcpyHostToDevice, s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_init_state(pl.d_probs, 1, s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_init_factors(pl.d_probs, pl.g, 1, s));
  if (int st = enqueue_mode_update(pl, mode, s, launches)) return st;
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_finalize(pl.d_probs, pl.g, mode, s));
  if (result) {
    State h;
    CPR_CUDA(cudaMemcpyAsync(&h, pl.d_states, sizeof(State), cudaMemcpyDeviceToHost, s));
    CPR_CUDA(cudaStreamSynchronize(s));
    result->iters = 0;
    result->status = h.status;
    result->fit_est = NAN;
    result->norm_x = NAN;
    result->kernel_launches = launches;
    result->ms_setup = result->ms_iterate = result->ms_finish = NAN;
  }
  return CPR_OK;
}

int cpr_fit_estimate(const cpr_tensor* X, const cpr_ktensor* K, int64_t P_hat, uint64_t seed, uint32_t b,
                     double norm_x, double* fit_host, void* ws, size_t ws_bytes, void* stream) {
  if (int st = check_tensor(X, true)) return st;
  if (!K || !fit_host) return CPR_EINVAL;
  const int R = K->rank;
  if (R < 1 || R > CPR_MAX_RANK) return CPR_EINVAL;
  if (int st = check_ktensor(K, X, R)) return st;
  if (P_hat < 1 || P_hat > INT32_MAX) return CPR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cpr_opts o = defaults();
  o.seed = seed;
  o.batch_index = b;
  o.fixed_iters = 1;
  o.fit_samples = P_hat;
  ProbSpec sp{X, R, 0, P_hat, &o, K->factors, K->lambda};
  const Plan measure = make_plan(1, &sp, 0, nullptr);
  if (int st = check_ws(ws, ws_bytes, measure.bytes)) return st;
  Plan pl = make_plan(1, &sp, 0, ws);
  int64_t launches = 0;
  CPR_CUDA(cudaMemcpyAsync(pl.d_probs, pl.probs.data(), sizeof(Prob), cudaMemcpyHostToDevice, s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_init_state(pl.d_probs, 1, s));
  if (norm_x < 0) {
    CPR_LAUNCH(CPR_KERNEL_OTHER, launch_sumsq(X->data, X->dtype, pl.probs[0].P, pl.d_normpart, pl.normblk, s));
    CPR_LAUNCH(CPR_KERNEL_OTHER, launch_sumsq_finish(pl.d_normpart, pl.normblk, nullptr, pl.d_states, 1, s));
  } else {
    CPR_CUDA(cudaMemcpyAsync(&pl.d_states[0].norm_x, &norm_x, sizeof(double), cudaMemcpyHostToDevice, s));
  }
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_init_factors(pl.d_probs, pl.g, 1, s));
  CPR_LAUNCH(CPR_KERNEL_OTHER, launch_fit_setup(pl.d_probs, pl.g, s));
  CPR_LAUNCH(CPR_KERNEL_FIT, launch_fit(pl.d_probs, pl.g, s));
  State h;
  CPR_CUDA(cudaMemcpyAsync(&h, pl.d_states, sizeof(State), cudaMemcpyDeviceToHost, s));
  CPR_CUDA(cudaStreamSynchronize(s));
  *fit_host = h.last_fit;
  return CPR_OK;
}

int cpr_mix_tensor(const cpr_tensor* X, void* out_dev, uint64_t seed, uint32_t b, void* ws, size_t ws_bytes,
                   void* stream) {
  if (int st = check_tensor(X, true)) return st;
  if (!out_dev || out_dev == X->data) return CPR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  const int N = X->order, dt = X->dtype;
  const int64_t P = prod_dims(X);
  Carver cv(nullptr);
  int64_t imax = 0;
  for (int n = 0; n < N; ++n) imax = std::max(imax, X->dims[n]);
  auto lay = [&](Carver& c, float** W32, float** Wlo, double** W64, double** F64, double** sg, double** table,
                 void** tmp, void** tmp2, int** err) {
    for (int n = 0; n < N; ++n) {
      const size_t I = (size_t)X->dims[n];
      W32[n] = dt == CPR_F64 ? nullptr : c.take<float>(I * I);
      Wlo[n] = dt == CPR_F32 ? c.take<float>(I * I) : nullptr;
      W64[n] = dt == CPR_F64 ? c.take<double>(I * I) : nullptr;
      F64[n] = c.take<double>(I * I);
      sg[n] = c.take<double>(I);
    }
    *table = c.take<double>((size_t)4 * imax);
    *tmp = c.take<unsigned char>((size_t)P * elem_size(dt));
    *tmp2 = dt == CPR_F32 ? c.take<unsigned char>((size_t)P * elem_size(dt)) : nullptr;
    *err = c.take<int>(16);   // [0] device error, [4..] mixing maxima
  };
  float *W32[kMaxOrder], *Wlo[kMaxOrder];
  double *W64[kMaxOrder], *F64[kMaxOrder], *sg[kMaxOrder], *table;
  void *tmp, *tmp2;
  int* derr;
  lay(cv, W32, Wlo, W64, F64, sg, &table, &tmp, &tmp2, &derr);
  if (int st = check_ws(ws, ws_bytes, align256(cv.off))) return st;
  Carver cw(ws);
  lay(cw, W32, Wlo, W64, F64, sg, &table, &tmp, &tmp2, &derr);
  CPR_CUDA(cudaMemsetAsync(derr, 0, sizeof(int), s));
  int64_t launches = 0;
  const bool fftm = fft_mixing(dt, N, X->dims) && W32[0] != nullptr;
  for (int n = 0; n < N; ++n)
    CPR_LAUNCH(CPR_KERNEL_OTHER, launch_build_mix_ops((int)X->dims[n], seed, b, n, table, fftm ? nullptr : W32[n],
                                                      W64[n], F64[n], sg[n], s, fftm ? W32[n] : nullptr));
  bool unused = false;
  if (int st = enqueue_mixing(X->data, out_dev, tmp, tmp2, nullptr, dt, N, X->dims, W32, Wlo, W64, sg, derr,
                              reinterpret_cast<unsigned*>(derr + 4), false, s, launches, &unused, nullptr))
    return st;
  return CPR_OK;
}

int cpr_unmix_factors(const cpr_ktensor* Khat, cpr_ktensor* out, uint64_t seed, uint32_t b, void* ws,
                      size_t ws_bytes, void* stream) {
  if (!Khat || !out || Khat->order != out->order || Khat->rank != out->rank) return CPR_EINVAL;
  if (Khat->order < 2 || Khat->order > CPR_MAX_ORDER || Khat->rank < 1 || Khat->rank > CPR_MAX_RANK)
    return CPR_EINVAL;
  const int N = Khat->order, R = Khat->rank;
  for (int n = 0; n < N; ++n) {
    if (Khat->dims[n] != out->dims[n] || Khat->dims[n] < 1 || Khat->dims[n] >= (int64_t(1) << 31)) return CPR_EINVAL;
    if (!Khat->factors[n] || !out->factors[n] || Khat->factors[n] == out->factors[n]) return CPR_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  Carver cv(nullptr);
  for (int n = 0; n < N; ++n) {
    cv.take<double>((size_t)Khat->dims[n] * Khat->dims[n]);
    cv.take<double>((size_t)Khat->dims[n]);
    cv.take<double>((size_t)4 * Khat->dims[n]);
  }
  if (int st = check_ws(ws, ws_bytes, align256(cv.off))) return st;
  Carver cw(ws);
  for (int n = 0; n < N; ++n) {
    const int I = (int)Khat->dims[n];
    double* F64 = cw.take<double>((size_t)I * I);
    double* sg = cw.take<double>((size_t)I);
    double* table = cw.take<double>((size_t)4 * I);
    CPR_CUDA(launch_build_mix_ops(I, seed, b, n, table, nullptr, nullptr, F64, sg, s));
    CPR_CUDA(launch_unmix(Khat->factors[n], out->factors[n], F64, sg, I, R, s));
  }
  if (Khat->lambda && out->lambda && Khat->lambda != out->lambda)
    CPR_CUDA(cudaMemcpyAsync(out->lambda, Khat->lambda, sizeof(double) * R, cudaMemcpyDeviceToDevice, s));
  return CPR_OK;
}

int cpr_cprand_mix_batched(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss, const cpr_opts* opts,
                           cpr_ktensor* outs, cpr_result* results, void* ws, size_t ws_bytes, void* stream) {
  return run_batched(B, Xs, Rs, Ss, opts, 1, outs, results, ws, ws_bytes, (cudaStream_t)stream);
}

int cpr_autotune(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss, const cpr_opts* opts, int mix,
                 cpr_ktensor* outs, void* ws, size_t ws_bytes, void* stream, int trial_iters, cpr_schedule* best) {
  if (B < 1 || !Xs || !Rs || !Ss || !outs || trial_iters < 1) return CPR_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  std::vector<cpr_opts> op(B);
  for (int b = 0; b < B; ++b) {
    op[b] = opts ? opts[b] : defaults();
    if (!opts) op[b].batch_index = (uint32_t)b;
    op[b].fixed_iters = trial_iters;     // the same iterations for every candidate
    op[b].fit_trace_dev = nullptr;
    op[b].user_samples = nullptr;
    op[b].user_S = 0;
  }
  std::vector<cpr_result> res(B);
  // candidates: the replicated / distributed clusters, the whole GPU with three split widths, the
  // graph with three split densities (those that do not apply return CPR_EINVAL and are skipped)
  std::vector<Schedule> cand;
  Schedule c;
  c.loop_path = 1; cand.push_back(c);
  c.loop_path = 4; cand.push_back(c);
  for (int gm : {16, 32, 64}) { c = Schedule{}; c.loop_path = 5; c.grid_min_split = gm; cand.push_back(c); }
  for (int sp : {1, 2, 4}) { c = Schedule{}; c.loop_path = 2; c.split_per_sm = sp; cand.push_back(c); }
  // warm-up (kernel loading), the default schedule
  Schedule d;
  if (int st = run_batched(B, Xs, Rs, Ss, op.data(), mix, outs, res.data(), ws, ws_bytes, s, &d)) return st;
  double best_ms = INFINITY;
  Schedule win;
  for (const Schedule& sc : cand) {
    const int st = run_batched(B, Xs, Rs, Ss, op.data(), mix, outs, res.data(), ws, ws_bytes, s, &sc);
    if (st == CPR_EINVAL) continue;   // this engine does not take the batch
    if (st != CPR_OK) return st;
    bool ok = true;
    int iters = 0;
    for (int b = 0; b < B; ++b) {
      ok = ok && res[b].status == CPR_OK;
      iters = std::max(iters, (int)res[b].iters);
    }
    if (!ok || iters < 1) continue;
    const double ms = res[0].ms_iterate / iters;
    if (ms < best_ms) {
      best_ms = ms;
      win = sc;
    }
  }
  if (!(best_ms < INFINITY)) return CPR_EINVAL;
  {
    TuneTable& t = tune_table();
    std::lock_guard<std::mutex> lk(t.mu);
    t.map[tune_key(B, Xs, Rs, Ss, mix)] = TuneEntry{win, best_ms};
  }
  if (best) {
    best->loop_path = win.loop_path;
    best->split_per_sm = win.split_per_sm;
    best->grid_min_split = win.grid_min_split;
    best->pad = 0;
    best->ms_per_iter = best_ms;
  }
  return CPR_OK;
}

int cpr_tune_lookup(int B, const cpr_tensor* Xs, const int* Rs, const int64_t* Ss, int mix, cpr_schedule* out) {
  if (B < 1 || !Xs || !Rs || !Ss || !out) return CPR_EINVAL;
  for (int b = 0; b < B; ++b)
    if (check_tensor(&Xs[b], false)) return CPR_EINVAL;
  Schedule sc;
  double ms = 0.0;
  if (!tune_lookup(tune_key(B, Xs, Rs, Ss, mix), &sc, &ms)) {
    memset(out, 0, sizeof(*out));
    return CPR_EINVAL;
  }
  out->loop_path = sc.loop_path;
  out->split_per_sm = sc.split_per_sm;
  out->grid_min_split = sc.grid_min_split;
  out->pad = 0;
  out->ms_per_iter = ms;
  return CPR_OK;
}

int cpr_tune_save(const char* path) {
  if (!path) return CPR_EINVAL;
  TuneTable& t = tune_table();
  std::lock_guard<std::mutex> lk(t.mu);
  FILE* f = fopen(path, "w");
  if (!f) return CPR_EINVAL;
  for (const auto& kv : t.map)
    fprintf(f, "%s %d %d %d %.17g\n", kv.first.c_str(), kv.second.sch.loop_path, kv.second.sch.split_per_sm,
            kv.second.sch.grid_min_split, kv.second.ms_per_iter);
  return fclose(f) == 0 ? CPR_OK : CPR_EINVAL;
}

int cpr_tune_load(const char* path) {
  if (!path) return CPR_EINVAL;
  TuneTable& t = tune_table();
  std::lock_guard<std::mutex> lk(t.mu);
  return tune_load_locked(t, path);
}

void cpr_tune_clear(void) {
  TuneTable& t = tune_table();
  std::lock_guard<std::mutex> lk(t.mu);
  t.map.clear();
  t.env_loaded = true;   // a cleared table stays empty until a load or a tuning run
}

int cpr_set_contract_engine(int engine) {
  if (engine < CPR_CONTRACT_AUTO || engine > CPR_CONTRACT_FMA) return -1;
  return g_contract_engine.exchange(engine);
}

int cpr_set_mix_engine(int engine) {
  if (engine != CPR_MIX_AUTO && engine != CPR_MIX_FFT && engine != CPR_MIX_DENSE) return -1;
  return g_mix_engine.exchange(engine);
}

int cpr_profile_begin(unsigned mask) {
  Profiler& p = prof();
  std::vector<ProfRec> old;
  {
    std::lock_guard<std::mutex> lk(p.mu);
    old.swap(p.recs);
    p.on = true;
    p.mask = mask;
    for (auto& c : p.counts) c = 0;
  }
  for (auto& r : old) {
    give_event(r.a);
    give_event(r.b);
  }
  return CPR_OK;
}

int cpr_profile_end(double* ms, int64_t* launches) {
  Profiler& p = prof();
  std::vector<ProfRec> recs;
  int64_t counts[CPR_KERNEL_CLASSES];
  {
    std::lock_guard<std::mutex> lk(p.mu);
    recs.swap(p.recs);
    p.on = false;
    memcpy(counts, p.counts, sizeof(counts));
  }
  double tot[CPR_KERNEL_CLASSES] = {};
  int st = CPR_OK;
  for (auto& r : recs) {
    float v = 0.f;
    if (cudaEventSynchronize(r.b) != cudaSuccess || cudaEventElapsedTime(&v, r.a, r.b) != cudaSuccess) st = CPR_ECUDA;
    tot[r.cls] += (double)v;
    give_event(r.a);
    give_event(r.b);
  }
  for (int c = 0; c < CPR_KERNEL_CLASSES; ++c) {
    if (ms) ms[c] = tot[c];
    if (launches) launches[c] = counts[c];
  }
  return st;
}

int cpr_tensor_norm(const cpr_tensor* X, double* norm_host, void* ws, size_t ws_bytes, void* stream) {
  if (int st = check_tensor(X, true)) return st;
  if (!norm_host) return CPR_EINVAL;
  const int64_t P = prod_dims(X);
  const int nblk = sumsq_blocks(P);
  const size_t need = cpr_workspace_size(CPR_METHOD_NORM, X, 1, 1, nullptr);
  if (int st = check_ws(ws, ws_bytes, need)) return st;
  Carver cw(ws);
  double* part = cw.take<double>(nblk);
  double* out = cw.take<double>(1);
  cudaStream_t s = (cudaStream_t)stream;
  CPR_CUDA(launch_sumsq(X->data, X->dtype, P, part, nblk, s));
  CPR_CUDA(launch_sumsq_finish(part, nblk, out, nullptr, 0, s));
  CPR_CUDA(cudaMemcpyAsync(norm_host, out, sizeof(double), cudaMemcpyDeviceToHost, s));
  CPR_CUDA(cudaStreamSynchronize(s));
  return CPR_OK;
}

}  // extern "C"
