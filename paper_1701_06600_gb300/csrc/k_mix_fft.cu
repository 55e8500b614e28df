// Mode-n mixing product by a factored DCT-II (the fast transform of Alg. 5's mixing step).
//
// One pass applies y = F_n D_n x to every mode-n fiber x of the tensor, where F_n is the orthonormal
// DCT-II of length I = I_n (F[k][i] = c_k cos(pi (2i + 1) k / (2I)), c_0 = sqrt(1/I), c_k = sqrt(2/I))
// and D_n the diagonal of random signs.  Instead of the dense I x I product (2I flops per entry) the
// DCT is computed through a complex DFT of the same length:
//   * reorder (even entries ascending, then odd entries descending):
//       v[m] = d[2m] x[2m] for 2m < I,   v[I-1-m] = d[2m+1] x[2m+1] for 2m+1 < I;
//   * V = DFT_I(v), with V[k] = sum_m v[m] exp(-2 pi i m k / I);
//   * y[k] = c_k Re(exp(-i pi k / (2I)) V[k]).
// Two real fibers go through one complex transform (one as the real part, one as the imaginary
// part); they are separated afterwards by the conjugate symmetry of real DFTs:
//   V1[k] = (W[k] + conj(W[I-k])) / 2,   V2[k] = (W[k] - conj(W[I-k])) / (2i).
// The DFT is a Stockham autosort FFT whose stages have radices up to 25: a stage of radix R = R1 R2
// holds the R values of a butterfly in registers and transforms them as R2 DFTs of length R1, a
// twiddle, and R1 DFTs of length R2 (Cooley-Tukey inside the butterfly), so that I = 400 = 25 x 16
// takes two shared-memory round trips.  About 5 I log2 I flops per pair of fibers instead of the
// dense product's 4 I^2.
//
// Data flow: a CTA owns BJ fibers that differ only in the index of one other mode v (consecutive
// i_v), loads them (each fiber is contiguous in the mode-n unfolding the pass reads; one bulk copy
// per fiber), transforms them in shared memory and writes the result in the mode-v unfolding layout,
// where those BJ fibers are adjacent for every output index k.  Choosing v = n + 1 makes every pass
// write exactly the layout the next pass reads, so the chain of N passes needs no transposition
// copies; the last pass (v = 0) writes the standard layout and, when asked, its own mode-n unfolding
// (the copy the sampled gathers of mode n read).
//
// Shared memory: the fibers land as rows (fiber f in row f, Ipad floats apart); the reorder turns
// rows 2p and 2p + 1 into the interleaved complex sequence p (Ipad complex values from row 2p on);
// the stages run in place (each thread keeps its butterflies in registers between a stage's reads
// and its writes); the final rotation writes (y_{2p}[k], y_{2p+1}[k]) back over the complex value k.
//
// Accuracy: FP32 arithmetic with twiddles rounded once from FP64; below 1e-6 relative for the sizes
// used here.  Every mbarrier wait is bounded: on expiry the kernel records an error and returns.
#include <string.h>

#include <algorithm>
#include <utility>

#include "internal.cuh"

namespace cpr {
namespace {

constexpr uint32_t kFftWaitLimit = 1u << 24;
constexpr uint32_t kFftDrainLimit = 1u << 26;   // second wait after an expiry, before the CTA leaves
constexpr int kSlots = 32;          // complex values a thread holds in a stage
constexpr int kMaxStages = 16;
constexpr int kFftMaxSmem = 200 * 1024;
constexpr int kMaxFftLen = 8192;    // keeps the multiply-high divisions exact
constexpr int kBsMinLen = 33;       // Bluestein form for I >= 33: its tables and FP64 scratch fit I^2 floats
constexpr int kBsMaxConv = 4096;    // longest Bluestein convolution
// the stage radices, in the order a plan's stages run; radix R = R1 x R2 (R2 = 1 for the plain ones)
constexpr int kNumRadices = 14;
constexpr int kRadR1[kNumRadices] = {5, 5, 4, 5, 4, 5, 3, 4, 7, 3, 5, 4, 3, 2};
constexpr int kRadR2[kNumRadices] = {5, 4, 4, 3, 3, 2, 3, 2, 1, 2, 1, 1, 1, 1};

struct StageTab {
  int L, Ns, tstep, rix;   // butterflies per sequence (I / R), radix product before, I / (Ns R), radix index
  uint32_t mL, mNs, r0, r1;   // ceil(2^32 / L), ceil(2^32 / Ns)
};

struct FftArgs {
  const void* U;        // input: the mode-n unfolding, fibers of length I contiguous
  void* yv;             // output in the mode-v unfolding layout
  void* ysame;          // optional output in the input's layout (mode-n unfolding)
  const float* tab;     // twiddles (2I), post-scales (2I), signs (I)
  int I, Ipad, BJ, S, nst, bulk;
  uint32_t mH2;         // ceil(2^32 / (I / 2 + 1))
  float cscale;         // complex transform: 1 / sqrt(I) (the unitary DFT)
  StageTab st[kMaxStages];
  int64_t Iv;           // extent of the mode the CTA's fibers run along
  int64_t rs_in_v;      // input row stride of one step in i_v
  int64_t out_k;        // output stride of one step in k (= i_n): I_v times the mode-v row stride of n
  int64_t nchunks;      // ceil(Iv / BJ)
  int64_t nblocks;      // fiber blocks of the pass (nchunks x the remaining modes' extents)
  int no;               // number of remaining modes (not n, not v)
  int64_t oext[kMaxOrder], o_in[kMaxOrder], o_out[kMaxOrder];
  int vec_v;            // the mode-v output admits 16-byte stores of 4 adjacent fibers
  int vec_in;           // BF16 input rows admit 8-byte loads of 4 entries
  int* err;
  // Bluestein (chirp-z) form for lengths with a prime factor above 7: the length-I DFT as a cyclic
  // convolution of length M (7-smooth, M >= 2 I - 1); st / nst then describe the length-M stages
  int M, Mpad;
  uint32_t mM, mI;      // ceil(2^32 / M), ceil(2^32 / I)
  // when given, CTA b writes the sum of squares of its input fibers to normpart[b] (FP64), so that
  // the pass that reads the caller's tensor also yields ||X||^2 (summed by launch_sumsq_finish)
  double* normpart;
};

__device__ __forceinline__ uint32_t smem_u32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ bool fft_mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}

__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}

template <typename T> __device__ __forceinline__ float ld_as_float(const T* p);
template <> __device__ __forceinline__ float ld_as_float<float>(const float* p) { return *p; }
template <> __device__ __forceinline__ float ld_as_float<__nv_bfloat16>(const __nv_bfloat16* p) {
  return __bfloat162float(*p);
}
template <typename T> __device__ __forceinline__ T from_float(float v);
template <> __device__ __forceinline__ float from_float<float>(float v) { return v; }
template <> __device__ __forceinline__ __nv_bfloat16 from_float<__nv_bfloat16>(float v) { return __float2bfloat16(v); }

// In-register DFT of R values, out[q] = sum_r v[r] w^(r q), w = exp(-2 pi i / R).  For odd R the
// terms r and R - r are combined: out[q] = v0 + sum_r cos(2 pi r q/R) (v_r + v_{R-r})
// - i sum_r sin(2 pi r q/R) (v_r - v_{R-r}) and out[R-q] the same with +i.  rc[m] = (cos, sin) of
// 2 pi m / R for m = 1 .. (R-1)/2.
template <int R>
__device__ __forceinline__ void dft(float2 (&v)[R], const float2 (&rc)[R / 2 + 1]) {
  if constexpr (R == 2) {
    const float2 a = v[0], b = v[1];
    v[0] = make_float2(a.x + b.x, a.y + b.y);
    v[1] = make_float2(a.x - b.x, a.y - b.y);
  } else if constexpr (R == 4) {
    const float2 a = make_float2(v[0].x + v[2].x, v[0].y + v[2].y);
    const float2 b = make_float2(v[0].x - v[2].x, v[0].y - v[2].y);
    const float2 c = make_float2(v[1].x + v[3].x, v[1].y + v[3].y);
    const float2 d = make_float2(v[1].x - v[3].x, v[1].y - v[3].y);   // -i d = (d.y, -d.x)
    v[0] = make_float2(a.x + c.x, a.y + c.y);
    v[2] = make_float2(a.x - c.x, a.y - c.y);
    v[1] = make_float2(b.x + d.y, b.y - d.x);
    v[3] = make_float2(b.x - d.y, b.y + d.x);
  } else {
    constexpr int H = (R - 1) / 2;
    float2 s[H], t[H];
    float2 sum = v[0];
#pragma unroll
    for (int r = 1; r <= H; ++r) {
      s[r - 1] = make_float2(v[r].x + v[R - r].x, v[r].y + v[R - r].y);
      t[r - 1] = make_float2(v[r].x - v[R - r].x, v[r].y - v[R - r].y);
      sum.x += s[r - 1].x;
      sum.y += s[r - 1].y;
    }
    const float2 v0 = v[0];
    v[0] = sum;
#pragma unroll
    for (int q = 1; q <= H; ++q) {
      float2 A = v0, B = make_float2(0.f, 0.f);
#pragma unroll
      for (int r = 1; r <= H; ++r) {
        const int m = (r * q) % R;                 // compile-time after unrolling
        const int mm = m <= H ? m : R - m;
        const float c = rc[mm].x;
        const float sn = m <= H ? rc[mm].y : -rc[mm].y;
        A.x = fmaf(c, s[r - 1].x, A.x);
        A.y = fmaf(c, s[r - 1].y, A.y);
        B.x = fmaf(sn, t[r - 1].x, B.x);
        B.y = fmaf(sn, t[r - 1].y, B.y);
      }
      v[q] = make_float2(A.x + B.y, A.y - B.x);      // A - iB
      v[R - q] = make_float2(A.x - B.y, A.y + B.x);  // A + iB
    }
  }
}

// n / d for n < 2^17 and 1 <= d <= 8192: one multiply-high by m = ceil(2^32 / d) (exact in that range:
// n (m - 2^32 / d) / 2^32 < n / 2^32 < 1 / d), or n itself when d = 1
__device__ __forceinline__ int fdiv(int n, int d, uint32_t m) { return d == 1 ? n : (int)__umulhi((uint32_t)n, m); }

// roots (cos, sin)(2 pi m / R) for m <= R / 2, read from the length-I twiddle table (step = I / R)
template <int R>
__device__ __forceinline__ void load_roots(float2 (&rc)[R / 2 + 1], const float2* tw, int step) {
  rc[0] = make_float2(1.f, 0.f);
#pragma unroll
  for (int m = 1; m <= R / 2; ++m) {
    const float2 w = tw[m * step];   // exp(-2 pi i m / R) = (cos, -sin)
    rc[m] = make_float2(w.x, -w.y);
  }
}

// In-register DFT of R = R1 R2 values (input index r = R2 r1 + r2, output index q = q1 + R1 q2):
// R2 DFTs of length R1 over r1, the twiddle w_R^(r2 q1), R1 DFTs of length R2 over r2.  L = I / R
// (w_R^m = tw[m L]).
template <int R1, int R2>
__device__ __forceinline__ void dft_comp(float2 (&v)[R1 * R2], const float2* tw, int L) {
  constexpr int R = R1 * R2;
  if constexpr (R2 == 1) {
    float2 rc[R1 / 2 + 1];
    load_roots<R1>(rc, tw, L);
    dft<R1>(v, rc);
  } else {
    float2 rc1[R1 / 2 + 1], rc2[R2 / 2 + 1];
    load_roots<R1>(rc1, tw, L * R2);
    load_roots<R2>(rc2, tw, L * R1);
#pragma unroll
    for (int r2 = 0; r2 < R2; ++r2) {
      float2 t[R1];
#pragma unroll
      for (int r1 = 0; r1 < R1; ++r1) t[r1] = v[R2 * r1 + r2];
      dft<R1>(t, rc1);
#pragma unroll
      for (int q1 = 0; q1 < R1; ++q1) v[R2 * q1 + r2] = (r2 && q1) ? cmul(t[q1], tw[r2 * q1 * L]) : t[q1];
    }
    float2 o[R];
#pragma unroll
    for (int q1 = 0; q1 < R1; ++q1) {
      float2 t[R2];
#pragma unroll
      for (int r2 = 0; r2 < R2; ++r2) t[r2] = v[R2 * q1 + r2];
      dft<R2>(t, rc2);
#pragma unroll
      for (int q2 = 0; q2 < R2; ++q2) o[q1 + R1 * q2] = t[q2];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = o[r];
  }
}

// One Stockham stage of radix R = R1 R2 over S interleaved complex sequences (sequence p at
// Z + p Ipad).  Butterfly j of a sequence reads entries j + r L (L = I / R), multiplies entry r by
// w_I^(r (j mod Ns) I / (Ns R)), transforms, and writes entry r to (j / Ns) Ns R + (j mod Ns) + r Ns.
// All reads of the stage finish before any write (the values wait in registers): in place.
// FIRST: the stage reads the real fibers instead (rows 2p and 2p + 1 of the loaded block) in the DCT
// reorder, times their signs: v_p[m] = d[s] (x_{2p}[s], x_{2p+1}[s]) with s = 2m (2m < I) or
// 2(I - 1 - m) + 1; Ns = 1, so no twiddles.
template <int R1, int R2, bool FIRST, int TPB>
__device__ __forceinline__ void fft_stage(float2* Z, int I, int Ipad, int S, const StageTab& sc, int tid,
                                          const float2* tw, const float* sg) {
  constexpr int R = R1 * R2, MAXB = kSlots / R;
  const int L = sc.L, Ns = FIRST ? 1 : sc.Ns, nbt = S * L, tstep = sc.tstep;
  float2 v[MAXB][R];
  int dst[MAXB];
#pragma unroll
  for (int q = 0; q < MAXB; ++q) {
    const int b = tid + q * TPB;
    dst[q] = -1;
    if (b < nbt) {
      const int p = fdiv(b, L, sc.mL), j = b - p * L;
      const int jn = FIRST ? j : fdiv(j, Ns, sc.mNs), k = j - jn * Ns;
      const float2* z = Z + p * Ipad;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const int m = j + r * L;
        float2 x;
        if constexpr (FIRST) {
          const int src = 2 * m < I ? 2 * m : 2 * (I - 1 - m) + 1;
          const float d = sg[src];
          const float* row = reinterpret_cast<const float*>(z);
          x = make_float2(row[src] * d, row[Ipad + src] * d);
        } else {
          x = z[m];
          if (r > 0 && k > 0) x = cmul(x, tw[r * k * tstep]);
        }
        v[q][r] = x;
      }
      dft_comp<R1, R2>(v[q], tw, L);
      dst[q] = p * Ipad + jn * Ns * R + k;
    }
    // one butterfly's loads at a time: otherwise the compiler issues the loads of every butterfly
    // up front and runs out of registers
    asm volatile("" ::: "memory");
  }
  __syncthreads();
#pragma unroll
  for (int q = 0; q < MAXB; ++q)
    if (dst[q] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) Z[dst[q] + r * Ns] = v[q][r];
    }
  __syncthreads();
}

__device__ __forceinline__ void fft_bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* bar) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   smem_u32(dst)),
               "l"(src), "r"(bytes), "r"(smem_u32(bar))
               : "memory");
}

// After a copy wait ran out: report it, then let the CTA's bulk copies land (a second bounded wait
// on the same mbarrier phase) before the CTA leaves, so that no copy targets the shared memory of a
// CTA that has exited.
__device__ __forceinline__ void fft_drain(uint64_t* bar, int* err, int tid) {
  if (tid == 0) {
    atomicExch(err, 1);
    for (uint32_t it = 0; it < kFftDrainLimit && !fft_mbar_try(bar, 0); ++it) __nanosleep(64);
  }
  __syncthreads();
}

// block blk of the pass: its fibers run along mode v from i_v = iv0; returns the fiber count and the
// first fiber's input row and output offset
__device__ __forceinline__ int fft_block(const FftArgs& a, int64_t blk, int64_t& row0, int64_t& out0) {
  const int64_t chunk = blk % a.nchunks;
  int64_t rest = blk / a.nchunks;
  const int64_t iv0 = chunk * a.BJ;
  row0 = iv0 * a.rs_in_v;
  out0 = 0;
  for (int m = 0; m < a.no; ++m) {   // the remaining modes: extent, input row stride, output stride
    const int64_t im = rest % a.oext[m];
    rest /= a.oext[m];
    row0 += im * a.o_in[m];
    out0 += im * a.o_out[m];
  }
  out0 = iv0 + a.Iv * out0;
  return (int)min((int64_t)a.BJ, a.Iv - iv0);
}

// ||fibers||^2 of the CTA's block, once its nf input rows (I FP32 entries each, rows Ipad floats
// apart, Ipad a multiple of 4) are in shared memory and before any stage writes them: 16-byte loads,
// four FP32 accumulators per thread, the warp's sum as an FP32 pair (error-free two-sums: the FP64
// pipe is too slow for one reduction per CTA of every pass), converted to FP64 into part[warp].  The
// caller adds the warps' partials in warp order after a later block barrier (fft_sumsq_store).
// the warp's sum of the lanes' v as an FP32 pair (error-free two-sums), stored in FP64 by lane 0
__device__ __forceinline__ void fft_sumsq_warp(float v, int lane, double* out) {
  float h = v, l = 0.f;
  for (int o = 16; o > 0; o >>= 1) {
    const float h2 = __shfl_xor_sync(0xffffffffu, h, o), l2 = __shfl_xor_sync(0xffffffffu, l, o);
    const float t = __fadd_rn(h, h2), bv = __fsub_rn(t, h);
    const float e = __fadd_rn(__fsub_rn(h, __fsub_rn(t, bv)), __fsub_rn(h2, bv));
    h = t;
    l = __fadd_rn(l, __fadd_rn(l2, e));
  }
  if (lane == 0) *out = (double)h + (double)l;
}
template <int TPB>
__device__ __forceinline__ void fft_sumsq_rows(const float* Y, int nf, int I, int Ipad, int tid, int lane,
                                               double* part) {
  const int I4 = I >> 2;
  float s0 = 0.f, s1 = 0.f, s2 = 0.f, s3 = 0.f;
#pragma unroll 4
  for (int e = tid; e < nf * I4; e += TPB) {
    const int f = e / I4, c = e - f * I4;
    const float4 v = *reinterpret_cast<const float4*>(Y + f * Ipad + 4 * c);
    s0 = fmaf(v.x, v.x, s0);
    s1 = fmaf(v.y, v.y, s1);
    s2 = fmaf(v.z, v.z, s2);
    s3 = fmaf(v.w, v.w, s3);
  }
  for (int e = tid; e < nf * (I - 4 * I4); e += TPB) {   // the entries past the last full vector
    const int f = e / (I - 4 * I4), c = 4 * I4 + e - f * (I - 4 * I4);
    const float x = Y[f * Ipad + c];
    s0 = fmaf(x, x, s0);
  }
  fft_sumsq_warp((s0 + s1) + (s2 + s3), lane, part + (tid >> 5));
}
template <int TPB>
__device__ __forceinline__ void fft_sumsq_store(const FftArgs& a, const double* part, int tid) {
  if (tid == 0) {
    double t = 0.0;
    for (int w = 0; w < TPB / 32; ++w) t += part[w];
    a.normpart[blockIdx.x] = t;
  }
}

// the stages of radix index RIX (one loop per radix: the register arrays of different radices are
// never live at once); the plan lists its stages in radix-index order
template <int RIX, int TPB>
__device__ __forceinline__ void fft_stages_of(float2* Z, int I, int Ipad, int S, int nst, const StageTab* stt, int& st,
                                              int tid, const float2* tw, const float* sg) {
  if (st == 0 && nst > 0 && stt[0].rix == RIX) {
    fft_stage<kRadR1[RIX], kRadR2[RIX], true, TPB>(Z, I, Ipad, S, stt[0], tid, tw, sg);
    ++st;
  }
  for (; st < nst && stt[st].rix == RIX; ++st)
    fft_stage<kRadR1[RIX], kRadR2[RIX], false, TPB>(Z, I, Ipad, S, stt[st], tid, tw, sg);
}

// One CTA per block of fibers (one bulk copy per fiber on the FP32 path).  Several CTAs share an SM,
// so one CTA's copies overlap the others' transforms.
template <typename T, int TPB>
__global__ void __launch_bounds__(TPB, 512 / TPB) k_mix_fft(const __grid_constant__ FftArgs a) {
  extern __shared__ float4 fft_smem4[];
  const int I = a.I, Ipad = a.Ipad, BJ = a.BJ, S = a.S;
  float* Y = reinterpret_cast<float*>(fft_smem4);
  float2* Z = reinterpret_cast<float2*>(Y);
  float2* tw = reinterpret_cast<float2*>(Y + BJ * Ipad);
  float2* post = tw + I;
  float* sg = reinterpret_cast<float*>(post + I);
  uint64_t* bar = reinterpret_cast<uint64_t*>(fft_smem4) + ((BJ * Ipad + 5 * I + 3) / 2);   // 8-byte aligned
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const T* U = static_cast<const T*>(a.U);
  __shared__ StageTab s_st[kMaxStages];
  __shared__ longlong4 s_blk;   // (first fiber's input row, first output offset, fiber count)
  if (tid < kMaxStages) s_st[tid] = a.st[tid];
  if (tid == 0) {   // the block's coordinates (64-bit divisions: once per CTA, not per thread)
    int64_t r0, o0;
    const int n = fft_block(a, blockIdx.x, r0, o0);
    s_blk = make_longlong4(r0, o0, n, 0);

    if (a.bulk) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __syncthreads();
  const int64_t row0 = s_blk.x, out0 = s_blk.y;
  const int nf = (int)s_blk.z;
  if (a.bulk) {   // the tx count may briefly go negative when a copy completes before the expect_tx
    if (tid == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                   "r"((uint32_t)(nf * I * sizeof(float)))
                   : "memory");
    if (tid < nf)
      fft_bulk_copy(Y + tid * Ipad, U + (row0 + (int64_t)tid * a.rs_in_v) * I, (uint32_t)(I * sizeof(float)), bar);
  } else {        // plain loads: one warp per fiber, lanes along the fiber
    for (int f = warp; f < nf; f += TPB / 32) {
      const T* src = U + (row0 + (int64_t)f * a.rs_in_v) * I;
      for (int k = lane; k < I; k += 32) Y[f * Ipad + k] = ld_as_float<T>(src + k);
    }
  }
  for (int e = tid; e < 5 * I; e += TPB) reinterpret_cast<float*>(tw)[e] = a.tab[e];
  for (int e = tid; e < (BJ - nf) * Ipad; e += TPB) Y[nf * Ipad + e] = 0.f;   // fibers past the end of mode v
  // one thread polls the copies' mbarrier (polling by every thread would take issue slots from the
  // other CTAs on the SM); the others wait in the block barrier and then observe the completed phase
  bool ok = true;
  if (a.bulk && tid == 0) {
    ok = false;
    for (uint32_t it = 0; it < kFftWaitLimit && !ok; ++it) ok = fft_mbar_try(bar, 0);
  }
  if (__syncthreads_or(!ok)) {   // the whole CTA leaves together if the wait ran out
    fft_drain(bar, a.err, tid);
    return;
  }
  if (a.bulk && tid != 0) (void)fft_mbar_try(bar, 0);   // completed: returns at once
  __shared__ double s_nrm[TPB / 32];
  if (a.normpart) fft_sumsq_rows<TPB>(Y, nf, I, Ipad, tid, lane, s_nrm);

  // the DFT stages of the S = BJ / 2 complex sequences (the first also reorders the real fibers into
  // interleaved complex values)
  const int nst = a.nst;
  int st = 0;
  fft_stages_of<0, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<1, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<2, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<3, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<4, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<5, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<6, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<7, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<8, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<9, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<10, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<11, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<12, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  fft_stages_of<13, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw, sg);
  if (st != nst && tid == 0) atomicExch(a.err, 1);   // a stage order the host never produces
  if (a.normpart) fft_sumsq_store<TPB>(a, s_nrm, tid);   // after the stages' block barriers

  // separate the two real fibers of each sequence and apply c_k exp(-i pi k / (2I)); the pair
  // (k, I - k) is read and written by one thread: (y_{2p}[k], y_{2p+1}[k]) replaces Z_p[k]
  {
    const int H2 = I / 2 + 1;
    for (int w = tid; w < S * H2; w += TPB) {
      const int p = fdiv(w, H2, a.mH2), k = w - p * H2;
      float2* z = Z + p * Ipad;
      const int kk = k == 0 ? 0 : I - k;
      const float2 A = z[k], B = z[kk];
      const float2 pk = post[k];
      z[k] = make_float2(pk.x * (A.x + B.x) + pk.y * (A.y - B.y), pk.x * (A.y + B.y) - pk.y * (A.x - B.x));
      if (kk != k) {
        const float2 pq = post[kk];
        z[kk] = make_float2(pq.x * (B.x + A.x) + pq.y * (B.y - A.y), pq.x * (B.y + A.y) - pq.y * (B.x - A.x));
      }
    }
  }
  __syncthreads();

  // stores: the mode-v layout (the CTA's fibers adjacent for each k); lanes = 8 fibers x 4 k (fiber f
  // is component f & 1 of sequence f / 2), so a warp reads 32 distinct banks (Ipad odd multiple of 4)
  // and writes four full 32-byte sectors.  The NW warps split the fiber groups (G8 = min(groups, NW)
  // of them at a time) and the groups of 4 k (NW / G8 warps per fiber group); addresses are stepped
  {
    T* yv = static_cast<T*>(a.yv);
    const int FW = BJ < 8 ? BJ : 8, KW = 32 / FW;
    constexpr int NW = TPB / 32;
    const int ngf = BJ / FW, G8 = ngf < NW ? ngf : NW, wpg = NW / G8;
    const int kstep = wpg * KW;
    for (int gf = warp % G8; gf < ngf; gf += G8) {
      const int f = gf * FW + lane % FW;
      int k = (warp / G8) * KW + lane / FW;
      if (f >= nf) continue;
      T* dst = yv + out0 + f + (int64_t)k * a.out_k;
      const int64_t dstep = (int64_t)kstep * a.out_k;
      const float* src = Y + (f >> 1) * 2 * Ipad + (f & 1) + 2 * k;
      for (; k < I; k += kstep, dst += dstep, src += 2 * kstep) *dst = from_float<T>(*src);
    }
  }
  if (a.ysame) {   // the input's own layout: each fiber a contiguous row
    T* ys = static_cast<T*>(a.ysame);
    for (int f = warp; f < nf; f += TPB / 32) {
      T* dst = ys + (row0 + (int64_t)f * a.rs_in_v) * I;
      const float* z = Y + (f >> 1) * 2 * Ipad + (f & 1);
      for (int k = lane; k < I; k += 32) dst[k] = from_float<T>(z[2 * k]);
    }
  }
}

// ---- the factored DCT-II for lengths I with a prime factor above 7 (Bluestein's chirp-z form) ----
// The pass is the one of k_mix_fft (the same fiber blocks, DCT reorder and signs, separation of the
// two real fibers of a sequence, post-rotation and stores); only the length-I DFT of the S complex
// sequences is computed differently.  With c_n = exp(-i pi n^2 / I), the identity
// n k = (n^2 + k^2 - (k - n)^2) / 2 gives Z_k = c_k sum_n (v_n c_n) conj(c_(k-n)): a linear
// convolution, computed as a cyclic one of length M >= 2 I - 1 by the same Stockham stages
// (FFT_M, times the FFT of the filter, FFT_M of the conjugate, conjugated back).  Tables behind the
// DCT's 5 I floats: c_n (I complex), the length-M twiddles (M complex), FFT_M of the filter divided
// by M (M complex).  Shared memory: the fiber rows (BJ x Ipad floats, the final spectra overwrite
// them), the S length-M sequences (Mpad complex each), the tables, the mbarrier.
template <int RIX, int TPB>
__device__ __forceinline__ void bs_stages_of(float2* W, int M, int Mpad, int S, int nst, const StageTab* stt, int& st,
                                             int tid, const float2* twm) {
  for (; st < nst && stt[st].rix == RIX; ++st)
    fft_stage<kRadR1[RIX], kRadR2[RIX], false, TPB>(W, M, Mpad, S, stt[st], tid, twm, nullptr);
}

template <int TPB>
__device__ __forceinline__ bool bs_transform(float2* W, int M, int Mpad, int S, int nst, const StageTab* stt, int tid,
                                             const float2* twm) {
  int st = 0;
  bs_stages_of<0, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<1, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<2, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<3, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<4, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<5, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<6, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<7, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<8, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<9, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<10, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<11, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<12, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  bs_stages_of<13, TPB>(W, M, Mpad, S, nst, stt, st, tid, twm);
  return st == nst;
}

template <typename T, int TPB>
__global__ void __launch_bounds__(TPB, 512 / TPB) k_mix_fft_bs(const __grid_constant__ FftArgs a) {
  extern __shared__ float4 fft_smem4[];
  const int I = a.I, Ipad = a.Ipad, BJ = a.BJ, S = a.S, M = a.M, Mpad = a.Mpad;
  float* Y = reinterpret_cast<float*>(fft_smem4);
  float2* Z = reinterpret_cast<float2*>(Y);                 // sequence p at Z + p Ipad (rows 2p, 2p + 1)
  float2* W = reinterpret_cast<float2*>(Y + BJ * Ipad);     // sequence p at W + p Mpad
  float2* post = W + S * Mpad;                              // I complex
  float2* chirp = post + I;                                 // I complex
  float2* twm = chirp + I;                                  // M complex
  float2* bf = twm + M;                                     // M complex
  float* sg = reinterpret_cast<float*>(bf + M);             // I floats
  uint64_t* bar = reinterpret_cast<uint64_t*>(fft_smem4) + ((BJ * Ipad + 2 * S * Mpad + 5 * I + 4 * M + 3) / 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const T* U = static_cast<const T*>(a.U);
  __shared__ StageTab s_st[kMaxStages];
  __shared__ longlong4 s_blk;
  if (tid < kMaxStages) s_st[tid] = a.st[tid];
  if (tid == 0) {
    int64_t r0, o0;
    const int n = fft_block(a, blockIdx.x, r0, o0);
    s_blk = make_longlong4(r0, o0, n, 0);
    if (a.bulk) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __syncthreads();
  const int64_t row0 = s_blk.x, out0 = s_blk.y;
  const int nf = (int)s_blk.z;
  if (a.bulk) {
    if (tid == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                   "r"((uint32_t)(nf * I * sizeof(float)))
                   : "memory");
    if (tid < nf)
      fft_bulk_copy(Y + tid * Ipad, U + (row0 + (int64_t)tid * a.rs_in_v) * I, (uint32_t)(I * sizeof(float)), bar);
  } else {
    for (int f = warp; f < nf; f += TPB / 32) {
      const T* src = U + (row0 + (int64_t)f * a.rs_in_v) * I;
      for (int k = lane; k < I; k += 32) Y[f * Ipad + k] = ld_as_float<T>(src + k);
    }
  }
  // the tables: post-scales and signs of the DCT, then the chirp, the length-M twiddles and the filter
  const float* tab = a.tab;
  for (int e = tid; e < 2 * I; e += TPB) reinterpret_cast<float*>(post)[e] = tab[2 * I + e];
  for (int e = tid; e < I; e += TPB) sg[e] = tab[4 * I + e];
  for (int e = tid; e < 2 * I + 4 * M; e += TPB) reinterpret_cast<float*>(chirp)[e] = tab[5 * I + e];
  for (int e = tid; e < (BJ - nf) * Ipad; e += TPB) Y[nf * Ipad + e] = 0.f;
  bool ok = true;
  if (a.bulk && tid == 0) {
    ok = false;
    for (uint32_t it = 0; it < kFftWaitLimit && !ok; ++it) ok = fft_mbar_try(bar, 0);
  }
  if (__syncthreads_or(!ok)) {
    fft_drain(bar, a.err, tid);
    return;
  }
  if (a.bulk && tid != 0) (void)fft_mbar_try(bar, 0);
  __shared__ double s_nrm[TPB / 32];
  if (a.normpart) fft_sumsq_rows<TPB>(Y, nf, I, Ipad, tid, lane, s_nrm);
  // a_p[m] = v_p[m] c_m (m < I), 0 past I: v_p[m] = d[s] (x_2p[s], x_2p+1[s]), s the DCT reorder of m
  for (int e = tid; e < S * M; e += TPB) {
    const int p = fdiv(e, M, a.mM), m = e - p * M;
    float2 x = make_float2(0.f, 0.f);
    if (m < I) {
      const int src = 2 * m < I ? 2 * m : 2 * (I - 1 - m) + 1;
      const float d = sg[src];
      const float* row = Y + 2 * p * Ipad;
      x = cmul(make_float2(row[src] * d, row[Ipad + src] * d), chirp[m]);
    }
    W[p * Mpad + m] = x;
  }
  __syncthreads();
  if (a.normpart) fft_sumsq_store<TPB>(a, s_nrm, tid);
  bool good = bs_transform<TPB>(W, M, Mpad, S, a.nst, s_st, tid, twm);
  for (int e = tid; e < S * M; e += TPB) {   // times FFT_M(filter) / M, conjugated
    const int p = fdiv(e, M, a.mM), m = e - p * M;
    const float2 y = cmul(W[p * Mpad + m], bf[m]);
    W[p * Mpad + m] = make_float2(y.x, -y.y);
  }
  __syncthreads();
  good = bs_transform<TPB>(W, M, Mpad, S, a.nst, s_st, tid, twm) && good;
  if (!good && tid == 0) atomicExch(a.err, 1);   // a stage order the host never produces
  // Z_p[k] = c_k conj(W_p[k]), k < I: the DFT of v_p, over the fiber rows (read in full above)
  for (int e = tid; e < S * I; e += TPB) {
    const int p = fdiv(e, I, a.mI), k = e - p * I;
    const float2 w = W[p * Mpad + k];
    Z[p * Ipad + k] = cmul(make_float2(w.x, -w.y), chirp[k]);
  }
  __syncthreads();
  // separation, post-rotation and stores: as in k_mix_fft
  {
    const int H2 = I / 2 + 1;
    for (int w = tid; w < S * H2; w += TPB) {
      const int p = fdiv(w, H2, a.mH2), k = w - p * H2;
      float2* z = Z + p * Ipad;
      const int kk = k == 0 ? 0 : I - k;
      const float2 A = z[k], B = z[kk];
      const float2 pk = post[k];
      z[k] = make_float2(pk.x * (A.x + B.x) + pk.y * (A.y - B.y), pk.x * (A.y + B.y) - pk.y * (A.x - B.x));
      if (kk != k) {
        const float2 pq = post[kk];
        z[kk] = make_float2(pq.x * (B.x + A.x) + pq.y * (B.y - A.y), pq.x * (B.y + A.y) - pq.y * (B.x - A.x));
      }
    }
  }
  __syncthreads();
  {
    T* yv = static_cast<T*>(a.yv);
    const int FW = BJ < 8 ? BJ : 8, KW = 32 / FW;
    constexpr int NW = TPB / 32;
    const int ngf = BJ / FW, G8 = ngf < NW ? ngf : NW, wpg = NW / G8;
    const int kstep = wpg * KW;
    for (int gf = warp % G8; gf < ngf; gf += G8) {
      const int f = gf * FW + lane % FW;
      int k = (warp / G8) * KW + lane / FW;
      if (f >= nf) continue;
      T* dst = yv + out0 + f + (int64_t)k * a.out_k;
      const int64_t dstep = (int64_t)kstep * a.out_k;
      const float* src = Y + (f >> 1) * 2 * Ipad + (f & 1) + 2 * k;
      for (; k < I; k += kstep, dst += dstep, src += 2 * kstep) *dst = from_float<T>(*src);
    }
  }
  if (a.ysame) {
    T* ys = static_cast<T*>(a.ysame);
    for (int f = warp; f < nf; f += TPB / 32) {
      T* dst = ys + (row0 + (int64_t)f * a.rs_in_v) * I;
      const float* z = Y + (f >> 1) * 2 * Ipad + (f & 1);
      for (int k = lane; k < I; k += 32) dst[k] = from_float<T>(z[2 * k]);
    }
  }
}

// The Bluestein tables of one length I behind its 5 I DCT floats (FP64, each rounded once to FP32):
// c_n = exp(-i pi n^2 / I) for n < I (the angle reduced exactly: n^2 mod 2 I), the length-M twiddles
// exp(-2 pi i m / M), and B_k / M with B = FFT_M(b), b_m = conj(c_m) for m < I, conj(c_(M-m)) for
// M - I < m < M, zero between.  First kernel: the FP64 roots exp(-2 pi i j / M) and conj(c_m) into
// scratch behind the FP32 tables, and the FP32 c_n and twiddles.  Second kernel: one warp per B_k,
// the lanes splitting the direct sum over the 2 I - 1 nonzero b_m (root indices stepped, no
// divisions), a fixed-order warp reduction.
__global__ void __launch_bounds__(256) k_build_bs_roots(int I, int M, float* out, double2* wm, double2* dm) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  float* chirp = out + 5 * I;
  float* twm = chirp + 2 * I;
  if (e < M) {
    double sn, cs;
    sincospi(2.0 * (double)e / (double)M, &sn, &cs);
    wm[e] = make_double2(cs, -sn);
    twm[2 * e] = (float)cs;
    twm[2 * e + 1] = (float)(-sn);
  } else if (e < M + I) {
    const int m = e - M;
    const int64_t q = ((int64_t)m * m) % (2 * (int64_t)I);
    double sn, cs;
    sincospi((double)q / (double)I, &sn, &cs);
    dm[m] = make_double2(cs, sn);
    chirp[2 * m] = (float)cs;
    chirp[2 * m + 1] = (float)(-sn);
  }
}

__global__ void __launch_bounds__(256) k_build_bs_tabs(int I, int M, float* out, const double2* __restrict__ wm,
                                                       const double2* __restrict__ dm) {
  const int k = blockIdx.x * 8 + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (k >= M) return;
  float* bf = out + 5 * I + 2 * I + 2 * M;
  double re = 0.0, im = 0.0;
  int j0 = (int)(((int64_t)lane * k) % M);   // (m k) mod M for m = lane, lane + 32, ...
  const int step = (int)(((int64_t)32 * k) % M);
  for (int m = lane; m < I; m += 32) {   // b_m = dm[m] at m and at M - m (m >= 1)
    const double2 b = dm[m];
    const double2 w0 = wm[j0];
    re += b.x * w0.x - b.y * w0.y;
    im += b.x * w0.y + b.y * w0.x;
    if (m > 0) {
      const double2 w1 = wm[j0 == 0 ? 0 : M - j0];
      re += b.x * w1.x - b.y * w1.y;
      im += b.x * w1.y + b.y * w1.x;
    }
    j0 += step;
    if (j0 >= M) j0 -= M;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    re += __shfl_xor_sync(0xffffffffu, re, o);
    im += __shfl_xor_sync(0xffffffffu, im, o);
  }
  if (lane == 0) {
    bf[2 * k] = (float)(re / M);
    bf[2 * k + 1] = (float)(im / M);
  }
}

// ---- the unitary DFT of the complex form of CPRAND-MIX (Alg. 4) ----
// A CTA owns BJ fibers, each its own complex sequence (fiber f at Z + f Ipad, interleaved): the
// fibers are loaded times the signs of the mode (real fibers get a zero imaginary part), transformed
// by the same Stockham stages (the first has no twiddles) and scaled by 1 / sqrt(I) on the way out to
// the mode-v unfolding layout (and, when asked, the input's own layout).
template <int RIX, int TPB>
__device__ __forceinline__ void cfft_stages_of(float2* Z, int I, int Ipad, int S, int nst, const StageTab* stt,
                                               int& st, int tid, const float2* tw) {
  for (; st < nst && stt[st].rix == RIX; ++st)
    fft_stage<kRadR1[RIX], kRadR2[RIX], false, TPB>(Z, I, Ipad, S, stt[st], tid, tw, nullptr);
}

template <typename TIN, int TPB>
__global__ void __launch_bounds__(TPB, 512 / TPB) k_mix_cfft(const __grid_constant__ FftArgs a) {
  extern __shared__ float4 fft_smem4[];
  const int I = a.I, Ipad = a.Ipad, BJ = a.BJ, S = a.S;
  float2* Z = reinterpret_cast<float2*>(fft_smem4);
  float2* tw = Z + BJ * Ipad;
  const float* sg = reinterpret_cast<const float*>(tw + 2 * I);   // after the (unused) post-scales
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  __shared__ StageTab s_st[kMaxStages];
  __shared__ longlong4 s_blk;
  if (tid < kMaxStages) s_st[tid] = a.st[tid];
  if (tid == 0) {
    int64_t r0, o0;
    const int n = fft_block(a, blockIdx.x, r0, o0);
    s_blk = make_longlong4(r0, o0, n, 0);
  }
  for (int e = tid; e < 5 * I; e += TPB) reinterpret_cast<float*>(tw)[e] = a.tab[e];
  __syncthreads();
  const int64_t row0 = s_blk.x, out0 = s_blk.y;
  const int nf = (int)s_blk.z;
  const TIN* U = static_cast<const TIN*>(a.U);
  for (int f = warp; f < BJ; f += TPB / 32) {   // one warp per fiber; fibers past the end: zero
    const TIN* src = U + (row0 + (int64_t)f * a.rs_in_v) * I;
    for (int k = lane; k < I; k += 32) {
      float2 x = make_float2(0.f, 0.f);
      if (f < nf) {
        const float d = sg[k];
        if constexpr (sizeof(TIN) == 8) {
          const float2 u = src[k];
          x = make_float2(u.x * d, u.y * d);
        } else {
          x = make_float2(src[k] * d, 0.f);
        }
      }
      Z[f * Ipad + k] = x;
    }
  }
  __syncthreads();
  const int nst = a.nst;
  int st = 0;
  cfft_stages_of<0, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<1, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<2, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<3, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<4, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<5, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<6, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<7, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<8, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<9, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<10, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<11, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<12, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  cfft_stages_of<13, TPB>(Z, I, Ipad, S, nst, s_st, st, tid, tw);
  if (st != nst && tid == 0) atomicExch(a.err, 1);   // a stage order the host never produces
  const float c = a.cscale;
  {
    float2* yv = static_cast<float2*>(a.yv);
    const int FW = BJ < 8 ? BJ : 8, KW = 32 / FW;
    constexpr int NW = TPB / 32;
    const int ngf = BJ / FW, G8 = ngf < NW ? ngf : NW, wpg = NW / G8;
    const int kstep = wpg * KW;
    for (int gf = warp % G8; gf < ngf; gf += G8) {
      const int f = gf * FW + lane % FW;
      int k = (warp / G8) * KW + lane / FW;
      if (f >= nf) continue;
      float2* dst = yv + out0 + f + (int64_t)k * a.out_k;
      const int64_t dstep = (int64_t)kstep * a.out_k;
      for (; k < I; k += kstep, dst += dstep) {
        const float2 z = Z[f * Ipad + k];
        *dst = make_float2(z.x * c, z.y * c);
      }
    }
  }
  if (a.ysame) {
    float2* ys = static_cast<float2*>(a.ysame);
    for (int f = warp; f < nf; f += TPB / 32) {
      float2* dst = ys + (row0 + (int64_t)f * a.rs_in_v) * I;
      for (int k = lane; k < I; k += 32) {
        const float2 z = Z[f * Ipad + k];
        dst[k] = make_float2(z.x * c, z.y * c);
      }
    }
  }
}


// ---- the same pass with the transform length and its plan fixed at compile time ----
// For a length with a compiled plan every stage constant (L, Ns, the twiddle steps) is known to the
// compiler, so shared-memory addresses take immediate offsets and the butterflies' roots of unity
// are FMA immediates.  Each later stage reads its twiddles from its own small table (rows indexed by
// k, so that the lanes of a warp read consecutive entries), whose row products give the stage's
// R - 1 twiddles.  The separation of the two real fibers of a sequence and the post-rotation are
// done by the stores: a lane reads the entries k and I - k once and writes the results at both (no
// extra pass over shared memory), 16 bytes per store.

// (cos, sin)(2 pi a / b) in double, evaluated by the compiler: the angle is split, in integers, into
// a multiple of pi / 4 and a rest in [0, pi / 4) whose sine and cosine are Taylor sums
struct CxPair {
  double c, s;
};
constexpr double cx_sin_series(double x) {
  double t = x, sum = x;
  for (int n = 1; n < 14; ++n) {
    t *= -x * x / ((2.0 * n) * (2.0 * n + 1.0));
    sum += t;
  }
  return sum;
}
constexpr double cx_cos_series(double x) {
  double t = 1.0, sum = 1.0;
  for (int n = 1; n < 14; ++n) {
    t *= -x * x / ((2.0 * n - 1.0) * (2.0 * n));
    sum += t;
  }
  return sum;
}
constexpr CxPair cx_quarter_turns(double c, double s, int q) {   // (c, s) rotated by q quarter turns
  return (q & 3) == 0 ? CxPair{c, s} : (q & 3) == 1 ? CxPair{-s, c} : (q & 3) == 2 ? CxPair{-c, -s} : CxPair{s, -c};
}
constexpr CxPair cx_cis_2pi(long a, long b) {
  constexpr double kQuarterPi = 0.78539816339744830961566084581988;
  const long t = 8 * (a % b);   // angle = (t / b) pi / 4
  const int o = (int)(t / b);
  const long rem = t - o * b;
  if (o % 2 == 0) {   // o pi / 4 + phi, phi = (pi / 4) rem / b
    const double phi = kQuarterPi * (double)rem / (double)b;
    return cx_quarter_turns(cx_cos_series(phi), cx_sin_series(phi), o / 2);
  }
  const double psi = kQuarterPi * (double)(b - rem) / (double)b;   // (o + 1) pi / 4 - psi
  return cx_quarter_turns(cx_cos_series(psi), -cx_sin_series(psi), (o + 1) / 2);
}
template <int R, int M>
struct CxRoot {   // exp(-2 pi i M / R) rounded to FP32
  static constexpr float re = (float)cx_cis_2pi(M, R).c;
  static constexpr float im = (float)-cx_cis_2pi(M, R).s;
};
template <int R, int... M>
__device__ __forceinline__ void ct_roots(float2 (&w)[R], std::integer_sequence<int, M...>) {
  ((w[M] = make_float2(CxRoot<R, M>::re, CxRoot<R, M>::im)), ...);
}

// dft_comp with the roots as constants: w[m] = exp(-2 pi i m / R)
template <int R1, int R2>
__device__ __forceinline__ void ct_dft_comp(float2 (&v)[R1 * R2]) {
  constexpr int R = R1 * R2;
  float2 w[R];
  ct_roots<R>(w, std::make_integer_sequence<int, R>{});
  float2 rc1[R1 / 2 + 1], rc2[R2 / 2 + 1];   // (cos, sin)(2 pi m / R1), (cos, sin)(2 pi m / R2)
#pragma unroll
  for (int m = 0; m <= R1 / 2; ++m) rc1[m] = make_float2(w[m * R2].x, -w[m * R2].y);
#pragma unroll
  for (int m = 0; m <= R2 / 2; ++m) rc2[m] = make_float2(w[m * R1].x, -w[m * R1].y);
  if constexpr (R2 == 1) {
    dft<R1>(v, rc1);
  } else {
#pragma unroll
    for (int r2 = 0; r2 < R2; ++r2) {
      float2 t[R1];
#pragma unroll
      for (int r1 = 0; r1 < R1; ++r1) t[r1] = v[R2 * r1 + r2];
      dft<R1>(t, rc1);
#pragma unroll
      for (int q1 = 0; q1 < R1; ++q1) v[R2 * q1 + r2] = (r2 && q1) ? cmul(t[q1], w[r2 * q1]) : t[q1];
    }
    float2 o[R];
#pragma unroll
    for (int q1 = 0; q1 < R1; ++q1) {
      float2 t[R2];
#pragma unroll
      for (int r2 = 0; r2 < R2; ++r2) t[r2] = v[R2 * q1 + r2];
      dft<R2>(t, rc2);
#pragma unroll
      for (int q2 = 0; q2 < R2; ++q2) o[q1 + R1 * q2] = t[q2];
    }
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = o[r];
  }
}

// table rows of a later stage of radix R1 R2: the twiddle of entry r = R2 r1 + r2 is the product
// of the rows w^(r2 k t) (r2 = 1 .. R2 - 1) and w^(R2 r1 k t) (r1 = 1 .. R1 - 1), rounded twice at most
constexpr int ct_twiddle_rows(int R1, int R2) { return R2 > 1 ? (R1 - 1) + (R2 - 1) : R1 - 1; }

template <int R1_, int R2_>
struct CtRadix {
  static constexpr int R1 = R1_, R2 = R2_, R = R1_ * R2_;
};

// a compiled plan: length, CTA width, fibers per CTA, the stages in order
template <int I_, int TPB_, int BJ_, int MINB_, class... Rs>
struct CtPlan {
  static constexpr int I = I_, TPB = TPB_, BJ = BJ_, S = BJ_ / 2, MINB = MINB_;
  static constexpr int NST = sizeof...(Rs);
  static constexpr int radix(int s) {
    const int rs[] = {Rs::R...};
    return rs[s];
  }
  // the first stage writes butterfly j's R0 outputs at j (R0 + 1) + r (stride R0 + 1, odd, instead
  // of the even R0: no bank conflicts); the second stage's reads follow (they stay immediate offsets
  // when R0 divides its L)
  static constexpr bool SKEW = NST >= 2 && radix(0) % 2 == 0 && (I_ / radix(1)) % radix(0) == 0;
  static constexpr int LEN = I_ + (SKEW ? I_ / radix(0) : 0);   // complex entries of a sequence
  // a sequence spans two fiber rows of IPAD floats: IPAD >= LEN, a multiple of 4 (16-byte rows for the
  // bulk copies) with IPAD / 4 odd (conflict-free column reads by the stores)
  static constexpr int IPAD = ((LEN + 3) / 4 * 4) % 8 == 0 ? (LEN + 3) / 4 * 4 + 4 : (LEN + 3) / 4 * 4;
  static constexpr int twiddles() {   // entries of the later stages' tables
    int ns = 1, n = 0;
    const int rs[] = {Rs::R...}, r1s[] = {Rs::R1...}, r2s[] = {Rs::R2...};
    for (int s = 0; s < NST; ++s) {
      if (s > 0) n += ct_twiddle_rows(r1s[s], r2s[s]) * ns;
      ns *= rs[s];
    }
    return n;
  }
  static constexpr int product() {
    int p = 1;
    const int rs[] = {Rs::R...};
    for (int s = 0; s < NST; ++s) p *= rs[s];
    return p;
  }
  // shared memory, in floats: the fiber rows, post-scales of k <= I/2 (those of I - k are the same
  // with swapped components), the first stage's sign masks (one word
  // per butterfly of a sequence, rounded up to even), the stage tables, then the mbarrier
  static constexpr int L0 = I_ / radix(0);
  static constexpr int OFF_POST = BJ_ * IPAD, OFF_SG = OFF_POST + 2 * (I_ / 2 + 1), OFF_T = OFF_SG + (L0 + 1) / 2 * 2,
                       OFF_BAR = OFF_T + 2 * twiddles();
  static constexpr size_t SMEM = (size_t)OFF_BAR * sizeof(float) + 16;
};

// one stage of the compiled plan (the Stockham stage of fft_stage with constant parameters).  smask:
// for butterfly j of the first stage, bit r set when the sign of its entry r (reorder order) is -1
// nrm (first stage only, when given): the warp's sum of squares of the entries it read, into
// nrm[warp] before the stage's block barrier
template <class PL, int R1, int R2, int NS, bool FIRST>
__device__ __forceinline__ void ct_stage(float2* Z, const float2* T, const uint32_t* smask, int tid, double* nrm) {
  constexpr int I = PL::I, IPAD = PL::IPAD, TPB = PL::TPB, R = R1 * R2, L = I / R, NB = PL::S * L;
  constexpr int NQ = (NB + TPB - 1) / TPB;
  constexpr bool SKW = FIRST && PL::SKEW, SKR = !FIRST && NS == PL::radix(0) && PL::SKEW;
  constexpr int R0 = PL::radix(0);
  float2 v[NQ][R];
  int dst[NQ];
  float sqx = 0.f, sqy = 0.f;
#pragma unroll
  for (int q = 0; q < NQ; ++q) {
    const int b = tid + q * TPB;
    dst[q] = -1;
    if (NB % TPB == 0 || b < NB) {
      const int p = b / L, j = b - p * L;
      if constexpr (FIRST) {   // v_p[m] = d[s] (x_{2p}[s], x_{2p+1}[s]), s = 2m or 2(I - 1 - m) + 1
        static_assert(R <= 32, "one sign mask word per butterfly");
        const float* row = reinterpret_cast<const float*>(Z + p * IPAD);
        const uint32_t msk = smask[j];
#pragma unroll
        for (int r = 0; r < R; ++r) {
          int src;
          if (2 * (r + 1) * L <= I) src = 2 * j + 2 * r * L;                 // every m of this r even-placed
          else if (2 * r * L >= I) src = (2 * I - 1 - 2 * r * L) - 2 * j;   // every m odd-placed
          else {
            const int m = j + r * L;
            src = 2 * m < I ? 2 * m : 2 * I - 1 - 2 * m;
          }
          const uint32_t flip = (msk << (31 - r)) & 0x80000000u;   // the sign bit of d
          v[q][r] = make_float2(__uint_as_float(__float_as_uint(row[src]) ^ flip),
                                __uint_as_float(__float_as_uint(row[IPAD + src]) ^ flip));
        }
        if (nrm) {
#pragma unroll
          for (int r = 0; r < R; ++r) {
            sqx = fmaf(v[q][r].x, v[q][r].x, sqx);
            sqy = fmaf(v[q][r].y, v[q][r].y, sqy);
          }
        }
      } else {
        const int k = j % NS;
        // entry m of the first stage's output sits at m + m / R0 when skewed (R0 divides L)
        const float2* z = Z + p * IPAD + j + (SKR ? j / R0 : 0);
        constexpr int LS = SKR ? L + L / R0 : L;
        const float2* t = T + k;
        v[q][0] = z[0];
        if constexpr (R2 > 1) {   // twiddle of r = R2 r1 + r2: the table rows' product
          float2 wa[R2], wb[R1];
#pragma unroll
          for (int r2 = 1; r2 < R2; ++r2) wa[r2] = t[(r2 - 1) * NS];
#pragma unroll
          for (int r1 = 1; r1 < R1; ++r1) wb[r1] = t[(R2 - 1 + r1 - 1) * NS];
#pragma unroll
          for (int r = 1; r < R; ++r) {
            const int r1 = r / R2, r2 = r % R2;
            const float2 w = r1 == 0 ? wa[r2] : (r2 == 0 ? wb[r1] : cmul(wb[r1], wa[r2]));
            v[q][r] = cmul(z[r * LS], w);
          }
        } else {
#pragma unroll
          for (int r = 1; r < R; ++r) v[q][r] = cmul(z[r * LS], t[(r - 1) * NS]);
        }
      }
      ct_dft_comp<R1, R2>(v[q]);
      dst[q] = p * IPAD + (SKW ? j * (R + 1) : (j / NS) * NS * R + j % NS);
    }
    asm volatile("" ::: "memory");
  }
  if (FIRST && nrm) fft_sumsq_warp(sqx + sqy, tid & 31, nrm + (tid >> 5));
  __syncthreads();
#pragma unroll
  for (int q = 0; q < NQ; ++q)
    if (NB % TPB == 0 || dst[q] >= 0) {
#pragma unroll
      for (int r = 0; r < R; ++r) Z[dst[q] + r * NS] = v[q][r];
    }
  __syncthreads();
}

template <class PL, int NS, bool FIRST, class R0, class... Rest>
__device__ __forceinline__ void ct_stages(float2* Z, const float2* T, const uint32_t* smask, int tid, double* nrm) {
  ct_stage<PL, R0::R1, R0::R2, NS, FIRST>(Z, T, smask, tid, nrm);
  if constexpr (sizeof...(Rest) > 0)
    ct_stages<PL, NS * R0::R, false, Rest...>(Z, FIRST ? T : T + ct_twiddle_rows(R0::R1, R0::R2) * NS, smask, tid,
                                              nullptr);
}

// the stage tables from the length-I twiddles in global memory (L2-resident): row e of a stage of
// radix R1 R2 (R2 > 1) holds w^(r2 k t) for e = r2 - 1 < R2 - 1, else w^(R2 r1 k t) for e = R2 - 2 + r1;
// a plain radix R1 holds w^(r k t) in row r - 1 (t = I / (NS R), k < NS)
template <class PL, int NS, bool FIRST, class R0, class... Rest>
__device__ __forceinline__ void ct_tables(float2* T, const float2* twg, int tid) {
  constexpr int ROWS = ct_twiddle_rows(R0::R1, R0::R2);
  if constexpr (!FIRST) {
    constexpr int CNT = ROWS * NS, TSTEP = PL::I / (NS * R0::R);
    for (int e = tid; e < CNT; e += PL::TPB) {
      const int row = e / NS, k = e - row * NS;
      const int mult = R0::R2 > 1 ? (row < R0::R2 - 1 ? row + 1 : R0::R2 * (row - (R0::R2 - 1) + 1)) : row + 1;
      T[e] = twg[mult * k * TSTEP];
    }
  }
  if constexpr (sizeof...(Rest) > 0)
    ct_tables<PL, NS * R0::R, false, Rest...>(FIRST ? T : T + ROWS * NS, twg, tid);
}

// y_{2p}[k], y_{2p+1}[k] from the transformed sequence p: A = Z_p[k], B = Z_p[(I - k) mod I]
__device__ __forceinline__ float2 ct_separate(float2 A, float2 B, float2 pk) {
  return make_float2(pk.x * (A.x + B.x) + pk.y * (A.y - B.y), pk.x * (A.y + B.y) - pk.y * (A.x - B.x));
}

template <typename T> __device__ __forceinline__ void st4(T* dst, float a, float b, float c, float d);
template <> __device__ __forceinline__ void st4<float>(float* dst, float a, float b, float c, float d) {
  *reinterpret_cast<float4*>(dst) = make_float4(a, b, c, d);
}
template <> __device__ __forceinline__ void st4<__nv_bfloat16>(__nv_bfloat16* dst, float a, float b, float c, float d) {
  const __nv_bfloat162 lo = __floats2bfloat162_rn(a, b), hi = __floats2bfloat162_rn(c, d);
  uint2 u;
  u.x = *reinterpret_cast<const uint32_t*>(&lo);
  u.y = *reinterpret_cast<const uint32_t*>(&hi);
  *reinterpret_cast<uint2*>(dst) = u;
}

template <class PL> struct CtStages;
template <int I_, int TPB_, int BJ_, int MINB_, class... Rs>
struct CtStages<CtPlan<I_, TPB_, BJ_, MINB_, Rs...>> {
  using P = CtPlan<I_, TPB_, BJ_, MINB_, Rs...>;
  static __device__ __forceinline__ void run(float2* Z, const float2* T, const uint32_t* smask, int tid, double* nrm) {
    ct_stages<P, 1, true, Rs...>(Z, T, smask, tid, nrm);
  }
  static __device__ __forceinline__ void tables(float2* T, const float2* twg, int tid) {
    ct_tables<P, 1, true, Rs...>(T, twg, tid);
  }
};

template <typename T, class PL>
__global__ void __launch_bounds__(PL::TPB, PL::MINB) k_mix_fft_ct(const __grid_constant__ FftArgs a) {
  constexpr int I = PL::I, IPAD = PL::IPAD, BJ = PL::BJ, S = PL::S, TPB = PL::TPB, NW = TPB / 32;
  static_assert(PL::product() == PL::I, "the plan's radices multiply to the length");
  // 4-fiber groups; a warp's lanes cover GW of them (GW <= 4 keeps the column reads conflict-free)
  constexpr int G4 = BJ / 4, GW = G4 < 4 ? G4 : 4, KPW = 32 / GW;
  static_assert(BJ % 4 == 0 && G4 % GW == 0 && TPB % 32 == 0, "4-fiber groups, whole warps");
  extern __shared__ float4 fft_smem4[];
  float* Y = reinterpret_cast<float*>(fft_smem4);
  float2* Z = reinterpret_cast<float2*>(Y);
  float2* post = reinterpret_cast<float2*>(Y + PL::OFF_POST);
  uint32_t* smask = reinterpret_cast<uint32_t*>(Y + PL::OFF_SG);
  float2* Tt = reinterpret_cast<float2*>(Y + PL::OFF_T);
  uint64_t* bar = reinterpret_cast<uint64_t*>(Y + PL::OFF_BAR);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const T* U = static_cast<const T*>(a.U);
  if (a.I != I) {   // the host launches a compiled plan for its own length only
    if (tid == 0) atomicExch(a.err, 1);
    return;
  }
  __shared__ longlong4 s_blk;
  if (tid == 0) {
    int64_t r0, o0;
    const int n = fft_block(a, blockIdx.x, r0, o0);
    s_blk = make_longlong4(r0, o0, n, 0);
    if (a.bulk) {
      asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(1) : "memory");
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
  }
  __syncthreads();
  const int64_t row0 = s_blk.x, out0 = s_blk.y;
  const int nf = (int)s_blk.z;
  if (a.bulk) {
    if (tid == 0)
      asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)),
                   "r"((uint32_t)(nf * I * sizeof(float)))
                   : "memory");
    if (tid < nf)
      fft_bulk_copy(Y + tid * IPAD, U + (row0 + (int64_t)tid * a.rs_in_v) * I, (uint32_t)(I * sizeof(float)), bar);
  } else if (sizeof(T) == 2 && I % 4 == 0 && a.vec_in) {
    // BF16 rows: 8-byte loads of 4 entries (widened exactly to FP32), four in flight per lane, 16-byte
    // shared stores
    constexpr int C4 = I / 4;
    for (int f = warp; f < nf; f += NW) {
      const uint2* src = reinterpret_cast<const uint2*>(U + (row0 + (int64_t)f * a.rs_in_v) * I);
      float4* dst = reinterpret_cast<float4*>(Y + f * IPAD);
      for (int c0 = 0; c0 < C4; c0 += 128) {
        uint2 u[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = c0 + 32 * i + lane;
          if (c < C4) u[i] = __ldg(src + c);
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int c = c0 + 32 * i + lane;
          if (c < C4)
            dst[c] = make_float4(__uint_as_float(u[i].x << 16), __uint_as_float(u[i].x & 0xffff0000u),
                                 __uint_as_float(u[i].y << 16), __uint_as_float(u[i].y & 0xffff0000u));
        }
      }
    }
  } else {
    for (int f = warp; f < nf; f += NW) {
      const T* src = U + (row0 + (int64_t)f * a.rs_in_v) * I;
      for (int k = lane; k < I; k += 32) Y[f * IPAD + k] = ld_as_float<T>(src + k);
    }
  }
  for (int e = tid; e < 2 * (I / 2 + 1); e += TPB) Y[PL::OFF_POST + e] = a.tab[2 * I + e];   // post-scales, k <= I/2
  for (int j = tid; j < PL::L0; j += TPB) {   // the signs of butterfly j's entries m = j + r L0
    uint32_t msk = 0;
    for (int r = 0; r < PL::radix(0); ++r) {
      const int m = j + r * PL::L0;
      msk |= (a.tab[4 * I + (2 * m < I ? 2 * m : 2 * I - 1 - 2 * m)] < 0.f ? 1u : 0u) << r;
    }
    smask[j] = msk;
  }
  CtStages<PL>::tables(Tt, reinterpret_cast<const float2*>(a.tab), tid);
  for (int e = tid; e < (BJ - nf) * IPAD; e += TPB) Y[nf * IPAD + e] = 0.f;
  bool ok = true;
  if (a.bulk && tid == 0) {
    ok = false;
    for (uint32_t it = 0; it < kFftWaitLimit && !ok; ++it) ok = fft_mbar_try(bar, 0);
  }
  if (__syncthreads_or(!ok)) {
    fft_drain(bar, a.err, tid);
    return;
  }
  if (a.bulk && tid != 0) (void)fft_mbar_try(bar, 0);
  __shared__ double s_nrm[TPB / 32];

  CtStages<PL>::run(Z, Tt, smask, tid, a.normpart ? s_nrm : nullptr);   // the first stage sums the squares
  if (a.normpart) fft_sumsq_store<TPB>(a, s_nrm, tid);   // after the stages' block barriers

  T* yv = static_cast<T*>(a.yv);
  constexpr int KH = I / 2;   // entries k <= KH and their partners I - k cover 0 .. I - 1
  if (a.vec_v && nf == BJ) {
    // lane (k = k0 + lane % KPW <= KH, 4-fiber group g = GW gq + lane / KPW): y_{4g .. 4g+3} at k and
    // at I - k from sequences 2g and 2g + 1 (each value read once), two 16-byte stores; a half warp
    // reads 32 distinct banks (IPAD / 4 odd)
    constexpr int NGQ = G4 / GW, NKO = (KH + 1 + KPW - 1) / KPW;
    for (int w = warp; w < NGQ * NKO; w += NW) {
      const int k = (w / NGQ) * KPW + lane % KPW, g = (w % NGQ) * GW + lane / KPW;
      if (k <= KH) {
        const int kk = k == 0 ? 0 : I - k;
        const float2* z0 = Z + 2 * g * IPAD;
        const float2 A0 = z0[k], B0 = z0[kk], A1 = z0[IPAD + k], B1 = z0[IPAD + kk];
        const float2 pk = post[k];
        const float2 y0 = ct_separate(A0, B0, pk), y1 = ct_separate(A1, B1, pk);
        st4<T>(yv + out0 + 4 * g + (int64_t)k * a.out_k, y0.x, y0.y, y1.x, y1.y);
        if (kk != k) {   // post(I - k) = post(k) with its components swapped (c_k = c_{I-k} for k >= 1)
          const float2 pq = make_float2(pk.y, pk.x);
          const float2 q0 = ct_separate(B0, A0, pq), q1 = ct_separate(B1, A1, pq);
          st4<T>(yv + out0 + 4 * g + (int64_t)kk * a.out_k, q0.x, q0.y, q1.x, q1.y);
        }
      }
    }
  } else {
    for (int e = tid; e < BJ * I; e += TPB) {
      const int f = e % BJ, k = e / BJ;
      if (f < nf) {
        const float2* z = Z + (f >> 1) * IPAD;
        const float2 pk = k <= I / 2 ? post[k] : make_float2(post[I - k].y, post[I - k].x);
        const float2 y = ct_separate(z[k], z[k == 0 ? 0 : I - k], pk);
        yv[out0 + f + (int64_t)k * a.out_k] = from_float<T>((f & 1) ? y.y : y.x);
      }
    }
  }
  if (a.ysame) {   // each fiber a row of the input's layout
    T* ys = static_cast<T*>(a.ysame);
    // a warp: sequence p, 32 consecutive k <= KH and their partners I - k (conflict-free reads of
    // Z_p[k], Z_p[I - k], post[k]); coalesced row segments of fibers 2p and 2p + 1
    constexpr int KC = (KH + 1 + 31) / 32;
    for (int w = warp; w < S * KC; w += NW) {
      const int p = w / KC, k = (w - p * KC) * 32 + lane;
      if (2 * p >= nf || k > KH) continue;
      const int kk = k == 0 ? 0 : I - k;
      const float2* z = Z + p * IPAD;
      const float2 A = z[k], B = z[kk];
      const float2 pk = post[k];
      const float2 y = ct_separate(A, B, pk);
      T* r0p = ys + (row0 + (int64_t)(2 * p) * a.rs_in_v) * I;
      T* r1p = ys + (row0 + (int64_t)(2 * p + 1) * a.rs_in_v) * I;
      const bool two = 2 * p + 1 < nf;
      r0p[k] = from_float<T>(y.x);
      if (two) r1p[k] = from_float<T>(y.y);
      if (kk != k) {
        const float2 q = ct_separate(B, A, make_float2(pk.y, pk.x));
        r0p[kk] = from_float<T>(q.x);
        if (two) r1p[kk] = from_float<T>(q.y);
      }
    }
  }
}

// the compiled plans:
//  * I = 400 = 20 x 20 (radix 20 = 5 x 4), 16 fibers per CTA, one butterfly per thread in both
//    stages, six CTAs per SM (64 registers, 30 KB of shared memory each);
//  * I = 1500 = 25 x 12 x 5, 8 fibers per CTA, 256 threads (240, 500 and 1200 butterflies: one, two
//    and five per thread), three CTAs per SM (65 KB each);
//  * I = 100 = 10 x 10 (radix 10 = 5 x 2), 16 fibers per CTA, 96 threads (80 butterflies a stage).
using CtPlan400 = CtPlan<400, 160, 16, 6, CtRadix<5, 4>, CtRadix<5, 4>>;
using CtPlan1500 = CtPlan<1500, 256, 8, 3, CtRadix<5, 5>, CtRadix<4, 3>, CtRadix<5, 1>>;
using CtPlan100 = CtPlan<100, 96, 16, 12, CtRadix<5, 2>, CtRadix<5, 2>>;

// the stage radices of I (every prime factor 2, 3, 5 or 7), grouped into the radices of kRadR1 x
// kRadR2, listed in radix-index order; among the groupings, the one that admits the widest fiber block
// (then the fewest stages).  CTAs of 128 threads (four per SM) unless that narrows the block below 8
// fibers where 256 threads (two per SM) would not
struct FftPlan {
  int tpb, BJ, Ipad, nst;
  int rix[kMaxStages];
  size_t smem;
};

// the fiber block (complex: two floats per entry), the tables, the mbarrier
size_t fft_smem_bytes(int BJ, int Ipad, int I, bool cplx = false) {
  return (size_t)((cplx ? 2 : 1) * BJ * Ipad + 5 * I + 4) * sizeof(float) + 16;
}

// the widest block (a power of two up to 128 fibers, not wider than mode v needs) whose stages fit
// the threads' register slots, within the shared memory that lets 512 / tpb CTAs share an SM
int fft_block_width(int I, int64_t Iv, int Ipad, const int* rix, int nst, int tpb, bool cplx) {
  int64_t cap = 2;
  while (cap < Iv && cap < 128) cap *= 2;
  const size_t smem_cap = (size_t)kFftMaxSmem / (512 / tpb);
  for (int BJ = 128; BJ >= 2; BJ /= 2) {
    if (BJ > cap) continue;
    const int S = cplx ? BJ : BJ / 2;   // complex: every fiber its own sequence
    bool ok = true;
    for (int s = 0; s < nst && ok; ++s) {
      const int R = kRadR1[rix[s]] * kRadR2[rix[s]];
      ok = ((int64_t)S * (I / R) + tpb - 1) / tpb <= kSlots / R;
    }
    const size_t sm = fft_smem_bytes(BJ, Ipad, I, cplx);
    if (ok && sm <= (size_t)kFftMaxSmem && (BJ <= 8 || sm <= smem_cap)) return BJ;
  }
  return 0;
}

void fft_search(int m, int from, int* cur, int depth, int I, int64_t Iv, int Ipad, int tpb, bool cplx,
                FftPlan* best) {
  if (m == 1) {
    if (depth == 0) return;
    const int BJ = fft_block_width(I, Iv, Ipad, cur, depth, tpb, cplx);
    if (BJ > best->BJ || (BJ == best->BJ && BJ > 0 && depth < best->nst)) {
      best->BJ = BJ;
      best->nst = depth;
      for (int s = 0; s < depth; ++s) best->rix[s] = cur[s];
    }
    return;
  }
  if (depth == kMaxStages) return;
  for (int r = from; r < kNumRadices; ++r) {
    const int R = kRadR1[r] * kRadR2[r];
    if (m % R) continue;
    cur[depth] = r;
    fft_search(m / R, r, cur, depth + 1, I, Iv, Ipad, tpb, cplx, best);
  }
}

bool fft_plan(int I, int64_t Iv, FftPlan* pl, bool cplx = false) {
  if (I < 2 || I > kMaxFftLen) return false;
  int m = I;
  for (int p : {2, 3, 5, 7})
    while (m % p == 0) m /= p;
  if (m != 1) return false;
  int Ipad = (I + 3) / 4 * 4;
  if ((Ipad / 4) % 2 == 0) Ipad += 4;   // Ipad / 4 odd: conflict-free column reads
  FftPlan best[2];
  const int tpbs[2] = {128, 256};
  for (int t = 0; t < 2; ++t) {
    memset(&best[t], 0, sizeof(FftPlan));
    int cur[kMaxStages];
    fft_search(I, 0, cur, 0, I, Iv, Ipad, tpbs[t], cplx, &best[t]);
    best[t].tpb = tpbs[t];
  }
  const int want = (int)std::min<int64_t>(8, Iv);
  const int pick = (best[0].BJ > 0 && (best[0].BJ >= want || best[0].BJ >= best[1].BJ)) ? 0 : 1;
  if (best[pick].BJ == 0) return false;
  *pl = best[pick];
  pl->Ipad = Ipad;
  pl->smem = fft_smem_bytes(pl->BJ, Ipad, I, cplx);
  return true;
}

// Bluestein form: the convolution length (the smallest 7-smooth M >= 2 I - 1, at most 4096), 0 when
// there is none or I is 7-smooth itself (the direct plan applies)
bool smooth7(int m) {
  for (int p : {2, 3, 5, 7})
    while (m % p == 0) m /= p;
  return m == 1;
}
int bs_length(int I) {
  if (I < kBsMinLen || smooth7(I)) return 0;
  for (int M = 2 * I - 1; M <= kBsMaxConv; ++M)
    if (smooth7(M)) return M;
  return 0;
}
// the fiber rows, the length-M sequences, the tables (5 I + 2 I + 4 M floats), the mbarrier
size_t bs_smem_bytes(int BJ, int Ipad, int Mpad, int I, int M) {
  return (size_t)(BJ * Ipad + BJ * Mpad + 7 * I + 4 * M + 4) * sizeof(float) + 16;
}
bool fft_plan_bs(int I, int64_t Iv, FftPlan* pl, int* Mout, int* Mpad_out) {
  const int M = bs_length(I);
  if (M == 0) return false;
  int Ipad = (I + 3) / 4 * 4;
  if ((Ipad / 4) % 2 == 0) Ipad += 4;
  int Mpad = (M + 3) / 4 * 4;
  if ((Mpad / 4) % 2 == 0) Mpad += 4;
  int64_t cap = 2;
  while (cap < Iv && cap < 128) cap *= 2;
  FftPlan best;
  memset(&best, 0, sizeof(best));
  const int tpbs[2] = {128, 256};
  for (int t = 0; t < 2; ++t) {
    const int tpb = tpbs[t];
    const size_t smem_cap = (size_t)kFftMaxSmem / (512 / tpb);
    // the stage plan of length M with the fewest stages, for the widest block that fits
    for (int BJ = 128; BJ >= 2; BJ /= 2) {
      if (BJ > cap) continue;
      const size_t sm = bs_smem_bytes(BJ, Ipad, Mpad, I, M);
      if (sm > (size_t)kFftMaxSmem || (BJ > 8 && sm > smem_cap)) continue;
      FftPlan cand;
      memset(&cand, 0, sizeof(cand));
      int cur[kMaxStages];
      fft_search(M, 0, cur, 0, M, (int64_t)BJ, Mpad, tpb, false, &cand);   // checks S = BJ / 2 sequences
      if (cand.BJ < BJ) continue;
      if (BJ > best.BJ) {
        best = cand;
        best.BJ = BJ;
        best.tpb = tpb;
        best.Ipad = Ipad;
        best.smem = sm;
      }
      break;
    }
  }
  if (best.BJ == 0) return false;
  *pl = best;
  *Mout = M;
  *Mpad_out = Mpad;
  return true;
}

template <typename T, int TPB>
cudaError_t launch_fft_kernel(const FftArgs& a, size_t smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_mix_fft<T, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftMaxSmem + 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (a.nblocks > INT32_MAX) return cudaErrorInvalidValue;
  k_mix_fft<T, TPB><<<(unsigned)a.nblocks, TPB, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, int TPB>
cudaError_t launch_fft_bs_kernel(const FftArgs& a, size_t smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_mix_fft_bs<T, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftMaxSmem + 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (a.nblocks > INT32_MAX) return cudaErrorInvalidValue;
  k_mix_fft_bs<T, TPB><<<(unsigned)a.nblocks, TPB, smem, s>>>(a);
  return cudaGetLastError();
}

template <typename T, class PL>
cudaError_t launch_fft_ct_kernel(const FftArgs& a, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mix_fft_ct<T, PL>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)PL::SMEM);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (a.nblocks > INT32_MAX) return cudaErrorInvalidValue;
  k_mix_fft_ct<T, PL><<<(unsigned)a.nblocks, PL::TPB, PL::SMEM, s>>>(a);
  return cudaGetLastError();
}

// the compiled plan of a pass, when there is one: the length matches and mode v is at least one
// CTA's block of fibers wide
template <class PL>
bool ct_plan_of(FftPlan* pl) {
  memset(pl, 0, sizeof(*pl));
  pl->tpb = PL::TPB;
  pl->BJ = PL::BJ;
  pl->Ipad = PL::IPAD;
  pl->smem = PL::SMEM;
  return true;
}
int ct_plan_id(int I, int64_t Iv) {
  if (I == CtPlan400::I && Iv >= CtPlan400::BJ) return 1;
  if (I == CtPlan1500::I && Iv >= CtPlan1500::BJ) return 2;
  if (I == CtPlan100::I && Iv >= CtPlan100::BJ) return 3;
  return 0;
}

template <typename TIN, int TPB>
cudaError_t launch_cfft_kernel(const FftArgs& a, size_t smem, cudaStream_t s) {
  static bool attr = false;
  if (!attr) {
    cudaError_t e =
        cudaFuncSetAttribute(k_mix_cfft<TIN, TPB>, cudaFuncAttributeMaxDynamicSharedMemorySize, kFftMaxSmem + 1024);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  if (a.nblocks > INT32_MAX) return cudaErrorInvalidValue;
  k_mix_cfft<TIN, TPB><<<(unsigned)a.nblocks, TPB, smem, s>>>(a);
  return cudaGetLastError();
}

uint32_t magic(int d) { return d > 1 ? (uint32_t)((((uint64_t)1 << 32) + d - 1) / d) : 0u; }

}  // namespace

bool mix_fft_supported(int dtype, int N, const int64_t* dims) {
  if (dtype != CPR_F32 && dtype != CPR_BF16) return false;
  if (N < 2) return false;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 5) return false;   // the tables live in the I x I operator buffer (5 I floats)
    FftPlan pl;
    int M, Mpad;
    if (!fft_plan((int)dims[n], dims[(n + 1) % N], &pl) &&
        !fft_plan_bs((int)dims[n], dims[(n + 1) % N], &pl, &M, &Mpad))
      return false;
  }
  return true;
}

cudaError_t launch_build_bs_tables(int I, float* fft_tab, cudaStream_t s) {
  const int M = bs_length(I);
  if (M == 0) return cudaSuccess;   // a 7-smooth length (or none): nothing to add
  // FP64 scratch behind the FP32 tables (7 I + 4 M floats), inside the I x I table buffer
  const int off = (7 * I + 4 * M + 3) / 4 * 4;
  double2* wm = reinterpret_cast<double2*>(fft_tab + off);
  double2* dm = wm + M;
  k_build_bs_roots<<<(M + I + 255) / 256, 256, 0, s>>>(I, M, fft_tab, wm, dm);
  k_build_bs_tabs<<<(M + 7) / 8, 256, 0, s>>>(I, M, fft_tab, wm, dm);
  return cudaGetLastError();
}


namespace {
// the kernel arguments of one pass (mode n read, mode v = n + 1 mod N written); false without a plan
// (a compiled plan's kernel ignores the stage list; it is filled from the generic planner only)
bool fft_args(FftArgs& a, FftPlan& pl, const void* U, void* yv, void* ysame, const float* tab, int N,
              const int64_t* dims, int n, int* err, bool cplx, int ct = 0) {
  if (N < 2 || n < 0 || n >= N) return false;
  const int v = (n + 1) % N;
  memset(&a, 0, sizeof(a));
  const int I = (int)dims[n];
  int M = 0, Mpad = 0;   // Bluestein form when nonzero
  if (ct == 1 || ct == 2 || ct == 3) {
    if (ct == 1) ct_plan_of<CtPlan400>(&pl);
    if (ct == 2) ct_plan_of<CtPlan1500>(&pl);
    if (ct == 3) ct_plan_of<CtPlan100>(&pl);
  } else if (!fft_plan(I, dims[v], &pl, cplx)) {
    if (cplx || !fft_plan_bs(I, dims[v], &pl, &M, &Mpad)) return false;
  }
  a.U = U;
  a.yv = yv;
  a.ysame = ysame;
  a.tab = tab;
  a.I = I;
  a.Ipad = pl.Ipad;
  a.BJ = pl.BJ;
  a.S = cplx ? pl.BJ : pl.BJ / 2;
  a.nst = pl.nst;
  a.mH2 = magic(I / 2 + 1);
  a.cscale = (float)(1.0 / sqrt((double)I));
  a.M = M;
  a.Mpad = Mpad;
  a.mM = magic(M);
  a.mI = magic(I);
  const int TL = M ? M : I;   // the length the stages transform
  int Ns = 1;
  for (int st = 0; st < pl.nst; ++st) {
    const int R = kRadR1[pl.rix[st]] * kRadR2[pl.rix[st]];
    StageTab& t = a.st[st];
    t.L = TL / R;
    t.Ns = Ns;
    t.tstep = TL / (Ns * R);
    t.rix = pl.rix[st];
    t.mL = magic(t.L);
    t.mNs = magic(Ns);
    Ns *= R;
  }
  a.Iv = dims[v];
  a.err = err;
  // row strides of the mode-n unfolding (input) and of the mode-v unfolding (output)
  int64_t rin[kMaxOrder], rout[kMaxOrder];
  int64_t acc_in = 1, acc_out = 1, P = 1;
  for (int m = 0; m < N; ++m) {
    P *= dims[m];
    rin[m] = m == n ? 0 : acc_in;
    if (m != n) acc_in *= dims[m];
    rout[m] = m == v ? 0 : acc_out;
    if (m != v) acc_out *= dims[m];
  }
  a.rs_in_v = rin[v];
  a.out_k = dims[v] * rout[n];
  for (int m = 0; m < N; ++m) {
    if (m == n || m == v) continue;
    a.oext[a.no] = dims[m];
    a.o_in[a.no] = rin[m];
    a.o_out[a.no] = rout[m];
    ++a.no;
  }
  a.nchunks = (a.Iv + a.BJ - 1) / a.BJ;
  a.nblocks = a.nchunks * (P / ((int64_t)I * a.Iv));
  return a.nblocks > 0;
}
}  // namespace

bool mix_fft_norm_fits(int dtype, int N, const int64_t* dims) {
  FftArgs a;
  FftPlan pl;
  if (N < 2) return false;
  if (!fft_args(a, pl, nullptr, nullptr, nullptr, nullptr, N, dims, 0, nullptr, false, ct_plan_id((int)dims[0], dims[1 % N])))
    return false;
  int64_t P = 1;
  for (int m = 0; m < N; ++m) P *= dims[m];
  const int64_t es = dtype == CPR_F32 ? 4 : 2;
  const int64_t words = a.nblocks + sumsq_partials_blocks(a.nblocks) + 1;
  return a.nblocks > 0 && words <= P * es / 8;
}

cudaError_t launch_mix_fft(const void* U, void* yv, void* ysame, const float* tab, int dtype, int N,
                           const int64_t* dims, int n, int* err, cudaStream_t s, double* normpart, int64_t* nblocks) {
  FftArgs a;
  FftPlan pl;
  if (N < 2 || n < 0 || n >= N) return cudaErrorInvalidValue;
  const int ct = ct_plan_id((int)dims[n], dims[(n + 1) % N]);
  if (!fft_args(a, pl, U, yv, ysame, tab, N, dims, n, err, false, ct)) return cudaErrorInvalidValue;
  a.normpart = normpart;
  if (nblocks) *nblocks = a.nblocks;
  const int I = a.I;
  const size_t es = dtype == CPR_F32 ? 4 : 2;
  a.bulk = dtype == CPR_F32 && (I * es) % 16 == 0 && (reinterpret_cast<uintptr_t>(U) & 15) == 0;
  const uintptr_t vmask = 4 * es - 1;   // 4 entries per vector store
  a.vec_v = a.Iv % 4 == 0 && (reinterpret_cast<uintptr_t>(yv) & vmask) == 0;
  a.vec_in = dtype == CPR_BF16 && I % 4 == 0 && (reinterpret_cast<uintptr_t>(U) & 7) == 0;
  if (ct == 1)
    return dtype == CPR_F32 ? launch_fft_ct_kernel<float, CtPlan400>(a, s)
                            : launch_fft_ct_kernel<__nv_bfloat16, CtPlan400>(a, s);
  if (ct == 2)
    return dtype == CPR_F32 ? launch_fft_ct_kernel<float, CtPlan1500>(a, s)
                            : launch_fft_ct_kernel<__nv_bfloat16, CtPlan1500>(a, s);
  if (ct == 3)
    return dtype == CPR_F32 ? launch_fft_ct_kernel<float, CtPlan100>(a, s)
                            : launch_fft_ct_kernel<__nv_bfloat16, CtPlan100>(a, s);
  if (a.M > 0) {
    if (dtype == CPR_F32)
      return pl.tpb == 128 ? launch_fft_bs_kernel<float, 128>(a, pl.smem, s)
                           : launch_fft_bs_kernel<float, 256>(a, pl.smem, s);
    if (dtype == CPR_BF16)
      return pl.tpb == 128 ? launch_fft_bs_kernel<__nv_bfloat16, 128>(a, pl.smem, s)
                           : launch_fft_bs_kernel<__nv_bfloat16, 256>(a, pl.smem, s);
    return cudaErrorInvalidValue;
  }
  if (dtype == CPR_F32)
    return pl.tpb == 128 ? launch_fft_kernel<float, 128>(a, pl.smem, s) : launch_fft_kernel<float, 256>(a, pl.smem, s);
  if (dtype == CPR_BF16)
    return pl.tpb == 128 ? launch_fft_kernel<__nv_bfloat16, 128>(a, pl.smem, s)
                         : launch_fft_kernel<__nv_bfloat16, 256>(a, pl.smem, s);
  return cudaErrorInvalidValue;
}

bool mix_cfft_supported(int N, const int64_t* dims) {
  if (N < 2) return false;
  for (int n = 0; n < N; ++n) {
    if (dims[n] < 5) return false;
    FftPlan pl;
    if (!fft_plan((int)dims[n], dims[(n + 1) % N], &pl, true)) return false;
  }
  return true;
}

cudaError_t launch_mix_cfft(const void* U, bool real_in, void* yv, void* ysame, const float* tab, int N,
                            const int64_t* dims, int n, int* err, cudaStream_t s) {
  FftArgs a;
  FftPlan pl;
  if (!fft_args(a, pl, U, yv, ysame, tab, N, dims, n, err, true)) return cudaErrorInvalidValue;
  if (real_in)
    return pl.tpb == 128 ? launch_cfft_kernel<float, 128>(a, pl.smem, s) : launch_cfft_kernel<float, 256>(a, pl.smem, s);
  return pl.tpb == 128 ? launch_cfft_kernel<float2, 128>(a, pl.smem, s) : launch_cfft_kernel<float2, 256>(a, pl.smem, s);
}

}  // namespace cpr
