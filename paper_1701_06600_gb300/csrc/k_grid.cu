// The whole outer-iteration loop of CPRAND (Alg. 3 with Alg. 2, the sampled fit of Sec. 3.4 and
// the stopping rules of Sec. 4.2) for one large problem at a time, spread over the whole GPU: a
// cooperative launch of one 512-thread CTA per SM, phases separated by grid-wide barriers.
//
// This is the path for problems whose factors and sampled fibers are far too large for one
// thread-block cluster (1500^3 with R = 50 and S = 2000: 12 MB of fibers and 2.5 million FP64 Gram
// products per mode update).  On this GPU FP64 issues at about 1.7 operations per clock per SM
// against 128 for FP32, so every FP64 step is spread evenly over all SMs and kept to a plain
// product form with every lane busy.  Per mode update n of outer iteration t:
//
//   P1  (concurrently, in disjoint warps of every CTA)
//       warps 0-3   partial FP64 Gram Z_S^T Z_S (packed upper triangle) of the CTA's ceil(S/G)
//                   samples: the Z_S rows (Alg. 2) as FP64 products of the FP32 factor rows times
//                   the lazy column scales.
//       warps 4-15  contraction units (96 fiber rows x one split of the samples): the split's
//                   Z_S rows in FP32, the sampled fibers (Sec. 3.2 index map) streamed through
//                   shared memory in chunks of 32 samples (the next chunk's loads in flight while
//                   the current one is multiplied), M_split = X_S Z_S with FP32 accumulation,
//                   stored column-major to global scratch.  The next mode update's fiber
//                   segments are prefetched into L2 (the draw depends on the Philox counter only).
//   --- grid barrier
//   P2  each CTA sums a slice of the packed Gram over the G partials (fixed order) and the split
//       partials of its own ceil(I_n/G) factor rows (FP64).
//   --- grid barrier
//   P3  every CTA reads G and inverts its Jacobi-scaled copy in FP32 (the sweep operator, one
//       block barrier per pivot; the same arithmetic in every CTA, so the same decisions), then
//       solves its rows: A0 = M G^-1 with the FP32 inverse, then refinement steps
//       A <- A + (M - A G) G^-1 with the residual M - A G in FP64 (a dense product, every lane
//       busy) until the correction is below 1e-5 of the row block, which leaves an error near its
//       square (at most three steps).  A
//       non-positive sweep pivot falls back to an FP64 Cholesky inverse; a non-positive Cholesky
//       pivot is a singular Gram (CPR_ESINGULAR).  The rows go to the FP64 factor and its FP32
//       copy (unnormalized), their column sums of squares to global scratch.
//   --- grid barrier
//   P4  every CTA sums the column partials (fixed order): lambda_r and the lazy scale 1/lambda_r.
// After the N modes: the CTA's share of the P_hat fixed fit entries (one warp per entry, FP32
// model, FP64 squares), a grid barrier, and every CTA sums the G partials in the same order and
// applies the stopping rules to its own copy of the loop state.
//
// Cross-CTA data is written before a barrier and read after it with L1-bypassing loads.  Every
// barrier wait is bounded (opts->wait_budget polls, default about a second): a CTA whose wait runs
// out sets the error flag and returns; CTAs that see the flag at a barrier return too, so the
// kernel always ends, and the call reports CPR_ETIMEOUT.  This kernel issues no asynchronous
// copies, so a CTA that returns early leaves nothing in flight.
#include <math.h>

#include "internal.cuh"
#include "small_spd.cuh"
#include "tc_util.cuh"

namespace cpr {

namespace {

constexpr int kGT = 512;                 // threads per CTA
constexpr int kGW = kGT / 32;            // warps per CTA
constexpr int kGramT = 128;              // threads of the Gram partial (warps 0-3)
constexpr int kCT = kGT - kGramT;        // contraction threads (warps 4-15)
constexpr int kTI = 96;                  // fiber rows per contraction tile
constexpr int kCG = kCT / kTI;           // column groups per tile row (4)
constexpr int kSC = 128;                 // samples per super-chunk (Z_S rows staged in shared memory)
constexpr int kXC = 32;                  // samples per fiber chunk
constexpr int kXPT = kXC * kTI / kCT;    // fiber elements per contraction thread and chunk (8)
constexpr int kGC = 32;                  // Gram samples per chunk
constexpr int kTM = 128;                 // tensor-core contraction: fiber rows per unit (MMA M)
constexpr int kTK = 32;                  // tensor-core contraction: samples per stage (128 bytes of FP32)
constexpr int kPPT = (kTM * (kTK / 4) + kCT - 1) / kCT;   // (row, 4-sample) pairs per contraction thread and stage
constexpr int kNEMax = kMaxRank * (kMaxRank + 1) / 2;
static_assert(kTI % 32 == 0 && kCT % kTI == 0 && (kXC * kTI) % kCT == 0, "tile shape");
static_assert(kTI <= kGridTileRows && kTM <= kGridTileRows, "the workspace sizes Mpart for the tile height");

__device__ __forceinline__ unsigned ld_acquire_u32(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void st_release_u32(unsigned* p, unsigned v) {
  asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_relaxed_i32(const int* p) {
  int v;
  asm volatile("ld.relaxed.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void prefetch_l2(const void* p) {
  asm volatile("prefetch.global.L2 [%0];" ::"l"(p));
}
__device__ __forceinline__ void named_sync(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
// Shared-memory accesses by shared-window address (a function that is not inlined cannot tell that a
// generic pointer points to shared memory).
__device__ __forceinline__ float lds_f32(uint32_t a) {
  float v;
  asm volatile("ld.shared.f32 %0, [%1];" : "=f"(v) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ float4 lds_v4f32(uint32_t a) {
  float4 v;
  asm volatile("ld.shared.v4.f32 {%0, %1, %2, %3}, [%4];" : "=f"(v.x), "=f"(v.y), "=f"(v.z), "=f"(v.w) : "r"(a) : "memory");
  return v;
}
__device__ __forceinline__ void sts_f32(uint32_t a, float v) {
  asm volatile("st.shared.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
// Arrives at block barrier id (n threads in all) without waiting; the threads that wait call named_sync.
__device__ __forceinline__ void named_arrive(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

// AND of v over the n threads of block barrier id (which all call it); also a barrier for them.
__device__ __forceinline__ bool named_and(int id, int n, bool v) {
  int r;
  asm volatile(
      "{\n .reg .pred p, q;\n setp.ne.s32 p, %1, 0;\n bar.red.and.pred q, %2, %3, p;\n selp.s32 %0, 1, 0, q;\n}\n"
      : "=r"(r)
      : "r"((int)v), "r"(id), "r"(n)
      : "memory");
  return r != 0;
}

template <typename T> __device__ __forceinline__ float gf(T v);
template <> __device__ __forceinline__ float gf<float>(float v) { return v; }
template <> __device__ __forceinline__ float gf<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Shared-memory layout (byte offsets), computed identically on the host and the device.  What is
// used after the contraction (G, its FP32 inverse, the row solve) overlays the P1 region.
struct GridSmem {
  int g2, x0, piv, dp;     // S: G as pairs (the FP64 fallback's inverse reuses it), Gs then X0 in place
                           // (FP32), the sweep's published pivot entries, the Jacobi scales D'
  int gids, Zd;            // P1, Gram warps
  int cids, coffs, Zf, xs; // P1, contraction warps (xs: SIMT fiber chunks)
  int stage;               // P1, tensor-core stages (aligned to 1024 bytes at run time)
  int mrow, m32, a2;       // P3 (overlays P1): M rows as pairs, FP32 scratch, A rows as pairs
  int G, fL, fT, fd, arow; // P3, FP64 fallback: G, Cholesky factor, triangular inverse, A rows
  int bytes;
  int ZP;                  // Zf row pitch (MAXR)
};
__host__ __device__ inline int ga16(int x) { return (x + 15) / 16 * 16; }

// S is written by the Gram warps while the contraction warps use P1, and read by the row solve (P3)
__host__ __device__ inline GridSmem grid_layout(int R, int MAXR, int tbytes) {
  GridSmem L;
  L.ZP = MAXR;
  int o = 0;
  L.g2 = o;    o = ga16(o + R * R * 8);
  L.x0 = o;    o = ga16(o + R * R * 4);
  L.piv = o;   o = ga16(o + 2 * 64 * 4);
  L.dp = o;    o = ga16(o + MAXR * 4);
  const int s_end = o;
  // P1: Gram warps, contraction warps (the SIMT fiber chunks or the tensor-core stages)
  L.gids = o;  o = ga16(o + kGC * kMaxOrder * 4);
  L.Zd = o;    o = ga16(o + kGC * R * 8);
  L.cids = o;  o = ga16(o + kSC * kMaxOrder * 4);
  L.coffs = o; o = ga16(o + kSC * 8);
  L.Zf = o;    o = ga16(o + kSC * MAXR * 4);
  L.xs = o;
  const int simt_end = ga16(o + 2 * kXC * kTI * tbytes);
  o = (o + 1023) / 1024 * 1024;          // + up to 1023 bytes of alignment of the dynamic base
  L.stage = o;
  const int tc_end = o + 1024 + 2 * (2 * kTM * kTK * 4 + 2 * MAXR * kTK * 4);
  const int p1 = simt_end > tc_end ? simt_end : tc_end;
  // P3, after the contraction (overlays P1): the row solve; the FP64 fallback's scratch behind it
  o = s_end;
  L.mrow = o;  o = ga16(o + kGridMaxRows * R * 8);
  L.m32 = o;   o = ga16(o + kGridMaxRows * R * 4);
  L.a2 = o;    o = ga16(o + kGridMaxRows * R * 8);
  L.G = o;     o = ga16(o + R * R * 8);
  L.fL = o;    o = ga16(o + R * R * 8);
  L.fT = o;    o = ga16(o + R * R * 8);
  L.fd = o;    o = ga16(o + R * 8);
  L.arow = o;  o = ga16(o + kGridMaxRows * R * 8);
  const int p3 = o;
  L.bytes = p1 > p3 ? p1 : p3;
  return L;
}

struct GridCtx {
  unsigned gen;       // barrier generation this CTA has passed
  int G, c;           // CTAs, this CTA
};

// Grid-wide barrier with a bounded wait.  Returns false (in every thread of the CTA) when the wait
// ran out or another CTA reported an error; the caller then returns.
// bar_id / nthr: the block barrier of the calling threads (0 / kGT: the whole CTA; thread 0 must be one
// of them, and every CTA's thread 0 calls the same sequence of grid barriers).
__device__ __forceinline__ bool grid_sync(const GridScratch& gs, GridCtx& x, int* s_flag, int bar_id = 0,
                                          int nthr = kGT) {
  named_sync(bar_id, nthr);
  if (threadIdx.x == 0) {
    int ok = 1;
    const unsigned my = x.gen;
    __threadfence();
    const unsigned arrived = atomicAdd(gs.bar, 1u) + 1u;
    if (arrived == (unsigned)x.G) {
      *((volatile unsigned*)gs.bar) = 0u;
      __threadfence();
      st_release_u32(gs.bar + 1, my + 1u);
    } else {
      uint32_t it = 0;
      while (ld_acquire_u32(gs.bar + 1) == my) {
        if (++it > gs.wait_limit) {
          ok = 0;
          break;
        }
        __nanosleep(32);
      }
    }
    __threadfence();
    if (ok && ld_relaxed_i32(gs.err) != 0) ok = 0;
    if (!ok) atomicExch(gs.err, 1);
    x.gen = my + 1u;
    *s_flag = ok;
  }
  named_sync(bar_id, nthr);
  return *s_flag != 0;
}

// ---- FP64-class quantities as unevaluated pairs of FP32 values, x = hi + lo.  On this part the FP64
// units run at about 1/75 of the FP32 rate (conversions between FP32 and FP64 included), so the
// Gram, M, the residual of the row solve and the column norms are carried as pairs and combined by
// error-free transformations: Dekker's exact product (a b = p + e, e by one FMA) and Knuth's two-sum
// (a + b = s + e).  A sum of pair products keeps about 2^-44 of the sum of the terms' magnitudes.
// Rounding-mode intrinsics keep the compiler from contracting or reordering these steps.

// x as a pair (hi = x rounded to FP32, lo = the remainder rounded: |x - hi - lo| <= 2^-48 |x|)
__device__ __forceinline__ float2 split_pair(double x) {
  const float h = (float)x;
  return make_float2(h, (float)(x - (double)h));
}
__device__ __forceinline__ double pair_value(float2 a) { return (double)a.x + (double)a.y; }

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float& s, float& e) {
  s = __fadd_rn(a, b);
  const float bv = __fsub_rn(s, a);
  e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bv)), __fsub_rn(b, bv));
}
// the pair (hi, lo) renormalized so that hi = fl(hi + lo)
__device__ __forceinline__ float2 pair_norm(float hi, float lo) {
  float s, e;
  two_sum(hi, lo, s, e);
  return make_float2(s, e);
}
// (sh, sl) += b for an FP32 value b
__device__ __forceinline__ void pair_acc(float b, float& sh, float& sl) {
  float s, e;
  two_sum(sh, b, s, e);
  sh = s;
  sl = __fadd_rn(sl, e);
}
// (sh, sl) += b for a pair b
__device__ __forceinline__ void pair_acc2(float2 b, float& sh, float& sl) {
  float s, e;
  two_sum(sh, b.x, s, e);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(e, b.y));
}
// a * b for a pair a and an FP32 value b
__device__ __forceinline__ float2 pair_mul_f(float2 a, float b) {
  const float p = __fmul_rn(a.x, b);
  const float e = __fmaf_rn(a.x, b, -p);
  return make_float2(p, __fmaf_rn(a.y, b, e));
}
// a * b for pairs (a.lo b.lo, below 2^-48 of the product, dropped)
__device__ __forceinline__ float2 pair_mul(float2 a, float2 b) {
  const float p = __fmul_rn(a.x, b.x);
  const float e = __fmaf_rn(a.x, b.x, -p);
  return pair_norm(p, __fmaf_rn(a.x, b.y, __fmaf_rn(a.y, b.x, e)));
}
// (sh, sl) += a * g for pairs a, g: the exact product of the high parts plus the two cross terms
__device__ __forceinline__ void pair_fma(float2 a, float2 g, float& sh, float& sl) {
  const float p = __fmul_rn(a.x, g.x);
  const float pe = __fmaf_rn(a.x, g.x, -p);
  const float cr = __fmaf_rn(a.x, g.y, __fmul_rn(a.y, g.x));
  float s, err;
  two_sum(sh, p, s, err);
  sh = s;
  sl = __fadd_rn(sl, __fadd_rn(err, __fadd_rn(pe, cr)));
}

// out[j] = sum over i < rows of src[i * stride + j] for j < cols (cols <= 64), from global scratch
// written by other CTAs: the rows are split into at most 32 chunks, each thread sums one (chunk,
// column) pair with its loads in flight together, and the chunk partials are then added in chunk
// order.  The order is fixed, so every CTA that sums the same data gets the same result.  part:
// nthr doubles of shared memory.  Called by threads 0 .. nthr-1 (block barrier bar_id); ends with
// that barrier.
__device__ void sum_rows(const double* src, int rows, int cols, int64_t stride, double* out, double* part,
                         int bar_id = 0, int nthr = kGT) {
  const int tid = threadIdx.x;
  int cp = 1;
  while (cp < cols) cp <<= 1;
  const int nch = min(nthr / cp, 32);
  const int j = tid % cp, q = tid / cp;
  double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
  if (j < cols && q < nch) {
    const int per = (rows + nch - 1) / nch;
    const int r0 = q * per, r1 = min(rows, r0 + per);
    int i = r0;
    for (; i + 3 < r1; i += 4) {
      a0 += __ldcg(src + (int64_t)i * stride + j);
      a1 += __ldcg(src + (int64_t)(i + 1) * stride + j);
      a2 += __ldcg(src + (int64_t)(i + 2) * stride + j);
      a3 += __ldcg(src + (int64_t)(i + 3) * stride + j);
    }
    for (; i < r1; ++i) a0 += __ldcg(src + (int64_t)i * stride + j);
  }
  if (q < nch) part[q * cp + j] = (a0 + a1) + (a2 + a3);
  named_sync(bar_id, nthr);
  if (tid < cols) {
    double b0 = 0.0, b1 = 0.0, b2 = 0.0, b3 = 0.0;
    int qq = 0;
    for (; qq + 3 < nch; qq += 4) {
      b0 += part[qq * cp + tid];
      b1 += part[(qq + 1) * cp + tid];
      b2 += part[(qq + 2) * cp + tid];
      b3 += part[(qq + 3) * cp + tid];
    }
    for (; qq < nch; ++qq) b0 += part[qq * cp + tid];
    out[tid] = (b0 + b1) + (b2 + b3);
  }
  named_sync(bar_id, nthr);
}

// The same fixed-order sum over rows for pair-valued entries (src: rows x cols pairs, row stride
// `stride`); out: cols pairs; part: scratch of nthr pairs.
__device__ void sum_pairs(const float2* src, int rows, int cols, int64_t stride, float2* out, float2* part,
                          int bar_id = 0, int nthr = kGT) {
  const int tid = threadIdx.x;
  int cp = 1;
  while (cp < cols) cp <<= 1;
  const int nch = min(nthr / cp, 32);
  const int j = tid % cp, q = tid / cp;
  float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
  if (j < cols && q < nch) {
    const int per = (rows + nch - 1) / nch;
    const int r0 = q * per, r1 = min(rows, r0 + per);
    int i = r0;
    for (; i + 7 < r1; i += 8) {   // eight loads in flight
      float2 v[8];
#pragma unroll
      for (int k = 0; k < 8; ++k) v[k] = __ldcg(src + (int64_t)(i + k) * stride + j);
#pragma unroll
      for (int k = 0; k < 8; k += 2) {
        pair_acc2(v[k], h0, l0);
        pair_acc2(v[k + 1], h1, l1);
      }
    }
    for (; i < r1; ++i) pair_acc2(__ldcg(src + (int64_t)i * stride + j), h0, l0);
    pair_acc2(make_float2(h1, l1), h0, l0);
  }
  if (q < nch) part[q * cp + j] = make_float2(h0, l0);
  named_sync(bar_id, nthr);
  if (tid < cols) {
    float h = 0.f, l = 0.f;
    for (int qq = 0; qq < nch; ++qq) pair_acc2(part[qq * cp + tid], h, l);
    out[tid] = pair_norm(h, l);
  }
  named_sync(bar_id, nthr);
}

// Sample j of mode update (n, t): indices by mode (mode-n slot 0) and the fiber's storage offset
// in the copy mode n reads (Philox stream 0, counter (j, n, t, b); the k-th mode other than n takes
// word k%4 of block k/4; i_m = floor(w I_m / 2^32)).  With a caller sample table (test hook), the
// multi-index is read from it instead.
__device__ __forceinline__ int64_t grid_draw(const Prob& p, int n, uint32_t t, uint32_t j, uint32_t* ids) {
  if (p.user_idx) {
    const uint32_t* u = p.user_idx + ((int64_t)n * p.S + j) * p.N;
    for (int m = 0; m < p.N; ++m) ids[m] = m == n ? 0u : u[m];
  } else {
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
    const uint4 w0 = philox10(make_uint4(j, counter_word1(kStreamSamples, 0, n), t, p.b), k0, k1);
    uint4 w1 = make_uint4(0u, 0u, 0u, 0u);
    if (p.N - 1 > 4) w1 = philox10(make_uint4(j, counter_word1(kStreamSamples, 1, n), t, p.b), k0, k1);
    int k = 0;
    for (int m = 0; m < p.N; ++m) {
      uint32_t im = 0;
      if (m != n) {
        const uint32_t w = k < 4 ? word_of(w0, k) : word_of(w1, k - 4);
        im = scale_index(w, (uint32_t)p.dims[m]);
        ++k;
      }
      ids[m] = im;
    }
  }
  int64_t stride;
  return fiber_offset(p, n, ids, &stride);
}

// Rows jj < cnt of the sampled Khatri-Rao product (Alg. 2) for the modes other than n:
// out[jj * pitch + r] = pre[r] * prod_{m != n} A32[m](ids[jj][m], r) for r < R (0 for R <= r < pitch),
// by nthr threads (a multiple of 64; t = this thread's index among them): thread t takes column
// t % 64 of every (nthr / 64)-th sample, and the factor-row loads of 8 samples of one mode are
// issued together (L2-resident rows: the latency, not the bandwidth, is what these loads cost).
template <typename OUT, int KB = 8>
__device__ __forceinline__ void build_rows(const Prob& p, int n, const uint32_t* ids, int cnt, const OUT* pre,
                                           OUT* out, int pitch, int t, int nthr) {
  // thread t: column r = t % 64 of samples t / 64 + k (nthr / 64), k < KB per round; every factor
  // row entry of a round is loaded before any is used
  const int R = p.R, N = p.N;
  const int r = t & 63, lanes = nthr >> 6;
  if (r >= pitch) return;
  for (int b = t >> 6; b < cnt; b += KB * lanes) {
    OUT z[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) z[k] = r < R ? pre[r] : OUT(0);
    for (int m = 0; m < N; ++m) {
      if (m == n) continue;
      const float* Am = p.A32[m];
      float v[KB];
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const int jj = b + k * lanes;
        v[k] = (jj < cnt && r < R) ? __ldcg(Am + (int64_t)ids[jj * kMaxOrder + m] * R + r) : 1.f;
      }
#pragma unroll
      for (int k = 0; k < KB; ++k) z[k] *= (OUT)v[k];
    }
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const int jj = b + k * lanes;
      if (jj < cnt) out[jj * pitch + r] = z[k];
    }
  }
}

// Work split of mode n over G CTAs.
struct ModeSplit {
  int I, ntile, nsplit, spl, units, rpc;
};

__device__ __forceinline__ ModeSplit mode_split(const Prob& p, int n, int G, int tile_rows) {
  ModeSplit s;
  s.I = (int)p.dims[n];
  s.ntile = (s.I + tile_rows - 1) / tile_rows;
  int ns = G / s.ntile;
  if (ns < 1) ns = 1;
  const int mins = p.grid_min_split > 0 ? p.grid_min_split : 16;
  const int most = (p.S + mins - 1) / mins;   // at least mins samples per split
  if (ns > most) ns = most;
  s.spl = (p.S + ns - 1) / ns;
  s.nsplit = (p.S + s.spl - 1) / s.spl;
  s.units = s.ntile * s.nsplit;
  s.rpc = (s.I + G - 1) / G;
  return s;
}

// ---- P1, Gram warps: partial Z'^T Z' over this CTA's samples (packed upper triangle) as pairs,
// where Z' are the sampled Khatri-Rao rows of the FP32 factor copies without the lazy column scales
// (Z_S = Z' Sc, so Z_S^T Z_S = Sc (Z'^T Z') Sc: the scales are applied to the reduced Gram).  A Z'
// entry is the product of N - 1 FP32 values, exact as a pair for N = 3.
__device__ __forceinline__ void build_pairs(const Prob& p, int n, const uint32_t* ids, int cnt, float2* out, int pitch,
                                            int t, int nthr) {
  const int R = p.R, N = p.N;
  const int r = t & 63, lanes = nthr >> 6;
  if (r >= pitch) return;
  constexpr int KB = kGC / (kGramT / 64);   // the chunk's samples in one round of loads
  for (int b = t >> 6; b < cnt; b += KB * lanes) {
    float2 z[KB];
#pragma unroll
    for (int k = 0; k < KB; ++k) z[k] = make_float2(1.f, 0.f);
    for (int m = 0; m < N; ++m) {
      if (m == n) continue;
      const float* Am = p.A32[m];
      float v[KB];
#pragma unroll
      for (int k = 0; k < KB; ++k) {
        const int jj = b + k * lanes;
        v[k] = (jj < cnt && r < R) ? __ldcg(Am + (int64_t)ids[jj * kMaxOrder + m] * R + r) : 0.f;
      }
#pragma unroll
      for (int k = 0; k < KB; ++k) z[k] = pair_mul_f(z[k], v[k]);
    }
#pragma unroll
    for (int k = 0; k < KB; ++k) {
      const int jj = b + k * lanes;
      if (jj < cnt) out[jj * pitch + r] = z[k];
    }
  }
}

// Not inlined: its register allocation then stays apart from the rest of the kernel (1500^3: 164.6 us
// per outer iteration, against 171.4 with the function inlined).
template <int MAXR>
__device__ __noinline__ void gram_partial(const Prob& p, const GridSmem& L, unsigned char* sm, const GridScratch& gs,
                                          const GridCtx& x, int n, uint32_t t, const unsigned char* ne_r,
                                          const unsigned char* ne_c) {
  const int tid = threadIdx.x, R = p.R, S = p.S;
  const int NE = R * (R + 1) / 2;
  const int gpc = (S + x.G - 1) / x.G;
  const int j0 = x.c * gpc;
  const int jn = min(S, j0 + gpc);
  uint32_t* ids = reinterpret_cast<uint32_t*>(sm + L.gids);
  float2* Zp = reinterpret_cast<float2*>(sm + L.Zd);
  float2* dst = gs.Gpart + (int64_t)x.c * NE;
  for (int c0 = j0; c0 < jn; c0 += kGC) {
    const int cnt = min(kGC, jn - c0);
    if (tid < cnt) grid_draw(p, n, t, (uint32_t)(c0 + tid), ids + tid * kMaxOrder);
    named_sync(1, kGramT);
    build_pairs(p, n, ids, cnt, Zp, R, tid, kGramT);
    named_sync(1, kGramT);
    // one entry at a time, its sum over the chunk's samples in two interleaved pair accumulators
    for (int e = tid; e < NE; e += kGramT) {
      const int r = ne_r[e], cc = ne_c[e];
      float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
      if (c0 > j0) {
        const float2 prev = dst[e];   // this thread's own earlier chunk
        h0 = prev.x;
        l0 = prev.y;
      }
      int jj = 0;
      for (; jj + 1 < cnt; jj += 2) {
        pair_fma(Zp[jj * R + r], Zp[jj * R + cc], h0, l0);
        pair_fma(Zp[(jj + 1) * R + r], Zp[(jj + 1) * R + cc], h1, l1);
      }
      if (jj < cnt) pair_fma(Zp[jj * R + r], Zp[jj * R + cc], h0, l0);
      pair_acc2(make_float2(h1, l1), h0, l0);
      dst[e] = pair_norm(h0, l0);
    }
    named_sync(1, kGramT);
  }
  if (j0 >= jn)
    for (int e = tid; e < NE; e += kGramT) dst[e] = make_float2(0.f, 0.f);
}

// ---- P1, contraction warps: M_split(tile rows, :) = X_S Z_S over the unit's samples, FP32.
template <typename T, int MAXR>
__device__ void contract_units(const Prob& p, const GridSmem& L, unsigned char* sm, const GridScratch& gs,
                               const GridCtx& x, int n, uint32_t t, const ModeSplit& ms, const float* scf) {
  constexpr int CW = MAXR / kCG;           // columns per thread
  static_assert(CW % 4 == 0, "float4 Z loads");
  const int ct = threadIdx.x - kGramT;     // 0 .. kCT-1
  const int ii = ct % kTI, g = ct / kTI;
  const int R = p.R, ZP = L.ZP;
  uint32_t* ids = reinterpret_cast<uint32_t*>(sm + L.cids);
  int64_t* offs = reinterpret_cast<int64_t*>(sm + L.coffs);
  float* Zf = reinterpret_cast<float*>(sm + L.Zf);
  T* xs = reinterpret_cast<T*>(sm + L.xs);
  const T* __restrict__ X = reinterpret_cast<const T*>(p.Xrep[n]);
  const int64_t stride = p.use_rep ? 1 : p.st[n];
  for (int u = x.c; u < ms.units; u += x.G) {
    const int tile = u % ms.ntile, split = u / ms.ntile;
    const int i0 = tile * kTI;
    const int js = split * ms.spl;
    const int cnt = min(ms.spl, p.S - js);
    float acc[CW];
#pragma unroll
    for (int k = 0; k < CW; ++k) acc[k] = 0.f;
    for (int s0 = 0; s0 < cnt; s0 += kSC) {
      const int scn = min(kSC, cnt - s0);
      named_sync(2, kCT);   // the previous super-chunk's Z rows and fibers are no longer read
      for (int jj = ct; jj < scn; jj += kCT)
        offs[jj] = grid_draw(p, n, t, (uint32_t)(js + s0 + jj), ids + jj * kMaxOrder);
      named_sync(2, kCT);
      // Z_S rows of the super-chunk in FP32 (zero-padded to the pitch)
      build_rows<float>(p, n, ids, scn, scf, Zf, ZP, ct, kCT);
      // fibers: chunks of kXC samples x kTI rows, the next chunk's loads in flight
      const int nch = (scn + kXC - 1) / kXC;
      T reg[kXPT];
      auto load_chunk = [&](int k) {
#pragma unroll
        for (int q = 0; q < kXPT; ++q) {
          const int e = ct + q * kCT;
          const int jj = k * kXC + e / kTI, r = e % kTI;
          T v = T(0.f);
          if (jj < scn && i0 + r < ms.I) v = X[offs[jj] + (int64_t)(i0 + r) * stride];
          reg[q] = v;
        }
      };
      auto store_chunk = [&](int k) {
        T* dst = xs + (k & 1) * (kXC * kTI);
#pragma unroll
        for (int q = 0; q < kXPT; ++q) dst[ct + q * kCT] = reg[q];
      };
      load_chunk(0);
      store_chunk(0);
      named_sync(2, kCT);
      for (int k = 0; k < nch; ++k) {
        if (k + 1 < nch) load_chunk(k + 1);
        const T* xb = xs + (k & 1) * (kXC * kTI);
        const int jn = min(kXC, scn - k * kXC);
        const float* zb = Zf + (k * kXC) * ZP + g * CW;
#pragma unroll 2
        for (int jj = 0; jj < jn; ++jj) {
          const float xv = gf<T>(xb[jj * kTI + ii]);
          const float4* z4 = reinterpret_cast<const float4*>(zb + jj * ZP);
#pragma unroll
          for (int v = 0; v < CW / 4; ++v) {
            const float4 zq = z4[v];
            acc[4 * v + 0] = fmaf(xv, zq.x, acc[4 * v + 0]);
            acc[4 * v + 1] = fmaf(xv, zq.y, acc[4 * v + 1]);
            acc[4 * v + 2] = fmaf(xv, zq.z, acc[4 * v + 2]);
            acc[4 * v + 3] = fmaf(xv, zq.w, acc[4 * v + 3]);
          }
        }
        if (k + 1 < nch) store_chunk(k + 1);
        named_sync(2, kCT);
      }
    }
    // M_split stored column-major (lanes = consecutive rows)
    const int i = i0 + ii;
    if (i < ms.I) {
      float* dst = gs.Mpart + (int64_t)split * R * ms.I + i;
#pragma unroll
      for (int k = 0; k < CW; ++k) {
        const int r = g * CW + k;
        if (r < R) dst[(int64_t)r * ms.I] = acc[k];
      }
    }
  }
}

// ---- P1, contraction warps on the tensor cores: the same M_split = X_S Z_S for 128-row units.
// Per stage of 32 samples the contraction warps write the unit's X_S tile (A: 128 rows x 32 samples)
// and the Z_S rows (B: MAXR columns x 32 samples) into shared memory as TF32 hi / lo halves in the
// swizzled K-major layout (each thread one row and four consecutive samples: the loads of a warp
// read 32 consecutive fiber entries, its 16-byte stores hit distinct banks), and one thread issues
// the MMAs hi*hi + hi*lo + lo*hi (lo*hi is exactly zero for BF16 tensors, whose values are TF32
// values, and is skipped) into a 128 x MAXR FP32 accumulator in TMEM.  Two stages alternate; a stage
// is rewritten once the MMAs that read it have completed (tcgen05.commit on its mbarrier).  After a
// unit's last stage the four warps 4-7 read the accumulator (one row per TMEM lane) and store the
// partial M column-major.  Every wait is bounded; one that runs out sets *s_tcerr, after which no
// more MMAs are issued and the CTA waits (bounded) for the ones in flight.
struct TcCtx {
  uint64_t* bar;        // [0], [1]: stage MMAs complete
  uint32_t tmem;        // accumulator base (128 lanes x MAXR columns)
  unsigned char* st;    // stage buffers, 1024-byte aligned
  uint32_t uses[2];     // commits made on each stage's mbarrier so far (uniform across the warps)
  uint32_t limit;
};

template <typename T, int MAXR>
__device__ void contract_units_tc(const Prob& p, const GridSmem& L, unsigned char* sm, const GridScratch& gs,
                                  const GridCtx& x, int n, uint32_t t, const ModeSplit& ms, const float* scf,
                                  TcCtx& tcx, volatile int* s_tcerr) {
  constexpr int NT = MAXR;                       // MMA N (a multiple of 16)
  constexpr int AH = kTM * kTK * 4;              // one A half: 16 KB
  constexpr int BH = NT * kTK * 4;               // one B half
  constexpr int STG = 2 * AH + 2 * BH;           // one stage
  constexpr bool kLoA = sizeof(T) == 4;          // FP32 tensors need the A lo half
  const int ct = threadIdx.x - kGramT;
  const int R = p.R, ZP = L.ZP;
  uint32_t* ids = reinterpret_cast<uint32_t*>(sm + L.cids);
  int64_t* offs = reinterpret_cast<int64_t*>(sm + L.coffs);
  float* Zf = reinterpret_cast<float*>(sm + L.Zf);
  const T* __restrict__ X = reinterpret_cast<const T*>(p.Xrep[n]);
  const int64_t stride = p.use_rep ? 1 : p.st[n];
  const uint32_t idesc = tc::idesc_tf32(kTM, NT);
  for (int u = x.c; u < ms.units; u += x.G) {
    const int tile = u % ms.ntile, split = u / ms.ntile;
    const int i0 = tile * kTM;
    const int js = split * ms.spl;
    const int cnt = min(ms.spl, p.S - js);
    bool first = true;                           // the unit's first MMA overwrites the accumulator
    for (int s0 = 0; s0 < cnt; s0 += kSC) {
      const int scn = min(kSC, cnt - s0);
      named_sync(2, kCT);                        // the previous super-chunk's ids and Z rows are free
      for (int jj = ct; jj < scn; jj += kCT)
        offs[jj] = grid_draw(p, n, t, (uint32_t)(js + s0 + jj), ids + jj * kMaxOrder);
      named_sync(2, kCT);
      build_rows<float, (kSC + kCT / 64 - 1) / (kCT / 64)>(p, n, ids, scn, scf, Zf, ZP, ct, kCT);
      named_sync(2, kCT);
      const int nch = (scn + kTK - 1) / kTK;
      // the X_S values of a chunk: thread ct takes (row r, 4-sample group c) pairs e = ct + u kCT; all
      // of a chunk's loads are issued together, as soon as the previous chunk's values are converted
      float va[kPPT][4];
      auto load_chunk = [&](int k, float (&v)[kPPT][4]) {
#pragma unroll
        for (int u = 0; u < kPPT; ++u) {
          const int e = ct + u * kCT;
          const int r = e % kTM, c = e / kTM;
          const int i = i0 + r;
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int jj = k * kTK + 4 * c + q;
            v[u][q] = (e < kTM * (kTK / 4) && jj < scn && i < ms.I) ? gf<T>(X[offs[jj] + (int64_t)i * stride]) : 0.f;
          }
        }
      };
      load_chunk(0, va);
      for (int k = 0; k < nch; ++k) {
        const int sidx = (int)((tcx.uses[0] + tcx.uses[1]) & 1);   // alternate the stages
        unsigned char* stg = tcx.st + sidx * STG;
        // the stage's previous MMAs must be complete before it is rewritten
        if (tcx.uses[sidx] > 0 && !*s_tcerr) {
          if (!tc::mbar_wait(tcx.bar + sidx, (tcx.uses[sidx] - 1) & 1, tcx.limit) && ct == 0) *s_tcerr = 1;
        }
        // A: (row r, 4-sample chunk c) pairs; B: (column r, chunk c) pairs
#pragma unroll
        for (int u = 0; u < kPPT; ++u) {
          const int e = ct + u * kCT;
          if (e < kTM * (kTK / 4)) {
            const int r = e % kTM, c = e / kTM;
            float4 h, l;
            h.x = tc::tf32_round(va[u][0]); h.y = tc::tf32_round(va[u][1]);
            h.z = tc::tf32_round(va[u][2]); h.w = tc::tf32_round(va[u][3]);
            l.x = tc::tf32_round(va[u][0] - h.x); l.y = tc::tf32_round(va[u][1] - h.y);
            l.z = tc::tf32_round(va[u][2] - h.z); l.w = tc::tf32_round(va[u][3] - h.w);
            const uint32_t off = tc::sw128_off(r, 4 * c);
            *reinterpret_cast<float4*>(stg + off) = h;
            if (kLoA) *reinterpret_cast<float4*>(stg + AH + off) = l;
          }
        }
        if (k + 1 < nch) load_chunk(k + 1, va);   // in flight through the B stores and the MMAs
        for (int e = ct; e < NT * (kTK / 4); e += kCT) {
          const int r = e % NT, c = e / NT;
          float v[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            const int jj = k * kTK + 4 * c + q;
            v[q] = jj < scn ? Zf[jj * ZP + r] : 0.f;
          }
          float4 h, l;
          h.x = tc::tf32_round(v[0]); h.y = tc::tf32_round(v[1]); h.z = tc::tf32_round(v[2]); h.w = tc::tf32_round(v[3]);
          l.x = tc::tf32_round(v[0] - h.x); l.y = tc::tf32_round(v[1] - h.y);
          l.z = tc::tf32_round(v[2] - h.z); l.w = tc::tf32_round(v[3] - h.w);
          const uint32_t off = tc::sw128_off(r, 4 * c);
          *reinterpret_cast<float4*>(stg + 2 * AH + off) = h;
          *reinterpret_cast<float4*>(stg + 2 * AH + BH + off) = l;
        }
        tc::fence_async_smem();
        named_sync(2, kCT);
        if (ct == 0 && !*s_tcerr) {
          tc::fence_after();
          const uint32_t ah = tc::saddr(stg), al = ah + AH, bh = ah + 2 * AH, bl = bh + BH;
#pragma unroll
          for (int kk = 0; kk < kTK / 8; ++kk) {
            const uint32_t o = kk * 32;
            tc::mma_tf32(tcx.tmem, tc::sw128_desc(ah + o), tc::sw128_desc(bh + o), idesc, (first && kk == 0) ? 0u : 1u);
            tc::mma_tf32(tcx.tmem, tc::sw128_desc(ah + o), tc::sw128_desc(bl + o), idesc, 1u);
            if (kLoA) tc::mma_tf32(tcx.tmem, tc::sw128_desc(al + o), tc::sw128_desc(bh + o), idesc, 1u);
          }
          tc::commit(tcx.bar + sidx);
        }
        tcx.uses[sidx] += 1;                       // (every contraction thread keeps the same count)
        first = false;
      }
    }
    // the unit's MMAs are complete when the last commit's phase is
    const int last = (int)((tcx.uses[0] + tcx.uses[1] + 1) & 1);
    bool drained = tc::mbar_wait(tcx.bar + last, (tcx.uses[last] - 1) & 1, tcx.limit);
    if (!drained && ct == 0) *s_tcerr = 1;
    tc::fence_after();
    // epilogue: warp w (4..15) reads TMEM lanes 32 (w % 4) .. + 31 (one row of the unit per lane), the
    // three warps of a lane quarter taking every third group of 16 columns
    {
      const int w = threadIdx.x >> 5;
      const int wq = w & 3, grp = (w - 4) >> 2;
      const int i = i0 + 32 * wq + (threadIdx.x & 31);
      float* dst = gs.Mpart + (int64_t)split * R * ms.I + i;
      for (int c0 = 16 * grp; c0 < NT && c0 < R; c0 += 48) {   // uniform in the warp
        float v[16];
        tc::tmem_ld16(tcx.tmem + ((uint32_t)(32 * wq) << 16) + (uint32_t)c0, v);
        if (i < ms.I) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (c0 + q < R) dst[(int64_t)(c0 + q) * ms.I] = v[q];
        }
      }
    }
    tc::fence_before();
    named_sync(2, kCT);                          // the accumulator is read before the next unit's MMAs
  }
}

// Prefetch into L2 the fiber segments the contraction units of the next mode update will read.
template <typename T>
__device__ void prefetch_next(const Prob& p, const GridCtx& x, int n, uint32_t t, const ModeSplit& ms, int tile_rows,
                              int ti, int nthr) {
  const T* X = reinterpret_cast<const T*>(p.Xrep[n]);
  if (!(p.use_rep || n == 0)) return;   // strided fibers: nothing contiguous to prefetch
  for (int u = x.c; u < ms.units; u += x.G) {
    const int tile = u % ms.ntile, split = u / ms.ntile;
    const int i0 = tile * tile_rows;
    const int rows = min(tile_rows, ms.I - i0);
    const int js = split * ms.spl;
    const int cnt = min(ms.spl, p.S - js);
    for (int jj = ti; jj < cnt; jj += nthr) {   // one draw per sample, then its row segment's lines
      uint32_t ids[kMaxOrder];
      const int64_t off = grid_draw(p, n, t, (uint32_t)(js + jj), ids);
      const uintptr_t end = reinterpret_cast<uintptr_t>(X + off + i0 + rows);
      for (uintptr_t a = reinterpret_cast<uintptr_t>(X + off + i0) & ~(uintptr_t)127; a < end; a += 128)
        prefetch_l2(reinterpret_cast<const void*>(a));
    }
  }
}

// X0 ~ Gs^-1 in FP32 for the Jacobi-scaled Gram Gs (unit diagonal) by the sweep operator: pivot k
// maps A to A' with A'_ij = A_ij - A_ik A_kj / A_kk (i, j != k), A'_ik = A_ik / A_kk,
// A'_kj = A_kj / A_kk, A'_kk = -1 / A_kk; after every pivot A = -Gs^-1.  The matrix lives in the
// registers of W warps (W = 1 for R <= 32, 2 for R <= 64): thread j (0 <= j < PAD = 32 W) holds column
// j, padded with zeros past R.  A stays symmetric, so row k is column k and each thread publishes its
// row-k entry to shared memory for the others (one barrier per pivot, two alternating slot sets).  The
// rows rotate by one position per pivot so that every register index is static: before pivot k,
// position p holds row (p + k) mod PAD, the pivot row is position 0, and the published entry of row i
// goes to slot (i - k - 1) mod PAD, which is where the update of the row's next position reads it.
// The column of the pivot itself takes A'_ik = A_ik - A_ik (1 - 1 / A_kk) from the same fused update
// (its own entries are the published ones).  A pivot below 1e-6 (relative to the unit diagonal) or
// not finite returns false in every thread.  src: Gs (R x R, FP32); dst: X0 (may be src: every read
// precedes the first barrier); piv: 2 PAD floats of scratch (16-byte aligned); src, dst and piv are
// shared-window addresses; bar_id: a block
// barrier for the PAD threads when W = 2; arrive_id: a block barrier of the whole CTA at which the
// PAD threads arrive once their columns are in registers.  Not inlined: the sweep's registers are
// then allocated apart from the rest of the kernel's live state (the caller saves that around the
// call), so the columns and the pivot row's loads stay in registers.
template <int W>
__device__ __noinline__ bool sweep_regs(uint32_t src, uint32_t dst, int R, uint32_t piv, int j, int bar_id,
                                        int arrive_id) {
  constexpr int PAD = 32 * W;
  float r[PAD];
#pragma unroll
  for (int p = 0; p < PAD; ++p) r[p] = (p < R && j < R) ? lds_f32(src + 4u * (p * R + j)) : 0.f;
  named_arrive(arrive_id, kGT);
  bool bad = false;
  for (int k = 0; k < R; ++k) {
    const uint32_t pv = piv + 4u * (k & 1) * PAD;
    sts_f32(pv + 4u * ((j - k - 1) & (PAD - 1)), r[0]);
    if (W == 1) __syncwarp();
    else named_sync(bar_id, PAD);
    const float d = lds_f32(pv + 4u * (PAD - 1));   // row k's entry of column k
    bad = bad || !(d > 1e-6f) || !isfinite(d);
    const float inv = __frcp_rn(d);
    const float akj = r[0];
    const float c = j == k ? 1.f - inv : akj * inv;
#pragma unroll
    for (int p = 0; p < PAD; p += 4) {
      const float4 q = lds_v4f32(pv + 4u * p);
      r[p] = fmaf(-q.x, c, r[p + 1]);
      r[p + 1] = fmaf(-q.y, c, r[p + 2]);
      r[p + 2] = fmaf(-q.z, c, r[p + 3]);
      if (p + 4 < PAD) r[p + 3] = fmaf(-q.w, c, r[p + 4]);
    }
    r[PAD - 1] = j == k ? -inv : akj * inv;   // the new pivot row, now at the last position
  }
  if (W == 1) __syncwarp();
  else named_sync(bar_id, PAD);
  if (j < R) {
#pragma unroll
    for (int p = 0; p < PAD; ++p) {
      const int row = (p + R) & (PAD - 1);
      if (row < R) sts_f32(dst + 4u * (row * R + j), -r[p]);
    }
  }
  return !bad;
}

// ---- after the Gram is reduced, by the NT threads of block barrier bar_id: G = Sc G' Sc as pairs in
// g2 (R x R; G' the reduced Gram of the unscaled rows, Sc the lazy column scales of the other modes),
// the Jacobi-scaled FP32 copy Gs = D' G' D' (D' = diag(1 / sqrt(G'_rr)), unit diagonal) in x0, and
// the scales of the row solve ds_r = D'_rr / Sc_rr, so that G^-1 ~ Ds X0 Ds for X0 ~ Gs^-1
// (they only precondition the refinement, whose residual uses G itself).  Returns whether every
// diagonal entry is positive and finite (identical in every CTA): else the FP32 start is skipped.
template <int MAXR, int NT>
__device__ bool solver_prepare(const Prob& p, const GridSmem& L, unsigned char* sm, const GridScratch& gs, float* ds,
                               const float2* scp, const unsigned char* ne_r, const unsigned char* ne_c, int bar_id) {
  const int tid = threadIdx.x, R = p.R, RR = R * R;
  const int NE = R * (R + 1) / 2;
  float2* g2 = reinterpret_cast<float2*>(sm + L.g2);
  float* sw = reinterpret_cast<float*>(sm + L.x0);
  float* dp = reinterpret_cast<float*>(sm + L.dp);
  constexpr int GPT = (MAXR * (MAXR + 1) / 2 + NT - 1) / NT;
  float2 gv[GPT];
#pragma unroll
  for (int q = 0; q < GPT; ++q) {       // every load in flight before the stores
    const int e = tid + q * NT;
    gv[q] = e < NE ? __ldcg(gs.Gfull + e) : make_float2(0.f, 0.f);
  }
#pragma unroll
  for (int q = 0; q < GPT; ++q) {
    const int e = tid + q * NT;
    if (e < NE) {
      const int r = ne_r[e], cc = ne_c[e];
      g2[r * R + cc] = gv[q];
      g2[cc * R + r] = gv[q];
    }
  }
  named_sync(bar_id, NT);
  bool good = true;
  for (int r = tid; r < R; r += NT) {
    const float d = g2[r * R + r].x;
    const bool ok = d > 0.f && isfinite(d);
    good = good && ok;
    const float y = ok ? rsqrtf(d) : 0.f;
    dp[r] = y;
    ds[r] = y / scp[r].x;
  }
  const bool fast = named_and(bar_id, NT, good);   // the same in every thread
  for (int e = tid; e < RR; e += NT) {
    const int r = e / R, cc = e - r * R;
    const float2 g = g2[e];
    sw[e] = g.x * dp[r] * dp[cc];
    g2[e] = pair_mul(pair_mul(g, scp[r]), scp[cc]);
  }
  named_sync(bar_id, NT);
  return fast;
}

// ---- all threads, after the contraction: this CTA's rows of A^(n) = M G^-1 (Alg. 3 least-squares
// step through the normal equations) from mrow (M rows as pairs) into a2 (pairs).  fast: the FP32
// inverse is usable: A0 = ((M Ds) X0) Ds, then refinement steps A += (M - A G) Ds X0 Ds with the
// residual summed in pairs; else the FP64 Cholesky inverse, which also decides singularity.  Returns
// false if the Gram is singular.
template <int MAXR>
__device__ bool solve_rows(const Prob& p, const GridSmem& L, unsigned char* sm, const GridCtx& x,
                           const ModeSplit& ms, const float* ds, bool fast, int* s_flag, unsigned* s_umax) {
  const int tid = threadIdx.x, R = p.R, RR = R * R;
  const float2* g2 = reinterpret_cast<const float2*>(sm + L.g2);
  const float2* mrow = reinterpret_cast<const float2*>(sm + L.mrow);
  float2* a2 = reinterpret_cast<float2*>(sm + L.a2);
  float* m32 = reinterpret_cast<float*>(sm + L.m32);
  const float* X0 = reinterpret_cast<const float*>(sm + L.x0);   // X0(r, c), scaled: G^-1 ~ Ds X0 Ds
  const int i0 = x.c * ms.rpc;
  const int nrows = max(0, min(ms.I, i0 + ms.rpc) - i0);
  const int NO = nrows * R;
  if (!fast) {
    // G in FP64, its FP64 Cholesky inverse (also the singularity test) over the pairs of G (read out
    // first), then A = M G^-1 in FP64
    double* G = reinterpret_cast<double*>(sm + L.G);
    for (int e = tid; e < RR; e += kGT) G[e] = pair_value(g2[e]);
    double* X = reinterpret_cast<double*>(sm + L.g2);
    if (tid == 0) *s_flag = 0;
    __syncthreads();
    spd_inverse_fp64(G, X, reinterpret_cast<double*>(sm + L.fL), reinterpret_cast<double*>(sm + L.fT),
                     reinterpret_cast<double*>(sm + L.fd), R, s_flag);
    __syncthreads();
    const bool singular = *s_flag != 0;
    double* arow = reinterpret_cast<double*>(sm + L.arow);
    for (int e = tid; e < NO; e += kGT) {
      const int li = e / R, cc = e - li * R;
      const float2* m = mrow + li * R;
      double a0 = 0.0;
      for (int l = 0; l < R; ++l) a0 = fma(pair_value(m[l]), X[l * R + cc], a0);
      arow[e] = a0;
    }
    __syncthreads();
    for (int e = tid; e < NO; e += kGT) a2[e] = split_pair(arow[e]);
    __syncthreads();
    return !singular;
  }
  // A0 = ((M Ds) X0) Ds in FP32
  for (int e = tid; e < NO; e += kGT) m32[e] = mrow[e].x * ds[e % R];
  __syncthreads();
  for (int e = tid; e < NO; e += kGT) {
    const int li = e / R, cc = e - li * R;
    const float* m = m32 + li * R;
    float a0 = 0.f, a1 = 0.f;
    int l = 0;
    for (; l + 1 < R; l += 2) {
      a0 = fmaf(m[l], X0[l * R + cc], a0);
      a1 = fmaf(m[l + 1], X0[(l + 1) * R + cc], a1);
    }
    if (l < R) a0 = fmaf(m[l], X0[l * R + cc], a0);
    a2[e] = make_float2((a0 + a1) * ds[cc], 0.f);
  }
  __syncthreads();
  // refinement: the residual M - A G summed in pairs from -M (to about 2^-44 of its terms), the
  // correction through the FP32 inverse, added to A as a pair
  for (int it = 0; it < 3; ++it) {
    if (tid == 0) s_umax[0] = s_umax[1] = 0u;
    for (int e = tid; e < NO; e += kGT) {
      const int li = e / R, cc = e - li * R;
      const float2* a = a2 + li * R;
      float sh = -mrow[e].x, sl = -mrow[e].y;
      for (int l = 0; l < R; ++l) pair_fma(a[l], g2[l * R + cc], sh, sl);
      m32[e] = -__fadd_rn(sh, sl) * ds[cc];
    }
    __syncthreads();
    float cm = 0.f, am = 0.f;
    for (int e = tid; e < NO; e += kGT) {
      const int li = e / R, cc = e - li * R;
      const float* m = m32 + li * R;
      float a0 = 0.f, a1 = 0.f;
      int l = 0;
      for (; l + 1 < R; l += 2) {
        a0 = fmaf(m[l], X0[l * R + cc], a0);
        a1 = fmaf(m[l + 1], X0[(l + 1) * R + cc], a1);
      }
      if (l < R) a0 = fmaf(m[l], X0[l * R + cc], a0);
      const float corr = (a0 + a1) * ds[cc];
      float2 a = a2[e];
      pair_acc(corr, a.x, a.y);
      a = pair_norm(a.x, a.y);
      a2[e] = a;
      cm = fmaxf(cm, fabsf(corr));
      am = fmaxf(am, fabsf(a.x));
    }
    cm = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(cm)));
    am = __uint_as_float(__reduce_max_sync(0xffffffffu, __float_as_uint(am)));
    if ((tid & 31) == 0) {
      atomicMax(s_umax, __float_as_uint(cm));
      atomicMax(s_umax + 1, __float_as_uint(am));
    }
    __syncthreads();
    // the error left after a correction of relative size c is about c^2 (the FP32 inverse's error
    // shrinks it by the same factor it shrank the previous one): stop once c < 1e-5
    const bool done = !(__uint_as_float(s_umax[0]) > 1e-5f * __uint_as_float(s_umax[1]));
    __syncthreads();
    if (done) break;
  }
  return true;
}

template <typename T, int MAXR>
__global__ void __launch_bounds__(kGT, 1) k_grid_run(const Prob* probs, int B, GridScratch gs) {
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ Prob P;
  __shared__ double sc[kMaxOrder * kMaxRank];
  __shared__ double lam[kMaxRank];
  __shared__ float ds[kMaxRank];
  __shared__ float2 scp[kMaxRank];
  __shared__ float scf[kMaxRank], wrf[kMaxRank];
  __shared__ double red[kGW];
  __shared__ double red64[kMaxRank], redp[kGT];
  float2* red2 = reinterpret_cast<float2*>(red64);   // the pair-valued sums reuse them
  float2* redp2 = reinterpret_cast<float2*>(redp);
  __shared__ unsigned char ne_r[kNEMax], ne_c[kNEMax];
  __shared__ int s_flag, s_flag2, s_done, s_status, s_iter, s_stall, s_fast, s_abort, s_invbad, s_gfast;
  __shared__ unsigned s_umax[2];
  __shared__ double s_best, s_last;
  __shared__ __align__(8) uint64_t tc_bar[2];
  __shared__ uint32_t tc_slot;
  __shared__ volatile int s_tcerr;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  GridCtx x;
  x.gen = 0u;
  x.G = (int)gridDim.x;
  x.c = (int)blockIdx.x;
  // the tensor-core contraction: two stage mbarriers and a TMEM accumulator of 128 lanes x MAXR
  // columns (allocated by warp 4, freed by it when the kernel ends)
  const bool use_tc = gs.use_tc != 0;
  constexpr uint32_t kTmemCols = MAXR <= 32 ? 32u : 64u;
  TcCtx tcx;
  tcx.uses[0] = tcx.uses[1] = 0u;
  tcx.limit = gs.wait_limit;
  if (use_tc) {
    if (tid == 0) {
      tc::mbar_init(&tc_bar[0], 1);
      tc::mbar_init(&tc_bar[1], 1);
      s_tcerr = 0;
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    if (warp == 4) tc::tmem_alloc(&tc_slot, kTmemCols);
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    tcx.bar = tc_bar;
    tcx.tmem = tc_slot;
  }
  bool quit = false;
  for (int b = 0; b < B && !quit; ++b) {
    {
      const int words = (int)(sizeof(Prob) / 4);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(probs + b);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&P);
      for (int w = tid; w < words; w += kGT) dst[w] = src[w];
    }
    __syncthreads();
    const Prob& p = P;
    const int R = p.R, N = p.N;
    const GridSmem L = grid_layout(R, MAXR, (int)sizeof(T));
    tcx.st = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(sm + L.stage) + 1023) & ~(uintptr_t)1023);
    State* st = p.state;
    if (tid == 0) {
      int e = 0;
      for (int r = 0; r < R; ++r)
        for (int cc = r; cc < R; ++cc, ++e) {
          ne_r[e] = (unsigned char)r;
          ne_c[e] = (unsigned char)cc;
        }
      s_done = st->done;
      s_status = st->status;
      s_iter = st->iter;
      s_stall = st->stall;
      s_best = st->best;
      s_last = st->last_fit;
    }
    if (tid == 0) {
      s_fast = 0;
      s_abort = 0;
      s_invbad = 0;
      s_gfast = 0;
    }
    for (int e = tid; e < N * R; e += kGT) sc[e] = p.scale[e / R][e % R];
    for (int r = tid; r < R; r += kGT) lam[r] = p.lambda[r];
    __syncthreads();
    const double inv_norm = 1.0 / st->norm_x;
    const double fit_scale = (double)p.P / (double)p.P_hat;
    const int cap = p.fixed_iters > 0 ? p.fixed_iters : p.max_iters;
    bool alive = true;
    while (alive && !s_done && s_iter < cap) {
      const uint32_t t = p.t0 + (uint32_t)s_iter;
      bool singular = false;
      for (int n = 0; n < N; ++n) {
        const ModeSplit ms = mode_split(p, n, x.G, use_tc ? kTM : kTI);
        // combined lazy scale of the other modes
        for (int r = tid; r < R; r += kGT) {
          double cmb = 1.0;
          for (int m = 0; m < N; ++m)
            if (m != n) cmb *= sc[m * R + r];
          scp[r] = split_pair(cmb);
          scf[r] = (float)cmb;
        }
        __syncthreads();
        // ---- P1: warps 0-3 Gram partial, grid barrier among themselves (A), their slice of the
        // reduced Gram, grid barrier (B); meanwhile warps 4-15 contract
        if (tid < kGramT) {
          gram_partial<MAXR>(p, L, sm, gs, x, n, t, ne_r, ne_c);
          bool gok = grid_sync(gs, x, &s_flag, 1, kGramT);
          if (gok) {
            const int NE = R * (R + 1) / 2;
            const int epc = (NE + x.G - 1) / x.G;      // at most 64 (NE <= 2080, G >= 33 on this path)
            const int e0 = x.c * epc;
            const int ne = max(0, min(NE, e0 + epc) - e0);
            if (ne > 0) {
              sum_pairs(gs.Gpart + e0, x.G, ne, NE, red2, redp2, 1, kGramT);
              for (int e = tid; e < ne; e += kGramT) gs.Gfull[e0 + e] = red2[e];
            }
            gok = grid_sync(gs, x, &s_flag, 1, kGramT);
          }
          if (!gok && tid == 0) s_abort = 1;
        } else {
          if (use_tc) {
            contract_units_tc<T, MAXR>(p, L, sm, gs, x, n, t, ms, scf, tcx, &s_tcerr);
            if (s_tcerr && threadIdx.x == kGramT) atomicExch(gs.err, 1);   // every CTA stops at a barrier
          } else {
            contract_units<T, MAXR>(p, L, sm, gs, x, n, t, ms, scf);
          }
        }
        __syncthreads();
        if (s_abort) {
          alive = false;
          break;
        }
        // G and its scaled FP32 copy by every warp; then the FP32 inverse X0 by W warps from warp 2 on (a
        // chain of pivots on their registers) while the other warps pass grid barrier C and reduce
        // this CTA's rows of M.  The M loads start once the sweep's columns are in registers (block
        // barrier 5): shared loads issued after them queue behind the partials' L2 loads.
        const bool gfast = solver_prepare<MAXR, kGT>(p, L, sm, gs, ds, scp, ne_r, ne_c, 0);
        const int W = (MAXR > 32 && R > 32) ? 2 : 1;
        const int nrest = kGT - 32 * W;
        const bool sweeper = tid >= 64 && tid < 64 + 32 * W;   // warps 2 (and 3)
        const int rt = tid < 64 ? tid : tid - 32 * W;          // index among the other threads
        if (sweeper) {
          if (gfast) {
            const uint32_t x0 = (uint32_t)__cvta_generic_to_shared(sm + L.x0);
            const uint32_t piv = (uint32_t)__cvta_generic_to_shared(sm + L.piv);
            bool iok;
            if constexpr (MAXR > 32) {
              iok = W == 2 ? sweep_regs<2>(x0, x0, R, piv, tid - 64, 3, 5)
                           : sweep_regs<1>(x0, x0, R, piv, tid - 64, 3, 5);
            } else {
              iok = sweep_regs<1>(x0, x0, R, piv, tid - 64, 3, 5);
            }
            if (tid == 64) s_invbad = iok ? 0 : 1;
          } else {
            named_arrive(5, kGT);
          }
        } else {
          const bool cok = grid_sync(gs, x, &s_flag, 4, nrest);   // (C) every split's partial M is stored
          named_sync(5, kGT);
          if (cok) {
            // ---- P3: the split partials of this CTA's rows, summed exactly into pairs
            float2* mrow = reinterpret_cast<float2*>(sm + L.mrow);
            const int i0 = x.c * ms.rpc;
            const int nrows = max(0, min(ms.I, i0 + ms.rpc) - i0);
            for (int e = rt; e < nrows * R; e += nrest) {   // rows fastest: a column's rows are adjacent in Mpart
              const int r = nrows > 0 ? e / nrows : 0, li = e - r * nrows;
              const float* src = gs.Mpart + (int64_t)r * ms.I + i0 + li;
              const int64_t sstr = (int64_t)R * ms.I;
              float h0 = 0.f, l0 = 0.f, h1 = 0.f, l1 = 0.f;
              int q = 0;
              for (; q + 7 < ms.nsplit; q += 8) {   // eight loads in flight
                float v[8];
#pragma unroll
                for (int k = 0; k < 8; ++k) v[k] = __ldcg(src + (q + k) * sstr);
#pragma unroll
                for (int k = 0; k < 8; k += 2) {
                  pair_acc(v[k], h0, l0);
                  pair_acc(v[k + 1], h1, l1);
                }
              }
              for (; q < ms.nsplit; ++q) pair_acc(__ldcg(src + q * sstr), h0, l0);
              pair_acc2(make_float2(h1, l1), h0, l0);
              mrow[li * R + r] = pair_norm(h0, l0);
            }
            // the next update's sampled fibers into L2, while warps 2-3 finish the inverse
            const int nn = n + 1 < N ? n + 1 : 0;
            const uint32_t nt = n + 1 < N ? t : t + 1;
            prefetch_next<T>(p, x, nn, nt, mode_split(p, nn, x.G, use_tc ? kTM : kTI), use_tc ? kTM : kTI, rt, nrest);
          }
        }
        __syncthreads();
        if (!(alive = s_flag != 0)) break;
        const bool fast = gfast && s_invbad == 0;   // the same in every CTA
        // ---- then A = M G^-1
        const bool ok = solve_rows<MAXR>(p, L, sm, x, ms, ds, fast, &s_flag2, s_umax);
        {
          const float2* a2 = reinterpret_cast<const float2*>(sm + L.a2);
          const int i0 = x.c * ms.rpc;
          const int nrows = max(0, min(ms.I, i0 + ms.rpc) - i0);
          double* A64 = p.A64[n] + (int64_t)i0 * R;
          float* A32 = p.A32[n] + (int64_t)i0 * R;
          for (int e = tid; e < nrows * R; e += kGT) {
            const float2 a = a2[e];
            A64[e] = pair_value(a);
            A32[e] = a.x;
          }
          for (int r = tid; r < R; r += kGT) {   // this CTA's part of the column sums of squares
            float sh = 0.f, sl = 0.f;
            for (int li = 0; li < nrows; ++li) pair_fma(a2[li * R + r], a2[li * R + r], sh, sl);
            gs.Npart[(int64_t)x.c * R + r] = pair_norm(sh, sl);
          }
        }
        if (!ok) singular = true;   // identical in every CTA (same G, same arithmetic)
        if (!(alive = grid_sync(gs, x, &s_flag))) break;   // (D) every row and column partial stored
        if (singular) break;
        // ---- P4: lambda and the lazy scales of mode n
        sum_pairs(gs.Npart, x.G, R, R, red2, redp2);
        for (int r = tid; r < R; r += kGT) {
          const double a = pair_value(red2[r]);
          const double y = a > 0.0 ? rsqrt64(a) : 0.0;
          const double nrm = a * y;
          lam[r] = nrm;
          sc[n * R + r] = nrm > 0.0 ? y : 1.0;
        }
        __syncthreads();
      }
      if (!alive) break;
      if (singular) {
        if (tid == 0) {
          s_status = CPR_ESINGULAR;
          s_done = 1;
        }
        __syncthreads();
        break;
      }
      // ---- sampled fit (Sec. 3.4) over the CTA's share of the fixed entries
      for (int r = tid; r < R; r += kGT) {
        double w = lam[r];
        for (int m = 0; m < N; ++m) w *= sc[m * R + r];
        wrf[r] = (float)w;
      }
      __syncthreads();
      {
        const int fpc = (p.P_hat + x.G - 1) / x.G;
        const int f0 = x.c * fpc;
        const int f1 = min(p.P_hat, f0 + fpc);
        double e2 = 0.0;
        // the CTA's fit entries staged in shared memory (the P1 region is free here) in chunks; four
        // entries per warp at a time, their factor-row loads issued together
        uint32_t* fids = reinterpret_cast<uint32_t*>(sm + L.Zf);
        double* fxs = reinterpret_cast<double*>(sm + L.cids);
        const int fchunk = kSC;              // entries per chunk (ids: kSC * N <= kSC * MAXR words)
        for (int c0 = f0; c0 < f1; c0 += fchunk) {
          const int cn = min(fchunk, f1 - c0);
          for (int e = tid; e < cn * N; e += kGT) fids[e] = p.fit_idx[(int64_t)c0 * N + e];
          for (int e = tid; e < cn; e += kGT) fxs[e] = p.fit_x[c0 + e];
          __syncthreads();
          for (int j0 = 4 * warp; j0 < cn; j0 += 4 * kGW) {
            float v[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
            for (int h = 0; h < 2; ++h) {          // R <= 64: two columns per lane
              const int r = lane + 32 * h;
              if (r < R) {
                float tt[4];
#pragma unroll
                for (int u = 0; u < 4; ++u) tt[u] = wrf[r];
                for (int m = 0; m < N; ++m) {
                  const float* Am = p.A32[m];
                  float a[4];
#pragma unroll
                  for (int u = 0; u < 4; ++u)
                    a[u] = j0 + u < cn ? __ldcg(Am + (int64_t)fids[(j0 + u) * N + m] * R + r) : 0.f;
#pragma unroll
                  for (int u = 0; u < 4; ++u) tt[u] *= a[u];
                }
#pragma unroll
                for (int u = 0; u < 4; ++u) v[u] += tt[u];
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              for (int o = 16; o > 0; o >>= 1) v[u] += __shfl_xor_sync(0xffffffffu, v[u], o);
              if (j0 + u < cn) {
                const double e = fxs[j0 + u] - (double)v[u];
                e2 = fma(e, e, e2);
              }
            }
          }
          __syncthreads();
        }
        if (lane == 0) red[warp] = e2;
        __syncthreads();
        if (tid == 0) {
          double a = 0.0;
          for (int q = 0; q < kGW; ++q) a += red[q];
          gs.fitpart[x.c] = a;
        }
      }
      if (!(alive = grid_sync(gs, x, &s_flag))) break;
      sum_rows(gs.fitpart, x.G, 1, 1, red64, redp);
      if (warp == 0) {
        const double a = red64[0];
        if (lane == 0) {
          const double v = fit_scale * a;
          const double fit = v > 0.0 ? 1.0 - v * rsqrt64(v) * inv_norm : (v == 0.0 ? 1.0 : NAN);
          const int t1 = s_iter + 1;
          bool stop = false;
          if (!isfinite(fit)) {
            s_status = CPR_ENONFINITE;
            stop = true;
          } else if (p.fixed_iters > 0) {
            stop = t1 >= p.fixed_iters;
          } else {
            if (fit > s_best) {
              s_best = fit;
              s_stall = 0;
            } else {
              s_stall += 1;
            }
            if (t1 >= p.max_iters) stop = true;
            if (t1 >= 2 && fabs(fit - s_last) <= p.tol) stop = true;
            if (p.eta >= 0.0 && fit >= 1.0 - 1.2 * p.eta) stop = true;
            if (p.stall_iters > 0 && s_stall >= p.stall_iters) stop = true;
          }
          if (x.c == 0 && p.trace) p.trace[s_iter] = fit;
          s_last = fit;
          s_iter = t1;
          if (stop) s_done = 1;
        }
      }
      __syncthreads();
    }
    if (!alive) {         // a barrier wait ran out (the error flag is set); no copy or MMA is in flight
      quit = true;
      break;
    }
    // publish the loop state, lambda and the lazy scales (CTA 0)
    if (x.c == 0) {
      for (int e = tid; e < N * R; e += kGT) p.scale[e / R][e % R] = sc[e];
      for (int r = tid; r < R; r += kGT) p.lambda[r] = lam[r];
      if (tid == 0) {
        st->done = 1;
        st->status = s_status;
        st->iter = s_iter;
        st->stall = s_stall;
        st->best = s_best;
        st->last_fit = s_last;
      }
    }
    // the next problem reuses the scratch: every CTA leaves this one first
    if (!grid_sync(gs, x, &s_flag)) quit = true;
  }
  if (use_tc) {
    // every MMA has completed (each unit waited for its last commit); after a wait that ran out, wait
    // again (bounded) for the last phase of each stage before the accumulator is freed
    if (s_tcerr && warp >= 4) {
      for (int sidx = 0; sidx < 2; ++sidx)
        if (tcx.uses[sidx] > 0) tc::mbar_wait(&tc_bar[sidx], (tcx.uses[sidx] - 1) & 1, 1u << 26);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
    if (warp == 4) tc::tmem_free(tcx.tmem, kTmemCols);
  }
}

template <typename T, int MAXR>
cudaError_t grid_launch(const Prob* probs, int B, const GridScratch& gs, int G, cudaStream_t s, int query,
                        int* capacity, int maxR) {
  auto kern = k_grid_run<T, MAXR>;
  const GridSmem L = grid_layout(maxR, MAXR, (int)sizeof(T));
  const int smem = L.bytes;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (query) {
    int per_sm = 0, dev = 0, sms = 0;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kGT, smem)) != cudaSuccess) return e;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    *capacity = per_sm >= 1 ? sms : 0;
    return cudaSuccess;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)G, 1, 1);
  cfg.blockDim = dim3(kGT, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, probs, B, gs);
}

template <typename T>
cudaError_t grid_dispatch_r(int maxR, const Prob* probs, int B, const GridScratch& gs, int G, cudaStream_t s,
                            int query, int* cap) {
  if (maxR <= 16) return grid_launch<T, 16>(probs, B, gs, G, s, query, cap, maxR);
  if (maxR <= 32) return grid_launch<T, 32>(probs, B, gs, G, s, query, cap, maxR);
  if (maxR <= 48) return grid_launch<T, 48>(probs, B, gs, G, s, query, cap, maxR);
  return grid_launch<T, 64>(probs, B, gs, G, s, query, cap, maxR);
}

}  // namespace

// CTAs of the grid loop on this device (one per SM), or 0 if it cannot be launched for this dtype
// and rank.
int grid_capacity(int dtype, int maxR) {
  int cap = 0;
  cudaError_t e = cudaSuccess;
  if (dtype == CPR_F32) e = grid_dispatch_r<float>(maxR, nullptr, 0, GridScratch{}, 0, nullptr, 1, &cap);
  else if (dtype == CPR_BF16) e = grid_dispatch_r<__nv_bfloat16>(maxR, nullptr, 0, GridScratch{}, 0, nullptr, 1, &cap);
  else return 0;
  if (e != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return cap > kGridMaxCTAs ? kGridMaxCTAs : cap;
}

// Whether a problem fits the grid loop's fixed limits (every mode's factor rows per CTA).
bool grid_fits(const Prob& p, int G) {
  if (p.dtype == CPR_F64 || p.R > kMaxRank || G < 33) return false;   // G >= 33: a CTA's Gram slice <= 64
  for (int n = 0; n < p.N; ++n)
    if ((p.dims[n] + G - 1) / G > kGridMaxRows) return false;
  return true;
}

cudaError_t launch_grid_run(const Prob* probs, int B, const GridScratch& gs, int dtype, int maxR, int G,
                            cudaStream_t s) {
  if (dtype == CPR_F32) return grid_dispatch_r<float>(maxR, probs, B, gs, G, s, 0, nullptr);
  return grid_dispatch_r<__nv_bfloat16>(maxR, probs, B, gs, G, s, 0, nullptr);
}

}  // namespace cpr
