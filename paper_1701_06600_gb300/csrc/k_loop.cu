// The whole outer-iteration loop of CPRAND (Alg. 3, with the sampled fit of Sec. 3.4 and the
// stopping rules of Sec. 4.2) in one 16-CTA thread-block cluster per problem, with every factor
// matrix replicated in each CTA's shared memory.
//
// Work split: CTA c draws samples [c*spc, (c+1)*spc) of every mode update and owns factor rows
// [c*rpc_n, (c+1)*rpc_n) of mode n.  Per mode update:
//   1. SKR (Alg. 2): the Z_S rows of this CTA's samples from the local factor copies times the
//      combined lazy column scale of the other modes (FP64; an FP32/FP64 copy feeds step 2).
//   2. Contraction M_c = X_S,c Z_S,c for every row i_n (FP32 accumulation, FP64 for FP64 tensors)
//      from the sampled fibers, which were copied into shared memory during the previous mode update
//      (one TMA bulk copy per contiguous fiber, cp.async otherwise): a mode update's sample draw
//      does not depend on the factors, so its fiber reads are issued one update ahead and never wait
//      on HBM in the dependent chain.  Each row's
//      partial is stored straight into the shared memory of the CTA owning that row.
//   3. Partial FP64 Gram of this CTA's Z rows, stored into every CTA's shared memory.
//   4. Cluster barrier (the next update's samples are drawn and its fiber copies issued between
//      the barrier's arrive and wait); every CTA sums the C partial Grams in one fixed order
//      (identical G everywhere) and inverts it: Gauss-Jordan elimination in FP32 with one thread
//      per entry of [G | I], then Newton-Schulz steps X <- X + X (I - G X) (one for FP32 tensors,
//      two for FP64) with the residual I - G X in FP64 and the small correction X (I - G X) in
//      FP32, each squaring the residual ||I - G X||; a residual above 1/4 or a
//      bad FP32 pivot falls back to an FP64 Cholesky inverse (which detects a singular Gram).
//   5. The CTA's rows: M rows summed over the C partials (fixed order), A = M G^-1 in FP64, written
//      to the FP64 result and stored into every CTA's copy of the factor; column sums of squares
//      of the rows are stored into every CTA.
//   6. Cluster barrier; lambda and the lazy column scales from the C column partials (fixed order).
// After the N modes each CTA evaluates its share of the P_hat fixed fit entries (indices and values
// staged in shared memory once per problem) against the local factor copies; after a cluster
// barrier every CTA sums the C partials in the same order and applies the stopping rules to its own
// copy of the loop state, so all CTAs take the same decision.
//
// Data only moves by stores into other CTAs' shared memory followed by a cluster barrier (release /
// acquire); no CTA reads another CTA's shared memory.  FP64 arithmetic issues at a low rate on this
// GPU (a warp's DFMA occupies an SM sub-partition's FP64 pipe for about 76 cycles), so FP64 work is
// packed into few warps spread over the four sub-partitions, and reductions never run redundantly
// in every warp.  Factor copies and Z rows are stored with rows padded to 16 bytes so that they
// move as vectors.
#include <cooperative_groups.h>
#include <math.h>

#include "internal.cuh"
#include "small_spd.cuh"

namespace cg = cooperative_groups;

namespace cpr {

namespace {

constexpr int kLT = 512;   // threads per CTA
constexpr int kLC = 16;    // CTAs per cluster

struct LoopSmem {          // byte offsets into the dynamic shared memory
  int F[kMaxOrder];        // full factor m, I_m x rp (ACC)
  int fib[2];              // sampled fibers of a mode update: spc rows of ldf elements (T)
  int ids[2];              // spc x kMaxOrder sampled indices
  int offs[2];             // spc fiber offsets
  int Zd, Zf;              // spc x R Z_S rows (FP64) and spc x rp (ACC)
  int Mrecv;               // C x R x rpcmax partial M columns received for this CTA's rows (ACC)
  int Grecv;               // C x NE partial Grams (packed upper triangle, FP64)
  int colrecv;             // C x R column sums of squares
  int fitrecv;             // C partial fit sums
  int fidx, fx;            // fpc x N fit indices, fpc fit values (ACC)
  int G, X, U, E, T2;      // R x R FP64
  int Gf;                  // R x R FP32 copy of G
  int gj;                  // 2 x R x 2R FP32: the Gauss-Jordan tableau, alternating by step
  int mrow, arow;          // rpcmax x R FP64
  int cpart;               // R x nchmax FP64
  int sc, lam, wr, dinv;   // N x R, R, rp (fit weights, ACC), R FP64
  int scomb;               // R: product of the other modes' lazy scales for the coming mode update
  int red;                 // kLT FP64 (block reduction)
  int bytes;
  int ldf, spc, rpcmax, fpc, NE, nchmax, rp;
};

__host__ __device__ inline int al16(int x) { return (x + 15) / 16 * 16; }

__host__ __device__ inline LoopSmem loop_layout(int N, int R, const int64_t* dims, int S, int P_hat, int tbytes,
                                                int abytes) {
  LoopSmem L;
  int o = 0, maxI = 0;
  L.rpcmax = 0;
  L.rp = (R * abytes + 15) / 16 * 16 / abytes;
  for (int m = 0; m < kMaxOrder; ++m) L.F[m] = 0;
  for (int m = 0; m < N; ++m) {
    const int I = (int)dims[m];
    maxI = I > maxI ? I : maxI;
    const int rpc = (I + kLC - 1) / kLC;
    L.rpcmax = rpc > L.rpcmax ? rpc : L.rpcmax;
    L.F[m] = o;
    o = al16(o + I * L.rp * abytes);
  }
  L.spc = (S + kLC - 1) / kLC;
  L.ldf = al16(maxI * tbytes) / tbytes;
  L.NE = R * (R + 1) / 2;
  L.fpc = (P_hat + kLC - 1) / kLC;
  L.nchmax = (L.rpcmax + 7) / 8;
  for (int q = 0; q < 2; ++q) {
    L.fib[q] = o;  o = al16(o + L.spc * L.ldf * tbytes);
  }
  for (int q = 0; q < 2; ++q) {
    L.ids[q] = o;  o = al16(o + L.spc * kMaxOrder * 4);
    L.offs[q] = o; o = al16(o + L.spc * 8);
  }
  L.Zd = o;      o = al16(o + L.spc * R * 8);
  L.Zf = o;      o = al16(o + L.spc * L.rp * abytes);
  L.Mrecv = o;   o = al16(o + kLC * L.rpcmax * R * abytes);
  L.Grecv = o;   o = al16(o + kLC * L.NE * 8);
  L.colrecv = o; o = al16(o + kLC * R * 8);
  L.fitrecv = o; o = al16(o + kLC * 8);
  L.fidx = o;    o = al16(o + L.fpc * N * 4);
  L.fx = o;      o = al16(o + L.fpc * abytes);
  L.G = o;       o = al16(o + R * R * 8);
  L.X = o;       o = al16(o + R * R * 8);
  L.U = o;       o = al16(o + R * R * 8);
  L.E = o;       o = al16(o + R * R * 8);
  L.T2 = o;      o = al16(o + R * R * 8);
  L.Gf = o;      o = al16(o + R * R * 4);
  L.gj = o;      o = al16(o + 2 * R * 2 * R * 4);
  L.mrow = o;    o = al16(o + L.rpcmax * R * 8);
  L.arow = o;    o = al16(o + L.rpcmax * R * 8);
  L.cpart = o;   o = al16(o + R * L.nchmax * 8);
  L.sc = o;      o = al16(o + N * R * 8);
  L.lam = o;     o = al16(o + R * 8);
  L.wr = o;      o = al16(o + L.rp * 8);
  L.dinv = o;    o = al16(o + R * 8);
  L.scomb = o;   o = al16(o + R * 8);
  L.red = o;     o = al16(o + kLT * 8);
  L.bytes = o;
  return L;
}

__device__ __forceinline__ uint32_t s32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

template <int B>
__device__ __forceinline__ void cp_async(void* dst, const void* src) {
  if constexpr (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(s32(dst)), "l"(src) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;" ::"r"(s32(dst)), "l"(src), "n"(B) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
__device__ __forceinline__ void cp_async_wait_all() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }

__device__ __forceinline__ void mbar_init(uint64_t* b) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(s32(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(s32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(s32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on a phase of an mbarrier: false if it did not complete within the limit.
__device__ __forceinline__ bool mbar_wait_bounded(uint64_t* b, uint32_t parity) {
  for (uint32_t it = 0; it < (1u << 24); ++it)
    if (mbar_try(b, parity)) return true;
  return false;
}
// One TMA bulk copy global -> this CTA's shared memory, completing bytes on the mbarrier.
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, uint32_t bytes, uint64_t* b) {
  asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
                   s32(dst)),
               "l"(src), "r"(bytes), "r"(s32(b))
               : "memory");
}

__device__ __forceinline__ void cluster_arrive() { asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory"); }
__device__ __forceinline__ void cluster_wait() { asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory"); }

template <typename T> __device__ __forceinline__ float tof(T v);
template <> __device__ __forceinline__ float tof<float>(float v) { return v; }
template <> __device__ __forceinline__ float tof<__nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

template <typename ACC, typename T>
__device__ __forceinline__ ACC to_acc(T v) {
  if constexpr (sizeof(ACC) == 8) return (ACC)v;
  else return tof<T>(v);
}

// Per-problem constants kept in shared memory (the descriptor in global memory is read once).
struct LoopConst {
  Prob p;
  LoopSmem L;
  int vec[kMaxOrder];      // bytes per cp.async of a mode's fiber copies (16, 8, 4), 0: plain loads
  int bulk[kMaxOrder];     // 1: a mode's fibers are contiguous and 16-byte aligned: one TMA bulk copy each
  int draw_late;           // 1: every mode copies by TMA and R^2 <= 384: the next update's samples are
                           // drawn (and copies issued) by the warps idle during the FP64 refinement
  int gs, gg;              // Gram: samples split over gs lanes; sum of the C partials over gg lanes
  unsigned char ne_r[32 * 33 / 2];   // packed upper-triangle entry e -> (row, column)
  unsigned char ne_c[32 * 33 / 2];
};

// Draw the samples of mode update (t, n) for this CTA (Philox stream 0, counter (j, n, t, b)):
// indices by mode and the storage offset of each sampled fiber in the copy that mode reads.
__device__ __forceinline__ void draw_samples(const Prob& p, int n, uint32_t t, int j0, int cnt, uint32_t* ids,
                                             int64_t* offs) {
  for (int jj = threadIdx.x; jj < cnt; jj += kLT) {
    const uint32_t j = (uint32_t)(j0 + jj);
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
      ids[jj * kMaxOrder + m] = im;
    }
    int64_t stride;
    offs[jj] = fiber_offset(p, n, ids + jj * kMaxOrder, &stride);
  }
}

// Copy the cnt sampled fibers of mode n into buf (row j at buf + j * ldf).  Contiguous, aligned
// fibers: one TMA bulk copy per fiber, all issued by thread 0 after it armed the buffer's mbarrier
// with the total byte count (returns true; the consumer waits on that barrier).  Otherwise cp.async
// copies (one commit group per call, possibly empty), or plain loads when no cp.async width fits.
template <typename T>
__device__ __forceinline__ bool fetch_fibers(const LoopConst& K, int n, const int64_t* offs, int cnt, T* buf,
                                             uint64_t* bar) {
  const Prob& p = K.p;
  const int I = (int)p.dims[n];
  const int ldf = K.L.ldf;
  const T* X = reinterpret_cast<const T*>(p.Xrep[n]);
  const int64_t stn = p.use_rep ? 1 : p.st[n];
  const int vec = K.vec[n];
  const int tid = threadIdx.x;
  if (K.bulk[n]) {
    if (tid == 0) {
      const uint32_t fb = (uint32_t)I * (uint32_t)sizeof(T);
      mbar_expect_tx(bar, fb * (uint32_t)cnt);
      for (int j = 0; j < cnt; ++j) bulk_copy(buf + j * ldf, X + offs[j], fb, bar);
    }
    return true;
  }
  if (stn == 1 && vec >= 4) {
    const int epc = vec / (int)sizeof(T);      // elements per copy
    const int cpf = I / epc;                    // copies per fiber
    for (int j = 0; j < cnt; ++j) {
      const T* src = X + offs[j];
      T* dst = buf + j * ldf;
      for (int q = tid; q < cpf; q += kLT) {
        if (vec == 16) cp_async<16>(dst + q * epc, src + (int64_t)q * epc);
        else if (vec == 8) cp_async<8>(dst + q * epc, src + (int64_t)q * epc);
        else cp_async<4>(dst + q * epc, src + (int64_t)q * epc);
      }
    }
  } else if (vec >= 4) {                        // strided fibers, one element per copy
    for (int j = 0; j < cnt; ++j)
      for (int i = tid; i < I; i += kLT) {
        if constexpr (sizeof(T) == 8) cp_async<8>(buf + j * ldf + i, X + offs[j] + (int64_t)i * stn);
        else cp_async<4>(buf + j * ldf + i, X + offs[j] + (int64_t)i * stn);
      }
  } else {
    for (int j = 0; j < cnt; ++j)
      for (int i = tid; i < I; i += kLT) buf[j * ldf + i] = X[offs[j] + (int64_t)i * stn];
  }
  cp_async_commit();
  return false;
}

// The next mode update's samples drawn by the threads [base, kLT) while the others refine the
// inverse, each drawing thread issuing the TMA bulk copy of its own fiber (every mode's fibers are
// contiguous and aligned when this is used); thread `base` arms the buffer's mbarrier.  An mbarrier
// transaction count may go transiently negative, so the arming need not precede the copies.
template <typename T>
__device__ __forceinline__ void draw_and_copy(const LoopConst& K, int n, uint32_t t, int j0, int cnt, uint32_t* ids,
                                              int64_t* offs, T* buf, uint64_t* bar, int base) {
  const Prob& p = K.p;
  const uint32_t fb = (uint32_t)p.dims[n] * (uint32_t)sizeof(T);
  const T* X = reinterpret_cast<const T*>(p.Xrep[n]);
  if ((int)threadIdx.x == base) mbar_expect_tx(bar, fb * (uint32_t)cnt);
  for (int jj = (int)threadIdx.x - base; jj < cnt; jj += kLT - base) {
    const uint32_t j = (uint32_t)(j0 + jj);
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
      ids[jj * kMaxOrder + m] = im;
    }
    int64_t stride;
    const int64_t off = fiber_offset(p, n, ids + jj * kMaxOrder, &stride);
    offs[jj] = off;
    bulk_copy(buf + jj * K.L.ldf, X + off, fb, bar);
  }
}

// Wait for the fibers of the buffer about to be read: its mbarrier phase when they came by TMA
// bulk copies (bounded; a wait that runs out sets *s_tout), and any cp.async groups.
__device__ __forceinline__ void wait_fibers(uint64_t* fbar, int b, uint32_t& fpar, uint32_t fblk, int* s_tout) {
  if ((fblk >> b) & 1u) {
    if (!mbar_wait_bounded(fbar + b, (fpar >> b) & 1u)) *s_tout = 1;
    fpar ^= 1u << b;
  }
  cp_async_wait_all();
}

// X0 = G^-1 in FP32 by Gauss-Jordan elimination without pivoting (G symmetric positive definite),
// one thread per entry of the R x 2R tableau [G | I], one block barrier per step (tableaus
// alternate between the two halves of gj).  Returns (the same in every thread) false when a pivot
// is not positive relative to the largest diagonal entry md; X0 is then columns R.. of the final
// tableau: gj[(R & 1) * 2R^2 + i * 2R + R + c].
template <int MAXR>
__device__ bool gauss_jordan_block(const float* Gf, float* gj, int R, float md) {
  constexpr int EPT = (2 * MAXR * MAXR + kLT - 1) / kLT;   // tableau entries per thread
  const int W = 2 * R, nent = R * W, tid = threadIdx.x;
  int ei[EPT], ec[EPT];
#pragma unroll
  for (int q = 0; q < EPT; ++q) {
    const int e = tid + q * kLT;
    ei[q] = e / W;
    ec[q] = e - ei[q] * W;
    if (e < nent) gj[e] = ec[q] < R ? Gf[ei[q] * R + ec[q]] : (ec[q] - R == ei[q] ? 1.f : 0.f);
  }
  __syncthreads();
  bool bad = false;
  for (int k = 0; k < R; ++k) {
    const float* o = gj + (k & 1) * nent;
    float* w = gj + ((k + 1) & 1) * nent;
    const float piv = o[k * W + k];
    bad = bad || !(piv > 1e-6f * md) || !isfinite(piv);
    const float inv = 1.f / piv;
#pragma unroll
    for (int q = 0; q < EPT; ++q) {
      const int e = tid + q * kLT;
      if (e < nent) {
        const float pkc = o[k * W + ec[q]] * inv;
        w[e] = ei[q] == k ? pkc : fmaf(-o[ei[q] * W + k], pkc, o[e]);
      }
    }
    __syncthreads();
  }
  return !bad;
}

template <typename T, typename ACC, int MAXR>
__device__ void loop_mode_update(const LoopConst& K, unsigned char* sm, cg::cluster_group& cl, int n, int cb,
                                 int nn, uint32_t nt, int* s_bad, unsigned* s_em, uint64_t* fbar, uint32_t& fpar,
                                 uint32_t& fblk, int* s_tout) {
  const Prob& p = K.p;
  const LoopSmem& L = K.L;
  const int rank = (int)cl.block_rank(), tid = threadIdx.x;
  const int R = p.R, N = p.N, S = p.S;
  const int I = (int)p.dims[n];
  const int spc = L.spc, rp = L.rp, ne = L.NE;
  const int cnt = max(0, min(S, rank * spc + spc) - rank * spc);
  double* sc = reinterpret_cast<double*>(sm + L.sc);
  double* lam = reinterpret_cast<double*>(sm + L.lam);
  double* scomb = reinterpret_cast<double*>(sm + L.scomb);
  double* Zd = reinterpret_cast<double*>(sm + L.Zd);
  ACC* Zf = reinterpret_cast<ACC*>(sm + L.Zf);
  const uint32_t* ids = reinterpret_cast<const uint32_t*>(sm + L.ids[cb]);
  const T* fib = reinterpret_cast<const T*>(sm + L.fib[cb]);
  ACC* Mrecv = reinterpret_cast<ACC*>(sm + L.Mrecv);
  double* Grecv = reinterpret_cast<double*>(sm + L.Grecv);
  double* colrecv = reinterpret_cast<double*>(sm + L.colrecv);
  double* G = reinterpret_cast<double*>(sm + L.G);
  float* Gf = reinterpret_cast<float*>(sm + L.Gf);
  double* mrow = reinterpret_cast<double*>(sm + L.mrow);
  double* arow = reinterpret_cast<double*>(sm + L.arow);
  double* cpart = reinterpret_cast<double*>(sm + L.cpart);

  // ---- 1. SKR rows of this CTA's samples (Alg. 2), from the local factor copies: the product of
  // the sampled rows (exact in FP64 for up to two FP32 factors) times the combined lazy scale
  for (int e = tid; e < cnt * rp; e += kLT) {
    const int jj = e / rp, r = e - jj * rp;
    if (r < R) {
      // a loop over the N - 1 other modes only: predicated-off FP64 multiplies of a loop unrolled to
      // the maximum order would still occupy the FP64 pipe
      double z = scomb[r];
#pragma unroll 1
      for (int m = 0; m < N; ++m)
        if (m != n) {
          const ACC* Fm = reinterpret_cast<const ACC*>(sm + L.F[m]);
          z *= (double)Fm[(int)ids[jj * kMaxOrder + m] * rp + r];
        }
      Zd[jj * R + r] = z;
      Zf[e] = (ACC)z;
    } else {
      Zf[e] = ACC(0);
    }
  }
  wait_fibers(fbar, cb, fpar, fblk, s_tout);   // this update's fibers (issued during the previous update)
  __syncthreads();

  // ---- 2. partial M = X_S,c Z_S,c, every row, stored into the owner CTA's receive buffer
  const int rpc = (I + kLC - 1) / kLC;
  constexpr int VZ = 16 / (int)sizeof(ACC);      // Z entries per 16-byte vector
  for (int i = tid; i < I; i += kLT) {
    ACC acc[MAXR];
#pragma unroll
    for (int r = 0; r < MAXR; ++r) acc[r] = ACC(0);
    const T* fi = fib + i;
#pragma unroll 2
    for (int j = 0; j < cnt; ++j) {
      const ACC x = to_acc<ACC, T>(fi[j * L.ldf]);
      const ACC* z = Zf + j * rp;
#pragma unroll
      for (int v = 0; v < MAXR; v += VZ) {
        if (v < R) {
          if constexpr (VZ == 4) {
            const float4 q = *reinterpret_cast<const float4*>(z + v);
            acc[v] = fma(x, q.x, acc[v]);
            acc[v + 1] = fma(x, q.y, acc[v + 1]);
            acc[v + 2] = fma(x, q.z, acc[v + 2]);
            acc[v + 3] = fma(x, q.w, acc[v + 3]);
          } else {
            const double2 q = *reinterpret_cast<const double2*>(z + v);
            acc[v] = fma(x, q.x, acc[v]);
            acc[v + 1] = fma(x, q.y, acc[v + 1]);
          }
        }
      }
    }
    // column-major receive layout: lanes (consecutive rows) store to consecutive addresses
    const int owner = i / rpc, li = i - owner * rpc;
    ACC* dst = cl.map_shared_rank(Mrecv, owner) + rank * R * L.rpcmax + li;
#pragma unroll
    for (int r = 0; r < MAXR; ++r)
      if (r < R) dst[r * L.rpcmax] = acc[r];
  }
  // ---- 3. partial Gram of this CTA's Z rows (upper triangle, gs lanes per entry), to every CTA
  {
    const int gs = K.gs;
    for (int t0 = 0; t0 < ne * gs; t0 += kLT) {
      const int t = t0 + tid;
      const int e = t / gs, s = t - e * gs;
      double a = 0.0;
      if (e < ne) {
        const int r = K.ne_r[e], c = K.ne_c[e];
        for (int jj = s; jj < cnt; jj += gs) a = fma(Zd[jj * R + r], Zd[jj * R + c], a);
      }
      for (int o = 1; o < gs; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (e < ne)
        for (int q = s; q < kLC; q += gs) cl.map_shared_rank(Grecv, q)[rank * ne + e] = a;
    }
  }
  cluster_arrive();
  // independent work while the barrier completes: the next mode update's samples and fiber copies
  // (unless the idle warps of the refinement step issue them)
  if (tid == 0) *s_em = 0u;
  if (!K.draw_late) {
    draw_samples(p, nn, nt, rank * spc, cnt, reinterpret_cast<uint32_t*>(sm + L.ids[cb ^ 1]),
                 reinterpret_cast<int64_t*>(sm + L.offs[cb ^ 1]));
    __syncthreads();
    if (fetch_fibers<T>(K, nn, reinterpret_cast<const int64_t*>(sm + L.offs[cb ^ 1]), cnt,
                       reinterpret_cast<T*>(sm + L.fib[cb ^ 1]), fbar + (cb ^ 1)))
      fblk |= 1u << (cb ^ 1);
    else
      fblk &= ~(1u << (cb ^ 1));
  }
  cluster_wait();   // every partial M row and Gram of the cluster has landed

  // ---- 4. G = sum of the C partial Grams (fixed order, gg lanes per entry); FP32 copy; max diag
  {
    const int gg = K.gg;
    for (int t0 = 0; t0 < ne * gg; t0 += kLT) {
      const int t = t0 + tid;
      const int e = t / gg, g = t - e * gg;
      double a = 0.0;
      if (e < ne)
        for (int q = g; q < kLC; q += gg) a += Grecv[q * ne + e];
      for (int o = 1; o < gg; o <<= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
      if (e < ne && g == 0) {
        const int r = K.ne_r[e], c = K.ne_c[e];
        G[r * R + c] = a;
        G[c * R + r] = a;
        const float af = (float)a;
        Gf[r * R + c] = af;
        Gf[c * R + r] = af;
        if (r == c && af > 0.f) atomicMax(s_em, __float_as_uint(af));   // positive floats order as ints
      }
    }
  }
  __syncthreads();
  const float md = __uint_as_float(*s_em);
  float* gj = reinterpret_cast<float*>(sm + L.gj);
  const bool ok = gauss_jordan_block<MAXR>(Gf, gj, R, md);
  const int W = 2 * R;
  const float* X0 = gj + (R & 1) * (R * W) + R;   // X0(i, c) = X0[i * W + c]
  double* X = reinterpret_cast<double*>(sm + L.X);
  {
    // ---- Newton-Schulz refinement (or the FP64 Cholesky inverse).  Step k: E = I - G X_k with the
    // residual in FP64, X_{k+1} = X_k + X0 E (the small correction in FP32 from the FP32 start X0,
    // which equals X_k to FP32 accuracy).  b = R max|E_ij| bounds ||E||_inf, and the step leaves a
    // residual of at most b^2 (plus the FP32 correction's rounding, about 1e-7 of b), so the steps stop
    // once b^2 is below the target (1e-7 for FP32 / BF16 tensors, 1e-13 for FP64); a start with
    // b >= 1/2, or no convergence within six steps, takes the FP64 Cholesky inverse instead (which
    // also reports a singular Gram).  Iterates alternate between X and U.
    double* U = reinterpret_cast<double*>(sm + L.U);
    double* E = reinterpret_cast<double*>(sm + L.E);
    const int RR = R * R;
    bool fast = ok;
    const double target = sizeof(ACC) == 8 ? 1e-13 : 1e-7;
    if (tid == 0) {
      s_em[1] = 0u;
      s_em[2] = 0u;
    }
    __syncthreads();
    const int dbase = (RR + 31) / 32 * 32;   // first thread not computing an entry of E
    // E in FP32 for the correction X E: |E| is small, so the FP32 product's rounding (about 1e-7 of
    // |X E|) stays far below the FP64 residual of the step; it lives in the tableau half X0 is not in
    float* Ef = gj + ((R + 1) & 1) * (R * W);
    bool drawn = false;
    const double* cur = nullptr;   // the current iterate (null: the FP32 start X0)
    for (int it = 0; fast; ++it) {
      unsigned* slot = s_em + 1 + (it & 1);
      if (tid == 0) s_em[1 + ((it + 1) & 1)] = 0u;   // the next step's slot (read two barriers ago)
      float em = 0.f;
      for (int e = tid; e < RR; e += kLT) {
        const int r = e / R, c = e - r * R;
        const double* g = G + r * R;
        double a0 = 0.0, a1 = 0.0;
        int l = 0;
        if (!cur) {
          for (; l + 1 < R; l += 2) {
            a0 = fma(g[l], (double)X0[l * W + c], a0);
            a1 = fma(g[l + 1], (double)X0[(l + 1) * W + c], a1);
          }
          if (l < R) a0 = fma(g[l], (double)X0[l * W + c], a0);
        } else {
          for (; l + 1 < R; l += 2) {
            a0 = fma(g[l], cur[l * R + c], a0);
            a1 = fma(g[l + 1], cur[(l + 1) * R + c], a1);
          }
          if (l < R) a0 = fma(g[l], cur[l * R + c], a0);
        }
        const double ev = (r == c ? 1.0 : 0.0) - (a0 + a1);
        E[e] = ev;
        Ef[e] = (float)ev;
        em = fmaxf(em, fabsf((float)ev));
      }
      const unsigned wm = __reduce_max_sync(0xffffffffu, __float_as_uint(em));
      if ((tid & 31) == 0 && wm) atomicMax(slot, wm);
      if (it == 0) {
        if (K.draw_late && tid >= dbase) {
          draw_and_copy<T>(K, nn, nt, rank * spc, cnt, reinterpret_cast<uint32_t*>(sm + L.ids[cb ^ 1]),
                           reinterpret_cast<int64_t*>(sm + L.offs[cb ^ 1]), reinterpret_cast<T*>(sm + L.fib[cb ^ 1]),
                           fbar + (cb ^ 1), dbase);
        }
        drawn = true;
      }
      __syncthreads();
      const float b = (float)R * __uint_as_float(*slot);
      if (!(b < 0.5f)) {
        fast = false;
        break;
      }
      const bool last = (double)b * (double)b < target;
      if (!last && it >= 6) {
        fast = false;
        break;
      }
      double* Xout = (it & 1) ? U : X;
      for (int e = tid; e < RR; e += kLT) {
        const int r = e / R, c = e - r * R;
        const float* xr = X0 + r * W;
        float a0 = 0.f, a1 = 0.f;
        int l = 0;
        for (; l + 1 < R; l += 2) {
          a0 = fmaf(xr[l], Ef[l * R + c], a0);
          a1 = fmaf(xr[l + 1], Ef[(l + 1) * R + c], a1);
        }
        if (l < R) a0 = fmaf(xr[l], Ef[l * R + c], a0);
        const double x = cur ? cur[e] : (double)xr[c];
        Xout[e] = x + (double)(a0 + a1);
      }
      __syncthreads();
      cur = Xout;
      if (last) break;
    }
    if (fast) X = const_cast<double*>(cur);
    if (K.draw_late && !drawn) {   // the refinement did not run: draw with every thread
      draw_and_copy<T>(K, nn, nt, rank * spc, cnt, reinterpret_cast<uint32_t*>(sm + L.ids[cb ^ 1]),
                       reinterpret_cast<int64_t*>(sm + L.offs[cb ^ 1]), reinterpret_cast<T*>(sm + L.fib[cb ^ 1]),
                       fbar + (cb ^ 1), 0);
    }
    if (K.draw_late) fblk |= 1u << (cb ^ 1);
    if (!fast) {
      X = reinterpret_cast<double*>(sm + L.X);
      spd_inverse_fp64(G, X, U, reinterpret_cast<double*>(sm + L.T2), reinterpret_cast<double*>(sm + L.dinv), R,
                       s_bad);
    }
  }

  // ---- 5. this CTA's rows: M rows (fixed-order sum over the C partials), A = M G^-1 (FP64)
  const int i0 = rank * rpc;
  const int nrows = max(0, min(I, i0 + rpc) - i0);
  for (int e = tid; e < nrows * R; e += kLT) {
    const int li = e / R, r = e - li * R;
    ACC a = ACC(0);
#pragma unroll
    for (int q = 0; q < kLC; ++q) a += Mrecv[(q * R + r) * L.rpcmax + li];
    mrow[e] = (double)a;
  }
  __syncthreads();
  ACC* Fn = reinterpret_cast<ACC*>(sm + L.F[n]);
  double* A64n = p.A64[n] + (int64_t)i0 * R;
  for (int e = tid; e < nrows * R; e += kLT) {
    const int li = e / R, r = e - li * R;
    const double* m = mrow + li * R;
    double s0 = 0.0, s1 = 0.0;
    int l = 0;
    for (; l + 1 < R; l += 2) {
      s0 = fma(m[l], X[l * R + r], s0);
      s1 = fma(m[l + 1], X[(l + 1) * R + r], s1);
    }
    if (l < R) s0 = fma(m[l], X[l * R + r], s0);
    const double a = s0 + s1;
    arow[e] = a;
    A64n[e] = a;                                    // FP64 result (read after the run)
    const ACC af = (ACC)a;
    const int off = (i0 + li) * rp + r;
#pragma unroll 4
    for (int q = 0; q < kLC; ++q) cl.map_shared_rank(Fn, q)[off] = af;   // every CTA's copy
  }
  __syncthreads();
  {
    // column sums of squares of this CTA's rows: 8-row chunks, then a fixed-order sum
    const int nch = (nrows + 7) / 8;
    for (int e = tid; e < R * nch; e += kLT) {
      const int r = e / nch, ch = e - r * nch;
      double sq = 0.0;
      for (int li = ch * 8; li < min(nrows, ch * 8 + 8); ++li) sq = fma(arow[li * R + r], arow[li * R + r], sq);
      cpart[e] = sq;
    }
    __syncthreads();
    // 16 destination CTAs x R columns: each (q, r) pair is one thread (a warp's stores to one CTA
    // are contiguous)
    for (int e = tid; e < R * kLC; e += kLT) {
      const int q = e / R, r = e - q * R;
      double sq = 0.0;
      for (int ch = 0; ch < nch; ++ch) sq += cpart[r * nch + ch];
      cl.map_shared_rank(colrecv, q)[rank * R + r] = sq;
    }
  }
  cluster_arrive();
  cluster_wait();   // new factor rows and column partials of every CTA have landed

  // ---- 6. lambda and the lazy scales of mode n (4 lanes per column, fixed order)
  const int nl = 4 * R;
  if (tid < (nl + 31) / 32 * 32) {       // whole warps (the shuffles need every lane)
    const bool v = tid < nl;
    const int r = tid >> 2, g = tid & 3;
    double a = 0.0;
    if (v)
      for (int q = g; q < kLC; q += 4) a += colrecv[q * R + r];
    a += __shfl_xor_sync(0xffffffffu, a, 1);
    a += __shfl_xor_sync(0xffffffffu, a, 2);
    if (v && g == 0) {
      const double y = a > 0.0 ? rsqrt64(a) : 0.0;
      const double nrm = a * y;
      const double scn = nrm > 0.0 ? y : 1.0;
      lam[r] = nrm;
      sc[n * R + r] = scn;
      double c = 1.0;                        // combined scale of the modes other than nn
      for (int m = 0; m < N; ++m)
        if (m != nn) c *= (m == n ? scn : sc[m * R + r]);
      scomb[r] = c;
    }
  }
  __syncthreads();
}

template <typename T, typename ACC, int MAXR>
__global__ void __launch_bounds__(kLT, 1) k_loop_rep(const Prob* probs, int B, int* queue) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ LoopConst K;
  __shared__ int s_prob, s_bad, s_done, s_status, s_iter, s_stall;
  __shared__ unsigned s_em[3];   // [0] diagonal maximum; [1], [2] refinement residuals
  __shared__ int s_tout;
  __shared__ double s_best, s_last;
  __shared__ double fitpart[4];
  __shared__ __align__(8) uint64_t fbar[2];   // completion of the TMA bulk fiber copies, per buffer
  while (true) {
    if (rank == 0 && tid == 0) s_prob = atomicAdd(queue, 1);
    cl.sync();
    const int b = *cl.map_shared_rank(&s_prob, 0);
    cl.sync();
    if (b >= B) break;
    // the problem descriptor and the layout, once
    {
      const int words = (int)(sizeof(Prob) / 4);
      const uint32_t* src = reinterpret_cast<const uint32_t*>(probs + b);
      uint32_t* dst = reinterpret_cast<uint32_t*>(&K.p);
      for (int w = tid; w < words; w += kLT) dst[w] = src[w];
    }
    __syncthreads();
    if (tid == 0) {
      const Prob& p = K.p;
      K.L = loop_layout(p.N, p.R, p.dims, p.S, p.P_hat, (int)sizeof(T), (int)sizeof(ACC));
      for (int m = 0; m < kMaxOrder; ++m) {
        int v = 0;
        if (m < p.N) {
          const bool contig = p.use_rep || m == 0;
          const uintptr_t base = reinterpret_cast<uintptr_t>(p.Xrep[m]);
          const int fb = (int)p.dims[m] * (int)sizeof(T);
          if (contig) {
            if (fb % 16 == 0 && base % 16 == 0) v = 16;
            else if (fb % 8 == 0 && base % 8 == 0) v = 8;
            else if (fb % 4 == 0 && base % 4 == 0 && sizeof(T) <= 4) v = 4;
          } else if (sizeof(T) >= 4) {
            v = (int)sizeof(T);
          }
        }
        K.vec[m] = v;
        K.bulk[m] = (m < p.N && (p.use_rep || m == 0) && v == 16) ? 1 : 0;
      }
      {
        int all_bulk = 1;
        for (int m = 0; m < p.N; ++m) all_bulk &= K.bulk[m];
        K.draw_late = (all_bulk && p.R * p.R <= kLT - 128) ? 1 : 0;
      }
      mbar_init(&fbar[0]);
      mbar_init(&fbar[1]);
      asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
      s_tout = 0;
      // Gram partial: gs lanes per entry; C-way sum: gg lanes per entry (fewest FP64 warp
      // instructions per SM sub-partition)
      const int ne = K.L.NE, spc = K.L.spc;
      int best = 1 << 30;
      for (int gs = 1; gs <= 8; gs <<= 1) {
        const int warps = (ne * gs + 31) / 32;
        const int cost = ((warps + 3) / 4) * ((spc + gs - 1) / gs + (gs > 1 ? 31 - __clz(gs) : 0)) * ((ne * gs + kLT - 1) / kLT);
        if (cost < best) {
          best = cost;
          K.gs = gs;
        }
      }
      best = 1 << 30;
      for (int gg = 1; gg <= 8; gg <<= 1) {
        const int warps = (ne * gg + 31) / 32;
        const int cost = ((warps + 3) / 4) * (kLC / gg - 1 + (gg > 1 ? 31 - __clz(gg) : 0)) * ((ne * gg + kLT - 1) / kLT);
        if (cost < best) {
          best = cost;
          K.gg = gg;
        }
      }
      int e = 0;
      for (int r = 0; r < p.R; ++r)
        for (int c = r; c < p.R; ++c, ++e) {
          K.ne_r[e] = (unsigned char)r;
          K.ne_c[e] = (unsigned char)c;
        }
    }
    __syncthreads();
    const Prob& p = K.p;
    const LoopSmem& L = K.L;
    const int R = p.R, N = p.N, rp = L.rp;
    double* sc = reinterpret_cast<double*>(sm + L.sc);
    double* lam = reinterpret_cast<double*>(sm + L.lam);
    ACC* wr = reinterpret_cast<ACC*>(sm + L.wr);
    double* red = reinterpret_cast<double*>(sm + L.red);
    double* fitrecv = reinterpret_cast<double*>(sm + L.fitrecv);
    uint32_t* fidx = reinterpret_cast<uint32_t*>(sm + L.fidx);
    ACC* fx = reinterpret_cast<ACC*>(sm + L.fx);
    State* st = p.state;
    // every factor in full (rows padded with zeros), the lazy scales, lambda, this CTA's fit entries
    for (int m = 0; m < N; ++m) {
      ACC* F = reinterpret_cast<ACC*>(sm + L.F[m]);
      const int cntm = (int)p.dims[m] * rp;
      for (int e = tid; e < cntm; e += kLT) {
        const int i = e / rp, r = e - i * rp;
        ACC v = ACC(0);
        if (r < R) {
          if constexpr (sizeof(ACC) == 8) v = p.A64[m][(int64_t)i * R + r];
          else v = p.A32[m][(int64_t)i * R + r];
        }
        F[e] = v;
      }
    }
    for (int e = tid; e < N * R; e += kLT) sc[e] = p.scale[e / R][e % R];
    for (int r = tid; r < R; r += kLT) lam[r] = p.lambda[r];
    const int f0 = rank * L.fpc;
    const int fcnt = max(0, min(p.P_hat, f0 + L.fpc) - f0);
    for (int e = tid; e < fcnt * N; e += kLT) fidx[e] = p.fit_idx[(int64_t)f0 * N + e];
    for (int e = tid; e < fcnt; e += kLT) fx[e] = (ACC)p.fit_x[f0 + e];
    for (int r = tid; r < rp; r += kLT) wr[r] = ACC(0);
    if (tid == 0) {
      s_done = st->done;
      s_status = st->status;
      s_iter = st->iter;
      s_stall = st->stall;
      s_best = st->best;
      s_last = st->last_fit;
      s_bad = 0;
    }
    const double fit_scale = (double)p.P / (double)p.P_hat;   // P / P_hat
    const double inv_norm = 1.0 / st->norm_x;
    // samples and fiber copies of the first mode update
    const int spc = L.spc;
    const int j0 = rank * spc;
    const int cnt = max(0, min(p.S, j0 + spc) - j0);
    draw_samples(p, 0, p.t0 + (uint32_t)st->iter, j0, cnt, reinterpret_cast<uint32_t*>(sm + L.ids[0]),
                 reinterpret_cast<int64_t*>(sm + L.offs[0]));
    __syncthreads();
    uint32_t fpar = 0u, fblk = 0u;   // per fiber buffer: mbarrier phase parity; last fetch was TMA bulk
    if (fetch_fibers<T>(K, 0, reinterpret_cast<const int64_t*>(sm + L.offs[0]), cnt,
                        reinterpret_cast<T*>(sm + L.fib[0]), &fbar[0]))
      fblk = 1u;
    {
      double* scomb = reinterpret_cast<double*>(sm + L.scomb);
      for (int r = tid; r < R; r += kLT) {   // combined scale of the modes other than the first
        double c = 1.0;
        for (int m = 1; m < N; ++m) c *= sc[m * R + r];
        scomb[r] = c;
      }
    }
    cl.sync();   // every CTA initialized before any stores into another
    const int cap = p.fixed_iters > 0 ? p.fixed_iters : p.max_iters;
    int u = 0;   // mode updates run (selects the sample / fiber buffer)
    while (!s_done && s_iter < cap) {
      const uint32_t t = p.t0 + (uint32_t)s_iter;
      for (int n = 0; n < N; ++n) {
        const int cb = u & 1;
        // the next mode update (its samples and fiber copies are issued during this one)
        const int nn = n + 1 < N ? n + 1 : 0;
        const uint32_t nt = n + 1 < N ? t : t + 1;
        loop_mode_update<T, ACC, MAXR>(K, sm, cl, n, cb, nn, nt, &s_bad, s_em, fbar, fpar, fblk, &s_tout);
        ++u;
        if (s_bad) break;   // identical in every CTA (same G, same factorization)
      }
      if (s_bad) {
        if (tid == 0) {
          s_status = CPR_ESINGULAR;
          s_done = 1;
        }
        __syncthreads();
        break;
      }
      // ---- sampled fit (Sec. 3.4) on this CTA's share of the fixed entries
      for (int r = tid; r < R; r += kLT) {
        double w = lam[r];
        for (int m = 0; m < N; ++m) w *= sc[m * R + r];
        wr[r] = (ACC)w;
      }
      __syncthreads();
      constexpr int VZ = 16 / (int)sizeof(ACC);
      ACC e2a = ACC(0);           // this thread's entries (at most a few), in the accumulation type
      for (int jj = tid; jj < fcnt; jj += kLT) {
        const uint32_t* id = fidx + jj * N;
        const ACC* rows[kMaxOrder];
#pragma unroll
        for (int m = 0; m < kMaxOrder; ++m)
          rows[m] = (m < N) ? reinterpret_cast<const ACC*>(sm + L.F[m]) + (int)id[m] * rp : nullptr;
        ACC acc = ACC(0);
#pragma unroll
        for (int v = 0; v < MAXR; v += VZ) {
          if (v < R) {
            if constexpr (VZ == 4) {
              float4 w = *reinterpret_cast<const float4*>(wr + v);
#pragma unroll
              for (int m = 0; m < kMaxOrder; ++m)
                if (m < N) {
                  const float4 q = *reinterpret_cast<const float4*>(rows[m] + v);
                  w.x *= q.x;
                  w.y *= q.y;
                  w.z *= q.z;
                  w.w *= q.w;
                }
              acc += (w.x + w.y) + (w.z + w.w);
            } else {
              double2 w = *reinterpret_cast<const double2*>(wr + v);
#pragma unroll
              for (int m = 0; m < kMaxOrder; ++m)
                if (m < N) {
                  const double2 q = *reinterpret_cast<const double2*>(rows[m] + v);
                  w.x *= q.x;
                  w.y *= q.y;
                }
              acc += w.x + w.y;
            }
          }
        }
        const ACC e = fx[jj] - acc;
        e2a = fma(e, e, e2a);
      }
      red[tid] = (double)e2a;
      __syncthreads();
      if (warp < 4) {   // four warps (one per SM sub-partition) sum 128 values each in FP64
        double a = red[warp * 128 + lane] + red[warp * 128 + 32 + lane];
        a += red[warp * 128 + 64 + lane] + red[warp * 128 + 96 + lane];
        for (int o = 16; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) fitpart[warp] = a;
      }
      __syncthreads();
      if (warp == 0 && lane < kLC) {
        const double tot = (fitpart[0] + fitpart[1]) + (fitpart[2] + fitpart[3]);
        cl.map_shared_rank(fitrecv, lane)[rank] = tot;
      }
      cluster_arrive();
      cluster_wait();
      if (warp == 0) {
        double a = lane < kLC ? fitrecv[lane] : 0.0;
        for (int o = 8; o > 0; o >>= 1) a += __shfl_xor_sync(0xffffffffu, a, o);
        if (lane == 0) {
          // F = 1 - sqrt(P mean e^2) / ||X||, the square root as v * rsqrt(v)
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
          if (rank == 0 && p.trace) p.trace[s_iter] = fit;
          s_last = fit;
          s_iter = t1;
          if (stop) s_done = 1;
        }
      }
      __syncthreads();
    }
    wait_fibers(fbar, u & 1, fpar, fblk, &s_tout);   // the copies issued for an update that will not run
    // publish the loop state, lambda and the lazy scales (CTA 0)
    if (rank == 0) {
      for (int e = tid; e < N * R; e += kLT) p.scale[e / R][e % R] = sc[e];
      for (int r = tid; r < R; r += kLT) p.lambda[r] = lam[r];
      if (tid == 0) {
        st->done = 1;
        st->status = s_status;
        st->iter = s_iter;
        st->stall = s_stall;
        st->best = s_best;
        st->last_fit = s_last;
      }
    }
    __syncthreads();
    cl.sync();  // no CTA reuses its shared memory while another may still store into it
    if (tid == 0 && s_tout) st->status = CPR_ETIMEOUT;   // after CTA 0 published the state
  }
}

template <typename T, typename ACC, int MAXR>
cudaError_t loop_launch(const Prob* probs, int B, int* queue, int smem, int nclusters, cudaStream_t s, int query,
                        int* capacity) {
  auto kern = k_loop_rep<T, ACC, MAXR>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  if (e != cudaSuccess) return e;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(kLC * (query ? 1 : nclusters)), 1, 1);
  cfg.blockDim = dim3(kLT, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)kLC;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  if (query) {
    int n = 0;
    e = cudaOccupancyMaxActiveClusters(&n, kern, &cfg);
    if (e != cudaSuccess) {
      cudaGetLastError();
      n = 0;
    }
    *capacity = n;
    return cudaSuccess;
  }
  return cudaLaunchKernelEx(&cfg, kern, probs, B, queue);
}

template <typename T, typename ACC>
cudaError_t loop_dispatch_r(int maxR, const Prob* probs, int B, int* queue, int smem, int ncl, cudaStream_t s,
                            int query, int* cap) {
  if (maxR <= 8) return loop_launch<T, ACC, 8>(probs, B, queue, smem, ncl, s, query, cap);
  if (maxR <= 16) return loop_launch<T, ACC, 16>(probs, B, queue, smem, ncl, s, query, cap);
  return loop_launch<T, ACC, 32>(probs, B, queue, smem, ncl, s, query, cap);
}

cudaError_t loop_dispatch(int dtype, int maxR, const Prob* probs, int B, int* queue, int smem, int ncl, cudaStream_t s,
                          int query, int* cap) {
  switch (dtype) {
    case CPR_F64: return loop_dispatch_r<double, double>(maxR, probs, B, queue, smem, ncl, s, query, cap);
    case CPR_F32: return loop_dispatch_r<float, float>(maxR, probs, B, queue, smem, ncl, s, query, cap);
    default: return loop_dispatch_r<__nv_bfloat16, float>(maxR, probs, B, queue, smem, ncl, s, query, cap);
  }
}

}  // namespace

// Shared memory of the replicated-factor loop for the largest problem of a batch, or -1 if some
// problem does not fit (rank above 32, or the layout above the per-CTA limit).
int loop_rep_smem_bytes(const Prob* probs_host, int B) {
  int most = 0;
  for (int b = 0; b < B; ++b) {
    const Prob& p = probs_host[b];
    if (p.R > 32) return -1;
    const int ab = p.dtype == CPR_F64 ? 8 : 4;
    const int tb = p.dtype == CPR_F64 ? 8 : (p.dtype == CPR_F32 ? 4 : 2);
    const LoopSmem L = loop_layout(p.N, p.R, p.dims, p.S, p.P_hat, tb, ab);
    most = most > L.bytes ? most : L.bytes;
  }
  return most <= 200 * 1024 ? most : -1;
}

int loop_rep_capacity(int dtype, int smem, int maxR) {
  int cap = 0;
  if (loop_dispatch(dtype, maxR, nullptr, 0, nullptr, smem, 0, nullptr, 1, &cap) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return cap;
}

cudaError_t launch_loop_rep(const Prob* probs, int B, int* queue, int dtype, int smem, int nclusters, int maxR,
                            cudaStream_t s) {
  return loop_dispatch(dtype, maxR, probs, B, queue, smem, nclusters, s, 0, nullptr);
}

}  // namespace cpr
