// Mode-n mixing product on the 5th-generation tensor cores (tcgen05, TMEM accumulators, TMA).
//
// One pass computes, for the column-major mode-n unfolding U = X_(n) (row j = fiber j, K = I_n
// contiguous entries) and the mixing operator W = F_n D_n (I_n x I_n, row-major):
//     C[j][c] = sum_k U[j][k] W[c][k]              (the fibers of X x_n W, Alg. 5 mixing step)
// and writes C in the standard column-major layout of the tensor and, optionally, as the mode-n
// unfolding of the result (C[j][c] at c + I_n j) and, in the first pass, as the mode-2 unfolding
// the second pass reads (then the standard layout is not needed).  Both operands are K-major; tiles arrive by TMA
// with the 128-byte swizzle, one thread issues tcgen05.mma (kind::tf32, M = 128, N = NT <= 256)
// into a TMEM accumulator, four warps read it back with tcgen05.ld for the stores.
//
// Accuracy: tf32 keeps 10 explicit mantissa bits.  With three_x, every operand is split into
// hi = x with its low 13 mantissa bits cleared and lo = x - hi (exact), and the product is
// hi*hi + hi*lo + lo*hi (the dropped lo*lo term is below FP32 rounding): FP32-level results at
// three MMAs per k-step.  W's halves come from global memory; the tile of U is split in shared
// memory by the epilogue warps while they wait.
//
// Roles (256 threads, one persistent CTA per SM): warp 0 lane 0 issues TMA; warp 1 owns TMEM (two
// accumulator buffers) and lane 0 issues MMAs; warps 2-3 split the U tiles; warps 4-7 drain TMEM.
// Two pipeline stages of 32 k-values, continuous across tiles.  Every mbarrier wait is bounded: on
// expiry the kernel records an error and stops issuing work.
#include <cuda.h>
#include <cuda_fp16.h>
#include <string.h>

#include <mutex>

#include "internal.cuh"

namespace cpr {
namespace {

constexpr int kTcThreads = 256;
constexpr int kBM = 128;             // rows (fibers) per tile
constexpr int kBK = 32;              // k-values per stage (128 bytes of fp32)
constexpr int kStages = 2;
constexpr int kAStage = kBM * kBK * 4;         // 16 KB
constexpr int kBStage = 256 * kBK * 4;         // 32 KB (room for NT = 256)
constexpr int kStageBytes = 2 * kAStage + 2 * kBStage;
constexpr int kBarOffset = kStages * kStageBytes;
constexpr int kTcSmem = kBarOffset + 256 + 1024;   // + barriers + alignment slack
constexpr uint32_t kWaitLimit = 1u << 22;

struct TcArgs {
  int64_t J;          // rows (fibers)
  int I;              // K = N extent
  int NT, NB;         // columns per CTA, column blocks
  int three_x;
  int n, N;
  int64_t dims[kMaxOrder];
  int64_t st[kMaxOrder];
  float* ystd;        // may be null
  float* yunf;        // may be null
  float* ynext;       // first pass only (n = 0), may be null: the result as the mode-2 unfolding
  int* err;
};

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(uint64_t* b, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(su32(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint64_t* b, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(su32(b)), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint64_t* b) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(su32(b)) : "memory");
}
__device__ __forceinline__ bool mbar_try(uint64_t* b, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(su32(b)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait on a phase of an mbarrier; false (and the CTA's error flag set) on expiry or if
// another role already gave up.
__device__ __forceinline__ bool mbar_wait(uint64_t* b, uint32_t parity, volatile int* err) {
  for (uint32_t it = 0; it < kWaitLimit; ++it) {
    if (mbar_try(b, parity)) return true;
    if (*err) return false;
  }
  *err = 1;
  return false;
}
__device__ __forceinline__ void tma_2d(void* dst, const CUtensorMap* map, int x, int y, uint64_t* bar) {
  asm volatile(
      "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%2, %3}], [%4];" ::"r"(
          su32(dst)),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(x), "r"(y), "r"(su32(bar))
      : "memory");
}
// Shared-memory matrix descriptor: K-major, 128-byte swizzle, 8-row groups 1024 bytes apart.
__device__ __forceinline__ uint64_t sw128_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(1024 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)2 << 61);
}
// Instruction descriptor: D = F32, A = B = TF32, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_tf32(int M, int N) {
  return (1u << 4) | (2u << 7) | (2u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_tf32(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
__device__ __forceinline__ void mma_commit(uint64_t* bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(su32(bar))
               : "memory");
}
__device__ __forceinline__ float tf32_hi(float x) { return __uint_as_float(__float_as_uint(x) & 0xFFFFE000u); }

// ---- FP16 split path -------------------------------------------------------------------------
// Shared-memory matrix descriptor: K-major, 64-byte swizzle (32 FP16 per row), 8-row groups 512 bytes
// apart.
__device__ __forceinline__ uint64_t sw64_desc(uint32_t saddr) {
  return (uint64_t)((saddr & 0x3FFFFu) >> 4) | ((uint64_t)1 << 16) | ((uint64_t)(512 >> 4) << 32) |
         ((uint64_t)1 << 46) | ((uint64_t)4 << 61);
}
// Instruction descriptor: D = F32, A = B = F16, both K-major, M x N.
__host__ __device__ constexpr uint32_t idesc_f16(int M, int N) {
  return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}
__device__ __forceinline__ void mma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(d),
      "l"(a), "l"(b), "r"(idesc), "r"(acc));
}
// x (already scaled by a power of two into FP16 range) = hi + lo with hi, lo FP16: lo carries the
// next 11 bits, so hi*hi + hi*lo + lo*hi reproduces a product to about 2^-21.
__device__ __forceinline__ void split_f16(float x, __half& h, __half& l) {
  h = __float2half_rn(x);
  l = __float2half_rn(x - __half2float(h));
}

// One mode-n product, persistent: CTA c takes output tiles c, c + gridDim.x, ... (tile t = (row block
// t / NB, column block t % NB)).  The TMA ring of kStages stages runs continuously across tiles, and
// the accumulator is double-buffered in TMEM (2 x 256 columns), so the epilogue of one tile overlaps
// the MMAs of the next.
//   warp 0, lane 0: TMA producer      warp 1: TMEM owner, lane 0 issues the MMAs
//   warps 2-3: split the U tiles into TF32 hi / lo halves      warps 4-7: epilogue (TMEM -> global)
__global__ void __launch_bounds__(kTcThreads, 1)
    k_mix_tc(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmWhi,
             const __grid_constant__ CUtensorMap tmWlo, TcArgs a) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kBarOffset);
  uint64_t* full = bars;                   // TMA landed (1 arrival + tx bytes)
  uint64_t* conv = bars + kStages;         // U tile split (64 arrivals)
  uint64_t* empty = bars + 2 * kStages;    // MMAs done with the stage (tcgen05.commit)
  uint64_t* accf = bars + 3 * kStages;     // accumulator buffer b complete (tcgen05.commit), 2 buffers
  uint64_t* acce = accf + 2;               // accumulator buffer b drained (128 arrivals), 2 buffers
  uint64_t* fin = acce + 2;                // every MMA issued by this CTA complete
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* err = reinterpret_cast<volatile int*>(fin + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t mtiles = (a.J + kBM - 1) / kBM;
  const int64_t ntiles = mtiles * a.NB;
  const int nk = (a.I + kBK - 1) / kBK;
  auto A_hi = [&](int s) { return sm + s * kStageBytes; };
  auto A_lo = [&](int s) { return sm + s * kStageBytes + kAStage; };
  auto B_hi = [&](int s) { return sm + s * kStageBytes + 2 * kAStage; };
  auto B_lo = [&](int s) { return sm + s * kStageBytes + 2 * kAStage + kBStage; };

  if (tid == 0) {
    for (int s = 0; s < kStages; ++s) {
      mbar_init(&full[s], 1);
      mbar_init(&conv[s], 64);
      mbar_init(&empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
    }
    mbar_init(fin, 1);
    *err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t bbytes = (uint32_t)a.NT * kBK * 4;

  if (warp == 0) {
    if (lane == 0) {   // producer: one continuous ring over all of this CTA's tiles
      int64_t it = 0, issued = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int nb = (int)(t % a.NB);
        const int j0 = (int)((t / a.NB) * kBM);
        const int c0 = nb * a.NT;
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = (int)(it % kStages);
          const uint32_t use = (uint32_t)(it / kStages);
          if (it >= kStages && !mbar_wait(&empty[s], (use - 1) & 1, err)) {
            ok = false;
            break;
          }
          mbar_expect_tx(&full[s], (uint32_t)kAStage + (a.three_x ? 2u : 1u) * bbytes);
          tma_2d(A_hi(s), &tmU, i * kBK, j0, &full[s]);
          tma_2d(B_hi(s), &tmWhi, i * kBK, c0, &full[s]);
          if (a.three_x) tma_2d(B_lo(s), &tmWlo, i * kBK, c0, &full[s]);
          issued = it + 1;
        }
      }
      if (*err) {   // never leave copies in flight: wait (bounded) for the last ones issued
        for (int64_t q = issued > kStages ? issued - kStages : 0; q < issued; ++q) {
          const int s = (int)(q % kStages);
          for (uint32_t w = 0; w < kWaitLimit && !mbar_try(&full[s], (uint32_t)(q / kStages) & 1); ++w) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      const uint32_t idesc = idesc_tf32(kBM, a.NT);
      int64_t it = 0, tl = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
        const int b = (int)(tl & 1);
        const uint32_t ub = (uint32_t)(tl >> 1);
        if (tl >= 2 && !mbar_wait(&acce[b], (ub - 1) & 1, err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * 256);
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = (int)(it % kStages);
          if (!mbar_wait(&conv[s], (uint32_t)(it / kStages) & 1, err)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ah = su32(A_hi(s)), al = su32(A_lo(s)), bh = su32(B_hi(s)), bl = su32(B_lo(s));
#pragma unroll
          for (int kk = 0; kk < kBK / 8; ++kk) {
            const uint32_t off = kk * 32;   // 8 tf32 values
            mma_tf32(d, sw128_desc(ah + off), sw128_desc(bh + off), idesc, (i | kk) != 0);
            if (a.three_x) {
              mma_tf32(d, sw128_desc(ah + off), sw128_desc(bl + off), idesc, 1u);
              mma_tf32(d, sw128_desc(al + off), sw128_desc(bh + off), idesc, 1u);
            }
          }
          mma_commit(&empty[s]);
        }
        if (ok) mma_commit(&accf[b]);
      }
      // every MMA this CTA issued has completed before the TMEM is released
      mma_commit(fin);
      for (uint32_t w = 0; w < kWaitLimit && !mbar_try(fin, 0); ++w) {
      }
    }
  } else if (warp < 4) {
    // split the U tiles into hi / lo halves (64 threads)
    const int ct = tid - 64;
    int64_t it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int i = 0; i < nk; ++i, ++it) {
        const int s = (int)(it % kStages);
        if (!mbar_wait(&full[s], (uint32_t)(it / kStages) & 1, err)) {
          ok = false;
          break;
        }
        if (a.three_x) {
          float4* hi = reinterpret_cast<float4*>(A_hi(s));
          float4* lo = reinterpret_cast<float4*>(A_lo(s));
#pragma unroll 4
          for (int v = ct; v < kAStage / 16; v += 64) {
            const float4 x = hi[v];
            const float4 h = make_float4(tf32_hi(x.x), tf32_hi(x.y), tf32_hi(x.z), tf32_hi(x.w));
            hi[v] = h;
            lo[v] = make_float4(x.x - h.x, x.y - h.y, x.z - h.z, x.w - h.w);
          }
          asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        }
        mbar_arrive(&conv[s]);
      }
    }
  } else {
    // epilogue: TMEM lanes 32 (warp - 4) .. + 31 hold rows j0 + those lanes of the tile
    int64_t tl = 0;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      const int b = (int)(tl & 1);
      if (!mbar_wait(&accf[b], (uint32_t)(tl >> 1) & 1, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int nb = (int)(t % a.NB);
      const int64_t j0 = (t / a.NB) * kBM;
      const int c0 = nb * a.NT;
      const int rl = 32 * (warp - 4) + lane;
      const int64_t j = j0 + rl;
      const bool row_ok = j < a.J;
      int64_t base = 0;
      if (a.ystd && row_ok) {   // standard-layout offset of fiber j (Sec. 2.1 index map, inverted)
        int64_t rem = j;
        for (int m = 0; m < a.N; ++m) {
          if (m == a.n) continue;
          const int64_t im = rem % a.dims[m];
          rem /= a.dims[m];
          base += im * a.st[m];
        }
      }
      const int64_t stn = a.st[a.n];
      for (int cc = 0; cc < a.NT; cc += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp - 4)) << 16) + (uint32_t)(b * 256 + cc);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!row_ok) continue;
        const int cb = c0 + cc;
        if (a.yunf) {
          float* dst = a.yunf + j * a.I + cb;
          if (cb + 16 <= a.I) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              reinterpret_cast<float4*>(dst)[q] =
                  make_float4(__uint_as_float(v[4 * q]), __uint_as_float(v[4 * q + 1]), __uint_as_float(v[4 * q + 2]),
                              __uint_as_float(v[4 * q + 3]));
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q)   // fully unrolled: v stays in registers
              if (cb + q < a.I) dst[q] = __uint_as_float(v[q]);
          }
        }
        if (a.ystd) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (cb + q < a.I) a.ystd[base + (int64_t)(cb + q) * stn] = __uint_as_float(v[q]);
        }
        if (a.ynext) {
          // first pass: row j = (i_2, i_3, ...) with i_2 fastest, column cb + q = i_1; in the
          // column-major mode-2 unfolding that entry sits at i_2 + I_2 (i_1 + I_1 rest), so the lanes
          // of a warp (consecutive i_2) store consecutive addresses for every column
          const int64_t I2 = a.dims[1];
          const int64_t i2 = j % I2, rest = j / I2;
          float* dst = a.ynext + i2 + I2 * ((int64_t)a.I * rest + cb);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (cb + q < a.I) dst[I2 * q] = __uint_as_float(v[q]);
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&acce[b]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
  if (tid == 0 && *err) atomicExch(a.err, 1);
}

constexpr int kStagesA = 4;                     // FP32 U staging ring (refilled as soon as it is converted)
constexpr int kStagesO = 3;                     // operand ring (FP16 halves of U and W, consumed by the MMAs)
constexpr int kA32Stage = kBM * kBK * 4;        // 16 KB: the FP32 U tile as TMA lands it (128B swizzle)
constexpr int kA16Stage = kBM * kBK * 2;        // 8 KB: one FP16 half of the U tile (64B swizzle)
constexpr int kB16Stage = 256 * kBK * 2;        // 16 KB: one FP16 half of the W tile (room for NT = 256)
constexpr int kOpStage = 2 * kA16Stage + 2 * kB16Stage;   // 48 KB
constexpr int kOpOffset = kStagesA * kA32Stage;           // 64 KB
constexpr int kBarOffsetH = kOpOffset + kStagesO * kOpStage;   // 208 KB
constexpr int kTcSmemH = kBarOffsetH + 256 + 1024;
constexpr int kConvWarps = 6;                   // converter warps (8 .. 13)
constexpr int kTcThreadsH = (8 + kConvWarps) * 32;   // 14 warps
constexpr int kWScaleExp = 14;                  // W (|w| <= 1) is stored times 2^14 in FP16

// The same persistent mode-n product with both operands split into FP16 halves and three
// tcgen05.mma kind::f16 per 16 k-values (hi*hi + hi*lo + lo*hi): twice the tensor rate of the TF32
// split at the same accuracy.  U is scaled by 2^ea so that max |U| < 2^14 (ea from *amax_in, the
// largest |entry| of the pass's input), W by 2^14 (pre-split in global memory); the epilogue undoes
// both scalings exactly and, when amax_out is set, records the largest |entry| of the result (the
// next pass's scale).  Two rings: the FP32 U tiles (HBM) land in a 4-deep staging ring that is
// released as soon as they are converted, so their loads run far ahead of the MMAs; the FP16 halves
// of U (written by the converter warps in the 64-byte swizzled layout the MMA reads) and of W (TMA)
// fill a 3-deep operand ring released by the MMAs.
//   warp 0: U producer   warp 1: TMEM owner and MMA issuer   warp 2: W producer
//   warps 4-7: epilogue (TMEM lane quarters 0-3)   warps 8-13: converter   warp 3: idle
__global__ void __launch_bounds__(kTcThreadsH, 1)
    k_mix_tc16(const __grid_constant__ CUtensorMap tmU, const __grid_constant__ CUtensorMap tmWhi,
               const __grid_constant__ CUtensorMap tmWlo, TcArgs a, const unsigned* __restrict__ amax_in,
               unsigned* amax_out) {
  extern __shared__ unsigned char smraw[];
  unsigned char* sm = reinterpret_cast<unsigned char*>((reinterpret_cast<uintptr_t>(smraw) + 1023) & ~(uintptr_t)1023);
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + kBarOffsetH);
  uint64_t* a_full = bars;                        // U tile landed (1 arrival + tx)
  uint64_t* a_empty = a_full + kStagesA;          // U tile converted (one arrival per converter thread)
  uint64_t* w_full = a_empty + kStagesA;          // W halves landed (1 arrival + tx)
  uint64_t* conv = w_full + kStagesO;             // U halves written (one arrival per converter thread)
  uint64_t* o_empty = conv + kStagesO;            // MMAs done with the operand stage (tcgen05.commit)
  uint64_t* accf = o_empty + kStagesO;            // accumulator buffer b complete, 2 buffers
  uint64_t* acce = accf + 2;                      // accumulator buffer b drained (128 arrivals), 2 buffers
  uint64_t* fin = acce + 2;                       // every MMA issued by this CTA complete
  uint32_t* tslot = reinterpret_cast<uint32_t*>(fin + 1);
  volatile int* err = reinterpret_cast<volatile int*>(fin + 2);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t mtiles = (a.J + kBM - 1) / kBM;
  const int64_t ntiles = mtiles * a.NB;
  const int nk = (a.I + kBK - 1) / kBK;
  auto A32 = [&](int s) { return sm + s * kA32Stage; };
  auto A_hi = [&](int s) { return sm + kOpOffset + s * kOpStage; };
  auto A_lo = [&](int s) { return sm + kOpOffset + s * kOpStage + kA16Stage; };
  auto B_hi = [&](int s) { return sm + kOpOffset + s * kOpStage + 2 * kA16Stage; };
  auto B_lo = [&](int s) { return sm + kOpOffset + s * kOpStage + 2 * kA16Stage + kB16Stage; };
  // scale of U: max |U| * 2^ea < 2^14
  int ea = 0;
  {
    const float m = __uint_as_float(*amax_in);
    if (m > 0.f && isfinite(m)) {
      int e;
      frexpf(m, &e);   // m = f 2^e, f in [0.5, 1)
      ea = 14 - e;
    }
  }
  const float uscale = ldexpf(1.f, ea);
  const float oscale = ldexpf(1.f, -(ea + kWScaleExp));

  if (tid == 0) {
    for (int s = 0; s < kStagesA; ++s) {
      mbar_init(&a_full[s], 1);
      mbar_init(&a_empty[s], 32 * kConvWarps);
    }
    for (int s = 0; s < kStagesO; ++s) {
      mbar_init(&w_full[s], 1);
      mbar_init(&conv[s], 32 * kConvWarps);
      mbar_init(&o_empty[s], 1);
    }
    for (int b = 0; b < 2; ++b) {
      mbar_init(&accf[b], 1);
      mbar_init(&acce[b], 128);
    }
    mbar_init(fin, 1);
    *err = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 1) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tslot)), "r"(512));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = *tslot;
  const uint32_t bbytes = (uint32_t)a.NT * kBK * 2;

  if (warp == 0 || warp == 2) {
    if (lane == 0) {   // producers: U tiles (warp 0) and W halves (warp 2), each in its own ring
      const bool isU = warp == 0;
      const int S = isU ? kStagesA : kStagesO;
      uint64_t* fullb = isU ? a_full : w_full;
      uint64_t* emptyb = isU ? a_empty : o_empty;
      int64_t it = 0, issued = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
        const int nb = (int)(t % a.NB);
        const int j0 = (int)((t / a.NB) * kBM);
        const int c0 = nb * a.NT;
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = (int)(it % S);
          const uint32_t use = (uint32_t)(it / S);
          if (it >= S && !mbar_wait(&emptyb[s], (use - 1) & 1, err)) {
            ok = false;
            break;
          }
          if (isU) {
            mbar_expect_tx(&fullb[s], (uint32_t)kA32Stage);
            tma_2d(A32(s), &tmU, i * kBK, j0, &fullb[s]);
          } else {
            mbar_expect_tx(&fullb[s], 2u * bbytes);
            tma_2d(B_hi(s), &tmWhi, i * kBK, c0, &fullb[s]);
            tma_2d(B_lo(s), &tmWlo, i * kBK, c0, &fullb[s]);
          }
          issued = it + 1;
        }
      }
      if (*err) {   // never leave copies in flight: wait (bounded) for the last ones issued
        for (int64_t q = issued > S ? issued - S : 0; q < issued; ++q) {
          const int s = (int)(q % S);
          for (uint32_t w = 0; w < kWaitLimit && !mbar_try(&fullb[s], (uint32_t)(q / S) & 1); ++w) {
          }
        }
      }
    }
  } else if (warp == 1) {
    if (lane == 0) {   // MMA issuer
      const uint32_t idesc = idesc_f16(kBM, a.NT);
      int64_t it = 0, tl = 0;
      bool ok = true;
      for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x, ++tl) {
        const int b = (int)(tl & 1);
        const uint32_t ub = (uint32_t)(tl >> 1);
        if (tl >= 2 && !mbar_wait(&acce[b], (ub - 1) & 1, err)) {
          ok = false;
          break;
        }
        asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
        const uint32_t d = tmem + (uint32_t)(b * 256);
        for (int i = 0; i < nk; ++i, ++it) {
          const int s = (int)(it % kStagesO);
          const uint32_t ph = (uint32_t)(it / kStagesO) & 1;
          if (!mbar_wait(&conv[s], ph, err) || !mbar_wait(&w_full[s], ph, err)) {
            ok = false;
            break;
          }
          asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
          const uint32_t ah = su32(A_hi(s)), al = su32(A_lo(s)), bh = su32(B_hi(s)), bl = su32(B_lo(s));
#pragma unroll
          for (int kk = 0; kk < kBK / 16; ++kk) {
            const uint32_t off = kk * 32;   // 16 FP16 values
            mma_f16(d, sw64_desc(ah + off), sw64_desc(bh + off), idesc, (i | kk) != 0);
            mma_f16(d, sw64_desc(ah + off), sw64_desc(bl + off), idesc, 1u);
            mma_f16(d, sw64_desc(al + off), sw64_desc(bh + off), idesc, 1u);
          }
          mma_commit(&o_empty[s]);
        }
        if (ok) mma_commit(&accf[b]);
      }
      mma_commit(fin);
      for (uint32_t w = 0; w < kWaitLimit && !mbar_try(fin, 0); ++w) {
      }
    }
  } else if (warp >= 8) {
    // converter (32 kConvWarps threads): FP16 halves of the U tile; work item = (row r, FP16 chunk q)
    const int ct = tid - 256;
    int64_t it = 0;
    bool ok = true;
    for (int64_t t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
      for (int i = 0; i < nk; ++i, ++it) {
        const int sa = (int)(it % kStagesA), so = (int)(it % kStagesO);
        if (!mbar_wait(&a_full[sa], (uint32_t)(it / kStagesA) & 1, err) ||
            (it >= kStagesO && !mbar_wait(&o_empty[so], (uint32_t)(it / kStagesO - 1) & 1, err))) {
          ok = false;
          break;
        }
        const unsigned char* src = A32(sa);
        unsigned char* hi = A_hi(so);
        unsigned char* lo = A_lo(so);
#pragma unroll 2
        for (int w = ct; w < kBM * 4; w += 32 * kConvWarps) {
          const int r = w >> 2, q = w & 3;
          // FP32 chunks 2q and 2q+1 of row r in the 128-byte swizzled tile: chunk c sits at c ^ (r & 7)
          const float4 x0 = *reinterpret_cast<const float4*>(src + r * 128 + (((2 * q) ^ (r & 7)) << 4));
          const float4 x1 = *reinterpret_cast<const float4*>(src + r * 128 + (((2 * q + 1) ^ (r & 7)) << 4));
          const float xv[8] = {x0.x * uscale, x0.y * uscale, x0.z * uscale, x0.w * uscale,
                               x1.x * uscale, x1.y * uscale, x1.z * uscale, x1.w * uscale};
          uint32_t hw[4], lw[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const __half2 h2 = __floats2half2_rn(xv[2 * u], xv[2 * u + 1]);
            const float2 hf = __half22float2(h2);
            const __half2 l2 = __floats2half2_rn(xv[2 * u] - hf.x, xv[2 * u + 1] - hf.y);
            hw[u] = *reinterpret_cast<const uint32_t*>(&h2);
            lw[u] = *reinterpret_cast<const uint32_t*>(&l2);
          }
          // FP16 chunk q of row r in the 64-byte swizzled tile sits at q ^ ((r >> 1) & 3)
          const int dst = r * 64 + ((q ^ ((r >> 1) & 3)) << 4);
          *reinterpret_cast<uint4*>(hi + dst) = make_uint4(hw[0], hw[1], hw[2], hw[3]);
          *reinterpret_cast<uint4*>(lo + dst) = make_uint4(lw[0], lw[1], lw[2], lw[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        mbar_arrive(&a_empty[sa]);
        mbar_arrive(&conv[so]);
      }
    }
  } else if (warp >= 4) {
    // epilogue: TMEM lanes 32 (warp - 4) .. + 31 hold rows j0 + those lanes of the tile
    int64_t tl = 0;
    float vmax = 0.f;
    for (int64_t t = blockIdx.x; t < ntiles; t += gridDim.x, ++tl) {
      const int b = (int)(tl & 1);
      if (!mbar_wait(&accf[b], (uint32_t)(tl >> 1) & 1, err)) break;
      asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
      const int nb = (int)(t % a.NB);
      const int64_t j0 = (t / a.NB) * kBM;
      const int c0 = nb * a.NT;
      const int rl = 32 * (warp - 4) + lane;
      const int64_t j = j0 + rl;
      const bool row_ok = j < a.J;
      int64_t base = 0;
      if (a.ystd && row_ok) {
        int64_t rem = j;
        for (int m = 0; m < a.N; ++m) {
          if (m == a.n) continue;
          const int64_t im = rem % a.dims[m];
          rem /= a.dims[m];
          base += im * a.st[m];
        }
      }
      const int64_t stn = a.st[a.n];
      for (int cc = 0; cc < a.NT; cc += 16) {
        uint32_t v[16];
        const uint32_t taddr = tmem + ((uint32_t)(32 * (warp - 4)) << 16) + (uint32_t)(b * 256 + cc);
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
              "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(taddr));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (!row_ok) continue;
        const int cb = c0 + cc;
        float y[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          y[q] = __uint_as_float(v[q]) * oscale;
          if (cb + q < a.I) vmax = fmaxf(vmax, fabsf(y[q]));
        }
        if (a.yunf) {
          float* dst = a.yunf + j * a.I + cb;
          if (cb + 16 <= a.I) {
#pragma unroll
            for (int q = 0; q < 4; ++q)
              reinterpret_cast<float4*>(dst)[q] = make_float4(y[4 * q], y[4 * q + 1], y[4 * q + 2], y[4 * q + 3]);
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q)   // fully unrolled: y stays in registers
              if (cb + q < a.I) dst[q] = y[q];
          }
        }
        if (a.ystd) {
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (cb + q < a.I) a.ystd[base + (int64_t)(cb + q) * stn] = y[q];
        }
        if (a.ynext) {
          const int64_t I2 = a.dims[1];
          const int64_t i2 = j % I2, rest = j / I2;
          float* dst = a.ynext + i2 + I2 * ((int64_t)a.I * rest + cb);
#pragma unroll
          for (int q = 0; q < 16; ++q)
            if (cb + q < a.I) dst[I2 * q] = y[q];
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
      mbar_arrive(&acce[b]);
    }
    if (amax_out) {   // the largest |entry| of the result: the next pass's scale
      const unsigned m = __reduce_max_sync(0xffffffffu, __float_as_uint(vmax));
      if (lane == 0 && m) atomicMax(amax_out, m);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 1) {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(512));
  }
  if (tid == 0 && *err) atomicExch(a.err, 1);
}

// W (FP32, |w| <= 1) times 2^14 as FP16 halves: hi in out[0, n), lo in out[n, 2n).
__global__ void k_split_f16(const float* __restrict__ w, __half* __restrict__ out, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  __half h, l;
  split_f16(ldexpf(w[i], kWScaleExp), h, l);
  out[i] = h;
  out[n + i] = l;
}

// Largest |x| over a tensor (as the bit pattern of a non-negative float, for atomicMax).
template <typename T>
__global__ void __launch_bounds__(256) k_absmax(const T* __restrict__ X, int64_t P, unsigned* out) {
  float m = 0.f;
  for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P; i += (int64_t)gridDim.x * blockDim.x) {
    float x;
    if constexpr (sizeof(T) == 2) x = __bfloat162float(X[i]);
    else x = (float)X[i];
    m = fmaxf(m, fabsf(x));
  }
  const unsigned r = __reduce_max_sync(0xffffffffu, __float_as_uint(m));
  if ((threadIdx.x & 31) == 0 && r) atomicMax(out, r);
}

__global__ void k_split_tf32(const float* __restrict__ w, float* __restrict__ hi, float* __restrict__ lo, int64_t n) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float x = w[i];
  const float h = tf32_hi(x);
  hi[i] = h;
  lo[i] = x - h;
}

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

EncodeTiledFn encode_fn() {
  static std::once_flag once;
  static EncodeTiledFn fn = nullptr;
  std::call_once(once, []() {
    void* p = nullptr;
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) == cudaSuccess &&
        q == cudaDriverEntryPointSuccess)
      fn = reinterpret_cast<EncodeTiledFn>(p);
  });
  return fn;
}

// 2D fp32 tensor map: rows of `inner` contiguous floats, `outer` rows, box {32, box_rows}, 128B swizzle.
bool make_map(CUtensorMap* m, const float* base, int64_t inner, int64_t outer, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * 4};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// 2D FP16 tensor map: rows of `inner` contiguous halves, `outer` rows, box {32, box_rows}, 64B swizzle.
bool make_map16(CUtensorMap* m, const __half* base, int64_t inner, int64_t outer, int box_rows) {
  EncodeTiledFn fn = encode_fn();
  if (!fn) return false;
  const cuuint64_t dims[2] = {(cuuint64_t)inner, (cuuint64_t)outer};
  const cuuint64_t strides[1] = {(cuuint64_t)inner * 2};
  const cuuint32_t box[2] = {(cuuint32_t)kBK, (cuuint32_t)box_rows};
  const cuuint32_t estr[2] = {1, 1};
  return fn(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, const_cast<__half*>(base), dims, strides, box, estr,
            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_64B, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

}  // namespace

bool mix_tc16_supported(int dtype, int I) {
  return dtype == CPR_F32 && I >= 1 && I % 8 == 0 && encode_fn() != nullptr;
}

cudaError_t launch_split_f16(const float* w, void* out16, int64_t n, cudaStream_t s) {
  k_split_f16<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, static_cast<__half*>(out16), n);
  return cudaGetLastError();
}

cudaError_t launch_absmax(const void* X, int dtype, int64_t P, unsigned* out, cudaStream_t s) {
  int dev = 0, sms = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
    sms = 1;
  int64_t blocks = (P + 255) / 256;   // grid-stride: eight blocks per SM at most
  if (blocks > (int64_t)sms * 8) blocks = (int64_t)sms * 8;
  if (blocks < 1) blocks = 1;
  switch (dtype) {
    case CPR_F64: k_absmax<double><<<(unsigned)blocks, 256, 0, s>>>((const double*)X, P, out); break;
    case CPR_F32: k_absmax<float><<<(unsigned)blocks, 256, 0, s>>>((const float*)X, P, out); break;
    default: k_absmax<__nv_bfloat16><<<(unsigned)blocks, 256, 0, s>>>((const __nv_bfloat16*)X, P, out);
  }
  return cudaGetLastError();
}

cudaError_t launch_mix_tc16(const float* U, float* ystd, float* yunf, float* ynext, const void* W16, int N,
                            const int64_t* dims, int n, const unsigned* amax_in, unsigned* amax_out, int* err,
                            cudaStream_t s) {
  if (ynext && n != 0) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mix_tc16, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmemH);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  TcArgs a;
  memset(&a, 0, sizeof(a));
  int64_t P = 1, st = 1;
  for (int m = 0; m < N; ++m) {
    a.dims[m] = dims[m];
    a.st[m] = st;
    st *= dims[m];
    P *= dims[m];
  }
  const int I = (int)dims[n];
  a.I = I;
  a.J = P / I;
  a.NB = (I + 255) / 256;
  a.NT = ((I + a.NB - 1) / a.NB + 15) / 16 * 16;
  a.three_x = 1;
  a.n = n;
  a.N = N;
  a.ystd = ystd;
  a.yunf = yunf;
  a.ynext = ynext;
  a.err = err;
  const __half* Wh = static_cast<const __half*>(W16);
  CUtensorMap mU, mH, mL;
  if (!make_map(&mU, U, I, a.J, kBM) || !make_map16(&mH, Wh, I, I, a.NT) ||
      !make_map16(&mL, Wh + (int64_t)I * I, I, I, a.NT))
    return cudaErrorInvalidValue;
  if (a.J > INT32_MAX) return cudaErrorInvalidValue;
  const int64_t tiles = ((a.J + kBM - 1) / kBM) * a.NB;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                     cudaSuccess)
      sms = 148;
  }
  const int64_t blocks = tiles < sms ? tiles : sms;
  k_mix_tc16<<<(unsigned)blocks, kTcThreadsH, kTcSmemH, s>>>(mU, mH, mL, a, amax_in, amax_out);
  return cudaGetLastError();
}

bool mix_tc_supported(int dtype, int I) { return dtype == CPR_F32 && I >= 1 && I % 4 == 0 && encode_fn() != nullptr; }

cudaError_t launch_split_tf32(const float* w, float* hi, float* lo, int64_t n, cudaStream_t s) {
  k_split_tf32<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(w, hi, lo, n);
  return cudaGetLastError();
}

cudaError_t launch_mix_tc(const float* U, float* ystd, float* yunf, float* ynext, const float* Whi, const float* Wlo,
                          int N, const int64_t* dims, int n, int three_x, int* err, cudaStream_t s) {
  if (ynext && n != 0) return cudaErrorInvalidValue;
  static bool attr = false;
  if (!attr) {
    cudaError_t e = cudaFuncSetAttribute(k_mix_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, kTcSmem);
    if (e != cudaSuccess) return e;
    attr = true;
  }
  TcArgs a;
  memset(&a, 0, sizeof(a));
  int64_t P = 1, st = 1;
  for (int m = 0; m < N; ++m) {
    a.dims[m] = dims[m];
    a.st[m] = st;
    st *= dims[m];
    P *= dims[m];
  }
  const int I = (int)dims[n];
  a.I = I;
  a.J = P / I;
  a.NB = (I + 255) / 256;
  a.NT = ((I + a.NB - 1) / a.NB + 15) / 16 * 16;
  a.three_x = three_x;
  a.n = n;
  a.N = N;
  a.ystd = ystd;
  a.yunf = yunf;
  a.ynext = ynext;
  a.err = err;
  CUtensorMap mU, mH, mL;
  if (!make_map(&mU, U, I, a.J, kBM) || !make_map(&mH, Whi, I, I, a.NT) || !make_map(&mL, Wlo, I, I, a.NT))
    return cudaErrorInvalidValue;
  const int64_t mtiles = (a.J + kBM - 1) / kBM;
  const int64_t tiles = mtiles * a.NB;
  if (a.J > INT32_MAX) return cudaErrorInvalidValue;
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                     cudaSuccess)
      sms = 148;
  }
  const int64_t blocks = tiles < sms ? tiles : sms;   // one persistent CTA per SM
  k_mix_tc<<<(unsigned)blocks, kTcThreads, kTcSmem, s>>>(mU, mH, mL, a);
  return cudaGetLastError();
}

}  // namespace cpr
