// Kernels of CP-ALS (Alg. 1): the exact mode-n update A^(n) = X_(n) Z^(n) (*_{m!=n} A^(m)T A^(m))^-1
// followed by column normalization, and the exact fit of Sec. 4.2 from Gram identities.
//
// Per mode n (one problem per call):
//   k_als_prep     V = Hadamard product of the other modes' Grams (Sec. 2.1: the Gram of the
//                  Khatri-Rao product Z^(n)), Cholesky V = L L^T in FP64; a non-positive pivot stops
//                  the run with CPR_ESINGULAR
//   k_mttkrp       M = X_(n) Z^(n) over the column-major unfolding copy X_(n) (i_n fastest): a CTA
//                  owns TI rows and a range of unfolding columns; the Z rows of a tile of columns are
//                  built on the fly from the factor rows (never the whole Khatri-Rao matrix);
//                  products in FP32 with FP32 sums over at most kMtFlush columns folded into FP64
//                  (FP64 throughout for an FP64 tensor); partial M per column split in FP64
//   k_mttkrp_fold  M = sum of the split partials in a fixed order, many blocks
//   k_als_solve    a_i L L^T = m_i in FP64 for the rows m_i of M, rows
//                  stored unnormalized; partial Grams of the new rows; the last block forms the
//                  Gram of the new factor, lambda, the lazy column scales and, after the last
//                  mode, the exact fit and the stopping rules
// The exact fit needs no pass over X:  ||X - X~||^2 = ||X||^2 - 2 <X, X~> + ||X~||^2 with
// <X, X~> = sum_{i,r} M_N(i,r) A_N(i,r) (A_N unnormalized, M_N the last mode's MTTKRP) and
// ||X~||^2 = sum_{r,s} V_N(r,s) (A_N^T A_N)(r,s), both available in the last mode update.
#include <math.h>

#include "internal.cuh"

namespace cpr {

constexpr int kAlsThreads = 128;
constexpr int kMtFlush = 256;     // FP32 partial sums of the MTTKRP span at most this many columns

int mttkrp_rank_groups(int R) {
  const int g = (R + 7) / 8;
  return g <= 1 ? 1 : (g <= 2 ? 2 : (g <= 4 ? 4 : 8));
}

// Thread tile: 4 rows x 8 rank columns; 128 threads = (TI / 4) row groups x RG rank groups.
// A tile of the unfolding holds TE = TI x JT entries (2048 FP32 / 1024 FP64).
template <typename ACC, int RG>
struct MtShape {
  static constexpr int ROWG = kAlsThreads / RG;
  static constexpr int TI = ROWG * 4;
  static constexpr int TE = sizeof(ACC) == 8 ? 1024 : 2048;
  static constexpr int JT = TE / TI;
  static constexpr int RP = 8 * RG;
  static constexpr int LPT = TE / kAlsThreads;    // tile entries each thread loads
};

int mttkrp_tile_rows(int rg, int) { return 4 * (kAlsThreads / rg); }
int mttkrp_tile_cols(int rg, int dtype) { return (dtype == CPR_F64 ? 1024 : 2048) / mttkrp_tile_rows(rg, dtype); }

template <typename ACC, typename T> __device__ __forceinline__ ACC to_acc(T v);
template <> __device__ __forceinline__ double to_acc<double, double>(double v) { return v; }
template <> __device__ __forceinline__ float to_acc<float, float>(float v) { return v; }
template <> __device__ __forceinline__ float to_acc<float, __nv_bfloat16>(__nv_bfloat16 v) { return __bfloat162float(v); }

// Z rows of a column tile (Z(j, r) = w_r prod_{m != n} A^(m)(j_m, r), (j_m) the multi-index of
// unfolding column j under the Sec. 2.1 index map: modes other than n in increasing order, the
// earliest fastest; w_r the product of those modes' lazy column scales).  Thread t owns column
// jj = t / TPC of every tile and EPT consecutive rank columns of it; it keeps the multi-index of its
// column and advances it by JT columns per tile (digit-wise addition with carry), so no division
// runs per entry.
template <typename ACC, int JT, int RP>
struct ZBuilder {
  static constexpr int TPC = kAlsThreads / JT;              // threads per column
  static constexpr int EPT = RP >= TPC ? RP / TPC : 1;      // rank columns per thread
  int jj, r0;
  bool active;
  int nm;                       // modes other than n
  uint32_t idx[kMaxOrder - 1];  // multi-index of column jb + k JT + jj over those modes
  uint32_t ext[kMaxOrder - 1];
  const ACC* rows[kMaxOrder - 1];

  __device__ void init(const Prob& p, int n, int64_t jfirst) {
    const int t = threadIdx.x;
    jj = t / TPC;
    r0 = (t % TPC) * EPT;
    active = r0 < RP;
    nm = 0;
    int64_t rem = jfirst + jj;
    for (int m = 0; m < p.N; ++m) {
      if (m == n) continue;
      const int64_t Im = p.dims[m];
      idx[nm] = (uint32_t)(rem % Im);
      rem /= Im;
      ext[nm] = (uint32_t)Im;
      if constexpr (sizeof(ACC) == 8) rows[nm] = p.A64[m];
      else rows[nm] = p.A32[m];
      ++nm;
    }
  }
  // writes the tile's Z rows (zero where j >= je or r >= R), then advances to the next tile
  __device__ void build(int64_t j0, int64_t je, int R, const ACC* w, ACC* Zs) {
    if (active) {
      const bool live = j0 + jj < je;
      ACC z[EPT];
#pragma unroll
      for (int c = 0; c < EPT; ++c) z[c] = (live && r0 + c < R) ? w[r0 + c] : (ACC)0;
      if (live) {
        for (int q = 0; q < nm; ++q) {
          const ACC* row = rows[q] + (int64_t)idx[q] * R + r0;
#pragma unroll
          for (int c = 0; c < EPT; ++c)
            if (r0 + c < R) z[c] *= row[c];
        }
      }
#pragma unroll
      for (int c = 0; c < EPT; ++c) Zs[jj * RP + r0 + c] = z[c];
    }
    uint32_t carry = JT;
    for (int q = 0; q < nm && carry; ++q) {
      const uint32_t v = idx[q] + carry;
      idx[q] = v % ext[q];
      carry = v / ext[q];
    }
  }
};

template <typename T, typename ACC, int RG>
__global__ void __launch_bounds__(kAlsThreads, 3) k_mttkrp(const Prob* probs, int n) {
  using Sh = MtShape<ACC, RG>;
  constexpr int TI = Sh::TI, JT = Sh::JT, RP = Sh::RP, ROWG = Sh::ROWG, LPT = Sh::LPT;
  constexpr int kFlushTiles = kMtFlush / JT > 0 ? kMtFlush / JT : 1;
  const Prob& p = probs[blockIdx.z];
  if (n >= p.N || is_done(p)) return;
  const int R = p.R;
  const int64_t I = p.dims[n];
  const int64_t J = p.P / I;
  const int64_t i0 = (int64_t)blockIdx.x * TI;
  const int sidx = blockIdx.y;
  if (i0 >= I || sidx >= p.als_nsplit[n]) return;
  const int64_t jb = (int64_t)sidx * p.jsplit[n];
  const int64_t je = min(J, jb + p.jsplit[n]);
  const T* __restrict__ Y = reinterpret_cast<const T*>(p.Xrep[n]);

  __shared__ __align__(16) ACC Ys[2][JT * TI];
  __shared__ __align__(16) ACC Zs[2][JT * RP];
  __shared__ ACC w[RP];
  const int tid = threadIdx.x;
  for (int r = tid; r < RP; r += kAlsThreads) {
    double v = 1.0;
    if (r < R)
      for (int m = 0; m < p.N; ++m)
        if (m != n) v *= p.scale[m][r];
    w[r] = (ACC)v;
  }
  const int g = tid % ROWG, h = tid / ROWG;
  ACC acc[4][8];
  double dacc[4][8];
#pragma unroll
  for (int a = 0; a < 4; ++a)
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      acc[a][c] = (ACC)0;
      dacc[a][c] = 0.0;
    }
  const int64_t ntile = je > jb ? (je - jb + JT - 1) / JT : 0;
  T ld[LPT];
  auto issue = [&](int64_t k) {
    const int64_t j0 = jb + k * JT;
    const T* Yt = Y + j0 * I + i0;
#pragma unroll
    for (int q = 0; q < LPT; ++q) {
      const int e = tid + q * kAlsThreads;
      const int jj = e / TI, ii = e - jj * TI;
      ld[q] = (j0 + jj < je && i0 + ii < I) ? Yt[(int64_t)jj * I + ii] : T(0.0f);
    }
  };
  ZBuilder<ACC, JT, RP> zb;
  zb.init(p, n, jb);
  auto commit = [&](int64_t k, int buf) {
#pragma unroll
    for (int q = 0; q < LPT; ++q) Ys[buf][tid + q * kAlsThreads] = to_acc<ACC, T>(ld[q]);
    zb.build(jb + k * JT, je, R, w, Zs[buf]);
  };
  __syncthreads();   // w ready
  if (ntile > 0) {
    issue(0);
    commit(0, 0);
  }
  __syncthreads();
  for (int64_t k = 0; k < ntile; ++k) {
    const int cur = (int)(k & 1);
    if (k + 1 < ntile) issue(k + 1);
    const ACC* ys = Ys[cur];
    const ACC* zs = Zs[cur];
#pragma unroll 4
    for (int jj = 0; jj < JT; ++jj) {
      ACC y[4], z[8];
      if constexpr (sizeof(ACC) == 4) {
        const float4 y4 = *reinterpret_cast<const float4*>(&ys[jj * TI + 4 * g]);
        const float4 za = *reinterpret_cast<const float4*>(&zs[jj * RP + 8 * h]);
        const float4 zb = *reinterpret_cast<const float4*>(&zs[jj * RP + 8 * h + 4]);
        y[0] = y4.x; y[1] = y4.y; y[2] = y4.z; y[3] = y4.w;
        z[0] = za.x; z[1] = za.y; z[2] = za.z; z[3] = za.w;
        z[4] = zb.x; z[5] = zb.y; z[6] = zb.z; z[7] = zb.w;
      } else {
#pragma unroll
        for (int a = 0; a < 4; ++a) y[a] = ys[jj * TI + 4 * g + a];
#pragma unroll
        for (int c = 0; c < 8; ++c) z[c] = zs[jj * RP + 8 * h + c];
      }
#pragma unroll
      for (int a = 0; a < 4; ++a)
#pragma unroll
        for (int c = 0; c < 8; ++c) acc[a][c] = fma(y[a], z[c], acc[a][c]);
    }
    if constexpr (sizeof(ACC) == 4) {
      if ((k + 1) % kFlushTiles == 0) {
#pragma unroll
        for (int a = 0; a < 4; ++a)
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            dacc[a][c] += (double)acc[a][c];
            acc[a][c] = 0.0f;
          }
      }
    }
    if (k + 1 < ntile) commit(k + 1, cur ^ 1);
    __syncthreads();
  }
  double* Mp = reinterpret_cast<double*>(p.Mpart) + (int64_t)sidx * p.imax * R;
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int64_t i = i0 + 4 * g + a;
    if (i >= I) continue;
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const int r = 8 * h + c;
      if (r < R) Mp[i * R + r] = dacc[a][c] + (double)acc[a][c];
    }
  }
}

template <typename T, typename ACC>
static cudaError_t mttkrp_go(const Prob* probs, const Prob& hp, int n, cudaStream_t s) {
  const int rg = hp.als_rg;
  const int TI = mttkrp_tile_rows(rg, hp.dtype);
  const dim3 grid((unsigned)((hp.dims[n] + TI - 1) / TI), (unsigned)hp.als_nsplit[n], 1);
  switch (rg) {
    case 1: k_mttkrp<T, ACC, 1><<<grid, kAlsThreads, 0, s>>>(probs, n); break;
    case 2: k_mttkrp<T, ACC, 2><<<grid, kAlsThreads, 0, s>>>(probs, n); break;
    case 4: k_mttkrp<T, ACC, 4><<<grid, kAlsThreads, 0, s>>>(probs, n); break;
    default: k_mttkrp<T, ACC, 8><<<grid, kAlsThreads, 0, s>>>(probs, n);
  }
  return cudaGetLastError();
}

cudaError_t launch_mttkrp(const Prob* probs, const Prob& hp, int n, cudaStream_t s) {
  switch (hp.dtype) {
    case CPR_F64: return mttkrp_go<double, double>(probs, hp, n, s);
    case CPR_F32: return mttkrp_go<float, float>(probs, hp, n, s);
    default: return mttkrp_go<__nv_bfloat16, float>(probs, hp, n, s);
  }
}

// ------------------------------------------------------------------------------------------------
// V = *_{m != n} Gram_m and its Cholesky factor (one block per problem).
// ------------------------------------------------------------------------------------------------
__global__ void k_als_prep(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.x];
  if (n >= p.N || is_done(p)) return;
  extern __shared__ double G[];
  const int R = p.R;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    double v = 1.0;
    for (int m = 0; m < p.N; ++m)
      if (m != n) v *= p.gram[m][e];
    G[e] = v;
    p.V[e] = v;
  }
  __syncthreads();
  const bool ok = block_cholesky(G, R);
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) p.L[e] = G[e];
  if (!ok && threadIdx.x == 0) {
    p.state->status = CPR_ESINGULAR;
    p.state->done = 1;
  }
}

cudaError_t launch_als_prep(const Prob* probs, const Prob& hp, int n, cudaStream_t s) {
  k_als_prep<<<1, 256, (size_t)hp.R * hp.R * sizeof(double), s>>>(probs, n);
  return cudaGetLastError();
}

// Partial Gram of the block's rows (rows x R in shared memory, row stride R1): upper triangle
// (r <= c) into out[r * R + c].
__device__ __forceinline__ void rows_gram(const double* Vr, int rows, int R, int R1, double* out) {
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    if (c < r) continue;
    double s0 = 0.0, s1 = 0.0;
    int li = 0;
    for (; li + 2 <= rows; li += 2) {
      s0 = fma(Vr[li * R1 + r], Vr[li * R1 + c], s0);
      s1 = fma(Vr[(li + 1) * R1 + r], Vr[(li + 1) * R1 + c], s1);
    }
    if (li < rows) s0 = fma(Vr[li * R1 + r], Vr[li * R1 + c], s0);
    out[e] = s0 + s1;
  }
}

// Last block of a mode: sum the nrb partial Grams in a fixed order into Gun (shared, R x R, both
// triangles), then lambda_r = sqrt(Gun_rr), the lazy scales and the normalized Gram of mode n.
__device__ void finish_gram(const Prob& p, int n, int nrb, double* Gun, bool set_lambda) {
  const int R = p.R;
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    if (c < r) continue;
    double a0 = 0.0, a1 = 0.0, a2 = 0.0, a3 = 0.0;
    int q = 0;
    for (; q + 4 <= nrb; q += 4) {
      a0 += __ldcg(&p.Gpart[(int64_t)(q + 0) * R * R + e]);
      a1 += __ldcg(&p.Gpart[(int64_t)(q + 1) * R * R + e]);
      a2 += __ldcg(&p.Gpart[(int64_t)(q + 2) * R * R + e]);
      a3 += __ldcg(&p.Gpart[(int64_t)(q + 3) * R * R + e]);
    }
    for (; q < nrb; ++q) a0 += __ldcg(&p.Gpart[(int64_t)q * R * R + e]);
    const double v = (a0 + a1) + (a2 + a3);
    Gun[r * R + c] = v;
    Gun[c * R + r] = v;
  }
  __syncthreads();
  for (int r = threadIdx.x; r < R; r += blockDim.x) {
    const double nrm = sqrt(Gun[r * R + r]);
    if (set_lambda) p.lambda[r] = nrm;
    p.scale[n][r] = nrm > 0.0 ? 1.0 / nrm : 1.0;
  }
  __syncthreads();
  for (int e = threadIdx.x; e < R * R; e += blockDim.x) {
    const int r = e / R, c = e - r * R;
    p.gram[n][e] = Gun[e] * p.scale[n][r] * p.scale[n][c];
  }
}

// Gram of a factor as it stands (initial factors): partial Grams of kAlsRows rows per block, the
// last block normalizes (lambda untouched).
__global__ void __launch_bounds__(kAlsThreads) k_als_gram(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.y];
  if (n >= p.N) return;
  const int R = p.R, R1 = R + 1;
  const int64_t I = p.dims[n];
  const int64_t i0 = (int64_t)blockIdx.x * kAlsRows;
  if (i0 >= I) return;
  const int nrb = (int)((I + kAlsRows - 1) / kAlsRows);
  const int rows = (int)min((int64_t)kAlsRows, I - i0);
  extern __shared__ double sm[];
  double* Vr = sm;                      // kAlsRows x R1
  double* Gun = sm + kAlsRows * R1;     // R x R
  for (int e = threadIdx.x; e < rows * R; e += blockDim.x) {
    const int li = e / R, r = e - li * R;
    Vr[li * R1 + r] = p.A64[n][(i0 + li) * R + r];
  }
  __syncthreads();
  rows_gram(Vr, rows, R, R1, p.Gpart + (int64_t)blockIdx.x * R * R);
  if (!arrive_last(p.state, (uint32_t)nrb)) return;
  finish_gram(p, n, nrb, Gun, false);
}

cudaError_t launch_als_gram(const Prob* probs, const Prob& hp, int n, cudaStream_t s) {
  const int R = hp.R;
  const size_t smem = ((size_t)kAlsRows * (R + 1) + (size_t)R * R) * sizeof(double);
  const dim3 grid((unsigned)((hp.dims[n] + kAlsRows - 1) / kAlsRows), 1);
  k_als_gram<<<grid, kAlsThreads, smem, s>>>(probs, n);
  return cudaGetLastError();
}

// M = sum over splits of the MTTKRP partials, in a fixed order: a block owns 32 consecutive entries
// of M (one per lane); warp w sums the splits s = w, w + kFoldWarps, ... (coalesced 256-byte reads),
// then the warp sums are added in warp order.
constexpr int kFoldWarps = 16;
__global__ void __launch_bounds__(32 * kFoldWarps) k_mttkrp_fold(const Prob* probs, int n, double* M) {
  const Prob& p = probs[blockIdx.y];
  if (n >= p.N || is_done(p)) return;
  const int64_t cnt = p.dims[n] * p.R;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t e = (int64_t)blockIdx.x * 32 + lane;
  const double* Mp = reinterpret_cast<const double*>(p.Mpart);
  const int ns = p.als_nsplit[n];
  const int64_t stride = (int64_t)p.imax * p.R;
  __shared__ double part[kFoldWarps][32];
  double a0 = 0.0, a1 = 0.0;
  if (e < cnt) {
    int s = w;
    for (; s + kFoldWarps < ns; s += 2 * kFoldWarps) {
      a0 += Mp[s * stride + e];
      a1 += Mp[(s + kFoldWarps) * stride + e];
    }
    if (s < ns) a0 += Mp[s * stride + e];
  }
  part[w][lane] = a0 + a1;
  __syncthreads();
  if (w == 0 && e < cnt) {
    double t = 0.0;
#pragma unroll
    for (int q = 0; q < kFoldWarps; ++q) t += part[q][lane];
    M[e] = t;
  }
}

cudaError_t launch_mttkrp_fold(const Prob* probs, const Prob& hp, int n, double* M, cudaStream_t s) {
  const int64_t cnt = hp.dims[n] * hp.R;
  k_mttkrp_fold<<<dim3((unsigned)((cnt + 31) / 32), 1), 32 * kFoldWarps, 0, s>>>(probs, n, M ? M : hp.Mfold);
  return cudaGetLastError();
}

// Rows [i0, i0 + kAlsRows) of the new factor: m_i = the folded MTTKRP row, a_i = m_i (L L^T)^-1
// by forward and backward substitution (FP64), stored unnormalized (FP64 and FP32).  Partial Gram
// and partial <M, A> of the block; the last block finishes the Gram, lambda and scales and, for
// the last mode, the exact fit and the stopping rules.
__global__ void __launch_bounds__(kAlsThreads) k_als_solve(const Prob* probs, int n) {
  const Prob& p = probs[blockIdx.y];
  if (n >= p.N || is_done(p)) return;
  const int R = p.R, R1 = R + 1;
  const int64_t I = p.dims[n];
  const int64_t i0 = (int64_t)blockIdx.x * kAlsRows;
  if (i0 >= I) return;
  const int nrb = (int)((I + kAlsRows - 1) / kAlsRows);
  const int rows = (int)min((int64_t)kAlsRows, I - i0);
  extern __shared__ double sm[];
  double* Ls = sm;                        // R x R1
  double* Vr = Ls + R * R1;               // kAlsRows x R1: solved rows
  double* Mr = Vr + kAlsRows * R1;        // kAlsRows x R1: MTTKRP rows
  double* Gun = Mr + kAlsRows * R1;       // R x R
  __shared__ double red[kAlsThreads / 32];
  const int tid = threadIdx.x;
  for (int e = tid; e < R * R; e += blockDim.x) Ls[(e / R) * R1 + e % R] = p.L[e];
  for (int e = tid; e < rows * R; e += blockDim.x) {
    const int li = e / R, r = e - li * R;
    const double m = p.Mfold[(i0 + li) * R + r];
    Mr[li * R1 + r] = m;
    Vr[li * R1 + r] = m;
  }
  __syncthreads();
  if (tid < rows) {
    double* v = Vr + tid * R1;
    for (int k = 0; k < R; ++k) {
      double s = v[k];
      for (int l = 0; l < k; ++l) s -= Ls[k * R1 + l] * v[l];
      v[k] = s / Ls[k * R1 + k];
    }
    for (int k = R - 1; k >= 0; --k) {
      double s = v[k];
      for (int l = k + 1; l < R; ++l) s -= Ls[l * R1 + k] * v[l];
      v[k] = s / Ls[k * R1 + k];
    }
  }
  __syncthreads();
  double* A = p.A64[n] + i0 * R;
  float* A32 = p.A32[n] + i0 * R;
  double inner = 0.0;
  for (int e = tid; e < rows * R; e += blockDim.x) {
    const int li = e / R, r = e - li * R;
    const double v = Vr[li * R1 + r];
    A[e] = v;
    A32[e] = (float)v;
    inner = fma(Mr[li * R1 + r], v, inner);
  }
  rows_gram(Vr, rows, R, R1, p.Gpart + (int64_t)blockIdx.x * R * R);
  for (int o = 16; o > 0; o >>= 1) inner += __shfl_down_sync(0xffffffffu, inner, o);
  if ((tid & 31) == 0) red[tid >> 5] = inner;
  __syncthreads();
  if (tid == 0) {
    double t = 0.0;
    for (int q = 0; q < kAlsThreads / 32; ++q) t += red[q];
    p.Npart[blockIdx.x] = t;
  }
  if (!arrive_last(p.state, (uint32_t)nrb)) return;
  finish_gram(p, n, nrb, Gun, true);
  if (n != p.N - 1) return;
  // exact fit after the last mode of the outer iteration
  __syncthreads();
  double xt = 0.0, in = 0.0;
  for (int e = tid; e < R * R; e += blockDim.x) xt = fma(Gun[e], p.V[e], xt);
  for (int q = tid; q < nrb; q += blockDim.x) in += __ldcg(&p.Npart[q]);
  __shared__ double r2[2][kAlsThreads / 32];
  for (int o = 16; o > 0; o >>= 1) {
    xt += __shfl_down_sync(0xffffffffu, xt, o);
    in += __shfl_down_sync(0xffffffffu, in, o);
  }
  if ((tid & 31) == 0) {
    r2[0][tid >> 5] = xt;
    r2[1][tid >> 5] = in;
  }
  __syncthreads();
  if (tid == 0) {
    double sxt = 0.0, sin = 0.0;
    for (int q = 0; q < kAlsThreads / 32; ++q) {
      sxt += r2[0][q];
      sin += r2[1][q];
    }
    State* st = p.state;
    const double nx = st->norm_x;
    const double res2 = nx * nx - 2.0 * sin + sxt;
    const double fit = 1.0 - sqrt(fmax(res2, 0.0)) / nx;
    apply_stop_rules(p, st, fit);
  }
}

cudaError_t launch_als_solve(const Prob* probs, const Prob& hp, int n, cudaStream_t s) {
  const int R = hp.R, R1 = R + 1;
  const size_t smem = ((size_t)R * R1 + 2 * (size_t)kAlsRows * R1 + (size_t)R * R) * sizeof(double);
  const dim3 grid((unsigned)((hp.dims[n] + kAlsRows - 1) / kAlsRows), 1);
  k_als_solve<<<grid, kAlsThreads, smem, s>>>(probs, n);
  return cudaGetLastError();
}

cudaError_t prepare_als_attributes() {
  const int R = kMaxRank, R1 = R + 1;
  const size_t solve = ((size_t)R * R1 + 2 * (size_t)kAlsRows * R1 + (size_t)R * R) * sizeof(double);
  const size_t gram = ((size_t)kAlsRows * R1 + (size_t)R * R) * sizeof(double);
  cudaError_t e = cudaFuncSetAttribute(k_als_solve, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)solve);
  if (e != cudaSuccess) return e;
  return cudaFuncSetAttribute(k_als_gram, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)gram);
}

}  // namespace cpr
