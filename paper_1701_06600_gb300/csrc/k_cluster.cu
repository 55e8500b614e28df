// The whole outer-iteration loop of CPRAND (Alg. 3 with the stopping test of Sec. 3.4 / 4.2) for
// problems small enough to live in one thread-block cluster.
//
// One cluster of C CTAs owns one problem at a time (a persistent scheduler hands out problems of a
// batch through a global counter).  Per mode n:
//   * CTA c draws samples [c*spc, (c+1)*spc) (Philox stream 0), builds their Z_S rows (Alg. 2) and
//     contracts its sampled fibers against them for EVERY row i_n: a partial M_c = X_S,c Z_S,c
//     (FP32 accumulation; FP64 for FP64 tensors) and a partial FP64 Gram, both in its own shared
//     memory.
//   * cluster barrier; every CTA sums the C partial Grams through distributed shared memory in a
//     fixed order and Cholesky-factors G (all CTAs get bit-identical factors and the same
//     singularity verdict); CTA c sums the partial M rows of its share of the rows, solves them in
//     FP64 (one warp per row) and writes them to global memory; column sums of squares per CTA.
//   * cluster barrier; every CTA sums the column partials: lambda and the lazy column scales.
// After the N modes, CTA c evaluates its share of the P_hat fit entries; after a cluster barrier
// every CTA sums the C partials in the same order and applies the stopping rules to its own copy of
// the loop state, so every CTA takes the same decision and all of them execute the same sequence of
// cluster barriers.  CTA 0 publishes the fit trace and the state.
#include <cooperative_groups.h>
#include <math.h>

#include "internal.cuh"
#include "small_spd.cuh"

namespace cg = cooperative_groups;

namespace cpr {

constexpr int kCT = 512;   // threads per CTA of the cluster kernel

struct ClusterSmem {       // offsets (bytes) into the dynamic shared memory
  int sc, lam, wr, dinv, Mp, Gp, G, Li, T, U, Gf, Lif, colp, Zd, Zf, ids, offs, V, fitp, bytes;
  int F[kMaxOrder];        // this CTA's rows of each factor
  int rpc[kMaxOrder];      // rows of factor m per CTA (CTA c owns rows [c rpc, (c+1) rpc))
};

__host__ __device__ inline int align_up(int x, int a) { return (x + a - 1) / a * a; }

__host__ __device__ inline ClusterSmem cluster_smem_layout(int N, int R, const int64_t* dims, int S, int C,
                                                            int acc_bytes) {
  ClusterSmem L;
  int maxI = 0, maxrpc = 0;
  int o = 0;
  for (int m = 0; m < kMaxOrder; ++m) {
    L.F[m] = 0;
    L.rpc[m] = 0;
  }
  for (int m = 0; m < N; ++m) {
    const int I = (int)dims[m];
    maxI = I > maxI ? I : maxI;
    L.rpc[m] = (I + C - 1) / C;
    maxrpc = L.rpc[m] > maxrpc ? L.rpc[m] : maxrpc;
    L.F[m] = o;
    o = align_up(o + L.rpc[m] * R * acc_bytes, 16);
  }
  const int spc = (S + C - 1) / C;
  L.sc = o;   o = align_up(o + N * R * 8, 16);
  L.lam = o;  o = align_up(o + R * 8, 16);
  L.wr = o;   o = align_up(o + (R + 3) / 4 * 4 * 8, 16);
  L.dinv = o; o = align_up(o + R * 8, 16);
  L.Mp = o;   o = align_up(o + maxI * R * acc_bytes, 16);
  L.Gp = o;   o = align_up(o + R * R * 8, 16);
  L.G = o;    o = align_up(o + R * R * 8, 16);
  L.Li = o;   o = align_up(o + R * R * 8, 16);
  L.T = o;    o = align_up(o + R * R * 8, 16);
  L.U = o;    o = align_up(o + R * R * 8, 16);
  L.Gf = o;   o = align_up(o + R * R * 4, 16);
  L.Lif = o;  o = align_up(o + R * R * 4, 16);
  L.colp = o; o = align_up(o + R * 8, 16);
  L.Zd = o;   o = align_up(o + spc * R * 8, 16);
  L.Zf = o;   o = align_up(o + spc * R * acc_bytes, 16);
  L.ids = o;  o = align_up(o + spc * kMaxOrder * 4, 16);
  L.offs = o; o = align_up(o + spc * 8, 16);
  L.V = o;    o = align_up(o + 2 * maxrpc * R * 8, 16);
  L.fitp = o; o = align_up(o + 16, 16);
  L.bytes = o;
  return L;
}

// Sum of v[q] over the C CTAs' copies of one shared-memory double, as a fixed pairwise tree (same
// rounding in every CTA; depth log2 C instead of a chain of C dependent FP64 adds).
template <int C>
__device__ __forceinline__ double cluster_tree_sum(cg::cluster_group& cl, const double* v) {
  double a[C];
#pragma unroll
  for (int q = 0; q < C; ++q) a[q] = cl.map_shared_rank(v, q)[0];
#pragma unroll
  for (int w = 1; w < C; w <<= 1)
#pragma unroll
    for (int q = 0; q + w < C; q += 2 * w) a[q] += a[q + w];
  return a[0];
}

// Factor row i of mode m, held by the CTA that owns it.
template <typename ACC, int C>
__device__ __forceinline__ const ACC* factor_row(cg::cluster_group& cl, unsigned char* sm, const ClusterSmem& Lo,
                                                 int m, uint32_t i, int R) {
  const int rpc = Lo.rpc[m];
  const int owner = (int)(i / (uint32_t)rpc);
  const int loc = (int)i - owner * rpc;
  const ACC* base = reinterpret_cast<const ACC*>(sm + Lo.F[m]);
  return cl.map_shared_rank(base, owner) + loc * R;
}

// Block-wide max of a non-negative value (every thread gets the result).
__device__ __forceinline__ double block_max(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmax(v, __shfl_xor_sync(0xffffffffu, v, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < (int)(blockDim.x >> 5); ++q) t = fmax(t, red[q]);
  __syncthreads();
  return t;
}

// X = G^-1 (R x R, FP64) in shared memory, identical in every CTA (no data-dependent thread
// counts, fixed operation order).  Small R: Cholesky and triangular inverse in FP32 (a short
// latency chain on the FP32 pipe), X0 = L^-T L^-1, then FP64 Newton-Schulz steps
// X <- X + X (I - G X), each squaring the residual ||I - G X||; the FP32 start is used only when
// that residual is below 1/4.  Otherwise (and for larger R) the Cholesky and the inverse are FP64.
// Returns through *s_bad a non-positive FP64 pivot (Gram matrix singular).
__device__ void gram_inverse(const double* G, double* X, double* Tm, double* Um, float* Gf, float* Lif,
                             double* dinv, double* Lw, int R, int ns_steps, int* s_bad, double* red) {
  const int tid = threadIdx.x;
  bool fast = R <= 16;
  if (fast) {
    for (int e = tid; e < R * R; e += blockDim.x) Gf[e] = (float)G[e];
    __syncthreads();
    __shared__ int fbad;
    if (tid < 32) {                      // FP32 Cholesky, lane i owns row i
      const int lane = tid;
      float md = lane < R ? Gf[lane * R + lane] : 0.f;
      for (int o = 16; o > 0; o >>= 1) md = fmaxf(md, __shfl_xor_sync(0xffffffffu, md, o));
      int bad = 0;
      for (int k = 0; k < R; ++k) {
        const float d = Gf[k * R + k];
        if (!(d > 1e-6f * md) || !isfinite(d)) bad = 1;
        const float y = rsqrtf(fmaxf(d, 1e-30f));
        __syncwarp();
        if (lane == 0) Gf[k * R + k] = d * y;
        if (lane > k && lane < R) Gf[lane * R + k] *= y;
        __syncwarp();
        if (lane > k && lane < R) {
          const float lik = Gf[lane * R + k];
          for (int c = k + 1; c <= lane; ++c) Gf[lane * R + c] = fmaf(-lik, Gf[c * R + k], Gf[lane * R + c]);
        }
        __syncwarp();
      }
      if (lane == 0) fbad = bad;
    }
    __syncthreads();
    fast = fbad == 0;
  }
  if (fast) {
    if (tid < R) {                       // L^-1 in FP32, column tid
      const int c = tid;
      for (int r = 0; r < c; ++r) Lif[r * R + c] = 0.f;
      Lif[c * R + c] = 1.f / Gf[c * R + c];
      for (int r = c + 1; r < R; ++r) {
        float acc = 0.f;
        for (int l = c; l < r; ++l) acc = fmaf(Gf[r * R + l], Lif[l * R + c], acc);
        Lif[r * R + c] = -acc / Gf[r * R + r];
      }
    }
    __syncthreads();
    for (int e = tid; e < R * R; e += blockDim.x) {   // X0 = L^-T L^-1
      const int r = e / R, c = e - r * R;
      float acc = 0.f;
      for (int l = max(r, c); l < R; ++l) acc = fmaf(Lif[l * R + r], Lif[l * R + c], acc);
      X[e] = (double)acc;
    }
    __syncthreads();
    for (int it = 0; it < ns_steps; ++it) {
      double emax = 0.0;
      for (int e = tid; e < R * R; e += blockDim.x) {   // E = I - G X
        const int r = e / R, c = e - r * R;
        double a0 = 0.0, a1 = 0.0;
        int l = 0;
        for (; l + 1 < R; l += 2) {
          a0 = fma(G[r * R + l], X[l * R + c], a0);
          a1 = fma(G[r * R + l + 1], X[(l + 1) * R + c], a1);
        }
        if (l < R) a0 = fma(G[r * R + l], X[l * R + c], a0);
        const double ev = (r == c ? 1.0 : 0.0) - (a0 + a1);
        Tm[e] = ev;
        emax = fmax(emax, fabs(ev));
      }
      emax = block_max(emax, red);
      if (it == 0 && !(emax < 0.25)) {
        fast = false;
        break;
      }
      for (int e = tid; e < R * R; e += blockDim.x) {   // X + X E
        const int r = e / R, c = e - r * R;
        double a0 = 0.0, a1 = 0.0;
        int l = 0;
        for (; l + 1 < R; l += 2) {
          a0 = fma(X[r * R + l], Tm[l * R + c], a0);
          a1 = fma(X[r * R + l + 1], Tm[(l + 1) * R + c], a1);
        }
        if (l < R) a0 = fma(X[r * R + l], Tm[l * R + c], a0);
        Um[e] = X[e] + (a0 + a1);
      }
      __syncthreads();
      for (int e = tid; e < R * R; e += blockDim.x) X[e] = Um[e];
      __syncthreads();
    }
    if (fast) return;
  }
  // FP64 path: Cholesky of G, triangular inverse, X = L^-T L^-1
  spd_inverse_fp64(G, X, Lw, Tm, dinv, R, s_bad);
}

template <typename T, typename ACC, int MAXR, int C>
__device__ void cluster_mode_update(const Prob& p, int n, uint32_t t, unsigned char* sm, const ClusterSmem& Lo,
                                    cg::cluster_group& cl, int* s_bad) {
  const int rank = (int)cl.block_rank(), tid = threadIdx.x;
  const int R = p.R, N = p.N, S = p.S;
  const int I = (int)p.dims[n];
  double* sc = reinterpret_cast<double*>(sm + Lo.sc);
  double* lam = reinterpret_cast<double*>(sm + Lo.lam);
  double* dinv = reinterpret_cast<double*>(sm + Lo.dinv);
  ACC* Mp = reinterpret_cast<ACC*>(sm + Lo.Mp);
  double* Gp = reinterpret_cast<double*>(sm + Lo.Gp);
  double* G = reinterpret_cast<double*>(sm + Lo.G);
  double* Li = reinterpret_cast<double*>(sm + Lo.Li);
  double* colp = reinterpret_cast<double*>(sm + Lo.colp);
  double* Zd = reinterpret_cast<double*>(sm + Lo.Zd);
  ACC* Zf = reinterpret_cast<ACC*>(sm + Lo.Zf);
  uint32_t* ids = reinterpret_cast<uint32_t*>(sm + Lo.ids);
  int64_t* offs = reinterpret_cast<int64_t*>(sm + Lo.offs);
  double* V1 = reinterpret_cast<double*>(sm + Lo.V);
  ACC* Fn = reinterpret_cast<ACC*>(sm + Lo.F[n]);

  // ---- samples of this CTA (Philox stream 0), SKR rows from the distributed factor slices
  const int spc = (S + C - 1) / C;
  const int j0 = rank * spc;
  const int cnt = max(0, min(S, j0 + spc) - j0);
  if (tid < cnt) {
    const uint32_t j = (uint32_t)(j0 + tid);
    const uint32_t k0 = (uint32_t)p.seed, k1 = (uint32_t)(p.seed >> 32);
    const uint4 w0 = philox10(make_uint4(j, counter_word1(kStreamSamples, 0, n), t, p.b), k0, k1);
    uint4 w1 = make_uint4(0u, 0u, 0u, 0u);
    if (N - 1 > 4) w1 = philox10(make_uint4(j, counter_word1(kStreamSamples, 1, n), t, p.b), k0, k1);
    int k = 0;
    for (int m = 0; m < N; ++m) {
      uint32_t im = 0;
      if (m != n) {
        const uint32_t w = k < 4 ? word_of(w0, k) : word_of(w1, k - 4);
        im = scale_index(w, (uint32_t)p.dims[m]);
        ++k;
      }
      ids[tid * kMaxOrder + m] = im;
    }
    int64_t stride;
    offs[tid] = fiber_offset(p, n, ids + tid * kMaxOrder, &stride);
  }
  __syncthreads();
  for (int e = tid; e < cnt * R; e += kCT) {
    const int jj = e / R, r = e - jj * R;
    ACC v[kMaxOrder];
#pragma unroll
    for (int m = 0; m < kMaxOrder; ++m)
      if (m < N && m != n) v[m] = factor_row<ACC, C>(cl, sm, Lo, m, ids[jj * kMaxOrder + m], R)[r];
    double z = 1.0;
#pragma unroll
    for (int m = 0; m < kMaxOrder; ++m) {
      if (m >= N) break;   // a branch, not predicated-off FP64 multiplies (they still occupy the pipe)
      if (m != n) z *= (double)v[m] * sc[m * R + r];
    }
    Zd[e] = z;
    Zf[e] = (ACC)z;
  }
  __syncthreads();
  // ---- partial M = X_S Z_S over this CTA's samples, every row (loads batched 8 at a time)
  const T* __restrict__ X = reinterpret_cast<const T*>(p.Xrep[n]);
  const int64_t stn = p.use_rep ? 1 : p.st[n];
  for (int i = tid; i < I; i += kCT) {
    ACC acc[MAXR];
#pragma unroll
    for (int r = 0; r < MAXR; ++r) acc[r] = ACC(0);
    const int64_t sti = (int64_t)i * stn;
    for (int j = 0; j < cnt; j += 8) {
      ACC x[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        x[q] = ACC(0);
        if (j + q < cnt) {
          if constexpr (sizeof(ACC) == 8) x[q] = (ACC)__ldg(&X[offs[j + q] + sti]);
          else if constexpr (sizeof(T) == 4) x[q] = __ldg(&X[offs[j + q] + sti]);
          else x[q] = __bfloat162float(X[offs[j + q] + sti]);
        }
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        if (j + q < cnt) {
          const ACC* z = Zf + (j + q) * R;
#pragma unroll
          for (int r = 0; r < MAXR; ++r)
            if (r < R) acc[r] = fma(x[q], z[r], acc[r]);
        }
      }
    }
#pragma unroll
    for (int r = 0; r < MAXR; ++r)
      if (r < R) Mp[i * R + r] = acc[r];
  }
  for (int e = tid; e < R * R; e += kCT) {
    const int r = e / R, c = e - r * R;
    if (c < r) continue;
    double a = 0.0;
    for (int jj = 0; jj < cnt; ++jj) a = fma(Zd[jj * R + r], Zd[jj * R + c], a);
    Gp[e] = a;
  }
  cl.sync();  // partial M and Gram of every CTA complete
  // ---- G = sum of the partial Grams in a fixed order (all C loads in flight), Cholesky, L^-1
  for (int e = tid; e < R * R; e += kCT) {
    const int r = e / R, c = e - r * R;
    if (c < r) continue;
    const double g = cluster_tree_sum<C>(cl, Gp + e);
    G[r * R + c] = g;
    G[c * R + r] = g;
  }
  __syncthreads();
  {
    __shared__ double red[kCT / 32];
    double* Tm = reinterpret_cast<double*>(sm + Lo.T);
    double* Um = reinterpret_cast<double*>(sm + Lo.U);
    float* Gf = reinterpret_cast<float*>(sm + Lo.Gf);
    float* Lif = reinterpret_cast<float*>(sm + Lo.Lif);
    // Li receives X = G^-1; U doubles as the FP64 Cholesky workspace of the fallback
    gram_inverse(G, Li, Tm, Um, Gf, Lif, dinv, Um, R, sizeof(ACC) == 8 ? 2 : 1, s_bad, red);
  }
  // ---- this CTA's rows: partial M rows summed through DSMEM (fixed order)
  const int rpc = Lo.rpc[n];
  const int i0 = rank * rpc;
  const int nrows = max(0, min(I, i0 + rpc) - i0);
  double* V2 = V1 + rpc * R;
  for (int e = tid; e < nrows * R; e += kCT) {
    ACC a = ACC(0);
#pragma unroll
    for (int q = 0; q < C; ++q) a += cl.map_shared_rank(Mp, q)[(int64_t)i0 * R + e];
    V1[e] = (double)a;
  }
  __syncthreads();
  // a = m X for every (row, column) in parallel (FP64; X = G^-1 is symmetric)
  for (int e = tid; e < nrows * R; e += kCT) {
    const int li = e / R, r = e - li * R;
    const double* m = V1 + li * R;
    double s0 = 0.0, s1 = 0.0;
    int l = 0;
    for (; l + 1 < R; l += 2) {
      s0 = fma(m[l], Li[l * R + r], s0);
      s1 = fma(m[l + 1], Li[(l + 1) * R + r], s1);
    }
    if (l < R) s0 = fma(m[l], Li[l * R + r], s0);
    const double a = s0 + s1;
    V2[e] = a;
    Fn[e] = (ACC)a;                               // this CTA's slice of the new factor
    p.A64[n][(int64_t)i0 * R + e] = a;            // FP64 result (read only after the run)
    reinterpret_cast<ACC*>(p.Apad[n])[(int64_t)(i0 + li) * ((R + 3) / 4 * 4) + r] = (ACC)a;   // for the fit
  }
  __syncthreads();
  for (int e = tid; e < nrows * R; e += kCT) V1[e] = V2[e];
  __syncthreads();
  {
    // column sums of squares of this CTA's rows: 8-row chunks in parallel, then a fixed-order sum
    double* cpart = V2;   // (R x ceil(nrows / 8)) partials; V2 is free again
    const int nch = (nrows + 7) / 8;
    for (int e = tid; e < R * nch; e += kCT) {
      const int r = e / nch, ch = e - r * nch;
      double sq = 0.0;
      for (int li = ch * 8; li < min(nrows, ch * 8 + 8); ++li) sq = fma(V1[li * R + r], V1[li * R + r], sq);
      cpart[e] = sq;
    }
    __syncthreads();
    for (int r = tid; r < R; r += kCT) {
      double sq = 0.0;
      for (int ch = 0; ch < nch; ++ch) sq += cpart[r * nch + ch];
      colp[r] = sq;
    }
  }
  if (n == N - 1) asm volatile("fence.acq_rel.cluster;" ::: "memory");   // padded rows read by the fit
  cl.sync();  // new factor slices and column partials of every CTA complete
  // ---- lambda and lazy scales of mode n in every CTA
  for (int r = tid; r < R; r += kCT) {
    const double nrm = sqrt(cluster_tree_sum<C>(cl, colp + r));
    lam[r] = nrm;
    sc[n * R + r] = nrm > 0.0 ? recip64(nrm) : 1.0;
  }
  __syncthreads();
}

__device__ __forceinline__ double cta_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double t = 0.0;
  for (int q = 0; q < kCT / 32; ++q) t += red[q];
  __syncthreads();
  return t;   // valid in every thread
}

template <typename T, typename ACC, int MAXR, int C>
__global__ void __launch_bounds__(kCT, 1) k_cluster_run(const Prob* probs, int B, int* queue) {
  cg::cluster_group cl = cg::this_cluster();
  const int rank = (int)cl.block_rank(), tid = threadIdx.x;
  extern __shared__ __align__(16) unsigned char sm[];
  __shared__ int s_prob;
  __shared__ int s_bad;
  __shared__ int s_done, s_status, s_iter, s_stall;
  __shared__ double s_best, s_last;
  __shared__ double red[kCT / 32];
  while (true) {
    if (rank == 0 && tid == 0) s_prob = atomicAdd(queue, 1);
    cl.sync();
    const int b = *cl.map_shared_rank(&s_prob, 0);
    cl.sync();
    if (b >= B) break;   // same value in every CTA of the cluster
    const Prob& p = probs[b];
    const int R = p.R, N = p.N;
    const ClusterSmem Lo = cluster_smem_layout(N, R, p.dims, p.S, C, (int)sizeof(ACC));
    double* sc = reinterpret_cast<double*>(sm + Lo.sc);
    double* lam = reinterpret_cast<double*>(sm + Lo.lam);
    double* wr = reinterpret_cast<double*>(sm + Lo.wr);
    double* fitp = reinterpret_cast<double*>(sm + Lo.fitp);
    State* st = p.state;
    // this CTA's rows of every factor (the starting point)
    const int Rp = (R + 3) / 4 * 4;
    for (int m = 0; m < N; ++m) {
      ACC* F = reinterpret_cast<ACC*>(sm + Lo.F[m]);
      ACC* Ap = reinterpret_cast<ACC*>(p.Apad[m]);
      const int i0 = rank * Lo.rpc[m];
      const int nr = max(0, min((int)p.dims[m], i0 + Lo.rpc[m]) - i0);
      for (int e = tid; e < nr * Rp; e += kCT) {
        const int li = e / Rp, r = e - li * Rp;
        ACC v = ACC(0);
        if (r < R) {
          if constexpr (sizeof(ACC) == 8) v = p.A64[m][(int64_t)(i0 + li) * R + r];
          else v = p.A32[m][(int64_t)(i0 + li) * R + r];
          F[li * R + r] = v;
        }
        Ap[(int64_t)(i0 + li) * Rp + r] = v;
      }
    }
    for (int e = tid; e < N * R; e += kCT) sc[e] = p.scale[e / R][e % R];
    for (int r = tid; r < R; r += kCT) lam[r] = p.lambda[r];
    if (tid == 0) {
      s_done = st->done;
      s_status = st->status;
      s_iter = st->iter;
      s_stall = st->stall;
      s_best = st->best;
      s_last = st->last_fit;
      s_bad = 0;
    }
    cl.sync();   // every slice loaded before any CTA reads another's
    const int cap = p.fixed_iters > 0 ? p.fixed_iters : p.max_iters;
    while (!s_done && s_iter < cap) {
      const uint32_t t = p.t0 + (uint32_t)s_iter;
      for (int n = 0; n < N; ++n) {
        cluster_mode_update<T, ACC, MAXR, C>(p, n, t, sm, Lo, cl, &s_bad);
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
      for (int r = tid; r < Rp; r += kCT) {
        double w = 0.0;
        if (r < R) {
          w = lam[r];
          for (int m = 0; m < N; ++m) w *= sc[m * R + r];
        }
        wr[r] = w;
      }
      __syncthreads();
      const int fpc = (p.P_hat + C - 1) / C;
      const int f0 = rank * fpc, f1 = min(p.P_hat, f0 + fpc);
      double e2 = 0.0;
      constexpr int VW = 16 / sizeof(ACC);          // elements per 16-byte vector
      const int nv = Rp / VW;
      for (int j = f0 + tid; j < f1; j += kCT) {
        const uint32_t* id = p.fit_idx + (int64_t)j * N;
        const uint4* rows[kMaxOrder];
#pragma unroll
        for (int m = 0; m < kMaxOrder; ++m)
          rows[m] = (m < N) ? reinterpret_cast<const uint4*>(reinterpret_cast<const ACC*>(p.Apad[m]) +
                                                             (int64_t)__ldg(&id[m]) * Rp)
                            : nullptr;
        ACC acc = ACC(0);
        for (int v = 0; v < nv; ++v) {
          uint4 q[kMaxOrder];
#pragma unroll
          for (int m = 0; m < kMaxOrder; ++m)
            if (m < N) q[m] = __ldcg(&rows[m][v]);
#pragma unroll
          for (int u = 0; u < VW; ++u) {
            ACC w = (ACC)wr[v * VW + u];
#pragma unroll
            for (int m = 0; m < kMaxOrder; ++m)
              if (m < N) w *= reinterpret_cast<const ACC*>(&q[m])[u];
            acc += w;
          }
        }
        const double e = p.fit_x[j] - (double)acc;
        e2 = fma(e, e, e2);
      }
      const double tot = cta_sum(e2, red);
      if (tid == 0) fitp[0] = tot;
      cl.sync();
      if (tid == 0) {
        const double s = cluster_tree_sum<C>(cl, fitp);
        const double fit = 1.0 - sqrt((double)p.P * (s / (double)p.P_hat)) / st->norm_x;
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
      __syncthreads();
    }
    // publish the loop state, lambda and the lazy scales (CTA 0)
    if (rank == 0) {
      for (int e = tid; e < N * R; e += kCT) p.scale[e / R][e % R] = sc[e];
      for (int r = tid; r < R; r += kCT) p.lambda[r] = lam[r];
      if (tid == 0) {
        st->done = 1;
        st->status = s_status;
        st->iter = s_iter;
        st->stall = s_stall;
        st->best = s_best;
        st->last_fit = s_last;
      }
    }
    cl.sync();  // no CTA reuses its shared memory while another may still read it
  }
}

// Shared memory of the cluster kernel for the largest problem of a batch, or -1 if a problem does
// not fit (then the multi-kernel path is used).
int cluster_smem_bytes(const Prob* probs_host, int B, int C) {
  int most = 0;
  for (int b = 0; b < B; ++b) {
    const Prob& p = probs_host[b];
    const int accb = p.dtype == CPR_F64 ? 8 : 4;
    const ClusterSmem L = cluster_smem_layout(p.N, p.R, p.dims, p.S, C, accb);
    most = max(most, L.bytes);
  }
  return most <= 180 * 1024 ? most : -1;
}

template <typename T, typename ACC, int MAXR, int C>
static cudaError_t cluster_launch(const Prob* probs, int B, int* queue, int smem, int nclusters, cudaStream_t s) {
  auto kern = k_cluster_run<T, ACC, MAXR, C>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  if (e != cudaSuccess) return e;
  if (C > 8) {
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    if (e != cudaSuccess) return e;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(C * nclusters), 1, 1);
  cfg.blockDim = dim3(kCT, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, probs, B, queue);
}

template <typename T, typename ACC, int MAXR, int C>
static int cluster_capacity_t(int smem) {
  auto kern = k_cluster_run<T, ACC, MAXR, C>;
  if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, smem) != cudaSuccess) return 0;
  if (C > 8 && cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1) != cudaSuccess) return 0;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)C, 1, 1);
  cfg.blockDim = dim3(kCT, 1, 1);
  cfg.dynamicSmemBytes = (size_t)smem;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)C;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int n = 0;
  if (cudaOccupancyMaxActiveClusters(&n, kern, &cfg) != cudaSuccess) {
    cudaGetLastError();
    return 0;
  }
  return n;
}

// One entry per (MAXR, C) instantiation: op 0 = launch, op 1 = capacity query.
template <typename T, typename ACC, int MAXR>
static int cluster_op_r(int op, int C, const Prob* probs, int B, int* queue, int smem, int nclusters, cudaStream_t s,
                        cudaError_t* err) {
  if (C == 16) {
    if (op == 1) return cluster_capacity_t<T, ACC, MAXR, 16>(smem);
    *err = cluster_launch<T, ACC, MAXR, 16>(probs, B, queue, smem, nclusters, s);
  } else {
    if (op == 1) return cluster_capacity_t<T, ACC, MAXR, 8>(smem);
    *err = cluster_launch<T, ACC, MAXR, 8>(probs, B, queue, smem, nclusters, s);
  }
  return 0;
}

template <typename T, typename ACC>
static int cluster_op(int op, int C, int maxR, const Prob* probs, int B, int* queue, int smem, int nclusters,
                      cudaStream_t s, cudaError_t* err) {
  if (maxR <= 8) return cluster_op_r<T, ACC, 8>(op, C, probs, B, queue, smem, nclusters, s, err);
  if (maxR <= 16) return cluster_op_r<T, ACC, 16>(op, C, probs, B, queue, smem, nclusters, s, err);
  if (maxR <= 32) return cluster_op_r<T, ACC, 32>(op, C, probs, B, queue, smem, nclusters, s, err);
  return cluster_op_r<T, ACC, 64>(op, C, probs, B, queue, smem, nclusters, s, err);
}

static int cluster_op_dt(int op, int dtype, int C, int maxR, const Prob* probs, int B, int* queue, int smem,
                         int nclusters, cudaStream_t s, cudaError_t* err) {
  switch (dtype) {
    case CPR_F64: return cluster_op<double, double>(op, C, maxR, probs, B, queue, smem, nclusters, s, err);
    case CPR_F32: return cluster_op<float, float>(op, C, maxR, probs, B, queue, smem, nclusters, s, err);
    default: return cluster_op<__nv_bfloat16, float>(op, C, maxR, probs, B, queue, smem, nclusters, s, err);
  }
}

// How many clusters of C CTAs with this shared memory can be resident at once (0: not launchable).
int cluster_capacity(int dtype, int C, int smem, int maxR) {
  if (C != 16 && C != 8) return 0;
  cudaError_t err = cudaSuccess;
  return cluster_op_dt(1, dtype, C, maxR, nullptr, 0, nullptr, smem, 0, nullptr, &err);
}

cudaError_t launch_cluster_run(const Prob* probs, int B, int* queue, int dtype, int C, int smem, int nclusters,
                               int maxR, cudaStream_t s) {
  if (C != 16 && C != 8) return cudaErrorInvalidValue;
  cudaError_t err = cudaSuccess;
  cluster_op_dt(0, dtype, C, maxR, probs, B, queue, smem, nclusters, s, &err);
  return err;
}

}  // namespace cpr
