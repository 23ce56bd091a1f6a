// factor.cu -- right-looking supernodal Cholesky (RL, Sec. II-A) on the GPU.
//
// Level by level of the supernodal elimination tree (leaves first), every
// supernode J of the level is factored (POTRF on the diagonal block, TRSM on
// the off-diagonal panel, Sec. II-A), its update matrix U_J = L_RJ L_RJ^T
// (the DSYRK of Sec. II-A) is formed in a workspace sized for the largest
// level (the preallocated update storage of Sec. II-A), and the update
// matrices of the level are scatter-added into their ancestors through the
// relative indices relind(J, K) (Sec. II-A assembly).
//
// Kernel classes
//   k_scatter        A's values into the zeroed panels (HBM-bound gather/scatter)
//   k_small          one CTA per small supernode: POTRF + TRSM + SYRK in shared memory
//   k_potrf          blocked path, diagonal block of one column step
//   k_trsm           blocked path, row tiles below the diagonal block
//   k_gemm_trailing  blocked path, trailing update of the panel (FP64 DFMA tiles)
//   k_syrk           blocked path, U_J tiles (lower triangle only)
//   k_assemble       relind scatter-add, pull-ordered: each task owns target
//                    columns and applies its contributors in a fixed order, so
//                    no atomics and a bitwise-deterministic result
//   k_logdet_*       2 sum log L_jj with a fixed-order reduction
#include <climits>
#include <cmath>
#include <cstring>

#include <cooperative_groups.h>

#include "device.h"
#include "mixed.h"
#include "assemble.cuh"
#include "potrf.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kSmallThreads = 128;
constexpr int kGemmThreads = 256;
constexpr int kAsmThreads = 256;

// ---------------------------------------------------------------------------
// dense Cholesky of the first s columns of a len x s column-major block in
// shared memory (right-looking, one column per step). A non-positive or NaN
// pivot records column fcol+k+1 in *status (smallest wins) and poisons the
// column with NaN so that the failure propagates without stopping the grid.
// ---------------------------------------------------------------------------
__device__ void dense_chol_smem(double* P, int ld, int len, int s, int fcol, int* status) {
  __shared__ double srk;
  for (int k = 0; k < s; ++k) {
    __syncthreads();
    if (threadIdx.x == 0) {
      // the pivot's root once, by one thread (FP64 sqrt and division are long
      // dependent sequences on the narrow FP64 pipe)
      const double d = P[k + k * ld];
      const bool bad = !(d > 0.0);
      double dk, rk;
      pivot_root(d, bad, dk, rk);
      P[k + k * ld] = dk;
      srk = rk;
      if (bad) atomicMin(status, fcol + k + 1);
    }
    __syncthreads();
    const double inv = srk;
    for (int r = k + 1 + threadIdx.x; r < len; r += blockDim.x) P[r + k * ld] *= inv;
    __syncthreads();
    // rank-1 update of the trailing columns, one thread per row
    for (int r = k + 1 + threadIdx.x; r < len; r += blockDim.x) {
      const double lrk = P[r + k * ld];
      const int jmax = r < s - 1 ? r : s - 1;
      for (int j = k + 1; j <= jmax; ++j) P[r + j * ld] -= lrk * P[j + k * ld];
    }
  }
  __syncthreads();
}

// Position of global row `key` in the sorted row structure rk[0, len).
__device__ __forceinline__ int row_position(const int32_t* __restrict__ rk, int len, int32_t key) {
  int lo = 0, hi = len;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (rk[mid] < key) lo = mid + 1; else hi = mid;
  }
  return lo;
}

__global__ void k_status_init(int* status) { *status = INT_MAX; }

__global__ void k_scatter(const double* __restrict__ vals, const int64_t* __restrict__ amap,
                          int64_t nnz, double* __restrict__ L) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz;
       t += (int64_t)gridDim.x * blockDim.x) {
#ifdef CHOL_BOUNDS_CHECK
    if (!CHOL_BC(amap[t] >= 0 && amap[t] < bc_lim.panel, kBcScatter)) continue;
#endif
    L[amap[t]] = vals[t];
  }
}

// One CTA per small supernode: the whole len x s panel lives in shared memory.
__device__ __forceinline__ void small_body(const SnodeDev& d, double* __restrict__ L, double* __restrict__ U,
                                           int* status, double* P) {
  const int len = d.len, s = d.s, b = len - s;
  double* G = L + d.loff;
  for (int c = 0; c < s; ++c)
    for (int r = threadIdx.x; r < len; r += blockDim.x) P[r + c * len] = G[r + (int64_t)c * d.ld];
  dense_chol_smem(P, len, len, s, d.f, status);
  for (int c = 0; c < s; ++c)
    for (int r = c + threadIdx.x; r < len; r += blockDim.x) G[r + (int64_t)c * d.ld] = P[r + c * len];
  if (b <= 0) return;
  // U_J = L_RJ L_RJ^T, lower triangle, column-major b x b. Flat walk over the
  // lower triangle: column c holds rows c..b-1.
  double* Uj = U + d.uoff;
  const double* R = P + s;  // row u of L_RJ is R[u + k*len]
  const int64_t total = (int64_t)b * (b + 1) / 2;
  int c = 0;
  int64_t cstart = 0;  // flat index of (c, c)
  for (int64_t q = threadIdx.x; q < total; q += blockDim.x) {
    while (q >= cstart + (b - c)) { cstart += b - c; ++c; }
    const int u = c + (int)(q - cstart);
    double acc = 0.0;
    for (int k = 0; k < s; ++k) acc += R[u + k * len] * R[c + k * len];
    Uj[u + (int64_t)c * b] = acc;
  }
}

__global__ void __launch_bounds__(kSmallThreads)
k_small(const SnodeDev* __restrict__ sn, const int32_t* __restrict__ list, double* __restrict__ L,
        double* __restrict__ U, int* status) {
  extern __shared__ double P[];
  small_body(sn[list[blockIdx.x]], L, U, status, P);
}

// RLB form of the one-CTA kernel: after the factorization in shared memory,
// every entry (u, c), u >= c, of L_RJ L_RJ^T is subtracted straight from the
// ancestor owning column c, pair by pair (row positions found once per pair).
__global__ void __launch_bounds__(kSmallThreads)
k_small_rlb(const SnodeDev* __restrict__ sn, const int32_t* __restrict__ list, const int4* __restrict__ pairs,
            const int32_t* __restrict__ pbeg, const int32_t* __restrict__ rows, double* __restrict__ L,
            int* status) {
  extern __shared__ double P[];
  __shared__ int32_t pos[kRlbSmallRows];
  const int32_t J = list[blockIdx.x];
  const SnodeDev d = sn[J];
  const int len = d.len, s = d.s, b = len - s;
  double* G = L + d.loff;
  for (int c = 0; c < s; ++c)
    for (int r = threadIdx.x; r < len; r += blockDim.x) P[r + c * len] = G[r + (int64_t)c * d.ld];
  dense_chol_smem(P, len, len, s, d.f, status);
  for (int c = 0; c < s; ++c)
    for (int r = c + threadIdx.x; r < len; r += blockDim.x) G[r + (int64_t)c * d.ld] = P[r + c * len];
  if (b <= 0) return;
  const double* R = P + s;   // row u of L_RJ is R[u + k*len]
  const int32_t* rj = rows + d.roff + s;
  for (int p = pbeg[J]; p < pbeg[J + 1]; ++p) {
    const int4 pr = pairs[p];
    const SnodeDev dk = sn[pr.x];
    __syncthreads();
    for (int u = pr.y + threadIdx.x; u < b; u += blockDim.x)
      pos[u - pr.y] = row_position(rows + dk.roff, dk.len, rj[u]);
    __syncthreads();
    // entries of columns [c0, c1), rows c..b-1: flat walk
    const int64_t total = (int64_t)(pr.z - pr.y) * b - ((int64_t)pr.z * (pr.z - 1) - (int64_t)pr.y * (pr.y - 1)) / 2;
    int c = pr.y;
    int64_t cstart = 0;   // flat index of (c, c)
    for (int64_t q = threadIdx.x; q < total; q += blockDim.x) {
      while (q >= cstart + (b - c)) { cstart += b - c; ++c; }
      const int u = c + (int)(q - cstart);
      double acc = 0.0;
      for (int k = 0; k < s; ++k) acc += R[u + k * len] * R[c + k * len];
      atomicAdd(L + dk.loff + pos[u - pr.y] + (int64_t)(rj[c] - dk.f) * dk.ld, -acc);
    }
  }
}

// Blocked path, step k0: factor the kb x kb (kb <= 64) diagonal block of each
// listed supernode (8-column panels on a shared-memory copy, potrf.cuh); a
// non-positive pivot records its column in *status.
constexpr int kPotrfThreads = kPkThreads;
__global__ void __launch_bounds__(kPotrfThreads)
k_potrf(const SnodeDev* __restrict__ sn, const int32_t* __restrict__ list, int k0, int nb,
        double* __restrict__ L, int* status) {
  __shared__ double As[64 * kPwLd];
  __shared__ int sok;
  const SnodeDev d = sn[list[blockIdx.x]];
  const int kb = min(nb, d.s - k0);
  double* G = L + d.loff + k0 + (int64_t)k0 * d.ld;
  potrf_panels<double, false>(G, d.ld, kb, -INFINITY, As, &sok, status, true, d.f + k0);
}

// Blocked path, step k0: rows [r0, r0 + kTrsmRows) of column block [k0, k0+kb) become
// X = B L_kk^{-T}. Eight lanes share a row, lane q holding columns q + 8m; the
// solved x_j is broadcast inside the 8-lane group with a shuffle and every lane
// updates its own columns (no barriers in the substitution loop).
constexpr int kTrsmThreads = 128;   // 8 lanes per row
constexpr int kTrsmRows = 16;
__global__ void __launch_bounds__(kTrsmThreads)
k_trsm(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, int nb,
       double* __restrict__ L) {
  __shared__ double Lk[64 * 65];
  __shared__ double inv[64];
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int kb = min(nb, d.s - t.k0);
  const double* Gd = L + d.loff + t.k0 + (int64_t)t.k0 * d.ld;
  {
    // stage the diagonal block: all loads of a thread issued before the
    // stores (column-major source: consecutive threads read consecutive rows)
    constexpr int kIt = 64 * 64 / kTrsmThreads;
    double v[kIt];
#pragma unroll
    for (int i = 0; i < kIt; ++i) {
      const int q = threadIdx.x + kTrsmThreads * i, r = q & 63, c = q >> 6;
      v[i] = (r < kb && c < kb) ? Gd[r + (int64_t)c * d.ld] : 0.0;
    }
#pragma unroll
    for (int i = 0; i < kIt; ++i) {
      const int q = threadIdx.x + kTrsmThreads * i;
      Lk[(q & 63) + (q >> 6) * 65] = v[i];
    }
  }
  __syncthreads();
  for (int c = threadIdx.x; c < kb; c += blockDim.x) inv[c] = 1.0 / Lk[c + c * 65];
  __syncthreads();
  const int g = threadIdx.x >> 3, q = threadIdx.x & 7;
  const int row = t.r0 + g;
  const bool live = row < d.len;
  double* Gx = L + d.loff + row + (int64_t)t.k0 * d.ld;
  double x[8];
#pragma unroll
  for (int m = 0; m < 8; ++m) {
    const int c = q + 8 * m;
    x[m] = (live && c < kb) ? Gx[(int64_t)c * d.ld] : 0.0;
  }
#pragma unroll
  for (int jm = 0; jm < 8; ++jm) {
#pragma unroll
    for (int jq = 0; jq < 8; ++jq) {
      const int j = jm * 8 + jq;
      if (j < kb) {
        const double cand = x[jm] * inv[j];
        const double xj = __shfl_sync(0xffffffffu, cand, jq, 8);
        if (q == jq) x[jm] = xj;
        // columns q + 8m with m < jm are already solved: not even issued
#pragma unroll
        for (int m = jm; m < 8; ++m) {
          const int c = q + 8 * m;
          if (c > j && c < kb) x[m] -= xj * Lk[c + j * 65];
        }
      }
    }
  }
  if (live) {
#pragma unroll
    for (int m = 0; m < 8; ++m) {
      const int c = q + 8 * m;
      if (c < kb) Gx[(int64_t)c * d.ld] = x[m];
    }
  }
}

// ---------------------------------------------------------------------------
// 64 x 64 FP64 tile of C (op)= A B^T with K-chunks of 16 staged in shared
// memory; 256 threads, 4 x 4 accumulators each (rows ty+16i, cols tx+16j).
// Only entries with (row + rdiag >= col) are written (lower triangle of the
// global matrix). SUB: C -= A B^T, else C = A B^T.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void gemm_nt_core(const double* __restrict__ A, int64_t lda,
                                             const double* __restrict__ B, int64_t ldb, int K, int M, int N,
                                             double (&acc)[4][4]) {
  constexpr int KC = 16;
  __shared__ double As[KC][kTile];
  __shared__ double Bs[KC][kTile];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j] = 0.0;
  for (int k = 0; k < K; k += KC) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + kGemmThreads * q;
      const int kk = idx >> 6, r = idx & 63;
      const bool kin = k + kk < K;
      As[kk][r] = (kin && r < M) ? A[r + (int64_t)(k + kk) * lda] : 0.0;
      Bs[kk][r] = (kin && r < N) ? B[r + (int64_t)(k + kk) * ldb] : 0.0;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      double a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
}

template <bool SUB>
__device__ __forceinline__ void gemm_nt_tile(const double* __restrict__ A, int64_t lda,
                                             const double* __restrict__ B, int64_t ldb, int K,
                                             double* __restrict__ C, int64_t ldc, int M, int N,
                                             int rdiag) {
  double acc[4][4];
  gemm_nt_core(A, lda, B, ldb, K, M, N, acc);
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      if (r < M && c < N && r + rdiag >= c) {
        double* p = C + r + (int64_t)c * ldc;
        *p = SUB ? (*p - acc[i][j]) : acc[i][j];
      }
    }
}

// Blocked path, step k0: trailing update of the panel,
// P[r, c] -= sum_{k in block} P[r, k] P[c, k] for r >= c, c >= k0 + kb.
__global__ void __launch_bounds__(kGemmThreads)
k_gemm_trailing(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, int nb,
                double* __restrict__ L) {
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int kb = min(nb, d.s - t.k0);
  double* P = L + d.loff;
  gemm_nt_tile<true>(P + t.r0 + (int64_t)t.k0 * d.ld, d.ld, P + t.c0 + (int64_t)t.k0 * d.ld, d.ld,
                     kb, P + t.r0 + (int64_t)t.c0 * d.ld, d.ld, min(kTile, d.len - t.r0),
                     min(kTile, d.s - t.c0), t.r0 - t.c0);
}

// Blocked path: U_J tile = L_RJ[r0.., :] L_RJ[c0.., :]^T (lower triangle).
__global__ void __launch_bounds__(kGemmThreads)
k_syrk(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks,
       const double* __restrict__ L, double* __restrict__ U) {
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int b = d.len - d.s;
  const double* R = L + d.loff + d.s;
  gemm_nt_tile<false>(R + t.r0, d.ld, R + t.c0, d.ld, d.s, U + d.uoff + t.r0 + (int64_t)t.c0 * b, b,
                      min(kTile, b - t.r0), min(kTile, b - t.c0), t.r0 - t.c0);
}

// RLB (Sec. II-B): the tile (rows r0.., columns c0..) of L_RJ L_RJ^T is
// subtracted straight from the ancestors' panels instead of being stored. The
// tile's columns fall into the (J, K) pairs of J (runs of J's rows owned by one
// ancestor K, in column order); for each pair the tile's rows are located in
// struct(K) (J's rows from the pair's first on all lie in it, and a run of
// consecutive global rows lands on consecutive positions), then every entry
// with row >= column is subtracted with an atomic add. Supernodes of a level
// update shared ancestors concurrently, so the order of the additions, and the
// rounding, varies from run to run.
__global__ void __launch_bounds__(kGemmThreads)
k_syrk_rlb(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, const int4* __restrict__ pairs,
           const int32_t* __restrict__ pbeg, const int32_t* __restrict__ rows, double* __restrict__ L) {
  __shared__ int32_t pos[kTile];
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int b = d.len - d.s;
  const double* R = L + d.loff + d.s;
  const int M = min(kTile, b - t.r0), N = min(kTile, b - t.c0);
  double acc[4][4];
  gemm_nt_core(R + t.r0, d.ld, R + t.c0, d.ld, d.s, M, N, acc);
  const int32_t* rj = rows + d.roff + d.s;
  const int tx = threadIdx.x & 15, ty = threadIdx.x >> 4;
  for (int p = pbeg[t.J]; p < pbeg[t.J + 1]; ++p) {
    const int4 pr = pairs[p];   // (K, first column, end column, -)
    if (pr.z <= t.c0) continue;
    if (pr.y >= t.c0 + N) break;
    const SnodeDev dk = sn[pr.x];
    __syncthreads();   // the previous pair is done with pos
    for (int i = threadIdx.x; i < M; i += blockDim.x) {
      const int u = t.r0 + i;
      pos[i] = u >= pr.y ? row_position(rows + dk.roff, dk.len, rj[u]) : -1;
    }
    __syncthreads();
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int r = ty + 16 * i, c = tx + 16 * j;
        const int u = t.r0 + r, cg = t.c0 + c;
        if (r < M && c < N && u >= cg && cg >= pr.y && cg < pr.z)
          atomicAdd(L + dk.loff + pos[r] + (int64_t)(rj[cg] - dk.f) * dk.ld, -acc[i][j]);
      }
  }
}

// Assembly of one task: for every segment (in J order) the rows ua..ub-1 of
// U_J are located in struct(K) by binary search over the task's position range
// (staged in shared memory), then a warp per column of the segment subtracts
// 32 rows at a time, kAsmUnroll (column, row chunk) items in flight per warp
// with all loads issued before the stores. Every entry of U_J hits a distinct
// entry of K (relind is injective) and a barrier separates segments, so the
// contributions to one entry are applied in a fixed order.
constexpr int kAsmUnroll = 4;

__device__ __forceinline__ void assemble_body(const AsmTask& t, const AsmSeg* __restrict__ segs,
                                              const SnodeDev* __restrict__ sn, const int32_t* __restrict__ rows,
                                              const double* __restrict__ U, double* __restrict__ L, int32_t* ssm) {
  __shared__ int32_t tcol[kAsmCols];
#ifdef CHOL_BOUNDS_CHECK
  if (!CHOL_BC(t.K >= 0 && t.K < bc_lim.ns, kBcTaskTarget)) return;
#endif
  const SnodeDev dk = sn[t.K];
  const int np = t.p1 - t.p0;
#ifdef CHOL_BOUNDS_CHECK
  if (!CHOL_BC(t.p0 >= 0 && np >= 0 && t.p1 <= dk.len && np <= kAsmPos && t.seg_begin >= 0 &&
                   t.seg_begin <= t.seg_end && t.seg_end <= bc_lim.nsegs,
               kBcTaskPositions))
    return;
#endif
  int32_t* sK = ssm;              // struct(K) at positions p0 .. p1-1
  int32_t* pos = ssm + kAsmPos;   // positions of rows ua .. ub-1 of the current segment
  const int32_t* rk = rows + dk.roff + t.p0;
  for (int i = threadIdx.x; i < np; i += blockDim.x) sK[i] = rk[i];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int nwarps = blockDim.x >> 5;
  for (int g = t.seg_begin; g < t.seg_end; ++g) {
    const AsmSeg sg = segs[g];
#ifdef CHOL_BOUNDS_CHECK
    if (!CHOL_BC(sg.J >= 0 && sg.J < bc_lim.ns, kBcSegSource)) continue;
#endif
    const SnodeDev dj = sn[sg.J];
    const int b = dj.len - dj.s;
    const int32_t* rj = rows + dj.roff + dj.s;
    const int nu = sg.ub - sg.ua, w = sg.cb - sg.ca;
#ifdef CHOL_BOUNDS_CHECK
    if (!CHOL_BC(sg.ua >= 0 && sg.ua <= sg.ub && sg.ub <= b && sg.ca >= 0 && sg.ca <= sg.cb && sg.cb <= b &&
                     nu <= kAsmPos && w <= kAsmCols,
                 kBcSegRange))
      continue;
#endif
    __syncthreads();   // sK loaded / previous segment finished with pos[] and tcol[]
    for (int i = threadIdx.x; i < nu; i += blockDim.x) {
      const int32_t key = rj[sg.ua + i];
      int lo = 0, hi = np;
      while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (sK[mid] < key) lo = mid + 1; else hi = mid;
      }
      pos[i] = t.p0 + lo;
#ifdef CHOL_BOUNDS_CHECK
      if (!CHOL_BC(lo < np && sK[lo] == key, kBcTargetRow)) pos[i] = -1;
#endif
    }
    for (int c = threadIdx.x; c < w; c += blockDim.x) {
      tcol[c] = rj[sg.ca + c] - dk.f;
#ifdef CHOL_BOUNDS_CHECK
      if (!CHOL_BC(tcol[c] >= 0 && tcol[c] < dk.s, kBcTargetCol)) tcol[c] = -1;
#endif
    }
    __syncthreads();
    const double* Uj = U + dj.uoff;
    double* Lk = L + dk.loff;
    const int nch = (nu + 31) >> 5;
    const int items = w * nch;   // (column, 32-row chunk) pairs
    for (int i0 = warp; i0 < items; i0 += nwarps * kAsmUnroll) {
      double v[kAsmUnroll], l[kAsmUnroll];
      int64_t off[kAsmUnroll];
#pragma unroll
      for (int q = 0; q < kAsmUnroll; ++q) {
        const int i = i0 + q * nwarps;
        off[q] = -1;
        if (i < items) {
          const int cc = i / nch;
          const int c = sg.ca + cc;
          const int u = sg.ua + (i - cc * nch) * 32 + lane;
          if (u < sg.ub && u >= c) {
#ifdef CHOL_BOUNDS_CHECK
            if (tcol[cc] < 0 || pos[u - sg.ua] < 0) continue;
#endif
            off[q] = (int64_t)tcol[cc] * dk.ld + pos[u - sg.ua];
            v[q] = Uj[(int64_t)c * b + u];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kAsmUnroll; ++q)
        if (off[q] >= 0) l[q] = Lk[off[q]];
#pragma unroll
      for (int q = 0; q < kAsmUnroll; ++q)
        if (off[q] >= 0) Lk[off[q]] = l[q] - v[q];
    }
  }
}

__global__ void __launch_bounds__(kAsmThreads)
k_assemble(const AsmTask* __restrict__ tasks, const AsmSeg* __restrict__ segs,
           const SnodeDev* __restrict__ sn, const int32_t* __restrict__ rows,
           const double* __restrict__ U, double* __restrict__ L) {
  extern __shared__ int32_t ssm[];
  assemble_body(tasks[blockIdx.x], segs, sn, rows, U, L, ssm);
}

// Persistent form for problems whose supernodes all take the one-CTA kernel
// (e.g. batches of small systems): one cooperative launch walks every level,
// grid-wide barriers separating the factor step of a level from its assembly
// and the assembly from the next level. The per-supernode and per-task work is
// the same code as the level-by-level kernels, so the results are identical.
template <int NT>
__global__ void __launch_bounds__(NT)
k_persist_factor(const SnodeDev* __restrict__ sn, const int32_t* __restrict__ small_list,
                 const AsmTask* __restrict__ tasks, const AsmSeg* __restrict__ segs,
                 const int32_t* __restrict__ rows, const PersistLevel* __restrict__ lv, int nlevels,
                 double* __restrict__ L, double* __restrict__ U, int* status) {
  extern __shared__ double psm[];
  cg::grid_group grid = cg::this_grid();
  for (int l = 0; l < nlevels; ++l) {
    const PersistLevel p = lv[l];
    for (int i = blockIdx.x; i < p.small_n; i += gridDim.x) {
      __syncthreads();
      small_body(sn[small_list[p.small_b + i]], L, U, status, psm);
    }
    grid.sync();
    for (int i = blockIdx.x; i < p.asm_n; i += gridDim.x) {
      __syncthreads();
      assemble_body(tasks[p.asm_b + i], segs, sn, rows, U, L, reinterpret_cast<int32_t*>(psm));
    }
    {
      // warp-sized tasks: one per warp of the grid, each warp in its own slice
      __syncthreads();
      int32_t* wsm = reinterpret_cast<int32_t*>(psm) + (threadIdx.x >> 5) * 2 * kAsmWarpPos;
      const int nw = NT / 32;
      for (int i = blockIdx.x * nw + (threadIdx.x >> 5); i < p.asmw_n; i += gridDim.x * nw)
        assemble_warp_task<double, false>(tasks[p.asm_b + p.asm_n + i], segs, sn, rows, U, L, wsm,
                                          wsm + kAsmWarpPos);
    }
    grid.sync();
  }
}

// log det: per-supernode partial sums, then one fixed-order reduction.
__global__ void k_logdet_part(const SnodeDev* __restrict__ sn, const double* __restrict__ L,
                              double* __restrict__ part) {
  __shared__ double red[128];
  const SnodeDev d = sn[blockIdx.x];
  double acc = 0.0;
  for (int c = threadIdx.x; c < d.s; c += blockDim.x) acc += log(L[d.loff + c + (int64_t)c * d.ld]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

// log det of every system: 2 x the supernode partials of its range, in order.
__global__ void k_logdet_sys(const double* __restrict__ part, const int32_t* __restrict__ sys_snode, int count,
                             double* __restrict__ out) {
  const int q = blockIdx.x * blockDim.x + threadIdx.x;
  if (q >= count) return;
  double acc = 0.0;
  for (int J = sys_snode[q]; J < sys_snode[q + 1]; ++J) acc += part[J];
  out[q] = 2.0 * acc;
}

__global__ void k_logdet_reduce(const double* __restrict__ part, int ns, double* out) {
  __shared__ double red[1024];
  double acc = 0.0;
  for (int i = threadIdx.x; i < ns; i += blockDim.x) acc += part[i];
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = 2.0 * red[0];
}

// out[t] = vals[src[t]]
__global__ void k_gather_src(const double* __restrict__ vals, const int64_t* __restrict__ src, int64_t m,
                             double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = vals[src[t]];
}

// out[t] = L[map[t]] (panel entries -> compressed sparse column order).
__global__ void k_gather(const double* __restrict__ L, const int64_t* __restrict__ map, int64_t nnz,
                         double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = L[map[t]];
}

template <class T>
int upload(chol_handle* h, T** dst, const std::vector<T>& v) {
  if (v.empty()) { *dst = nullptr; return CHOL_OK; }
  int rc = chol_dalloc(h, (void**)dst, v.size() * sizeof(T));
  if (rc) return rc;
  CHOL_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return CHOL_OK;
}

inline unsigned grid1d(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g > 0 ? g : 1);
}

}  // namespace

void chol_prof_resolve(chol_handle* h) {
  Profiler* p = h->prof;
  if (!p || p->pending.empty()) return;
  for (auto& q : p->pending) cudaEventSynchronize(q.b);   // launches may be on several streams
  for (auto& q : p->pending) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, q.a, q.b) == cudaSuccess) {
      p->st[q.cls].ms += ms;
      p->st[q.cls].timed++;
    }
    p->pool.push_back(q.a);
    p->pool.push_back(q.b);
  }
  p->pending.clear();
  cudaGetLastError();
}

void chol_prof_free(chol_handle* h) {
  Profiler* p = h->prof;
  if (!p) return;
  chol_prof_resolve(h);
  for (cudaEvent_t e : p->pool) cudaEventDestroy(e);
  delete p;
  h->prof = nullptr;
}

extern "C" int chol_profile(chol_handle* h, uint32_t timing_mask) {
  if (!h) return -1;
  chol_prof_resolve(h);
  chol_prof(h)->mask = timing_mask;
  return CHOL_OK;
}

extern "C" int chol_get_stats(chol_handle* h, chol_kernel_stat* out, int32_t reset) {
  if (!h) return -1;
  if (!out) return -2;
  chol_prof_resolve(h);
  Profiler* p = chol_prof(h);
  std::memcpy(out, p->st, sizeof(p->st));
  if (reset) std::memset(p->st, 0, sizeof(p->st));
  return CHOL_OK;
}

void chol_status_init(int* status, cudaStream_t st) { k_status_init<<<1, 1, 0, st>>>(status); }

int chol_dalloc(chol_handle* h, void** p, size_t bytes) {
  DeviceState* D = h->dev;
  *p = nullptr;
  if (bytes == 0) return CHOL_OK;
  if (h->opt.device_mem_cap > 0 && D->bytes + (int64_t)bytes > h->opt.device_mem_cap) return CHOL_ENOMEM;
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? CHOL_ENOMEM : CHOL_ECUDA;
  }
  D->bytes += (int64_t)bytes;
  return CHOL_OK;
}

void chol_device_free(chol_handle* h) {
  chol_prof_free(h);
  DeviceState* D = h->dev;
  if (!D) return;
  int cur = -1;
  cudaGetDevice(&cur);
  if (D->device >= 0) cudaSetDevice(D->device);
  chol_adjoint_free(h);
  void* ptrs[] = {D->L, D->U, D->sn, D->rows, D->amap, D->small_list, D->potrf_list,
                  D->level_snodes, D->trsm, D->gemm, D->syrk, D->asm_tasks, D->asm_segs, D->tri, D->rlb_pairs, D->rlb_pbeg, D->zrr_ws,
                  D->tri_flags, D->tri_sync, D->sv_err, D->bpanel, D->gemv, D->bpart, D->bred, D->P32, D->plevels, D->vals, D->sys_snode, D->sys_out,
                  D->ssmall, D->Zp, D->Tw, D->Ww, D->Uh, D->a_col, D->a_row, D->adj_xb, D->perm, D->status, D->part, D->scalar_dev, D->Y, D->W,
                  D->mx_diagpos, D->mx_aij, D->mx_d, D->mx_fallbacks, D->csr_ptr, D->csr_col, D->csr_src,
                  D->csr_val, D->Lbf, D->tmaps, D->tc_err, D->R, D->Z, D->Pv, D->Q, D->red, D->Y32, D->W32,
                  D->rhs_scale, D->host_vals, D->host_rhs, D->panel, D->pflags, D->dinv, D->split_part, D->split_cnt, D->hand32};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  if (D->status_host) cudaFreeHost(D->status_host);
  if (D->scalar_host) cudaFreeHost(D->scalar_host);
  if (D->red_host) cudaFreeHost(D->red_host);
  if (D->graph_exec) cudaGraphExecDestroy(D->graph_exec);
  if (D->gstream) cudaStreamDestroy(D->gstream);
  if (D->lstream) cudaStreamDestroy(D->lstream);
  if (D->hstream) cudaStreamDestroy(D->hstream);
  if (D->istream) cudaStreamDestroy(D->istream);
  for (cudaEvent_t e : D->lev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : D->iev)
    if (e) cudaEventDestroy(e);
  for (cudaEvent_t e : D->gev)
    if (e) cudaEventDestroy(e);
  if (cur >= 0) cudaSetDevice(cur);
  delete D;
  h->dev = nullptr;
}

int chol_device_ensure(chol_handle* h) {
  if (h->dev) {
    int cur = -1;
    CHOL_CUDA_TRY(cudaGetDevice(&cur));
    return cur == h->dev->device ? CHOL_OK : CHOL_ESTATE;
  }
  h->dev = new DeviceState();
  DeviceState* D = h->dev;
  int rc = CHOL_OK;
  auto fail = [&](int code) {
    chol_device_free(h);
    return code;
  };
  if (cudaGetDevice(&D->device) != cudaSuccess) return fail(CHOL_ECUDA);
  {
    // the lookahead's critical path (POTRF, TRSM, next column block) runs on a
    // highest-priority stream so that its CTAs are placed ahead of the side
    // stream's trailing tiles
    int lo = 0, hi = 0;
    if (cudaDeviceGetStreamPriorityRange(&lo, &hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&D->hstream, cudaStreamNonBlocking, hi) != cudaSuccess ||
        cudaStreamCreateWithPriority(&D->lstream, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaStreamCreateWithPriority(&D->istream, cudaStreamNonBlocking, lo) != cudaSuccess ||
        cudaEventCreateWithFlags(&D->iev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&D->iev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&D->lev[0], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&D->lev[1], cudaEventDisableTiming) != cudaSuccess ||
        cudaEventCreateWithFlags(&D->lev[2], cudaEventDisableTiming) != cudaSuccess)
      return fail(CHOL_ECUDA);
  }
  if (cudaDeviceGetAttribute(&D->sms, cudaDevAttrMultiProcessorCount, D->device) != cudaSuccess) return fail(CHOL_ECUDA);
  if (h->opt.precision != CHOL_PREC_FP64) {
    // the tensor-core and binary32 kernels are built for this architecture only
    cudaDeviceProp prop;
    if (cudaGetDeviceProperties(&prop, D->device) != cudaSuccess) return fail(CHOL_ECUDA);
    if (prop.major != 10) return fail(CHOL_ENOTSUP);
  }
  const size_t esz = h->opt.precision == CHOL_PREC_FP64 ? sizeof(double) : sizeof(float);
  if ((rc = chol_dalloc(h, (void**)&D->L, esz * (size_t)std::max<int64_t>(h->panel_doubles, 1)))) return fail(rc);
  if ((rc = chol_dalloc(h, (void**)&D->U, esz * (size_t)std::max<int64_t>(h->update_doubles, 1)))) return fail(rc);
  if ((rc = upload(h, &D->csr_ptr, h->csr_ptr))) return fail(rc);
  if ((rc = upload(h, &D->csr_col, h->csr_col))) return fail(rc);
  if ((rc = upload(h, &D->csr_src, h->csr_src))) return fail(rc);
  if ((rc = chol_dalloc(h, (void**)&D->csr_val, sizeof(double) * (size_t)std::max<int64_t>(h->csr_ptr[h->n], 1))))
    return fail(rc);
  if ((rc = upload(h, &D->sn, h->snodes))) return fail(rc);
  if ((rc = upload(h, &D->rows, h->rows))) return fail(rc);
  if ((rc = upload(h, &D->amap, h->amap))) return fail(rc);
  if ((rc = upload(h, &D->small_list, h->small_list))) return fail(rc);
  if ((rc = upload(h, &D->potrf_list, h->potrf_list))) return fail(rc);
  if ((rc = upload(h, &D->level_snodes, h->level_snodes))) return fail(rc);
  if ((rc = upload(h, &D->trsm, h->trsm_tasks))) return fail(rc);
  if ((rc = upload(h, &D->gemm, h->gemm_tasks))) return fail(rc);
  if ((rc = upload(h, &D->syrk, h->syrk_tasks))) return fail(rc);
  if ((rc = upload(h, &D->asm_tasks, h->asm_tasks))) return fail(rc);
  if ((rc = upload(h, &D->asm_segs, h->asm_segs))) return fail(rc);
  if ((rc = upload(h, &D->tri, h->tri_items))) return fail(rc);
  if (h->opt.update_mode == CHOL_UPDATE_RLB) {
    std::vector<int4> pr(h->rel_J.size());
    for (size_t p = 0; p < pr.size(); ++p) pr[p] = make_int4(h->rel_K[p], h->rel_c0[p], h->rel_c1[p], 0);
    if ((rc = upload(h, &D->rlb_pairs, pr))) return fail(rc);
    if ((rc = upload(h, &D->rlb_pbeg, h->pair_beg))) return fail(rc);
  }
  // one flag per diagonal block and right-hand-side column of a chunk
  const size_t nflags = (size_t)std::max(h->tri_nflags, 1) * kSolveChunk;
  if ((rc = chol_dalloc(h, (void**)&D->tri_flags, sizeof(int32_t) * nflags))) return fail(rc);
  if (h->opt.precision == CHOL_PREC_FP64) {
    if ((rc = chol_dalloc(h, &D->dinv, sizeof(double) * 64 * 64 * (size_t)std::max(h->tri_nflags, 1))))
      return fail(rc);
    const size_t slots = (size_t)std::max<int64_t>(h->split_slots_max, 1);
    if ((rc = chol_dalloc(h, (void**)&D->split_part, sizeof(double) * 64 * kSolveChunk * slots))) return fail(rc);
    if ((rc = chol_dalloc(h, (void**)&D->split_cnt, sizeof(int32_t) * slots))) return fail(rc);
    if (cudaMemset(D->split_cnt, 0, sizeof(int32_t) * slots) != cudaSuccess) return fail(CHOL_ECUDA);
  }
  if ((rc = chol_dalloc(h, (void**)&D->tri_sync, sizeof(int32_t) * 2))) return fail(rc);
  if ((rc = chol_dalloc(h, (void**)&D->sv_err, sizeof(int32_t)))) return fail(rc);
  if (cudaMemset(D->tri_flags, 0, sizeof(int32_t) * nflags) != cudaSuccess ||
      cudaMemset(D->tri_sync, 0, sizeof(int32_t) * 2) != cudaSuccess ||
      cudaMemset(D->sv_err, 0, sizeof(int32_t)) != cudaSuccess)
    return fail(CHOL_ECUDA);
  if ((rc = upload(h, &D->ssmall, h->ssmall_list))) return fail(rc);
  if ((rc = upload(h, &D->bpanel, h->bpanel_tasks))) return fail(rc);
  if ((rc = upload(h, &D->gemv, h->gemv_tasks))) return fail(rc);
  if ((rc = upload(h, &D->bpart, h->bpart_tasks))) return fail(rc);
  if ((rc = upload(h, &D->bred, h->bred_tasks))) return fail(rc);
  if ((rc = upload(h, &D->plevels, h->persist_levels))) return fail(rc);
  if ((rc = upload(h, &D->perm, h->perm))) return fail(rc);
  if ((rc = chol_dalloc(h, (void**)&D->status, sizeof(int32_t)))) return fail(rc);
  if ((rc = chol_dalloc(h, (void**)&D->part, sizeof(double) * (size_t)std::max(h->ns, 1)))) return fail(rc);
  if ((rc = chol_dalloc(h, (void**)&D->scalar_dev, sizeof(double)))) return fail(rc);
  if (cudaMallocHost((void**)&D->status_host, 4 * sizeof(int32_t)) != cudaSuccess) return fail(CHOL_ENOMEM);
  if (cudaMallocHost((void**)&D->scalar_host, sizeof(double)) != cudaSuccess) return fail(CHOL_ENOMEM);
  static bool attrs_done = false;
  if (!attrs_done) {
    if (cudaFuncSetAttribute(k_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
      return fail(CHOL_ECUDA);
    if (cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize, 24576 * 8) != cudaSuccess)
      return fail(CHOL_ECUDA);
    if (cudaFuncSetAttribute(k_small_rlb, cudaFuncAttributeMaxDynamicSharedMemorySize, 24576 * 8) != cudaSuccess)
      return fail(CHOL_ECUDA);
    attrs_done = true;
  }
  return CHOL_OK;
}

namespace {

// Enqueue the binary64 factorization (no synchronization).
int enqueue_factor_fp64(chol_handle* h, const double* values, cudaStream_t st) {
  DeviceState* D = h->dev;
  const int nb = h->opt.block_cols;
  k_status_init<<<1, 1, 0, st>>>(D->status);
  CHOL_CUDA_TRY(cudaMemsetAsync(D->L, 0, sizeof(double) * (size_t)h->panel_doubles, st));
  if (h->nnz_a > 0) {
    KScope ks(h, CHOL_K_SCATTER, st, 0.0, 24.0 * (double)h->nnz_a);
    k_scatter<<<grid1d(h->nnz_a, 256), 256, 0, st>>>(values, D->amap, h->nnz_a, D->L);
    // binary64 copy of A in CSR order for residuals (chol_solve_refine)
    const int64_t m = h->csr_ptr[h->n];
    k_gather_src<<<grid1d(m, 256), 256, 0, st>>>(values, D->csr_src, m, D->csr_val);
  }
  if (h->opt.persistent) {
    if (h->n_large > 0 || h->opt.update_mode != CHOL_UPDATE_RL) return CHOL_ENOTSUP;
    double fl = 0.0, by = 0.0;
    for (const LevelPlan& P : h->levels) { fl += P.small_flops; by += P.small_bytes; }
    {
      KScope ks(h, CHOL_K_SMALL, st, fl, by);
      const int rc = chol_launch_persistent(h, (void*)D->L, (void*)D->U, st);
      if (rc) return rc;
    }
    return chol_diag_inv(h, 0, (int)h->tri_items.size(), st);
  }
  // levels with blocked supernodes run on the high-priority stream (forked from
  // and joined back to the caller's stream)
  const cudaStream_t caller = st;
  if (h->n_large > 0) {
    CHOL_CUDA_TRY(cudaEventRecord(D->lev[2], caller));
    CHOL_CUDA_TRY(cudaStreamWaitEvent(D->hstream, D->lev[2], 0));
    st = D->hstream;
  }
  bool inv_pending = false;
  for (const LevelPlan& P : h->levels) {
    NvtxRange nvtx_level("level", (long long)(&P - h->levels.data()));
    const bool rlb = h->opt.update_mode == CHOL_UPDATE_RLB;
    if (P.small_n > 0) {
      KScope ks(h, CHOL_K_SMALL, st, P.small_flops, P.small_bytes);
      if (rlb)
        k_small_rlb<<<P.small_n, kSmallThreads, sizeof(double) * P.small_max_panel, st>>>(
            D->sn, D->small_list + P.small_b, D->rlb_pairs, D->rlb_pbeg, D->rows, D->L, D->status);
      else
        k_small<<<P.small_n, kSmallThreads, sizeof(double) * P.small_max_panel, st>>>(
            D->sn, D->small_list + P.small_b, D->L, D->U, D->status);
    }
    // One-step lookahead: the trailing tiles of step k other than the next
    // block column ("rest") run on the side stream, beside the POTRF and TRSM
    // of step k + 1 on the main stream. Before step k + 1's own trailing tiles,
    // the main stream waits for step k's rest (they share tiles); the side
    // stream keeps the rests in order. Each tile still receives its updates in
    // step order, so the result is the same as without lookahead.
    bool rest_pending = false;
    for (size_t k = 0; k < P.steps.size(); ++k) {
      const StepRange& s = P.steps[k];
      const int k0 = (int)k * nb;
      if (s.potrf_n > 0) {
        KScope ks(h, CHOL_K_POTRF, st, s.potrf_flops, 16.0 * nb * nb * s.potrf_n);
        k_potrf<<<s.potrf_n, kPotrfThreads, 0, st>>>(D->sn, D->potrf_list + s.potrf_b, k0, nb, D->L,
                                                     D->status);
      }
      if (s.trsm_n > 0) {
        KScope ks(h, CHOL_K_TRSM, st, s.trsm_flops, 16.0 * kTrsmRows * nb * s.trsm_n);
        k_trsm<<<s.trsm_n, kTrsmThreads, 0, st>>>(D->sn, D->trsm + s.trsm_b, nb, D->L);
      }
      const int nrest = s.gemm_n - s.gemm_next;
      if (nrest > 0) {
        CHOL_CUDA_TRY(cudaEventRecord(D->lev[0], st));   // step k's panel is final
        CHOL_CUDA_TRY(cudaStreamWaitEvent(D->lstream, D->lev[0], 0));
      }
      if (rest_pending) {
        CHOL_CUDA_TRY(cudaStreamWaitEvent(st, D->lev[1], 0));   // step k-1's rest
        rest_pending = false;
      }
      if (s.gemm_n > 0) {
        const double frac = (double)s.gemm_next / s.gemm_n;
        if (s.gemm_next > 0) {
          KScope ks(h, CHOL_K_GEMM, st, s.gemm_flops * frac, 16.0 * kTile * kTile * s.gemm_next);
          k_gemm_trailing<<<s.gemm_next, kGemmThreads, 0, st>>>(D->sn, D->gemm + s.gemm_b, nb, D->L);
        }
        if (nrest > 0) {
          KScope ks(h, CHOL_K_GEMM, D->lstream, s.gemm_flops * (1.0 - frac), 16.0 * kTile * kTile * nrest);
          k_gemm_trailing<<<nrest, kGemmThreads, 0, D->lstream>>>(D->sn, D->gemm + s.gemm_b + s.gemm_next, nb,
                                                                  D->L);
          CHOL_CUDA_TRY(cudaEventRecord(D->lev[1], D->lstream));
          rest_pending = true;
        }
      }
    }
    if (rest_pending) CHOL_CUDA_TRY(cudaStreamWaitEvent(st, D->lev[1], 0));   // join before SYRK
    // the level's diagonal blocks are final: their inverses (for the triangle
    // solves) on a side stream, beside the SYRK, the assembly and later levels
    if (P.tri_n > 0) {
      CHOL_CUDA_TRY(cudaEventRecord(D->iev[0], st));
      CHOL_CUDA_TRY(cudaStreamWaitEvent(D->istream, D->iev[0], 0));
      if (int rc = chol_diag_inv(h, P.tri_b, P.tri_n, D->istream)) return rc;
      inv_pending = true;
    }
    if (P.syrk_n > 0) {
      KScope ks(h, CHOL_K_SYRK, st, P.syrk_flops, 8.0 * kTile * kTile * P.syrk_n);
      if (rlb)
        k_syrk_rlb<<<P.syrk_n, kGemmThreads, 0, st>>>(D->sn, D->syrk + P.syrk_b, D->rlb_pairs, D->rlb_pbeg, D->rows,
                                                       D->L);
      else
        k_syrk<<<P.syrk_n, kGemmThreads, 0, st>>>(D->sn, D->syrk + P.syrk_b, D->L, D->U);
    }
    if (!rlb && P.asm_n + P.asmw_n > 0) {
      KScope ks(h, CHOL_K_ASSEMBLE, st, P.asm_entries, 24.0 * P.asm_entries);
      ks.launches((P.asm_n > 0) + (P.asmw_n > 0));
      if (P.asm_n > 0)
        k_assemble<<<P.asm_n, kAsmThreads, sizeof(int32_t) * 2 * kAsmPos, st>>>(
            D->asm_tasks + P.asm_b, D->asm_segs, D->sn, D->rows, D->U, D->L);
      if (P.asmw_n > 0)
        k_assemble_warp<double, false><<<(P.asmw_n + 7) / 8, 256, 0, st>>>(
            D->asm_tasks + P.asm_b + P.asm_n, P.asmw_n, D->asm_segs, D->sn, D->rows, D->U, D->L);
    }
  }
  if (inv_pending) {   // the inverses join the factor's stream before it ends
    CHOL_CUDA_TRY(cudaEventRecord(D->iev[1], D->istream));
    CHOL_CUDA_TRY(cudaStreamWaitEvent(st, D->iev[1], 0));
  }
  if (st != caller) {
    CHOL_CUDA_TRY(cudaEventRecord(D->lev[2], st));
    CHOL_CUDA_TRY(cudaStreamWaitEvent(caller, D->lev[2], 0));
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

int enqueue_factor(chol_handle* h, const double* values, cudaStream_t st) {
  if (h->opt.precision == CHOL_PREC_FP64) return enqueue_factor_fp64(h, values, st);   // inverses inside
  const int rc = chol_enqueue_factor_mixed(h, values, st);
  if (rc) return rc;
  // the binary32 triangle solve multiplies by the diagonal blocks' inverses
  return chol_diag_inv(h, 0, (int)h->tri_items.size(), st);
}

void drop_graph(chol_handle* h) {
  DeviceState* D = h->dev;
  if (D && D->graph_exec) {
    cudaGraphExecDestroy(D->graph_exec);
    D->graph_exec = nullptr;
  }
}

}  // namespace

// The one-CTA-per-supernode levels in a single cooperative launch.
int chol_launch_persistent(chol_handle* h, void* L, void* U, cudaStream_t st) {
  DeviceState* D = h->dev;
  const bool fp64 = h->opt.precision == CHOL_PREC_FP64;
  const size_t esz = fp64 ? sizeof(double) : sizeof(float);
  const size_t smem = std::max(esz * (size_t)std::max(h->small_panel_max, 1),
                               sizeof(int32_t) * 2 * (size_t)std::max(kAsmPos, 8 * kAsmWarpPos)) + 64;
  const int threads = h->persist_threads == 256 ? 256 : 128;
  const void* fn = chol_persistent_kernel(h->opt.precision, threads);
  if (!fn) return CHOL_ENOTSUP;
  CHOL_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int per_sm = 0, sms = 0;
  CHOL_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, threads, smem));
  CHOL_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, D->device));
  if (per_sm < 1) return CHOL_ENOTSUP;
  if (h->persist_ctas > 0) per_sm = std::min(per_sm, h->persist_ctas);
  const int grid = per_sm * sms;
  int nlevels = h->nlevels;
  D->mx_spiv = h->opt.static_pivot ? (float)h->opt.pivot_tau : 0.f;
  void* args[] = {(void*)&D->sn, (void*)&D->small_list, (void*)&D->asm_tasks, (void*)&D->asm_segs,
                  (void*)&D->rows, (void*)&D->plevels, (void*)&nlevels, (void*)&L, (void*)&U,
                  (void*)&D->status, (void*)&D->mx_spiv, (void*)&D->mx_fallbacks};
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(threads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  CHOL_CUDA_TRY(cudaLaunchKernelExC(&cfg, fn, args));
  return CHOL_OK;
}

const void* chol_persistent_kernel(int precision, int threads) {
  if (precision == CHOL_PREC_FP64)
    return threads == 256 ? (const void*)k_persist_factor<256> : (const void*)k_persist_factor<128>;
  return chol_persistent_kernel_mixed(threads);
}

extern "C" int chol_factor(chol_handle* h, const double* values, void* stream) {
  NvtxRange nvtx_range("chol_factor");
  if (!h) return -1;
  if (!values && h->nnz_a > 0) return -2;
  int rc = chol_device_ensure(h);
  if (rc) return rc;
  DeviceState* D = h->dev;
  cudaStream_t st = (cudaStream_t)stream;
  h->factored = false;
  h->selinv_valid = false;
  if (h->opt.precision != CHOL_PREC_FP64 && (rc = chol_mixed_ensure(h))) return rc;
  h->bounds_code = 0;
#ifdef CHOL_BOUNDS_CHECK
  if (bc_begin(h) || chol_bc_begin_mixed(h)) return CHOL_ECUDA;
#endif
  if (h->opt.use_graph) {
    // replay a graph of the whole launch sequence; the values go through a copy
    // owned by the handle so that the captured pointers stay valid. Capture and
    // replay run on a stream of the handle (any caller stream can be captured
    // from that way, the legacy default stream included), joined to the
    // caller's stream with events on both sides.
    if (!D->gstream) {
      CHOL_CUDA_TRY(cudaStreamCreateWithFlags(&D->gstream, cudaStreamNonBlocking));
      CHOL_CUDA_TRY(cudaEventCreateWithFlags(&D->gev[0], cudaEventDisableTiming));
      CHOL_CUDA_TRY(cudaEventCreateWithFlags(&D->gev[1], cudaEventDisableTiming));
    }
    const cudaStream_t caller = st;
    CHOL_CUDA_TRY(cudaEventRecord(D->gev[0], caller));
    CHOL_CUDA_TRY(cudaStreamWaitEvent(D->gstream, D->gev[0], 0));
    st = D->gstream;
    if (!D->vals && h->nnz_a > 0) {
      if ((rc = chol_dalloc(h, (void**)&D->vals, sizeof(double) * (size_t)h->nnz_a))) return rc;
    }
    if (h->nnz_a > 0)
      CHOL_CUDA_TRY(cudaMemcpyAsync(D->vals, values, sizeof(double) * (size_t)h->nnz_a, cudaMemcpyDeviceToDevice, st));
    Profiler* pr = chol_prof(h);
    if (!D->graph_exec) {
      chol_prof_resolve(h);
      chol_kernel_stat before[CHOL_K_NCLASSES];
      std::memcpy(before, pr->st, sizeof(before));
      const uint32_t mask = pr->mask;
      pr->mask = 0;   // no event timing inside the captured sequence
      cudaGraph_t graph = nullptr;
      CHOL_CUDA_TRY(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
      rc = enqueue_factor(h, D->vals, st);
      const cudaError_t ce = cudaStreamEndCapture(st, &graph);
      pr->mask = mask;
      if (rc) { if (graph) cudaGraphDestroy(graph); return rc; }
      if (ce != cudaSuccess) { cudaGetLastError(); return CHOL_ECUDA; }
      const cudaError_t ie = cudaGraphInstantiate(&D->graph_exec, graph, 0);
      cudaGraphDestroy(graph);
      if (ie != cudaSuccess) { cudaGetLastError(); D->graph_exec = nullptr; return CHOL_ECUDA; }
      for (int c = 0; c < CHOL_K_NCLASSES; ++c) {     // per-replay launch accounting
        D->graph_delta[c].launches = pr->st[c].launches - before[c].launches;
        D->graph_delta[c].flops = pr->st[c].flops - before[c].flops;
        D->graph_delta[c].bytes = pr->st[c].bytes - before[c].bytes;
      }
      std::memcpy(pr->st, before, sizeof(before));
    }
    CHOL_CUDA_TRY(cudaGraphLaunch(D->graph_exec, st));
    for (int c = 0; c < CHOL_K_NCLASSES; ++c) {
      pr->st[c].launches += D->graph_delta[c].launches;
      pr->st[c].flops += D->graph_delta[c].flops;
      pr->st[c].bytes += D->graph_delta[c].bytes;
    }
    CHOL_CUDA_TRY(cudaEventRecord(D->gev[1], st));
    CHOL_CUDA_TRY(cudaStreamWaitEvent(caller, D->gev[1], 0));
    st = caller;
  } else {
    if ((rc = enqueue_factor(h, values, st))) return rc;
  }
  return chol_finish_factor(h, st);
}

// Read the status word (and the mixed-mode counters) after a factorization.
int chol_finish_factor(chol_handle* h, cudaStream_t st) {
  DeviceState* D = h->dev;
  CHOL_CUDA_TRY(cudaGetLastError());
  CHOL_CUDA_TRY(cudaMemcpyAsync(D->status_host, D->status, sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  if (h->opt.precision != CHOL_PREC_FP64)
    CHOL_CUDA_TRY(cudaMemcpyAsync(&D->status_host[1], D->mx_fallbacks, 2 * sizeof(int32_t), cudaMemcpyDeviceToHost, st));
  CHOL_CUDA_TRY(cudaStreamSynchronize(st));
  if (h->opt.precision != CHOL_PREC_FP64) {
    h->fp64_fallbacks = D->status_host[1];
    h->perturbed_pivots = D->status_host[2];
  }
#ifdef CHOL_BOUNDS_CHECK
  {
    const int e1 = bc_read(), e2 = chol_bc_read_mixed();
    if (e1 < 0 || e2 < 0) return CHOL_ECUDA;
    if (e1 || e2) {
      h->bounds_code = e1 ? e1 : e2;
      return CHOL_EBOUNDS;
    }
  }
#endif
  const int32_t s = D->status_host[0];
  if (s != INT_MAX) return s;
  if (h->opt.precision != CHOL_PREC_FP64) {
    const int rc = chol_tc_status(h);
    if (rc) return rc;
  }
  {
    const int rc = chol_solve_status(h);
    if (rc) return rc;
  }
  h->factored = true;
  return CHOL_OK;
}

extern "C" int chol_test_corrupt_plan(chol_handle* h, int32_t kind) {
#ifdef CHOL_BOUNDS_CHECK
  if (!h) return -1;
  if (h->dev) return CHOL_ESTATE;   // the plan is uploaded by the first factorization
  // first level with a CTA-sized (kind 1-3) or a warp-sized (kind 5) assembly task
  const LevelPlan* cta = nullptr;
  const LevelPlan* warp = nullptr;
  for (const LevelPlan& P : h->levels) {
    if (!cta && P.asm_n > 0) cta = &P;
    if (!warp && P.asmw_n > 0) warp = &P;
  }
  switch (kind) {
    case 1:   // a segment's source supernode out of range
      if (!cta) return CHOL_ENOTSUP;
      h->asm_segs[h->asm_tasks[cta->asm_b].seg_begin].J = h->ns + 5;
      return CHOL_OK;
    case 2: {  // a segment's rows past U_J
      if (!cta) return CHOL_ENOTSUP;
      AsmSeg& g = h->asm_segs[h->asm_tasks[cta->asm_b].seg_begin];
      g.ub = h->snodes[g.J].len - h->snodes[g.J].s + 100;
      return CHOL_OK;
    }
    case 3: {  // a task's row positions past the target
      if (!cta) return CHOL_ENOTSUP;
      AsmTask& t = h->asm_tasks[cta->asm_b];
      t.p1 = h->snodes[t.K].len + 50;
      return CHOL_OK;
    }
    case 4:   // a value's panel position past the panels
      if (h->amap.empty()) return CHOL_ENOTSUP;
      h->amap[0] = h->panel_doubles + 1000;
      return CHOL_OK;
    case 5:   // a warp task's segment source out of range (negative)
      if (!warp) return CHOL_ENOTSUP;
      h->asm_segs[h->asm_tasks[warp->asm_b + warp->asm_n].seg_begin].J = -3;
      return CHOL_OK;
    default:
      return -2;
  }
#else
  (void)h;
  (void)kind;
  return CHOL_ENOTSUP;
#endif
}

extern "C" int chol_autotune(chol_handle* h, const double* values, void* stream) {
  NvtxRange nvtx_range("chol_autotune");
  if (!h) return -1;
  if (!values && h->nnz_a > 0) return -2;
  cudaStream_t st = (cudaStream_t)stream;
  struct Cand { int persistent, graph, threads, ctas; };
  std::vector<Cand> cands = {{0, 0, 128, 0}, {0, 1, 128, 0}};
  if (h->n_large == 0 && h->opt.update_mode == CHOL_UPDATE_RL)   // the persistent kernel assembles through U
    for (int t : {128, 256})
      for (int c : {1, 2, 4, 0}) cands.push_back({1, 1, t, c});
  float best = 1e30f;
  Cand win = cands[0];
  int rc = CHOL_OK;
  cudaEvent_t e0, e1;
  CHOL_CUDA_TRY(cudaEventCreate(&e0));
  CHOL_CUDA_TRY(cudaEventCreate(&e1));
  for (const Cand& c : cands) {
    h->opt.persistent = c.persistent;
    h->opt.use_graph = c.graph;
    h->persist_threads = c.threads;
    h->persist_ctas = c.ctas;
    if (h->dev) drop_graph(h);
    if ((rc = chol_factor(h, values, stream))) break;   // warm-up (and capture)
    float tmin = 1e30f;
    for (int rep = 0; rep < 2; ++rep) {
      cudaEventRecord(e0, st);
      if ((rc = chol_factor(h, values, stream))) break;
      cudaEventRecord(e1, st);
      cudaEventSynchronize(e1);
      float ms = 0.f;
      cudaEventElapsedTime(&ms, e0, e1);
      tmin = std::min(tmin, ms);
    }
    if (rc) break;
    if (tmin < best) { best = tmin; win = c; }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  h->opt.persistent = win.persistent;
  h->opt.use_graph = win.graph;
  h->persist_threads = win.threads;
  h->persist_ctas = win.ctas;
  if (h->dev) drop_graph(h);
  if (rc) return rc;
  return chol_factor(h, values, stream);
}

extern "C" int chol_logdet_batch(chol_handle* h, double* out, void* stream) {
  if (!h) return -1;
  if (!out) return -2;
  if (int rc_state = chol_factored_here(h)) return rc_state;
  DeviceState* D = h->dev;
  cudaStream_t st = (cudaStream_t)stream;
  const int count = (int)h->sys_ptr.size() - 1;
  if (count <= 0) return CHOL_OK;
  int rc;
  if (!D->sys_snode) {
    if ((rc = upload(h, &D->sys_snode, h->sys_snode_ptr))) return rc;
    if ((rc = chol_dalloc(h, (void**)&D->sys_out, sizeof(double) * (size_t)count))) return rc;
  }
  if (h->ns > 0) {
    if (h->opt.precision == CHOL_PREC_FP64)
      k_logdet_part<<<h->ns, 128, 0, st>>>(D->sn, D->L, D->part);
    else if ((rc = chol_logdet_parts_mixed(h, st)))
      return rc;
  }
  k_logdet_sys<<<(count + 127) / 128, 128, 0, st>>>(D->part, D->sys_snode, count, D->sys_out);
  CHOL_CUDA_TRY(cudaGetLastError());
  CHOL_CUDA_TRY(cudaMemcpyAsync(out, D->sys_out, sizeof(double) * (size_t)count, cudaMemcpyDeviceToHost, st));
  CHOL_CUDA_TRY(cudaStreamSynchronize(st));
  return CHOL_OK;
}

extern "C" int chol_logdet(chol_handle* h, double* out, void* stream) {
  if (!h) return -1;
  if (!out) return -2;
  if (int rc_state = chol_factored_here(h)) return rc_state;
  DeviceState* D = h->dev;
  cudaStream_t st = (cudaStream_t)stream;
  if (h->opt.precision != CHOL_PREC_FP64) return chol_logdet_mixed(h, out, st);
  if (h->ns > 0) {
    KScope ks(h, CHOL_K_LOGDET, st, (double)h->n, 8.0 * h->n);
    k_logdet_part<<<h->ns, 128, 0, st>>>(D->sn, D->L, D->part);
    k_logdet_reduce<<<1, 1024, 0, st>>>(D->part, h->ns, D->scalar_dev);
  } else {
    CHOL_CUDA_TRY(cudaMemsetAsync(D->scalar_dev, 0, sizeof(double), st));
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  CHOL_CUDA_TRY(cudaMemcpyAsync(D->scalar_host, D->scalar_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  CHOL_CUDA_TRY(cudaStreamSynchronize(st));
  *out = *D->scalar_host;
  return CHOL_OK;
}

extern "C" int chol_factor_solve_host(chol_handle* h, const double* values, const double* b, double* x,
                                      int32_t nrhs, double* logdet, void* stream) {
  NvtxRange nvtx_range("chol_factor_solve_host");
  if (!h) return -1;
  if (!values && h->nnz_a > 0) return -2;
  if (!b && nrhs > 0 && h->n > 0) return -3;
  if (!x && nrhs > 0 && h->n > 0) return -4;
  if (nrhs < 0) return -5;
  int rc = chol_device_ensure(h);
  if (rc) return rc;
  DeviceState* D = h->dev;
  cudaStream_t st = (cudaStream_t)stream;
  const size_t nb = (size_t)h->n * (size_t)nrhs;
  if (h->nnz_a > 0 && !D->host_vals) {
    if ((rc = chol_dalloc(h, (void**)&D->host_vals, sizeof(double) * (size_t)h->nnz_a))) return rc;
  }
  if (nb > (size_t)D->host_rhs_cap) {
    if (D->host_rhs) {
      cudaFree(D->host_rhs);
      D->bytes -= sizeof(double) * (size_t)D->host_rhs_cap;
      D->host_rhs = nullptr;
      D->host_rhs_cap = 0;
    }
    if ((rc = chol_dalloc(h, (void**)&D->host_rhs, sizeof(double) * nb))) return rc;
    D->host_rhs_cap = (int64_t)nb;
  }
  if (h->nnz_a > 0)
    CHOL_CUDA_TRY(cudaMemcpyAsync(D->host_vals, values, sizeof(double) * (size_t)h->nnz_a, cudaMemcpyHostToDevice, st));
  if ((rc = chol_factor(h, D->host_vals, stream))) return rc;
  if (nb > 0) {
    CHOL_CUDA_TRY(cudaMemcpyAsync(D->host_rhs, b, sizeof(double) * nb, cudaMemcpyHostToDevice, st));
    if ((rc = chol_solve(h, D->host_rhs, nrhs, stream))) return rc;
  }
  if (logdet && (rc = chol_logdet(h, logdet, stream))) return rc;
  if (nb > 0) CHOL_CUDA_TRY(cudaMemcpyAsync(x, D->host_rhs, sizeof(double) * nb, cudaMemcpyDeviceToHost, st));
  CHOL_CUDA_TRY(cudaStreamSynchronize(st));
  return chol_solve_status(h);
}

extern "C" int chol_get_factor(chol_handle* h, int64_t* lp, int32_t* li, double* lx, void* stream) {
  if (!h) return -1;
  if (int rc_state = chol_factored_here(h)) return rc_state;
  DeviceState* D = h->dev;
  cudaStream_t st = (cudaStream_t)stream;
  const int32_t n = h->n;
  const int32_t cns = (int32_t)h->c_sptr.size() - 1;
  std::vector<int64_t> hp(n + 1, 0);
  for (int32_t j = 0; j < n; ++j) hp[j + 1] = hp[j] + h->colcount[j];
  if (lp) std::memcpy(lp, hp.data(), sizeof(int64_t) * hp.size());
  // canonical column j: rows of its maximal supernode's structure from j on
  if (li) {
    for (int32_t K = 0; K < cns; ++K) {
      const int32_t f = h->c_sptr[K];
      const int32_t* r = h->c_rows.data() + h->c_rowptr[K];
      const int32_t len = (int32_t)(h->c_rowptr[K + 1] - h->c_rowptr[K]);
      for (int32_t c = 0; c < h->c_sptr[K + 1] - f; ++c)
        for (int32_t t = c; t < len; ++t) li[hp[f + c] + (t - c)] = r[t];
    }
  }
  if (lx && h->nnz_l > 0) {
    if (h->cscmap.empty()) {
      // entry of canonical column j -> its position in the storage panel
      h->cscmap.assign(h->nnz_l, 0);
      std::vector<int32_t> csnode(n), pos(n, -1);
      for (int32_t K = 0; K < cns; ++K)
        for (int32_t j = h->c_sptr[K]; j < h->c_sptr[K + 1]; ++j) csnode[j] = K;
      for (int32_t J = 0; J < h->ns; ++J) {
        const SnodeDev& d = h->snodes[J];
        const int32_t* r = h->rows.data() + d.roff;
        for (int32_t t = 0; t < d.len; ++t) pos[r[t]] = t;
        for (int32_t c = 0; c < d.s; ++c) {
          const int32_t j = d.f + c, K = csnode[j];
          const int32_t* rk = h->c_rows.data() + h->c_rowptr[K];
          const int32_t lenk = (int32_t)(h->c_rowptr[K + 1] - h->c_rowptr[K]);
          const int32_t ck = j - h->c_sptr[K];
          for (int32_t t = ck; t < lenk; ++t)
            h->cscmap[hp[j] + (t - ck)] = h->opt.precision == CHOL_PREC_FP64
                                              ? d.loff + (int64_t)c * d.ld + pos[rk[t]]
                                              : d.loff + (int64_t)pos[rk[t]] * d.ld + c;
        }
        for (int32_t t = 0; t < d.len; ++t) pos[r[t]] = -1;
      }
    }
    int64_t* dmap = nullptr;
    double* dlx = nullptr;
    int rc = chol_dalloc(h, (void**)&dmap, sizeof(int64_t) * (size_t)h->nnz_l);
    if (rc) return rc;
    rc = chol_dalloc(h, (void**)&dlx, sizeof(double) * (size_t)h->nnz_l);
    if (rc) {
      cudaFree(dmap);
      D->bytes -= sizeof(int64_t) * (size_t)h->nnz_l;
      return rc;
    }
    CHOL_CUDA_TRY(cudaMemcpyAsync(dmap, h->cscmap.data(), sizeof(int64_t) * (size_t)h->nnz_l,
                                  cudaMemcpyHostToDevice, st));
    if (h->opt.precision == CHOL_PREC_FP64) {
      k_gather<<<grid1d(h->nnz_l, 256), 256, 0, st>>>(D->L, dmap, h->nnz_l, dlx);
    } else {
      // L = D^{-1} L~: needs the permuted row of every entry
      std::vector<int32_t> lrow(h->nnz_l);
      for (int32_t K = 0; K < cns; ++K) {
        const int32_t f = h->c_sptr[K];
        const int32_t* r = h->c_rows.data() + h->c_rowptr[K];
        const int32_t len = (int32_t)(h->c_rowptr[K + 1] - h->c_rowptr[K]);
        for (int32_t c = 0; c < h->c_sptr[K + 1] - f; ++c)
          for (int32_t t = c; t < len; ++t) lrow[hp[f + c] + (t - c)] = r[t];
      }
      int32_t* dlrow = nullptr;
      rc = chol_dalloc(h, (void**)&dlrow, sizeof(int32_t) * (size_t)h->nnz_l);
      if (rc) return rc;
      CHOL_CUDA_TRY(cudaMemcpyAsync(dlrow, lrow.data(), sizeof(int32_t) * (size_t)h->nnz_l, cudaMemcpyHostToDevice, st));
      rc = chol_gather_mixed(h, dmap, dlrow, dlx, st);
      CHOL_CUDA_TRY(cudaStreamSynchronize(st));
      cudaFree(dlrow);
      D->bytes -= (int64_t)sizeof(int32_t) * h->nnz_l;
      if (rc) return rc;
    }
    CHOL_CUDA_TRY(cudaMemcpyAsync(lx, dlx, sizeof(double) * (size_t)h->nnz_l, cudaMemcpyDeviceToHost, st));
    CHOL_CUDA_TRY(cudaStreamSynchronize(st));
    cudaFree(dmap);
    cudaFree(dlx);
    D->bytes -= (int64_t)(sizeof(int64_t) + sizeof(double)) * h->nnz_l;
  }
  return CHOL_OK;
}
