// mixed.cu -- the mixed-precision form of the RL factorization (Sec. II-A) and
// the binary64 refinement around it.
//
// The matrix is scaled to D A D (D = diag(A)^{-1/2}, unit diagonal) while its
// values are scattered into binary32 panels. The panels are row-major, so both
// operands of every update GEMM are K-major, which the tensor cores want. The
// per-supernode steps are those of binary64 (Sec. II-A), grouped differently:
// - one panel launch per 256-column outer block does the POTRF of its 64-column
//   diagonal blocks (binary32; a block whose pivots fall below pivot_tau is
//   redone in binary64), the TRSM of the rows below and the updates inside the
//   block (k_mx_panel);
// - the columns right of the block get one update with K = 256, and the SYRK
//   forms the update matrix;
// - the pull-ordered relind scatter-add.
// In CHOL_PREC_FP32 the updates run on binary32 SIMT tiles; in TF32/BF16 they
// run on tcgen05 tensor-core tiles (tc_gemm.cuh). Accuracy is won back by
// iterative refinement with binary64 residuals (refine.cu).
#include <climits>
#include <cmath>
#include <cstring>

#include <cooperative_groups.h>
#include <cuda_bf16.h>

#include "device.h"
#include "mixed.h"
#include "assemble.cuh"
#include "potrf.cuh"

namespace cg = cooperative_groups;

namespace {

constexpr int kMxThreads = 256;

// d[i] = 1/sqrt(A_ii) of P A P^T; a non-positive diagonal keeps d = 1 (the
// factorization then reports the failing pivot itself).
__global__ void k_mx_scale(const double* __restrict__ vals, const int64_t* __restrict__ diagpos, int n,
                           double* __restrict__ d) {
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    const double a = vals[diagpos[i]];
    d[i] = a > 0.0 ? 1.0 / sqrt(a) : 1.0;
  }
}

__global__ void k_mx_scatter(const double* __restrict__ vals, const int64_t* __restrict__ amap,
                             const int32_t* __restrict__ aij, const double* __restrict__ d, int64_t nnz,
                             float* __restrict__ L) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x) {
#ifdef CHOL_BOUNDS_CHECK
    if (!CHOL_BC(amap[t] >= 0 && amap[t] < bc_lim.panel, kBcScatter)) continue;
#endif
    L[amap[t]] = (float)(vals[t] * d[aij[2 * t]] * d[aij[2 * t + 1]]);
  }
}

// Dense right-looking Cholesky of the first s columns of a len x s row-major
// block in shared memory (ld = s). Same failure convention as the binary64 path.
template <class T>
__device__ void dense_chol_rowmajor(T* P, int len, int s, int fcol, int* status, T spiv, int* nperturbed) {
  for (int k = 0; k < s; ++k) {
    __syncthreads();
    T dv = P[k * s + k];
    if (spiv > T(0) && !(dv >= spiv)) {      // static pivoting: max(|d|, tau)
      dv = fabs(dv) >= spiv ? T(fabs(dv)) : spiv;
      if (threadIdx.x == 0) atomicAdd(nperturbed, 1);
    }
    const bool bad = !(dv > T(0));
    const T dk = bad ? T(__longlong_as_double(0x7ff8000000000000LL)) : sqrt(dv);
    const T inv = T(1) / dk;
    for (int r = k + 1 + threadIdx.x; r < len; r += blockDim.x) P[r * s + k] *= inv;
    __syncthreads();
    if (threadIdx.x == 0) {
      P[k * s + k] = dk;
      if (bad) atomicMin(status, fcol + k + 1);
    }
    for (int r = k + 1 + threadIdx.x; r < len; r += blockDim.x) {
      const T lrk = P[r * s + k];
      const int jmax = r < s - 1 ? r : s - 1;
      for (int j = k + 1; j <= jmax; ++j) P[r * s + j] -= lrk * P[j * s + k];
    }
  }
  __syncthreads();
}

// One CTA per small supernode: binary32 panel in shared memory, U_J row-major
// lower (row u holds columns c <= u, leading dimension ldu = b rounded to 8).
__device__ __forceinline__ void mx_small_body(const SnodeDev& d, float* __restrict__ L, float* __restrict__ U,
                                              int* status, float spiv, int* counters, float* Pf) {
  const int len = d.len, s = d.s, b = len - s;
  float* G = L + d.loff;
  for (int q = threadIdx.x; q < len * s; q += blockDim.x) Pf[q] = G[(int64_t)(q / s) * d.ld + q % s];
  dense_chol_rowmajor<float>(Pf, len, s, d.f, status, spiv, counters + 1);
  for (int q = threadIdx.x; q < len * s; q += blockDim.x) {
    const int r = q / s, c = q % s;
    if (r >= c) G[(int64_t)r * d.ld + c] = Pf[q];
  }
  if (b <= 0) return;
  const int ldu = (b + 7) & ~7;
  float* Uj = U + d.uoff;
  const float* R = Pf + s * s;   // row u of L_RJ at R[u * s]
  const int64_t total = (int64_t)b * (b + 1) / 2;
  int u = 0;
  int64_t ustart = 0;            // flat index of (u, 0)
  for (int64_t q = threadIdx.x; q < total; q += blockDim.x) {
    while (q >= ustart + u + 1) { ustart += u + 1; ++u; }
    const int c = (int)(q - ustart);
    float acc = 0.f;
    for (int k = 0; k < s; ++k) acc = fmaf(R[u * s + k], R[c * s + k], acc);
    Uj[(int64_t)u * ldu + c] = acc;
  }
}

__global__ void __launch_bounds__(128)
k_mx_small(const SnodeDev* __restrict__ sn, const int32_t* __restrict__ list, float* __restrict__ L,
           float* __restrict__ U, int* status, float spiv, int* counters) {
  extern __shared__ float Pf[];
  mx_small_body(sn[list[blockIdx.x]], L, U, status, spiv, counters, Pf);
}

// ---------------------------------------------------------------------------
// Panel factorization of one outer column block [ob, ob + w), w <= kTcOuter,
// of every large supernode of a level (Sec. II-A: the POTRF, TRSM and update
// steps of the block's 64-column sub-blocks), binary32, in one launch.
//
// A CTA takes 64-row tiles of the block (PanelItem) from a work counter in
// list order and keeps its tile (64 x w) in shared memory through every
// sub-step. The tile holding the rows of sub-block d (a "diagonal tile"):
// for each j < d, the TRSM of its sub-block j against L_jj and the update of
// its sub-blocks j+1..d; then the POTRF of its diagonal block. A tile below
// the block does the TRSM and update for every sub-block. Tiles hand results
// to each other through global memory and one progress flag per diagonal
// tile: prog(d) = j + 1 once its TRSM of sub-block j is stored (j < d), and
// d + 1 once its L_dd is stored. A tile waits for prog(j) >= j + 1 (L_jj) and
// for prog(j') >= j + 1 (rows of sub-block j', columns of j) before using
// them. Every wait points to a diagonal tile with a smaller d, which comes
// earlier in the list, and items are taken in list order by running CTAs, so
// the smallest unfinished item can always proceed (no co-residency needed).
// Waits are bounded: one that runs out sets *err and carries on (the factor
// is then invalid and chol_factor reports CHOL_ETIMEOUT).
//
// Arithmetic per entry is that of the 64-column steps: the diagonal block in
// 8-column panels (binary64 redo below tau), the TRSM by substitution with
// the reciprocal pivots, the in-block updates as binary32 fused
// multiply-subtracts in column order.
// ---------------------------------------------------------------------------
constexpr int kPnW = kTcOuter;          // outer block width
static_assert(kPnW == 256, "the tile staging below indexes columns with 8 bits");
constexpr int kPnLd = kPnW + 4;         // shared tile row stride (floats)
constexpr int kPvLd = 68;              // row stride of the staged L_jj and Xo tiles: rows start on 16 bytes
static_assert(kPvLd >= kPwLd && kPvLd % 4 == 0 && kPnLd % 4 == 0, "16-byte row starts");
constexpr size_t kPnSmem = sizeof(float) * ((size_t)64 * kPnLd + 2 * 64 * kPvLd + 64);
constexpr long long kPanelMaxPolls = 1ll << 21;   // about a second with the back-off

__device__ __forceinline__ int pn_ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void pn_st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// One thread waits (bounded) until *flag >= need; then the CTA proceeds. Once
// any wait of the launch has run out (*err set), the others give up at once,
// so a launch with a broken hand-off ends after one wait limit.
__device__ __forceinline__ void pn_wait(const int* flag, int need, long long max_polls, int* err) {
  if (threadIdx.x == 0) {
    long long polls = 0;
    while (pn_ld_acquire(flag) < need) {
      if (++polls > max_polls) { atomicExch(err, 1); break; }
      if ((polls & 255) == 0 && *(volatile int*)err != 0) break;
      if (polls > 2048) __nanosleep(64);
    }
  }
  __syncthreads();
}

// Publish after the CTA's global stores: the barrier orders every thread's
// stores before thread 0's release store, and the release (gpu scope,
// cumulative) makes them visible to a consumer whose acquire load sees v.
__device__ __forceinline__ void pn_publish(int* flag, int v) {
  __syncthreads();
  if (threadIdx.x == 0) pn_st_release(flag, v);
}

__global__ void __launch_bounds__(256, 2)
k_mx_panel(const SnodeDev* __restrict__ sn, const PanelItem* __restrict__ items, int nitems, int ob,
           float* __restrict__ L, __nv_bfloat16* __restrict__ Lb, int* ticket, int* flags, int* err,
           long long max_polls, float tau, int static_pivot, int* status, int* counters) {
  extern __shared__ __align__(16) float pn_smem[];
  float* Own = pn_smem;                 // the tile: 64 rows x w columns (row stride kPnLd)
  float* Lk = Own + 64 * kPnLd;         // L_jj, column-major (ld kPvLd); POTRF staging (row-major, ld kPwLd)
  float* Xo = Lk + 64 * kPvLd;          // rows of sub-block j', columns of j (row-major, ld kPvLd)
  float* inv = Xo + 64 * kPvLd;         // reciprocal pivots of L_jj
  __shared__ int s_item, s_ok;
  __shared__ double colk_d[64];
  __shared__ double sinv_d;
  const int tid = threadIdx.x;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_item = atomicAdd(ticket, 1);
    __syncthreads();
    const int it = s_item;
    if (it >= nitems) break;
    const PanelItem item = items[it];
    const SnodeDev d = sn[item.J];
    const int w = min(kPnW, d.s - ob);
    const int nsub = (w + 63) >> 6;
    const int dd = item.d;                           // -1: below the block
    // valid rows: a diagonal tile holds exactly the rows of its diagonal block
    const int m = dd >= 0 ? min(64, w - dd * 64) : min(64, d.len - item.r0);
    const int jend = dd >= 0 ? dd : nsub;            // TRSM sub-steps of this tile
    int* fl = flags + item.fbase;
    float* G = L + d.loff + (int64_t)item.r0 * d.ld + ob;   // row 0, column 0 of the tile
    // stage the tile's nsub 64-column sub-blocks (the only columns any step
    // reads; zero past w and below the valid rows): 16-byte loads, all of a
    // thread's loads issued before its stores
#pragma unroll
    for (int s0 = 0; s0 < 4; s0 += 2) {   // two sub-blocks at a time: 8 loads in flight
      if (s0 >= nsub) break;
      float4 v[8];
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int sb = s0 + (q >> 2), e = tid + 256 * (q & 3), r = e >> 4, c = sb * 64 + (e & 15) * 4;
        float4 x = make_float4(0.f, 0.f, 0.f, 0.f);
        if (sb < nsub && r < m) {
          const float* g = G + (int64_t)r * d.ld + c;
          if (c + 4 <= w) {
            x = *reinterpret_cast<const float4*>(g);
          } else if (c < w) {
            x.x = g[0];
            if (c + 1 < w) x.y = g[1];
            if (c + 2 < w) x.z = g[2];
          }
        }
        v[q] = x;
      }
#pragma unroll
      for (int q = 0; q < 8; ++q) {
        const int sb = s0 + (q >> 2), e = tid + 256 * (q & 3), r = e >> 4, c = sb * 64 + (e & 15) * 4;
        if (sb < nsub) *reinterpret_cast<float4*>(Own + r * kPnLd + c) = v[q];
      }
    }
    __syncthreads();   // the tile is staged (a d = 0 tile reads it right away)
    for (int j = 0; j < jend; ++j) {
      const int c0 = j * 64, kb = min(64, w - c0);
      // L_jj (stored by the diagonal tile j) and its reciprocal pivots
      pn_wait(fl + j, j + 1, max_polls, err);
      {
        const float* Gd = L + d.loff + (int64_t)(ob + c0) * d.ld + ob + c0;
        float v[16];
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int q = tid + 256 * i, r = q >> 6, c = q & 63;
          v[i] = (r < kb && c <= r) ? __ldcg(Gd + (int64_t)r * d.ld + c) : 0.f;
        }
#pragma unroll
        for (int i = 0; i < 16; ++i) {
          const int q = tid + 256 * i;
          Lk[(q >> 6) + (q & 63) * kPvLd] = v[i];
        }
      }
      __syncthreads();
      // reciprocal pivots; zero past kb, where the tile's columns and L_jj are
      // zero too, so the substitution below needs no bounds on kb
      if (tid < 64) inv[tid] = tid < kb ? 1.0f / Lk[tid + tid * kPvLd] : 0.f;
      __syncthreads();
      // TRSM of the tile's sub-block j: two threads per row (threads 0-127),
      // thread h of row r holding columns [32 h, 32 h + 32) in registers. The
      // low half substitutes its columns and passes them through shared memory
      // (Xo is free until the updates); the high half then subtracts their
      // products, in column order, and substitutes its own. Per entry the same
      // fused multiply-subtracts in the same order as a column-by-column
      // substitution with the reciprocal pivots.
      if (tid < 128) {
        const int r = tid & 63, h = tid >> 6;
        float* Xr = Own + r * kPnLd + c0 + 32 * h;
        float* xs = Xo + r * 33;
        float x[32];
#pragma unroll
        for (int k4 = 0; k4 < 8; ++k4) {
          const float4 a = *reinterpret_cast<const float4*>(Xr + 4 * k4);
          x[4 * k4] = a.x; x[4 * k4 + 1] = a.y; x[4 * k4 + 2] = a.z; x[4 * k4 + 3] = a.w;
        }
        // substitution of columns [32 h, 32 h + 32) of this row
        auto substitute = [&](int cb) {
#pragma unroll
          for (int jl = 0; jl < 32; ++jl) {
            const int jj = cb + jl;
            x[jl] = x[jl] * inv[jj];
            const float xj = x[jl];
#pragma unroll
            for (int k4 = (jl + 1) >> 2; k4 < 8; ++k4) {
              const float4 l4 = *reinterpret_cast<const float4*>(Lk + jj * kPvLd + cb + 4 * k4);
              const float lv[4] = {l4.x, l4.y, l4.z, l4.w};
#pragma unroll
              for (int u = 0; u < 4; ++u)
                if (4 * k4 + u > jl) x[4 * k4 + u] = fmaf(-xj, lv[u], x[4 * k4 + u]);
            }
          }
        };
        if (h == 0) {
          substitute(0);
#pragma unroll
          for (int jl = 0; jl < 32; ++jl) xs[jl] = x[jl];
        }
        asm volatile("bar.sync 1, 128;" ::: "memory");
        if (h == 1) {
#pragma unroll 4
          for (int jj = 0; jj < 32; ++jj) {
            const float xj = xs[jj];
#pragma unroll
            for (int k4 = 0; k4 < 8; ++k4) {
              const float4 l4 = *reinterpret_cast<const float4*>(Lk + jj * kPvLd + 32 + 4 * k4);
              x[4 * k4] = fmaf(-xj, l4.x, x[4 * k4]);
              x[4 * k4 + 1] = fmaf(-xj, l4.y, x[4 * k4 + 1]);
              x[4 * k4 + 2] = fmaf(-xj, l4.z, x[4 * k4 + 2]);
              x[4 * k4 + 3] = fmaf(-xj, l4.w, x[4 * k4 + 3]);
            }
          }
          substitute(32);
        }
#pragma unroll
        for (int k4 = 0; k4 < 8; ++k4)
          *reinterpret_cast<float4*>(Xr + 4 * k4) =
              make_float4(x[4 * k4], x[4 * k4 + 1], x[4 * k4 + 2], x[4 * k4 + 3]);
      }
      __syncthreads();
      // the solved sub-block to the panel (and its bf16 copy): 16-byte stores,
      // a warp writing two rows of 256 contiguous bytes
      {
        __nv_bfloat16* Bt = Lb ? Lb + d.loff + (int64_t)item.r0 * d.ld + ob + c0 : nullptr;
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const int e = tid + 256 * i, r = e >> 4, c = (e & 15) * 4;
          if (r < m && c < kb) {
            const float4 v = *reinterpret_cast<const float4*>(Own + r * kPnLd + c0 + c);
            float* Gx = G + (int64_t)r * d.ld + c0 + c;
            __nv_bfloat16* Bx = Bt ? Bt + (int64_t)r * d.ld + c : nullptr;
            if (c + 4 <= kb) {
              *reinterpret_cast<float4*>(Gx) = v;
              if (Bx) {
                const __nv_bfloat162 lo = __floats2bfloat162_rn(v.x, v.y), hi = __floats2bfloat162_rn(v.z, v.w);
                uint2 u;
                u.x = *reinterpret_cast<const uint32_t*>(&lo);
                u.y = *reinterpret_cast<const uint32_t*>(&hi);
                *reinterpret_cast<uint2*>(Bx) = u;
              }
            } else {
              const float vv[4] = {v.x, v.y, v.z, v.w};
              for (int u = 0; u < 4 && c + u < kb; ++u) {
                Gx[u] = vv[u];
                if (Bx) Bx[u] = __float2bfloat16_rn(vv[u]);
              }
            }
          }
        }
      }
      if (dd >= 0) pn_publish(fl + dd, j + 1);   // this tile's rows of sub-block j are stored
      __syncthreads();
      // updates of the later sub-blocks j' this tile holds: below the block
      // every j' < nsub; a diagonal tile up to its own diagonal block
      const int jlast = dd >= 0 ? dd : nsub - 1;
      for (int jp = j + 1; jp <= jlast; ++jp) {
        const int cp = jp * 64, kbp = min(64, w - cp);
        const float* Y;   // rows of sub-block j' (columns of j), row stride yld
        int yld;
        if (jp == dd) {
          Y = Own + c0;
          yld = kPnLd;
        } else {
          pn_wait(fl + jp, j + 1, max_polls, err);
          const float* Gy = L + d.loff + (int64_t)(ob + cp) * d.ld + ob + c0;
          float v[16];
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int q = tid + 256 * i, r = q >> 6, c = q & 63;
            v[i] = (r < kbp && c < kb) ? __ldcg(Gy + (int64_t)r * d.ld + c) : 0.f;
          }
#pragma unroll
          for (int i = 0; i < 16; ++i) {
            const int q = tid + 256 * i;
            Xo[(q >> 6) * kPvLd + (q & 63)] = v[i];
          }
          __syncthreads();
          Y = Xo;
          yld = kPvLd;
        }
        // Own[:, j'] -= Own[:, j] Y^T: thread (tx, ty) owns rows ty + 16 i,
        // columns tx + 16 l; K in column order
        const int tx = tid & 15, ty = tid >> 4;
        float acc[4][4] = {};
        const int k4 = kb & ~3;
        for (int k = 0; k < k4; k += 4) {   // four k at a time from 16-byte loads, k in order
          float4 a[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = *reinterpret_cast<const float4*>(Own + (ty + 16 * i) * kPnLd + c0 + k);
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            const float4 bv = *reinterpret_cast<const float4*>(Y + (tx + 16 * l) * yld + k);
#pragma unroll
            for (int i = 0; i < 4; ++i) {
              acc[i][l] = fmaf(a[i].x, bv.x, acc[i][l]);
              acc[i][l] = fmaf(a[i].y, bv.y, acc[i][l]);
              acc[i][l] = fmaf(a[i].z, bv.z, acc[i][l]);
              acc[i][l] = fmaf(a[i].w, bv.w, acc[i][l]);
            }
          }
        }
        for (int k = k4; k < kb; ++k) {
          float a[4], bv[4];
#pragma unroll
          for (int i = 0; i < 4; ++i) a[i] = Own[(ty + 16 * i) * kPnLd + c0 + k];
#pragma unroll
          for (int l = 0; l < 4; ++l) bv[l] = Y[(tx + 16 * l) * yld + k];
#pragma unroll
          for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int l = 0; l < 4; ++l) acc[i][l] = fmaf(a[i], bv[l], acc[i][l]);
        }
        __syncthreads();   // every read of Own[:, j] and Y is done
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
          for (int l = 0; l < 4; ++l) {
            const int c = tx + 16 * l;
            if (c < kbp) Own[(ty + 16 * i) * kPnLd + cp + c] -= acc[i][l];
          }
        __syncthreads();
      }
    }
    if (dd >= 0) {
      // POTRF of the diagonal block dd (rows and columns [cd, cd + kbd) of the tile)
      const int cd = dd * 64, kbd = min(64, w - cd);
      for (int q = tid; q < 64 * 64; q += 256) {
        const int r = q >> 6, c = q & 63;
        Lk[r * kPwLd + c] = (r < kbd && c <= r) ? Own[r * kPnLd + cd + c] : 0.f;
      }
      const bool ok = potrf_panels_smem<float>(kbd, tau, Lk, &s_ok, status, false, d.f + ob + cd);
      float* Gd = G + cd;   // the tile's rows are those of the diagonal block
      if (ok) {
        for (int q = tid; q < 64 * 64; q += 256) {
          const int r = q >> 6, c = q & 63;
          if (r < kbd && c <= r) Gd[(int64_t)r * d.ld + c] = Lk[r * kPwLd + c];
        }
      } else {
        // binary64 redo from the updated (unfactored) block
        if (tid == 0) atomicAdd(counters, 1);
        for (int q = tid; q < 64 * 64; q += 256) {
          const int r = q >> 6, c = q & 63;
          if (r < kbd && c <= r) Gd[(int64_t)r * d.ld + c] = Own[r * kPnLd + cd + c];
        }
        __syncthreads();
        potrf_block<double, true, float>(Gd, d.ld, kbd, static_pivot ? (double)tau : 0.0, counters + 1, nullptr,
                                         status, true, d.f + ob + cd, colk_d, &sinv_d, -INFINITY);
      }
      pn_publish(fl + dd, dd + 1);
    }
  }
}

// 64 x 64 binary32 SIMT tile of C (op)= A B^T with row-major A, B (K
// contiguous) and row-major C; entries with row + rdiag >= col only.
template <bool SUB>
__device__ __forceinline__ void gemm_nt_tile_f32(const float* __restrict__ A, int64_t lda,
                                                 const float* __restrict__ B, int64_t ldb, int K,
                                                 float* __restrict__ C, int64_t ldc, int M, int N,
                                                 int rdiag) {
  constexpr int KC = 16;
  __shared__ float As[KC][kTile + 4];
  __shared__ float Bs[KC][kTile + 4];
  const int tid = threadIdx.x;
  const int tx = tid & 15, ty = tid >> 4;
  float acc[4][4] = {};
  for (int k = 0; k < K; k += KC) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + 256 * q;
      const int kk = idx & 15, r = idx >> 4;
      const bool kin = k + kk < K;
      As[kk][r] = (kin && r < M) ? A[r * lda + k + kk] : 0.f;
      Bs[kk][r] = (kin && r < N) ? B[r * ldb + k + kk] : 0.f;
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      float a[4], bb[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) bb[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fmaf(a[i], bb[j], acc[i][j]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = ty + 16 * i, c = tx + 16 * j;
      if (r < M && c < N && r + rdiag >= c) {
        float* p = C + r * ldc + c;
        *p = SUB ? (*p - acc[i][j]) : acc[i][j];
      }
    }
}

__global__ void __launch_bounds__(256)
k_mx_gemm_simt(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, int nb,
               float* __restrict__ L) {
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int kb = min(nb, d.s - t.k0);
  float* P = L + d.loff;
  gemm_nt_tile_f32<true>(P + (int64_t)t.r0 * d.ld + t.k0, d.ld, P + (int64_t)t.c0 * d.ld + t.k0, d.ld, kb,
                         P + (int64_t)t.r0 * d.ld + t.c0, d.ld, min(kTile, d.len - t.r0),
                         min(kTile, d.s - t.c0), t.r0 - t.c0);
}

__global__ void __launch_bounds__(256)
k_mx_syrk_simt(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks,
               const float* __restrict__ L, float* __restrict__ U) {
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int b = d.len - d.s;
  const int ldu = (b + 7) & ~7;
  const float* R = L + d.loff + (int64_t)d.s * d.ld;
  gemm_nt_tile_f32<false>(R + (int64_t)t.r0 * d.ld, d.ld, R + (int64_t)t.c0 * d.ld, d.ld, d.s,
                          U + d.uoff + (int64_t)t.r0 * ldu + t.c0, ldu, min(kTile, b - t.r0),
                          min(kTile, b - t.c0), t.r0 - t.c0);
}

// Binary32 assembly of one task (row-major U_J and panels). Row positions as in
// the binary64 kernel; the segment's columns are spread over groups of 4, 8, 16
// or 32 lanes (the smallest that covers them, twice for 33..64 columns), so a
// warp covers 32 / group rows per pass and issues kMxAsmUnroll passes' loads
// before their stores.
constexpr int kMxAsmUnroll = 4;

__device__ __forceinline__ void mx_assemble_body(const AsmTask& t, const AsmSeg* __restrict__ segs,
                                                 const SnodeDev* __restrict__ sn, const int32_t* __restrict__ rows,
                                                 const float* __restrict__ U, float* __restrict__ L, int32_t* ssm) {
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
  int32_t* sK = ssm;
  int32_t* pos = ssm + kAsmPos;
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
    const int ldu = (b + 7) & ~7;
    const int32_t* rj = rows + dj.roff + dj.s;
    const int nu = sg.ub - sg.ua, w = sg.cb - sg.ca;
#ifdef CHOL_BOUNDS_CHECK
    if (!CHOL_BC(sg.ua >= 0 && sg.ua <= sg.ub && sg.ub <= b && sg.ca >= 0 && sg.ca <= sg.cb && sg.cb <= b &&
                     nu <= kAsmPos && w <= kAsmCols,
                 kBcSegRange))
      continue;
#endif
    __syncthreads();
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
    const float* Uj = U + dj.uoff;
    float* Lk = L + dk.loff;
    const int gs = w <= 4 ? 4 : w <= 8 ? 8 : w <= 16 ? 16 : 32;   // lanes per row
    const int gsh = gs == 4 ? 2 : gs == 8 ? 3 : gs == 16 ? 4 : 5;
    const int rpw = 32 >> gsh;                                   // rows per warp pass
    const int nc = w > 32 ? 2 : 1;                               // column chunks per row
    const int sub = lane >> gsh, cl = lane & (gs - 1);
    const int items = nu * nc;                                   // (row, column chunk) pairs
    for (int i0 = warp * rpw; i0 < items; i0 += nwarps * rpw * kMxAsmUnroll) {
      float v[kMxAsmUnroll], l[kMxAsmUnroll];
      int64_t off[kMxAsmUnroll];
#pragma unroll
      for (int q = 0; q < kMxAsmUnroll; ++q) {
        const int i = i0 + q * nwarps * rpw + sub;
        off[q] = -1;
        if (i < items) {
          const int ui = nc == 2 ? (i >> 1) : i;
          const int cc = (nc == 2 ? (i & 1) * 32 : 0) + cl;
          const int u = sg.ua + ui, c = sg.ca + cc;
          if (cc < w && c <= u) {
#ifdef CHOL_BOUNDS_CHECK
            if (tcol[cc] < 0 || pos[ui] < 0) continue;
#endif
            off[q] = (int64_t)pos[ui] * dk.ld + tcol[cc];
            v[q] = Uj[(int64_t)u * ldu + c];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kMxAsmUnroll; ++q)
        if (off[q] >= 0) l[q] = Lk[off[q]];
#pragma unroll
      for (int q = 0; q < kMxAsmUnroll; ++q)
        if (off[q] >= 0) Lk[off[q]] = l[q] - v[q];
    }
  }
}

__global__ void __launch_bounds__(kMxThreads)
k_mx_assemble(const AsmTask* __restrict__ tasks, const AsmSeg* __restrict__ segs,
              const SnodeDev* __restrict__ sn, const int32_t* __restrict__ rows,
              const float* __restrict__ U, float* __restrict__ L) {
  extern __shared__ int32_t ssm[];
  mx_assemble_body(tasks[blockIdx.x], segs, sn, rows, U, L, ssm);
}

// Persistent form of the one-CTA levels (binary32 panels), see the binary64
// k_persist_factor.
template <int NT>
__global__ void __launch_bounds__(NT)
k_persist_factor_mx(const SnodeDev* __restrict__ sn, const int32_t* __restrict__ small_list,
                    const AsmTask* __restrict__ tasks, const AsmSeg* __restrict__ segs,
                    const int32_t* __restrict__ rows, const PersistLevel* __restrict__ lv, int nlevels,
                    float* __restrict__ L, float* __restrict__ U, int* status, float spiv, int* counters) {
  extern __shared__ float psmf[];
  cg::grid_group grid = cg::this_grid();
  for (int l = 0; l < nlevels; ++l) {
    const PersistLevel p = lv[l];
    for (int i = blockIdx.x; i < p.small_n; i += gridDim.x) {
      __syncthreads();
      mx_small_body(sn[small_list[p.small_b + i]], L, U, status, spiv, counters, psmf);
    }
    grid.sync();
    for (int i = blockIdx.x; i < p.asm_n; i += gridDim.x) {
      __syncthreads();
      mx_assemble_body(tasks[p.asm_b + i], segs, sn, rows, U, L, reinterpret_cast<int32_t*>(psmf));
    }
    {
      __syncthreads();
      int32_t* wsm = reinterpret_cast<int32_t*>(psmf) + (threadIdx.x >> 5) * 2 * kAsmWarpPos;
      const int nw = NT / 32;
      for (int i = blockIdx.x * nw + (threadIdx.x >> 5); i < p.asmw_n; i += gridDim.x * nw)
        assemble_warp_task<float, true>(tasks[p.asm_b + p.asm_n + i], segs, sn, rows, U, L, wsm,
                                        wsm + kAsmWarpPos);
    }
    grid.sync();
  }
}

// log det: per-supernode partial sums of log(L~_jj) - log(d_j) (A = D^-1 A~ D^-1).
__global__ void k_mx_logdet_part(const SnodeDev* __restrict__ sn, const float* __restrict__ L,
                                 const double* __restrict__ dsc, double* __restrict__ part) {
  __shared__ double red[128];
  const SnodeDev d = sn[blockIdx.x];
  double acc = 0.0;
  for (int c = threadIdx.x; c < d.s; c += blockDim.x)
    acc += log((double)L[d.loff + (int64_t)c * d.ld + c]) - log(dsc[d.f + c]);
  red[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) part[blockIdx.x] = red[0];
}

__global__ void k_mx_logdet_reduce(const double* __restrict__ part, int ns, double* out) {
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

// L = D^{-1} L~ in compressed sparse column order: out[t] = L~[map[t]] / d[row(t)].
__global__ void k_mx_gather(const float* __restrict__ L, const int64_t* __restrict__ map,
                            const int32_t* __restrict__ lrow, const double* __restrict__ dsc, int64_t nnz,
                            double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = (double)L[map[t]] / dsc[lrow[t]];
}

__global__ void k_mx_gather_vals(const double* __restrict__ vals, const int64_t* __restrict__ src, int64_t m,
                                 double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = vals[src[t]];
}

inline unsigned grid1d(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g > 0 ? g : 1);
}

template <class T>
int upload_vec(chol_handle* h, T** dst, const std::vector<T>& v) {
  if (v.empty()) { *dst = nullptr; return CHOL_OK; }
  int rc = chol_dalloc(h, (void**)dst, v.size() * sizeof(T));
  if (rc) return rc;
  CHOL_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return CHOL_OK;
}

}  // namespace

// Device buffers of the mixed modes (allocated once, by the first factor).
int chol_mixed_ensure(chol_handle* h) {
  DeviceState* D = h->dev;
  if (D->mx_ready) return CHOL_OK;
  int rc;
  std::vector<int64_t> diagpos(h->n);
  // diagonal of P A P^T at permuted i is A's diagonal of column perm[i]: the
  // first entry of that column (validated by chol_analyze)
  for (int32_t i = 0; i < h->n; ++i) diagpos[i] = h->diagpos_orig[h->perm[i]];
  if ((rc = upload_vec(h, &D->mx_diagpos, diagpos))) return rc;
  if ((rc = upload_vec(h, &D->mx_aij, h->aij))) return rc;
  if ((rc = chol_dalloc(h, (void**)&D->mx_d, sizeof(double) * (size_t)std::max(h->n, 1)))) return rc;
  if ((rc = chol_dalloc(h, (void**)&D->mx_fallbacks, 2 * sizeof(int32_t)))) return rc;
  if ((rc = chol_tc_prepare(h))) return rc;
  if (!D->tc_err) {
    if ((rc = chol_dalloc(h, (void**)&D->tc_err, sizeof(int32_t)))) return rc;
    CHOL_CUDA_TRY(cudaMemset(D->tc_err, 0, sizeof(int32_t)));
  }
  if ((rc = upload_vec(h, &D->panel, h->panel_items))) return rc;
  // per diagonal block of the solve: its inverse and the two last-dependency products
  if ((rc = chol_dalloc(h, &D->dinv, sizeof(float) * 3 * 64 * 64 * (size_t)std::max(h->tri_nflags, 1)))) return rc;
  if ((rc = chol_dalloc(h, (void**)&D->pflags, sizeof(int32_t) * (size_t)std::max(h->panel_ntickets + h->panel_nflags, 1))))
    return rc;
  if (cudaFuncSetAttribute(k_mx_panel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kPnSmem) != cudaSuccess)
    return CHOL_ECUDA;
  {
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_mx_panel, 256, kPnSmem) != cudaSuccess || per_sm < 1)
      return CHOL_ECUDA;
    D->panel_ctas = per_sm * D->sms;
  }
  if (cudaFuncSetAttribute(k_mx_assemble, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024) != cudaSuccess)
    return CHOL_ECUDA;
  if (cudaFuncSetAttribute(k_mx_small, cudaFuncAttributeMaxDynamicSharedMemorySize, 24576 * 4) != cudaSuccess)
    return CHOL_ECUDA;
  D->mx_ready = true;
  return CHOL_OK;
}

int chol_enqueue_factor_mixed(chol_handle* h, const double* values, cudaStream_t st) {
  int rc = CHOL_OK;
  DeviceState* D = h->dev;
  float* L = (float*)D->L;
  float* U = (float*)D->U;
  const int nb = h->opt.block_cols;
  const bool tc = h->opt.precision == CHOL_PREC_TF32 || h->opt.precision == CHOL_PREC_BF16;
  chol_status_init(D->status, st);
  h->tc_shallow = h->tc_deep = h->panel_launches = 0;
  CHOL_CUDA_TRY(cudaMemsetAsync(D->mx_fallbacks, 0, 2 * sizeof(int32_t), st));
  const float spiv = h->opt.static_pivot ? (float)h->opt.pivot_tau : 0.f;
  CHOL_CUDA_TRY(cudaMemsetAsync(L, 0, sizeof(float) * (size_t)h->panel_doubles, st));
  if (h->n > 0) {
    KScope ks(h, CHOL_K_SCATTER, st, 0.0, 16.0 * h->n);
    k_mx_scale<<<grid1d(h->n, 256), 256, 0, st>>>(values, D->mx_diagpos, h->n, D->mx_d);
  }
  if (h->nnz_a > 0) {
    KScope ks(h, CHOL_K_SCATTER, st, 0.0, 28.0 * (double)h->nnz_a);
    k_mx_scatter<<<grid1d(h->nnz_a, 256), 256, 0, st>>>(values, D->amap, D->mx_aij, D->mx_d, h->nnz_a, L);
    const int64_t m = h->csr_ptr[h->n];
    k_mx_gather_vals<<<grid1d(m, 256), 256, 0, st>>>(values, D->csr_src, m, D->csr_val);
  }
  if (h->opt.persistent) {
    if (h->n_large > 0) return CHOL_ENOTSUP;
    double fl = 0.0, by = 0.0;
    for (const LevelPlan& P : h->levels) { fl += P.small_flops; by += P.small_bytes / 2; }
    KScope ks(h, CHOL_K_SMALL, st, fl, by);
    return chol_launch_persistent(h, (void*)L, (void*)U, st);
  }
  // levels with blocked supernodes: critical path on the high-priority stream
  const cudaStream_t caller = st;
  if (h->n_large > 0) {
    CHOL_CUDA_TRY(cudaEventRecord(D->lev[2], caller));
    CHOL_CUDA_TRY(cudaStreamWaitEvent(D->hstream, D->lev[2], 0));
    st = D->hstream;
  }
  // outer-update tiles of a step (K = kk: one or two outer blocks, from each task's k0)
  auto gemm = [&](const TileTask* tasks, int n, int kk, double flops, cudaStream_t s2) -> int {
    if (n <= 0) return CHOL_OK;
    KScope ks(h, CHOL_K_GEMM, s2, flops, 0.0);
    if (tc) return chol_tc_gemm(h, tasks, n, kk, 0, s2);
    k_mx_gemm_simt<<<n, 256, 0, s2>>>(D->sn, tasks, kk, L);
    return CHOL_OK;
  };
  // progress flags and work counters of this factorization's panel launches
  if (h->panel_ntickets > 0)
    CHOL_CUDA_TRY(cudaMemsetAsync(D->pflags, 0, sizeof(int32_t) * (size_t)(h->panel_ntickets + h->panel_nflags), st));
  for (const LevelPlan& P : h->levels) {
    NvtxRange nvtx_level("level", (long long)(&P - h->levels.data()));
    if (P.small_n > 0) {
      KScope ks(h, CHOL_K_SMALL, st, P.small_flops, P.small_bytes / 2);
      k_mx_small<<<P.small_n, 128, sizeof(float) * P.small_max_panel, st>>>(D->sn, D->small_list + P.small_b, L, U,
                                                                              D->status, spiv, D->mx_fallbacks);
    }
    // one launch per outer column block: the panel kernel (its POTRF, TRSM and
    // in-block update steps), then the outer update of a pair of blocks (the
    // next block's columns after the first block, everything right of the pair
    // after the second); the columns the next panels need on the critical
    // stream, the rest on the side stream beside the next panels (lookahead)
    bool rest_pending = false;
    for (size_t k = 0; k < P.steps.size(); ++k) {
      const StepRange& s = P.steps[k];
      if (s.panel_n > 0) {
        KScope ks(h, CHOL_K_PANEL, st, s.panel_flops, 0.0);
        ++h->panel_launches;
        const int grid = std::min(s.panel_n, D->panel_ctas);
        k_mx_panel<<<grid, 256, kPnSmem, st>>>(
            D->sn, D->panel + s.panel_b, s.panel_n, s.ok0, L,
            (__nv_bfloat16*)(h->opt.precision == CHOL_PREC_BF16 ? D->Lbf : nullptr), D->pflags + s.panel_ticket,
            D->pflags + h->panel_ntickets, D->tc_err, h->opt.wait_polls > 0 ? (long long)h->opt.wait_polls : kPanelMaxPolls,
            (float)h->opt.pivot_tau, h->opt.static_pivot, D->status, D->mx_fallbacks);
      }
      const int orest = s.ogemm_n - s.ogemm_next;
      if (orest > 0) {
        CHOL_CUDA_TRY(cudaEventRecord(D->lev[0], st));   // the block's panel is final
        CHOL_CUDA_TRY(cudaStreamWaitEvent(D->lstream, D->lev[0], 0));
      }
      // the side stream's update of a pair reaches the columns of the next
      // pair's second block onwards: wait for it before updating those
      if (rest_pending && s.join_rest) {
        CHOL_CUDA_TRY(cudaStreamWaitEvent(st, D->lev[1], 0));
        rest_pending = false;
      }
      const double fo = s.ogemm_n > 0 ? (double)s.ogemm_next / s.ogemm_n : 0.0;
      if ((rc = gemm(D->gemm + s.ogemm_b, s.ogemm_next, s.okb, s.ogemm_flops * fo, st))) return rc;
      if (orest > 0) {
        if ((rc = gemm(D->gemm + s.ogemm_b + s.ogemm_next, orest, s.okb, s.ogemm_flops * (1.0 - fo), D->lstream)))
          return rc;
        CHOL_CUDA_TRY(cudaEventRecord(D->lev[1], D->lstream));
        rest_pending = true;
      }
    }
    if (rest_pending) CHOL_CUDA_TRY(cudaStreamWaitEvent(st, D->lev[1], 0));   // join before SYRK
    if (P.syrk_n > 0) {
      KScope ks(h, CHOL_K_SYRK, st, P.syrk_flops, 0.0);
      if (tc) {
        if ((rc = chol_tc_syrk(h, D->syrk + P.syrk_b, P.syrk_n, st))) return rc;
      } else {
        k_mx_syrk_simt<<<P.syrk_n, 256, 0, st>>>(D->sn, D->syrk + P.syrk_b, L, U);
      }
    }
    if (P.asm_n + P.asmw_n > 0) {
      KScope ks(h, CHOL_K_ASSEMBLE, st, P.asm_entries, 12.0 * P.asm_entries);
      ks.launches((P.asm_n > 0) + (P.asmw_n > 0));
      if (P.asm_n > 0)
        k_mx_assemble<<<P.asm_n, kMxThreads, sizeof(int32_t) * 2 * kAsmPos, st>>>(
            D->asm_tasks + P.asm_b, D->asm_segs, D->sn, D->rows, U, L);
      if (P.asmw_n > 0)
        k_assemble_warp<float, true><<<(P.asmw_n + 7) / 8, 256, 0, st>>>(
            D->asm_tasks + P.asm_b + P.asm_n, P.asmw_n, D->asm_segs, D->sn, D->rows, U, L);
    }
  }
  if (st != caller) {
    CHOL_CUDA_TRY(cudaEventRecord(D->lev[2], st));
    CHOL_CUDA_TRY(cudaStreamWaitEvent(caller, D->lev[2], 0));
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

const void* chol_persistent_kernel_mixed(int threads) {
  return threads == 256 ? (const void*)k_persist_factor_mx<256> : (const void*)k_persist_factor_mx<128>;
}

int chol_logdet_parts_mixed(chol_handle* h, cudaStream_t st) {
  DeviceState* D = h->dev;
  k_mx_logdet_part<<<h->ns, 128, 0, st>>>(D->sn, (const float*)D->L, D->mx_d, D->part);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

int chol_logdet_mixed(chol_handle* h, double* out, cudaStream_t st) {
  DeviceState* D = h->dev;
  if (h->ns > 0) {
    KScope ks(h, CHOL_K_LOGDET, st, (double)h->n, 4.0 * h->n);
    k_mx_logdet_part<<<h->ns, 128, 0, st>>>(D->sn, (const float*)D->L, D->mx_d, D->part);
    k_mx_logdet_reduce<<<1, 1024, 0, st>>>(D->part, h->ns, D->scalar_dev);
  } else {
    CHOL_CUDA_TRY(cudaMemsetAsync(D->scalar_dev, 0, sizeof(double), st));
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  CHOL_CUDA_TRY(cudaMemcpyAsync(D->scalar_host, D->scalar_dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  CHOL_CUDA_TRY(cudaStreamSynchronize(st));
  *out = *D->scalar_host;
  return CHOL_OK;
}

// Gather L = D^{-1} L~ (binary64) in canonical CSC order (map built by the caller).
int chol_gather_mixed(chol_handle* h, const int64_t* dmap, const int32_t* dlrow, double* dlx, cudaStream_t st) {
  DeviceState* D = h->dev;
  k_mx_gather<<<grid1d(h->nnz_l, 256), 256, 0, st>>>((const float*)D->L, dmap, dlrow, D->mx_d, h->nnz_l, dlx);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

// CHOL_BOUNDS_CHECK build: the limits and the error word of this translation
// unit's checked kernels (no-ops in the normal build).
int chol_bc_begin_mixed(const chol_handle* h) {
#ifdef CHOL_BOUNDS_CHECK
  return bc_begin(h);
#else
  (void)h;
  return 0;
#endif
}

int chol_bc_read_mixed() {
#ifdef CHOL_BOUNDS_CHECK
  return bc_read();
#else
  return 0;
#endif
}
