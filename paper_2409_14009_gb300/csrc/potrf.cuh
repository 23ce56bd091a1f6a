// potrf.cuh -- Cholesky of one kb x kb (kb <= 64) diagonal block in one CTA of
// 256 threads (the diagonal POTRF of a column step of the blocked path, Sec.
// II-A). Two routines with the same per-entry arithmetic:
//
// potrf_panels (the diagonal POTRF of both precisions) stages the block in
// shared memory and works in 8-column panels: one warp factors a panel in
// registers, all warps apply its rank-8 update to the trailing triangle.
//
// potrf_block (the binary64 redo of a rejected binary32 block, with static
// pivoting) keeps the lower triangle in registers, enumerated column by
// column, e = off(c) + (r - c) with off(c) = c kb - c (c - 1) / 2; entry e lives
// in register slot e / 256 of thread e % 256. Right-looking, one column per
// step: the owner of (k, k) takes the square root, the owners of column k scale
// it into shared memory, and the owners of every later column subtract the
// rank-1 term. The entries still being updated at step k are exactly those
// with e >= off(k + 1), a suffix of the enumeration, so whole warps drop out as
// the factorization advances.
#pragma once
#include <cstdint>

constexpr int kPkThreads = 256;
constexpr int kPkSlots = 9;   // ceil(64 * 65 / 2 / 256)

__device__ __forceinline__ int pk_off(int c, int kb) { return c * kb - (c * (c - 1)) / 2; }

// (r, c) of entry e of the packed lower triangle of a kb x kb block.
__device__ __forceinline__ void pk_coord(int e, int kb, int& r, int& c) {
  const float fk = (float)kb + 0.5f;
  int cc = (int)(fk - sqrtf(fmaxf(fk * fk - 2.0f * (float)e, 0.0f)));
  cc = max(0, min(cc, kb - 1));
  while (cc > 0 && pk_off(cc, kb) > e) --cc;
  while (cc + 1 < kb && pk_off(cc + 1, kb) <= e) ++cc;
  c = cc;
  r = cc + (e - pk_off(cc, kb));
}

// Square root of a pivot and its reciprocal. binary32 (the low-precision
// factor of the mixed modes, refined in binary64 afterwards): the hardware
// reciprocal square root rsqrtf (a few ulps) and sqrt(d) = d rsqrt(d), which
// keeps the pivot chain short. binary64: on this GPU every FP64 instruction of the serial pivot chain holds
// the narrow FP64 pipe for many cycles, and sqrt plus a division expand to
// long dependent sequences; instead the reciprocal square root starts from the
// binary32 estimate and takes two Newton-Raphson steps y <- y (3 - d y^2) / 2
// (each roughly doubles the correct bits: ~23 -> ~46 -> full precision, within
// a few ulps), then sqrt(d) = d y. Pivots outside the binary32 normal range
// take sqrt and a division.
__device__ __forceinline__ void pivot_root(float d, bool bad, float& root, float& rroot) {
  rroot = bad ? __int_as_float(0x7fc00000) : rsqrtf(d);
  root = d * rroot;
}
__device__ __forceinline__ void pivot_root(double d, bool bad, double& root, double& rroot) {
  if (bad) {
    root = __longlong_as_double(0x7ff8000000000000LL);
    rroot = root;
  } else if (d > 1e-30 && d < 1e30) {
    double y = (double)rsqrtf((float)d);
    y = y * fma(-0.5 * d, y * y, 1.5);
    y = y * fma(-0.5 * d, y * y, 1.5);
    root = d * y;
    rroot = y;
  } else {
    root = sqrt(d);
    rroot = 1.0 / root;
  }
}

// Factor the block at G (row-major with leading dimension ld if RM, else
// column-major) in arithmetic T, reading and writing the storage type GT.
//   spiv       > 0: static pivoting, a pivot below spiv becomes max(|d|, spiv)
//              (counted in *nperturbed)
//   sminpiv    shared, receives the smallest pivot seen (-1 for a non-positive
//              or NaN one); may be null
//   status     when `record`, a non-positive or NaN pivot records column
//              fcol + k + 1 (smallest wins) and the column becomes NaN
//   colk, sinv shared scratch: 64 entries and one
//   accept     the factor is stored back to G unless a pivot (before its
//              square root) fell below this value (needs sminpiv); the
//              return value, uniform across the CTA, says whether it was
template <class T, bool RM, class GT>
__device__ bool potrf_block(GT* __restrict__ G, int64_t ld, int kb, T spiv, int* nperturbed, float* sminpiv,
                            int* status, bool record, int fcol, T* colk, T* sinv, float accept) {
  const int tid = threadIdx.x;
  const int E = kb * (kb + 1) / 2;
  T v[kPkSlots];
  int rr[kPkSlots], cc[kPkSlots];
#pragma unroll
  for (int q = 0; q < kPkSlots; ++q) {
    const int e = tid + kPkThreads * q;
    if (e < E) {
      pk_coord(e, kb, rr[q], cc[q]);
      v[q] = (T)(RM ? G[(int64_t)rr[q] * ld + cc[q]] : G[rr[q] + (int64_t)cc[q] * ld]);
    } else {
      rr[q] = 0;
      cc[q] = -1;   // never in a column that is scaled or updated
      v[q] = T(0);
    }
  }
  for (int k = 0; k < kb; ++k) {
    const int ek = pk_off(k, kb);
    if (tid == (ek & (kPkThreads - 1))) {
      const int qk = ek / kPkThreads;
      T dv = T(0);
#pragma unroll
      for (int q = 0; q < kPkSlots; ++q)
        if (q == qk) dv = v[q];
      if (spiv > T(0) && !(dv >= spiv)) {
        dv = fabs(dv) >= spiv ? T(fabs(dv)) : spiv;
        atomicAdd(nperturbed, 1);
      }
      const bool bad = !(dv > T(0));
      if (sminpiv && ((float)dv < *sminpiv || bad)) *sminpiv = bad ? -1.f : (float)dv;
      if (bad && record) atomicMin(status, fcol + k + 1);
      T dk, rk;
      pivot_root(dv, bad, dk, rk);
#pragma unroll
      for (int q = 0; q < kPkSlots; ++q)
        if (q == qk) v[q] = dk;
      *sinv = rk;
    }
    __syncthreads();
    const T inv = *sinv;
#pragma unroll
    for (int q = 0; q < kPkSlots; ++q)
      if (cc[q] == k && rr[q] > k) {
        v[q] *= inv;
        colk[rr[q]] = v[q];
      }
    __syncthreads();
    const int act = pk_off(k + 1, kb);   // entries e >= act are still being updated
#pragma unroll
    for (int q = 0; q < kPkSlots; ++q)
      if (tid + kPkThreads * q >= act && tid + kPkThreads * q < E) v[q] -= colk[rr[q]] * colk[cc[q]];
  }
  __syncthreads();
  const bool ok = !(sminpiv && !(*sminpiv >= accept));
  if (ok) {
#pragma unroll
    for (int q = 0; q < kPkSlots; ++q)
      if (tid + kPkThreads * q < E) {
        if (RM) G[(int64_t)rr[q] * ld + cc[q]] = (GT)v[q];
        else G[rr[q] + (int64_t)cc[q] * ld] = (GT)v[q];
      }
  }
  return ok;
}

// A CTA of kPkThreads factors a kb x kb (kb <= 64) block, row-major with
// leading dimension ld if RM, else column-major, in 8-column panels on a
// shared-memory copy (As: 64 rows of 65 entries):
// - staging: every thread issues its 16 loads before storing any, so the
//   block arrives in about one memory latency;
// - panel (warp 0): lane l holds rows c0 + l and c0 + l + 32 of the panel's 8
//   columns in registers; right-looking, one column at a time, with the pivot
//   and the column entries L(c0 + jj, k) passed by shuffles;
// - trailing update (all warps): entry (r, j), c0 + w <= j <= r, subtracts
//   the panel's w products L(r, k) L(j, k) in column order; a thread owns row
//   r = c0 + w + tid / 4 and every fourth column of it.
// Per entry this is exactly the arithmetic of potrf_block (the same fused
// multiply-subtracts, scalings and pivot roots, in the same column order), so
// the factor is bitwise the same; the difference is 2 CTA barriers per panel
// instead of 2 per column, and no per-slot bookkeeping.
//   accept   a pivot (before its square root) below it, or a NaN or
//            non-positive one, rejects the block: nothing is stored back and
//            the return value (uniform across the CTA) is false; -INFINITY
//            accepts every block
//   record   a non-positive or NaN pivot records column fcol + k + 1 in
//            *status (smallest wins); its column becomes NaN
//   sok      shared scratch word
constexpr int kPwLd = 65;
template <class T>
__device__ __forceinline__ T fmsub(T a, T b, T c) {   // c - a b, one rounding
  if constexpr (sizeof(T) == 8) return fma(-a, b, c);
  else return fmaf(-a, b, c);
}
// Warp 0 factors the 8-column panel [c0, c0 + w) of As in registers (lane l
// holds rows c0 + l and c0 + l + 32): right-looking, one column at a time, the
// pivot and the column entries L(c0 + jj, k) passed by shuffles. Clears *sok
// if a pivot (before its square root) is below `accept` (when accept >
// -INFINITY), zero, negative or NaN.
template <class T>
__device__ __forceinline__ void potrf_panel_warp(T* __restrict__ As, int c0, int w, float accept, int* sok,
                                                 int* status, bool record, int fcol) {
  const int lane = threadIdx.x & 31;
  const int ra = c0 + lane, rb = ra + 32;
  T xa[8], xb[8];
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    xa[t] = ra < 64 ? As[ra * kPwLd + c0 + t] : T(0);
    xb[t] = rb < 64 ? As[rb * kPwLd + c0 + t] : T(0);
  }
  bool ok = true;
  const bool check = accept > -INFINITY;
#pragma unroll
  for (int kk = 0; kk < 8; ++kk) {
    if (kk < w) {
      const T dk = __shfl_sync(0xffffffffu, xa[kk], kk);
      const bool bad = !(dk > T(0));
      ok = ok && (!check || (!bad && (float)dk >= accept));
      if (bad && record && lane == 0) atomicMin(status, fcol + c0 + kk + 1);
      T root, rroot;
      pivot_root(dk, bad, root, rroot);
      const int rk = c0 + kk;
      xa[kk] = ra == rk ? root : (ra > rk ? xa[kk] * rroot : xa[kk]);
      xb[kk] = xb[kk] * rroot;   // rb >= c0 + 32 > rk
#pragma unroll
      for (int jj = kk + 1; jj < 8; ++jj) {
        const T cj = __shfl_sync(0xffffffffu, xa[kk], jj);   // L(c0 + jj, rk)
        xa[jj] = fmsub(xa[kk], cj, xa[jj]);
        xb[jj] = fmsub(xb[kk], cj, xb[jj]);
      }
    }
  }
#pragma unroll
  for (int t = 0; t < 8; ++t) {
    if (ra < 64) As[ra * kPwLd + c0 + t] = xa[t];
    if (rb < 64) As[rb * kPwLd + c0 + t] = xb[t];
  }
  if (lane == 0 && !ok) *sok = 0;
}

// Entry (r, j) -= sum_t L(r, c0 + t) L(j, c0 + t), t < w, in t order.
template <class T>
__device__ __forceinline__ void potrf_rank8(T* __restrict__ As, int r, int j, int c0, int w) {
  const T* Ar = As + r * kPwLd + c0;
  const T* Aj = As + j * kPwLd + c0;
  T acc = As[r * kPwLd + j];
#pragma unroll
  for (int t = 0; t < 8; ++t)
    if (t < w) acc = fmsub(Ar[t], Aj[t], acc);
  As[r * kPwLd + j] = acc;
}

// The panel loop of potrf_panels on a block already staged in As (64 rows of
// kPwLd entries, lower triangle of a kb x kb block), with a one-panel
// lookahead. For each panel p: first every thread subtracts panel p's rank-8
// product from panel p + 1's columns (a short step), then warp 0 factors panel
// p + 1 while warps 1-7 subtract panel p's product from the columns right of
// it. Every entry still receives its panel products in panel order, each as w
// fused multiply-subtracts in column order, so the factor is bitwise that of
// the plain panel loop; the trailing update is off the critical path. Uniform
// return value as below. Nothing is read from or written to global memory
// except *status.
template <class T>
__device__ __forceinline__ bool potrf_panels_smem(int kb, float accept, T* __restrict__ As, int* sok, int* status,
                                                  bool record, int fcol) {
  const int tid = threadIdx.x;
  if (tid == 0) *sok = 1;
  __syncthreads();
  if (tid < 32 && kb > 0) potrf_panel_warp<T>(As, 0, min(8, kb), accept, sok, status, record, fcol);
  __syncthreads();
  for (int c0 = 0; c0 < kb; c0 += 8) {
    const int w = min(8, kb - c0), n0 = c0 + w;        // panel p = [c0, n0), next panel [n0, n1)
    const int nw = min(8, kb - n0), n1 = n0 + nw;
    if (n0 >= kb) break;                                // uniform: p was the last panel
    // panel p+1's columns: entry (r, j), n0 <= j < n1, j <= r; thread owns row
    // n0 + tid / 4 and columns n0 + (tid & 3), n0 + (tid & 3) + 4
    {
      const int r = n0 + (tid >> 2);
      if (r < kb)
        for (int j = n0 + (tid & 3); j < n1 && j <= r; j += 4) potrf_rank8<T>(As, r, j, c0, w);
    }
    __syncthreads();
    if (tid < 32) {
      potrf_panel_warp<T>(As, n0, nw, accept, sok, status, record, fcol);
    } else {
      // the columns right of panel p+1: entry (r, j), n1 <= j <= r; a thread
      // owns row r = n1 + (tid - 32) / 4 and every fourth column of it
      const int t2 = tid - 32;
      const int r = n1 + (t2 >> 2);
      if (r < kb)
        for (int j = n1 + (t2 & 3); j <= r; j += 4) potrf_rank8<T>(As, r, j, c0, w);
    }
    __syncthreads();
  }
  return *sok != 0;
}

template <class T, bool RM>
__device__ __forceinline__ bool potrf_panels(T* __restrict__ G, int64_t ld, int kb, float accept, T* __restrict__ As,
                                             int* sok, int* status, bool record, int fcol) {
  const int tid = threadIdx.x;
  {
    T v[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int q = tid + kPkThreads * i;
      const int r = RM ? q >> 6 : q & 63, c = RM ? q & 63 : q >> 6;   // coalesced either way
      v[i] = (r < kb && c <= r) ? (RM ? G[(int64_t)r * ld + c] : G[r + (int64_t)c * ld]) : T(0);
    }
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int q = tid + kPkThreads * i;
      const int r = RM ? q >> 6 : q & 63, c = RM ? q & 63 : q >> 6;
      As[r * kPwLd + c] = v[i];
    }
  }
  const bool ok = potrf_panels_smem<T>(kb, accept, As, sok, status, record, fcol);
  if (ok) {
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      const int q = tid + kPkThreads * i;
      const int r = RM ? q >> 6 : q & 63, c = RM ? q & 63 : q >> 6;
      if (r < kb && c <= r) {
        if (RM) G[(int64_t)r * ld + c] = As[r * kPwLd + c];
        else G[r + (int64_t)c * ld] = As[r * kPwLd + c];
      }
    }
  }
  return ok;
}

