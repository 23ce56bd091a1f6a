// assemble.cuh -- warp-sized relind scatter-add tasks (Sec. II-A assembly).
//
// Small assembly tasks (at most kAsmWarpPos row positions of the target and
// kAsmWarpEntries entries in all) take one warp each instead of one CTA, so an
// SM keeps dozens of them in flight; their cost is the chain of dependent loads
// (task, descriptors, row structures), not the bytes moved. The warp stages
// the task's slice of struct(K) and the positions of each segment's rows in its
// own shared-memory slice, then subtracts the segment's entries of U_J,
// kAsmWarpUnroll per lane with the loads issued before the stores. Segments
// are applied in order, so each entry of K receives its contributions in a
// fixed order, exactly as in the CTA-sized tasks.
#pragma once
#include <cstdint>

#include "internal.h"
#include "bounds.cuh"

constexpr int kAsmWarpUnroll = 4;

// One warp, one task. ROWMAJOR: U_J row-major (ld = b rounded up to 8) and
// row-major panels (the binary32 modes); else U_J column-major (ld = b) and
// column-major panels (binary64). sK and pos: kAsmWarpPos ints each, private to
// the warp.
template <class T, bool ROWMAJOR>
__device__ __forceinline__ void assemble_warp_task(const AsmTask& t, const AsmSeg* __restrict__ segs,
                                                   const SnodeDev* __restrict__ sn,
                                                   const int32_t* __restrict__ rows, const T* __restrict__ U,
                                                   T* __restrict__ L, int32_t* sK, int32_t* pos) {
  const int lane = threadIdx.x & 31;
#ifdef CHOL_BOUNDS_CHECK
  if (!CHOL_BC(t.K >= 0 && t.K < bc_lim.ns, kBcTaskTarget)) return;
#endif
  const SnodeDev dk = sn[t.K];
  const int np = t.p1 - t.p0;
#ifdef CHOL_BOUNDS_CHECK
  if (!CHOL_BC(t.p0 >= 0 && np >= 0 && t.p1 <= dk.len && np <= kAsmWarpPos && t.seg_begin >= 0 &&
                   t.seg_begin <= t.seg_end && t.seg_end <= bc_lim.nsegs,
               kBcTaskPositions))
    return;
#endif
  const int32_t* rk = rows + dk.roff + t.p0;
  for (int i = lane; i < np; i += 32) sK[i] = rk[i];
  T* Lk = L + dk.loff;
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
                     nu <= kAsmWarpPos,
                 kBcSegRange))
      continue;
#endif
    __syncwarp();   // sK staged / previous segment done with pos[]
    for (int i = lane; i < nu; i += 32) {
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
    __syncwarp();
    const T* Uj = U + dj.uoff;
    const int ldu = ROWMAJOR ? ((b + 7) & ~7) : b;
    const int total = nu * w;
    for (int e0 = lane; e0 < total; e0 += 32 * kAsmWarpUnroll) {
      T v[kAsmWarpUnroll], l[kAsmWarpUnroll];
      int64_t off[kAsmWarpUnroll];
#pragma unroll
      for (int q = 0; q < kAsmWarpUnroll; ++q) {
        const int e = e0 + 32 * q;
        off[q] = -1;
        if (e < total) {
          // consecutive lanes take consecutive entries of the contiguous dimension
          const int ui = ROWMAJOR ? e / w : e % nu;
          const int ci = ROWMAJOR ? e - ui * w : e / nu;
          const int u = sg.ua + ui, c = sg.ca + ci;
          if (c <= u) {
            const int64_t col = rj[c] - dk.f;
#ifdef CHOL_BOUNDS_CHECK
            if (!CHOL_BC(col >= 0 && col < dk.s, kBcTargetCol) || pos[ui] < 0) continue;
#endif
            off[q] = ROWMAJOR ? (int64_t)pos[ui] * dk.ld + col : col * dk.ld + pos[ui];
            v[q] = ROWMAJOR ? Uj[(int64_t)u * ldu + c] : Uj[(int64_t)c * ldu + u];
          }
        }
      }
#pragma unroll
      for (int q = 0; q < kAsmWarpUnroll; ++q)
        if (off[q] >= 0) l[q] = Lk[off[q]];
#pragma unroll
      for (int q = 0; q < kAsmWarpUnroll; ++q)
        if (off[q] >= 0) Lk[off[q]] = l[q] - v[q];
    }
  }
}

// One launch of warp tasks: blockDim.x / 32 tasks per CTA.
template <class T, bool ROWMAJOR>
__global__ void __launch_bounds__(256)
k_assemble_warp(const AsmTask* __restrict__ tasks, int ntasks, const AsmSeg* __restrict__ segs,
                const SnodeDev* __restrict__ sn, const int32_t* __restrict__ rows, const T* __restrict__ U,
                T* __restrict__ L) {
  __shared__ int32_t wsm[8][2 * kAsmWarpPos];
  const int warp = threadIdx.x >> 5;
  const int i = blockIdx.x * (blockDim.x >> 5) + warp;
  if (i >= ntasks) return;
  assemble_warp_task<T, ROWMAJOR>(tasks[i], segs, sn, rows, U, L, wsm[warp], wsm[warp] + kAsmWarpPos);
}
