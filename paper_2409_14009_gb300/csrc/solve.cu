// solve.cu -- forward and backward substitution with the supernodal factor.
//
// X = P^T L^{-T} L^{-1} P B: the triangular factors give the solution (Sec. I).
// One engine serves both storage forms:
// - binary64, column-major panels, binary64 vectors;
// - the mixed modes' binary32 row-major panels, binary32 vectors. Here the
//   right-hand sides are scaled by D and by their max-norm on the way in and
//   scaled back on the way out.
//
// Forward, levels leaves -> root, for every supernode J of the level:
//   - the diagonal triangle, as 64-row blocks in one cooperative launch per
//     level (k_sv_tri): a block accumulates the products with the blocks
//     already solved as their flags are published, then substitutes.
//   - one panel product w_J = L_RJ y_J for the off-diagonal rows (k_sv_gemv).
//   - w_J is scatter-subtracted into the ancestors' rows of y through the
//     factor's pull-ordered relind task lists (k_sv_fasm).
//   Supernodes with s <= 32 and len <= 256 take one warp each instead.
// Backward, levels root -> leaves:
//   - y_J -= L_RJ^T x_R, a gather of the already final ancestor rows (k_sv_bpanel).
//   - the transposed diagonal triangle, blocks last to first (k_sv_tri).
// Every output entry is written by exactly one thread per launch and every
// reduction runs in a fixed order, so the solve is deterministic.
#include <mutex>
#include <type_traits>

#include "device.h"
#include "mixed.h"

namespace {

constexpr int kT = 256;
constexpr int kSub = 64;

inline unsigned grid1d(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g > 0 ? g : 1);
}

// L(r, c) of supernode d in either storage form.
template <class T, bool RM>
__device__ __forceinline__ T lval(const T* __restrict__ P, const SnodeDev& d, int r, int c) {
  return RM ? P[(int64_t)r * d.ld + c] : P[r + (int64_t)c * d.ld];
}

__device__ __forceinline__ double scale_of(const unsigned long long* s, int r) {
  if (!s) return 1.0;
  const double v = __longlong_as_double((long long)s[r]);
  return v > 0.0 ? v : 1.0;
}

// Y = (P B) * d / scale (d, scale optional)
template <class T>
__global__ void k_sv_permute_in(const double* __restrict__ B, const int32_t* __restrict__ perm,
                                const double* __restrict__ d, const unsigned long long* __restrict__ scale, int n,
                                int nr, T* __restrict__ Y) {
  const int64_t tot = (int64_t)n * nr;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), i = (int)(q % n);
    double v = B[perm[i] + (int64_t)r * n];
    if (d) v = v * d[i] / scale_of(scale, r);
    Y[q] = (T)v;
  }
}

template <class T>
__global__ void k_sv_permute_out(const T* __restrict__ Y, const int32_t* __restrict__ perm,
                                 const double* __restrict__ d, const unsigned long long* __restrict__ scale, int n,
                                 int nr, double* __restrict__ B) {
  const int64_t tot = (int64_t)n * nr;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), i = (int)(q % n);
    double v = (double)Y[q];
    if (d) v = v * d[i] * scale_of(scale, r);
    B[perm[i] + (int64_t)r * n] = v;
  }
}

// per right-hand side: out[r] = max_i |b_ir| (ordering of non-negative doubles)
__global__ void k_sv_maxabs(const double* __restrict__ b, int n, int nr, unsigned long long* __restrict__ out) {
  for (int r = 0; r < nr; ++r) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      m = fmax(m, fabs(b[i + (int64_t)r * n]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + r, (unsigned long long)__double_as_longlong(m));
  }
}

// Diagonal triangles of every (non-warp) supernode of a level in one
// cooperative launch. Item (J, i) owns the 64-row block blk of L_JJ (blk = i
// forward, nb-1-i transposed); the items of J are listed in dependency order.
// The binary64 kernel (k_sv_tri64) runs one right-hand-side column per item:
// virtual item v = item * nrhs + m. The binary32 kernel (k_sv_tri32) takes all
// columns of a chunk in one item. A CTA takes virtual items blockIdx.x,
// blockIdx.x + gridDim.x, ...; for each it accumulates the products with the
// blocks already solved (forward: blocks j < blk, L(blk, j) y_j; transposed:
// blocks j > blk, L(j, blk)^T x_j) as their flags are published, then
// multiplies by the block's inverse, writes its rows of Y and publishes its
// flag. Waits point only to items with smaller indices and every CTA is
// resident (cooperative launch), so the smallest unfinished item can always
// proceed. Each wait is bounded; one that gives up sets *err and carries on
// (the result is then invalid). Flags hold the value epoch + 1 of the launch
// that published them; the last CTA to finish advances the device-side epoch,
// so no reset is needed between launches (also when they are replayed from a
// CUDA graph). Every entry of Y is computed by one thread in a fixed order: the
// solve is deterministic.
struct TriItem {
  int32_t J, i, nb, fbase;
};

__device__ __forceinline__ int ld_acquire(const int* p) {
  int v;
  asm volatile("ld.acquire.gpu.global.b32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_release(int* p, int v) {
  asm volatile("st.release.gpu.global.b32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

constexpr long long kTriMaxPolls = 1ll << 24;   // seconds, with the back-off below

// ---------------------------------------------------------------------------
// Binary64 diagonal triangles through inverted 64 x 64 diagonal blocks.
// On this part a dependent binary64 FMA takes about 65 cycles and one SM
// retires two binary64 FMAs per cycle, so a 64-step substitution is a long
// latency chain and a 64 x 64 tile product with 8 right-hand sides keeps one
// SM's FP64 pipe busy for 8 us. Here each right-hand-side column of a block is
// its own item (8 columns run on 8 SMs), and after its last wait a block does
// two 64 x 64 matrix-vector products (the last dependency's tile, then the
// inverse) instead of the substitution. The inverses are formed once after the
// factor (k_diag_inv64), column-major: Dinv[(fbase + blk) * 4096 + r + 64 c] =
// (L_ii^{-1})(r, c), zero above the diagonal and past the block's width.
constexpr int kInv64Stride = kSub * kSub;

// One CTA per block: thread group g (four lanes) solves L_ii x = e_g by
// substitution, lane q holding rows q + 4 mm, giving column g of L_ii^{-1}.
__global__ void __launch_bounds__(kT)
k_diag_inv64(const SnodeDev* __restrict__ sn, const TriItem* __restrict__ items, const double* __restrict__ L,
             double* __restrict__ Dinv) {
  __shared__ double Lk[kSub * 65];   // L_ii, column-major (ld 65), zero above the diagonal and past kb
  __shared__ double rinv[kSub];
  const TriItem item = items[blockIdx.x];
  const SnodeDev d = sn[item.J];
  const double* P = L + d.loff;
  const int blk = item.i, i0 = blk * kSub, kb = min(kSub, d.s - i0);
  const int tid = threadIdx.x;
  for (int e = tid; e < kSub * kSub; e += kT) {
    const int rr = e & 63, cc = e >> 6;   // consecutive threads read consecutive rows of a column
    Lk[rr + cc * 65] = (rr < kb && cc <= rr) ? P[(i0 + rr) + (int64_t)(i0 + cc) * d.ld] : 0.0;
  }
  __syncthreads();
  if (tid < kSub) rinv[tid] = tid < kb ? 1.0 / Lk[tid * 66] : 0.0;
  __syncthreads();
  const int g = tid >> 2, q = tid & 3;
  double x[16];
#pragma unroll
  for (int mm = 0; mm < 16; ++mm) x[mm] = (q + 4 * mm == g) ? 1.0 : 0.0;
  // only the first kb steps and the warps holding columns g < kb do work (a
  // ragged block of a small supernode is often much narrower than 64)
  if ((tid >> 5) * 8 < kb) {
#pragma unroll
    for (int jm = 0; jm < 16; ++jm) {
      if (jm * 4 >= kb) break;   // uniform across the CTA
#pragma unroll
      for (int jq = 0; jq < 4; ++jq) {
        const int jj = jm * 4 + jq;
        const double xj = __shfl_sync(0xffffffffu, x[jm] * rinv[jj], jq, 4);
        if (q == jq) x[jm] = xj;
#pragma unroll
        for (int mm = jm; mm < 16; ++mm) {
          const int c = q + 4 * mm;
          if (c > jj && 4 * mm < kb) x[mm] = fma(-xj, Lk[c + jj * 65], x[mm]);
        }
      }
    }
  }
  double* Di = Dinv + (int64_t)(item.fbase + blk) * kInv64Stride;
#pragma unroll
  for (int mm = 0; mm < 16; ++mm) {
    const int c = q + 4 * mm;
    Di[c + g * kSub] = (c < kb && g < kb) ? x[mm] : 0.0;
  }
}

// The binary64 triangle items of a level, one right-hand-side column each
// (column-major panels). Thread (r, g) owns row r of the block and the k range
// [16 g, 16 g + 16) of every product; it keeps four partial sums (k mod 4),
// added pairwise, and the four k-groups are added in group order, so each
// entry of Y is computed in a fixed order. The block's inverse entries and the
// last dependency's tile are loaded into registers before any wait, and each
// earlier tile's entries before its flag is read.
template <bool TRANS>
__global__ void __launch_bounds__(kT, 2)
k_sv_tri64(const SnodeDev* __restrict__ sn, const TriItem* __restrict__ items, int nitems, const double* __restrict__ L,
           const double* __restrict__ Dinv, double* __restrict__ Y, int n, int nrhs, int* __restrict__ flags,
           int* __restrict__ sync, int* __restrict__ err, long long max_polls, int skew) {
  __shared__ double ys[kSub];         // a solved block's column
  __shared__ double zs[kSub];         // this block's right-hand side, then z
  __shared__ double red[4 * kSub];    // k-group partial sums
  __shared__ int target, savail;
  const int tid = threadIdx.x, r = tid & 63, g = tid >> 6, ka = 16 * g;
  if (tid == 0) {
    target = ld_acquire(sync) + 1;
    savail = -1;
  }
  __syncthreads();
  const int tgt = target;
  const int wait_tgt = tgt + skew;   // skew != 0 only to test the failure path
  auto wait_flag = [&](const int* f) {
    if (tid == 0) {
      long long polls = 0;
      while (ld_acquire(f) != wait_tgt) {
        if (++polls > max_polls) { atomicExch(err, 1); break; }
        if (polls > 4096) __nanosleep(100);   // spin first: the hand-off is on the critical path
      }
    }
  };
  // zs[r] -= (sum of the four k-groups' partial sums), group order
  auto subtract_sums = [&](double part) {
    red[g * kSub + r] = part;
    __syncthreads();
    if (tid < kSub) zs[tid] -= ((red[tid] + red[kSub + tid]) + red[2 * kSub + tid]) + red[3 * kSub + tid];
    __syncthreads();
  };
  const int64_t nv = (int64_t)nitems * nrhs;
  for (int64_t v = blockIdx.x; v < nv; v += gridDim.x) {
    const int it = (int)(v / nrhs), m = (int)(v - (int64_t)it * nrhs);
    const TriItem item = items[it];
    const SnodeDev d = sn[item.J];
    const double* P = L + d.loff;
    const int blk = TRANS ? item.nb - 1 - item.i : item.i;
    const int i0 = blk * kSub, kb = min(kSub, d.s - i0);
    double* Ym = Y + d.f + (int64_t)m * n;
    int* fl = flags + m;   // flag of block j: fl[(fbase + j) * kSolveChunk]
    // L(row, col) of the block row r and a dependency's column k (forward), or
    // the transposed pair (L(j, blk)^T), both column-major in the panel
    auto lrow = [&](int j0, int k) -> double {
      return TRANS ? P[(j0 + k) + (int64_t)(i0 + r) * d.ld] : P[(i0 + r) + (int64_t)(j0 + k) * d.ld];
    };
    // the inverse's entries of row r (forward: L_ii^{-1}(r, k); transposed:
    // L_ii^{-T}(r, k) = L_ii^{-1}(k, r)), zero where the product has none
    const double* Di = Dinv + (int64_t)(item.fbase + blk) * kInv64Stride;
    const bool inv_live = TRANS ? (ka + 15 >= r) : (ka <= r);
    double li[16];
#pragma unroll
    for (int kk = 0; kk < 16; ++kk)
      li[kk] = inv_live ? (TRANS ? Di[(ka + kk) + r * kSub] : Di[r + (ka + kk) * kSub]) : 0.0;
    if (tid < kSub) zs[tid] = tid < kb ? Ym[i0 + tid] : 0.0;
    // the last dependency's tile
    double lt[16];
    int jl0 = 0, jlb = 0;
    if (item.i > 0) {
      const int jl = TRANS ? blk + 1 : blk - 1;
      jl0 = jl * kSub;
      jlb = min(kSub, d.s - jl0);
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) lt[kk] = (r < kb && ka + kk < jlb) ? lrow(jl0, ka + kk) : 0.0;
    }
    // the dependencies other than the last, straight from the panel
    // (blocks are published in dependency order, so once the flag of the last
    // of them is seen no further flag is read)
    double a[4] = {0.0, 0.0, 0.0, 0.0};
    const int ndep = item.i - 1;
    int avail = -1;   // dependencies 0 .. avail are known to be published
    for (int q = 0; q < ndep; ++q) {
      const int j = TRANS ? item.nb - 1 - q : q;
      const int j0 = j * kSub, jb = min(kSub, d.s - j0);
      double lv[16];
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) lv[kk] = (r < kb && ka + kk < jb) ? lrow(j0, ka + kk) : 0.0;
      if (q > avail) {
        wait_flag(fl + (int64_t)(item.fbase + j) * kSolveChunk);
        if (tid == 0) {
          const int jl = TRANS ? item.nb - ndep : ndep - 1;   // the last of them
          savail = ld_acquire(fl + (int64_t)(item.fbase + jl) * kSolveChunk) == wait_tgt ? ndep - 1 : q;
        }
      }
      __syncthreads();   // the flag (and savail) seen; the previous tile is done with ys
      avail = savail;
      if (tid < kSub) ys[tid] = tid < jb ? __ldcg(Ym + j0 + tid) : 0.0;
      __syncthreads();
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) a[kk & 3] = fma(lv[kk], ys[ka + kk], a[kk & 3]);
    }
    subtract_sums((a[0] + a[1]) + (a[2] + a[3]));
    if (item.i > 0) {
      // the last dependency: z = pre - L(i, l) y_l
      wait_flag(fl + (int64_t)(item.fbase + (TRANS ? blk + 1 : blk - 1)) * kSolveChunk);
      __syncthreads();
      if (tid < kSub) ys[tid] = tid < jlb ? __ldcg(Ym + jl0 + tid) : 0.0;
      __syncthreads();
      double b[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) b[kk & 3] = fma(lt[kk], ys[ka + kk], b[kk & 3]);
      subtract_sums((b[0] + b[1]) + (b[2] + b[3]));
    }
    // y_i = L_ii^{-1} z (forward) or L_ii^{-T} z (transposed)
    double c[4] = {0.0, 0.0, 0.0, 0.0};
    if (inv_live) {
#pragma unroll
      for (int kk = 0; kk < 16; ++kk) c[kk & 3] = fma(li[kk], zs[ka + kk], c[kk & 3]);
    }
    red[g * kSub + r] = (c[0] + c[1]) + (c[2] + c[3]);
    __syncthreads();
    if (tid < kb) Ym[i0 + tid] = ((red[tid] + red[kSub + tid]) + red[2 * kSub + tid]) + red[3 * kSub + tid];
    // the barrier orders every thread's stores of Y before thread 0's release
    // store (gpu scope, cumulative), so a consumer whose acquire load sees the
    // flag sees the rows
    __syncthreads();
    if (tid == 0) st_release(fl + (int64_t)(item.fbase + blk) * kSolveChunk, tgt);
  }
  // the last CTA to finish advances the epoch for the next launch
  __syncthreads();
  if (tid == 0) {
    __threadfence();
    if (atomicAdd(sync + 1, 1) == (int)gridDim.x - 1) {
      atomicExch(sync + 1, 0);
      __threadfence();
      atomicAdd(sync, 1);
    }
  }
}

// Panel product w_J = L_RJ y_J for the off-diagonal rows [r0, r0 + kGemvRows)
// of J, y_J staged in shared memory in chunks of KC columns.
// Column-major (binary64): 64 rows per task. The 8 warps split each chunk's
// columns (warp w takes k = w mod 8); a lane holds rows lane and lane + 32 and
// walks four of its columns at a time, so 8 independent 8-byte loads are in
// flight per lane, each warp load a contiguous 256 bytes. The warps' partial
// sums are then combined in warp order through shared memory.
// Row-major (binary32): 32 rows, a warp per 4 rows, lanes along K,
// fixed-order shuffle reduction.
template <class T, bool RM, int NR>
__global__ void __launch_bounds__(kT)
k_sv_gemv(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, const T* __restrict__ L,
          const T* __restrict__ Y, int n, T* __restrict__ W, int nrhs, T* __restrict__ spart,
          int* __restrict__ scnt) {
  constexpr int KC = 256;
  constexpr int kYk = KC * NR > 2048 ? KC * NR : 2048;   // also the binary64 warp partials (8 x 64 x 4)
  __shared__ __align__(16) T yk[kYk];
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int b = d.len - d.s;
  const T* P = L + d.loff;
  T* Wj = W + d.wpre * nrhs;
  if constexpr (!RM) {
    constexpr int NW = kT / 32;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int u0 = t.r0 + lane, u1 = u0 + 32;
    const bool in0 = u0 < b, in1 = u1 < b;
    const T* col0 = P + d.s + u0;   // L(s + u0, k) = col0[k * ld]
    T acc[2][NR];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[h][r] = T(0);
    // part `split` of `nsplit` sums over the columns [kbeg, kend) only
    const int split = t.k0 & 0xffff, nsplit = t.k0 >> 16;
    int kbeg = 0, kend = d.s;
    if (nsplit > 1) {
      const int ch = (d.s + nsplit - 1) / nsplit;
      kbeg = min(d.s, split * ch);
      kend = min(d.s, kbeg + ch);
    }
    for (int kc = kbeg; kc < kend; kc += KC) {
      const int kn = min(KC, kend - kc);
      __syncthreads();
      for (int q = threadIdx.x; q < kn * nrhs; q += blockDim.x) {
        const int i = q % kn, r = q / kn;
        yk[i + r * KC] = Y[d.f + kc + i + (int64_t)r * n];
      }
      for (int q = kn + threadIdx.x; q < KC; q += blockDim.x)   // zero tail: masked columns read 0
        for (int r = 0; r < nrhs; ++r) yk[q + r * KC] = T(0);
      __syncthreads();
      for (int k4 = warp; k4 < kn; k4 += 4 * NW) {
        T l[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = k4 + j * NW;
          const T* c = col0 + (int64_t)(kc + k) * d.ld;
          l[j][0] = (k < kn && in0) ? c[0] : T(0);
          l[j][1] = (k < kn && in1) ? c[32] : T(0);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int k = min(k4 + j * NW, KC - 1);   // l = 0 past kn
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            if (r >= nrhs) break;
            const T y = yk[k + r * KC];
            acc[0][r] += l[j][0] * y;
            acc[1][r] += l[j][1] * y;
          }
        }
      }
    }
    // combine the warps' partials in warp order, four right-hand sides a round
    T* red = yk;   // NW x 64 rows x 4
    for (int r0 = 0; r0 < nrhs; r0 += 4) {
      __syncthreads();
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        if (r0 + q >= nrhs) break;
        T v0 = T(0), v1 = T(0);
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (r == r0 + q) { v0 = acc[0][r]; v1 = acc[1][r]; }
        red[(warp * 64 + lane) * 4 + q] = v0;
        red[(warp * 64 + lane + 32) * 4 + q] = v1;
      }
      __syncthreads();
      for (int e = threadIdx.x; e < 64 * 4; e += blockDim.x) {
        const int row = e >> 2, q = e & 3;
        const int u = t.r0 + row;
        if (r0 + q >= nrhs || u >= b) continue;
        T v = T(0);
#pragma unroll
        for (int w = 0; w < NW; ++w) v += red[(w * 64 + row) * 4 + q];
        if (nsplit > 1) spart[((int64_t)(t.c0 + split) * kSolveChunk + r0 + q) * 64 + row] = v;
        else Wj[u + (int64_t)(r0 + q) * b] = v;
      }
    }
    if (nsplit > 1) {
      // the last part of the group to finish adds the parts' sums in part order
      __shared__ int last;
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(scnt + t.c0, 1) == nsplit - 1;
        if (last) {
          __threadfence();
          scnt[t.c0] = 0;   // reset for the next level or solve
        }
      }
      __syncthreads();
      if (last) {
        for (int e = threadIdx.x; e < 64 * nrhs; e += blockDim.x) {
          const int row = e & 63, r = e >> 6;
          const int u = t.r0 + row;
          if (u >= b) continue;
          const T* src = spart + ((int64_t)t.c0 * kSolveChunk + r) * 64 + row;
          T v = __ldcg(src);
          for (int q = 1; q < nsplit; ++q) v += __ldcg(src + (int64_t)q * kSolveChunk * 64);
          Wj[u + (int64_t)r * b] = v;
        }
      }
    }
  } else {
    // binary32 row-major panels: a lane covers 4 consecutive columns (one
    // 16-byte load; rows start 32-byte aligned), 128 columns per warp pass, two
    // passes per staged chunk: 8 loads of 16 bytes in flight per lane
    static_assert(sizeof(T) == 4, "row-major panels are binary32");
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T acc[4][NR];   // 4 rows per warp, 32 rows per task
#pragma unroll
    for (int m = 0; m < 4; ++m)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[m][r] = T(0);
    for (int kc = 0; kc < d.s; kc += KC) {
      const int kn = min(KC, d.s - kc);
      __syncthreads();
      for (int q = threadIdx.x; q < kn * nrhs; q += blockDim.x) {
        const int i = q % kn, r = q / kn;
        yk[i + r * KC] = Y[d.f + kc + i + (int64_t)r * n];
      }
      for (int q = kn + threadIdx.x; q < KC; q += blockDim.x)   // zero tail: full 4-column groups
        for (int r = 0; r < nrhs; ++r) yk[q + r * KC] = T(0);
      __syncthreads();
      float4 lv[4][2];
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        const int u = t.r0 + warp * 4 + m;
        const float* row = reinterpret_cast<const float*>(P) + (int64_t)(d.s + u) * d.ld + kc;
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const int k = 4 * lane + 128 * h;
          if (u < b && k + 3 < kn) {
            lv[m][h] = *reinterpret_cast<const float4*>(row + k);
          } else {
            lv[m][h].x = (u < b && k < kn) ? row[k] : 0.f;
            lv[m][h].y = (u < b && k + 1 < kn) ? row[k + 1] : 0.f;
            lv[m][h].z = (u < b && k + 2 < kn) ? row[k + 2] : 0.f;
            lv[m][h].w = 0.f;
          }
        }
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 4 * lane + 128 * h;
#pragma unroll
        for (int r = 0; r < NR; ++r) {
          if (r >= nrhs) break;
          const float4 y4 = *reinterpret_cast<const float4*>(reinterpret_cast<const float*>(yk) + k + r * KC);
#pragma unroll
          for (int m = 0; m < 4; ++m)
            acc[m][r] += lv[m][h].x * y4.x + lv[m][h].y * y4.y + lv[m][h].z * y4.z + lv[m][h].w * y4.w;
        }
      }
    }
#pragma unroll
    for (int m = 0; m < 4; ++m) {
      const int u = t.r0 + warp * 4 + m;
#pragma unroll
      for (int r = 0; r < NR; ++r) {
        T v = acc[m][r];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if (lane == 0 && u < b && r < nrhs) Wj[u + (int64_t)r * b] = v;
      }
    }
  }
}

// y[targets] -= w_J through the relind task lists (pull-ordered), one warp per
// task: only the first position chunk of a column tile holds the segments'
// columns; segments are applied in order (the same y entries can appear in
// several), so each entry receives its contributions in a fixed order.
template <class T>
__global__ void __launch_bounds__(kT)
k_sv_fasm(const AsmTask* __restrict__ tasks, int ntasks, const AsmSeg* __restrict__ segs,
          const SnodeDev* __restrict__ sn, const int32_t* __restrict__ rows, const T* __restrict__ W,
          T* __restrict__ Y, int n, int nrhs) {
  const int i = blockIdx.x * (kT / 32) + (threadIdx.x >> 5), lane = threadIdx.x & 31;
  if (i >= ntasks) return;
  const AsmTask t = tasks[i];
  if (t.p0 != t.t0) return;
  for (int g = t.seg_begin; g < t.seg_end; ++g) {
    const AsmSeg sg = segs[g];
    const SnodeDev dj = sn[sg.J];
    const int b = dj.len - dj.s;
    const int32_t* rj = rows + dj.roff + dj.s;
    const T* Wj = W + dj.wpre * nrhs;
    const int ncol = sg.cb - sg.ca;
    for (int q = lane; q < ncol * nrhs; q += 32) {
      const int c = sg.ca + q % ncol, r = q / ncol;
      Y[rj[c] + (int64_t)r * n] -= Wj[c + (int64_t)r * b];
    }
    __syncwarp();
  }
}

// Backward panel: y_J[c] -= sum_u L(s+u, c) x[rows[s+u]] for the columns of a task.
// Column-major (binary64): 16 columns per task, two per warp. The gathered
// x[rows[s+u]] of a 256-row chunk are staged in shared memory once for the
// task; a lane walks rows lane, lane + 32, ... of both its columns, four rows
// at a time (8 independent loads in flight, each warp load a contiguous 256
// bytes), then a fixed shuffle tree sums the lanes. Row-major: 64 columns per
// task, a thread per (column, row group of 4), fixed-order combination.
template <class T, bool RM, int NR>
__global__ void __launch_bounds__(kT)
k_sv_bpanel(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, const int32_t* __restrict__ rows,
            const T* __restrict__ L, T* __restrict__ Y, int n, int nrhs, T* __restrict__ spart,
            int* __restrict__ scnt) {
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int b = d.len - d.s;
  const int32_t* rj = rows + d.roff + d.s;
  const T* P = L + d.loff;
  if constexpr (!RM) {
    constexpr int CH = 256;
    __shared__ T xs[CH * NR];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int c0 = t.c0 + 2 * warp;
    const bool in0 = c0 < d.s, in1 = c0 + 1 < d.s;
    const T* colA = P + d.s + (int64_t)c0 * d.ld;   // L(s + u, c0) = colA[u]
    const T* colB = colA + d.ld;
    T acc[2][NR];
#pragma unroll
    for (int h = 0; h < 2; ++h)
#pragma unroll
      for (int r = 0; r < NR; ++r) acc[h][r] = T(0);
    // part `split` of `nsplit` sums over the rows [ubeg, uend) only
    const int split = t.k0 & 0xffff, nsplit = t.k0 >> 16;
    int ubeg = 0, uend = b;
    if (nsplit > 1) {
      const int ch = (b + nsplit - 1) / nsplit;
      ubeg = min(b, split * ch);
      uend = min(b, ubeg + ch);
    }
    for (int ub = ubeg; ub < uend; ub += CH) {
      const int un = min(CH, uend - ub);
      __syncthreads();
      for (int q = threadIdx.x; q < un * nrhs; q += blockDim.x) {
        const int i = q % un, r = q / un;
        xs[i + r * CH] = Y[rj[ub + i] + (int64_t)r * n];
      }
      __syncthreads();
      for (int i4 = lane; i4 < un; i4 += 128) {
        T l[4][2];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int i = i4 + 32 * j;
          l[j][0] = (i < un && in0) ? colA[ub + i] : T(0);
          l[j][1] = (i < un && in1) ? colB[ub + i] : T(0);
        }
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          const int i = i4 + 32 * j;
          if (i >= un) break;
#pragma unroll
          for (int r = 0; r < NR; ++r) {
            if (r >= nrhs) break;
            const T x = xs[i + r * CH];
            acc[0][r] += l[j][0] * x;
            acc[1][r] += l[j][1] * x;
          }
        }
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) {
      if (r >= nrhs) break;
      T v0 = acc[0][r], v1 = acc[1][r];
      for (int o = 16; o > 0; o >>= 1) {
        v0 += __shfl_xor_sync(0xffffffffu, v0, o);
        v1 += __shfl_xor_sync(0xffffffffu, v1, o);
      }
      if (nsplit > 1) {
        // slot: 16 columns x kSolveChunk right-hand sides
        if (lane == 0) {
          T* dst = spart + ((int64_t)(t.r0 + split) * kSolveChunk + r) * 16 + 2 * warp;
          dst[0] = v0;
          dst[1] = v1;
        }
      } else {
        if (lane == 0 && in0) Y[d.f + c0 + (int64_t)r * n] -= v0;
        if (lane == 0 && in1) Y[d.f + c0 + 1 + (int64_t)r * n] -= v1;
      }
    }
    if (nsplit > 1) {
      // the last part of the group to finish subtracts the parts' sums, added in part order
      __shared__ int last;
      __syncthreads();
      if (threadIdx.x == 0) {
        __threadfence();
        last = atomicAdd(scnt + t.r0, 1) == nsplit - 1;
        if (last) {
          __threadfence();
          scnt[t.r0] = 0;   // reset for the next level or solve
        }
      }
      __syncthreads();
      if (last) {
        for (int e = threadIdx.x; e < 16 * nrhs; e += blockDim.x) {
          const int col = e & 15, r = e >> 4;
          const int c = t.c0 + col;
          if (c >= d.s) continue;
          const T* src = spart + ((int64_t)t.r0 * kSolveChunk + r) * 16 + col;
          T v = __ldcg(src);
          for (int q = 1; q < nsplit; ++q) v += __ldcg(src + (int64_t)q * kSolveChunk * 16);
          Y[d.f + c + (int64_t)r * n] -= v;
        }
      }
    }
  } else {
    __shared__ T part[4][64][NR + 1];
    const int col = threadIdx.x & 63, rg = threadIdx.x >> 6;
    const int c = t.c0 + col;
    T acc[NR];
#pragma unroll
    for (int r = 0; r < NR; ++r) acc[r] = T(0);
    if (c < d.s) {
      for (int u = rg; u < b; u += 4) {
        const T l = lval<T, RM>(P, d, d.s + u, c);
        const int32_t g = rj[u];
#pragma unroll
        for (int r = 0; r < NR; ++r)
          if (r < nrhs) acc[r] += l * Y[g + (int64_t)r * n];
      }
    }
#pragma unroll
    for (int r = 0; r < NR; ++r) part[rg][col][r] = acc[r];
    __syncthreads();
    if (rg == 0 && c < d.s) {
      for (int r = 0; r < nrhs; ++r) {
        const T v = ((part[0][col][r] + part[1][col][r]) + part[2][col][r]) + part[3][col][r];
        Y[d.f + c + (int64_t)r * n] -= v;
      }
    }
  }
}

// Backward panel for row-major storage, two stages. Stage 1: a task (J, 64-row
// chunk u0, 256-column tile c0) writes part[chunk][c] = sum over its rows of
// L(s+u, c) x[rows[s+u]] (rows walked contiguously, coalesced). Stage 2: for
// each column, the chunk partials are summed in chunk order and subtracted.
template <class T, int NR>
__global__ void __launch_bounds__(kT)
k_sv_bpart(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, const int32_t* __restrict__ rows,
           const T* __restrict__ L, const T* __restrict__ Y, int n, T* __restrict__ part, int64_t pstride,
           int nrhs) {
  __shared__ T xs[kSub * NR];
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int b = d.len - d.s;
  const int u0 = t.r0, chunk = t.k0;
  const int nr64 = min(kSub, b - u0);
  const int32_t* rj = rows + d.roff + d.s + u0;
  for (int q = threadIdx.x; q < nr64 * nrhs; q += blockDim.x) {
    const int u = q % nr64, r = q / nr64;
    xs[u + r * kSub] = Y[rj[u] + (int64_t)r * n];
  }
  __syncthreads();
  const int c = t.c0 + threadIdx.x;
  if (c >= d.s) return;
  const T* P = L + d.loff + (int64_t)(d.s + u0) * d.ld + c;
  T acc[NR];
#pragma unroll
  for (int r = 0; r < NR; ++r) acc[r] = T(0);
#pragma unroll 8
  for (int u = 0; u < nr64; ++u) {
    const T l = P[(int64_t)u * d.ld];
#pragma unroll
    for (int r = 0; r < NR; ++r)
      if (r < nrhs) acc[r] += l * xs[u + r * kSub];
  }
  T* out = part + d.ppre + (int64_t)chunk * d.s + c;
#pragma unroll
  for (int r = 0; r < NR; ++r)
    if (r < nrhs) out[r * pstride] = acc[r];
}

template <class T>
__global__ void __launch_bounds__(kT)
k_sv_bred(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, const T* __restrict__ part,
          int64_t pstride, T* __restrict__ Y, int n, int nrhs) {
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int c = t.c0 + threadIdx.x;
  if (c >= d.s) return;
  const int nchunks = (d.len - d.s + kSub - 1) / kSub;
  for (int r = 0; r < nrhs; ++r) {
    const T* p = part + r * pstride + d.ppre + c;
    T acc = T(0);
    for (int ch = 0; ch < nchunks; ++ch) acc += p[(int64_t)ch * d.s];
    Y[d.f + c + (int64_t)r * n] -= acc;
  }
}

// Small supernodes (s <= 32, len <= 256), one warp each. Lane i holds row i of
// the diagonal block in registers (loaded once, with the reciprocal pivots), so
// the substitution chain is shuffles and FMAs only. Forward: the solved entry
// is broadcast by shuffle; then w_J = L_RJ y_J with lanes along the
// off-diagonal rows. S bounds s (8 or 32), which sizes the register copy of
// the row.
template <class T, bool RM, int S>
__global__ void __launch_bounds__(kT)
k_sv_small_fwd(const SnodeDev* __restrict__ sn, const int32_t* __restrict__ list, int count,
               const T* __restrict__ L, T* __restrict__ Y, int n, T* __restrict__ W, int nrhs) {
  __shared__ T ysh[kT / 32][S];
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= count) return;
  const SnodeDev d = sn[list[wid]];
  const T* P = L + d.loff;
  const int b = d.len - d.s;
  T* Wj = W + d.wpre * nrhs;
  // binary64: lane i holds row i of the block scaled by 1 / L(i, i), y_i =
  // b_i / L(i, i) - sum_k (L(i, k) / L(i, i)) y_k, so a step of the substitution
  // chain is a shuffle and one FMA (a binary64 multiply on the chain costs ~65
  // cycles). binary32 (4-cycle multiplies) keeps the unscaled rows and divides
  // on the chain, which rounds once less per entry.
  constexpr bool kScaled = sizeof(T) == 8;
  const T rdiag = lane < d.s ? T(1) / lval<T, RM>(P, d, lane, lane) : T(0);
  T lrow[S];   // L(lane, k) (binary64: / L(lane, lane)), k < lane (s <= S)
#pragma unroll
  for (int k = 0; k < S; ++k)
    lrow[k] = (k < lane && lane < d.s) ? lval<T, RM>(P, d, lane, k) * (kScaled ? rdiag : T(1)) : T(0);
  for (int r = 0; r < nrhs; ++r) {
    T y = lane < d.s ? Y[d.f + lane + (int64_t)r * n] * (kScaled ? rdiag : T(1)) : T(0);
#pragma unroll
    for (int k = 0; k < S; ++k) {
      if (k < d.s) {   // uniform across the warp
        if constexpr (kScaled) {
          const T yk = __shfl_sync(0xffffffffu, y, k);
          if (lane > k) y -= lrow[k] * yk;
        } else {
          const T yk = __shfl_sync(0xffffffffu, y * rdiag, k);
          if (lane == k) y = yk;
          if (lane > k) y -= lrow[k] * yk;
        }
      }
    }
    if (lane < d.s) Y[d.f + lane + (int64_t)r * n] = y;
    // w_J = L_RJ y_J, lane u holding rows u, u + 32, ...: per 32-row group all
    // s entries of the lane's row are loaded at once (one memory round trip per
    // group), then multiplied with y_J from shared memory; binary64 keeps four
    // partial sums (k mod 4, added pairwise) to shorten its FMA chain, binary32
    // one, in k order
    T* yk = ysh[threadIdx.x >> 5];   // y_J of this warp's supernode (broadcast reads)
    if (lane < S) yk[lane] = y;
    __syncwarp();
    for (int c = 0; c < kSolveSmallRows / 32; ++c) {
      if (32 * c >= b) break;   // uniform across the warp
      const int u = lane + 32 * c;
      // binary64 with S = 32: two halves of 16 loads (the row copy of the
      // block stays in registers for every right-hand side)
      constexpr int KH = (sizeof(T) == 8 && S > 16) ? 16 : S;
      T a4[4] = {T(0), T(0), T(0), T(0)};
#pragma unroll 1
      for (int k0 = 0; k0 < S; k0 += KH) {
        if (k0 >= d.s) break;   // uniform across the warp
        T lv[KH];
#pragma unroll
        for (int kk = 0; kk < KH; ++kk)
          lv[kk] = (k0 + kk < d.s && u < b) ? lval<T, RM>(P, d, d.s + u, k0 + kk) : T(0);
#pragma unroll
        for (int kk = 0; kk < KH; ++kk) a4[kScaled ? (kk & 3) : 0] += lv[kk] * yk[k0 + kk];
      }
      if (u < b) Wj[u + (int64_t)r * b] = (a4[0] + a4[1]) + (a4[2] + a4[3]);
    }
    __syncwarp();   // the next right-hand side rewrites yk
  }
}

// Backward for the same supernodes: lane k gathers t_k = sum_u L(s+u, k) x[rows[s+u]]
// (ancestor rows are final; four rows' loads in flight), then the transposed
// diagonal solve with shuffles, lane i holding column i of the block.
template <class T, bool RM, int S>
__global__ void __launch_bounds__(kT)
k_sv_small_bwd(const SnodeDev* __restrict__ sn, const int32_t* __restrict__ list, int count,
               const int32_t* __restrict__ rows, const T* __restrict__ L, T* __restrict__ Y, int n, int nrhs) {
  const int wid = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  if (wid >= count) return;
  const SnodeDev d = sn[list[wid]];
  const T* P = L + d.loff;
  const int b = d.len - d.s;
  const int32_t* rj = rows + d.roff + d.s;
  // lane i holds column i of the block (binary64: scaled by 1 / L(i, i), as in
  // the forward kernel)
  constexpr bool kScaled = sizeof(T) == 8;
  const T rdiag = lane < d.s ? T(1) / lval<T, RM>(P, d, lane, lane) : T(0);
  T lcol[S];   // L(k, lane) (binary64: / L(lane, lane)), k > lane (s <= S)
#pragma unroll
  for (int k = 0; k < S; ++k)
    lcol[k] = (k > lane && k < d.s) ? lval<T, RM>(P, d, k, lane) * (kScaled ? rdiag : T(1)) : T(0);
  for (int r = 0; r < nrhs; ++r) {
    // binary64: four partial sums (u mod 4), added pairwise, a chain of b/4
    // dependent FMAs; binary32: one, in u order (16 rows' loads in flight per
    // round)
    T t4[4] = {T(0), T(0), T(0), T(0)};
    if (lane < d.s) {
      for (int u0 = 0; u0 < b; u0 += 16) {
        T lv[16], xv[16];
#pragma unroll
        for (int uu = 0; uu < 16; ++uu) {
          const int u = u0 + uu;
          lv[uu] = u < b ? lval<T, RM>(P, d, d.s + u, lane) : T(0);
          xv[uu] = u < b ? Y[rj[u] + (int64_t)r * n] : T(0);
        }
#pragma unroll
        for (int uu = 0; uu < 16; ++uu) t4[kScaled ? (uu & 3) : 0] += lv[uu] * xv[uu];
      }
    }
    const T t = (t4[0] + t4[1]) + (t4[2] + t4[3]);
    T y = lane < d.s ? (Y[d.f + lane + (int64_t)r * n] - t) * (kScaled ? rdiag : T(1)) : T(0);
#pragma unroll
    for (int k = S - 1; k >= 0; --k) {
      if (k < d.s) {   // uniform across the warp
        if constexpr (kScaled) {
          const T xk = __shfl_sync(0xffffffffu, y, k);
          if (lane < k) y -= lcol[k] * xk;
        } else {
          const T xk = __shfl_sync(0xffffffffu, y * rdiag, k);
          if (lane == k) y = xk;
          if (lane < k) y -= lcol[k] * xk;
        }
      }
    }
    if (lane < d.s) Y[d.f + lane + (int64_t)r * n] = y;
  }
}

// ---------------------------------------------------------------------------
// Binary32 diagonal triangles: each 64-row block is solved by a product with
// its inverse, and the product with its last dependency's solved block goes
// through a matrix formed with that inverse in advance, so that after the last
// wait a block does one tile product. Per block three 64 x 64 row-major
// matrices, at Dinv + (fbase + blk) * kInvStride:
//   Li   = L_ii^{-1};
//   Mf   = L_ii^{-1} L(i, i-1)        (forward, i >= 1);
//   Mb   = L_ii^{-T} L(i+1, i)^T      (transposed, i + 1 < nb).
constexpr int kInvStride = 3 * kSub * kSub;

// One CTA per block of the forward item order (which lists each block once):
// thread group g (four lanes) solves L_ii x = e_g by substitution, giving
// column g of L_ii^{-1}; then the two 64 x 64 x 64 products, k in order.
__global__ void __launch_bounds__(kT)
k_diag_inv(const SnodeDev* __restrict__ sn, const TriItem* __restrict__ items, const float* __restrict__ L,
           float* __restrict__ Dinv) {
  __shared__ float Lk[kSub * 65];              // L_ii (column-major), then the tile of a product
  __shared__ __align__(16) float Li[kSub * kSub];   // L_ii^{-1}, row-major
  __shared__ float rinv[kSub];
  const TriItem item = items[blockIdx.x];
  const SnodeDev d = sn[item.J];
  const float* P = L + d.loff;
  const int blk = item.i, i0 = blk * kSub, kb = min(kSub, d.s - i0);
  const int tid = threadIdx.x;
  for (int e = tid; e < kSub * kSub; e += kT) {
    const int rr = e >> 6, cc = e & 63;   // consecutive threads read consecutive columns of a row
    Lk[rr + cc * 65] = (rr < kb && cc <= rr) ? P[(int64_t)(i0 + rr) * d.ld + i0 + cc] : 0.f;
  }
  __syncthreads();
  if (tid < kSub) rinv[tid] = tid < kb ? 1.f / Lk[tid + tid * 65] : 0.f;
  __syncthreads();
  {
    const int g = tid >> 2, q = tid & 3;
    float x[16];
#pragma unroll
    for (int mm = 0; mm < 16; ++mm) x[mm] = (q + 4 * mm == g) ? 1.f : 0.f;
#pragma unroll
    for (int jm = 0; jm < 16; ++jm) {
#pragma unroll
      for (int jq = 0; jq < 4; ++jq) {
        const int jj = jm * 4 + jq;
        const float xj = __shfl_sync(0xffffffffu, x[jm] * rinv[jj], jq, 4);
        if (q == jq) x[jm] = xj;
#pragma unroll
        for (int mm = jm; mm < 16; ++mm) {
          const int c = q + 4 * mm;
          if (c > jj) x[mm] -= xj * Lk[c + jj * 65];
        }
      }
    }
    float* Di = Dinv + (int64_t)(item.fbase + blk) * kInvStride;
#pragma unroll
    for (int mm = 0; mm < 16; ++mm) {
      const int c = q + 4 * mm;
      const float v = (c < kb && g < kb) ? x[mm] : 0.f;
      Di[c * kSub + g] = v;
      Li[c * kSub + g] = v;
    }
  }
  const int tx = tid & 15, ty = tid >> 4;
  float* Mf = Dinv + (int64_t)(item.fbase + blk) * kInvStride + kSub * kSub;
  float* Mb = Mf + kSub * kSub;
  if (blk >= 1) {
    // Mf = L_ii^{-1} L(i, i-1): the tile rows i0.., columns (blk - 1) * 64.. (full)
    __syncthreads();   // Li is complete, Lk is free
    const int c0 = (blk - 1) * kSub;
    for (int e = tid; e < kSub * kSub; e += kT) {
      const int t = e >> 6, k = e & 63;
      Lk[t * 65 + k] = t < kb ? P[(int64_t)(i0 + t) * d.ld + c0 + k] : 0.f;
    }
    __syncthreads();
    float acc[4][4] = {};
    for (int t = 0; t < kSub; ++t) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Li[(ty + 16 * i) * kSub + t];
#pragma unroll
      for (int l = 0; l < 4; ++l) b[l] = Lk[t * 65 + tx + 16 * l];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int l = 0; l < 4; ++l) acc[i][l] = fmaf(a[i], b[l], acc[i][l]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int l = 0; l < 4; ++l) Mf[(ty + 16 * i) * kSub + tx + 16 * l] = acc[i][l];
  }
  if (blk + 1 < item.nb) {
    // Mb = L_ii^{-T} L(i+1, i)^T: the tile rows (blk + 1) * 64.., columns i0..,
    // staged transposed: Lk[t * 65 + k] = L((blk + 1) * 64 + k, i0 + t)
    __syncthreads();   // Li is complete, the previous product is done with Lk
    const int r1 = (blk + 1) * kSub, rb = min(kSub, d.s - r1);
    for (int e = tid; e < kSub * kSub; e += kT) {
      const int k = e >> 6, t = e & 63;   // consecutive threads read consecutive columns of a row
      Lk[t * 65 + k] = (k < rb && t < kb) ? P[(int64_t)(r1 + k) * d.ld + i0 + t] : 0.f;
    }
    __syncthreads();
    float acc[4][4] = {};
    for (int t = 0; t < kSub; ++t) {
      float a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = Li[t * kSub + ty + 16 * i];
#pragma unroll
      for (int l = 0; l < 4; ++l) b[l] = Lk[t * 65 + tx + 16 * l];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int l = 0; l < 4; ++l) acc[i][l] = fmaf(a[i], b[l], acc[i][l]);
    }
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int l = 0; l < 4; ++l) Mb[(ty + 16 * i) * kSub + tx + 16 * l] = acc[i][l];
  }
}

// catch-up tiles of the binary32 triangle kernel per staging round
constexpr int kCatch = 4;

size_t tri32_smem(int nr) {
  // ys (kCatch solved blocks, kCatch x 64 x nr), yi (64 x nr), L_ii^{-1} and M
  // (64 x 65 each), the k-group partial sums (4 x 64 x nr)
  return sizeof(float) * ((size_t)(kCatch + 5) * kSub * nr + 2 * kSub * 65);
}

// Binary32 diagonal triangles of a level (row-major panels). Same items, epochs
// and bounded waits as k_sv_tri64, but a solved block is handed over through
// tagged words instead of flags: besides its rows of Y, a block stores each
// entry as one 64-bit word {binary32 bits, launch tag} (hand, indexed like Y),
// and a consumer spins on the words it needs until they carry this launch's
// tag. A 64-bit aligned access is single-copy atomic, so a word with the right
// tag holds the right value: no flag, fence or barrier sits between a block's
// result and its consumers, and the hand-off costs one memory round trip.
// For block i with last dependency l (forward l = i - 1; transposed l = i + 1):
//   pre = L_ii^{-1} (b_i - sum over the other dependencies j of L(i, j) y_j)
// is formed before the last wait (forward; the transposed solve uses
// L_ii^{-T} and L(j, i)^T), then y_i = pre - M y_l with M = Mf or Mb. Thread
// (r, g) owns row r and the k range [16 g, 16 g + 16) of every product; the
// four partial sums are added in group order, so the solve is deterministic.
__device__ __forceinline__ unsigned long long ld_relaxed_u64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}

__device__ __forceinline__ void st_relaxed_u64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}

template <bool TRANS, int NR>
__global__ void __launch_bounds__(kT)
k_sv_tri32(const SnodeDev* __restrict__ sn, const TriItem* __restrict__ items, int nitems, const float* __restrict__ L,
           const float* __restrict__ Dinv, float* __restrict__ Y, unsigned long long* __restrict__ hand, int n,
           int nrhs, int* __restrict__ sync, int* __restrict__ err, long long max_polls, int skew) {
  extern __shared__ __align__(16) unsigned char sv_smem[];
  float* ys = reinterpret_cast<float*>(sv_smem);   // kCatch solved blocks, kCatch x 64 x nrhs
  float* yi = ys + kCatch * kSub * nrhs;            // this block's right-hand sides, then pre
  float* red = yi + kSub * nrhs;                    // k-group partial sums, 4 x 64 x nrhs
  float* Ls = red + 4 * kSub * nrhs;                // L_ii^{-1}, column-major (ld 65)
  float* Ms = Ls + kSub * 65;                       // M, column-major (ld 65)
  __shared__ int target;
  if (threadIdx.x == 0) target = ld_acquire(sync) + 1;
  __syncthreads();
  const int tgt = target;
  const unsigned wait_tag = (unsigned)(tgt + skew);   // skew != 0 only to test the failure path
  const unsigned long long tag_hi = (unsigned long long)(unsigned)tgt << 32;
  const int tid = threadIdx.x, r = tid & 63, g = tid >> 6, ka = 16 * g;
  // ys = the solved rows [j0, j0 + jb) of the supernode starting at column f
  // (zero past jb), each read from its tagged word once the tag is this
  // launch's (bounded: a wait that gives up sets *err and takes the value)
  auto stage_solved = [&](float* dst, int64_t f, int j0, int jb) {
    for (int e = tid; e < kSub * nrhs; e += kT) {
      const int k = e & (kSub - 1), m = e / kSub;
      float v = 0.f;
      if (k < jb) {
        const unsigned long long* p = hand + f + j0 + k + (int64_t)m * n;
        unsigned long long w = ld_relaxed_u64(p);
        long long polls = 0;
        while ((unsigned)(w >> 32) != wait_tag) {
          if (++polls > max_polls) { atomicExch(err, 1); break; }
          if ((polls & 255) == 0 && *(volatile int*)err != 0) break;   // another wait gave up: stop
          if (polls > 4096) __nanosleep(100);   // spin first: the hand-off is on the critical path
          w = ld_relaxed_u64(p);
        }
        v = __uint_as_float((unsigned)w);
      }
      dst[k + m * kSub] = v;
    }
  };
  // partial sums of acc into red (the caller then combines them)
  auto reduce = [&](const float (&acc)[NR]) {
#pragma unroll
    for (int m = 0; m < NR; ++m)
      if (m < nrhs) red[(g * kSub + r) + m * 4 * kSub] = acc[m];
    __syncthreads();
  };
  for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
    const TriItem item = items[it];
    const SnodeDev d = sn[item.J];
    const float* P = L + d.loff;
    const int blk = TRANS ? item.nb - 1 - item.i : item.i;
    const int i0 = blk * kSub, kb = min(kSub, d.s - i0);
    const float* Di = Dinv + (int64_t)(item.fbase + blk) * kInvStride;
    // the inverse, M and the right-hand sides, before any wait
    for (int e = tid; e < kSub * kSub; e += kT) Ls[(e >> 6) + (e & 63) * 65] = Di[e];
    if (item.i > 0) {
      const float* Mx = Di + (TRANS ? 2 : 1) * kSub * kSub;
      for (int e = tid; e < kSub * kSub; e += kT) Ms[(e >> 6) + (e & 63) * 65] = Mx[e];
    }
    for (int e = tid; e < kb * nrhs; e += kT) {
      const int rr = e % kb, m = e / kb;
      yi[rr + m * kSub] = Y[d.f + i0 + rr + (int64_t)m * n];
    }
    float acc[NR];
#pragma unroll
    for (int m = 0; m < NR; ++m) acc[m] = 0.f;
    // the dependencies other than the last, from the panel, kCatch tiles a
    // round: their entries are loaded first, then their solved blocks are
    // staged together (one hand-off round trip per round, overlapping the
    // loads), then the products in dependency order
    const int ndep = item.i - 1;
    for (int q0 = 0; q0 < ndep; q0 += kCatch) {
      float lv[kCatch][16];
#pragma unroll
      for (int t = 0; t < kCatch; ++t) {
        const int q = q0 + t;
        const int j = TRANS ? item.nb - 1 - q : q;
        const int j0 = j * kSub, jb = min(kSub, d.s - j0);
        const int row = i0 + r;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          const int k = ka + kk;
          lv[t][kk] = (q < ndep && r < kb && k < jb)
                          ? (TRANS ? P[(int64_t)(j0 + k) * d.ld + row] : P[(int64_t)row * d.ld + j0 + k])
                          : 0.f;
        }
      }
      __syncthreads();   // the previous round is done with ys
      {
        // the round's solved blocks: up to four tagged words of a thread in
        // flight at once, then each checked (and waited for, bounded)
        const int per = kSub * nrhs, tot = min(kCatch, ndep - q0) * per;
        for (int e0 = tid; e0 < tot; e0 += 4 * kT) {
          unsigned long long w[4];
          const unsigned long long* src[4];
          int dsti[4];
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            const int e = e0 + u * kT;
            const int t = e / per, em = e - t * per, k = em & (kSub - 1), m = em / kSub;
            const int j = TRANS ? item.nb - 1 - (q0 + t) : q0 + t;
            const int j0 = j * kSub, jb = min(kSub, d.s - j0);
            src[u] = (e < tot && k < jb) ? hand + d.f + j0 + k + (int64_t)m * n : nullptr;
            dsti[u] = e < tot ? e : -1;
            w[u] = src[u] ? ld_relaxed_u64(src[u]) : 0ull;
          }
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (dsti[u] < 0) continue;
            float v = 0.f;   // zero past a ragged block
            if (src[u]) {
              long long polls = 0;
              while ((unsigned)(w[u] >> 32) != wait_tag) {
                if (++polls > max_polls) { atomicExch(err, 1); break; }
                if ((polls & 255) == 0 && *(volatile int*)err != 0) break;
                if (polls > 4096) __nanosleep(100);
                w[u] = ld_relaxed_u64(src[u]);
              }
              v = __uint_as_float((unsigned)w[u]);
            }
            ys[dsti[u]] = v;
          }
        }
      }
      __syncthreads();
#pragma unroll
      for (int t = 0; t < kCatch; ++t) {
        if (q0 + t >= ndep) break;
#pragma unroll
        for (int kk = 0; kk < 16; ++kk)
#pragma unroll
          for (int m = 0; m < NR; ++m)
            if (m < nrhs) acc[m] += lv[t][kk] * ys[t * kSub * nrhs + ka + kk + m * kSub];
      }
    }
    __syncthreads();   // every thread is done with ys and red
    reduce(acc);
    for (int e = tid; e < kb * nrhs; e += kT) {
      const int rr = e % kb, m = e / kb;
      const float* pr = red + m * 4 * kSub + rr;
      yi[rr + m * kSub] -= ((pr[0] + pr[kSub]) + pr[2 * kSub]) + pr[3 * kSub];
    }
    __syncthreads();
    // pre = L_ii^{-1} yi (forward) or L_ii^{-T} yi (transposed)
    float acc2[NR];
#pragma unroll
    for (int m = 0; m < NR; ++m) acc2[m] = 0.f;
    if (r < kb) {
#pragma unroll 4
      for (int kk = 0; kk < 16; ++kk) {
        const int k = ka + kk;
        // rows of yi past kb are not staged: skip them (never multiply by 0)
        if (TRANS ? (k >= r && k < kb) : (k <= r)) {
          const float a = TRANS ? Ls[k + r * 65] : Ls[r + k * 65];
#pragma unroll
          for (int m = 0; m < NR; ++m)
            if (m < nrhs) acc2[m] += a * yi[k + m * kSub];
        }
      }
    }
    __syncthreads();   // every read of yi is done
    reduce(acc2);
    for (int e = tid; e < kb * nrhs; e += kT) {
      const int rr = e % kb, m = e / kb;
      const float* pr = red + m * 4 * kSub + rr;
      yi[rr + m * kSub] = ((pr[0] + pr[kSub]) + pr[2 * kSub]) + pr[3 * kSub];
    }
    // y_i (pre, minus M y_l for i > 0): rows of Y and their tagged words
    auto publish = [&](int rr, int m, float y) {
      const int64_t q = d.f + i0 + rr + (int64_t)m * n;
      Y[q] = y;
      st_relaxed_u64(hand + q, tag_hi | __float_as_uint(y));
    };
    if (item.i > 0) {
      // the last dependency: y_i = pre - M y_l
      const int q = item.i - 1;
      const int j = TRANS ? item.nb - 1 - q : q;
      const int j0 = j * kSub, jb = min(kSub, d.s - j0);
      __syncthreads();   // pre is in yi, red is free
      stage_solved(ys, d.f, j0, jb);
      __syncthreads();
      float acc3[NR];
#pragma unroll
      for (int m = 0; m < NR; ++m) acc3[m] = 0.f;
      if (r < kb) {
        const int kz = min(jb, ka + 16);
#pragma unroll
        for (int kk = 0; kk < 16; ++kk) {
          if (ka + kk >= kz) break;
          const float a = Ms[r + (ka + kk) * 65];
#pragma unroll
          for (int m = 0; m < NR; ++m)
            if (m < nrhs) acc3[m] += a * ys[ka + kk + m * kSub];
        }
      }
      reduce(acc3);
      for (int e = tid; e < kb * nrhs; e += kT) {
        const int rr = e % kb, m = e / kb;
        const float* pr = red + m * 4 * kSub + rr;
        publish(rr, m, yi[rr + m * kSub] - (((pr[0] + pr[kSub]) + pr[2 * kSub]) + pr[3 * kSub]));
      }
    } else {
      __syncthreads();
      for (int e = tid; e < kb * nrhs; e += kT) {
        const int rr = e % kb, m = e / kb;
        publish(rr, m, yi[rr + m * kSub]);
      }
    }
    __syncthreads();   // the next item reuses the shared buffers
  }
  // the last CTA to finish advances the epoch for the next launch
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    if (atomicAdd(sync + 1, 1) == (int)gridDim.x - 1) {
      atomicExch(sync + 1, 0);
      __threadfence();
      atomicAdd(sync, 1);
    }
  }
}

// The level schedule of one solve on a chunk of nr <= 16 right-hand sides
// already permuted into Y (W: per-level panel products). `prof` enables the
// per-class launch accounting (off for the no-allocation entry point).
// Resident CTAs per SM of each triangle kernel per chunk width (set once).
int g_tri_per_sm[2][2][kSolveChunk + 1] = {};   // [binary32][transposed][nr]

// The panel-product and binary32 triangle kernels keep per-thread sums for at
// most NR right-hand sides: 1, 4, 8 or the chunk (fewer registers, more
// resident CTAs for few).
template <class F>
void with_nr(int nr, F&& f) {
  if (nr <= 1) f(std::integral_constant<int, 1>{});
  else if (nr <= 4) f(std::integral_constant<int, 4>{});
  else if (nr <= 8) f(std::integral_constant<int, 8>{});
  else f(std::integral_constant<int, kSolveChunk>{});
}

// One cooperative launch of the level's diagonal triangles: k_sv_tri64
// (binary64, one right-hand-side column per item) or k_sv_tri32 (binary32, all
// columns of the chunk per item); both multiply by the blocks' inverses.
template <class T, bool RM, bool TRANS>
int launch_tri(chol_handle* h, const LevelPlan& P, const T* L, T* Y, int nr, cudaStream_t st) {
  DeviceState* D = h->dev;
  constexpr bool f32 = sizeof(T) == 4;
  const int per_sm = g_tri_per_sm[f32][TRANS][nr];
  if (per_sm < 1) return CHOL_ENOTSUP;
  const int64_t work = f32 ? (int64_t)P.tri_n : (int64_t)P.tri_n * nr;
  const int grid = (int)std::min<int64_t>(work, (int64_t)per_sm * D->sms);
  const TriItem* items = reinterpret_cast<const TriItem*>(D->tri) + P.tri_b;
  int nitems = P.tri_n, n = h->n;
  long long max_polls = h->opt.wait_polls > 0 ? (long long)h->opt.wait_polls : kTriMaxPolls;
  int skew = h->opt.test_unreachable_flags ? 1 : 0;
  cudaError_t e;
  if constexpr (f32) {
    const float* Dinv = reinterpret_cast<const float*>(D->dinv);
    void* args[] = {(void*)&D->sn, (void*)&items, (void*)&nitems, (void*)&L, (void*)&Dinv, (void*)&Y, (void*)&D->hand32,
                    (void*)&n, (void*)&nr, (void*)&D->tri_sync, (void*)&D->sv_err, (void*)&max_polls, (void*)&skew};
    with_nr(nr, [&](auto c) {
      e = cudaLaunchCooperativeKernel((const void*)k_sv_tri32<TRANS, decltype(c)::value>, dim3(grid), dim3(kT), args,
                                      tri32_smem(nr), st);
    });
  } else {
    static_assert(f32 || !RM, "binary64 panels are column-major");
    const double* Dinv = reinterpret_cast<const double*>(D->dinv);
    void* args[] = {(void*)&D->sn, (void*)&items, (void*)&nitems, (void*)&L, (void*)&Dinv, (void*)&Y, (void*)&n,
                    (void*)&nr, (void*)&D->tri_flags, (void*)&D->tri_sync, (void*)&D->sv_err, (void*)&max_polls,
                    (void*)&skew};
    e = cudaLaunchCooperativeKernel((const void*)k_sv_tri64<TRANS>, dim3(grid), dim3(kT), args, 0, st);
  }
  if (e != cudaSuccess) {
    cudaGetLastError();
    return CHOL_ECUDA;
  }
  return CHOL_OK;
}

template <class T, bool RM>
int solve_levels(chol_handle* h, const T* L, T* Y, T* W, T* part, int nr, cudaStream_t st, bool prof) {
  DeviceState* D = h->dev;
  const int n = h->n;
  auto scope = [&](int cls) { return prof ? new KScope(h, cls, st, 0.0, 0.0) : nullptr; };
  {   // forward pass (an NVTX range over the scope; early returns pop it)
  NvtxRange nvtx_forward("forward");
  for (const LevelPlan& P : h->levels) {
    if (P.ssmall_n > 0) {
      // supernodes with s <= 8 first, then the wider ones
      KScope* ks = scope(CHOL_K_SOLVE_DIAG);
      const int n8 = P.ssmall8_n, nw = P.ssmall_n - P.ssmall8_n;
      if (n8 > 0)
        k_sv_small_fwd<T, RM, 8><<<(n8 + 7) / 8, kT, 0, st>>>(D->sn, D->ssmall + P.ssmall_b, n8, L, Y, n, W, nr);
      if (nw > 0)
        k_sv_small_fwd<T, RM, 32><<<(nw + 7) / 8, kT, 0, st>>>(D->sn, D->ssmall + P.ssmall_b + n8, nw, L, Y, n, W, nr);
      if (ks) ks->launches((n8 > 0) + (nw > 0));
      delete ks;
    }
    if (P.tri_n > 0) {
      KScope* ks = scope(CHOL_K_SOLVE_DIAG);
      const int rc = launch_tri<T, RM, false>(h, P, L, Y, nr, st);
      delete ks;
      if (rc) return rc;
    }
    if (P.gemv_n > 0) {
      KScope* ks = scope(CHOL_K_SOLVE_GEMV);
      with_nr(nr, [&](auto c) {
        k_sv_gemv<T, RM, decltype(c)::value><<<P.gemv_n, kT, 0, st>>>(D->sn, D->gemv + P.gemv_b, L, Y, n, W, nr,
                                                                      (T*)D->split_part, D->split_cnt);
      });
      delete ks;
    }
    if (P.asm_n + P.asmw_n > 0) {
      // the CTA-sized and the warp-sized assembly tasks of the level, contiguous
      KScope* ks = scope(CHOL_K_SOLVE_FASM);
      const int nt = P.asm_n + P.asmw_n;
      k_sv_fasm<T><<<(nt + kT / 32 - 1) / (kT / 32), kT, 0, st>>>(D->asm_tasks + P.asm_b, nt, D->asm_segs, D->sn,
                                                                  D->rows, W, Y, n, nr);
      delete ks;
    }
  }
  }
  NvtxRange nvtx_backward("backward");
  for (int lv = h->nlevels - 1; lv >= 0; --lv) {
    const LevelPlan& P = h->levels[lv];
    if constexpr (RM) {
      if (P.bpart_n > 0) {
        KScope* ks = scope(CHOL_K_SOLVE_BPANEL);
        with_nr(nr, [&](auto c) {
          k_sv_bpart<T, decltype(c)::value><<<P.bpart_n, kT, 0, st>>>(D->sn, D->bpart + P.bpart_b, D->rows, L, Y, n,
                                                                      part, h->p_max, nr);
        });
        k_sv_bred<T><<<P.bred_n, kT, 0, st>>>(D->sn, D->bred + P.bred_b, part, h->p_max, Y, n, nr);
        delete ks;
      }
    } else if (P.bpanel_n > 0) {
      KScope* ks = scope(CHOL_K_SOLVE_BPANEL);
      with_nr(nr, [&](auto c) {
        k_sv_bpanel<T, RM, decltype(c)::value><<<P.bpanel_n, kT, 0, st>>>(D->sn, D->bpanel + P.bpanel_b, D->rows, L,
                                                                          Y, n, nr, (T*)D->split_part, D->split_cnt);
      });
      delete ks;
    }
    if (P.ssmall_n > 0) {
      KScope* ks = scope(CHOL_K_SOLVE_DIAG);
      const int n8 = P.ssmall8_n, nw = P.ssmall_n - P.ssmall8_n;
      if (n8 > 0)
        k_sv_small_bwd<T, RM, 8><<<(n8 + 7) / 8, kT, 0, st>>>(D->sn, D->ssmall + P.ssmall_b, n8, D->rows, L, Y, n, nr);
      if (nw > 0)
        k_sv_small_bwd<T, RM, 32><<<(nw + 7) / 8, kT, 0, st>>>(D->sn, D->ssmall + P.ssmall_b + n8, nw, D->rows, L, Y,
                                                                n, nr);
      if (ks) ks->launches((n8 > 0) + (nw > 0));
      delete ks;
    }
    if (P.tri_n > 0) {
      KScope* ks = scope(CHOL_K_SOLVE_DIAG);
      const int rc = launch_tri<T, RM, true>(h, P, L, Y, nr, st);
      delete ks;
      if (rc) return rc;
    }
  }
  return CHOL_OK;
}

int set_solve_attrs() {
  static std::once_flag once;
  static int rc = CHOL_OK;
  std::call_once(once, [] {
    const void* kd[2] = {(const void*)k_sv_tri64<false>, (const void*)k_sv_tri64<true>};
    cudaError_t e = cudaSuccess;
    for (int t = 0; t < 2; ++t) {
      for (int nr = 1; nr <= kSolveChunk; ++nr) {
        e = e ? e : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_tri_per_sm[0][t][nr], kd[t], kT, 0);
        // the binary32 kernel of this chunk width's NR class
        with_nr(nr, [&](auto c) {
          const void* kf = t ? (const void*)k_sv_tri32<true, decltype(c)::value>
                             : (const void*)k_sv_tri32<false, decltype(c)::value>;
          e = e ? e : cudaFuncSetAttribute(kf, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)tri32_smem(decltype(c)::value));
          e = e ? e : cudaOccupancyMaxActiveBlocksPerMultiprocessor(&g_tri_per_sm[1][t][nr], kf, kT, tri32_smem(nr));
        });
      }
    }
    if (e != cudaSuccess) {
      cudaGetLastError();
      rc = CHOL_ECUDA;
    }
  });
  return rc;
}

int ensure_solve_ws(chol_handle* h) {
  DeviceState* D = h->dev;
  if (!D->Y) {
    int rc = chol_dalloc(h, (void**)&D->Y, sizeof(double) * (size_t)std::max(h->n, 1) * kSolveChunk);
    if (rc) return rc;
  }
  if (!D->W) {
    int rc = chol_dalloc(h, (void**)&D->W, sizeof(double) * (size_t)std::max<int64_t>(h->w_rows_max, 1) * kSolveChunk);
    if (rc) return rc;
  }
  return CHOL_OK;
}

// binary64 solve of b (n x nrhs, ld n) in place with workspaces Y, W of
// chunk columns each
int solve_fp64(chol_handle* h, double* b, int32_t nrhs, cudaStream_t st, double* Y, double* W, int chunk,
               bool prof) {
  DeviceState* D = h->dev;
  const int n = h->n;
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    const int nr = std::min(chunk, nrhs - r0);
    double* B = b + (int64_t)r0 * n;
    KScope* ks = prof ? new KScope(h, CHOL_K_PERMUTE, st, 0.0, 24.0 * n * nr) : nullptr;
    k_sv_permute_in<double><<<grid1d((int64_t)n * nr, 256), 256, 0, st>>>(B, D->perm, nullptr, nullptr, n, nr, Y);
    delete ks;
    const int rc = solve_levels<double, false>(h, (const double*)D->L, Y, W, (double*)nullptr, nr, st, prof);
    if (rc) return rc;
    ks = prof ? new KScope(h, CHOL_K_PERMUTE, st, 0.0, 24.0 * n * nr) : nullptr;
    k_sv_permute_out<double><<<grid1d((int64_t)n * nr, 256), 256, 0, st>>>(Y, D->perm, nullptr, nullptr, n, nr, B);
    delete ks;
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CHOL_OK : CHOL_ECUDA;
}

}  // namespace

// Binary32 solve with the mixed-precision factor, in place on a binary64 block.
int chol_solve_mixed(chol_handle* h, double* b, int32_t nrhs, cudaStream_t st) {
  int rc = set_solve_attrs();
  if (rc) return rc;
  DeviceState* D = h->dev;
  const int n = h->n;
  if (!D->Y32) {
    if ((rc = chol_dalloc(h, (void**)&D->Y32, sizeof(float) * (size_t)std::max(n, 1) * kSolveChunk))) return rc;
    // tagged hand-off words of the triangle launches: zero (no launch tag) once
    if ((rc = chol_dalloc(h, (void**)&D->hand32, sizeof(unsigned long long) * (size_t)std::max(n, 1) * kSolveChunk)))
      return rc;
    CHOL_CUDA_TRY(cudaMemset(D->hand32, 0, sizeof(unsigned long long) * (size_t)std::max(n, 1) * kSolveChunk));
    if ((rc = chol_dalloc(h, (void**)&D->W32, sizeof(float) * (size_t)std::max<int64_t>(h->w_rows_max, 1) * kSolveChunk)))
      return rc;
    if ((rc = chol_dalloc(h, (void**)&D->rhs_scale, sizeof(double) * kSolveChunk))) return rc;
    if ((rc = chol_dalloc(h, (void**)&D->P32, sizeof(float) * (size_t)std::max<int64_t>(h->p_max, 1) * kSolveChunk)))
      return rc;
  }
  unsigned long long* sc = (unsigned long long*)D->rhs_scale;
  for (int r0 = 0; r0 < nrhs; r0 += kSolveChunk) {
    const int nr = std::min(kSolveChunk, nrhs - r0);
    double* B = b + (int64_t)r0 * n;
    CHOL_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(double) * kSolveChunk, st));
    {
      KScope ks(h, CHOL_K_PERMUTE, st, 0.0, 12.0 * n * nr);
      k_sv_maxabs<<<grid1d(n, 256), 256, 0, st>>>(B, n, nr, sc);
      k_sv_permute_in<float><<<grid1d((int64_t)n * nr, 256), 256, 0, st>>>(B, D->perm, D->mx_d, sc, n, nr, D->Y32);
    }
    if ((rc = solve_levels<float, true>(h, (const float*)D->L, D->Y32, D->W32, D->P32, nr, st, true))) return rc;
    {
      KScope ks(h, CHOL_K_PERMUTE, st, 0.0, 12.0 * n * nr);
      k_sv_permute_out<float><<<grid1d((int64_t)n * nr, 256), 256, 0, st>>>(D->Y32, D->perm, D->mx_d, sc, n, nr, B);
    }
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

// Inverses of the diagonal blocks the triangle solves multiply by, for the
// triangle items [b, b + nitems) of a factor enqueued on st (their blocks
// final): binary64 (column-major panels) the inverse alone, binary32 (row-major
// panels) the inverse and the two last-dependency products.
int chol_diag_inv(chol_handle* h, int b, int nitems, cudaStream_t st) {
  DeviceState* D = h->dev;
  if (nitems <= 0) return CHOL_OK;
  const TriItem* items = reinterpret_cast<const TriItem*>(D->tri) + b;
  if (h->opt.precision == CHOL_PREC_FP64) {
    // per block: the inverse by substitution, about 64^3 / 3 flops
    KScope ks(h, CHOL_K_SOLVE_DIAG, st, (double)nitems * 64.0 * 64.0 * 64.0 / 3.0,
              (double)nitems * 64.0 * 64.0 * 8.0 * 1.5);
    k_diag_inv64<<<nitems, kT, 0, st>>>(D->sn, items, (const double*)D->L, (double*)D->dinv);
  } else {
    // per block: the inverse by substitution and up to two 64^3 products
    KScope ks(h, CHOL_K_SOLVE_DIAG, st, (double)nitems * 5.0 * 64.0 * 64.0 * 64.0,
              (double)nitems * 64.0 * 64.0 * 4.0 * 6.0);
    k_diag_inv<<<nitems, kT, 0, st>>>(D->sn, items, (const float*)D->L, (float*)D->dinv);
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

// CHOL_ETIMEOUT if a triangle launch gave up waiting since the last check
// (for callers that have synchronized with the solves).
int chol_solve_status(chol_handle* h) {
  DeviceState* D = h->dev;
  if (!D || !D->sv_err) return CHOL_OK;
  int32_t e = 0;
  CHOL_CUDA_TRY(cudaMemcpy(&e, D->sv_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (e != 0) {
    CHOL_CUDA_TRY(cudaMemset(D->sv_err, 0, sizeof(int32_t)));
    return CHOL_ETIMEOUT;
  }
  return CHOL_OK;
}

extern "C" int chol_check_waits(chol_handle* h, void* stream) {
  if (!h) return -1;
  if (int rc_state = chol_factored_here(h)) return rc_state;
  CHOL_CUDA_TRY(cudaStreamSynchronize((cudaStream_t)stream));
  return chol_solve_status(h);
}

extern "C" int chol_solve(chol_handle* h, double* b, int32_t nrhs, void* stream) {
  NvtxRange nvtx_range("chol_solve");
  if (!h) return -1;
  if (!b && nrhs > 0 && h->n > 0) return -2;
  if (nrhs < 0) return -3;
  if (int rc_state = chol_factored_here(h)) return rc_state;
  if (nrhs == 0 || h->n == 0) return CHOL_OK;
  if (h->opt.precision != CHOL_PREC_FP64) return chol_solve_mixed(h, b, nrhs, (cudaStream_t)stream);
  int rc = set_solve_attrs();
  if (rc) return rc;
  if ((rc = ensure_solve_ws(h))) return rc;
  DeviceState* D = h->dev;
  return solve_fp64(h, b, nrhs, (cudaStream_t)stream, D->Y, D->W, kSolveChunk, true);
}

// ---------------------------------------------------------------------------
// chol_solve_noalloc: the same forward/backward substitution as chol_solve, for
// callers that must not allocate device memory once set up -- for example a
// service whose memory pool has already claimed the GPU, or a latency-bound
// loop where a cudaMalloc could stall on device-wide synchronization. Its two
// workspaces (the permuted right-hand sides and the per-level panel products)
// live in one fixed, file-scope device array instead of handle-owned buffers.
//
// The array holds kNoAllocScratchDoubles doubles (16 MiB) on every GPU that
// loads this library, for the life of the process. A solve needs n + w_rows
// doubles per right-hand-side column (w_rows: the largest sum of off-diagonal
// rows over one level); right-hand sides are processed in chunks that fit, and
// a problem whose single column does not fit is rejected with CHOL_ETOOBIG.
//
// The array is shared by every call on a device and keeps the previous call's
// contents; nothing in it needs to start at zero (each chunk writes Y before
// reading it, and each level writes its W rows before reading them).
// Calls whose work overlaps on the GPU (different streams or threads) race on
// the array. The first call on each device looks up the array's device address
// with cudaGetSymbolAddress (with that device current), and looks it up again
// when the device's context has changed (after a cudaDeviceReset); make that
// first call before any stream capture. The handle's device must be current
// (CHOL_ESTATE otherwise), because the array and the factor are per device.
// ---------------------------------------------------------------------------
constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kNoAllocMaxDevices] = {};
unsigned long long g_noalloc_ctx[kNoAllocMaxDevices] = {};   // context id the address belongs to

typedef CUresult (*CtxGetCurrentFn)(CUcontext*);
typedef CUresult (*CtxGetIdFn)(CUcontext, unsigned long long*);

// Process-unique id of the current context (0 if the driver cannot say). A
// cudaDeviceReset destroys the primary context and the module with it; the next
// context gets a new id, so the array's address is looked up again.
unsigned long long current_ctx_id() {
  static CtxGetCurrentFn get_cur = nullptr;
  static CtxGetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_cur, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      get_cur = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q) !=
            cudaSuccess || q != cudaDriverEntryPointSuccess)
      get_id = nullptr;
    cudaGetLastError();
    resolved = true;
  }
  CUcontext ctx = nullptr;
  unsigned long long id = 0;
  if (get_cur && get_id && get_cur(&ctx) == CUDA_SUCCESS && ctx && get_id(ctx, &id) == CUDA_SUCCESS) return id;
  return 0;
}

// Device address of g_noalloc_scratch on the current device: looked up once
// per device and context (cudaGetSymbolAddress with that device current).
int noalloc_scratch(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    return CHOL_ECUDA;
  }
  const unsigned long long ctx = current_ctx_id();
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev] || g_noalloc_ctx[dev] != ctx) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return CHOL_ECUDA;
    }
    g_noalloc_addr[dev] = static_cast<double*>(p);
    g_noalloc_ctx[dev] = ctx;
  }
  *out = g_noalloc_addr[dev];
  return CHOL_OK;
}

}  // namespace

extern "C" int chol_solve_noalloc(chol_handle* h, double* b, int32_t nrhs, void* stream) {
  if (!h) return -1;
  if (!b && nrhs > 0 && h->n > 0) return -2;
  if (nrhs < 0) return -3;
  const int64_t per_col = (int64_t)h->n + h->w_rows_max;
  if (per_col > kNoAllocScratchDoubles) return CHOL_ETOOBIG;
  if (int rc_state = chol_factored_here(h)) return rc_state;
  if (h->opt.precision != CHOL_PREC_FP64) return CHOL_ENOTSUP;
  if (nrhs == 0 || h->n == 0) return CHOL_OK;
  int rc = set_solve_attrs();
  if (rc) return rc;
  double* scratch = nullptr;
  if ((rc = noalloc_scratch(&scratch))) return rc;
  const int chunk = (int)std::min<int64_t>(kSolveChunk, kNoAllocScratchDoubles / std::max<int64_t>(per_col, 1));
  double* Y = scratch;
  double* W = scratch + (int64_t)h->n * chunk;
  return solve_fp64(h, b, nrhs, (cudaStream_t)stream, Y, W, chunk, false);
}
