// adjoint.cu -- selected inverse and gradients of x = A^{-1} b and log det A.
//
// The loss l = sum_k w_k^T x_k + alpha log det A, with X = A^{-1} B, has
//   dl/dB = Xbar = A^{-1} W          (two triangular solves with the factor)
//   dl/dA = -Xbar X^T + alpha A^{-1}
// and, for the stored lower entries (a_ij and a_ji move together):
//   g_ii = G_ii,  g_ij = G_ij + G_ji (i > j).
// Only the entries of A^{-1} on the pattern of A are needed. They come from
// the selected inverse Z = (P A P^T)^{-1} on the pattern of L. Z is computed
// supernode by supernode from the root down, with dense blocks:
//   T    = L_JJ^{-1}
//   Uhat = L_RJ T
//   Z_RJ = -Z_RR Uhat          (Z_RR gathered from the ancestors through the
//                               relative positions, the factor's scatter in
//                               reverse)
//   Z_JJ = T^T T - Uhat^T Z_RJ
// Z is stored in the layout of the factor's panels (binary64, column-major).
#include <cstring>
#include <vector>

#include "device.h"
#include "mixed.h"

namespace {

constexpr int kGT = 256;
constexpr int kGTile = 64;

// Generic strided binary64 GEMM tile: C = beta C + alpha A B over a 64 x 64
// tile. A(i,k) = A[i*ar + k*ac], B(k,j) = B[k*br + j*bc], C(i,j) = C[i*cr + j*cc].
// amode: 0 general, 1 A lower triangular (A(i,k) = 0 for k > i), 2 A symmetric
// stored in its lower triangle. bmode: 0 general, 1 B lower triangular
// (B(k,j) = 0 for j > k). lower_c: write only i >= j.
struct GenGemm {
  const double* A;
  int64_t ar, ac;
  const double* B;
  int64_t br, bc;
  double* C;
  int64_t cr, cc;
  int M, N, K;
  double alpha, beta;
  int amode, bmode, lower_c;
  int ksplit, kchunk;   // K split over ksplit CTAs of kchunk (a multiple of 16) each
  int64_t part;         // split: first partial tile of this product in the workspace
};

// Grouped form: one CTA per (descriptor, tile i, tile j) entry of a task list,
// so the GEMMs of every supernode of a level run in one launch.
struct GemmTile {
  int32_t desc, ti, tj, kc;   // product, output tile, K chunk
};

__device__ __forceinline__ void gen_gemm_tile(const GenGemm& g, int i0, int j0, int kc, double* __restrict__ part_ws,
                                              int64_t tile_idx) {
  constexpr int KC = 16;
  __shared__ double As[KC][kGTile + 1];
  __shared__ double Bs[KC][kGTile + 1];
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int kbeg = 0, kend = g.K;
  if (g.amode == 1) kend = min(kend, i0 + kGTile);
  if (g.bmode == 1) kbeg = (j0 / KC) * KC;
  if (g.ksplit > 1) {
    kbeg = max(kbeg, kc * g.kchunk);
    kend = min(kend, (kc + 1) * g.kchunk);
  }
  double acc[4][4] = {};
  // the thread -> element map of each operand follows its contiguous index
  const bool bkf = g.br == 1 && g.bc != 1;
  for (int k = kbeg; k < kend; k += KC) {
    // symmetric A: the chunk reads its stored transpose wholly above the diagonal
    const bool akf = g.amode == 2 ? (k >= i0 + kGTile ? g.ar == 1 : (g.ac == 1 && g.ar != 1))
                                  : (g.ac == 1 && g.ar != 1);
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + kGT * q;
      {
        const int kk = akf ? (idx & 15) : (idx >> 6), r = akf ? (idx >> 4) : (idx & 63);
        const int kg = k + kk, ia = i0 + r;
        double av = 0.0;
        if (kg < kend && ia < g.M) {
          if (g.amode == 0 || (g.amode == 1 && kg <= ia)) av = g.A[ia * g.ar + kg * g.ac];
          else if (g.amode == 2) av = kg <= ia ? g.A[ia * g.ar + kg * g.ac] : g.A[kg * g.ar + ia * g.ac];
        }
        As[kk][r] = av;
      }
      {
        const int kk = bkf ? (idx & 15) : (idx >> 6), r = bkf ? (idx >> 4) : (idx & 63);
        const int kg = k + kk, jb = j0 + r;
        double bv = 0.0;
        if (kg < kend && jb < g.N && (g.bmode == 0 || jb <= kg)) bv = g.B[kg * g.br + jb * g.bc];
        Bs[kk][r] = bv;
      }
    }
    __syncthreads();
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      double a[4], b[4];
#pragma unroll
      for (int i = 0; i < 4; ++i) a[i] = As[kk][ty + 16 * i];
#pragma unroll
      for (int j = 0; j < 4; ++j) b[j] = Bs[kk][tx + 16 * j];
#pragma unroll
      for (int i = 0; i < 4; ++i)
#pragma unroll
        for (int j = 0; j < 4; ++j) acc[i][j] = fma(a[i], b[j], acc[i][j]);
    }
    __syncthreads();
  }
  if (g.ksplit > 1) {
    // partial tile (row-major 64 x 64), summed by k_gen_reduce
    double* pp = part_ws + g.part + (tile_idx * g.ksplit + kc) * (kGTile * kGTile);
#pragma unroll
    for (int i = 0; i < 4; ++i)
#pragma unroll
      for (int j = 0; j < 4; ++j) pp[(ty + 16 * i) * kGTile + tx + 16 * j] = acc[i][j];
    return;
  }
#pragma unroll
  for (int i = 0; i < 4; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      const int r = i0 + ty + 16 * i, c = j0 + tx + 16 * j;
      if (r < g.M && c < g.N && (!g.lower_c || r >= c)) {
        double* p = g.C + r * g.cr + c * g.cc;
        *p = (g.beta == 0.0 ? 0.0 : g.beta * *p) + g.alpha * acc[i][j];
      }
    }
}

__global__ void __launch_bounds__(kGT, 3)
k_gen_gemm_grouped(const GenGemm* __restrict__ descs, const GemmTile* __restrict__ tiles,
                   double* __restrict__ part_ws) {
  const GemmTile t = tiles[blockIdx.x];
  const GenGemm g = descs[t.desc];
  const int64_t ntj = (g.N + kGTile - 1) / kGTile;
  gen_gemm_tile(g, t.ti * kGTile, t.tj * kGTile, t.kc, part_ws, t.ti * ntj + t.tj);
}

// Split products: C = beta C + alpha sum_kc partial(kc), the partials added in
// chunk order (deterministic); one CTA per output tile.
__global__ void __launch_bounds__(kGT)
k_gen_reduce(const GenGemm* __restrict__ descs, const GemmTile* __restrict__ tiles,
             const double* __restrict__ part_ws) {
  const GemmTile t = tiles[blockIdx.x];
  const GenGemm g = descs[t.desc];
  const int64_t ntj = (g.N + kGTile - 1) / kGTile;
  const double* pp = part_ws + g.part + (t.ti * ntj + t.tj) * g.ksplit * (kGTile * kGTile);
  for (int e = threadIdx.x; e < kGTile * kGTile; e += kGT) {
    const int r = t.ti * kGTile + e / kGTile, c = t.tj * kGTile + e % kGTile;
    if (r >= g.M || c >= g.N || (g.lower_c && r < c)) continue;
    double acc = 0.0;
    for (int kc = 0; kc < g.ksplit; ++kc) acc += pp[(int64_t)kc * (kGTile * kGTile) + e];
    double* p = g.C + r * g.cr + c * g.cc;
    *p = (g.beta == 0.0 ? 0.0 : g.beta * *p) + g.alpha * acc;
  }
}

struct InvTask {
  const double* src;
  int64_t lds;
  double* dst;
  int64_t ldt;
  int32_t kb, pad;
};

// Inverse of a kb x kb (kb <= 64) lower-triangular block (column-major,
// leading dimensions lds / ldt): thread j computes column j of the inverse by
// forward substitution on the unit vector e_j.
__device__ __forceinline__ void inv64_body(const double* __restrict__ Lsrc, int64_t lds, int kb,
                                           double* __restrict__ T, int64_t ldt) {
  __shared__ double Ls[64 * 65];
  for (int e = threadIdx.x; e < kb * kb; e += blockDim.x) {
    const int r = e % kb, c = e / kb;
    Ls[r + c * 65] = r >= c ? Lsrc[r + c * lds] : 0.0;
  }
  __syncthreads();
  const int j = threadIdx.x;
  if (j >= kb) return;
  double x[64];
#pragma unroll
  for (int i = 0; i < 64; ++i) x[i] = 0.0;
  for (int i = j; i < kb; ++i) {
    double s = (i == j) ? 1.0 : 0.0;
    for (int k = j; k < i; ++k) s -= Ls[i + k * 65] * x[k];
    x[i] = s / Ls[i + i * 65];
  }
  for (int i = 0; i < kb; ++i) T[i + j * ldt] = i >= j ? x[i] : 0.0;
}

__global__ void k_inv64_grouped(const InvTask* __restrict__ tasks) {
  const InvTask t = tasks[blockIdx.x];
  inv64_body(t.src, t.lds, t.kb, t.dst, t.ldt);
}

// One gather task: the part of pair (J, K) with J's off-diagonal rows
// u in [u0, u1) (at most kGatherRows of them).
struct LevelPair {
  int32_t J, K, c0, c1, u0, u1;
};
constexpr int kGatherRows = 512;
constexpr int kGatherUnroll = 4;

// Z_RR of every supernode J of a level (lower, column-major b x b, stored in the
// update workspace at U_J's place), gathered from the ancestors' Z panels. A
// task covers columns [c0, c1) of J's pair with K and a chunk of rows: it
// stages struct(K) in shared memory, finds the positions of its rows by binary
// search, then a warp per column copies 32 rows at a time, kGatherUnroll
// (column, row chunk) items in flight per warp. Tasks write disjoint entries.
__global__ void __launch_bounds__(kGT)
k_gather_zrr_level(const LevelPair* __restrict__ pairs, const SnodeDev* __restrict__ sn,
                   const int32_t* __restrict__ rows, const double* __restrict__ Z, double* __restrict__ U) {
  extern __shared__ int32_t gsm2[];
  const LevelPair pr = pairs[blockIdx.x];
  const SnodeDev dj = sn[pr.J];
  const SnodeDev dk = sn[pr.K];
  const int b = dj.len - dj.s;
  double* ZRR = U + dj.uoff;
  int32_t* sK = gsm2;
  int32_t* pos = gsm2 + dk.len;
  const int32_t* rk = rows + dk.roff;
  const int32_t* rj = rows + dj.roff + dj.s;
  for (int i = threadIdx.x; i < dk.len; i += blockDim.x) sK[i] = rk[i];
  __syncthreads();
  const int nu = pr.u1 - pr.u0;
  for (int i = threadIdx.x; i < nu; i += blockDim.x) {
    const int32_t key = rj[pr.u0 + i];
    int lo = 0, hi = dk.len;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sK[mid] < key) lo = mid + 1; else hi = mid;
    }
    pos[i] = lo;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = kGT / 32;
  const int nch = (nu + 31) >> 5, w = pr.c1 - pr.c0;
  const int items = w * nch;
  for (int i0 = warp; i0 < items; i0 += nw * kGatherUnroll) {
    double v[kGatherUnroll];
    int64_t dst[kGatherUnroll];
#pragma unroll
    for (int q = 0; q < kGatherUnroll; ++q) {
      const int i = i0 + q * nw;
      dst[q] = -1;
      if (i < items) {
        const int cc = i / nch;
        const int c = pr.c0 + cc;
        const int ui = (i - cc * nch) * 32 + lane;
        const int u = pr.u0 + ui;
        if (ui < nu && u >= c) {
          v[q] = Z[dk.loff + (int64_t)(rj[c] - dk.f) * dk.ld + pos[ui]];
          dst[q] = u + (int64_t)c * b;
        }
      }
    }
#pragma unroll
    for (int q = 0; q < kGatherUnroll; ++q)
      if (dst[q] >= 0) ZRR[dst[q]] = v[q];
  }
}

// g[t] = -(xbar_r . x_c + [r != c] xbar_c . x_r) + alpha (1 + [r != c]) Z(entry t)
__global__ void k_adj_grad(const int32_t* __restrict__ rowind, const int32_t* __restrict__ colidx,
                           const int64_t* __restrict__ amap, const double* __restrict__ Z, double alpha,
                           const double* __restrict__ Xb, const double* __restrict__ X, int n, int nrhs, int64_t nnz,
                           double* __restrict__ g) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < nnz; t += (int64_t)gridDim.x * blockDim.x) {
    const int r = rowind[t], c = colidx[t];
    double s = 0.0;
    for (int k = 0; k < nrhs; ++k) s = fma(Xb[r + (int64_t)k * n], X[c + (int64_t)k * n], s);
    if (r != c)
      for (int k = 0; k < nrhs; ++k) s = fma(Xb[c + (int64_t)k * n], X[r + (int64_t)k * n], s);
    double v = -s;
    if (Z) v += alpha * (r != c ? 2.0 : 1.0) * Z[amap[t]];
    g[t] = v;
  }
}

__global__ void k_take(const double* __restrict__ Z, const int64_t* __restrict__ map, int64_t m,
                       double* __restrict__ out) {
  for (int64_t t = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; t < m; t += (int64_t)gridDim.x * blockDim.x)
    out[t] = Z[map[t]];
}

inline unsigned grid1d(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g > 0 ? g : 1);
}

GenGemm mk(const double* A, int64_t ar, int64_t ac, const double* B, int64_t br, int64_t bc, double* C, int64_t cr,
           int64_t cc, int M, int N, int K, double alpha, double beta, int amode = 0, int bmode = 0, int lower = 0) {
  GenGemm g;
  g.A = A; g.ar = ar; g.ac = ac; g.B = B; g.br = br; g.bc = bc; g.C = C; g.cr = cr; g.cc = cc;
  g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.beta = beta; g.amode = amode; g.bmode = bmode; g.lower_c = lower;
  g.ksplit = 1; g.kchunk = K; g.part = 0;
  return g;
}

template <class T>
int upload_v(chol_handle* h, T** dst, const std::vector<T>& v) {
  if (v.empty()) { *dst = nullptr; return CHOL_OK; }
  int rc = chol_dalloc(h, (void**)dst, v.size() * sizeof(T));
  if (rc) return rc;
  CHOL_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice));
  return CHOL_OK;
}

int ensure_adjoint(chol_handle* h) {
  DeviceState* D = h->dev;
  if (D->Zp) return CHOL_OK;
  int rc;
  if ((rc = chol_dalloc(h, (void**)&D->Zp, sizeof(double) * (size_t)std::max<int64_t>(h->panel_doubles, 1)))) return rc;
  // column index of every stored entry of A (original ordering)
  std::vector<int32_t> colidx(h->nnz_a), rowidx(h->nnz_a);
  for (int32_t c = 0; c < h->n; ++c)
    for (int64_t t = h->a_colptr[c]; t < h->a_colptr[c + 1]; ++t) colidx[t] = c;
  if ((rc = upload_v(h, &D->a_col, colidx))) return rc;
  if ((rc = upload_v(h, &D->a_row, h->a_rowind))) return rc;
  return CHOL_OK;
}

// Level plan of the selected inverse (built once, on first use).
// Products launched together: their tiles (incl. K chunks) and, for the split
// ones, the output tiles of the reduction.
struct Group {
  int32_t tb = 0, tn = 0, rb = 0, rn = 0;
  double flops = 0.0;
};
struct SiStep {
  int32_t inv_b, inv_n;
  Group g1, g2;
  double flops;                         // algorithmic flops of the step
};
struct SiLevel {
  int64_t t_doubles;                    // T workspace of the level (zeroed first)
  std::vector<SiStep> steps;            // the L_JJ^{-1} recurrence, batched
  Group uh, zrj, zjj1, zjj2;
  int32_t pair_b, pair_n;
  double gemm_flops;                    // Uhat, Z_RJ and Z_JJ products
};

// Algorithmic flops of a descriptor: 2 M N K, halved for a triangular operand
// and for a triangular output.
double gemm_flops(const GenGemm& g) {
  double f = 2.0 * g.M * (double)g.N * g.K;
  if (g.amode == 1 || g.bmode == 1) f *= 0.5;
  if (g.lower_c) f *= 0.5;
  return f;
}

struct SiPlan {
  std::vector<SiLevel> levels;
  std::vector<GenGemm> descs;
  std::vector<GemmTile> tiles, rtiles;
  std::vector<InvTask> invs;
  std::vector<LevelPair> pairs;
  int64_t part_max = 0;                 // partial-tile workspace (doubles)
  GenGemm* d_descs = nullptr;
  GemmTile* d_tiles = nullptr;
  GemmTile* d_rtiles = nullptr;
  InvTask* d_invs = nullptr;
  LevelPair* d_pairs = nullptr;
  double* d_part = nullptr;
};

// Emit the tiles of products launched together. Products with K > 256 may be
// split over K chunks (of at least 128): each chunk writes a partial tile to
// the workspace and a second launch adds them in chunk order. The split factor
// is chosen per group for the fill of whole waves of resident CTAs (tiles of
// unequal cost counted alike): a small group is spread over the SMs, and a
// group of, say, 384 tiles on 456 CTA slots, which would leave some SMs idle
// for a third of the launch, becomes 7 x 384 = 5.9 waves. Only groups below
// two waves are split, and a split must gain at least 8% of fill to pay for
// its partial tiles.
constexpr int kGenCtasPerSm = 3;   // __launch_bounds__ of k_gen_gemm_grouped
Group emit_group(SiPlan& pl, const std::vector<GenGemm>& gs, int sms) {
  Group gr;
  gr.tb = (int32_t)pl.tiles.size();
  gr.rb = (int32_t)pl.rtiles.size();
  auto out_tiles = [](const GenGemm& g) {
    int64_t n = 0;
    for (int ti = 0; ti * kGTile < g.M; ++ti)
      for (int tj = 0; tj * kGTile < g.N; ++tj)
        if (!g.lower_c || ti * kGTile + kGTile - 1 >= tj * kGTile) ++n;
    return n;
  };
  const int64_t slots = (int64_t)kGenCtasPerSm * sms;
  auto split_of = [](const GenGemm& g, int ks) {
    return g.K > 256 ? (int)std::min<int64_t>(ks, (g.K + 127) / 128) : 1;
  };
  auto fill = [&](int ks) {
    int64_t t = 0;
    for (const GenGemm& g : gs)
      if (g.M > 0 && g.N > 0) t += out_tiles(g) * split_of(g, ks);
    return t == 0 ? 1.0 : (double)t / ((double)((t + slots - 1) / slots) * (double)slots);
  };
  int64_t nt = 0;
  for (const GenGemm& g : gs)
    if (g.M > 0 && g.N > 0) nt += out_tiles(g);
  int ksel = 1;
  double best = fill(1);
  const double base = best;
  // from two waves on, tiles of unequal cost already even out the tail
  for (int ks = 2; ks <= 32 && nt < 2 * slots; ++ks) {
    const double f = fill(ks);
    if (f > best + 0.02) { best = f; ksel = ks; }
  }
  if (best < base + 0.08) ksel = 1;
  int64_t part = 0;
  for (GenGemm g : gs) {
    if (g.M <= 0 || g.N <= 0) continue;
    gr.flops += gemm_flops(g);
    int ks = split_of(g, ksel);
    if (ks > 1) {
      g.kchunk = (((g.K + ks - 1) / ks) + 15) / 16 * 16;
      ks = (g.K + g.kchunk - 1) / g.kchunk;
    }
    g.ksplit = ks;
    if (ks == 1) g.kchunk = g.K;
    g.part = part;
    const int32_t d = (int32_t)pl.descs.size();
    pl.descs.push_back(g);
    const int ntj = (g.N + kGTile - 1) / kGTile;
    for (int ti = 0; ti * kGTile < g.M; ++ti)
      for (int tj = 0; tj < ntj; ++tj) {
        if (g.lower_c && ti * kGTile + kGTile - 1 < tj * kGTile) continue;
        for (int kc = 0; kc < ks; ++kc) pl.tiles.push_back({d, ti, tj, kc});
        if (ks > 1) pl.rtiles.push_back({d, ti, tj, 0});
      }
    if (ks > 1) part += (int64_t)((g.M + kGTile - 1) / kGTile) * ntj * ks * kGTile * kGTile;
  }
  gr.tn = (int32_t)pl.tiles.size() - gr.tb;
  gr.rn = (int32_t)pl.rtiles.size() - gr.rb;
  pl.part_max = std::max(pl.part_max, part);
  return gr;
}

int build_si_plan(chol_handle* h) {
  DeviceState* D = h->dev;
  if (D->si_plan) return CHOL_OK;
  SiPlan* pl = new SiPlan();
  const double* L = D->L;
  // Z_RR of a level lives in the update workspace, at U_J's place; an RLB
  // handle has none, so it gets its own
  if (h->update_doubles < h->update_doubles_rl && !D->zrr_ws) {
    const int rz = chol_dalloc(h, (void**)&D->zrr_ws, sizeof(double) * (size_t)h->update_doubles_rl);
    if (rz) { delete pl; return rz; }
  }
  double* ZRR = D->zrr_ws ? D->zrr_ws : D->U;
  double* Z = D->Zp;
  int64_t tmax = 0, hmax = 0, wmax = 0;
  // per-level offsets of T (s^2), Uhat (b s) and W (s^2 / 2)
  std::vector<int64_t> toff(h->ns), hoff(h->ns), woff(h->ns);
  for (const LevelPlan& P : h->levels) {
    int64_t t = 0, u = 0, w = 0;
    for (int32_t q = 0; q < P.snode_n; ++q) {
      const int32_t J = h->level_snodes[P.snode_b + q];
      const SnodeDev& d = h->snodes[J];
      toff[J] = t; hoff[J] = u; woff[J] = w;
      t += (int64_t)d.s * d.s;
      u += (int64_t)(d.len - d.s) * d.s;
      w += ((int64_t)d.s * d.s + 1) / 2;   // B A^{-1} of one doubling step: at most s^2 / 2
    }
    tmax = std::max(tmax, t); hmax = std::max(hmax, u); wmax = std::max(wmax, w);
  }
  int rc;
  if ((rc = chol_dalloc(h, (void**)&D->Tw, sizeof(double) * (size_t)std::max<int64_t>(tmax, 1)))) return rc;
  if ((rc = chol_dalloc(h, (void**)&D->Uh, sizeof(double) * (size_t)std::max<int64_t>(hmax, 1)))) return rc;
  if ((rc = chol_dalloc(h, (void**)&D->Ww, sizeof(double) * (size_t)std::max<int64_t>(wmax, 1)))) return rc;
  std::vector<std::vector<int64_t>> pairs_of(h->ns);
  for (size_t p = 0; p < h->rel_J.size(); ++p) pairs_of[h->rel_J[p]].push_back((int64_t)p);
  for (int lv = h->nlevels - 1; lv >= 0; --lv) {
    const LevelPlan& P = h->levels[lv];
    SiLevel sl{};
    std::vector<int32_t> Js(h->level_snodes.begin() + P.snode_b, h->level_snodes.begin() + P.snode_b + P.snode_n);
    int maxnbk = 0;
    int64_t tl = 0;
    for (int32_t J : Js) {
      maxnbk = std::max(maxnbk, (h->snodes[J].s + 63) / 64);
      tl += (int64_t)h->snodes[J].s * h->snodes[J].s;
    }
    sl.t_doubles = tl;
    // T = L_JJ^{-1} by recursive doubling: first every 64 x 64 diagonal block
    // is inverted (all at once), then blocks of size bs = 64, 128, ... are
    // combined pairwise, [A 0; B C]^{-1} = [A^{-1} 0; -C^{-1} B A^{-1} C^{-1}],
    // W = B A^{-1} then the off-diagonal block = -C^{-1} W, every pair of every
    // supernode of the level in one launch per product
    {
      SiStep st{};
      st.inv_b = (int32_t)pl->invs.size();
      for (int32_t J : Js) {
        const SnodeDev& d = h->snodes[J];
        double* T = D->Tw + toff[J];
        for (int k0 = 0; k0 < d.s; k0 += 64) {
          const int kb = std::min(64, d.s - k0);
          pl->invs.push_back({L + d.loff + k0 + (int64_t)k0 * d.ld, d.ld, T + k0 + (int64_t)k0 * d.s, d.s, kb, 0});
          st.flops += (double)kb * kb * kb / 3.0;
        }
      }
      st.inv_n = (int32_t)pl->invs.size() - st.inv_b;
      sl.steps.push_back(st);
    }
    for (int bs = 64; bs < maxnbk * 64; bs *= 2) {
      SiStep st{};
      st.inv_b = (int32_t)pl->invs.size();
      std::vector<GenGemm> g1s, g2s;
      for (int32_t J : Js) {
        const SnodeDev& d = h->snodes[J];
        double* T = D->Tw + toff[J];
        double* Wp = D->Ww + woff[J];
        for (int i0 = 0; i0 + bs < d.s; i0 += 2 * bs) {
          const int c0 = i0 + bs, mc = std::min(c0 + bs, d.s) - c0;
          g1s.push_back(mk(L + d.loff + c0 + (int64_t)i0 * d.ld, 1, d.ld, T + i0 + (int64_t)i0 * d.s, 1, d.s, Wp, 1, mc,
                           mc, bs, bs, 1.0, 0.0, 0, 1, 0));
          g2s.push_back(mk(T + c0 + (int64_t)c0 * d.s, 1, d.s, Wp, 1, mc, T + c0 + (int64_t)i0 * d.s, 1, d.s, mc, bs, mc,
                           -1.0, 0.0, 1, 0, 0));
          Wp += (int64_t)mc * bs;
        }
      }
      st.g1 = emit_group(*pl, g1s, D->sms);
      st.g2 = emit_group(*pl, g2s, D->sms);
      st.flops = st.g1.flops + st.g2.flops;
      sl.steps.push_back(st);
    }
    // Uhat = L_RJ T
    std::vector<GenGemm> gs;
    for (int32_t J : Js) {
      const SnodeDev& d = h->snodes[J];
      const int b = d.len - d.s;
      if (b > 0)
        gs.push_back(mk(L + d.loff + d.s, 1, d.ld, D->Tw + toff[J], 1, d.s, D->Uh + hoff[J], 1, b, b, d.s, d.s, 1.0,
                        0.0, 0, 1, 0));
    }
    sl.uh = emit_group(*pl, gs, D->sms);
    // Z_RR gather pairs
    sl.pair_b = (int32_t)pl->pairs.size();
    for (int32_t J : Js)
      for (int64_t p : pairs_of[J]) {
        const SnodeDev& d = h->snodes[J];
        const int32_t b = d.len - d.s;
        // rows u >= c0 of J are the ones in K (and later ancestors' rows are
        // in struct(K) too); chunks of kGatherRows
        for (int32_t u0 = h->rel_c0[p]; u0 < b; u0 += kGatherRows)
          pl->pairs.push_back({J, h->rel_K[p], h->rel_c0[p], h->rel_c1[p], u0, std::min(b, u0 + kGatherRows)});
      }
    sl.pair_n = (int32_t)pl->pairs.size() - sl.pair_b;
    // Z_RJ = -Z_RR Uhat  (Z_RR at U_J's place in the update workspace)
    gs.clear();
    for (int32_t J : Js) {
      const SnodeDev& d = h->snodes[J];
      const int b = d.len - d.s;
      if (b > 0)
        gs.push_back(mk(ZRR + d.uoff, 1, b, D->Uh + hoff[J], 1, b, Z + d.loff + d.s, 1, d.ld, b, d.s, b, -1.0, 0.0, 2,
                        0, 0));
    }
    sl.zrj = emit_group(*pl, gs, D->sms);
    // Z_JJ = T^T T, then -= Uhat^T Z_RJ
    gs.clear();
    for (int32_t J : Js) {
      const SnodeDev& d = h->snodes[J];
      double* T = D->Tw + toff[J];
      gs.push_back(mk(T, d.s, 1, T, 1, d.s, Z + d.loff, 1, d.ld, d.s, d.s, d.s, 1.0, 0.0, 0, 0, 1));
    }
    sl.zjj1 = emit_group(*pl, gs, D->sms);
    gs.clear();
    for (int32_t J : Js) {
      const SnodeDev& d = h->snodes[J];
      const int b = d.len - d.s;
      if (b > 0)
        gs.push_back(mk(D->Uh + hoff[J], b, 1, Z + d.loff + d.s, 1, d.ld, Z + d.loff, 1, d.ld, d.s, d.s, b, -1.0, 1.0, 0,
                        0, 1));
    }
    sl.zjj2 = emit_group(*pl, gs, D->sms);
    sl.gemm_flops = sl.uh.flops + sl.zrj.flops + sl.zjj1.flops + sl.zjj2.flops;
    pl->levels.push_back(std::move(sl));
  }
  auto up = [&](auto** dst, const auto& v) -> int {
    if (v.empty()) return CHOL_OK;
    int r = chol_dalloc(h, (void**)dst, v.size() * sizeof(v[0]));
    if (r) return r;
    CHOL_CUDA_TRY(cudaMemcpy(*dst, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice));
    return CHOL_OK;
  };
  if ((rc = up(&pl->d_descs, pl->descs))) return rc;
  if ((rc = up(&pl->d_tiles, pl->tiles))) return rc;
  if ((rc = up(&pl->d_rtiles, pl->rtiles))) return rc;
  if (pl->part_max > 0 && (rc = chol_dalloc(h, (void**)&pl->d_part, sizeof(double) * (size_t)pl->part_max))) return rc;
  if ((rc = up(&pl->d_invs, pl->invs))) return rc;
  if ((rc = up(&pl->d_pairs, pl->pairs))) return rc;
  D->si_plan = pl;
  CHOL_CUDA_TRY(cudaFuncSetAttribute(k_gather_zrr_level, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  return CHOL_OK;
}

// Selected inverse into D->Zp (once per factorization), level by level from the
// root, every supernode of a level at once.
int selinv(chol_handle* h, cudaStream_t st) {
  if (h->selinv_valid) return CHOL_OK;
  // the Z_RR gather stages struct(K) and the positions in shared memory
  if ((int64_t)(h->max_len + kGatherRows) * (int64_t)sizeof(int32_t) > 200 * 1024) return CHOL_ENOTSUP;
  int rc = ensure_adjoint(h);
  if (rc) return rc;
  if ((rc = build_si_plan(h))) return rc;
  DeviceState* D = h->dev;
  SiPlan* pl = (SiPlan*)D->si_plan;
  auto launch = [&](const Group& gr) {
    if (gr.tn > 0) k_gen_gemm_grouped<<<gr.tn, kGT, 0, st>>>(pl->d_descs, pl->d_tiles + gr.tb, pl->d_part);
    if (gr.rn > 0) k_gen_reduce<<<gr.rn, kGT, 0, st>>>(pl->d_descs, pl->d_rtiles + gr.rb, pl->d_part);
  };
  auto nl = [](const Group& gr) { return (gr.tn > 0) + (gr.rn > 0); };
  for (const SiLevel& sl : pl->levels) {
    CHOL_CUDA_TRY(cudaMemsetAsync(D->Tw, 0, sizeof(double) * (size_t)sl.t_doubles, st));
    for (const SiStep& q : sl.steps) {
      KScope ks(h, CHOL_K_SELINV_INV, st, q.flops, 0.0);
      ks.launches((q.inv_n > 0) + nl(q.g1) + nl(q.g2));
      if (q.inv_n > 0) k_inv64_grouped<<<q.inv_n, 64, 0, st>>>(pl->d_invs + q.inv_b);
      launch(q.g1);
      launch(q.g2);
    }
    if (sl.pair_n > 0) {
      KScope ks(h, CHOL_K_SELINV_GATHER, st, 0.0, 0.0);
      k_gather_zrr_level<<<sl.pair_n, kGT, sizeof(int32_t) * (h->max_len + kGatherRows), st>>>(pl->d_pairs + sl.pair_b, D->sn,
                                                                                   D->rows, D->Zp, D->zrr_ws ? D->zrr_ws : D->U);
    }
    {
      KScope ks(h, CHOL_K_SELINV_GEMM, st, sl.gemm_flops, 0.0);
      ks.launches(nl(sl.uh) + nl(sl.zrj) + nl(sl.zjj1) + nl(sl.zjj2));
      launch(sl.uh);
      launch(sl.zrj);
      launch(sl.zjj1);
      launch(sl.zjj2);
    }
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  h->selinv_valid = true;
  return CHOL_OK;
}

}  // namespace

void chol_adjoint_free(chol_handle* h) {
  DeviceState* D = h->dev;
  if (!D || !D->si_plan) return;
  SiPlan* pl = (SiPlan*)D->si_plan;
  void* ptrs[] = {pl->d_descs, pl->d_tiles, pl->d_rtiles, pl->d_invs, pl->d_pairs, pl->d_part};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  delete pl;
  D->si_plan = nullptr;
}

extern "C" int chol_selected_inverse(chol_handle* h, double* zvals, void* stream) {
  NvtxRange nvtx_range("chol_selected_inverse");
  if (!h) return -1;
  if (!zvals && h->nnz_a > 0) return -2;
  if (int rc_state = chol_factored_here(h)) return rc_state;
  if (h->opt.precision != CHOL_PREC_FP64) return CHOL_ENOTSUP;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = selinv(h, st);
  if (rc) return rc;
  DeviceState* D = h->dev;
  if (h->nnz_a > 0) k_take<<<grid1d(h->nnz_a, 256), 256, 0, st>>>(D->Zp, D->amap, h->nnz_a, zvals);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

extern "C" int chol_adjoint(chol_handle* h, const double* w, const double* x, int32_t nrhs, double logdet_weight,
                            double* bbar, double* grad, void* stream) {
  NvtxRange nvtx_range("chol_adjoint");
  if (!h) return -1;
  if (!w && nrhs > 0) return -2;
  if (!x && nrhs > 0) return -3;
  if (nrhs < 0) return -4;
  if (!grad && h->nnz_a > 0) return -7;
  if (int rc_state = chol_factored_here(h)) return rc_state;
  if (h->opt.precision != CHOL_PREC_FP64) return CHOL_ENOTSUP;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_adjoint(h);
  if (rc) return rc;
  DeviceState* D = h->dev;
  double* xb = bbar;
  if (nrhs > 0) {
    if (!xb) {
      if (D->adj_cap < nrhs) {
        if (D->adj_xb) cudaFree(D->adj_xb);
        D->adj_xb = nullptr;
        if ((rc = chol_dalloc(h, (void**)&D->adj_xb, sizeof(double) * (size_t)h->n * nrhs))) return rc;
        D->adj_cap = nrhs;
      }
      xb = D->adj_xb;
    }
    // Xbar = A^{-1} W
    CHOL_CUDA_TRY(cudaMemcpyAsync(xb, w, sizeof(double) * (size_t)h->n * nrhs, cudaMemcpyDeviceToDevice, st));
    if ((rc = chol_solve(h, xb, nrhs, (void*)st))) return rc;
  }
  if (logdet_weight != 0.0 && (rc = selinv(h, st))) return rc;
  if (h->nnz_a > 0) {
    KScope ks(h, CHOL_K_ADJOINT, st, 4.0 * nrhs * (double)h->nnz_a, 0.0);
    k_adj_grad<<<grid1d(h->nnz_a, 256), 256, 0, st>>>(D->a_row, D->a_col, D->amap,
                                                      logdet_weight != 0.0 ? D->Zp : nullptr, logdet_weight, xb, x,
                                                      h->n, nrhs, h->nnz_a, grad);
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}
