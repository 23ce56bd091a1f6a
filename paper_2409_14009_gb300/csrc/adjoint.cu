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
};

__global__ void __launch_bounds__(kGT) k_gen_gemm(GenGemm g) {
  constexpr int KC = 16;
  __shared__ double As[KC][kGTile + 1];
  __shared__ double Bs[KC][kGTile + 1];
  const int i0 = blockIdx.x * kGTile, j0 = blockIdx.y * kGTile;
  if (g.lower_c && i0 + kGTile - 1 < j0) return;
  const int tid = threadIdx.x, tx = tid & 15, ty = tid >> 4;
  int kbeg = 0, kend = g.K;
  if (g.amode == 1) kend = min(kend, i0 + kGTile);          // A(i,k) = 0 for k > i
  if (g.bmode == 1) kbeg = (j0 / KC) * KC;                   // B(k,j) = 0 for k < j
  double acc[4][4] = {};
  for (int k = kbeg; k < kend; k += KC) {
#pragma unroll
    for (int q = 0; q < 4; ++q) {
      const int idx = tid + kGT * q;
      const int kk = idx >> 6, r = idx & 63;
      const int kg = k + kk;
      const int ia = i0 + r, jb = j0 + r;
      double av = 0.0, bv = 0.0;
      if (kg < g.K && ia < g.M) {
        if (g.amode == 0 || (g.amode == 1 && kg <= ia)) av = g.A[ia * g.ar + kg * g.ac];
        else if (g.amode == 2) av = kg <= ia ? g.A[ia * g.ar + kg * g.ac] : g.A[kg * g.ar + ia * g.ac];
      }
      if (kg < g.K && jb < g.N && (g.bmode == 0 || jb <= kg)) bv = g.B[kg * g.br + jb * g.bc];
      As[kk][r] = av;
      Bs[kk][r] = bv;
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

// Inverse of a kb x kb (kb <= 64) lower-triangular block (column-major,
// leading dimensions lds / ldt): thread j computes column j of the inverse by
// forward substitution on the unit vector e_j.
__global__ void k_inv64(const double* __restrict__ Lsrc, int64_t lds, int kb, double* __restrict__ T, int64_t ldt) {
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

// Z_RR of supernode J (lower, column-major b x b) gathered from the ancestors'
// Z panels: one block per (J, K) pair, positions of J's rows in struct(K) found
// by binary search in shared memory.
struct PairDev {
  int32_t K, c0, c1, pad;
};

__global__ void __launch_bounds__(kGT)
k_gather_zrr(const PairDev* __restrict__ pairs, SnodeDev dj, const SnodeDev* __restrict__ sn,
             const int32_t* __restrict__ rows, const double* __restrict__ Z, double* __restrict__ ZRR) {
  extern __shared__ int32_t gsm[];
  const PairDev pr = pairs[blockIdx.x];
  const SnodeDev dk = sn[pr.K];
  const int b = dj.len - dj.s;
  int32_t* sK = gsm;
  int32_t* pos = gsm + dk.len;
  const int32_t* rk = rows + dk.roff;
  const int32_t* rj = rows + dj.roff + dj.s;
  for (int i = threadIdx.x; i < dk.len; i += blockDim.x) sK[i] = rk[i];
  __syncthreads();
  for (int u = pr.c0 + threadIdx.x; u < b; u += blockDim.x) {
    const int32_t key = rj[u];
    int lo = 0, hi = dk.len;
    while (lo < hi) {
      const int mid = (lo + hi) >> 1;
      if (sK[mid] < key) lo = mid + 1; else hi = mid;
    }
    pos[u - pr.c0] = lo;
  }
  __syncthreads();
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  for (int c = pr.c0 + warp; c < pr.c1; c += kGT / 32) {
    const double* Zc = Z + dk.loff + (int64_t)(rj[c] - dk.f) * dk.ld;
    for (int u = c + lane; u < b; u += 32) ZRR[u + (int64_t)c * b] = Zc[pos[u - pr.c0]];
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

void gemm(cudaStream_t st, const GenGemm& g) {
  if (g.M <= 0 || g.N <= 0) return;
  dim3 grid((g.M + kGTile - 1) / kGTile, (g.N + kGTile - 1) / kGTile);
  k_gen_gemm<<<grid, kGT, 0, st>>>(g);
}

GenGemm mk(const double* A, int64_t ar, int64_t ac, const double* B, int64_t br, int64_t bc, double* C, int64_t cr,
           int64_t cc, int M, int N, int K, double alpha, double beta, int amode = 0, int bmode = 0, int lower = 0) {
  GenGemm g;
  g.A = A; g.ar = ar; g.ac = ac; g.B = B; g.br = br; g.bc = bc; g.C = C; g.cr = cr; g.cc = cc;
  g.M = M; g.N = N; g.K = K; g.alpha = alpha; g.beta = beta; g.amode = amode; g.bmode = bmode; g.lower_c = lower;
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
  int32_t maxs = 0, maxb = 0;
  for (const SnodeDev& d : h->snodes) {
    maxs = std::max(maxs, d.s);
    maxb = std::max(maxb, d.len - d.s);
  }
  const size_t ms = std::max(maxs, 1), mb = std::max(maxb, 1);
  if ((rc = chol_dalloc(h, (void**)&D->Zp, sizeof(double) * (size_t)std::max<int64_t>(h->panel_doubles, 1)))) return rc;
  if ((rc = chol_dalloc(h, (void**)&D->Tw, sizeof(double) * ms * ms))) return rc;
  if ((rc = chol_dalloc(h, (void**)&D->Ww, sizeof(double) * ms * 64))) return rc;
  if ((rc = chol_dalloc(h, (void**)&D->Uh, sizeof(double) * mb * ms))) return rc;
  if ((rc = chol_dalloc(h, (void**)&D->Zrr, sizeof(double) * mb * mb))) return rc;
  std::vector<PairDev> pairs(h->rel_J.size());
  for (size_t p = 0; p < pairs.size(); ++p) pairs[p] = {h->rel_K[p], h->rel_c0[p], h->rel_c1[p], 0};
  if ((rc = upload_v(h, (PairDev**)&D->pairs, pairs))) return rc;
  h->pair_begin.assign(h->ns + 1, 0);
  for (size_t p = 0; p < h->rel_J.size(); ++p) h->pair_begin[h->rel_J[p] + 1]++;
  for (int32_t J = 0; J < h->ns; ++J) h->pair_begin[J + 1] += h->pair_begin[J];
  // column index of every stored entry of A (original ordering)
  std::vector<int32_t> colidx(h->nnz_a), rowidx(h->nnz_a);
  for (int32_t c = 0; c < h->n; ++c)
    for (int64_t t = h->a_colptr[c]; t < h->a_colptr[c + 1]; ++t) colidx[t] = c;
  if ((rc = upload_v(h, &D->a_col, colidx))) return rc;
  if ((rc = upload_v(h, &D->a_row, h->a_rowind))) return rc;
  CHOL_CUDA_TRY(cudaFuncSetAttribute(k_gather_zrr, cudaFuncAttributeMaxDynamicSharedMemorySize, 200 * 1024));
  return CHOL_OK;
}

// Selected inverse into D->Zp (once per factorization).
int selinv(chol_handle* h, cudaStream_t st) {
  if (h->selinv_valid) return CHOL_OK;
  int rc = ensure_adjoint(h);
  if (rc) return rc;
  DeviceState* D = h->dev;
  const double* L = D->L;
  double* Z = D->Zp;
  const PairDev* pairs = (const PairDev*)D->pairs;
  for (int32_t J = h->ns - 1; J >= 0; --J) {
    const SnodeDev& d = h->snodes[J];
    const int s = d.s, b = d.len - d.s;
    const int64_t ld = d.ld;
    const double* Lp = L + d.loff;
    double* Zp = Z + d.loff;
    double* T = D->Tw;
    CHOL_CUDA_TRY(cudaMemsetAsync(T, 0, sizeof(double) * (size_t)s * s, st));
    // T = L_JJ^{-1}, block columns right to left:
    // T_kk = inv(L_kk), T_{>k,k} = -T_{>k,>k} L_{>k,k} T_kk
    const int nbk = (s + 63) / 64;
    for (int k = nbk - 1; k >= 0; --k) {
      const int k0 = 64 * k, kb = std::min(64, s - k0);
      k_inv64<<<1, 64, 0, st>>>(Lp + k0 + k0 * ld, ld, kb, T + k0 + (int64_t)k0 * s, s);
      const int m = s - (k0 + kb);
      if (m > 0) {
        gemm(st, mk(T + (k0 + kb) + (int64_t)(k0 + kb) * s, 1, s, Lp + (k0 + kb) + (int64_t)k0 * ld, 1, ld, D->Ww, 1, m,
                    m, kb, m, 1.0, 0.0, 1, 0, 0));
        gemm(st, mk(D->Ww, 1, m, T + k0 + (int64_t)k0 * s, 1, s, T + (k0 + kb) + (int64_t)k0 * s, 1, s, m, kb, kb, -1.0,
                    0.0, 0, 1, 0));
      }
    }
    if (b > 0) {
      // Uhat = L_RJ T   (b x s)
      gemm(st, mk(Lp + s, 1, ld, T, 1, s, D->Uh, 1, b, b, s, s, 1.0, 0.0, 0, 1, 0));
      // Z_RR from the ancestors
      const int np = h->pair_begin[J + 1] - h->pair_begin[J];
      if (np > 0)
        k_gather_zrr<<<np, kGT, sizeof(int32_t) * 2 * h->max_len, st>>>(pairs + h->pair_begin[J], d, D->sn, D->rows, Z,
                                                                         D->Zrr);
      // Z_RJ = -Z_RR Uhat
      gemm(st, mk(D->Zrr, 1, b, D->Uh, 1, b, Zp + s, 1, ld, b, s, b, -1.0, 0.0, 2, 0, 0));
    }
    // Z_JJ = T^T T - Uhat^T Z_RJ  (lower)
    gemm(st, mk(T, s, 1, T, 1, s, Zp, 1, ld, s, s, s, 1.0, 0.0, 0, 0, 1));
    if (b > 0) gemm(st, mk(D->Uh, b, 1, Zp + s, 1, ld, Zp, 1, ld, s, s, b, -1.0, 1.0, 0, 0, 1));
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  h->selinv_valid = true;
  return CHOL_OK;
}

}  // namespace

extern "C" int chol_selected_inverse(chol_handle* h, double* zvals, void* stream) {
  if (!h) return -1;
  if (!zvals && h->nnz_a > 0) return -2;
  if (!h->factored) return CHOL_ESTATE;
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
  if (!h) return -1;
  if (!w && nrhs > 0) return -2;
  if (!x && nrhs > 0) return -3;
  if (nrhs < 0) return -4;
  if (!grad && h->nnz_a > 0) return -7;
  if (!h->factored) return CHOL_ESTATE;
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
  if (h->nnz_a > 0)
    k_adj_grad<<<grid1d(h->nnz_a, 256), 256, 0, st>>>(D->a_row, D->a_col, D->amap,
                                                      logdet_weight != 0.0 ? D->Zp : nullptr, logdet_weight, xb, x,
                                                      h->n, nrhs, h->nnz_a, grad);
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}
