// solve.cu -- forward and backward substitution with the supernodal factor.
//
// X = P^T L^{-T} L^{-1} P B (the triangular factors give the solution, Sec. I).
// Forward, levels leaves->root: per column block k of each supernode J,
//   y_k <- L_kk^{-1} y_k                                  (k_fwd_diag)
//   y_i -= L_ik y_k for rows i of J below the block; rows of the off-diagonal
//   panel accumulate w_J = L_RJ y_J instead             (k_fwd_update)
// then w_J is scatter-subtracted into the ancestors' rows of y through the same
// pull-ordered task lists as the factor's relind assembly  (k_fwd_assemble).
// Backward, levels root->leaves:
//   y_J -= L_RJ^T x_R (gather of already-final ancestor rows)   (k_bwd_panel)
//   per column block k, last to first: x_k <- L_kk^{-T} y_k      (k_bwd_diag)
//   and y_c -= L_kc^T x_k for the column blocks c left of k       (k_bwd_update)
// Every output entry is written by exactly one thread per launch; reductions
// run in a fixed order, so the solve is deterministic.
#include <mutex>

#include "device.h"
#include "mixed.h"

namespace {

constexpr int kSolveThreads = 256;

__global__ void k_permute_in(const double* __restrict__ B, const int32_t* __restrict__ perm, int n,
                             int64_t ldb, int nrhs, double* __restrict__ Y) {
  const int64_t tot = (int64_t)n * nrhs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), i = (int)(q % n);
    Y[q] = B[perm[i] + r * ldb];
  }
}

__global__ void k_permute_out(const double* __restrict__ Y, const int32_t* __restrict__ perm, int n,
                              int64_t ldb, int nrhs, double* __restrict__ B) {
  const int64_t tot = (int64_t)n * nrhs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), i = (int)(q % n);
    B[perm[i] + r * ldb] = Y[q];
  }
}

// Triangular solve with the kb x kb (kb <= 64) diagonal block at step k0, in
// place in Y, for up to 16 right-hand sides. Sixteen lanes share a right-hand
// side, lane q holding rows q + 16a; the solved entry is broadcast inside the
// 16-lane group with a shuffle (no barriers in the substitution loop).
template <bool TRANS>
__global__ void __launch_bounds__(kSolveThreads)
k_diag(const SnodeDev* __restrict__ sn, const int32_t* __restrict__ list, int k0, int nb,
       const double* __restrict__ L, double* __restrict__ Y, int n, int nrhs) {
  __shared__ double Lk[64 * 65];
  __shared__ double inv[64];
  const SnodeDev d = sn[list[blockIdx.x]];
  const int kb = min(nb, d.s - k0);
  const double* G = L + d.loff + k0 + (int64_t)k0 * d.ld;
  for (int q = threadIdx.x; q < kb * kb; q += blockDim.x) {
    const int r = q % kb, c = q / kb;
    Lk[r + c * 65] = G[r + (int64_t)c * d.ld];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < kb; c += blockDim.x) inv[c] = 1.0 / Lk[c + c * 65];
  __syncthreads();
  const int rr = threadIdx.x >> 4, q = threadIdx.x & 15;
  const bool live = rr < nrhs;
  double* Yb = Y + d.f + k0 + (int64_t)rr * n;
  double y[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = q + 16 * a;
    y[a] = (live && i < kb) ? Yb[i] : 0.0;
  }
  if (!TRANS) {
#pragma unroll
    for (int ka = 0; ka < 4; ++ka) {
#pragma unroll
      for (int kq = 0; kq < 16; ++kq) {
        const int k = ka * 16 + kq;
        if (k < kb) {
          const double yk = __shfl_sync(0xffffffffu, y[ka] * inv[k], kq, 16);
          if (q == kq) y[ka] = yk;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = q + 16 * a;
            if (i > k && i < kb) y[a] -= Lk[i + k * 65] * yk;
          }
        }
      }
    }
  } else {
#pragma unroll
    for (int ka = 3; ka >= 0; --ka) {
#pragma unroll
      for (int kq = 15; kq >= 0; --kq) {
        const int k = ka * 16 + kq;
        if (k < kb) {
          const double yk = __shfl_sync(0xffffffffu, y[ka] * inv[k], kq, 16);
          if (q == kq) y[ka] = yk;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = q + 16 * a;
            if (i < k) y[a] -= Lk[k + i * 65] * yk;
          }
        }
      }
    }
  }
  if (live) {
#pragma unroll
    for (int a = 0; a < 4; ++a) {
      const int i = q + 16 * a;
      if (i < kb) Yb[i] = y[a];
    }
  }
}

// Forward update below the diagonal block of step k0, rows [r0, r0+64):
// acc = L[rows, k0:k0+kb] y_k; rows < s update y, rows >= s build w_J.
__global__ void __launch_bounds__(kSolveThreads)
k_fwd_update(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, int nb,
             const double* __restrict__ L, double* __restrict__ Y, int n, double* __restrict__ W,
             int nrhs) {
  __shared__ double yk[64 * kSolveChunk];
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int kb = min(nb, d.s - t.k0);
  for (int q = threadIdx.x; q < kb * nrhs; q += blockDim.x) {
    const int r = q % kb, c = q / kb;
    yk[q] = Y[d.f + t.k0 + r + (int64_t)c * n];
  }
  __syncthreads();
  const int row = threadIdx.x & 63, rg = threadIdx.x >> 6;   // 4 rhs groups
  const int gr = t.r0 + row;
  if (gr >= d.len) return;
  const double* Lr = L + d.loff + gr + (int64_t)t.k0 * d.ld;
  double acc[kSolveChunk / 4];
#pragma unroll
  for (int j = 0; j < kSolveChunk / 4; ++j) acc[j] = 0.0;
  for (int k = 0; k < kb; ++k) {
    const double l = Lr[(int64_t)k * d.ld];
#pragma unroll
    for (int j = 0; j < kSolveChunk / 4; ++j) {
      const int r = rg + 4 * j;
      if (r < nrhs) acc[j] = fma(l, yk[k + r * kb], acc[j]);
    }
  }
  const int b = d.len - d.s;
#pragma unroll
  for (int j = 0; j < kSolveChunk / 4; ++j) {
    const int r = rg + 4 * j;
    if (r >= nrhs) continue;
    if (gr < d.s) {
      Y[d.f + gr + (int64_t)r * n] -= acc[j];
    } else {
      double* w = W + d.wpre * nrhs + (gr - d.s) + (int64_t)r * b;
      *w = (t.k0 == 0) ? acc[j] : (*w + acc[j]);
    }
  }
}

// y[targets] -= w_J through the relind task lists (pull-ordered).
__global__ void __launch_bounds__(kSolveThreads)
k_fwd_assemble(const AsmTask* __restrict__ tasks, const AsmSeg* __restrict__ segs,
               const SnodeDev* __restrict__ sn, const int32_t* __restrict__ rows,
               const double* __restrict__ W, double* __restrict__ Y, int n, int nrhs) {
  const AsmTask t = tasks[blockIdx.x];
  for (int g = t.seg_begin; g < t.seg_end; ++g) {
    const AsmSeg sg = segs[g];
    const SnodeDev dj = sn[sg.J];
    const int b = dj.len - dj.s;
    const int32_t* rj = rows + dj.roff + dj.s;
    const double* Wj = W + dj.wpre * nrhs;
    const int ncol = sg.cb - sg.ca;
    for (int q = threadIdx.x; q < ncol * nrhs; q += blockDim.x) {
      const int c = sg.ca + q % ncol, r = q / ncol;
      Y[rj[c] + (int64_t)r * n] -= Wj[c + (int64_t)r * b];
    }
    __syncthreads();
  }
}

// Backward: y_J[c] -= sum_u L[s+u, c] x[rows[s+u]] for the 64 columns of a task.
__global__ void __launch_bounds__(kSolveThreads)
k_bwd_panel(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks,
            const int32_t* __restrict__ rows, const double* __restrict__ L, double* __restrict__ Y,
            int n, int nrhs) {
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int b = d.len - d.s;
  const int32_t* rj = rows + d.roff + d.s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cend = min(d.s, t.c0 + kBwdCols);
  for (int c = t.c0 + warp; c < cend; c += kSolveThreads / 32) {
    const double* Lc = L + d.loff + d.s + (int64_t)c * d.ld;
    double acc[kSolveChunk];
#pragma unroll
    for (int r = 0; r < kSolveChunk; ++r) acc[r] = 0.0;
    for (int u = lane; u < b; u += 32) {
      const double l = Lc[u];
      const int32_t g = rj[u];
#pragma unroll
      for (int r = 0; r < kSolveChunk; ++r)
        if (r < nrhs) acc[r] = fma(l, Y[g + (int64_t)r * n], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < kSolveChunk; ++r) {
      double v = acc[r];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[r] = v;
    }
    if (lane < nrhs) {
      double v = 0.0;
#pragma unroll
      for (int r = 0; r < kSolveChunk; ++r)
        if (r == lane) v = acc[r];
      Y[d.f + c + (int64_t)lane * n] -= v;
    }
  }
}

// Backward update of step k0: y[c0..c0+64) -= L[k0:k0+kb, c0..c0+64)^T x_k.
__global__ void __launch_bounds__(kSolveThreads)
k_bwd_update(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, int nb,
             const double* __restrict__ L, double* __restrict__ Y, int n, int nrhs) {
  __shared__ double xk[64 * kSolveChunk];
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int kb = min(nb, d.s - t.k0);
  for (int q = threadIdx.x; q < kb * nrhs; q += blockDim.x) {
    const int r = q % kb, c = q / kb;
    xk[q] = Y[d.f + t.k0 + r + (int64_t)c * n];
  }
  __syncthreads();
  const int col = threadIdx.x & 63, rg = threadIdx.x >> 6;
  const int gc = t.c0 + col;
  if (gc >= t.k0) return;               // only the column blocks left of step k0
  const double* Lc = L + d.loff + t.k0 + (int64_t)gc * d.ld;
  double acc[kSolveChunk / 4];
#pragma unroll
  for (int j = 0; j < kSolveChunk / 4; ++j) acc[j] = 0.0;
  for (int k = 0; k < kb; ++k) {
    const double l = Lc[k];
#pragma unroll
    for (int j = 0; j < kSolveChunk / 4; ++j) {
      const int r = rg + 4 * j;
      if (r < nrhs) acc[j] = fma(l, xk[k + r * kb], acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < kSolveChunk / 4; ++j) {
    const int r = rg + 4 * j;
    if (r < nrhs) Y[d.f + gc + (int64_t)r * n] -= acc[j];
  }
}

inline unsigned grid1d(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g > 0 ? g : 1);
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

}  // namespace

extern "C" int chol_solve(chol_handle* h, double* b, int32_t nrhs, void* stream) {
  if (!h) return -1;
  if (!b && nrhs > 0 && h->n > 0) return -2;
  if (nrhs < 0) return -3;
  if (!h->factored) return CHOL_ESTATE;
  if (nrhs == 0 || h->n == 0) return CHOL_OK;
  if (h->opt.precision != CHOL_PREC_FP64) return chol_solve_mixed(h, b, nrhs, (cudaStream_t)stream);
  int rc = ensure_solve_ws(h);
  if (rc) return rc;
  DeviceState* D = h->dev;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = h->opt.block_cols;
  const int n = h->n;
  for (int r0 = 0; r0 < nrhs; r0 += kSolveChunk) {
    const int nr = std::min(kSolveChunk, nrhs - r0);
    double* B = b + (int64_t)r0 * n;
    {
      KScope ks(h, CHOL_K_PERMUTE, st, 0.0, 24.0 * n * nr);
      k_permute_in<<<grid1d((int64_t)n * nr, 256), 256, 0, st>>>(B, D->perm, n, n, nr, D->Y);
    }
    for (const LevelPlan& P : h->levels) {
      for (size_t k = 0; k < P.ssteps.size(); ++k) {
        const SolveStep& s = P.ssteps[k];
        const int k0 = (int)k * nb;
        if (s.diag_n > 0) {
          KScope ks(h, CHOL_K_SOLVE_DIAG, st, 0.0, 0.0);
          k_diag<false><<<s.diag_n, kSolveThreads, 0, st>>>(
              D->sn, D->sdiag + s.diag_b, k0, nb, D->L, D->Y, n, nr);
        }
        if (s.fupd_n > 0) {
          KScope ks(h, CHOL_K_SOLVE_FUPD, st, 0.0, 0.0);
          k_fwd_update<<<s.fupd_n, kSolveThreads, 0, st>>>(D->sn, D->fupd + s.fupd_b, nb, D->L, D->Y, n,
                                                           D->W, nr);
        }
      }
      if (P.asm_n > 0) {
        KScope ks(h, CHOL_K_SOLVE_FASM, st, 0.0, 0.0);
        k_fwd_assemble<<<P.asm_n, kSolveThreads, 0, st>>>(D->asm_tasks + P.asm_b, D->asm_segs, D->sn,
                                                          D->rows, D->W, D->Y, n, nr);
      }
    }
    for (int lv = h->nlevels - 1; lv >= 0; --lv) {
      const LevelPlan& P = h->levels[lv];
      if (P.bpanel_n > 0) {
        KScope ks(h, CHOL_K_SOLVE_BPANEL, st, 0.0, 0.0);
        k_bwd_panel<<<P.bpanel_n, kSolveThreads, 0, st>>>(D->sn, D->bpanel + P.bpanel_b, D->rows, D->L,
                                                          D->Y, n, nr);
      }
      for (int k = (int)P.ssteps.size() - 1; k >= 0; --k) {
        const SolveStep& s = P.ssteps[k];
        const int k0 = k * nb;
        if (s.diag_n > 0) {
          KScope ks(h, CHOL_K_SOLVE_DIAG, st, 0.0, 0.0);
          k_diag<true><<<s.diag_n, kSolveThreads, 0, st>>>(
              D->sn, D->sdiag + s.diag_b, k0, nb, D->L, D->Y, n, nr);
        }
        if (s.bupd_n > 0) {
          KScope ks(h, CHOL_K_SOLVE_BUPD, st, 0.0, 0.0);
          k_bwd_update<<<s.bupd_n, kSolveThreads, 0, st>>>(D->sn, D->bupd + s.bupd_b, nb, D->L, D->Y, n,
                                                           nr);
        }
      }
    }
    {
      KScope ks(h, CHOL_K_PERMUTE, st, 0.0, 24.0 * n * nr);
      k_permute_out<<<grid1d((int64_t)n * nr, 256), 256, 0, st>>>(D->Y, D->perm, n, n, nr, B);
    }
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
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
// reading it, and the first column step writes each W row before accumulating).
// Calls whose work overlaps on the GPU (different streams or threads) race on
// the array. The first call on each device looks up the array's device address
// with cudaGetSymbolAddress (with that device current); make that first call
// before any stream capture.
// ---------------------------------------------------------------------------
constexpr int64_t kNoAllocScratchDoubles = int64_t(1) << 21;
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

namespace {

constexpr int kNoAllocMaxDevices = 64;
std::mutex g_noalloc_mu;
double* g_noalloc_addr[kNoAllocMaxDevices] = {};

// Device address of g_noalloc_scratch on the current device (looked up once).
int noalloc_scratch(double** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kNoAllocMaxDevices) {
    cudaGetLastError();
    return CHOL_ECUDA;
  }
  std::lock_guard<std::mutex> lock(g_noalloc_mu);
  if (!g_noalloc_addr[dev]) {
    void* p = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) {
      cudaGetLastError();
      return CHOL_ECUDA;
    }
    g_noalloc_addr[dev] = static_cast<double*>(p);
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
  if (!h->factored || !h->dev) return CHOL_ESTATE;
  if (h->opt.precision != CHOL_PREC_FP64) return CHOL_ENOTSUP;
  if (nrhs == 0 || h->n == 0) return CHOL_OK;
  double* scratch = nullptr;
  int rc = noalloc_scratch(&scratch);
  if (rc) return rc;
  const int chunk = (int)std::min<int64_t>(kSolveChunk, kNoAllocScratchDoubles / std::max<int64_t>(per_col, 1));
  DeviceState* D = h->dev;
  cudaStream_t st = (cudaStream_t)stream;
  const int nb = h->opt.block_cols;
  const int n = h->n;
  double* Y = scratch;
  double* W = scratch + (int64_t)n * chunk;
  for (int r0 = 0; r0 < nrhs; r0 += chunk) {
    const int nr = std::min(chunk, nrhs - r0);
    double* B = b + (int64_t)r0 * n;
    k_permute_in<<<grid1d((int64_t)n * nr, 256), 256, 0, st>>>(B, D->perm, n, n, nr, Y);
    for (const LevelPlan& P : h->levels) {
      for (size_t k = 0; k < P.ssteps.size(); ++k) {
        const SolveStep& s = P.ssteps[k];
        const int k0 = (int)k * nb;
        if (s.diag_n > 0)
          k_diag<false><<<s.diag_n, kSolveThreads, 0, st>>>(D->sn, D->sdiag + s.diag_b, k0, nb, D->L, Y, n, nr);
        if (s.fupd_n > 0)
          k_fwd_update<<<s.fupd_n, kSolveThreads, 0, st>>>(D->sn, D->fupd + s.fupd_b, nb, D->L, Y, n, W, nr);
      }
      if (P.asm_n > 0)
        k_fwd_assemble<<<P.asm_n, kSolveThreads, 0, st>>>(D->asm_tasks + P.asm_b, D->asm_segs, D->sn, D->rows,
                                                          W, Y, n, nr);
    }
    for (int lv = h->nlevels - 1; lv >= 0; --lv) {
      const LevelPlan& P = h->levels[lv];
      if (P.bpanel_n > 0)
        k_bwd_panel<<<P.bpanel_n, kSolveThreads, 0, st>>>(D->sn, D->bpanel + P.bpanel_b, D->rows, D->L, Y, n, nr);
      for (int k = (int)P.ssteps.size() - 1; k >= 0; --k) {
        const SolveStep& s = P.ssteps[k];
        const int k0 = k * nb;
        if (s.diag_n > 0)
          k_diag<true><<<s.diag_n, kSolveThreads, 0, st>>>(D->sn, D->sdiag + s.diag_b, k0, nb, D->L, Y, n, nr);
        if (s.bupd_n > 0)
          k_bwd_update<<<s.bupd_n, kSolveThreads, 0, st>>>(D->sn, D->bupd + s.bupd_b, nb, D->L, Y, n, nr);
      }
    }
    k_permute_out<<<grid1d((int64_t)n * nr, 256), 256, 0, st>>>(Y, D->perm, n, n, nr, B);
  }
  const cudaError_t e = cudaGetLastError();
  return e == cudaSuccess ? CHOL_OK : CHOL_ECUDA;
}
