// refine.cu -- the binary32 triangular solves of the mixed modes, and binary64
// iterative refinement / preconditioned conjugate gradients around any factor.
//
// Mixed solve, x = A^{-1} b with A = D^{-1} L~ L~^T D^{-1}: the right-hand
// sides are permuted, multiplied by D and divided by their max-norm, solved
// with the binary32 factor (row-major panels, the same blocked schedule as the
// binary64 solve), then multiplied back and returned in binary64.
//
// Refinement works in binary64 on the original A (full CSR, the values of the
// last factorization): r = b - A x, d = solve(r), x += d, until the normwise
// backward error reaches the tolerance. If that stagnates, conjugate gradients
// preconditioned by the same factor take over. All reductions use fixed orders
// (deterministic).
#include <cmath>
#include <cstring>
#include <vector>

#include "device.h"
#include "mixed.h"

namespace {

constexpr int kT = 256;
constexpr int kChunk = kSolveChunk;

inline unsigned grid1d(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g > 0 ? g : 1);
}

// ---- binary32 solve kernels (row-major panels) ------------------------------

// per right-hand side: scale[r] = max_i |b_ir| (1 if zero); uses the ordering of
// non-negative doubles as unsigned integers
__global__ void k_maxabs_cols(const double* __restrict__ b, int n, int nr, unsigned long long* __restrict__ out) {
  for (int r = 0; r < nr; ++r) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      m = fmax(m, fabs(b[i + (int64_t)r * n]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + r, (unsigned long long)__double_as_longlong(m));
  }
}

__global__ void k_mx_permute_in(const double* __restrict__ B, const int32_t* __restrict__ perm,
                                const double* __restrict__ d, const unsigned long long* __restrict__ scale_bits,
                                int n, int nr, float* __restrict__ Y) {
  const int64_t tot = (int64_t)n * nr;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), i = (int)(q % n);
    double s = __longlong_as_double((long long)scale_bits[r]);
    if (!(s > 0.0)) s = 1.0;
    Y[q] = (float)(B[perm[i] + (int64_t)r * n] * d[i] / s);
  }
}

__global__ void k_mx_permute_out(const float* __restrict__ Y, const int32_t* __restrict__ perm,
                                 const double* __restrict__ d, const unsigned long long* __restrict__ scale_bits,
                                 int n, int nr, double* __restrict__ B) {
  const int64_t tot = (int64_t)n * nr;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n), i = (int)(q % n);
    double s = __longlong_as_double((long long)scale_bits[r]);
    if (!(s > 0.0)) s = 1.0;
    B[perm[i] + (int64_t)r * n] = (double)Y[q] * d[i] * s;
  }
}

template <bool TRANS>
__global__ void __launch_bounds__(kT)
k_mx_diag(const SnodeDev* __restrict__ sn, const int32_t* __restrict__ list, int k0, int nb,
          const float* __restrict__ L, float* __restrict__ Y, int n, int nrhs) {
  __shared__ float Lk[64 * 65];
  __shared__ float inv[64];
  const SnodeDev d = sn[list[blockIdx.x]];
  const int kb = min(nb, d.s - k0);
  const float* G = L + d.loff + (int64_t)k0 * d.ld + k0;
  for (int q = threadIdx.x; q < kb * kb; q += blockDim.x) {
    const int r = q / kb, c = q % kb;
    Lk[r + c * 65] = G[(int64_t)r * d.ld + c];
  }
  __syncthreads();
  for (int c = threadIdx.x; c < kb; c += blockDim.x) inv[c] = 1.0f / Lk[c + c * 65];
  __syncthreads();
  const int rr = threadIdx.x >> 4, q = threadIdx.x & 15;
  const bool live = rr < nrhs;
  float* Yb = Y + d.f + k0 + (int64_t)rr * n;
  float y[4];
#pragma unroll
  for (int a = 0; a < 4; ++a) {
    const int i = q + 16 * a;
    y[a] = (live && i < kb) ? Yb[i] : 0.f;
  }
  if (!TRANS) {
#pragma unroll
    for (int ka = 0; ka < 4; ++ka)
#pragma unroll
      for (int kq = 0; kq < 16; ++kq) {
        const int k = ka * 16 + kq;
        if (k < kb) {
          const float yk = __shfl_sync(0xffffffffu, y[ka] * inv[k], kq, 16);
          if (q == kq) y[ka] = yk;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = q + 16 * a;
            if (i > k && i < kb) y[a] = fmaf(-Lk[i + k * 65], yk, y[a]);
          }
        }
      }
  } else {
#pragma unroll
    for (int ka = 3; ka >= 0; --ka)
#pragma unroll
      for (int kq = 15; kq >= 0; --kq) {
        const int k = ka * 16 + kq;
        if (k < kb) {
          const float yk = __shfl_sync(0xffffffffu, y[ka] * inv[k], kq, 16);
          if (q == kq) y[ka] = yk;
#pragma unroll
          for (int a = 0; a < 4; ++a) {
            const int i = q + 16 * a;
            if (i < k) y[a] = fmaf(-Lk[k + i * 65], yk, y[a]);
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

__global__ void __launch_bounds__(kT)
k_mx_fwd_update(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, int nb,
                const float* __restrict__ L, float* __restrict__ Y, int n, float* __restrict__ W, int nrhs) {
  __shared__ float yk[64 * kChunk];
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int kb = min(nb, d.s - t.k0);
  for (int q = threadIdx.x; q < kb * nrhs; q += blockDim.x) {
    const int r = q % kb, c = q / kb;
    yk[q] = Y[d.f + t.k0 + r + (int64_t)c * n];
  }
  __syncthreads();
  const int row = threadIdx.x & 63, rg = threadIdx.x >> 6;
  const int gr = t.r0 + row;
  if (gr >= d.len) return;
  const float* Lr = L + d.loff + (int64_t)gr * d.ld + t.k0;
  float acc[kChunk / 4];
#pragma unroll
  for (int j = 0; j < kChunk / 4; ++j) acc[j] = 0.f;
  for (int k = 0; k < kb; ++k) {
    const float l = Lr[k];
#pragma unroll
    for (int j = 0; j < kChunk / 4; ++j) {
      const int r = rg + 4 * j;
      if (r < nrhs) acc[j] = fmaf(l, yk[k + r * kb], acc[j]);
    }
  }
  const int b = d.len - d.s;
#pragma unroll
  for (int j = 0; j < kChunk / 4; ++j) {
    const int r = rg + 4 * j;
    if (r >= nrhs) continue;
    if (gr < d.s) {
      Y[d.f + gr + (int64_t)r * n] -= acc[j];
    } else {
      float* w = W + d.wpre * nrhs + (gr - d.s) + (int64_t)r * b;
      *w = (t.k0 == 0) ? acc[j] : (*w + acc[j]);
    }
  }
}

__global__ void __launch_bounds__(kT)
k_mx_fwd_assemble(const AsmTask* __restrict__ tasks, const AsmSeg* __restrict__ segs,
                  const SnodeDev* __restrict__ sn, const int32_t* __restrict__ rows,
                  const float* __restrict__ W, float* __restrict__ Y, int n, int nrhs) {
  const AsmTask t = tasks[blockIdx.x];
  for (int g = t.seg_begin; g < t.seg_end; ++g) {
    const AsmSeg sg = segs[g];
    const SnodeDev dj = sn[sg.J];
    const int b = dj.len - dj.s;
    const int32_t* rj = rows + dj.roff + dj.s;
    const float* Wj = W + dj.wpre * nrhs;
    const int ncol = sg.cb - sg.ca;
    for (int q = threadIdx.x; q < ncol * nrhs; q += blockDim.x) {
      const int c = sg.ca + q % ncol, r = q / ncol;
      Y[rj[c] + (int64_t)r * n] -= Wj[c + (int64_t)r * b];
    }
    __syncthreads();
  }
}

__global__ void __launch_bounds__(kT)
k_mx_bwd_panel(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks,
               const int32_t* __restrict__ rows, const float* __restrict__ L, float* __restrict__ Y, int n,
               int nrhs) {
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int b = d.len - d.s;
  const int32_t* rj = rows + d.roff + d.s;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int cend = min(d.s, t.c0 + kBwdCols);
  for (int c = t.c0 + warp; c < cend; c += kT / 32) {
    const float* Lc = L + d.loff + (int64_t)d.s * d.ld + c;
    float acc[kChunk];
#pragma unroll
    for (int r = 0; r < kChunk; ++r) acc[r] = 0.f;
    for (int u = lane; u < b; u += 32) {
      const float l = Lc[(int64_t)u * d.ld];
      const int32_t g = rj[u];
#pragma unroll
      for (int r = 0; r < kChunk; ++r)
        if (r < nrhs) acc[r] = fmaf(l, Y[g + (int64_t)r * n], acc[r]);
    }
#pragma unroll
    for (int r = 0; r < kChunk; ++r) {
      float v = acc[r];
      for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
      acc[r] = v;
    }
    if (lane < nrhs) {
      float v = 0.f;
#pragma unroll
      for (int r = 0; r < kChunk; ++r)
        if (r == lane) v = acc[r];
      Y[d.f + c + (int64_t)lane * n] -= v;
    }
  }
}

__global__ void __launch_bounds__(kT)
k_mx_bwd_update(const SnodeDev* __restrict__ sn, const TileTask* __restrict__ tasks, int nb,
                const float* __restrict__ L, float* __restrict__ Y, int n, int nrhs) {
  __shared__ float xk[64 * kChunk];
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
  if (gc >= t.k0) return;
  const float* Lc = L + d.loff + (int64_t)t.k0 * d.ld + gc;
  float acc[kChunk / 4];
#pragma unroll
  for (int j = 0; j < kChunk / 4; ++j) acc[j] = 0.f;
  for (int k = 0; k < kb; ++k) {
    const float l = Lc[(int64_t)k * d.ld];
#pragma unroll
    for (int j = 0; j < kChunk / 4; ++j) {
      const int r = rg + 4 * j;
      if (r < nrhs) acc[j] = fmaf(l, xk[k + r * kb], acc[j]);
    }
  }
#pragma unroll
  for (int j = 0; j < kChunk / 4; ++j) {
    const int r = rg + 4 * j;
    if (r < nrhs) Y[d.f + gc + (int64_t)r * n] -= acc[j];
  }
}

// ---- binary64 vector kernels for refinement -----------------------------------

// R = B - A X (full CSR, warp per row, fixed-order lane reduction); also
// rmax[r] = max_i |R_ir| via the ordering of non-negative doubles.
__global__ void __launch_bounds__(kT)
k_residual(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const double* __restrict__ av,
           const double* __restrict__ X, const double* __restrict__ B, int n, int nrhs, double* __restrict__ R,
           unsigned long long* __restrict__ rmax) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    for (int r = 0; r < nrhs; ++r) {
      const double* x = X + (int64_t)r * n;
      double s = 0.0;
      for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) s = fma(av[t], x[ci[t]], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) {
        const double v = B[i + (int64_t)r * n] - s;
        R[i + (int64_t)r * n] = v;
        atomicMax(rmax + r, (unsigned long long)__double_as_longlong(fabs(v)));
      }
    }
  }
}

// Y = A X (full CSR), for conjugate gradients.
__global__ void __launch_bounds__(kT)
k_spmv(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const double* __restrict__ av,
       const double* __restrict__ X, int n, int nrhs, double* __restrict__ Y) {
  const int lane = threadIdx.x & 31;
  const int warps = (gridDim.x * blockDim.x) >> 5;
  for (int i = (blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < n; i += warps) {
    for (int r = 0; r < nrhs; ++r) {
      const double* x = X + (int64_t)r * n;
      double s = 0.0;
      for (int64_t t = rp[i] + lane; t < rp[i + 1]; t += 32) s = fma(av[t], x[ci[t]], s);
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
      if (lane == 0) Y[i + (int64_t)r * n] = s;
    }
  }
}

// ||A||_inf = max_i sum_j |A_ij| (one value)
__global__ void k_anorm(const int64_t* __restrict__ rp, const double* __restrict__ av, int n,
                        unsigned long long* __restrict__ out) {
  double m = 0.0;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
    double s = 0.0;
    for (int64_t t = rp[i]; t < rp[i + 1]; ++t) s += fabs(av[t]);
    m = fmax(m, s);
  }
  for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
  if ((threadIdx.x & 31) == 0) atomicMax(out, (unsigned long long)__double_as_longlong(m));
}

// X += alpha_r * Y per column (alpha from device memory, or 1)
__global__ void k_axpy_cols(const double* __restrict__ Y, const double* __restrict__ alpha, int n, int nrhs,
                            double* __restrict__ X) {
  const int64_t tot = (int64_t)n * nrhs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n);
    X[q] += (alpha ? alpha[r] : 1.0) * Y[q];
  }
}

// P = Z + beta_r P
__global__ void k_xpby_cols(const double* __restrict__ Z, const double* __restrict__ beta, int n, int nrhs,
                            double* __restrict__ P) {
  const int64_t tot = (int64_t)n * nrhs;
  for (int64_t q = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; q < tot; q += (int64_t)gridDim.x * blockDim.x) {
    const int r = (int)(q / n);
    P[q] = Z[q] + beta[r] * P[q];
  }
}

// Deterministic dot products per column: block partials in a fixed tree, then a
// fixed-order sum over the blocks. part has gridDim.x * nrhs entries.
constexpr int kDotBlocks = 304;
__global__ void k_dot_part(const double* __restrict__ A, const double* __restrict__ B, int n, int nrhs,
                           double* __restrict__ part) {
  __shared__ double red[kT];
  for (int r = 0; r < nrhs; ++r) {
    double s = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      s = fma(A[i + (int64_t)r * n], B[i + (int64_t)r * n], s);
    red[threadIdx.x] = s;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
      if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
      __syncthreads();
    }
    if (threadIdx.x == 0) part[blockIdx.x + r * gridDim.x] = red[0];
    __syncthreads();
  }
}

__global__ void k_dot_final(const double* __restrict__ part, int nblocks, int nrhs, double* __restrict__ out) {
  const int r = threadIdx.x;
  if (r >= nrhs) return;
  double s = 0.0;
  for (int b = 0; b < nblocks; ++b) s += part[b + r * nblocks];
  out[r] = s;
}

// CG scalars: alpha = rz / pq, then rz is kept; beta = rz_new / rz_old
__global__ void k_ratio(const double* __restrict__ num, const double* __restrict__ den, int nrhs,
                        double* __restrict__ out, const unsigned char* __restrict__ active) {
  const int r = threadIdx.x;
  if (r < nrhs) out[r] = (active[r] && den[r] != 0.0) ? num[r] / den[r] : 0.0;
}

}  // namespace

// Binary32 solve with the mixed-precision factor, in place on a binary64 block.
int chol_solve_mixed(chol_handle* h, double* b, int32_t nrhs, cudaStream_t st) {
  DeviceState* D = h->dev;
  const int n = h->n, nb = h->opt.block_cols;
  if (!D->Y32) {
    int rc = chol_dalloc(h, (void**)&D->Y32, sizeof(float) * (size_t)std::max(n, 1) * kChunk);
    if (rc) return rc;
    rc = chol_dalloc(h, (void**)&D->W32, sizeof(float) * (size_t)std::max<int64_t>(h->w_rows_max, 1) * kChunk);
    if (rc) return rc;
    rc = chol_dalloc(h, (void**)&D->rhs_scale, sizeof(double) * kChunk);
    if (rc) return rc;
  }
  const float* L = (const float*)D->L;
  unsigned long long* sc = (unsigned long long*)D->rhs_scale;
  for (int r0 = 0; r0 < nrhs; r0 += kChunk) {
    const int nr = std::min(kChunk, nrhs - r0);
    double* B = b + (int64_t)r0 * n;
    CHOL_CUDA_TRY(cudaMemsetAsync(sc, 0, sizeof(double) * kChunk, st));
    {
      KScope ks(h, CHOL_K_PERMUTE, st, 0.0, 8.0 * n * nr);
      k_maxabs_cols<<<grid1d(n, 256), 256, 0, st>>>(B, n, nr, sc);
      k_mx_permute_in<<<grid1d((int64_t)n * nr, 256), 256, 0, st>>>(B, D->perm, D->mx_d, sc, n, nr, D->Y32);
    }
    for (const LevelPlan& P : h->levels) {
      for (size_t k = 0; k < P.ssteps.size(); ++k) {
        const SolveStep& s = P.ssteps[k];
        const int k0 = (int)k * nb;
        if (s.diag_n > 0) {
          KScope ks(h, CHOL_K_SOLVE_DIAG, st, 0.0, 0.0);
          k_mx_diag<false><<<s.diag_n, kT, 0, st>>>(D->sn, D->sdiag + s.diag_b, k0, nb, L, D->Y32, n, nr);
        }
        if (s.fupd_n > 0) {
          KScope ks(h, CHOL_K_SOLVE_FUPD, st, 0.0, 0.0);
          k_mx_fwd_update<<<s.fupd_n, kT, 0, st>>>(D->sn, D->fupd + s.fupd_b, nb, L, D->Y32, n, D->W32, nr);
        }
      }
      if (P.asm_n > 0) {
        KScope ks(h, CHOL_K_SOLVE_FASM, st, 0.0, 0.0);
        k_mx_fwd_assemble<<<P.asm_n, kT, 0, st>>>(D->asm_tasks + P.asm_b, D->asm_segs, D->sn, D->rows, D->W32,
                                                  D->Y32, n, nr);
      }
    }
    for (int lv = h->nlevels - 1; lv >= 0; --lv) {
      const LevelPlan& P = h->levels[lv];
      if (P.bpanel_n > 0) {
        KScope ks(h, CHOL_K_SOLVE_BPANEL, st, 0.0, 0.0);
        k_mx_bwd_panel<<<P.bpanel_n, kT, 0, st>>>(D->sn, D->bpanel + P.bpanel_b, D->rows, L, D->Y32, n, nr);
      }
      for (int k = (int)P.ssteps.size() - 1; k >= 0; --k) {
        const SolveStep& s = P.ssteps[k];
        const int k0 = k * nb;
        if (s.diag_n > 0) {
          KScope ks(h, CHOL_K_SOLVE_DIAG, st, 0.0, 0.0);
          k_mx_diag<true><<<s.diag_n, kT, 0, st>>>(D->sn, D->sdiag + s.diag_b, k0, nb, L, D->Y32, n, nr);
        }
        if (s.bupd_n > 0) {
          KScope ks(h, CHOL_K_SOLVE_BUPD, st, 0.0, 0.0);
          k_mx_bwd_update<<<s.bupd_n, kT, 0, st>>>(D->sn, D->bupd + s.bupd_b, nb, L, D->Y32, n, nr);
        }
      }
    }
    {
      KScope ks(h, CHOL_K_PERMUTE, st, 0.0, 12.0 * n * nr);
      k_mx_permute_out<<<grid1d((int64_t)n * nr, 256), 256, 0, st>>>(D->Y32, D->perm, D->mx_d, sc, n, nr, B);
    }
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  return CHOL_OK;
}

namespace {

int ensure_refine_ws(chol_handle* h, int nrhs) {
  DeviceState* D = h->dev;
  if (D->refine_cap >= nrhs) return CHOL_OK;
  for (double** p : {&D->R, &D->Z, &D->Pv, &D->Q}) {
    if (*p) { cudaFree(*p); D->bytes -= sizeof(double) * (size_t)std::max(h->n, 1) * D->refine_cap; *p = nullptr; }
  }
  if (D->red) { cudaFree(D->red); D->red = nullptr; }
  if (D->red_host) { cudaFreeHost(D->red_host); D->red_host = nullptr; }
  int rc;
  for (double** p : {&D->R, &D->Z, &D->Pv, &D->Q})
    if ((rc = chol_dalloc(h, (void**)p, sizeof(double) * (size_t)std::max(h->n, 1) * nrhs))) return rc;
  // reduction scratch: [rmax | xmax | bmax | anorm | rz | pq | rznew | alpha | beta | active(bytes)] + partials
  const size_t nred = (size_t)(9 * nrhs + 1 + kDotBlocks * nrhs + nrhs);
  if ((rc = chol_dalloc(h, (void**)&D->red, sizeof(double) * nred))) return rc;
  if (cudaMallocHost((void**)&D->red_host, sizeof(double) * (4 * nrhs + 1)) != cudaSuccess) return CHOL_ENOMEM;
  D->refine_cap = nrhs;
  return CHOL_OK;
}

// Low-precision correction solve (or the binary64 solve in CHOL_PREC_FP64).
int correction_solve(chol_handle* h, double* v, int nrhs, cudaStream_t st) {
  if (h->opt.precision == CHOL_PREC_FP64) return chol_solve(h, v, nrhs, (void*)st);
  return chol_solve_mixed(h, v, nrhs, st);
}

}  // namespace

extern "C" int chol_solve_refine(chol_handle* h, const double* b, double* x, int32_t nrhs, double tol,
                                 int32_t max_iter, int32_t* iters, double* berr, void* stream) {
  if (!h) return -1;
  if (!b && nrhs > 0) return -2;
  if (!x && nrhs > 0) return -3;
  if (nrhs < 0 || nrhs > 1024) return -4;
  if (!(tol > 0.0)) return -5;
  if (max_iter < 1) return -6;
  if (!h->factored) return CHOL_ESTATE;
  if (iters) *iters = 0;
  if (nrhs == 0 || h->n == 0) return CHOL_OK;
  cudaStream_t st = (cudaStream_t)stream;
  int rc = ensure_refine_ws(h, nrhs);
  if (rc) return rc;
  DeviceState* D = h->dev;
  const int n = h->n;
  const size_t nb = sizeof(double) * (size_t)n * nrhs;
  double* red = D->red;
  unsigned long long* rmax = (unsigned long long*)red;
  unsigned long long* xmax = rmax + nrhs;
  unsigned long long* bmax = xmax + nrhs;
  unsigned long long* anorm = bmax + nrhs;
  double* rz = red + 3 * nrhs + 1;
  double* pq = rz + nrhs;
  double* rznew = pq + nrhs;
  double* alpha = rznew + nrhs;
  double* beta = alpha + nrhs;
  double* part = beta + nrhs;
  unsigned char* active = (unsigned char*)(part + kDotBlocks * nrhs);
  const unsigned gsp = grid1d((int64_t)n * 32, kT);

  // ||A||_inf and ||b||_inf
  CHOL_CUDA_TRY(cudaMemsetAsync(red, 0, sizeof(double) * (3 * nrhs + 1), st));
  k_anorm<<<grid1d(n, 256), 256, 0, st>>>(D->csr_ptr, D->csr_val, n, anorm);
  k_maxabs_cols<<<grid1d(n, 256), 256, 0, st>>>(b, n, nrhs, bmax);
  // x0 = solve(b)
  CHOL_CUDA_TRY(cudaMemcpyAsync(x, b, nb, cudaMemcpyDeviceToDevice, st));
  if ((rc = correction_solve(h, x, nrhs, st))) return rc;

  std::vector<double> eta(nrhs, 1.0), prev(nrhs, 1e300);
  std::vector<unsigned char> act(nrhs, 1);
  auto measure = [&]() -> int {
    // R = b - A x; eta = ||R|| / (||A|| ||x|| + ||b||)
    CHOL_CUDA_TRY(cudaMemsetAsync(rmax, 0, sizeof(double) * 2 * nrhs, st));
    k_residual<<<gsp, kT, 0, st>>>(D->csr_ptr, D->csr_col, D->csr_val, x, b, n, nrhs, D->R, rmax);
    k_maxabs_cols<<<grid1d(n, 256), 256, 0, st>>>(x, n, nrhs, xmax);
    CHOL_CUDA_TRY(cudaMemcpyAsync(D->red_host, red, sizeof(double) * (3 * nrhs + 1), cudaMemcpyDeviceToHost, st));
    CHOL_CUDA_TRY(cudaStreamSynchronize(st));
    const unsigned long long* hb = (const unsigned long long*)D->red_host;
    double an;
    std::memcpy(&an, &hb[3 * nrhs], 8);
    for (int r = 0; r < nrhs; ++r) {
      double rm, xm, bm;
      std::memcpy(&rm, &hb[r], 8);
      std::memcpy(&xm, &hb[nrhs + r], 8);
      std::memcpy(&bm, &hb[2 * nrhs + r], 8);
      const double den = an * xm + bm;
      eta[r] = den > 0.0 ? rm / den : 0.0;
    }
    return CHOL_OK;
  };
  auto done = [&]() {
    for (int r = 0; r < nrhs; ++r)
      if (!(eta[r] <= tol)) return false;
    return true;
  };
  int it = 0;
  if ((rc = measure())) return rc;
  bool use_cg = false;
  // plain refinement: x += solve(b - A x)
  while (!done() && it < max_iter) {
    bool stagnating = true;
    for (int r = 0; r < nrhs; ++r)
      if (eta[r] > tol && eta[r] < 0.5 * prev[r]) stagnating = false;
    if (it > 0 && stagnating) { use_cg = true; break; }
    prev = eta;
    CHOL_CUDA_TRY(cudaMemcpyAsync(D->Z, D->R, nb, cudaMemcpyDeviceToDevice, st));
    if ((rc = correction_solve(h, D->Z, nrhs, st))) return rc;
    k_axpy_cols<<<grid1d((int64_t)n * nrhs, 256), 256, 0, st>>>(D->Z, nullptr, n, nrhs, x);
    ++it;
    if ((rc = measure())) return rc;
  }
  if (use_cg && !done()) {
    // conjugate gradients on A, preconditioned by the factor; R holds b - A x
    CHOL_CUDA_TRY(cudaMemcpyAsync(D->Z, D->R, nb, cudaMemcpyDeviceToDevice, st));
    if ((rc = correction_solve(h, D->Z, nrhs, st))) return rc;
    CHOL_CUDA_TRY(cudaMemcpyAsync(D->Pv, D->Z, nb, cudaMemcpyDeviceToDevice, st));
    k_dot_part<<<kDotBlocks, kT, 0, st>>>(D->R, D->Z, n, nrhs, part);
    k_dot_final<<<1, 1024, 0, st>>>(part, kDotBlocks, nrhs, rz);
    while (!done() && it < max_iter) {
      for (int r = 0; r < nrhs; ++r) act[r] = eta[r] > tol ? 1 : 0;
      CHOL_CUDA_TRY(cudaMemcpyAsync(active, act.data(), nrhs, cudaMemcpyHostToDevice, st));
      k_spmv<<<gsp, kT, 0, st>>>(D->csr_ptr, D->csr_col, D->csr_val, D->Pv, n, nrhs, D->Q);
      k_dot_part<<<kDotBlocks, kT, 0, st>>>(D->Pv, D->Q, n, nrhs, part);
      k_dot_final<<<1, 1024, 0, st>>>(part, kDotBlocks, nrhs, pq);
      k_ratio<<<1, 1024, 0, st>>>(rz, pq, nrhs, alpha, active);
      k_axpy_cols<<<grid1d((int64_t)n * nrhs, 256), 256, 0, st>>>(D->Pv, alpha, n, nrhs, x);
      ++it;
      if ((rc = measure())) return rc;    // true residual of the new x in R
      if (done() || it >= max_iter) break;
      CHOL_CUDA_TRY(cudaMemcpyAsync(D->Z, D->R, nb, cudaMemcpyDeviceToDevice, st));
      if ((rc = correction_solve(h, D->Z, nrhs, st))) return rc;
      k_dot_part<<<kDotBlocks, kT, 0, st>>>(D->R, D->Z, n, nrhs, part);
      k_dot_final<<<1, 1024, 0, st>>>(part, kDotBlocks, nrhs, rznew);
      k_ratio<<<1, 1024, 0, st>>>(rznew, rz, nrhs, beta, active);
      k_xpby_cols<<<grid1d((int64_t)n * nrhs, 256), 256, 0, st>>>(D->Z, beta, n, nrhs, D->Pv);
      CHOL_CUDA_TRY(cudaMemcpyAsync(rz, rznew, sizeof(double) * nrhs, cudaMemcpyDeviceToDevice, st));
    }
  }
  CHOL_CUDA_TRY(cudaGetLastError());
  if (iters) *iters = it;
  if (berr) std::memcpy(berr, eta.data(), sizeof(double) * nrhs);
  return done() ? CHOL_OK : CHOL_ENOCONV;
}
