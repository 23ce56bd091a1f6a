// refine.cu -- binary64 iterative refinement / preconditioned conjugate
// gradients around any factor (the correction solves use the factor's own
// precision: binary32 for the mixed modes, see solve.cu).
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

inline unsigned grid1d(int64_t n, int threads) {
  int64_t g = (n + threads - 1) / threads;
  if (g > 152 * 32) g = 152 * 32;
  return (unsigned)(g > 0 ? g : 1);
}

// per right-hand side: out[r] = max_i |b_ir| (ordering of non-negative doubles)
__global__ void k_maxabs_cols(const double* __restrict__ b, int n, int nr, unsigned long long* __restrict__ out) {
  for (int r = 0; r < nr; ++r) {
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x)
      m = fmax(m, fabs(b[i + (int64_t)r * n]));
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(out + r, (unsigned long long)__double_as_longlong(m));
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

// The same residual with a thread per row, for matrices with few entries per
// row (at most 16 on average, e.g. 5-point grids): each row's sum in entry
// order, the maxima reduced per warp before one atomic per warp and column.
__global__ void __launch_bounds__(kT)
k_residual_rows(const int64_t* __restrict__ rp, const int32_t* __restrict__ ci, const double* __restrict__ av,
                const double* __restrict__ X, const double* __restrict__ B, int n, int nrhs,
                double* __restrict__ R, unsigned long long* __restrict__ rmax) {
  for (int r = 0; r < nrhs; ++r) {
    const double* x = X + (int64_t)r * n;
    double m = 0.0;
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < n; i += gridDim.x * blockDim.x) {
      double s = 0.0;
      for (int64_t t = rp[i]; t < rp[i + 1]; ++t) s = fma(av[t], x[ci[t]], s);
      const double v = B[i + (int64_t)r * n] - s;
      R[i + (int64_t)r * n] = v;
      m = fmax(m, fabs(v));
    }
    for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
    if ((threadIdx.x & 31) == 0) atomicMax(rmax + r, (unsigned long long)__double_as_longlong(m));
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
  NvtxRange nvtx_range("chol_solve_refine");
  if (!h) return -1;
  if (!b && nrhs > 0) return -2;
  if (!x && nrhs > 0) return -3;
  if (nrhs < 0 || nrhs > 1024) return -4;
  if (!(tol > 0.0)) return -5;
  if (max_iter < 1) return -6;
  if (int rc_state = chol_factored_here(h)) return rc_state;
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
  // a warp per row wastes most lanes on rows of a few entries
  const bool few_per_row = h->csr_ptr[n] <= 16 * (int64_t)n;

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
    if (few_per_row)
      k_residual_rows<<<grid1d(n, kT), kT, 0, st>>>(D->csr_ptr, D->csr_col, D->csr_val, x, b, n, nrhs, D->R, rmax);
    else
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
  {
    const int rc = chol_solve_status(h);
    if (rc) return rc;
  }
  return done() ? CHOL_OK : CHOL_ENOCONV;
}
