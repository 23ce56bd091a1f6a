// tc_gemm.cu -- host side and launch wrappers of the tcgen05 update tiles.
//
// One TMA tensor map per supernode describes its row-major panel (binary32 for
// CHOL_PREC_TF32, the bf16 copy for CHOL_PREC_BF16): dimensions {s, len}, row
// stride ld, box {128 bytes of K, 128 rows}, 128-byte swizzle, zero fill out of
// bounds. The maps live in device memory; each CTA uses the map of its task's
// supernode.
#include <cstring>
#include <vector>

#include "device.h"
#include "mixed.h"
#include "tc_gemm.cuh"

namespace {

typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*, const cuuint64_t*,
                                  const cuuint64_t*, const cuuint32_t*, const cuuint32_t*, CUtensorMapInterleave,
                                  CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

// Trailing update of a panel (C -= A B^T on the lower part) with K range
// [k0, k0 + nb). inner = 1: a column step's own update, whose columns stop at
// the end of the kTcOuter-wide block holding k0; inner = 0: the update of the
// columns right of a finished outer block (K = the block).
template <int KIND>
__global__ void __launch_bounds__(tc::kThreads, 1)
k_tc_trailing(const CUtensorMap* __restrict__ maps, const TileTask* __restrict__ tasks,
              const SnodeDev* __restrict__ sn, int nb, int inner, float* __restrict__ L, int stages, int* err) {
  extern __shared__ uint8_t smem[];
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int kb = min(nb, d.s - t.k0);
  const int cend = inner ? min(d.s, (t.k0 / kTcOuter + 1) * kTcOuter) : d.s;
  tc::TileJob job;
  job.map = maps + t.J;
  job.a_row = t.r0;
  job.b_row = t.c0;
  job.k_begin = t.k0;
  job.k_end = t.k0 + kb;
  job.C = L + d.loff + (int64_t)t.r0 * d.ld + t.c0;
  job.ldc = d.ld;
  job.m = min(tc::kTileM, d.len - t.r0);
  job.n = min(tc::kTileN, cend - t.c0);
  job.rdiag = t.r0 - t.c0;
  job.sub = true;
  tc::tile_body<KIND>(job, smem, stages, err);
}

// U_J tile (row-major lower, leading dimension b rounded to 8) = L_RJ L_RJ^T.
template <int KIND>
__global__ void __launch_bounds__(tc::kThreads, 1)
k_tc_syrk(const CUtensorMap* __restrict__ maps, const TileTask* __restrict__ tasks,
          const SnodeDev* __restrict__ sn, float* __restrict__ U, int stages, int* err) {
  extern __shared__ uint8_t smem[];
  const TileTask t = tasks[blockIdx.x];
  const SnodeDev d = sn[t.J];
  const int b = d.len - d.s;
  const int ldu = (b + 7) & ~7;
  tc::TileJob job;
  job.map = maps + t.J;
  job.a_row = d.s + t.r0;
  job.b_row = d.s + t.c0;
  job.k_begin = 0;
  job.k_end = d.s;
  job.C = U + d.uoff + (int64_t)t.r0 * ldu + t.c0;
  job.ldc = ldu;
  job.m = min(tc::kTileM, b - t.r0);
  job.n = min(tc::kTileN, b - t.c0);
  job.rdiag = t.r0 - t.c0;
  job.sub = false;
  tc::tile_body<KIND>(job, smem, stages, err);
}

}  // namespace

int chol_tc_prepare(chol_handle* h) {
  const int prec = h->opt.precision;
  if (prec != CHOL_PREC_TF32 && prec != CHOL_PREC_BF16) return CHOL_OK;
  DeviceState* D = h->dev;
  int rc;
  if (!D->tc_err) {
    if ((rc = chol_dalloc(h, (void**)&D->tc_err, sizeof(int32_t)))) return rc;
    CHOL_CUDA_TRY(cudaMemset(D->tc_err, 0, sizeof(int32_t)));
  }
  void* base = D->L;
  size_t esz = 4;
  if (prec == CHOL_PREC_BF16) {
    if ((rc = chol_dalloc(h, (void**)&D->Lbf, sizeof(__nv_bfloat16) * (size_t)std::max<int64_t>(h->panel_doubles, 1))))
      return rc;
    CHOL_CUDA_TRY(cudaMemset(D->Lbf, 0, sizeof(__nv_bfloat16) * (size_t)std::max<int64_t>(h->panel_doubles, 1)));
    base = D->Lbf;
    esz = 2;
  }
  EncodeTiledFn encode = nullptr;
  cudaDriverEntryPointQueryResult q;
  if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&encode, 12000, cudaEnableDefault, &q) !=
          cudaSuccess ||
      !encode || q != cudaDriverEntryPointSuccess) {
    cudaGetLastError();
    return CHOL_ECUDA;
  }
  std::vector<CUtensorMap> maps(std::max(h->ns, 1));
  std::memset(maps.data(), 0, sizeof(CUtensorMap) * maps.size());
  for (int32_t J = 0; J < h->ns; ++J) {
    const SnodeDev& d = h->snodes[J];
    cuuint64_t gdim[2] = {(cuuint64_t)d.s, (cuuint64_t)d.len};
    cuuint64_t gstr[1] = {(cuuint64_t)d.ld * esz};
    cuuint32_t box[2] = {(cuuint32_t)(128 / esz), (cuuint32_t)tc::kTileM};
    cuuint32_t estr[2] = {1, 1};
    void* addr = (char*)base + (size_t)d.loff * esz;
    const CUresult cr = encode(&maps[J], prec == CHOL_PREC_TF32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32
                                                                 : CU_TENSOR_MAP_DATA_TYPE_BFLOAT16,
                               2, addr, gdim, gstr, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (cr != CUDA_SUCCESS) return CHOL_ECUDA;
  }
  if ((rc = chol_dalloc(h, (void**)&D->tmaps, sizeof(CUtensorMap) * maps.size()))) return rc;
  CHOL_CUDA_TRY(cudaMemcpy(D->tmaps, maps.data(), sizeof(CUtensorMap) * maps.size(), cudaMemcpyHostToDevice));
  const void* kernels[] = {(const void*)k_tc_trailing<0>, (const void*)k_tc_trailing<1>, (const void*)k_tc_syrk<0>,
                           (const void*)k_tc_syrk<1>};
  for (const void* k : kernels)
    CHOL_CUDA_TRY(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, tc::kSmemMax));
  return CHOL_OK;
}

int chol_tc_gemm(chol_handle* h, const TileTask* tasks, int n, int nb, int inner, cudaStream_t st) {
  DeviceState* D = h->dev;
  const int ns = tc::stages_for(n, D->sms);
  ++(ns == tc::kFewStages ? h->tc_shallow : h->tc_deep);
  const int sm = tc::smem_bytes(ns);
  if (h->opt.precision == CHOL_PREC_TF32)
    k_tc_trailing<0><<<n, tc::kThreads, sm, st>>>(D->tmaps, tasks, D->sn, nb, inner, (float*)D->L, ns, D->tc_err);
  else
    k_tc_trailing<1><<<n, tc::kThreads, sm, st>>>(D->tmaps, tasks, D->sn, nb, inner, (float*)D->L, ns, D->tc_err);
  return CHOL_OK;
}

int chol_tc_syrk(chol_handle* h, const TileTask* tasks, int n, cudaStream_t st) {
  DeviceState* D = h->dev;
  const int ns = tc::stages_for(n, D->sms);
  ++(ns == tc::kFewStages ? h->tc_shallow : h->tc_deep);
  const int sm = tc::smem_bytes(ns);
  if (h->opt.precision == CHOL_PREC_TF32)
    k_tc_syrk<0><<<n, tc::kThreads, sm, st>>>(D->tmaps, tasks, D->sn, (float*)D->U, ns, D->tc_err);
  else
    k_tc_syrk<1><<<n, tc::kThreads, sm, st>>>(D->tmaps, tasks, D->sn, (float*)D->U, ns, D->tc_err);
  return CHOL_OK;
}

// After a synchronized factorization: CHOL_ETIMEOUT if any tile gave up waiting.
int chol_tc_status(chol_handle* h) {
  DeviceState* D = h->dev;
  if (!D->tc_err) return CHOL_OK;
  int32_t e = 0;
  CHOL_CUDA_TRY(cudaMemcpy(&e, D->tc_err, sizeof(int32_t), cudaMemcpyDeviceToHost));
  if (e != 0) {
    CHOL_CUDA_TRY(cudaMemset(D->tc_err, 0, sizeof(int32_t)));
    return CHOL_ETIMEOUT;
  }
  return CHOL_OK;
}
