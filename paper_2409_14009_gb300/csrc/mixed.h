// mixed.h -- entry points of the mixed-precision factor, the tensor-core tiles
// and the refinement, shared between translation units.
#pragma once
#include <cuda_runtime.h>

#include "internal.h"

int chol_mixed_ensure(chol_handle* h);
int chol_enqueue_factor_mixed(chol_handle* h, const double* values, cudaStream_t st);
int chol_finish_factor(chol_handle* h, cudaStream_t st);
int chol_launch_persistent(chol_handle* h, void* L, void* U, cudaStream_t st);
const void* chol_persistent_kernel(int precision, int threads);
const void* chol_persistent_kernel_mixed(int threads);
int chol_logdet_parts_mixed(chol_handle* h, cudaStream_t st);
int chol_logdet_mixed(chol_handle* h, double* out, cudaStream_t st);
int chol_gather_mixed(chol_handle* h, const int64_t* dmap, const int32_t* dlrow, double* dlx, cudaStream_t st);
int chol_solve_mixed(chol_handle* h, double* b, int32_t nrhs, cudaStream_t st);
void chol_status_init(int* status, cudaStream_t st);

int chol_tc_prepare(chol_handle* h);
int chol_tc_gemm(chol_handle* h, const TileTask* tasks, int n, int nb, int inner, cudaStream_t st);
int chol_tc_syrk(chol_handle* h, const TileTask* tasks, int n, cudaStream_t st);
int chol_tc_status(chol_handle* h);
void chol_adjoint_free(chol_handle* h);
int chol_solve_status(chol_handle* h);
int chol_diag_inv(chol_handle* h, int b, int nitems, cudaStream_t st);
int chol_bc_begin_mixed(const chol_handle* h);
int chol_bc_read_mixed();
