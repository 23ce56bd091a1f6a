// bounds.cuh -- the CHOL_BOUNDS_CHECK build of the library: range checks of the
// relind assembly (task and segment fields, the target positions found by the
// binary searches, the target columns) and of the value scatter into the
// panels. A failed check records its code in a device word (the first failure
// wins) and the access is skipped, so a corrupt plan gives CHOL_EBOUNDS from
// chol_factor instead of a memory fault. In the normal build every check
// compiles to nothing.
//
// The limits and the error word are per translation unit (static), set by
// bc_begin before a factorization and read by bc_read after it; one
// factorization at a time per process in the checked build.
#pragma once
#include <cstdint>

#include "internal.h"

enum : int {
  kBcNone = 0,
  kBcTaskTarget = 1,     // assembly task: target supernode out of range
  kBcTaskPositions = 2,  // assembly task: row positions or segment range out of range
  kBcSegSource = 3,      // segment: source supernode out of range
  kBcSegRange = 4,       // segment: rows or columns outside U_J (or the task's scratch)
  kBcTargetRow = 5,      // a row of U_J not found in the target's structure
  kBcTargetCol = 6,      // a column of U_J outside the target's columns
  kBcScatter = 7         // value scatter: position past the panels
};

#ifdef CHOL_BOUNDS_CHECK
#include <cuda_runtime.h>
struct BcLimits {
  int32_t ns;        // storage supernodes
  int32_t pad;
  int64_t nsegs;     // assembly segments
  int64_t panel;     // panel entries (L storage)
};
static __constant__ BcLimits bc_lim;
static __device__ int bc_err;
__device__ __forceinline__ bool bc_ok(bool cond, int code) {
  if (!cond) atomicCAS(&bc_err, 0, code);
  return cond;
}
static inline int bc_begin(const chol_handle* h) {
  BcLimits l{h->ns, 0, (int64_t)h->asm_segs.size(), h->panel_doubles};
  int zero = 0;
  if (cudaMemcpyToSymbol(bc_lim, &l, sizeof(l)) != cudaSuccess ||
      cudaMemcpyToSymbol(bc_err, &zero, sizeof(zero)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return 0;
}
static inline int bc_read() {
  int e = 0;
  if (cudaMemcpyFromSymbol(&e, bc_err, sizeof(e)) != cudaSuccess) {
    cudaGetLastError();
    return -1;
  }
  return e;
}
#define CHOL_BC(cond, code) bc_ok((cond), (code))
#else
#define CHOL_BC(cond, code) true
#endif
