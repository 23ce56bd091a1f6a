// device.h -- device-side state of a handle and helpers shared by the CUDA
// translation units.
#pragma once
#include <cuda.h>
#include <cuda_runtime.h>

#include <vector>

#include "internal.h"

struct DeviceState {
  int device = -1;
  int sms = 152;                // streaming multiprocessors of the device
  int64_t bytes = 0;            // bytes allocated so far (for the optional cap)
  double* L = nullptr;          // supernodal panels
  double* U = nullptr;          // update-matrix workspace (one level)
  SnodeDev* sn = nullptr;
  int32_t* rows = nullptr;
  int64_t* amap = nullptr;
  int32_t* small_list = nullptr;
  int32_t* potrf_list = nullptr;
  int32_t* level_snodes = nullptr;
  TileTask* trsm = nullptr;
  TileTask* gemm = nullptr;
  TileTask* syrk = nullptr;
  AsmTask* asm_tasks = nullptr;
  AsmSeg* asm_segs = nullptr;
  TriItemHost* tri = nullptr;   // solve: diagonal-triangle items
  int4* rlb_pairs = nullptr;    // RLB: (K, c0, c1, -) of every (J, K) pair, J-major
  int32_t* rlb_pbeg = nullptr;  // RLB: first pair of every supernode
  double* zrr_ws = nullptr;     // adjoint: Z_RR workspace when there is no update workspace (RLB)
  int32_t* tri_flags = nullptr; // solve: one flag per diagonal block and chunk column (zeroed once)
  void* dinv = nullptr;         // per 64-row diagonal block of the solve: binary64 L_ii^{-1}; mixed modes: L_ii^{-1} and two products (binary32)
  int32_t* tri_sync = nullptr;  // solve: {epoch, CTAs done} of the triangle launches
  int32_t* sv_err = nullptr;    // solve: set when a bounded wait gave up
  int32_t* ssmall = nullptr;
  TileTask* bpanel = nullptr;
  TileTask* gemv = nullptr;
  TileTask* bpart = nullptr;
  TileTask* bred = nullptr;
  int32_t* perm = nullptr;
  int32_t* status = nullptr;    // device status word (first failing column + 1)
  int32_t* status_host = nullptr;  // pinned
  double* part = nullptr;       // logdet partial sums (one per supernode)
  double* split_part = nullptr; // binary64 solve: partial sums of split panel products (split_slots_max x 64 x chunk)
  int32_t* split_cnt = nullptr; // ... and one arrival counter per slot (zero between uses)
  double* scalar_host = nullptr;   // pinned
  double* scalar_dev = nullptr;
  // mixed modes
  bool mx_ready = false;
  int64_t* mx_diagpos = nullptr;   // position of A_ii of P A P^T in the values array
  int32_t* mx_aij = nullptr;       // (row, col) of P A P^T per entry of A
  double* mx_d = nullptr;          // D = diag(P A P^T)^{-1/2}
  int32_t* mx_fallbacks = nullptr; // diagonal blocks redone in binary64
  int64_t* csr_ptr = nullptr;      // full symmetric A, original ordering (refinement)
  int32_t* csr_col = nullptr;
  int64_t* csr_src = nullptr;
  double* csr_val = nullptr;
  void* Lbf = nullptr;             // bf16 copy of the panels (CHOL_PREC_BF16)
  CUtensorMap* tmaps = nullptr;    // one TMA map per supernode
  int32_t* tc_err = nullptr;       // tensor-core tile / panel wait timeout flag
  PanelItem* panel = nullptr;      // panel-launch tiles (mixed modes)
  int32_t* pflags = nullptr;       // panel work counters, then progress flags (zeroed per factorization)
  int panel_ctas = 0;              // resident panel CTAs on the device
  // refinement workspaces
  double* R = nullptr;
  double* Z = nullptr;
  double* Pv = nullptr;
  double* Q = nullptr;
  double* red = nullptr;           // reduction scratch
  double* red_host = nullptr;      // pinned
  int refine_cap = 0;
  float* Y32 = nullptr;            // binary32 solve workspaces
  float* W32 = nullptr;
  float* P32 = nullptr;             // row-major backward-panel partials
  unsigned long long* hand32 = nullptr;   // binary32 triangle solve: tagged hand-off words, n x chunk
  double* rhs_scale = nullptr;
  // batches, persistent launches and graphs
  PersistLevel* plevels = nullptr;
  double* vals = nullptr;          // handle-owned copy of the values (graph replays)
  int32_t* sys_snode = nullptr;    // storage-supernode range of every system
  double* sys_out = nullptr;
  cudaGraphExec_t graph_exec = nullptr;
  cudaStream_t gstream = nullptr;  // capture / replay stream of the handle
  cudaEvent_t gev[2] = {nullptr, nullptr};
  cudaStream_t lstream = nullptr;  // side stream of the lookahead trailing updates (lowest priority)
  cudaStream_t hstream = nullptr;  // critical path of the blocked levels (highest priority)
  cudaEvent_t lev[3] = {nullptr, nullptr, nullptr};   // panel final / rest done / fork-join
  cudaStream_t istream = nullptr;  // binary64: diagonal-block inverses of finished levels (lowest priority)
  cudaEvent_t iev[2] = {nullptr, nullptr};            // level factored / inverses done
  chol_kernel_stat graph_delta[CHOL_K_NCLASSES] = {};
  float mx_spiv = 0.f;             // static-pivot threshold passed to the persistent kernel
  // selected inverse and adjoint
  double* Zp = nullptr;            // Z = (P A P^T)^{-1} on the pattern of L, panel layout
  double* Tw = nullptr;            // L_JJ^{-1}
  double* Ww = nullptr;
  double* Uh = nullptr;            // L_RJ L_JJ^{-1}
  int32_t* a_col = nullptr;        // column / row of every stored entry of A
  int32_t* a_row = nullptr;
  double* adj_xb = nullptr;
  void* si_plan = nullptr;         // level plan of the selected inverse (adjoint.cu)
  int adj_cap = 0;
  // solve workspaces (grown on demand)
  double* Y = nullptr;          // permuted right-hand sides, n x chunk
  double* W = nullptr;          // per-level panel products, w_rows_max x chunk
  // staging of chol_factor_solve_host (host-buffer entry point)
  double* host_vals = nullptr;  // nnz(A) values
  double* host_rhs = nullptr;   // n x nrhs right-hand sides / solutions
  int64_t host_rhs_cap = 0;
};

// Right-hand sides are processed in chunks of at most this many columns.
constexpr int kSolveChunk = 16;

#define CHOL_CUDA_TRY(expr)                 \
  do {                                      \
    cudaError_t e_ = (expr);                \
    if (e_ != cudaSuccess) {                \
      return e_ == cudaErrorMemoryAllocation ? CHOL_ENOMEM : CHOL_ECUDA; \
    }                                       \
  } while (0)

// Launch accounting: counts, algorithmic flops/bytes, and (for the classes in
// the mask) CUDA-event timing of each launch on its stream.
struct Profiler {
  uint32_t mask = 0;
  chol_kernel_stat st[CHOL_K_NCLASSES] = {};
  struct Pending {
    int cls;
    cudaEvent_t a, b;
  };
  std::vector<Pending> pending;
  std::vector<cudaEvent_t> pool;
  cudaStream_t last = nullptr;
};

inline Profiler* chol_prof(chol_handle* h) {
  if (!h->prof) h->prof = new Profiler();
  return h->prof;
}

// RAII scope around one kernel launch.
struct KScope {
  Profiler* p;
  int cls;
  cudaStream_t st;
  cudaEvent_t a = nullptr, b = nullptr;
  KScope(chol_handle* h, int cls_, cudaStream_t st_, double flops, double bytes)
      : p(chol_prof(h)), cls(cls_), st(st_) {
    p->st[cls].launches++;
    p->st[cls].flops += flops;
    p->st[cls].bytes += bytes;
    p->last = st;
    if (p->mask & (1u << cls)) {
      for (cudaEvent_t* e : {&a, &b}) {
        if (!p->pool.empty()) { *e = p->pool.back(); p->pool.pop_back(); }
        else if (cudaEventCreate(e) != cudaSuccess) { *e = nullptr; }
      }
      if (a && b) cudaEventRecord(a, st);
    }
  }
  // the scope holds `n` launches instead of one
  void launches(int n) { p->st[cls].launches += n - 1; }
  ~KScope() {
    if (a && b) {
      cudaEventRecord(b, st);
      p->pending.push_back({cls, a, b});
    } else {
      if (a) p->pool.push_back(a);
      if (b) p->pool.push_back(b);
    }
  }
};

void chol_prof_resolve(chol_handle* h);   // sum the pending event pairs
void chol_prof_free(chol_handle* h);

int chol_device_ensure(chol_handle* h);   // allocate and upload on first use

// CHOL_ESTATE unless the handle holds a factorization on the current device.
// Calls after chol_factor launch on whichever device is current, while the
// handle's buffers live on the device it was factored on; a mismatch would
// make kernels read another device's memory, so it is refused up front.
inline int chol_factored_here(const chol_handle* h) {
  if (!h->factored || !h->dev) return CHOL_ESTATE;
  int cur = -1;
  if (cudaGetDevice(&cur) != cudaSuccess) {
    cudaGetLastError();
    return CHOL_ECUDA;
  }
  return cur == h->dev->device ? CHOL_OK : CHOL_ESTATE;
}
int chol_dalloc(chol_handle* h, void** p, size_t bytes);
