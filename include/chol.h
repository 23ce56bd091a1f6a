/*
 * chol.h -- C ABI of the GB300 supernodal sparse Cholesky library.
 *
 * The library computes A = L L^T for a sparse symmetric positive definite A
 * (Karsavuran, Ng, Peyton, "GPU Accelerated Sparse Cholesky Factorization",
 * Sec. II: problem statement A = L L^T, elimination tree, supernodes, relative
 * indices) with the right-looking supernodal method RL of Sec. II-A: per
 * supernode J a dense POTRF of the diagonal block, a TRSM of the off-diagonal
 * panel, a SYRK update matrix, and the scatter-add of that update matrix into
 * the ancestor supernodes through relative indices. The triangular factors
 * then give the solution (Sec. I, abstract).
 *
 * Conventions shared by every call
 *   - A is passed once as a pattern: the lower triangle including the
 *     diagonal in compressed sparse column form, 0-based, row indices sorted
 *     ascending and unique in every column, every diagonal entry present.
 *   - perm is new->old: row/column i of P A P^T is row/column perm[i] of A.
 *     NULL means the identity. The library never reorders on its own.
 *   - Host arrays passed to chol_analyze are copied; the caller keeps them.
 *   - Device arrays (values, right-hand sides, gradients) belong to the
 *     caller and must stay valid until the call's work on `stream` is done.
 *   - `stream` is a cudaStream_t passed as void*; NULL is the legacy default
 *     stream. Work is ordered on that stream only.
 *   - Return codes: CHOL_OK (0); -k: argument k (1-based) is invalid;
 *     +j: A is not positive definite, the first failing pivot is column j
 *     (1-based) of P A P^T (LAPACK "info" convention); CHOL_E* below.
 *     No call aborts, prints, traps or asserts.
 *   - A handle is not thread-safe: calls on one handle must be serialized.
 */
#ifndef CHOL_H_
#define CHOL_H_

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct chol_handle chol_handle;

enum {
  CHOL_OK = 0,
  CHOL_ENOMEM = -1001,    /* host or device allocation failed (or over cap) */
  CHOL_ECUDA = -1002,     /* a CUDA runtime call failed */
  CHOL_ETIMEOUT = -1003,  /* a bounded device wait ran out */
  CHOL_ENOCONV = -1004,   /* iterative refinement did not reach the tolerance */
  CHOL_ESTATE = -1005,    /* call made in the wrong state (e.g. solve before factor) */
  CHOL_ENOTSUP = -1006,   /* option combination not supported */
  CHOL_ETOOBIG = -1007,   /* problem exceeds a fixed-size workspace */
  CHOL_EBOUNDS = -1008    /* CHOL_BOUNDS_CHECK build: a range check failed (access skipped) */
};

/*
 * Precision modes. The mixed modes scale A to D A D (D = diag(A)^{-1/2}, unit
 * diagonal) before rounding it to binary32, keep binary32 panels (row-major),
 * and win the accuracy back with binary64 iterative refinement
 * (chol_solve_refine): binary64 residual r = b - A x, binary64 update of x.
 * A diagonal block whose binary32 pivots fall below pivot_tau is refactored in
 * binary64. The paper computes in binary64 only (D-prefixed BLAS, Sec. II-A);
 * these modes are an extension.
 */
enum {
  CHOL_PREC_FP64 = 0,     /* every operation in IEEE binary64 */
  CHOL_PREC_FP32 = 1,     /* binary32 storage and SIMT arithmetic */
  CHOL_PREC_TF32 = 2,     /* binary32 storage; SYRK/GEMM tiles on tensor cores, TF32 operands */
                          /* (tcgen05 kind::tf32, operands truncated by the hardware), FP32 accumulate */
  CHOL_PREC_BF16 = 3      /* binary32 storage; SYRK/GEMM tiles on tensor cores, BF16 operands */
                          /* (round-to-nearest-even copies), FP32 accumulate */
};

typedef struct chol_options {
  int32_t precision;       /* CHOL_PREC_*; default CHOL_PREC_FP64 */
  int32_t small_max_cols;  /* supernodes with at most this many columns and at   */
  int32_t small_max_panel; /* most this many panel entries (len*cols, at most   */
                           /* 24576) take the one-CTA-per-supernode kernel;      */
                           /* default 64 / 4096                                  */
  int32_t block_cols;      /* column block of the blocked large-supernode path  */
                           /* (POTRF/TRSM/update step); default 64               */
  int64_t device_mem_cap;  /* refuse device allocations above this many bytes;  */
                           /* 0 = no cap (for testing the ENOMEM path)          */
  double merge_growth;     /* relaxed supernode merging budget (Sec. IV setup): */
                           /* merge adjacent (J, parent(J)) pairs, fewest added */
                           /* explicit zeros first (ties: smaller J), while the */
                           /* stored entries grow by at most this fraction of   */
                           /* nnz(L); 0 = off (the maximal partition, default)  */
  int32_t small_max_rows;  /* rows limit of the one-CTA kernel; default 128     */
  int32_t persistent;      /* 1 = one cooperative launch walks every level (needs */
                           /* every supernode on the one-CTA kernel, e.g. batches */
                           /* of small systems); 0 = one launch per level and     */
                           /* kernel class (default)                              */
  double pivot_tau;        /* mixed modes: a diagonal block with a binary32 pivot */
                           /* L_jj^2 below this (scaled matrix) is refactored in  */
                           /* binary64; default 1e-3                              */
  int32_t static_pivot;    /* mixed modes: 1 = a pivot d still below pivot_tau   */
                           /* after the binary64 redo becomes max(|d|, pivot_tau)  */
                           /* (counted), leaving the correction to               */
                           /* chol_solve_refine; 0 = report it as not positive   */
                           /* definite (default)                                 */
  int32_t use_graph;       /* 1 = the factorization's launches are captured in a  */
                           /* CUDA graph on the first chol_factor and replayed by */
                           /* the later ones (values are copied into the handle   */
                           /* first); 0 = direct launches (default)               */
  int32_t update_mode;     /* CHOL_UPDATE_RL (default): each supernode's update  */
                           /* matrix U_J = L_RJ L_RJ^T is formed in a workspace   */
                           /* and assembled into its ancestors by relative index  */
                           /* (Sec. II-A, RL), bitwise reproducible.              */
                           /* CHOL_UPDATE_RLB: the update products are subtracted */
                           /* straight into the ancestors' panels block by block  */
                           /* (the right-looking blocked variant, Sec. II-B): no  */
                           /* update workspace, atomic adds, so results agree to  */
                           /* rounding but not bit for bit between runs.         */
                           /* CHOL_PREC_FP64 and persistent = 0 only.            */
  int64_t wait_polls;      /* bounded device waits of the triangle solve give up */
                           /* after this many polls of a flag or hand-off word   */
                           /* (the solve is then                                 */
                           /* invalid and chol_check_waits reports              */
                           /* CHOL_ETIMEOUT); 0 = default 2^24 (seconds)        */
  int32_t test_unreachable_flags; /* testing the failure path only: 1 = the   */
                           /* triangle solve's dependent blocks wait for a flag  */
                           /* value that no block publishes, so every such wait  */
                           /* runs out after wait_polls polls; 0 = off (default) */
  int32_t reserved_opt;
} chol_options;

enum { CHOL_UPDATE_RL = 0, CHOL_UPDATE_RLB = 1 };

/*
 * A fill-reducing ordering for a general sparsity pattern (host only). The
 * paper orders its matrices with METIS nested dissection (Sec. IV); this is a
 * self-contained nested dissection: connected components separately; parts
 * above 64 vertices split by the smaller of two vertex separators (the
 * minimum vertex cover of a multilevel edge bisection's cut, and the trimmed
 * middle level of a breadth-first level structure from a pseudo-peripheral
 * vertex), sides first and separator last; small parts by minimum degree.
 * Deterministic: the ordering does not depend on the number of host threads
 * (large independent parts of the recursion run on threads of their own, up
 * to the hardware concurrency). O(nnz log n) work, O(nnz) memory.
 *   n       matrix order, >= 0
 *   colptr  host, n+1 entries (lower triangle incl. diagonal, as chol_analyze)
 *   rowind  host, colptr[n] entries
 *   perm    host, n entries, receives the ordering (new -> old), ready for
 *           chol_analyze
 * Errors: -1..-4 for invalid arguments (a row index above the diagonal or
 * out of range is -3), CHOL_ENOMEM.
 */
int chol_order_nd(int32_t n, const int64_t* colptr, const int32_t* rowind, int32_t* perm);

/* Fill *opt with the defaults. */
void chol_default_options(chol_options* opt);

/*
 * Symbolic analysis on the host (Sec. II): forms the pattern of P A P^T,
 * the elimination tree (parent(j) = min{i > j : L_ij != 0}), column counts,
 * the maximal supernode partition (columns j, j+1 share a supernode iff
 * parent(j) = j+1 and colcount(j) = colcount(j+1) + 1), the supernodal
 * elimination tree, the row structure of every supernode, the relative
 * indices relind(J, K) of Sec. II-A for every supernode J and every ancestor
 * K that J updates, the level schedule and the kernel task lists.
 *   n       matrix order, >= 0
 *   colptr  host, n+1 entries, colptr[0] = 0, non-decreasing
 *   rowind  host, colptr[n] entries (lower triangle incl. diagonal)
 *   perm    host, n entries (new->old) or NULL
 *   opt     host or NULL for defaults
 *   out     receives a new handle (library-owned; free with chol_destroy)
 * Errors: -1..-5 for invalid arguments (malformed CSC: -2 or -3; bad
 * permutation: -4), CHOL_ENOMEM. No device memory is touched here: device
 * buffers are created by the first chol_factor.
 */
int chol_analyze(int32_t n, const int64_t* colptr, const int32_t* rowind,
                 const int32_t* perm, const chol_options* opt, chol_handle** out);

/*
 * Numeric factorization A = L L^T (Sec. II-A, RL): scatters the values into
 * the supernodal panels, then, level by level of the supernodal elimination
 * tree (leaves first), POTRF of each diagonal block, TRSM of each panel,
 * SYRK of each update matrix U_J = L_RJ L_RJ^T and the relind scatter-add of
 * U_J into the ancestors (pull-ordered, atomic-free, deterministic). It ends
 * by inverting the 64x64 diagonal blocks the triangle solves multiply by
 * (binary64: the inverse; mixed modes: also the last-dependency products).
 *   values  device, colptr[n] doubles in the order of the analyzed rowind
 *   stream  cudaStream_t as void*
 * Returns CHOL_OK, +j (not positive definite at column j of P A P^T), or an
 * error. Synchronizes `stream` once at the end to read the status word.
 */
int chol_factor(chol_handle* h, const double* values, void* stream);

/*
 * Solve A X = B with the computed factor: X = P^T L^{-T} L^{-1} P B
 * (forward substitution over the levels leaves->root, backward substitution
 * root->leaves; the diagonal triangles of a level in one cooperative launch,
 * 64-row blocks handed from block to block and multiplied by their inverses).
 *   b      device, n x nrhs column-major (leading dimension n); overwritten by X
 *   nrhs   >= 0
 * Returns CHOL_ESTATE without a successful chol_factor. Asynchronous. The
 * blocks of a triangle wait (bounded, chol_options.wait_polls) for the blocks
 * they depend on; a wait that runs out leaves X invalid and is reported as
 * CHOL_ETIMEOUT by chol_check_waits, or by the next chol_factor or
 * chol_solve_refine on the handle. Calls on one handle must not overlap on the
 * GPU (they share workspaces). CHOL_ESTATE if the current device is not the
 * one the handle was factored on.
 */
int chol_solve(chol_handle* h, double* b, int32_t nrhs, void* stream);

/*
 * Report the bounded waits of the solves enqueued so far on this handle
 * (chol_solve, chol_solve_batch, chol_solve_noalloc, and the solves inside
 * chol_solve_refine). Synchronizes `stream` (the stream the solves ran on),
 * then returns CHOL_ETIMEOUT if any wait of a diagonal-triangle block gave up
 * since the last check (the solutions of those calls are invalid) and clears
 * the record; CHOL_OK otherwise. CHOL_ESTATE without a factorization on the
 * current device. The paper's solves are host-driven library calls with no
 * device-side waits; this check belongs to the cooperative triangle kernel.
 */
int chol_check_waits(chol_handle* h, void* stream);

/*
 * chol_solve without any device allocation. The paper has no counterpart: it
 * exists for callers that cannot call cudaMalloc once they are set up (a
 * process whose memory pool already owns the GPU, or a latency-bound loop in
 * which an allocation could stall on device-wide synchronization). Arguments,
 * layout and result are those of chol_solve; the handle must hold a factor.
 * Its workspaces live in one fixed device array of 2^21 doubles (16 MiB) that
 * every GPU loading the library keeps until the process exits; a problem needs
 * n + (largest per-level sum of off-diagonal supernode rows) doubles per
 * right-hand-side column and is refused with CHOL_ETOOBIG if one column does
 * not fit (wider blocks of right-hand sides are processed in chunks that fit).
 * All calls on a device share that array, so calls that overlap on the GPU
 * race; nothing in it needs to start at zero. The first call on each device
 * looks up the array's device address (cudaGetSymbolAddress, with that device
 * current), and again after the device's context was replaced (cudaDeviceReset):
 * make that first call before any stream capture. The device the handle was
 * factored on must be current (CHOL_ESTATE otherwise). Returns CHOL_ENOTSUP
 * for a mixed-precision handle. A bounded wait that runs out is reported by
 * chol_check_waits. Asynchronous.
 */
int chol_solve_noalloc(chol_handle* h, double* b, int32_t nrhs, void* stream);

/*
 * Factor, solve and log det for a caller whose data lives in host memory
 * (Sec. II-A factorization, then the triangular solves of Sec. I): copies the
 * values and the right-hand sides to the device, runs chol_factor, chol_solve
 * and (when logdet != NULL) chol_logdet on `stream`, copies X back and
 * synchronizes. The staging buffers (nnz(A) values, n x nrhs right-hand
 * sides) belong to the handle and are created by the first call (grown when
 * nrhs grows). Page-locked host buffers make the copies asynchronous and
 * faster; pageable ones also work.
 *   values  host, colptr[n] doubles in the order of the analyzed rowind
 *   b       host, n x nrhs column-major (ld n)
 *   x       host, n x nrhs column-major output (may be b)
 *   logdet  host, one double, or NULL
 * Returns what chol_factor returns (+j, errors), then solve errors; a bounded
 * wait of the solve that ran out gives CHOL_ETIMEOUT (x is then invalid).
 */
int chol_factor_solve_host(chol_handle* h, const double* values, const double* b, double* x, int32_t nrhs,
                           double* logdet, void* stream);

/*
 * log det A = 2 sum_j log L_jj, reduced in a fixed order (deterministic).
 *   out    host pointer to one double
 * Synchronizes `stream`.
 */
int chol_logdet(chol_handle* h, double* out, void* stream);

/*
 * Iteratively refined solve (mixed modes; in CHOL_PREC_FP64 it is one solve
 * plus the backward-error check). x_0 = solve(b); then, until the normwise
 * backward error eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf) of
 * every right-hand side is <= tol: r = b - A x in binary64 (with the values of
 * the last chol_factor), d = solve(r) with the low-precision factor, x += d in
 * binary64. When plain refinement stagnates (eta shrinks by less than 2x per
 * iteration) it switches to conjugate gradients in binary64 preconditioned by
 * the same factor.
 *   b        device, n x nrhs column-major (ld n), not modified
 *   x        device, n x nrhs column-major (ld n), output
 *   tol      target backward error (> 0)
 *   max_iter iteration cap (>= 1)
 *   iters    host, receives the iterations used (may be NULL)
 *   berr     host, nrhs doubles, receives the final eta per right-hand side (may be NULL)
 * Returns CHOL_OK, CHOL_ENOCONV if tol was not reached, or an error.
 * Synchronizes `stream` once per iteration.
 */
int chol_solve_refine(chol_handle* h, const double* b, double* x, int32_t nrhs, double tol,
                      int32_t max_iter, int32_t* iters, double* berr, void* stream);

/*
 * Selected inverse: zvals[t] = (A^{-1})_ij for every stored entry t = (i, j)
 * of the analyzed lower pattern of A (device, colptr[n] doubles). Computed
 * once per factorization, level by level of the supernodal tree from the
 * root down, every supernode of a level at once (dense blocks: T = L_JJ^{-1},
 * Uhat = L_RJ T, Z_RJ = -Z_RR Uhat with Z_RR gathered from the ancestors
 * through the relative positions, Z_JJ = T^T T - Uhat^T Z_RJ). The first call
 * builds the level plan and its workspaces (largest level's sum of s^2,
 * b s and 64 s doubles). CHOL_PREC_FP64 handles only (else CHOL_ENOTSUP).
 * Asynchronous.
 */
int chol_selected_inverse(chol_handle* h, double* zvals, void* stream);

/*
 * Adjoint of x = A^{-1} b and log det A for the loss
 *   l = sum_k w_k^T x_k + logdet_weight * log det A,   X = A^{-1} B.
 * Gives dl/dB = Xbar = A^{-1} W and the gradient with respect to the stored
 * lower entries of A (a_ij and a_ji move together):
 *   G = -Xbar X^T + logdet_weight A^{-1},  g_ii = G_ii,  g_ij = G_ij + G_ji.
 *   w     device, n x nrhs column-major (ld n)
 *   x     device, n x nrhs, the solution X of the forward solve
 *   bbar  device, n x nrhs output (dl/dB), or NULL (not returned)
 *   grad  device, colptr[n] doubles output, in the order of the analyzed rowind
 * Reuses the factor: two triangular solves, plus the selected inverse when
 * logdet_weight != 0. CHOL_PREC_FP64 handles only. Asynchronous.
 */
int chol_adjoint(chol_handle* h, const double* w, const double* x, int32_t nrhs, double logdet_weight,
                 double* bbar, double* grad, void* stream);

/* Sizes of the symbolic structure, for sizing the chol_get_symbolic arrays. */
typedef struct chol_info {
  int32_t n;
  int32_t nsuper;          /* number of supernodes */
  int32_t nlevels;         /* levels of the supernodal elimination tree */
  int32_t max_cols;        /* widest supernode */
  int64_t nnz_a;           /* entries of the lower triangle of A */
  int64_t nnz_l;           /* entries of L (diagonal included) */
  int64_t n_relind_pairs;  /* (J, K) pairs with relind(J, K) */
  int64_t relind_len;      /* total relind entries */
  int64_t panel_doubles;   /* device storage of the supernodal panels */
  int64_t update_doubles;  /* update-matrix workspace (largest level) */
  double flops;            /* sum_j c_j^2, c_j = nnz(L_{*,j}) incl. diagonal */
  int32_t n_small;         /* supernodes on the one-CTA kernel */
  int32_t n_large;         /* supernodes on the blocked path */
  int32_t nsuper_storage;  /* supernodes after relaxed merging (= nsuper if off) */
  int32_t reserved;
  int64_t nnz_stored;      /* stored factor entries incl. explicit zeros of merging */
  double flops_stored;     /* sum over stored columns of their stored count^2 */
  int32_t precision;       /* CHOL_PREC_* of the handle */
  int32_t fp64_fallbacks;  /* mixed modes: diagonal blocks refactored in binary64 by the last factor */
  int32_t perturbed_pivots; /* mixed modes with static_pivot: pivots raised to pivot_tau */
  int32_t nsys;            /* independent systems (chol_analyze_batch), else 1 */
  int32_t persistent_ok;   /* 1 if every supernode takes the one-CTA kernel */
  int32_t persistent_threads; /* launch shape of the persistent kernel (0 = default) */
  int32_t persistent_ctas_per_sm;
  int32_t launch_mode;     /* bit 0: persistent kernel in use, bit 1: CUDA-graph replay */
  int32_t tc_launches_shallow; /* tensor-core modes, last factorization: update launches on the */
  int32_t tc_launches_deep;    /* 2-stage ring (3 CTAs per SM, grids of >= 2 tiles per SM) and */
                               /* on the 6-stage ring (one CTA per SM)                        */
  int32_t panel_launches;      /* mixed modes, last factorization: panel launches (outer blocks) */
  int32_t bounds_code;         /* CHOL_BOUNDS_CHECK build: first failed check of the last */
                               /* factorization (1 task target, 2 task positions, 3 segment */
                               /* source, 4 segment range, 5 target row, 6 target column,  */
                               /* 7 value scatter); 0 otherwise                            */
} chol_info;

int chol_get_info(const chol_handle* h, chol_info* info);

/*
 * Batches of independent SPD systems (many small systems of uneven sizes).
 * The systems are passed as one block-diagonal matrix: system q owns rows and
 * columns [sys_ptr[q], sys_ptr[q+1]); colptr / rowind / perm use global
 * indices, no entry may couple two systems, and perm must map every system's
 * range onto itself. The analysis is that of the block-diagonal matrix (its
 * elimination tree is a forest, one tree per system), so every level of the
 * schedule batches the supernodes of all systems; chol_factor, chol_solve and
 * chol_solve_refine then work on the concatenated values and right-hand sides.
 *   count    number of systems, >= 0
 *   sys_ptr  host, count+1 offsets (sys_ptr[0] = 0, non-decreasing)
 * Errors as chol_analyze, plus -2 for a bad sys_ptr and -4 for an entry or a
 * permutation that crosses systems.
 */
int chol_analyze_batch(int32_t count, const int32_t* sys_ptr, const int64_t* colptr, const int32_t* rowind,
                       const int32_t* perm, const chol_options* opt, chol_handle** out);

/* log det of every system of a batch handle (out: host, count doubles; a
 * single-system handle fills out[0]). Fixed-order reductions. Synchronizes. */
int chol_logdet_batch(chol_handle* h, double* out, void* stream);

/* The batch forms of chol_factor and chol_solve, with the same arguments and
 * errors; any handle is accepted (a single-system handle is a batch of one).
 *   values  device, the entries of every system concatenated in the order of
 *           the block-diagonal matrix given to chol_analyze_batch
 *   b       device, n_total x nrhs column-major (system q in rows
 *           [sys_ptr[q], sys_ptr[q+1])), overwritten by the solutions
 * All systems are factored (solved) together, level by level, in one launch
 * sequence (or one graph replay / persistent launch, as analysed). */
int chol_factor_batch(chol_handle* h, const double* values, void* stream);
int chol_solve_batch(chol_handle* h, double* b, int32_t nrhs, void* stream);

/*
 * The bounds-checked build (compiled with -DCHOL_BOUNDS_CHECK; the package's
 * build(checked=True) makes it beside the normal library). Its kernels
 * range-check what comes from the plan before using it: every relind assembly
 * task (target supernode, row positions, segment range) and segment (source
 * supernode, rows and columns of U_J), every target row found by the binary
 * search (it must be present in the target's structure) and every target
 * column, and every position of the value scatter into the panels. A failed
 * check records its code (chol_info.bounds_code) and skips the access, and
 * chol_factor returns CHOL_EBOUNDS. (The paper's assembly is CPU code; this is
 * a debugging aid of the GPU form.)
 *
 * chol_test_corrupt_plan damages the host copy of a handle's plan before its
 * first chol_factor uploads it, for testing the checks without a fault:
 * kind 1: a segment's source supernode out of range; 2: a segment's rows past
 * U_J; 3: a task's row positions past the target; 4: a value's panel position
 * past the panels; 5: a warp-sized task's segment with a negative source.
 * CHOL_ESTATE after the first factorization; CHOL_ENOTSUP in the normal build
 * or when the plan has no task of that kind; -2 for an unknown kind.
 */
int chol_test_corrupt_plan(chol_handle* h, int32_t kind);

/*
 * Autotuner of the launch configuration: factors `values` (device, as for
 * chol_factor) once per candidate and keeps the fastest:
 * - level-by-level launches, with and without CUDA-graph replay;
 * - when every supernode takes the one-CTA kernel, the persistent
 *   cooperative kernel with 128 or 256 threads per CTA and 1 to 4 CTAs per SM.
 * The handle keeps the winner (reported by chol_get_info) and ends up
 * factored. Returns the status of the last factorization.
 */
int chol_autotune(chol_handle* h, const double* values, void* stream);

/*
 * Analysis-level autotuner for batches (the schedule of many small systems
 * picked by measurement; the paper's own choice is a fixed size threshold
 * between its CPU and GPU code paths, Sec. III-IV). Searches which
 * supernodes take the one-CTA kernel and how much relaxed merging to allow:
 * (small_max_cols, small_max_panel, small_max_rows) in {(64, 4096, 128),
 * (128, 16384, 256), (160, 24576, 512)} x merge_growth in {0, 0.1, 0.25}; for
 * each, analyzes a sample of the batch (every sample_every-th system), picks
 * the launch configuration with chol_autotune and times three factorizations;
 * keeps the fastest. Arguments as chol_analyze_batch, plus:
 *   values        device, the whole batch's values (the sample is copied out)
 *   base          options to start from (precision, update mode, ...) or NULL
 *   sample_every  >= 1 (1 = the whole batch)
 *   cache_path    a text file of earlier results, or NULL: a line whose key
 *                 (hash of the pattern, precision, update mode and device)
 *                 matches is used without searching; a new result is appended
 *   best          receives the chosen options (persistent, use_graph included)
 *   best_ms       the sample's factor time with them (may be NULL)
 *   from_cache    1 if the cache answered (may be NULL)
 * The caller then analyzes the whole batch with *best (and may call
 * chol_autotune on it to fit the launch shape to the whole batch).
 * Errors: -1..-10 for invalid arguments, errors of the calls it makes.
 */
int chol_tune_batch(int32_t count, const int32_t* sys_ptr, const int64_t* colptr, const int32_t* rowind,
                    const int32_t* perm, const double* values, const chol_options* base, int32_t sample_every,
                    const char* cache_path, chol_options* best, double* best_ms, int32_t* from_cache, void* stream);

/*
 * Copy out the symbolic results (host arrays, sized from chol_info; any
 * pointer may be NULL to skip it):
 *   parent[n]            etree parent of each column of P A P^T (-1 = root)
 *   colcount[n]          nnz(L_{*,j}) including the diagonal
 *   snode_ptr[nsuper+1]  first column of each supernode
 *   snode_parent[nsuper] supernodal etree parent (-1 = root)
 *   row_ptr[nsuper+1]    offsets into rows[] (int64)
 *   rows[]               struct(J) ascending (J's own columns first)
 *   relind_ptr[pairs+1]  offsets into relind[] (int64); pairs are ordered by
 *                        J ascending, then K ascending
 *   relind_target[pairs] K of each pair
 *   relind[]             relind(J, K): for each row i of struct(J) ∩
 *                        struct(K), in ascending i, the distance of i from the
 *                        bottom of struct(K) (Sec. II-A definition)
 */
int chol_get_symbolic(const chol_handle* h, int32_t* parent, int32_t* colcount,
                      int32_t* snode_ptr, int32_t* snode_parent, int64_t* row_ptr,
                      int32_t* rows, int64_t* relind_ptr, int32_t* relind_target,
                      int32_t* relind);

/*
 * The storage partition actually used by the numeric kernels (the maximal
 * partition, or the coarser one after relaxed merging): snode_ptr[nsuper_storage+1],
 * snode_parent[nsuper_storage], row_ptr[nsuper_storage+1] and rows[] (struct of
 * each stored supernode: union of the structures of its columns). NULL skips.
 */
int chol_get_partition(const chol_handle* h, int32_t* snode_ptr, int32_t* snode_parent,
                       int64_t* row_ptr, int32_t* rows);

/*
 * Copy the factor to the host in compressed sparse column form of L (rows of
 * each column ascending, diagonal first): lp[n+1] (int64), li[nnz_l],
 * lx[nnz_l]. Synchronizes `stream`. CHOL_ESTATE before a factorization.
 */
int chol_get_factor(chol_handle* h, int64_t* lp, int32_t* li, double* lx, void* stream);

/*
 * Per-kernel-class launch statistics (tracing). Launch counts and the
 * algorithmic flops and bytes of every launch are always accumulated; device
 * time is measured with CUDA events on the launching stream only for the
 * classes whose bit is set in the mask given to chol_profile (bit k = class k
 * of chol_kernel_class). Times of asynchronous calls are resolved when the
 * stats are read (which synchronizes the handle's last stream).
 */
enum chol_kernel_class {
  CHOL_K_SCATTER = 0, CHOL_K_SMALL, CHOL_K_POTRF, CHOL_K_TRSM, CHOL_K_GEMM, CHOL_K_SYRK,
  CHOL_K_ASSEMBLE, CHOL_K_SOLVE_DIAG,
  CHOL_K_SELINV_INV,     /* selected inverse: L_JJ^{-1} (block inverses and their products) */
  CHOL_K_SOLVE_FASM, CHOL_K_SOLVE_BPANEL,
  CHOL_K_SELINV_GEMM,    /* selected inverse: Uhat, Z_RJ and Z_JJ products */
  CHOL_K_PERMUTE, CHOL_K_LOGDET, CHOL_K_SOLVE_GEMV,
  CHOL_K_SELINV_GATHER,  /* selected inverse: Z_RR gathered from the ancestors */
  CHOL_K_ADJOINT,        /* per-entry gradient */
  CHOL_K_PANEL,          /* mixed modes: POTRF, TRSM and in-block updates of an outer column block */
  CHOL_K_NCLASSES
};

typedef struct chol_kernel_stat {
  int64_t launches;   /* kernel launches of this class */
  double flops;       /* algorithmic floating-point operations of those launches */
  double bytes;       /* algorithmic DRAM bytes of those launches */
  double ms;          /* summed device time of the timed launches */
  int64_t timed;      /* how many launches were timed */
} chol_kernel_stat;

int chol_profile(chol_handle* h, uint32_t timing_mask);
/* out[CHOL_K_NCLASSES]; reset != 0 clears the counters after reading. */
int chol_get_stats(chol_handle* h, chol_kernel_stat* out, int32_t reset);

/*
 * Measured binary64 throughput of the current GPU (the paper has no
 * counterpart; a measurement aid for the roofline of the binary64 factor,
 * whose dense updates run on the FP64 FMA pipe). kind 0: DFMA, independent
 * fused multiply-add chains on every SM; kind 1: DMMA, mma.sync m8n8k4 f64.
 * Tries 8 and 16 independent chains per thread and 2, 4 and 6 CTAs of 256
 * threads per SM, each shape with reps + 1 timed launches of a few
 * milliseconds (the first a warm-up), and returns the best rate in *gflops
 * (2 flops per multiply-add) and, in *sm_ghz (may be NULL), the SM clock that
 * run actually had (SM cycles over wall time of one CTA; a long FP64 burst on
 * every SM can run below the maximum clock under the power limit; 0 for DMMA,
 * which does not record it). Allocates
 * and frees 24 bytes of device memory. Synchronizes `stream`.
 * Errors: -1 bad kind, -2 reps < 1, -3 gflops NULL, CHOL_ECUDA.
 */
int chol_probe_fp64(int32_t kind, int32_t reps, double* gflops, double* sm_ghz, void* stream);

/* Release the handle and all its device memory. NULL is a no-op. */
void chol_destroy(chol_handle* h);

/* Static description of a return code. */
const char* chol_strerror(int code);

#ifdef __cplusplus
}
#endif

#endif /* CHOL_H_ */
