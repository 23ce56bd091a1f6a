// internal.h -- handle layout shared by the host analysis and the CUDA driver.
#pragma once
#include <cstdint>
#include <vector>

#include "chol.h"

#include <cstdio>
#include <nvtx3/nvToolsExt.h>

// An NVTX range over a scope, on the host timeline of the calling thread, so
// that timeline tools and ncu's --nvtx filters can select a phase (e.g. one
// level of one factorization). A no-op unless such a tool is attached.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  NvtxRange(const char* prefix, long long index) {
    char buf[48];
    std::snprintf(buf, sizeof(buf), "%s %lld", prefix, index);
    nvtxRangePushA(buf);
  }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

// Per-supernode descriptor (device copy).
struct SnodeDev {
  int64_t loff;  // offset of the panel in L storage (doubles), column-major, leading dim ld
  int64_t roff;  // offset of struct(J) in the rows[] array
  int64_t uoff;  // offset of U_J (b x b, column-major, ld b) in the update workspace
  int64_t wpre;  // prefix of b over the level (solve workspace offset = wpre * nrhs)
  int64_t ppre;  // prefix over the level of ceil(b/64) * s (backward-panel partials, row-major)
  int32_t f;     // first column
  int32_t s;     // number of columns
  int32_t len;   // |struct(J)| (rows of the panel)
  int32_t ld;    // leading dimension of the panel
};

// Blocked large-supernode task: supernode J, column step k0, tile origin (r0, c0).
struct TileTask {
  int32_t J, k0, r0, c0;
};

// Pull-ordered assembly: one task owns columns [t0, t1) and row positions
// [p0, p1) of target supernode K (disjoint entries of K across tasks) and
// applies its segments in order; a segment is the part of U_J that lands
// there: columns [ca, cb), rows [ua, ub) (entries with row >= column only).
// The positions of a (K, column tile) pair are split into chunks of at most
// kAsmPos; the first chunk starts at t0 and holds every segment's columns.
struct AsmTask {
  int32_t K, t0, t1, seg_begin, seg_end, p0, p1, pad;
};
struct AsmSeg {
  int32_t J, ca, cb, ua, ub, pad;
};

// One column step of the blocked large-supernode path. In the tensor-core
// modes the trailing update is blocked twice: the step's own update (gemm_*)
// stays inside its kTcOuter-wide column block, and after the last step of a
// block the columns right of it are updated once with K = the block's width
// (ogemm_*, K range starting at ok0).
// binary64: the step's trailing tiles are ordered with the first column tile
// of every supernode first (gemm_next of them: the next step's block column),
// then the rest, so the rest can run beside the next POTRF and TRSM
// (one-step lookahead).
// Mixed modes: a step is one outer block [ok0, ok0 + kTcOuter) of columns; its
// POTRF, TRSM and in-block updates run in one panel launch (panel_*: 64-row
// tiles, see PanelItem; panel_ticket: the launch's work counter), then an
// outer update with K = okb from each task's k0 (ogemm_*, the columns the next
// panels need first). With tensor-core updates blocks go in pairs: the first
// block updates the next block's columns (okb = kTcOuter), the second every
// column right of the pair (okb = 2 kTcOuter); join_rest: wait for the previous
// side-stream update first.
struct StepRange {
  int32_t potrf_b, potrf_n, trsm_b, trsm_n, gemm_b, gemm_n, ogemm_b, ogemm_n, ok0, okb;
  int32_t gemm_next, ogemm_next;
  int32_t panel_b, panel_n, panel_ticket, join_rest;
  double potrf_flops, trsm_flops, gemm_flops, ogemm_flops, panel_flops;
};

// One 64-row tile of a supernode's outer column block in a panel launch:
// supernode J, first row r0 of the tile, d = index of the 64-column sub-block
// whose diagonal block the rows hold (-1: the rows lie below the outer block),
// fbase = first of J's four progress flags in the launch. Items are listed
// with every diagonal tile (by d, then J) before the tiles below.
struct PanelItem {
  int32_t J, r0, d, fbase;
};

// Blocked triangular-solve step k0 of one level: diagonal blocks of every
// supernode with s > k0, the row tiles below them (forward) and the column
// tiles left of them (backward).
// Triangular solve of one 64-row block of a supernode's diagonal triangle:
// supernode J, processing index i of nb blocks, flag index of block 0.
struct TriItemHost {
  int32_t J, i, nb, fbase;
};

struct LevelPlan {
  int32_t snode_b, snode_n;   // all supernodes of the level (in level_snodes)
  int32_t small_b, small_n;   // one-CTA supernodes (in small_list)
  int32_t small_max_panel;    // largest len*s among them (shared memory sizing)
  std::vector<StepRange> steps;
  int32_t syrk_b, syrk_n;     // U tiles (in syrk_tasks)
  int32_t asm_b, asm_n;       // assembly tasks, one CTA each
  int32_t asmw_n;             // then (from asm_b + asm_n) small tasks, one warp each
  int32_t tri_b, tri_n;       // diagonal-triangle solve items (in tri_items), dependency order
  int32_t ssmall_b, ssmall_n; // supernodes solved by one warp each (in ssmall_list),
  int32_t ssmall8_n;          // the first ssmall8_n of them with s <= 8
  int32_t gemv_b, gemv_n;     // forward-solve panel products (TileTask: J, r0)
  int32_t bpart_b, bpart_n;   // row-major backward panel, stage 1 (J, chunk, u0, c0)
  int32_t bred_b, bred_n;     // row-major backward panel, stage 2 (J, c0)
  int32_t bpanel_b, bpanel_n; // backward-solve panel column blocks (TileTask: J, c0)
  int64_t u_doubles;          // update workspace used by this level
  int64_t w_rows;             // sum of b over the level (solve workspace rows)
  double small_flops, syrk_flops, asm_entries;   // algorithmic work per launch
  double small_bytes;
};

// One level of the persistent (cooperative) factorization.
struct PersistLevel {
  int32_t small_b, small_n, asm_b, asm_n, asmw_n, pad;
};

struct DeviceState;  // defined in the CUDA driver
struct Profiler;     // defined in the CUDA driver

struct chol_handle {
  chol_options opt;
  int32_t n = 0;
  int64_t nnz_a = 0;
  std::vector<int32_t> perm, iperm;
  // symbolic: the canonical (maximal) partition of Fig. 1 ...
  std::vector<int32_t> parent, colcount;
  std::vector<int32_t> c_sptr, c_sparent;
  std::vector<int64_t> c_rowptr;
  std::vector<int32_t> c_rows;
  // ... and the storage partition the kernels use (canonical, or merged)
  int32_t ns = 0, nlevels = 0, max_cols = 0;
  std::vector<int32_t> sptr, sparent, level;
  std::vector<int64_t> rowptr;
  std::vector<int32_t> rows;
  std::vector<int64_t> cscmap;      // canonical CSC entry -> panel position (built on request)
  std::vector<SnodeDev> snodes;
  std::vector<int64_t> amap;        // entry t of A -> position in L storage
  std::vector<int32_t> aij;         // entry t of A -> (row, col) of P A P^T (pairs)
  std::vector<int64_t> csr_ptr;     // full symmetric A in its original ordering (CSR)
  std::vector<int32_t> csr_col;
  std::vector<int64_t> csr_src;     // CSR entry -> entry of the lower CSC input
  int32_t fp64_fallbacks = 0;
  int32_t tc_shallow = 0, tc_deep = 0, panel_launches = 0;   // launch shapes of the last factorization
  int32_t bounds_code = 0;          // CHOL_BOUNDS_CHECK build: first failed check of the last factorization
  std::vector<int64_t> a_colptr;    // the analyzed pattern of A (for gradients)
  std::vector<int32_t> a_rowind;
  bool selinv_valid = false;        // selected inverse of the current factor computed
  int32_t perturbed_pivots = 0;
  std::vector<int64_t> diagpos_orig;  // position of A_jj in the values array, per original column
  int64_t nnz_l = 0, panel_doubles = 0, update_doubles = 0, w_rows_max = 0, nnz_stored = 0;
  double flops = 0.0, flops_stored = 0.0;
  // (J, K) pairs: J updates ancestor K through U_J columns [c0, c1) (J ascending, K ascending)
  std::vector<int32_t> rel_J, rel_K, rel_c0, rel_c1;
  std::vector<int32_t> pair_beg;    // first (J, K) pair of every supernode (pairs are J-major)
  int64_t update_doubles_rl = 0;    // the RL update workspace (also sizes the Z_RR gathers)
  int64_t relind_len = 0;           // sum over pairs of (b_J - c0)
  int32_t max_len = 0;              // longest struct(J)
  // schedule
  std::vector<LevelPlan> levels;
  std::vector<int32_t> level_snodes, small_list, potrf_list;
  std::vector<TileTask> trsm_tasks, gemm_tasks, syrk_tasks, bpanel_tasks;
  std::vector<TriItemHost> tri_items;          // solve: diagonal-triangle blocks per level
  int32_t tri_nflags = 0;                      // solve: one flag per 64-row diagonal block
  std::vector<int32_t> ssmall_list;            // solve: one-warp supernodes per level
  std::vector<TileTask> gemv_tasks;             // solve: (J, r0) off-diagonal row tiles
  std::vector<TileTask> bpart_tasks, bred_tasks; // solve: row-major backward panel stages
  int64_t p_max = 0;                            // largest per-level partial-sum rows
  int64_t split_slots_max = 0;                  // binary64 solve: largest per-level count of split-sum slots
  std::vector<PanelItem> panel_items;           // mixed modes: panel-launch tiles, step by step
  int32_t panel_nflags = 0, panel_ntickets = 0; // progress flags and work counters of all panel launches
  std::vector<AsmTask> asm_tasks;
  std::vector<AsmSeg> asm_segs;
  int32_t n_small = 0, n_large = 0;
  // batches and launch configuration
  std::vector<int32_t> sys_ptr;       // count+1 column offsets of the systems
  std::vector<int32_t> sys_snode_ptr; // count+1 storage-supernode offsets of the systems
  std::vector<PersistLevel> persist_levels;
  int32_t small_panel_max = 0;        // largest len*s on the one-CTA kernel
  int32_t persist_threads = 128;      // chosen by chol_autotune
  int32_t persist_ctas = 0;           // CTAs per SM (0 = as many as fit)
  // numeric state
  bool factored = false;
  DeviceState* dev = nullptr;
  Profiler* prof = nullptr;
};

// Tile sizes shared by the schedule builder and the kernels.
constexpr int kTile = 64;        // SIMT GEMM/SYRK tile edge
constexpr int kTileTC = 128;     // tensor-core (tcgen05) GEMM/SYRK tile edge
constexpr int kTcOuter = 256;    // outer column block of the tensor-core trailing update
constexpr int kAsmCols = 32;     // assembly task width (target columns)
constexpr int kAsmPos = 64;      // assembly task height (row positions of the target)
constexpr int kAsmWarpPos = 256;       // warp-sized assembly tasks: at most this many positions
constexpr int kAsmWarpEntries = 4096;  // ... and this many entries over all segments
constexpr int kTrsmRowsHost = 32; // TRSM task height (rows; binary64 tasks take half)
constexpr int kSolveSmallCols = 32;   // supernodes solved by one warp: s <= 32 and
constexpr int kSolveSmallRows = 256;  // len <= 256
constexpr int kSplitTasks = 608;      // binary64 solve panel products: split levels with fewer tasks (4 x 152 SMs)
constexpr int kMaxSplit = 16;         // ... into at most this many parts
constexpr int kSplitMin = 128;        // ... of at least this many columns (gemv) or rows (bpanel)
constexpr int kRlbSmallRows = 1024;   // RLB: rows of a supernode on the one-CTA kernel (small_max_rows cap)

void chol_device_free(chol_handle* h);  // CUDA side
