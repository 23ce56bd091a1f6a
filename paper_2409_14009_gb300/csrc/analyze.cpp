// analyze.cpp -- host symbolic analysis and schedule construction.
//
// Sec. II of the paper defines the pieces computed here: the elimination tree
// (parent(j) = min{i > j : L_ij != 0}), supernodes (contiguous columns with the
// same structure; the maximal partition of Fig. 1), the supernodal elimination
// tree, and the relative indices relind(J, K) of Sec. II-A used to scatter the
// update matrix of J into its ancestor K. On top of those the level schedule
// and the task lists of the CUDA kernels are built once, here, on the host.
#include <algorithm>
#include <limits>
#include <array>
#include <cstring>
#include <new>
#include <numeric>
#include <queue>
#include <tuple>
#include <stdexcept>

#include "internal.h"

extern "C" void chol_default_options(chol_options* opt) {
  if (!opt) return;
  std::memset(opt, 0, sizeof(*opt));
  opt->precision = CHOL_PREC_FP64;
  opt->small_max_cols = 64;
  opt->small_max_panel = 4096;
  opt->block_cols = 64;
  opt->device_mem_cap = 0;
  opt->merge_growth = 0.0;
  opt->small_max_rows = 128;
  opt->pivot_tau = 1e-3;
  opt->static_pivot = 0;
  opt->persistent = 0;
  opt->use_graph = 0;
  opt->update_mode = CHOL_UPDATE_RL;
  opt->wait_polls = 0;
  opt->test_unreachable_flags = 0;
}

namespace {

int validate(int32_t n, const int64_t* colptr, const int32_t* rowind, const int32_t* perm,
             const chol_options* opt) {
  if (n < 0) return -1;
  if (!colptr) return -2;
  if (n > 0 && !rowind && colptr[n] > 0) return -3;
  if (colptr[0] != 0) return -2;
  for (int32_t j = 0; j < n; ++j)
    if (colptr[j + 1] < colptr[j]) return -2;
  for (int32_t j = 0; j < n; ++j) {
    int64_t a = colptr[j], b = colptr[j + 1];
    if (a == b || rowind[a] != j) return -3;  // diagonal first and present
    for (int64_t t = a + 1; t < b; ++t)
      if (rowind[t] <= rowind[t - 1] || rowind[t] >= n) return -3;
  }
  if (perm) {
    std::vector<char> seen(n, 0);
    for (int32_t i = 0; i < n; ++i) {
      if (perm[i] < 0 || perm[i] >= n || seen[perm[i]]) return -4;
      seen[perm[i]] = 1;
    }
  }
  if (opt) {
    if (opt->precision < CHOL_PREC_FP64 || opt->precision > CHOL_PREC_BF16) return -5;
    if (!(opt->pivot_tau > 0.0) || opt->pivot_tau >= 1.0) return -5;
    if (opt->static_pivot != 0 && opt->static_pivot != 1) return -5;
    // tensor-core K chunks are 32 (tf32) / 64 (bf16) wide and must not cross a column step
    if (opt->precision == CHOL_PREC_TF32 && opt->block_cols % 32 != 0) return -5;
    if (opt->precision == CHOL_PREC_BF16 && opt->block_cols % 64 != 0) return -5;
    if (opt->small_max_cols < 1 || opt->small_max_panel < 1 || opt->small_max_panel > 24576) return -5;
    if (opt->persistent != 0 && opt->persistent != 1) return -5;
    if (opt->use_graph != 0 && opt->use_graph != 1) return -5;
    if (opt->update_mode != CHOL_UPDATE_RL && opt->update_mode != CHOL_UPDATE_RLB) return -5;
    if (opt->update_mode == CHOL_UPDATE_RLB &&
        (opt->precision != CHOL_PREC_FP64 || opt->persistent || opt->small_max_rows > kRlbSmallRows))
      return -5;
    if (opt->block_cols < 8 || opt->block_cols > 64) return -5;
    if (opt->device_mem_cap < 0) return -5;
    if (!(opt->merge_growth >= 0.0) || opt->merge_growth > 100.0) return -5;
    if (opt->small_max_rows < 1) return -5;
  }
  return 0;
}

// Supernodal elimination tree of a contiguous partition: parent of J = the
// supernode holding parent(last column of J).
void supernode_tree(int32_t n, const std::vector<int32_t>& sptr, const std::vector<int32_t>& parent,
                    std::vector<int32_t>& sparent) {
  const int32_t ns = (int32_t)sptr.size() - 1;
  std::vector<int32_t> snode_of(n);
  for (int32_t J = 0; J < ns; ++J)
    for (int32_t j = sptr[J]; j < sptr[J + 1]; ++j) snode_of[j] = J;
  sparent.assign(ns, -1);
  for (int32_t J = 0; J < ns; ++J) {
    int32_t p = parent[sptr[J + 1] - 1];
    sparent[J] = p >= 0 ? snode_of[p] : -1;
  }
}

// struct(J) for every supernode of a partition: J's columns, then the rows
// below J of B's columns in J and of the children's structures, ascending.
// For the maximal partition this is exactly struct(first column of J); for a
// merged one it is the union of the structures of J's columns.
void build_structs(int32_t n, const std::vector<int32_t>& sptr, const std::vector<int32_t>& sparent,
                   const std::vector<int64_t>& bp, const std::vector<std::pair<int32_t, int64_t>>& ent,
                   std::vector<int64_t>& rowptr, std::vector<int32_t>& rows) {
  const int32_t ns = (int32_t)sptr.size() - 1;
  std::vector<int32_t> chead(ns, -1), cnext(ns, -1);
  for (int32_t J = ns - 1; J >= 0; --J)
    if (sparent[J] >= 0) {
      cnext[J] = chead[sparent[J]];
      chead[sparent[J]] = J;
    }
  rowptr.assign(ns + 1, 0);
  rows.clear();
  std::vector<int32_t> mark(n, -1), buf;
  for (int32_t J = 0; J < ns; ++J) {
    const int32_t f = sptr[J], l = sptr[J + 1] - 1;
    buf.clear();
    for (int32_t j = f; j <= l; ++j) buf.push_back(j);
    const size_t first_off = buf.size();
    for (int32_t j = f; j <= l; ++j)
      for (int64_t t = bp[j]; t < bp[j + 1]; ++t) {
        int32_t i = ent[t].first;
        if (i > l && mark[i] != J) { mark[i] = J; buf.push_back(i); }
      }
    for (int32_t C = chead[J]; C != -1; C = cnext[C])
      for (int64_t t = rowptr[C]; t < rowptr[C + 1]; ++t) {
        int32_t i = rows[t];
        if (i > l && mark[i] != J) { mark[i] = J; buf.push_back(i); }
      }
    std::sort(buf.begin() + first_off, buf.end());
    rows.insert(rows.end(), buf.begin(), buf.end());
    rowptr[J + 1] = (int64_t)rows.size();
  }
}

// Stored entries of a supernode with s columns and len rows (lower trapezoid).
inline double stored_entries(double s, double len) { return s * len - s * (s - 1.0) / 2.0; }

// Relaxed supernode merging (Sec. IV setup): repeatedly merge the adjacent pair
// (J, P) with P = parent(J) = the next supernode in column order that adds the
// fewest explicit zeros (ties: smaller first column of J), while the cumulative
// added zeros stay within the budget. The merged structure is J's columns plus
// struct(P), because struct(J) minus J's columns lies in struct(P).
void relaxed_merge(const std::vector<int32_t>& csptr, const std::vector<int32_t>& csparent,
                   const std::vector<int64_t>& crowptr, double budget, std::vector<int32_t>& sptr) {
  const int32_t ns = (int32_t)csptr.size() - 1;
  std::vector<double> s(ns), len(ns);
  std::vector<int32_t> nxt(ns), prv(ns), rep(ns), ver(ns, 0), lastc(ns);
  std::vector<char> alive(ns, 1);
  for (int32_t J = 0; J < ns; ++J) {
    s[J] = csptr[J + 1] - csptr[J];
    len[J] = (double)(crowptr[J + 1] - crowptr[J]);
    nxt[J] = J + 1 < ns ? J + 1 : -1;
    prv[J] = J - 1;
    rep[J] = J;
    lastc[J] = J;   // canonical member holding the last column
  }
  auto find = [&](int32_t x) {
    while (rep[x] != x) {
      rep[x] = rep[rep[x]];
      x = rep[x];
    }
    return x;
  };
  // current parent of a live supernode = representative of the canonical parent
  // of its last canonical member
  auto cur_parent = [&](int32_t J) {
    const int32_t p = csparent[lastc[J]];
    return p < 0 ? -1 : find(p);
  };
  auto cost = [&](int32_t J, int32_t P) {
    return stored_entries(s[J] + s[P], s[J] + len[P]) - stored_entries(s[J], len[J]) -
           stored_entries(s[P], len[P]);
  };
  typedef std::tuple<double, int32_t, int32_t, int32_t> Item;  // cost, first column, J, version
  std::priority_queue<Item, std::vector<Item>, std::greater<Item>> pq;
  auto push = [&](int32_t J) {
    ++ver[J];
    const int32_t P = nxt[J];
    if (P >= 0 && cur_parent(J) == P) pq.push(Item(cost(J, P), csptr[J], J, ver[J]));
  };
  for (int32_t J = 0; J < ns; ++J) push(J);
  double total = 0.0;
  while (!pq.empty()) {
    const Item it = pq.top();
    pq.pop();
    const int32_t J = std::get<2>(it);
    if (!alive[J] || std::get<3>(it) != ver[J]) continue;
    const int32_t P = nxt[J];
    if (P < 0 || cur_parent(J) != P) continue;
    const double c = std::get<0>(it);
    if (total + c > budget) break;
    total += c;
    len[J] = s[J] + len[P];   // J absorbs P
    s[J] += s[P];
    lastc[J] = lastc[P];
    alive[P] = 0;
    rep[P] = J;
    nxt[J] = nxt[P];
    if (nxt[P] >= 0) prv[nxt[P]] = J;
    push(J);
    if (prv[J] >= 0) push(prv[J]);
  }
  sptr.clear();
  for (int32_t J = 0; J < ns; ++J)
    if (alive[J]) sptr.push_back(csptr[J]);
  sptr.push_back(csptr[ns]);
}


void build(chol_handle* h, const int64_t* colptr, const int32_t* rowind) {
  const int32_t n = h->n;
  const int64_t nnz = h->nnz_a;
  // ---- B = P A P^T: lower pattern, plus the A entry behind each B entry ----
  std::vector<int64_t> bp(n + 1, 0);
  for (int32_t c = 0; c < n; ++c)
    for (int64_t t = colptr[c]; t < colptr[c + 1]; ++t) {
      int32_t a = h->iperm[rowind[t]], b = h->iperm[c];
      bp[std::min(a, b) + 1]++;
    }
  for (int32_t j = 0; j < n; ++j) bp[j + 1] += bp[j];
  std::vector<std::pair<int32_t, int64_t>> ent(nnz);
  {
    std::vector<int64_t> nx(bp.begin(), bp.end() - 1);
    for (int32_t c = 0; c < n; ++c)
      for (int64_t t = colptr[c]; t < colptr[c + 1]; ++t) {
        int32_t a = h->iperm[rowind[t]], b = h->iperm[c];
        ent[nx[std::min(a, b)]++] = {std::max(a, b), t};
      }
    for (int32_t j = 0; j < n; ++j) std::sort(ent.begin() + bp[j], ent.begin() + bp[j + 1]);
  }
  // ---- permuted (row, col) of every entry of A, and the full-matrix CSR of A in
  //      its original ordering (both triangles) for binary64 residuals ----
  h->aij.assign(2 * nnz, 0);
  for (int32_t j = 0; j < n; ++j)
    for (int64_t t = bp[j]; t < bp[j + 1]; ++t) {
      h->aij[2 * ent[t].second] = ent[t].first;
      h->aij[2 * ent[t].second + 1] = j;
    }
  h->csr_ptr.assign(n + 1, 0);
  for (int32_t c = 0; c < n; ++c)
    for (int64_t t = colptr[c]; t < colptr[c + 1]; ++t) {
      h->csr_ptr[rowind[t] + 1]++;
      if (rowind[t] != c) h->csr_ptr[c + 1]++;
    }
  for (int32_t i = 0; i < n; ++i) h->csr_ptr[i + 1] += h->csr_ptr[i];
  h->csr_col.assign(h->csr_ptr[n], 0);
  h->csr_src.assign(h->csr_ptr[n], 0);
  {
    std::vector<int64_t> nx(h->csr_ptr.begin(), h->csr_ptr.end() - 1);
    for (int32_t c = 0; c < n; ++c)
      for (int64_t t = colptr[c]; t < colptr[c + 1]; ++t) {
        const int32_t r = rowind[t];
        h->csr_col[nx[r]] = c; h->csr_src[nx[r]++] = t;
        if (r != c) { h->csr_col[nx[c]] = r; h->csr_src[nx[c]++] = t; }
      }
  }
  // ---- row lists of B's strictly lower part (k < i with B_ik != 0) ----
  std::vector<int64_t> rp(n + 1, 0);
  for (int32_t j = 0; j < n; ++j)
    for (int64_t t = bp[j]; t < bp[j + 1]; ++t)
      if (ent[t].first > j) rp[ent[t].first + 1]++;
  for (int32_t i = 0; i < n; ++i) rp[i + 1] += rp[i];
  std::vector<int32_t> rl(rp[n]);
  {
    std::vector<int64_t> nx(rp.begin(), rp.end() - 1);
    for (int32_t j = 0; j < n; ++j)
      for (int64_t t = bp[j]; t < bp[j + 1]; ++t)
        if (ent[t].first > j) rl[nx[ent[t].first]++] = j;
  }
  // ---- elimination tree (Liu's algorithm with path compression) ----
  h->parent.assign(n, -1);
  {
    std::vector<int32_t> anc(n, -1);
    for (int32_t i = 0; i < n; ++i)
      for (int64_t t = rp[i]; t < rp[i + 1]; ++t) {
        int32_t r = rl[t];
        while (anc[r] != -1 && anc[r] != i) {
          int32_t nxt = anc[r];
          anc[r] = i;
          r = nxt;
        }
        if (anc[r] == -1) {
          anc[r] = i;
          h->parent[r] = i;
        }
      }
  }
  // ---- column counts by row subtrees: row i of L covers the etree paths from
  //      every k with B_ik != 0 up to i ----
  h->colcount.assign(n, 1);
  {
    std::vector<int32_t> mark(n, -1);
    for (int32_t i = 0; i < n; ++i) {
      mark[i] = i;
      for (int64_t t = rp[i]; t < rp[i + 1]; ++t)
        for (int32_t j = rl[t]; mark[j] != i; j = h->parent[j]) {
          mark[j] = i;
          h->colcount[j]++;
        }
    }
  }
  h->nnz_l = 0;
  h->flops = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    h->nnz_l += h->colcount[j];
    h->flops += (double)h->colcount[j] * (double)h->colcount[j];
  }
  // ---- maximal supernodes (Fig. 1): the canonical partition ----
  h->c_sptr.clear();
  for (int32_t j = 0; j < n; ++j) {
    bool join = j > 0 && h->parent[j - 1] == j && h->colcount[j - 1] == h->colcount[j] + 1;
    if (!join) h->c_sptr.push_back(j);
  }
  h->c_sptr.push_back(n);
  supernode_tree(n, h->c_sptr, h->parent, h->c_sparent);
  build_structs(n, h->c_sptr, h->c_sparent, bp, ent, h->c_rowptr, h->c_rows);
  for (size_t J = 0; J + 1 < h->c_sptr.size(); ++J)
    if (h->c_rowptr[J + 1] - h->c_rowptr[J] != h->colcount[h->c_sptr[J]])
      throw std::logic_error("structure/count mismatch");
  // ---- storage partition: canonical, or coarser after relaxed merging ----
  if (h->opt.merge_growth > 0.0) {
    relaxed_merge(h->c_sptr, h->c_sparent, h->c_rowptr, (double)h->nnz_l * h->opt.merge_growth, h->sptr);
    supernode_tree(n, h->sptr, h->parent, h->sparent);
    build_structs(n, h->sptr, h->sparent, bp, ent, h->rowptr, h->rows);
  } else {
    h->sptr = h->c_sptr;
    h->sparent = h->c_sparent;
    h->rowptr = h->c_rowptr;
    h->rows = h->c_rows;
  }
  const int32_t ns = (int32_t)h->sptr.size() - 1;
  h->ns = ns;
  std::vector<int32_t> snode_of(n);
  for (int32_t J = 0; J < ns; ++J)
    for (int32_t j = h->sptr[J]; j < h->sptr[J + 1]; ++j) snode_of[j] = J;
  std::vector<int32_t> chead(ns, -1), cnext(ns, -1);
  for (int32_t J = ns - 1; J >= 0; --J)
    if (h->sparent[J] >= 0) {
      cnext[J] = chead[h->sparent[J]];
      chead[h->sparent[J]] = J;
    }
  // ---- levels (height in the supernodal tree) ----
  h->level.assign(ns, 0);
  h->nlevels = ns > 0 ? 1 : 0;
  for (int32_t J = 0; J < ns; ++J) {
    int32_t lv = 0;
    for (int32_t C = chead[J]; C != -1; C = cnext[C]) lv = std::max(lv, h->level[C] + 1);
    h->level[J] = lv;
    h->nlevels = std::max(h->nlevels, lv + 1);
  }
  // ---- panel layout ----
  h->snodes.assign(ns, SnodeDev{});
  h->nnz_stored = 0;
  h->flops_stored = 0.0;
  int64_t off = 0;
  h->max_cols = 0;
  h->max_len = 0;
  for (int32_t J = 0; J < ns; ++J) {
    SnodeDev& d = h->snodes[J];
    d.f = h->sptr[J];
    d.s = h->sptr[J + 1] - h->sptr[J];
    d.len = (int32_t)(h->rowptr[J + 1] - h->rowptr[J]);
    d.roff = h->rowptr[J];
    d.loff = off;
    if (h->opt.precision == CHOL_PREC_FP64) {
      d.ld = (d.len + 1) & ~1;             // column-major, binary64
      off += (int64_t)d.ld * d.s;
      off = (off + 15) & ~int64_t(15);
    } else {
      d.ld = (d.s + 7) & ~7;               // row-major, binary32 (16-byte rows for TMA;
      off += (int64_t)d.ld * d.len;        // 8-element rows also fit the BF16 copy)
      off = (off + 31) & ~int64_t(31);
    }
    h->max_cols = std::max(h->max_cols, d.s);
    h->max_len = std::max(h->max_len, d.len);
    for (int32_t c = 0; c < d.s; ++c) {
      h->nnz_stored += d.len - c;
      h->flops_stored += (double)(d.len - c) * (double)(d.len - c);
    }
  }
  h->panel_doubles = off;
  // ---- value scatter map: A entry -> L storage position ----
  h->amap.assign(nnz, -1);
  {
    std::vector<int32_t> pos(n, -1);
    for (int32_t J = 0; J < ns; ++J) {
      const SnodeDev& d = h->snodes[J];
      const int32_t* r = h->rows.data() + d.roff;
      for (int32_t t = 0; t < d.len; ++t) pos[r[t]] = t;
      for (int32_t j = d.f; j < d.f + d.s; ++j)
        for (int64_t t = bp[j]; t < bp[j + 1]; ++t)
          h->amap[ent[t].second] = h->opt.precision == CHOL_PREC_FP64
                                       ? d.loff + (int64_t)(j - d.f) * d.ld + pos[ent[t].first]
                                       : d.loff + (int64_t)pos[ent[t].first] * d.ld + (j - d.f);
    }
  }
  // ---- relind pairs (J ascending, K ascending) ----
  h->rel_J.clear(); h->rel_K.clear(); h->rel_c0.clear(); h->rel_c1.clear();
  for (int32_t J = 0; J < ns; ++J) {
    const SnodeDev& d = h->snodes[J];
    const int32_t* r = h->rows.data() + d.roff;
    int32_t b = d.len - d.s;
    int32_t u = 0;
    while (u < b) {
      int32_t K = snode_of[r[d.s + u]];
      int32_t u1 = u;
      while (u1 < b && snode_of[r[d.s + u1]] == K) ++u1;
      h->rel_J.push_back(J); h->rel_K.push_back(K); h->rel_c0.push_back(u); h->rel_c1.push_back(u1);
      u = u1;
    }
  }
  const int64_t np = (int64_t)h->rel_J.size();
  h->pair_beg.assign(ns + 1, 0);
  for (int64_t p = 0; p < np; ++p) h->pair_beg[h->rel_J[p] + 1]++;
  for (int32_t J = 0; J < ns; ++J) h->pair_beg[J + 1] += h->pair_beg[J];
  h->relind_len = 0;
  for (int64_t p = 0; p < np; ++p)
    h->relind_len += (h->snodes[h->rel_J[p]].len - h->snodes[h->rel_J[p]].s) - h->rel_c0[p];
  // ---- level schedule and task lists ----
  const int nb = h->opt.block_cols;
  // solve super-step: one CTA solves this many diagonal columns. Binary64 keeps
  // it at one 64-column block (a single SM's FP64 rate is the limit); binary32
  // takes 256 to cut the number of dependent launches.
  const bool tc_modes = h->opt.precision == CHOL_PREC_TF32 || h->opt.precision == CHOL_PREC_BF16;
  const bool mixed = h->opt.precision != CHOL_PREC_FP64;
  const int tg = tc_modes ? kTileTC : kTile;
  std::vector<std::vector<int32_t>> by_level(h->nlevels);
  for (int32_t J = 0; J < ns; ++J) by_level[h->level[J]].push_back(J);
  // pairs by contributor level, then K, then J
  std::vector<std::vector<int64_t>> pairs_by_level(h->nlevels);
  for (int64_t p = 0; p < np; ++p) pairs_by_level[h->level[h->rel_J[p]]].push_back(p);
  std::vector<int64_t> kcount(ns, 0), sorted;   // scratch of the per-level sort by K
  std::vector<int32_t> touched;
  std::vector<std::array<int32_t, 3>> tile_segs;  // scratch: segments of one column tile
  h->levels.assign(h->nlevels, LevelPlan{});
  h->level_snodes.clear(); h->small_list.clear(); h->potrf_list.clear();
  h->trsm_tasks.clear(); h->gemm_tasks.clear(); h->syrk_tasks.clear();
  h->panel_items.clear(); h->panel_nflags = 0; h->panel_ntickets = 0;
  h->bpanel_tasks.clear(); h->tri_items.clear(); h->tri_nflags = 0;
  h->ssmall_list.clear();
  h->gemv_tasks.clear(); h->bpart_tasks.clear(); h->bred_tasks.clear();
  h->p_max = 0;
  h->split_slots_max = 0;
  h->asm_tasks.clear(); h->asm_segs.clear();
  h->n_small = h->n_large = 0;
  h->update_doubles = 0;
  h->update_doubles_rl = 0;
  h->w_rows_max = 0;
  for (int32_t lv = 0; lv < h->nlevels; ++lv) {
    LevelPlan& P = h->levels[lv];
    const auto& Js = by_level[lv];
    P.snode_b = (int32_t)h->level_snodes.size();
    P.snode_n = (int32_t)Js.size();
    h->level_snodes.insert(h->level_snodes.end(), Js.begin(), Js.end());
    std::vector<int32_t> large;
    P.small_b = (int32_t)h->small_list.size();
    P.small_max_panel = 0;
    int64_t uo = 0, wo = 0;
    for (int32_t J : Js) {
      SnodeDev& d = h->snodes[J];
      int32_t b = d.len - d.s;
      d.uoff = uo;
      uo += (int64_t)b * (h->opt.precision == CHOL_PREC_FP64 ? b : ((b + 7) & ~7));
      d.wpre = wo;
      wo += b;
      bool small = d.s <= h->opt.small_max_cols && (int64_t)d.len * d.s <= h->opt.small_max_panel &&
                   d.len <= h->opt.small_max_rows;
      if (small) {
        for (int32_t j = d.f; j < d.f + d.s; ++j) P.small_flops += (double)h->colcount[j] * h->colcount[j];
        P.small_bytes += 16.0 * (double)d.len * d.s + 8.0 * (double)b * (b + 1) / 2.0;
        h->small_list.push_back(J);
        P.small_max_panel = std::max(P.small_max_panel, d.len * d.s);
        h->n_small++;
      } else {
        large.push_back(J);
        h->n_large++;
      }
    }
    P.small_n = (int32_t)h->small_list.size() - P.small_b;
    P.u_doubles = uo;
    P.w_rows = wo;
    h->update_doubles_rl = std::max(h->update_doubles_rl, uo);
    if (h->opt.update_mode == CHOL_UPDATE_RL) h->update_doubles = std::max(h->update_doubles, uo);
    h->w_rows_max = std::max(h->w_rows_max, wo);
    int32_t maxs = 0;
    for (int32_t J : large) maxs = std::max(maxs, h->snodes[J].s);
    // binary64 TRSM tasks are half as tall: each CTA's substitution is DFMA-bound
    const int32_t trsm_rows = h->opt.precision == CHOL_PREC_FP64 ? kTrsmRowsHost / 2 : kTrsmRowsHost;
    // mixed modes: one panel launch per outer block of kTcOuter columns (its
    // 64-column POTRF/TRSM/update steps inside, tile by tile), then the update
    // of the columns right of it with K = the block
    for (int32_t ob = 0; mixed && ob < maxs; ob += kTcOuter) {
      StepRange st{};
      st.potrf_b = (int32_t)h->potrf_list.size();
      st.trsm_b = (int32_t)h->trsm_tasks.size();
      st.gemm_b = (int32_t)h->gemm_tasks.size();
      st.panel_b = (int32_t)h->panel_items.size();
      st.panel_ticket = h->panel_ntickets++;
      std::vector<int32_t> fb(large.size(), -1);
      for (int32_t dsub = 0; dsub < kTcOuter / 64; ++dsub)
        for (size_t q = 0; q < large.size(); ++q) {
          const SnodeDev& d = h->snodes[large[q]];
          if (d.s <= ob) continue;
          if (fb[q] < 0) { fb[q] = h->panel_nflags; h->panel_nflags += kTcOuter / 64; }
          const int32_t w = std::min(kTcOuter, d.s - ob);
          if (dsub * 64 < w) h->panel_items.push_back({large[q], ob + dsub * 64, dsub, fb[q]});
        }
      for (size_t q = 0; q < large.size(); ++q) {
        const SnodeDev& d = h->snodes[large[q]];
        if (d.s <= ob) continue;
        const int32_t w = std::min(kTcOuter, d.s - ob);
        // diagonal tiles hold the rows [ob, ob + w); every row below is in a tile
        for (int32_t r0 = ob + w; r0 < d.len; r0 += 64) h->panel_items.push_back({large[q], r0, -1, fb[q]});
        // flop convention: the block's columns contribute sum c^2; the part of
        // their outer products right of the block is the outer update's
        for (int32_t j = ob; j < ob + w; ++j) st.panel_flops += (double)(d.len - j) * (d.len - j);
      }
      st.panel_n = (int32_t)h->panel_items.size() - st.panel_b;
      st.ogemm_b = (int32_t)h->gemm_tasks.size();
      st.ok0 = ob;
      const int32_t oend = ob + kTcOuter;
      // the block's outer products right of it belong to the outer updates
      // (flop convention), whichever launch applies them
      for (int32_t J : large) {
        const SnodeDev& d = h->snodes[J];
        if (d.s <= oend) continue;
        const double w = (double)(d.s - oend), hgt = (double)(d.len - oend);
        st.panel_flops -= 2.0 * kTcOuter * (w * hgt - w * (w - 1.0) / 2.0);
      }
      // With the tensor-core updates, outer blocks go in pairs, so that most
      // of the trailing matrix is read and written once per 512 columns
      // instead of once per 256:
      // - the first block of a pair updates only the next block's columns
      //   (K = the block), which the next panel needs;
      // - the second updates every column right of it with K = both blocks
      //   (the next pair's two blocks' columns first, on the critical stream;
      //   the rest beside the next panels).
      // Otherwise (binary32 SIMT tiles) every block updates every column right
      // of it with K = the block, the next block's columns first. Every entry
      // receives the blocks' updates in block order either way.
      const bool pairs = h->opt.precision == CHOL_PREC_TF32 || h->opt.precision == CHOL_PREC_BF16;
      const bool second = pairs && ((ob / kTcOuter) & 1);
      const bool first = pairs && !second;
      const int32_t kbeg = second ? ob - kTcOuter : ob;
      st.okb = second ? 2 * kTcOuter : kTcOuter;
      // the critical stream waits for the previous side-stream update before
      // this step's outer update (with pairs: only where that update's columns
      // reach the side stream's)
      st.join_rest = pairs ? (second ? 1 : 0) : 1;
      const int32_t next_end = oend + (second ? 2 * kTcOuter : kTcOuter);
      for (int32_t J : large) {
        const SnodeDev& d = h->snodes[J];
        if (d.s <= oend) continue;
        const int32_t cend = first ? std::min(d.s, next_end) : d.s;
        const double kk = (double)std::min(st.okb, d.s - kbeg);
        const double w = (double)(cend - oend), hgt = (double)(d.len - oend);
        st.ogemm_flops += 2.0 * kk * (w * hgt - w * (w - 1.0) / 2.0);
      }
      // the columns the next panels need first
      for (int pass = 0; pass < 2; ++pass) {
        for (int32_t J : large) {
          const SnodeDev& d = h->snodes[J];
          if (d.s <= oend) continue;
          const int32_t cend = first ? std::min(d.s, next_end) : d.s;
          for (int32_t c0 = oend; c0 < cend; c0 += tg) {
            if ((pass == 0) != (c0 < next_end)) continue;
            for (int32_t r0 = c0; r0 < d.len; r0 += tg) h->gemm_tasks.push_back({J, kbeg, r0, c0});
          }
        }
        if (pass == 0) st.ogemm_next = (int32_t)h->gemm_tasks.size() - st.ogemm_b;
      }
      st.ogemm_n = (int32_t)h->gemm_tasks.size() - st.ogemm_b;
      P.steps.push_back(st);
    }
    for (int32_t k0 = 0; !mixed && k0 < maxs; k0 += nb) {
      StepRange st{};
      st.potrf_b = (int32_t)h->potrf_list.size();
      st.potrf_flops = st.trsm_flops = st.gemm_flops = st.ogemm_flops = 0.0;
      st.trsm_b = (int32_t)h->trsm_tasks.size();
      st.gemm_b = (int32_t)h->gemm_tasks.size();
      for (int32_t J : large) {
        const SnodeDev& d = h->snodes[J];
        if (d.s <= k0) continue;
        int32_t kb = std::min(nb, d.s - k0);
        h->potrf_list.push_back(J);  // k0 is implied by the step
        // flop convention sum c_j^2: a kb x kb Cholesky is sum_{j<kb} (kb-j)^2
        for (int32_t j = 0; j < kb; ++j) st.potrf_flops += (double)(kb - j) * (kb - j);
        const double below = (double)(d.len - k0 - kb);
        st.trsm_flops += below * (double)kb * (double)kb;   // kb divisions + 2*kb(kb-1)/2 per row
        for (int32_t r0 = k0 + kb; r0 < d.len; r0 += trsm_rows) h->trsm_tasks.push_back({J, k0, r0, 0});
        // trailing update: 2 kb flops per entry (r, c) with c in [k0+kb, s), r in [c, len)
        const int32_t cend = d.s;
        {
          const double w = (double)(cend - k0 - kb), hgt = (double)(d.len - k0 - kb);
          st.gemm_flops += 2.0 * kb * (w * hgt - w * (w - 1.0) / 2.0);
        }
      }
      // the step's own trailing update covers columns [k0+kb, cend) of each
      // supernode: first column tiles of all supernodes, then the others
      for (int pass = 0; pass < 2; ++pass) {
        for (int32_t J : large) {
          const SnodeDev& d = h->snodes[J];
          if (d.s <= k0) continue;
          const int32_t kb = std::min(nb, d.s - k0);
          for (int32_t c0 = k0 + kb; c0 < d.s; c0 += tg) {
            if ((pass == 0) != (c0 == k0 + kb)) continue;
            for (int32_t r0 = c0; r0 < d.len; r0 += tg) h->gemm_tasks.push_back({J, k0, r0, c0});
          }
        }
        if (pass == 0) st.gemm_next = (int32_t)h->gemm_tasks.size() - st.gemm_b;
      }
      st.potrf_n = (int32_t)h->potrf_list.size() - st.potrf_b;
      st.trsm_n = (int32_t)h->trsm_tasks.size() - st.trsm_b;
      st.gemm_n = (int32_t)h->gemm_tasks.size() - st.gemm_b;
      st.ogemm_b = (int32_t)h->gemm_tasks.size();
      st.ok0 = k0;
      st.okb = 0;
      st.ogemm_next = 0;
      st.ogemm_n = (int32_t)h->gemm_tasks.size() - st.ogemm_b;
      P.steps.push_back(st);
    }
    P.syrk_b = (int32_t)h->syrk_tasks.size();
    P.syrk_flops = 0.0;
    for (int32_t J : large) {
      const SnodeDev& d = h->snodes[J];
      int32_t b = d.len - d.s;
      P.syrk_flops += 2.0 * d.s * ((double)b * (b + 1) / 2.0);
      for (int32_t c0 = 0; c0 < b; c0 += tg)
        for (int32_t r0 = c0; r0 < b; r0 += tg) h->syrk_tasks.push_back({J, 0, r0, c0});
    }
    P.syrk_n = (int32_t)h->syrk_tasks.size() - P.syrk_b;
    // triangular solves over every supernode of the level: the diagonal
    // triangles as 64-row blocks in dependency order (one cooperative launch per
    // level and direction), then one panel product per level for the
    // off-diagonal rows; small supernodes take one warp each
    auto warp_solved = [&](int32_t J) {
      return h->snodes[J].s <= kSolveSmallCols && h->snodes[J].len <= kSolveSmallRows;
    };
    P.ssmall_b = (int32_t)h->ssmall_list.size();
    for (int32_t J : Js)
      if (warp_solved(J) && h->snodes[J].s <= 8) h->ssmall_list.push_back(J);
    P.ssmall8_n = (int32_t)h->ssmall_list.size() - P.ssmall_b;
    for (int32_t J : Js)
      if (warp_solved(J) && h->snodes[J].s > 8) h->ssmall_list.push_back(J);
    P.ssmall_n = (int32_t)h->ssmall_list.size() - P.ssmall_b;
    P.tri_b = (int32_t)h->tri_items.size();
    for (int32_t J : Js) {
      if (warp_solved(J)) continue;
      const int32_t nb = (h->snodes[J].s + 63) / 64;
      for (int32_t i = 0; i < nb; ++i) h->tri_items.push_back({J, i, nb, h->tri_nflags});
      h->tri_nflags += nb;
    }
    P.tri_n = (int32_t)h->tri_items.size() - P.tri_b;
    const int32_t gemv_rows = h->opt.precision == CHOL_PREC_FP64 ? 64 : 32;
    const int32_t bpanel_cols = h->opt.precision == CHOL_PREC_FP64 ? 16 : 64;
    P.gemv_b = (int32_t)h->gemv_tasks.size();
    P.bpanel_b = (int32_t)h->bpanel_tasks.size();
    // Binary64: a level with fewer tasks than kSplitTasks (the top of the tree:
    // few supernodes with long panels) splits each task's sum (gemv: over the
    // columns, bpanel: over the rows) into up to kMaxSplit parts of at least
    // kSplitMin, so that its products spread over the GPU. Parts write partial
    // sums to slots [slot, slot + parts) and the last part to finish adds them
    // in part order. Task fields: k0 = part | parts << 16; gemv: c0 = slot;
    // bpanel: r0 = slot.
    int32_t gemv_groups = 0, bpanel_groups = 0;
    for (int32_t J : Js) {
      const SnodeDev& d = h->snodes[J];
      const int32_t b = d.len - d.s;
      if (b <= 0 || warp_solved(J)) continue;
      gemv_groups += (b + gemv_rows - 1) / gemv_rows;
      bpanel_groups += (d.s + bpanel_cols - 1) / bpanel_cols;
    }
    const bool fp64 = h->opt.precision == CHOL_PREC_FP64;
    auto level_split = [&](int32_t groups) {
      if (!fp64 || groups <= 0 || groups >= kSplitTasks) return 1;
      return std::min(kMaxSplit, (kSplitTasks + groups - 1) / groups);
    };
    const int32_t gemv_split = level_split(gemv_groups), bpanel_split = level_split(bpanel_groups);
    int32_t gemv_slots = 0, bpanel_slots = 0;
    for (int32_t J : Js) {
      const SnodeDev& d = h->snodes[J];
      const int32_t b = d.len - d.s;
      if (b <= 0 || warp_solved(J)) continue;
      const int32_t gs = std::max(1, std::min(gemv_split, d.s / kSplitMin));
      for (int32_t r0 = 0; r0 < b; r0 += gemv_rows) {
        for (int32_t q = 0; q < gs; ++q) h->gemv_tasks.push_back({J, q | (gs << 16), r0, gs > 1 ? gemv_slots : 0});
        if (gs > 1) gemv_slots += gs;
      }
      const int32_t bs = std::max(1, std::min(bpanel_split, b / kSplitMin));
      for (int32_t c0 = 0; c0 < d.s; c0 += bpanel_cols) {
        for (int32_t q = 0; q < bs; ++q) h->bpanel_tasks.push_back({J, q | (bs << 16), bs > 1 ? bpanel_slots : 0, c0});
        if (bs > 1) bpanel_slots += bs;
      }
    }
    h->split_slots_max = std::max<int64_t>(h->split_slots_max, std::max(gemv_slots, bpanel_slots));
    P.gemv_n = (int32_t)h->gemv_tasks.size() - P.gemv_b;
    // row-major backward panel: 64-row chunks x 256-column tiles, then a reduction
    P.bpart_b = (int32_t)h->bpart_tasks.size();
    P.bred_b = (int32_t)h->bred_tasks.size();
    int64_t pp = 0;
    for (int32_t J : Js) {
      SnodeDev& d = h->snodes[J];
      const int32_t b = d.len - d.s;
      d.ppre = pp;
      if (b <= 0 || h->opt.precision == CHOL_PREC_FP64 || warp_solved(J)) continue;
      const int32_t nch = (b + 63) / 64;
      for (int32_t ch = 0; ch < nch; ++ch)
        for (int32_t c0 = 0; c0 < d.s; c0 += 256) h->bpart_tasks.push_back({J, ch, ch * 64, c0});
      for (int32_t c0 = 0; c0 < d.s; c0 += 256) h->bred_tasks.push_back({J, 0, 0, c0});
      pp += (int64_t)nch * d.s;
    }
    P.bpart_n = (int32_t)h->bpart_tasks.size() - P.bpart_b;
    P.bred_n = (int32_t)h->bred_tasks.size() - P.bred_b;
    h->p_max = std::max(h->p_max, pp);
    P.bpanel_n = (int32_t)h->bpanel_tasks.size() - P.bpanel_b;
    // assembly: group this level's pairs by target K (then J ascending)
    auto& pl = pairs_by_level[lv];
    {
      // pl is in J order already (pairs are generated by J), so a stable
      // counting sort by K gives (K, then J) order
      touched.clear();
      for (int64_t pz : pl)
        if (kcount[h->rel_K[pz]]++ == 0) touched.push_back(h->rel_K[pz]);
      std::sort(touched.begin(), touched.end());
      int64_t off = 0;
      for (int32_t K : touched) {
        const int64_t c = kcount[K];
        kcount[K] = off;
        off += c;
      }
      sorted.resize(pl.size());
      for (int64_t pz : pl) sorted[kcount[h->rel_K[pz]]++] = pz;
      pl.swap(sorted);
      for (int32_t K : touched) kcount[K] = 0;
    }
    P.asm_b = (int32_t)h->asm_tasks.size();
    P.asm_entries = 0.0;
    std::vector<AsmTask> warp_tasks;   // placed after the level's CTA tasks
    size_t q = 0;
    while (q < pl.size()) {
      int32_t K = h->rel_K[pl[q]];
      size_t q1 = q;
      while (q1 < pl.size() && h->rel_K[pl[q1]] == K) ++q1;
      const SnodeDev& dk = h->snodes[K];
      const int32_t* rk = h->rows.data() + dk.roff;
      for (int32_t t0 = 0; t0 < dk.s; t0 += kAsmCols) {
        int32_t t1 = std::min(dk.s, t0 + kAsmCols);
        // the segments of this column tile
        tile_segs.clear();
        for (size_t z = q; z < q1; ++z) {
          int64_t p = pl[z];
          const SnodeDev& dj = h->snodes[h->rel_J[p]];
          const int32_t* rj = h->rows.data() + dj.roff;
          int32_t ca = h->rel_c0[p], cb = h->rel_c1[p];
          while (ca < cb && rj[dj.s + ca] - dk.f < t0) ++ca;
          int32_t ce = ca;
          while (ce < cb && rj[dj.s + ce] - dk.f < t1) ++ce;
          if (ce > ca) {
            tile_segs.push_back({h->rel_J[p], ca, ce});
            const double bj = dj.len - dj.s;
            for (int32_t c = ca; c < ce; ++c) P.asm_entries += bj - c;
          }
        }
        if (tile_segs.empty()) continue;
        // split the row positions [t0, len) of K into chunks; a segment's rows
        // in a chunk are those between the chunk's first and next row indices
        for (int32_t p0 = t0; p0 < dk.len; p0 += kAsmPos) {
          const int32_t p1 = std::min(dk.len, p0 + kAsmPos);
          const int32_t r0 = rk[p0];
          const int32_t r1 = p1 < dk.len ? rk[p1] : std::numeric_limits<int32_t>::max();
          AsmTask task{K, t0, t1, (int32_t)h->asm_segs.size(), 0, p0, p1, 0};
          int64_t entries = 0;
          for (const auto& sgm : tile_segs) {
            const SnodeDev& dj = h->snodes[sgm[0]];
            const int32_t* ro = h->rows.data() + dj.roff + dj.s;
            const int32_t b = dj.len - dj.s;
            const int32_t ua = (int32_t)(std::lower_bound(ro + sgm[1], ro + b, r0) - ro);
            const int32_t ub = (int32_t)(std::lower_bound(ro + ua, ro + b, r1) - ro);
            if (ub > ua) {
              h->asm_segs.push_back({sgm[0], sgm[1], sgm[2], ua, ub, 0});
              entries += (int64_t)(ub - ua) * (sgm[2] - sgm[1]);
            }
          }
          task.seg_end = (int32_t)h->asm_segs.size();
          if (task.seg_end > task.seg_begin) {
            if (p1 - p0 <= kAsmWarpPos && entries <= kAsmWarpEntries) warp_tasks.push_back(task);
            else h->asm_tasks.push_back(task);
          }
        }
      }
      q = q1;
    }
    P.asm_n = (int32_t)h->asm_tasks.size() - P.asm_b;
    P.asmw_n = (int32_t)warp_tasks.size();
    h->asm_tasks.insert(h->asm_tasks.end(), warp_tasks.begin(), warp_tasks.end());
  }
  h->persist_levels.clear();
  h->small_panel_max = 0;
  for (const LevelPlan& P : h->levels) {
    h->persist_levels.push_back({P.small_b, P.small_n, P.asm_b, P.asm_n, P.asmw_n, 0});
    h->small_panel_max = std::max(h->small_panel_max, P.small_max_panel);
  }
  // one system unless chol_analyze_batch says otherwise
  h->sys_ptr = {0, n};
  h->sys_snode_ptr = {0, ns};
}

}  // namespace

extern "C" int chol_analyze(int32_t n, const int64_t* colptr, const int32_t* rowind,
                            const int32_t* perm, const chol_options* opt, chol_handle** out) {
  NvtxRange nvtx_range("chol_analyze");
  if (!out) return -6;
  *out = nullptr;
  int rc = validate(n, colptr, rowind, perm, opt);
  if (rc) return rc;
  chol_handle* h = new (std::nothrow) chol_handle();
  if (!h) return CHOL_ENOMEM;
  try {
    if (opt) h->opt = *opt; else chol_default_options(&h->opt);
    h->n = n;
    h->nnz_a = colptr[n];
    h->perm.resize(n);
    h->iperm.resize(n);
    for (int32_t i = 0; i < n; ++i) h->perm[i] = perm ? perm[i] : i;
    for (int32_t i = 0; i < n; ++i) h->iperm[h->perm[i]] = i;
    h->diagpos_orig.assign(colptr, colptr + n);   // diagonal = first entry of each column
    h->a_colptr.assign(colptr, colptr + n + 1);
    h->a_rowind.assign(rowind, rowind + colptr[n]);
    build(h, colptr, rowind);
  } catch (const std::bad_alloc&) {
    delete h;
    return CHOL_ENOMEM;
  } catch (...) {
    delete h;
    return CHOL_ESTATE;
  }
  *out = h;
  return CHOL_OK;
}

namespace {
void canonical_pairs(const chol_handle* h, std::vector<int32_t>& pj, std::vector<int32_t>& pk,
                     std::vector<int32_t>& pc0);
}

extern "C" int chol_analyze_batch(int32_t count, const int32_t* sys_ptr, const int64_t* colptr,
                                  const int32_t* rowind, const int32_t* perm, const chol_options* opt,
                                  chol_handle** out) {
  if (!out) return -7;
  *out = nullptr;
  if (count < 0) return -1;
  if (!sys_ptr || sys_ptr[0] != 0) return -2;
  for (int32_t q = 0; q < count; ++q)
    if (sys_ptr[q + 1] < sys_ptr[q]) return -2;
  const int32_t n = sys_ptr[count];
  int rc = validate(n, colptr, rowind, perm, opt);
  if (rc) return rc;
  // no coupling between systems, and perm keeps every system in place
  std::vector<int32_t> sys_of(n);
  for (int32_t q = 0; q < count; ++q)
    for (int32_t j = sys_ptr[q]; j < sys_ptr[q + 1]; ++j) sys_of[j] = q;
  for (int32_t c = 0; c < n; ++c)
    for (int64_t t = colptr[c]; t < colptr[c + 1]; ++t)
      if (sys_of[rowind[t]] != sys_of[c]) return -4;
  if (perm)
    for (int32_t i = 0; i < n; ++i)
      if (sys_of[perm[i]] != sys_of[i]) return -4;
  if ((rc = chol_analyze(n, colptr, rowind, perm, opt, out))) return rc;
  chol_handle* h = *out;
  h->sys_ptr.assign(sys_ptr, sys_ptr + count + 1);
  // storage supernodes never span systems (no coupling): map ranges
  h->sys_snode_ptr.assign(count + 1, 0);
  int32_t J = 0;
  for (int32_t q = 0; q < count; ++q) {
    while (J < h->ns && h->sptr[J] < sys_ptr[q + 1]) ++J;
    h->sys_snode_ptr[q + 1] = J;
  }
  return CHOL_OK;
}

// The batch forms of the factor and the solve: a batch handle is one
// block-diagonal system, so they are chol_factor and chol_solve.
extern "C" int chol_factor_batch(chol_handle* h, const double* values, void* stream) {
  return chol_factor(h, values, stream);
}

extern "C" int chol_solve_batch(chol_handle* h, double* b, int32_t nrhs, void* stream) {
  return chol_solve(h, b, nrhs, stream);
}

extern "C" int chol_get_info(const chol_handle* h, chol_info* info) {
  if (!h) return -1;
  if (!info) return -2;
  std::memset(info, 0, sizeof(*info));
  info->n = h->n;
  info->nsuper = (int32_t)h->c_sptr.size() - 1;
  info->nsuper_storage = h->ns;
  info->precision = h->opt.precision;
  info->nsys = (int32_t)h->sys_ptr.size() - 1;
  info->persistent_ok = h->n_large == 0 ? 1 : 0;
  info->persistent_threads = h->persist_threads;
  info->persistent_ctas_per_sm = h->persist_ctas;
  info->launch_mode = (h->opt.persistent ? 1 : 0) | (h->opt.use_graph ? 2 : 0);
  info->fp64_fallbacks = h->fp64_fallbacks;
  info->tc_launches_shallow = h->tc_shallow;
  info->tc_launches_deep = h->tc_deep;
  info->panel_launches = h->panel_launches;
  info->bounds_code = h->bounds_code;
  info->perturbed_pivots = h->perturbed_pivots;
  info->nnz_stored = h->nnz_stored;
  info->flops_stored = h->flops_stored;
  info->nlevels = h->nlevels;
  info->max_cols = h->max_cols;
  info->nnz_a = h->nnz_a;
  info->nnz_l = h->nnz_l;
  {
    std::vector<int32_t> pj, pk, pc0;
    canonical_pairs(h, pj, pk, pc0);
    info->n_relind_pairs = (int64_t)pj.size();
    int64_t tot = 0;
    for (size_t p = 0; p < pj.size(); ++p) {
      const int32_t J = pj[p];
      const int64_t b = (h->c_rowptr[J + 1] - h->c_rowptr[J]) - (h->c_sptr[J + 1] - h->c_sptr[J]);
      tot += b - pc0[p];
    }
    info->relind_len = tot;
  }
  info->panel_doubles = h->panel_doubles;
  info->update_doubles = h->update_doubles;
  info->flops = h->flops;
  info->n_small = h->n_small;
  info->n_large = h->n_large;
  return CHOL_OK;
}

namespace {

// (J, K) pairs of the canonical partition: K = every supernode owning a row of
// struct(J) below J's columns, ascending; c0 = first such row's index in
// struct(J) minus J's columns.
void canonical_pairs(const chol_handle* h, std::vector<int32_t>& pj, std::vector<int32_t>& pk,
                     std::vector<int32_t>& pc0) {
  const int32_t ns = (int32_t)h->c_sptr.size() - 1;
  std::vector<int32_t> snode_of(h->n);
  for (int32_t J = 0; J < ns; ++J)
    for (int32_t j = h->c_sptr[J]; j < h->c_sptr[J + 1]; ++j) snode_of[j] = J;
  for (int32_t J = 0; J < ns; ++J) {
    const int32_t s = h->c_sptr[J + 1] - h->c_sptr[J];
    const int32_t* r = h->c_rows.data() + h->c_rowptr[J];
    const int32_t len = (int32_t)(h->c_rowptr[J + 1] - h->c_rowptr[J]);
    int32_t prevK = -1;
    for (int32_t u = s; u < len; ++u) {
      const int32_t K = snode_of[r[u]];
      if (K == prevK) continue;
      prevK = K;
      pj.push_back(J); pk.push_back(K); pc0.push_back(u - s);
    }
  }
}

}  // namespace

extern "C" int chol_get_symbolic(const chol_handle* h, int32_t* parent, int32_t* colcount,
                                 int32_t* snode_ptr, int32_t* snode_parent, int64_t* row_ptr,
                                 int32_t* rows, int64_t* relind_ptr, int32_t* relind_target,
                                 int32_t* relind) {
  if (!h) return -1;
  auto cp = [](auto* dst, const auto& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  cp(parent, h->parent);
  cp(colcount, h->colcount);
  cp(snode_ptr, h->c_sptr);
  cp(snode_parent, h->c_sparent);
  cp(row_ptr, h->c_rowptr);
  cp(rows, h->c_rows);
  if (relind_ptr || relind_target || relind) {
    // relind(J, K) by its definition (Sec. II-A), on request: for each row i of
    // struct(J) from the first row owned by K on (all of them lie in struct(K)),
    // the distance of i from the bottom of struct(K).
    std::vector<int32_t> pj, pk, pc0;
    canonical_pairs(h, pj, pk, pc0);
    cp(relind_target, pk);
    std::vector<int32_t> pos(h->n, -1);
    int64_t off = 0;
    if (relind_ptr) relind_ptr[0] = 0;
    for (size_t p = 0; p < pj.size(); ++p) {
      const int32_t J = pj[p], K = pk[p];
      const int32_t sJ = h->c_sptr[J + 1] - h->c_sptr[J];
      const int32_t* rj = h->c_rows.data() + h->c_rowptr[J];
      const int32_t lenJ = (int32_t)(h->c_rowptr[J + 1] - h->c_rowptr[J]);
      const int32_t* rk = h->c_rows.data() + h->c_rowptr[K];
      const int32_t lenK = (int32_t)(h->c_rowptr[K + 1] - h->c_rowptr[K]);
      for (int32_t t = 0; t < lenK; ++t) pos[rk[t]] = t;
      for (int32_t u = sJ + pc0[p]; u < lenJ; ++u) {
        const int32_t ps = pos[rj[u]];
        if (relind) relind[off] = ps < 0 ? -1 : lenK - 1 - ps;
        ++off;
      }
      for (int32_t t = 0; t < lenK; ++t) pos[rk[t]] = -1;
      if (relind_ptr) relind_ptr[p + 1] = off;
    }
  }
  return CHOL_OK;
}

extern "C" int chol_get_partition(const chol_handle* h, int32_t* snode_ptr, int32_t* snode_parent,
                                  int64_t* row_ptr, int32_t* rows) {
  if (!h) return -1;
  auto cp = [](auto* dst, const auto& v) {
    if (dst && !v.empty()) std::memcpy(dst, v.data(), v.size() * sizeof(v[0]));
  };
  cp(snode_ptr, h->sptr);
  cp(snode_parent, h->sparent);
  cp(row_ptr, h->rowptr);
  cp(rows, h->rows);
  return CHOL_OK;
}

extern "C" void chol_destroy(chol_handle* h) {
  if (!h) return;
  chol_device_free(h);
  delete h;
}

extern "C" const char* chol_strerror(int code) {
  switch (code) {
    case CHOL_OK: return "success";
    case CHOL_ENOMEM: return "out of memory (host, device, or over the configured device cap)";
    case CHOL_ECUDA: return "a CUDA runtime call failed";
    case CHOL_ETIMEOUT: return "a bounded device wait ran out";
    case CHOL_ENOCONV: return "iterative refinement did not converge";
    case CHOL_ESTATE: return "call made in the wrong state";
    case CHOL_ENOTSUP: return "option combination not supported";
    case CHOL_ETOOBIG: return "problem exceeds the fixed-size workspace of this call";
    case CHOL_EBOUNDS: return "a range check of the bounds-checked build failed (the access was skipped)";
    default: break;
  }
  if (code > 0) return "matrix is not positive definite (return value = failing column, 1-based)";
  if (code < 0 && code > -100) return "invalid argument (return value = -argument position)";
  return "unknown error";
}
