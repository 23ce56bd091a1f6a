// analyze.cpp -- host symbolic analysis and schedule construction.
//
// Sec. II of the paper defines the pieces computed here: the elimination tree
// (parent(j) = min{i > j : L_ij != 0}), supernodes (contiguous columns with the
// same structure; the maximal partition of Fig. 1), the supernodal elimination
// tree, and the relative indices relind(J, K) of Sec. II-A used to scatter the
// update matrix of J into its ancestor K. On top of those the level schedule
// and the task lists of the CUDA kernels are built once, here, on the host.
#include <algorithm>
#include <cstring>
#include <new>
#include <numeric>
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
    if (opt->precision != CHOL_PREC_FP64) return -5;
    if (opt->small_max_cols < 1 || opt->small_max_panel < 1 || opt->small_max_panel > 4096) return -5;
    if (opt->block_cols < 8 || opt->block_cols > 64) return -5;
    if (opt->device_mem_cap < 0) return -5;
  }
  return 0;
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
  // ---- maximal supernodes and the supernodal tree ----
  h->sptr.clear();
  for (int32_t j = 0; j < n; ++j) {
    bool join = j > 0 && h->parent[j - 1] == j && h->colcount[j - 1] == h->colcount[j] + 1;
    if (!join) h->sptr.push_back(j);
  }
  h->sptr.push_back(n);
  const int32_t ns = (int32_t)h->sptr.size() - 1;
  h->ns = ns;
  std::vector<int32_t> snode_of(n);
  for (int32_t J = 0; J < ns; ++J)
    for (int32_t j = h->sptr[J]; j < h->sptr[J + 1]; ++j) snode_of[j] = J;
  h->sparent.assign(ns, -1);
  for (int32_t J = 0; J < ns; ++J) {
    int32_t p = h->parent[h->sptr[J + 1] - 1];
    h->sparent[J] = p >= 0 ? snode_of[p] : -1;
  }
  std::vector<int32_t> chead(ns, -1), cnext(ns, -1);
  for (int32_t J = ns - 1; J >= 0; --J)
    if (h->sparent[J] >= 0) {
      cnext[J] = chead[h->sparent[J]];
      chead[h->sparent[J]] = J;
    }
  // ---- struct(J): J's columns, B's rows below J, children's rows below J ----
  h->rowptr.assign(ns + 1, 0);
  for (int32_t J = 0; J < ns; ++J) h->rowptr[J + 1] = h->rowptr[J] + h->colcount[h->sptr[J]];
  h->rows.assign(h->rowptr[ns], 0);
  {
    std::vector<int32_t> mark(n, -1);
    for (int32_t J = 0; J < ns; ++J) {
      int32_t f = h->sptr[J], l = h->sptr[J + 1] - 1;
      int32_t* out = h->rows.data() + h->rowptr[J];
      int32_t cnt = 0;
      for (int32_t j = f; j <= l; ++j) out[cnt++] = j;
      int32_t first_off = cnt;
      for (int32_t j = f; j <= l; ++j)
        for (int64_t t = bp[j]; t < bp[j + 1]; ++t) {
          int32_t i = ent[t].first;
          if (i > l && mark[i] != J) { mark[i] = J; out[cnt++] = i; }
        }
      for (int32_t C = chead[J]; C != -1; C = cnext[C]) {
        const int32_t* cr = h->rows.data() + h->rowptr[C];
        int32_t clen = (int32_t)(h->rowptr[C + 1] - h->rowptr[C]);
        for (int32_t t = 0; t < clen; ++t) {
          int32_t i = cr[t];
          if (i > l && mark[i] != J) { mark[i] = J; out[cnt++] = i; }
        }
      }
      std::sort(out + first_off, out + cnt);
      if (cnt != h->colcount[f]) throw std::logic_error("structure/count mismatch");
    }
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
  int64_t off = 0;
  h->max_cols = 0;
  h->max_len = 0;
  for (int32_t J = 0; J < ns; ++J) {
    SnodeDev& d = h->snodes[J];
    d.f = h->sptr[J];
    d.s = h->sptr[J + 1] - h->sptr[J];
    d.len = (int32_t)(h->rowptr[J + 1] - h->rowptr[J]);
    d.ld = (d.len + 1) & ~1;
    d.roff = h->rowptr[J];
    d.loff = off;
    off += (int64_t)d.ld * d.s;
    off = (off + 15) & ~int64_t(15);
    h->max_cols = std::max(h->max_cols, d.s);
    h->max_len = std::max(h->max_len, d.len);
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
          h->amap[ent[t].second] = d.loff + (int64_t)(j - d.f) * d.ld + pos[ent[t].first];
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
  h->relind_len = 0;
  for (int64_t p = 0; p < np; ++p)
    h->relind_len += (h->snodes[h->rel_J[p]].len - h->snodes[h->rel_J[p]].s) - h->rel_c0[p];
  // ---- level schedule and task lists ----
  const int nb = h->opt.block_cols;
  std::vector<std::vector<int32_t>> by_level(h->nlevels);
  for (int32_t J = 0; J < ns; ++J) by_level[h->level[J]].push_back(J);
  // pairs by contributor level, then K, then J
  std::vector<std::vector<int64_t>> pairs_by_level(h->nlevels);
  for (int64_t p = 0; p < np; ++p) pairs_by_level[h->level[h->rel_J[p]]].push_back(p);
  h->levels.assign(h->nlevels, LevelPlan{});
  h->level_snodes.clear(); h->small_list.clear(); h->potrf_list.clear();
  h->trsm_tasks.clear(); h->gemm_tasks.clear(); h->syrk_tasks.clear();
  h->bpanel_tasks.clear(); h->sdiag_list.clear(); h->fupd_tasks.clear(); h->bupd_tasks.clear();
  h->asm_tasks.clear(); h->asm_segs.clear();
  h->n_small = h->n_large = 0;
  h->update_doubles = 0;
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
      uo += (int64_t)b * b;
      d.wpre = wo;
      wo += b;
      bool small = d.s <= h->opt.small_max_cols && (int64_t)d.len * d.s <= h->opt.small_max_panel;
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
    h->update_doubles = std::max(h->update_doubles, uo);
    h->w_rows_max = std::max(h->w_rows_max, wo);
    int32_t maxs = 0;
    for (int32_t J : large) maxs = std::max(maxs, h->snodes[J].s);
    for (int32_t k0 = 0; k0 < maxs; k0 += nb) {
      StepRange st{};
      st.potrf_b = (int32_t)h->potrf_list.size();
      st.potrf_flops = st.trsm_flops = st.gemm_flops = 0.0;
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
        for (int32_t r0 = k0 + kb; r0 < d.len; r0 += kTile) h->trsm_tasks.push_back({J, k0, r0, 0});
        for (int32_t c0 = k0 + kb; c0 < d.s; c0 += kTile)
          for (int32_t r0 = c0; r0 < d.len; r0 += kTile) h->gemm_tasks.push_back({J, k0, r0, c0});
        // trailing update: 2 kb flops per entry (r, c) with c in [k0+kb, s), r in [c, len)
        {
          const double w = (double)(d.s - k0 - kb), hgt = (double)(d.len - k0 - kb);
          st.gemm_flops += 2.0 * kb * (w * hgt - w * (w - 1.0) / 2.0);
        }
      }
      st.potrf_n = (int32_t)h->potrf_list.size() - st.potrf_b;
      st.trsm_n = (int32_t)h->trsm_tasks.size() - st.trsm_b;
      st.gemm_n = (int32_t)h->gemm_tasks.size() - st.gemm_b;
      P.steps.push_back(st);
    }
    P.syrk_b = (int32_t)h->syrk_tasks.size();
    P.syrk_flops = 0.0;
    for (int32_t J : large) {
      const SnodeDev& d = h->snodes[J];
      int32_t b = d.len - d.s;
      P.syrk_flops += 2.0 * d.s * ((double)b * (b + 1) / 2.0);
      for (int32_t c0 = 0; c0 < b; c0 += kTile)
        for (int32_t r0 = c0; r0 < b; r0 += kTile) h->syrk_tasks.push_back({J, 0, r0, c0});
    }
    P.syrk_n = (int32_t)h->syrk_tasks.size() - P.syrk_b;
    // blocked triangular solves over every supernode of the level
    int32_t maxs_all = 0;
    for (int32_t J : Js) maxs_all = std::max(maxs_all, h->snodes[J].s);
    for (int32_t k0 = 0; k0 < maxs_all; k0 += nb) {
      SolveStep st{};
      st.diag_b = (int32_t)h->sdiag_list.size();
      st.fupd_b = (int32_t)h->fupd_tasks.size();
      st.bupd_b = (int32_t)h->bupd_tasks.size();
      for (int32_t J : Js) {
        const SnodeDev& d = h->snodes[J];
        if (d.s <= k0) continue;
        int32_t kb = std::min(nb, d.s - k0);
        h->sdiag_list.push_back(J);
        for (int32_t r0 = k0 + kb; r0 < d.len; r0 += kTile) h->fupd_tasks.push_back({J, k0, r0, 0});
        for (int32_t c0 = 0; c0 < k0; c0 += kTile) h->bupd_tasks.push_back({J, k0, 0, c0});
      }
      st.diag_n = (int32_t)h->sdiag_list.size() - st.diag_b;
      st.fupd_n = (int32_t)h->fupd_tasks.size() - st.fupd_b;
      st.bupd_n = (int32_t)h->bupd_tasks.size() - st.bupd_b;
      P.ssteps.push_back(st);
    }
    P.bpanel_b = (int32_t)h->bpanel_tasks.size();
    for (int32_t J : Js) {
      const SnodeDev& d = h->snodes[J];
      if (d.len - d.s <= 0) continue;
      for (int32_t c0 = 0; c0 < d.s; c0 += kBwdCols) h->bpanel_tasks.push_back({J, 0, 0, c0});
    }
    P.bpanel_n = (int32_t)h->bpanel_tasks.size() - P.bpanel_b;
    // assembly: group this level's pairs by target K (then J ascending)
    auto& pl = pairs_by_level[lv];
    std::stable_sort(pl.begin(), pl.end(), [&](int64_t a, int64_t b) {
      if (h->rel_K[a] != h->rel_K[b]) return h->rel_K[a] < h->rel_K[b];
      return h->rel_J[a] < h->rel_J[b];
    });
    P.asm_b = (int32_t)h->asm_tasks.size();
    P.asm_entries = 0.0;
    size_t q = 0;
    while (q < pl.size()) {
      int32_t K = h->rel_K[pl[q]];
      size_t q1 = q;
      while (q1 < pl.size() && h->rel_K[pl[q1]] == K) ++q1;
      const SnodeDev& dk = h->snodes[K];
      for (int32_t t0 = 0; t0 < dk.s; t0 += kAsmCols) {
        int32_t t1 = std::min(dk.s, t0 + kAsmCols);
        AsmTask task{K, t0, t1, (int32_t)h->asm_segs.size(), 0, 0, 0, 0};
        for (size_t z = q; z < q1; ++z) {
          int64_t p = pl[z];
          const SnodeDev& dj = h->snodes[h->rel_J[p]];
          const int32_t* rj = h->rows.data() + dj.roff;
          int32_t ca = h->rel_c0[p], cb = h->rel_c1[p];
          while (ca < cb && rj[dj.s + ca] - dk.f < t0) ++ca;
          int32_t ce = ca;
          while (ce < cb && rj[dj.s + ce] - dk.f < t1) ++ce;
          if (ce > ca) {
            h->asm_segs.push_back({h->rel_J[p], ca, ce, 0});
            const double bj = dj.len - dj.s;
            for (int32_t c = ca; c < ce; ++c) P.asm_entries += bj - c;
          }
        }
        task.seg_end = (int32_t)h->asm_segs.size();
        if (task.seg_end > task.seg_begin) h->asm_tasks.push_back(task);
      }
      q = q1;
    }
    P.asm_n = (int32_t)h->asm_tasks.size() - P.asm_b;
  }
}

}  // namespace

extern "C" int chol_analyze(int32_t n, const int64_t* colptr, const int32_t* rowind,
                            const int32_t* perm, const chol_options* opt, chol_handle** out) {
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

extern "C" int chol_get_info(const chol_handle* h, chol_info* info) {
  if (!h) return -1;
  if (!info) return -2;
  std::memset(info, 0, sizeof(*info));
  info->n = h->n;
  info->nsuper = h->ns;
  info->nlevels = h->nlevels;
  info->max_cols = h->max_cols;
  info->nnz_a = h->nnz_a;
  info->nnz_l = h->nnz_l;
  info->n_relind_pairs = (int64_t)h->rel_J.size();
  info->relind_len = h->relind_len;
  info->panel_doubles = h->panel_doubles;
  info->update_doubles = h->update_doubles;
  info->flops = h->flops;
  info->n_small = h->n_small;
  info->n_large = h->n_large;
  return CHOL_OK;
}

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
  cp(snode_ptr, h->sptr);
  cp(snode_parent, h->sparent);
  cp(row_ptr, h->rowptr);
  cp(rows, h->rows);
  cp(relind_target, h->rel_K);
  if (relind_ptr || relind) {
    // relind(J, K) by its definition, computed on request: for each row i of
    // struct(J) from the first row in K on (all of them lie in struct(K)), the
    // distance of i from the bottom of struct(K).
    const int64_t np = (int64_t)h->rel_J.size();
    int64_t off = 0;
    std::vector<int32_t> pos(h->n, -1);
    if (relind_ptr) relind_ptr[0] = 0;
    for (int64_t p = 0; p < np; ++p) {
      const SnodeDev& dj = h->snodes[h->rel_J[p]];
      const SnodeDev& dk = h->snodes[h->rel_K[p]];
      const int32_t* rj = h->rows.data() + dj.roff;
      const int32_t* rk = h->rows.data() + dk.roff;
      for (int32_t t = 0; t < dk.len; ++t) pos[rk[t]] = t;
      const int32_t b = dj.len - dj.s;
      for (int32_t u = h->rel_c0[p]; u < b; ++u) {
        int32_t ps = pos[rj[dj.s + u]];
        if (relind) relind[off] = ps < 0 ? -1 : dk.len - 1 - ps;
        ++off;
      }
      for (int32_t t = 0; t < dk.len; ++t) pos[rk[t]] = -1;
      if (relind_ptr) relind_ptr[p + 1] = off;
    }
  }
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
    default: break;
  }
  if (code > 0) return "matrix is not positive definite (return value = failing column, 1-based)";
  if (code < 0 && code > -100) return "invalid argument (return value = -argument position)";
  return "unknown error";
}
