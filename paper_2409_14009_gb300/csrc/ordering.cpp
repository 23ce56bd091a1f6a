// ordering.cpp -- a fill-reducing ordering for general sparsity patterns.
//
// The paper orders its matrices with METIS nested dissection (Sec. IV); that
// library is not part of this project. chol_order_nd computes a nested
// dissection ordering from the graph alone, so that user-supplied matrices
// with irregular structure can be factored without an external orderer:
// - each connected component is dissected on its own;
// - a part with more than kNdLeaf vertices is bisected by a multilevel edge
//   bisection: heavy-edge matching coarsens the graph to about kCoarse
//   vertices, greedy growing from several seeds partitions the coarsest
//   graph, and Fiduccia-Mattheyses passes refine the cut on the way back up;
// - the cut edges form a bipartite graph whose minimum vertex cover (Konig's
//   theorem, from a Hopcroft-Karp maximum matching) is the separator;
// - a level-structure separator (the middle breadth-first level from a
//   pseudo-peripheral vertex, trimmed to the vertices that touch the next
//   level) is the second candidate; the smaller of the two is used;
// - the two sides are ordered recursively, then the separator last;
// - parts of at most kNdLeaf vertices are ordered by minimum degree on their
//   own subgraph (exact degrees, eliminated vertices' neighbours joined into
//   cliques).
// Host only; deterministic (every tie goes to the smallest vertex index), and
// independent of the number of threads: large independent parts of the
// recursion run on threads of their own, their outputs joined in order.
#include <algorithm>
#include <atomic>
#include <climits>
#include <cstdint>
#include <cstdlib>
#include <exception>
#include <memory>
#include <set>
#include <system_error>
#include <thread>
#include <vector>

#include "internal.h"

namespace {

constexpr int kNdLeaf = 64;

struct Graph {
  std::vector<int64_t> ptr;
  std::vector<int32_t> adj;
};

// symmetric adjacency (no self loops) from the lower triangle in CSC
Graph build_graph(int32_t n, const int64_t* colptr, const int32_t* rowind) {
  std::vector<int64_t> deg(n + 1, 0);
  for (int32_t j = 0; j < n; ++j)
    for (int64_t t = colptr[j]; t < colptr[j + 1]; ++t)
      if (rowind[t] != j) { deg[j]++; deg[rowind[t]]++; }
  Graph g;
  g.ptr.assign(n + 1, 0);
  for (int32_t i = 0; i < n; ++i) g.ptr[i + 1] = g.ptr[i] + deg[i];
  g.adj.resize(g.ptr[n]);
  std::vector<int64_t> fill(g.ptr.begin(), g.ptr.end() - 1);
  for (int32_t j = 0; j < n; ++j)
    for (int64_t t = colptr[j]; t < colptr[j + 1]; ++t) {
      const int32_t i = rowind[t];
      if (i == j) continue;
      g.adj[fill[j]++] = i;
      g.adj[fill[i]++] = j;
    }
  return g;
}

// State shared by the dissection, which may run on several threads: a part
// (a set of vertices) is worked on by one thread at a time and parts are
// disjoint, so lvl_of and loc are only touched at the part's own vertices;
// part tags (unique per part) are read at neighbours too, hence atomic.
struct Shared {
  explicit Shared(int32_t n) : part(new std::atomic<int32_t>[n]), lvl_of(n, -1), loc(n, -1) {
    for (int32_t v = 0; v < n; ++v) part[v].store(0, std::memory_order_relaxed);
  }
  std::unique_ptr<std::atomic<int32_t>[]> part;
  std::vector<int32_t> lvl_of, loc;
  std::atomic<int32_t> next_tag{1};
  std::atomic<int> spare_threads{0};   // threads that may still be started
  int32_t tag_of(int32_t v) const { return part[v].load(std::memory_order_relaxed); }
  void set_tag(int32_t v, int32_t t) { part[v].store(t, std::memory_order_relaxed); }
};

// Breadth-first search from `root` inside the part marked `part == tag`;
// returns the vertices in visiting order and their levels.
void bfs(const Graph& g, Shared& sh, int32_t tag, int32_t root, std::vector<int32_t>& order,
         std::vector<int32_t>& level) {
  std::vector<int32_t>& lvl_of = sh.lvl_of;
  order.clear();
  level.clear();
  order.push_back(root);
  lvl_of[root] = 0;
  for (size_t h = 0; h < order.size(); ++h) {
    const int32_t v = order[h];
    level.push_back(lvl_of[v]);
    for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t) {
      const int32_t w = g.adj[t];
      if (sh.tag_of(w) == tag && lvl_of[w] < 0) {
        lvl_of[w] = lvl_of[v] + 1;
        order.push_back(w);
      }
    }
  }
}

// Minimum degree on a small vertex set (exact degrees, clique elimination).
void min_degree(const Graph& g, const std::vector<int32_t>& verts, std::vector<int32_t>& out) {
  const int m = (int)verts.size();
  std::vector<std::set<int>> nb(m);
  // map global -> local by sorted search
  std::vector<std::pair<int32_t, int>> key(m);
  for (int i = 0; i < m; ++i) key[i] = {verts[i], i};
  std::sort(key.begin(), key.end());
  auto loc = [&](int32_t v) -> int {
    auto it = std::lower_bound(key.begin(), key.end(), std::make_pair(v, -1));
    return (it != key.end() && it->first == v) ? it->second : -1;
  };
  for (int i = 0; i < m; ++i)
    for (int64_t t = g.ptr[verts[i]]; t < g.ptr[verts[i] + 1]; ++t) {
      const int j = loc(g.adj[t]);
      if (j >= 0 && j != i) nb[i].insert(j);
    }
  std::vector<char> done(m, 0);
  for (int step = 0; step < m; ++step) {
    int best = -1;
    for (int i = 0; i < m; ++i)
      if (!done[i] && (best < 0 || nb[i].size() < nb[best].size() ||
                       (nb[i].size() == nb[best].size() && verts[i] < verts[best])))
        best = i;
    done[best] = 1;
    out.push_back(verts[best]);
    std::vector<int> ns(nb[best].begin(), nb[best].end());
    for (int a : ns) {
      nb[a].erase(best);
      for (int c : ns)
        if (c != a) nb[a].insert(c);
    }
    nb[best].clear();
  }
}

// ---------------------------------------------------------------------------
// multilevel edge bisection

constexpr int kCoarse = 120;   // coarsening stops near this many vertices
constexpr int kSeeds = 6;      // greedy-growing seeds on the coarsest graph

struct WGraph {
  int32_t n = 0;
  std::vector<int64_t> ptr;
  std::vector<int32_t> adj, ew, vw;   // neighbours, edge weights, vertex weights
};

// the subgraph induced by `verts`, the part tagged `tag` (local index i is
// verts[i]); sh.loc is a global -> local scratch map, read only at the part's
// own vertices and reset to -1 before returning
WGraph subgraph(const Graph& g, const std::vector<int32_t>& verts, Shared& sh, int32_t tag) {
  std::vector<int32_t>& loc = sh.loc;
  WGraph s;
  s.n = (int32_t)verts.size();
  for (int32_t i = 0; i < s.n; ++i) loc[verts[i]] = i;
  s.ptr.assign(s.n + 1, 0);
  for (int32_t i = 0; i < s.n; ++i) {
    for (int64_t t = g.ptr[verts[i]]; t < g.ptr[verts[i] + 1]; ++t) {
      if (sh.tag_of(g.adj[t]) != tag) continue;
      s.adj.push_back(loc[g.adj[t]]);
      s.ew.push_back(1);
    }
    s.ptr[i + 1] = (int64_t)s.adj.size();
  }
  s.vw.assign(s.n, 1);
  for (int32_t v : verts) loc[v] = -1;
  return s;
}

// Heavy-edge matching: vertices visited by increasing degree, each matched to
// the unmatched neighbour across its heaviest edge. Returns false when the
// graph shrinks by less than 5%.
bool coarsen(const WGraph& g, WGraph& c, std::vector<int32_t>& cmap) {
  const int32_t n = g.n;
  int64_t tot = 0;
  for (int32_t w : g.vw) tot += w;
  const int64_t maxvw = std::max<int64_t>(1, (3 * tot) / (2 * kCoarse));
  std::vector<int32_t> order(n);
  for (int32_t i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int32_t x, int32_t y) {
    return g.ptr[x + 1] - g.ptr[x] < g.ptr[y + 1] - g.ptr[y];
  });
  std::vector<int32_t> match(n, -1);
  cmap.assign(n, -1);
  int32_t nc = 0;
  for (int32_t v : order) {
    if (match[v] >= 0) continue;
    int32_t best = -1, bw = -1;
    for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t) {
      const int32_t u = g.adj[t];
      if (match[u] >= 0 || u == v || g.vw[u] + g.vw[v] > maxvw) continue;
      if (g.ew[t] > bw || (g.ew[t] == bw && u < best)) { best = u; bw = g.ew[t]; }
    }
    if (best >= 0) {
      match[v] = best; match[best] = v;
      cmap[v] = cmap[best] = nc++;
    } else {
      match[v] = v;
      cmap[v] = nc++;
    }
  }
  if ((int64_t)nc * 20 > (int64_t)n * 19) return false;
  // members of each coarse vertex (one or two fine vertices)
  std::vector<int32_t> m0(nc, -1), m1(nc, -1);
  for (int32_t v = 0; v < n; ++v) (m0[cmap[v]] < 0 ? m0[cmap[v]] : m1[cmap[v]]) = v;
  c = WGraph();
  c.n = nc;
  c.ptr.assign(nc + 1, 0);
  c.vw.assign(nc, 0);
  std::vector<int64_t> pos(nc, -1);
  for (int32_t cv = 0; cv < nc; ++cv) {
    const int64_t start = (int64_t)c.adj.size();
    for (int32_t v : {m0[cv], m1[cv]}) {
      if (v < 0) continue;
      c.vw[cv] += g.vw[v];
      for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t) {
        const int32_t cu = cmap[g.adj[t]];
        if (cu == cv) continue;
        if (pos[cu] >= start && c.adj[pos[cu]] == cu) {
          c.ew[pos[cu]] += g.ew[t];
        } else {
          pos[cu] = (int64_t)c.adj.size();
          c.adj.push_back(cu);
          c.ew.push_back(g.ew[t]);
        }
      }
    }
    c.ptr[cv + 1] = (int64_t)c.adj.size();
  }
  return true;
}

int64_t cut_of(const WGraph& g, const std::vector<int8_t>& where) {
  int64_t cut = 0;
  for (int32_t v = 0; v < g.n; ++v)
    for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t)
      if (where[g.adj[t]] != where[v]) cut += g.ew[t];
  return cut / 2;
}

// Fiduccia-Mattheyses passes on a two-way cut: single vertex moves by best
// gain (edge weight to the other side minus to its own), each vertex moved at
// most once a pass, no side heavier than `maxside`; each pass is rolled back to
// its best prefix (smallest cut, then best balance). The candidates of each
// side sit in a binary heap ordered by (gain, then smallest vertex); an entry
// whose vertex changed since it was pushed is skipped when it reaches the top.
struct FmItem {
  int64_t gain;
  int32_t v;
  uint32_t stamp;
};
struct FmOrder {   // max-heap: larger gain first, then the smaller vertex
  bool operator()(const FmItem& a, const FmItem& b) const {
    return a.gain != b.gain ? a.gain < b.gain : a.v > b.v;
  }
};
void fm_refine(const WGraph& g, std::vector<int8_t>& where, int64_t maxside, int passes) {
  const int32_t n = g.n;
  std::vector<int64_t> id(n, 0), ed(n, 0);
  int64_t w[2] = {0, 0};
  for (int32_t v = 0; v < n; ++v) {
    w[where[v]] += g.vw[v];
    for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t) (where[g.adj[t]] == where[v] ? id[v] : ed[v]) += g.ew[t];
  }
  int64_t cut = 0;
  for (int32_t v = 0; v < n; ++v) cut += ed[v];
  cut /= 2;
  std::vector<char> locked(n, 0);
  std::vector<uint32_t> stamp(n, 0);
  std::vector<int32_t> moves;
  std::vector<FmItem> hv[2];
  auto move = [&](int32_t v) {
    const int s = where[v];
    where[v] = (int8_t)(1 - s);
    w[s] -= g.vw[v];
    w[1 - s] += g.vw[v];
    cut -= ed[v] - id[v];
    std::swap(id[v], ed[v]);
    for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t) {
      const int32_t u = g.adj[t];
      if (where[u] == where[v]) { id[u] += g.ew[t]; ed[u] -= g.ew[t]; }
      else { id[u] -= g.ew[t]; ed[u] += g.ew[t]; }
    }
  };
  auto push = [&](int32_t v) {
    auto& h = hv[where[v]];
    h.push_back({ed[v] - id[v], v, stamp[v]});
    std::push_heap(h.begin(), h.end(), FmOrder());
  };
  // the live top of side s, or null
  auto top = [&](int s) -> const FmItem* {
    auto& h = hv[s];
    while (!h.empty()) {
      const FmItem& f = h.front();
      if (f.stamp == stamp[f.v] && !locked[f.v] && where[f.v] == s && ed[f.v] > 0) return &h.front();
      std::pop_heap(h.begin(), h.end(), FmOrder());
      h.pop_back();
    }
    return nullptr;
  };
  const int limit = std::max(30, std::min(300, n / 50));
  for (int pass = 0; pass < passes; ++pass) {
    std::fill(locked.begin(), locked.end(), 0);
    hv[0].clear();
    hv[1].clear();
    for (int32_t v = 0; v < n; ++v)
      if (ed[v] > 0) { ++stamp[v]; push(v); }
    moves.clear();
    int64_t best_cut = cut, best_imb = std::llabs(w[0] - w[1]);
    size_t best_len = 0;
    int since = 0;
    while (since < limit) {
      int side = -1;
      const FmItem* pick = nullptr;
      for (int s = 0; s < 2; ++s) {
        const FmItem* f = top(s);
        if (!f) continue;
        if (w[1 - s] + g.vw[f->v] > maxside) continue;   // would unbalance
        if (w[s] > maxside) { side = s; pick = f; break; } // must shed weight
        if (side < 0 || f->gain > pick->gain || (f->gain == pick->gain && w[s] > w[side])) { side = s; pick = f; }
      }
      if (side < 0) break;
      const int32_t v = pick->v;
      std::pop_heap(hv[side].begin(), hv[side].end(), FmOrder());
      hv[side].pop_back();
      locked[v] = 1;
      move(v);
      for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t) {
        const int32_t u = g.adj[t];
        if (locked[u]) continue;
        ++stamp[u];   // older entries of u are stale
        if (ed[u] > 0) push(u);
      }
      moves.push_back(v);
      const int64_t imb = std::llabs(w[0] - w[1]);
      const bool balanced = w[0] <= maxside && w[1] <= maxside;
      if (balanced && (cut < best_cut || (cut == best_cut && imb < best_imb))) {
        best_cut = cut; best_imb = imb; best_len = moves.size(); since = 0;
      } else {
        ++since;
      }
    }
    for (size_t i = moves.size(); i > best_len; --i) move(moves[i - 1]);
    if (best_len == 0) break;
  }
}

// Greedy growing on the (small) coarsest graph: from each seed, side 0 grows
// breadth-first to half the weight; the best refined cut wins.
void initial_bisection(const WGraph& g, std::vector<int8_t>& where, int64_t maxside) {
  const int32_t n = g.n;
  int64_t tot = 0;
  for (int32_t w : g.vw) tot += w;
  int64_t best = -1;
  std::vector<int8_t> cur(n);
  std::vector<int32_t> queue;
  std::vector<char> seen(n);
  for (int k = 0; k < kSeeds; ++k) {
    const int32_t seed = (int32_t)(((int64_t)k * n) / kSeeds);
    std::fill(cur.begin(), cur.end(), (int8_t)1);
    std::fill(seen.begin(), seen.end(), 0);
    int64_t w0 = 0;
    queue.clear();
    queue.push_back(seed);
    seen[seed] = 1;
    int32_t next = 0;
    for (size_t h = 0; w0 * 2 < tot;) {
      if (h == queue.size()) {   // component exhausted: restart at the next unseen vertex
        while (next < n && seen[next]) ++next;
        if (next == n) break;
        queue.push_back(next);
        seen[next] = 1;
      }
      const int32_t v = queue[h++];
      if (w0 + g.vw[v] > maxside) continue;
      cur[v] = 0;
      w0 += g.vw[v];
      for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t)
        if (!seen[g.adj[t]]) { seen[g.adj[t]] = 1; queue.push_back(g.adj[t]); }
    }
    fm_refine(g, cur, maxside, 8);
    const int64_t c = cut_of(g, cur);
    if (best < 0 || c < best) { best = c; where = cur; }
  }
}

// Two-way partition of g (where[v] in {0, 1}) with both sides at most 55% of
// the weight.
void ml_bisect(const WGraph& g, std::vector<int8_t>& where) {
  int64_t tot = 0;
  for (int32_t w : g.vw) tot += w;
  const int64_t maxside = (tot * 11 + 19) / 20;
  std::vector<WGraph> levels;
  std::vector<std::vector<int32_t>> cmaps;
  const WGraph* cur = &g;
  while (cur->n > kCoarse) {
    WGraph c;
    std::vector<int32_t> cmap;
    if (!coarsen(*cur, c, cmap)) break;
    levels.push_back(std::move(c));
    cmaps.push_back(std::move(cmap));
    cur = &levels.back();
  }
  std::vector<int8_t> w;
  initial_bisection(*cur, w, maxside);
  for (size_t l = levels.size(); l-- > 0;) {
    const WGraph& fine = l == 0 ? g : levels[l - 1];
    std::vector<int8_t> fw(fine.n);
    for (int32_t v = 0; v < fine.n; ++v) fw[v] = w[cmaps[l][v]];
    fm_refine(fine, fw, maxside, 4);
    w.swap(fw);
  }
  where.swap(w);
}

// Minimum vertex cover of the cut edges (Konig's theorem): a Hopcroft-Karp
// maximum matching between side-0 and side-1 boundary vertices, then the
// alternating search from unmatched side-0 vertices; the cover is the
// unreached side-0 vertices and the reached side-1 vertices. Marks them 2.
void cover_cut(const WGraph& g, std::vector<int8_t>& where) {
  const int32_t n = g.n;
  std::vector<int32_t> idx(n, -1), L, R;
  for (int32_t v = 0; v < n; ++v) {
    bool bnd = false;
    for (int64_t t = g.ptr[v]; t < g.ptr[v + 1] && !bnd; ++t) bnd = where[g.adj[t]] != where[v];
    if (!bnd) continue;
    if (where[v] == 0) { idx[v] = (int32_t)L.size(); L.push_back(v); }
    else { idx[v] = (int32_t)R.size(); R.push_back(v); }
  }
  const int32_t nl = (int32_t)L.size(), nr = (int32_t)R.size();
  std::vector<int64_t> lp(nl + 1, 0);
  std::vector<int32_t> la;
  for (int32_t i = 0; i < nl; ++i) {
    const int32_t v = L[i];
    for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t)
      if (where[g.adj[t]] == 1) la.push_back(idx[g.adj[t]]);
    lp[i + 1] = (int64_t)la.size();
  }
  std::vector<int32_t> mateL(nl, -1), mateR(nr, -1), dist(nl), st, via;
  std::vector<int64_t> it(nl);
  const int32_t kInf = INT32_MAX;
  for (;;) {
    // layered search from the free side-0 vertices
    std::vector<int32_t> q;
    for (int32_t u = 0; u < nl; ++u) {
      dist[u] = mateL[u] < 0 ? 0 : kInf;
      if (mateL[u] < 0) q.push_back(u);
    }
    bool found = false;
    for (size_t h = 0; h < q.size(); ++h) {
      const int32_t u = q[h];
      for (int64_t t = lp[u]; t < lp[u + 1]; ++t) {
        const int32_t l2 = mateR[la[t]];
        if (l2 < 0) found = true;
        else if (dist[l2] == kInf) { dist[l2] = dist[u] + 1; q.push_back(l2); }
      }
    }
    if (!found) break;
    for (int32_t u = 0; u < nl; ++u) it[u] = lp[u];
    for (int32_t root = 0; root < nl; ++root) {
      if (mateL[root] >= 0) continue;
      st.assign(1, root);
      via.clear();
      while (!st.empty()) {
        const int32_t u = st.back();
        if (it[u] == lp[u + 1]) {   // dead end
          dist[u] = kInf;
          st.pop_back();
          if (!via.empty()) via.pop_back();
          continue;
        }
        const int32_t r = la[it[u]++];
        const int32_t l2 = mateR[r];
        if (l2 < 0) {   // augmenting path: flip it
          via.push_back(r);
          for (size_t i = 0; i < st.size(); ++i) { mateL[st[i]] = via[i]; mateR[via[i]] = st[i]; }
          break;
        }
        if (dist[l2] == dist[u] + 1) { via.push_back(r); st.push_back(l2); }
      }
    }
  }
  std::vector<char> reachL(nl, 0), reachR(nr, 0);
  std::vector<int32_t> q;
  for (int32_t u = 0; u < nl; ++u)
    if (mateL[u] < 0) { reachL[u] = 1; q.push_back(u); }
  for (size_t h = 0; h < q.size(); ++h) {
    const int32_t u = q[h];
    for (int64_t t = lp[u]; t < lp[u + 1]; ++t) {
      const int32_t r = la[t];
      if (reachR[r]) continue;
      reachR[r] = 1;
      const int32_t l2 = mateR[r];
      if (l2 >= 0 && !reachL[l2]) { reachL[l2] = 1; q.push_back(l2); }
    }
  }
  for (int32_t u = 0; u < nl; ++u)
    if (!reachL[u]) where[L[u]] = 2;
  for (int32_t r = 0; r < nr; ++r)
    if (reachR[r]) where[R[r]] = 2;
}

// Level-structure separator: breadth-first levels from a pseudo-peripheral
// vertex (the far end of repeated searches), cut where the running count
// passes half; the separator is the vertices of that level with a neighbour
// in the next one (the rest of the level joins side 0). Returns false when the
// structure is too shallow to cut.
bool level_separator(const WGraph& g, std::vector<int8_t>& where) {
  const int32_t n = g.n;
  std::vector<int32_t> lvl(n), order;
  auto search = [&](int32_t root) {
    std::fill(lvl.begin(), lvl.end(), -1);
    order.assign(1, root);
    lvl[root] = 0;
    for (size_t h = 0; h < order.size(); ++h) {
      const int32_t v = order[h];
      for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t)
        if (lvl[g.adj[t]] < 0) { lvl[g.adj[t]] = lvl[v] + 1; order.push_back(g.adj[t]); }
    }
    return lvl[order.back()];
  };
  int32_t root = 0;
  int depth = -1;
  for (int it = 0; it < 8; ++it) {
    const int d = search(root);
    if (d <= depth) break;
    depth = d;
    int32_t far = -1;
    int64_t fdeg = 0;
    for (int32_t v : order)
      if (lvl[v] == d) {
        const int64_t dg = g.ptr[v + 1] - g.ptr[v];
        if (far < 0 || dg < fdeg || (dg == fdeg && v < far)) { far = v; fdeg = dg; }
      }
    if (far == root) break;
    root = far;
  }
  const int d = search(root);
  if (d < 2) return false;
  std::vector<int64_t> cnt(d + 1, 0);
  for (int32_t v = 0; v < n; ++v) cnt[lvl[v]]++;
  int64_t run = 0;
  int mid = 1;
  for (int l = 0; l <= d; ++l) {
    run += cnt[l];
    if (2 * run >= n) { mid = l; break; }
  }
  mid = std::max(1, std::min(mid, d - 1));
  where.assign(n, 0);
  for (int32_t v = 0; v < n; ++v) {
    if (lvl[v] > mid) { where[v] = 1; continue; }
    if (lvl[v] < mid) continue;
    for (int64_t t = g.ptr[v]; t < g.ptr[v + 1]; ++t)
      if (lvl[g.adj[t]] > mid) { where[v] = 2; break; }
  }
  return true;
}

// A side of at least this many vertices may go to its own thread.
constexpr size_t kNdThreadMin = 4096;

void dissect(const Graph& g, Shared& sh, int32_t tag, std::vector<int32_t> verts, std::vector<int32_t>& out);

// Order one side of a split (possibly several components, each on its own).
void order_side(const Graph& g, Shared& sh, const std::vector<int32_t>& side, std::vector<int32_t>& out) {
  const int32_t stag = sh.next_tag.fetch_add(1);
  for (int32_t v : side) sh.set_tag(v, stag);
  for (int32_t v : side) sh.lvl_of[v] = -1;
  std::vector<int32_t> comp, clev;
  for (int32_t s : side) {
    if (sh.tag_of(s) != stag) continue;   // already placed in a component
    const int32_t ctag = sh.next_tag.fetch_add(1);
    bfs(g, sh, stag, s, comp, clev);
    for (int32_t v : comp) sh.set_tag(v, ctag);
    dissect(g, sh, ctag, comp, out);
  }
}

// Order the vertices of part `tag` (all connected), appending to `out`.
// The two sides of a split are independent: the second may run on a thread
// of its own (its output is appended after the first side's), so the
// ordering is the same with any number of threads.
void dissect(const Graph& g, Shared& sh, int32_t tag, std::vector<int32_t> verts, std::vector<int32_t>& out) {
  if ((int)verts.size() <= kNdLeaf) {
    min_degree(g, verts, out);
    return;
  }
  std::sort(verts.begin(), verts.end());
  // two candidate separators, the smaller one wins
  std::vector<int8_t> where, lw;
  {
    const WGraph s = subgraph(g, verts, sh, tag);
    ml_bisect(s, where);
    cover_cut(s, where);
    if (level_separator(s, lw) &&
        std::count(lw.begin(), lw.end(), (int8_t)2) < std::count(where.begin(), where.end(), (int8_t)2))
      where.swap(lw);
  }
  std::vector<int32_t> a, b, sep;
  for (size_t i = 0; i < verts.size(); ++i)
    (where[i] == 0 ? a : where[i] == 1 ? b : sep).push_back(verts[i]);
  if (a.empty() || b.empty() || 2 * sep.size() > verts.size()) {
    // no useful separator (nearly a clique): the order hardly matters here
    if ((int)verts.size() <= 16 * kNdLeaf) min_degree(g, verts, out);
    else out.insert(out.end(), verts.begin(), verts.end());
    return;
  }
  bool spawn = false;
  if (b.size() >= kNdThreadMin && a.size() >= kNdThreadMin) {
    int spare = sh.spare_threads.load();
    while (spare > 0 && !sh.spare_threads.compare_exchange_weak(spare, spare - 1)) {}
    spawn = spare > 0;
  }
  if (spawn) {
    std::vector<int32_t> out_b;
    std::exception_ptr err;
    std::thread t([&] {
      try {
        order_side(g, sh, b, out_b);
      } catch (...) {
        err = std::current_exception();
      }
    });
    try {
      order_side(g, sh, a, out);
    } catch (...) {
      t.join();
      sh.spare_threads.fetch_add(1);
      throw;
    }
    t.join();
    sh.spare_threads.fetch_add(1);
    if (err) std::rethrow_exception(err);
    out.insert(out.end(), out_b.begin(), out_b.end());
  } else {
    order_side(g, sh, a, out);
    order_side(g, sh, b, out);
  }
  for (int32_t v : sep) sh.set_tag(v, -2);   // ordered
  out.insert(out.end(), sep.begin(), sep.end());
}

}  // namespace

extern "C" int chol_order_nd(int32_t n, const int64_t* colptr, const int32_t* rowind, int32_t* perm) {
  if (n < 0) return -1;
  if (n > 0 && !colptr) return -2;
  if (n > 0 && !rowind) return -3;
  if (n > 0 && !perm) return -4;
  if (n == 0) return CHOL_OK;
  if (colptr[0] != 0) return -2;
  for (int32_t j = 0; j < n; ++j) {
    if (colptr[j + 1] < colptr[j]) return -2;
    for (int64_t t = colptr[j]; t < colptr[j + 1]; ++t)
      if (rowind[t] < j || rowind[t] >= n) return -3;
  }
  try {
    const Graph g = build_graph(n, colptr, rowind);
    Shared sh(n);
    const unsigned hw = std::thread::hardware_concurrency();
    sh.spare_threads.store(hw > 1 ? (int)hw - 1 : 0);
    std::vector<int32_t> out;
    out.reserve(n);
    // connected components of the whole graph, each dissected on its own
    std::vector<int32_t> comp, clev;
    for (int32_t s = 0; s < n; ++s) {
      if (sh.tag_of(s) != 0) continue;
      const int32_t ctag = sh.next_tag.fetch_add(1);
      bfs(g, sh, 0, s, comp, clev);
      for (int32_t v : comp) sh.set_tag(v, ctag);
      dissect(g, sh, ctag, comp, out);
    }
    if ((int32_t)out.size() != n) return CHOL_ESTATE;   // cannot happen: every vertex is placed once
    std::copy(out.begin(), out.end(), perm);
  } catch (const std::bad_alloc&) {
    return CHOL_ENOMEM;
  } catch (const std::system_error&) {   // a thread could not be started
    return CHOL_ENOMEM;
  }
  return CHOL_OK;
}
