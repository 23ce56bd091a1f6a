/*
 * oracle.c -- plain, slow, obviously correct FP64 CPU sparse Cholesky.
 *
 * TEST INFRASTRUCTURE ONLY. Nothing in the library's compute path may call,
 * link or load this file; it exists so that tests, the smoke check and the
 * benchmark's CPU-baseline leg can compare the GPU results against a direct
 * restatement of the definitions in "GPU Accelerated Sparse Cholesky
 * Factorization" (Karsavuran, Ng, Peyton):
 *
 *   - Sec. II: A = L L^T for sparse SPD A (n x n); the elimination tree has
 *     parent(j) = the minimum row index i > j with L_ij != 0, and the row
 *     structure of column j (minus j) is contained in that of parent(j).
 *   - Sec. II: relative indices relind(J, J'): for every global row index i in
 *     struct(J) ∩ struct(J'), the distance of i from the bottom of the index set
 *     of J'.
 *   - Sec. II / Fig. 1: a supernode is a set of contiguous columns with the same
 *     structure; the partition used is the maximal one (columns j and j+1 share
 *     a supernode iff parent(j) = j+1 and colcount(j) = colcount(j+1) + 1).
 *   - Sec. I: the triangular factors give the solution (forward and backward
 *     substitution).
 *
 * Numeric factorization: left-looking column Cholesky (cmod / cdiv) with a dense
 * accumulator per column -- deliberately *not* the right-looking supernodal
 * method of the paper, so the two share no algorithmic structure.
 *
 * Conventions: 0-based indices, lower-triangular CSC (diagonal included, rows
 * ascending and unique), perm is new->old.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* small helpers                                                            */
/* ------------------------------------------------------------------------ */

typedef struct { int32_t r; double v; } rv_t;

static int cmp_i32(const void* a, const void* b) {
  int32_t x = *(const int32_t*)a, y = *(const int32_t*)b;
  return (x > y) - (x < y);
}
static int cmp_rv(const void* a, const void* b) {
  int32_t x = ((const rv_t*)a)->r, y = ((const rv_t*)b)->r;
  return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------ */
/* B = P A P^T (lower CSC). Returns 0 or -1 on a malformed permutation.      */
/* ------------------------------------------------------------------------ */
int orc_permute(int32_t n, const int64_t* colptr, const int32_t* rowind, const double* vals,
                const int32_t* perm, int64_t* bcolptr, int32_t* browind, double* bvals) {
  int32_t* iperm = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) iperm[i] = -1;
  for (int32_t i = 0; i < n; ++i) {
    int32_t p = perm ? perm[i] : i;
    if (p < 0 || p >= n || iperm[p] != -1) { free(iperm); return -1; }
    iperm[p] = i;
  }
  int64_t nnz = colptr[n];
  memset(bcolptr, 0, sizeof(int64_t) * (size_t)(n + 1));
  for (int32_t c = 0; c < n; ++c)
    for (int64_t t = colptr[c]; t < colptr[c + 1]; ++t) {
      int32_t a = iperm[rowind[t]], b = iperm[c];
      int32_t col = a < b ? a : b;
      bcolptr[col + 1]++;
    }
  for (int32_t c = 0; c < n; ++c) bcolptr[c + 1] += bcolptr[c];
  int64_t* next = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t c = 0; c < n; ++c) next[c] = bcolptr[c];
  rv_t* tmp = (rv_t*)malloc(sizeof(rv_t) * (size_t)(nnz > 0 ? nnz : 1));
  for (int32_t c = 0; c < n; ++c)
    for (int64_t t = colptr[c]; t < colptr[c + 1]; ++t) {
      int32_t a = iperm[rowind[t]], b = iperm[c];
      int32_t col = a < b ? a : b, row = a < b ? b : a;
      tmp[next[col]].r = row;
      tmp[next[col]].v = vals ? vals[t] : 0.0;
      next[col]++;
    }
  for (int32_t c = 0; c < n; ++c)
    qsort(tmp + bcolptr[c], (size_t)(bcolptr[c + 1] - bcolptr[c]), sizeof(rv_t), cmp_rv);
  for (int64_t t = 0; t < nnz; ++t) {
    browind[t] = tmp[t].r;
    if (bvals) bvals[t] = tmp[t].v;
  }
  free(tmp); free(next); free(iperm);
  return 0;
}

/* ------------------------------------------------------------------------ */
/* Symbolic factorization by definition.                                     */
/*   struct(j) = {j} ∪ {i > j : B_ij != 0} ∪ ⋃_{c : parent(c) = j} struct(c)\{c}
 *   parent(j) = min(struct(j) \ {j})   (Sec. II definition of the etree)      */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n;
  int32_t* parent;
  int32_t* colcount;
  int64_t* lp;   /* n+1 */
  int32_t* li;   /* nnz(L), rows of each column ascending, diagonal first */
} orc_sym;

void* orc_sym_new(int32_t n, const int64_t* bcolptr, const int32_t* browind) {
  orc_sym* s = (orc_sym*)calloc(1, sizeof(orc_sym));
  s->n = n;
  s->parent = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  s->colcount = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t** cols = (int32_t**)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t*));
  int32_t* head = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));   /* child lists */
  int32_t* nxt = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* mark = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  int32_t* buf = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t j = 0; j < n; ++j) { head[j] = -1; mark[j] = -1; }
  for (int32_t j = 0; j < n; ++j) {
    int32_t cnt = 0;
    buf[cnt++] = j; mark[j] = j;
    for (int64_t t = bcolptr[j]; t < bcolptr[j + 1]; ++t) {
      int32_t i = browind[t];
      if (i > j && mark[i] != j) { mark[i] = j; buf[cnt++] = i; }
    }
    for (int32_t c = head[j]; c != -1; c = nxt[c]) {
      for (int32_t t = 0; t < s->colcount[c]; ++t) {
        int32_t i = cols[c][t];
        if (i != c && mark[i] != j) { mark[i] = j; buf[cnt++] = i; }
      }
    }
    qsort(buf, (size_t)cnt, sizeof(int32_t), cmp_i32);
    cols[j] = (int32_t*)malloc(sizeof(int32_t) * (size_t)cnt);
    memcpy(cols[j], buf, sizeof(int32_t) * (size_t)cnt);
    s->colcount[j] = cnt;
    s->parent[j] = cnt > 1 ? buf[1] : -1;
    if (cnt > 1) { nxt[j] = head[buf[1]]; head[buf[1]] = j; }
  }
  s->lp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  s->lp[0] = 0;
  for (int32_t j = 0; j < n; ++j) s->lp[j + 1] = s->lp[j] + s->colcount[j];
  s->li = (int32_t*)malloc(sizeof(int32_t) * (size_t)(s->lp[n] > 0 ? s->lp[n] : 1));
  for (int32_t j = 0; j < n; ++j) {
    memcpy(s->li + s->lp[j], cols[j], sizeof(int32_t) * (size_t)s->colcount[j]);
    free(cols[j]);
  }
  free(cols); free(head); free(nxt); free(mark); free(buf);
  return s;
}

int64_t orc_sym_nnz(void* h) { orc_sym* s = (orc_sym*)h; return s->lp[s->n]; }

void orc_sym_get(void* h, int32_t* parent, int32_t* colcount, int64_t* lp, int32_t* li) {
  orc_sym* s = (orc_sym*)h;
  if (parent) memcpy(parent, s->parent, sizeof(int32_t) * (size_t)s->n);
  if (colcount) memcpy(colcount, s->colcount, sizeof(int32_t) * (size_t)s->n);
  if (lp) memcpy(lp, s->lp, sizeof(int64_t) * (size_t)(s->n + 1));
  if (li) memcpy(li, s->li, sizeof(int32_t) * (size_t)s->lp[s->n]);
}

void orc_sym_free(void* h) {
  orc_sym* s = (orc_sym*)h;
  if (!s) return;
  free(s->parent); free(s->colcount); free(s->lp); free(s->li); free(s);
}

/* Maximal supernode partition (Fig. 1 groups columns this way).            */
/* snode_ptr has room for n+1 entries; returns the number of supernodes.    */
int32_t orc_supernodes(int32_t n, const int32_t* parent, const int32_t* colcount,
                       int32_t* snode_ptr, int32_t* snode_parent) {
  int32_t ns = 0;
  for (int32_t j = 0; j < n; ++j) {
    int join = j > 0 && parent[j - 1] == j && colcount[j - 1] == colcount[j] + 1;
    if (!join) snode_ptr[ns++] = j;
  }
  snode_ptr[ns] = n;
  if (snode_parent) {
    for (int32_t J = 0; J < ns; ++J) {
      int32_t last = snode_ptr[J + 1] - 1;
      int32_t p = parent[last];
      int32_t K = -1;
      if (p >= 0) {
        for (int32_t q = J + 1; q < ns; ++q)
          if (snode_ptr[q] <= p && p < snode_ptr[q + 1]) { K = q; break; }
      }
      snode_parent[J] = K;
    }
  }
  return ns;
}

/* relind by definition: for each supernode J (ascending) and each supernode K
 * (ascending) that owns a column in struct(J) below J, the list, in J's
 * ascending row order, of (|struct(K)| - 1 - position of i in struct(K)) for
 * every i in struct(J) ∩ struct(K), found by linear search.
 * Call once with out arrays NULL to get the sizes (npairs, total length).      */
void orc_relind(int32_t n, int32_t ns, const int32_t* snode_ptr, const int64_t* lp,
                const int32_t* li, int64_t* npairs, int64_t* total,
                int64_t* relind_ptr, int32_t* relind_target, int32_t* relind) {
  int32_t* snode_of = (int32_t*)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t J = 0; J < ns; ++J)
    for (int32_t j = snode_ptr[J]; j < snode_ptr[J + 1]; ++j) snode_of[j] = J;
  int64_t np = 0, tot = 0;
  if (relind_ptr) relind_ptr[0] = 0;
  for (int32_t J = 0; J < ns; ++J) {
    int32_t f = snode_ptr[J];
    const int32_t* sJ = li + lp[f];
    int32_t lenJ = (int32_t)(lp[f + 1] - lp[f]);
    int32_t prevK = -1;
    for (int32_t t = 0; t < lenJ; ++t) {
      int32_t i = sJ[t];
      if (i < snode_ptr[J + 1]) continue;
      int32_t K = snode_of[i];
      if (K == prevK) continue;
      prevK = K;
      int32_t fK = snode_ptr[K];
      const int32_t* sK = li + lp[fK];
      int32_t lenK = (int32_t)(lp[fK + 1] - lp[fK]);
      for (int32_t u = 0; u < lenJ; ++u) {
        int32_t r = sJ[u];
        for (int32_t v = 0; v < lenK; ++v)
          if (sK[v] == r) {
            if (relind) relind[tot] = lenK - 1 - v;
            tot++;
            break;
          }
      }
      if (relind_target) relind_target[np] = K;
      np++;
      if (relind_ptr) relind_ptr[np] = tot;
    }
  }
  *npairs = np; *total = tot;
  free(snode_of);
}

/* ------------------------------------------------------------------------ */
/* Numeric: left-looking column Cholesky with a dense accumulator.           */
/* For column j: w = B_{*,j}; w -= L_{*,k} L_jk for every k < j with L_jk!=0  */
/* (cmod); L_jj = sqrt(w_j), L_ij = w_i / L_jj (cdiv). The pattern of column */
/* j is the set of touched positions, found independently of orc_sym_new.    */
/* ------------------------------------------------------------------------ */
typedef struct {
  int32_t n;
  int32_t info;     /* 0, or j+1 for a non-positive pivot at column j */
  int64_t* lp;
  int32_t* li;
  double* lx;
} orc_num;

void* orc_factor_new(int32_t n, const int64_t* bcolptr, const int32_t* browind, const double* bvals) {
  orc_num* f = (orc_num*)calloc(1, sizeof(orc_num));
  f->n = n;
  size_t nn = (size_t)(n > 0 ? n : 1);
  int32_t** ci = (int32_t**)calloc(nn, sizeof(int32_t*));
  double** cx = (double**)calloc(nn, sizeof(double*));
  int32_t* cc = (int32_t*)calloc(nn, sizeof(int32_t));
  double* w = (double*)calloc(nn, sizeof(double));
  int32_t* touched = (int32_t*)malloc(sizeof(int32_t) * nn);
  char* on = (char*)calloc(nn, 1);
  int32_t* head = (int32_t*)malloc(sizeof(int32_t) * nn);  /* row lists */
  int32_t* link = (int32_t*)malloc(sizeof(int32_t) * nn);
  int32_t* ptr = (int32_t*)malloc(sizeof(int32_t) * nn);   /* next row position of col k */
  for (int32_t j = 0; j < n; ++j) head[j] = -1;
  int32_t done = 0;
  for (int32_t j = 0; j < n && !f->info; ++j) {
    int32_t nt = 0;
    for (int64_t t = bcolptr[j]; t < bcolptr[j + 1]; ++t) {
      int32_t i = browind[t];
      w[i] += bvals[t];
      if (!on[i]) { on[i] = 1; touched[nt++] = i; }
    }
    if (!on[j]) { on[j] = 1; touched[nt++] = j; }
    int32_t k = head[j];
    head[j] = -1;
    while (k != -1) {
      int32_t knext = link[k];
      int32_t p = ptr[k];
      double ljk = cx[k][p];
      for (int32_t q = p; q < cc[k]; ++q) {
        int32_t i = ci[k][q];
        w[i] -= cx[k][q] * ljk;
        if (!on[i]) { on[i] = 1; touched[nt++] = i; }
      }
      ptr[k] = p + 1;
      if (p + 1 < cc[k]) {
        int32_t r = ci[k][p + 1];
        link[k] = head[r];
        head[r] = k;
      }
      k = knext;
    }
    qsort(touched, (size_t)nt, sizeof(int32_t), cmp_i32);
    double d = w[j];
    if (!(d > 0.0)) f->info = j + 1;
    double ljj = sqrt(d);
    ci[j] = (int32_t*)malloc(sizeof(int32_t) * (size_t)nt);
    cx[j] = (double*)malloc(sizeof(double) * (size_t)nt);
    cc[j] = nt;
    for (int32_t q = 0; q < nt; ++q) {
      int32_t i = touched[q];
      ci[j][q] = i;
      cx[j][q] = (i == j) ? ljj : w[i] / ljj;
      w[i] = 0.0;
      on[i] = 0;
    }
    if (nt > 1) {
      ptr[j] = 1;
      int32_t r = ci[j][1];
      link[j] = head[r];
      head[r] = j;
    }
    done = j + 1;
  }
  f->lp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  f->lp[0] = 0;
  for (int32_t j = 0; j < n; ++j) f->lp[j + 1] = f->lp[j] + (j < done ? cc[j] : 0);
  int64_t nnz = f->lp[n];
  f->li = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  f->lx = (double*)malloc(sizeof(double) * (size_t)(nnz > 0 ? nnz : 1));
  for (int32_t j = 0; j < done; ++j) {
    memcpy(f->li + f->lp[j], ci[j], sizeof(int32_t) * (size_t)cc[j]);
    memcpy(f->lx + f->lp[j], cx[j], sizeof(double) * (size_t)cc[j]);
    free(ci[j]); free(cx[j]);
  }
  free(ci); free(cx); free(cc); free(w); free(touched); free(on); free(head); free(link); free(ptr);
  return f;
}

/* ------------------------------------------------------------------------ */
/* The same numeric loops, multi-threaded (timing variant of the baseline).  */
/* Column j needs exactly the columns k < j with L_jk != 0, all of which are */
/* descendants of j in the elimination tree; so the columns of one etree     */
/* height are independent and are factored in parallel (OpenMP, one dense    */
/* accumulator per thread), heights in increasing order. A height with fewer */
/* columns than threads (the chains of the top separators, where most of the */
/* flops are) splits each column's cmod terms over the threads instead, and  */
/* adds their accumulators in thread order. The pattern comes                */
/* from the symbolic factor (lp, li: the output of orc_sym_new), and the     */
/* columns k that update column j are walked in increasing k, so the result  */
/* matches orc_factor_new up to the order of the cmod sums. Without OpenMP   */
/* it runs on one thread. info = smallest j + 1 with a non-positive pivot.   */
/* ------------------------------------------------------------------------ */
#ifdef _OPENMP
#include <omp.h>
#endif
/* Staged form: orc_mt_begin builds the row lists and the height classes,     */
/* orc_mt_run factors the heights [h0, h1) (heights must be run in increasing */
/* order, each once), orc_mt_finish returns the factor. orc_factor_new_mt     */
/* runs all heights in one go; splitting them changes nothing in the result.  */
typedef struct {
  orc_num* f;
  const int64_t* bcolptr;
  const int32_t* browind;
  const double* bvals;
  int64_t *rp, *rq, *hp;
  int32_t *rk, *byh;
  int32_t maxh, nt;
  double* wall;
  int32_t first_bad;   /* smallest j + 1 with a non-positive pivot */
} orc_mt;

void* orc_mt_begin(int32_t n, const int64_t* bcolptr, const int32_t* browind, const double* bvals,
                   const int32_t* parent, const int64_t* lp, const int32_t* li, int32_t nthreads) {
  orc_mt* m = (orc_mt*)calloc(1, sizeof(orc_mt));
  orc_num* f = (orc_num*)calloc(1, sizeof(orc_num));
  m->f = f;
  m->bcolptr = bcolptr; m->browind = browind; m->bvals = bvals;
  f->n = n;
  size_t nn = (size_t)(n > 0 ? n : 1);
  int64_t nnz = lp[n];
  f->lp = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
  memcpy(f->lp, lp, sizeof(int64_t) * (size_t)(n + 1));
  f->li = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  memcpy(f->li, li, sizeof(int32_t) * (size_t)nnz);
  f->lx = (double*)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
  /* row lists: for row j, the columns k < j with L_jk != 0 (ascending) and */
  /* the position of L_jk in column k                                       */
  int64_t* rp = (int64_t*)calloc(nn + 1, sizeof(int64_t));
  for (int32_t k = 0; k < n; ++k)
    for (int64_t q = lp[k] + 1; q < lp[k + 1]; ++q) rp[li[q] + 1]++;
  for (int32_t j = 0; j < n; ++j) rp[j + 1] += rp[j];
  int32_t* rk = (int32_t*)malloc(sizeof(int32_t) * (size_t)(rp[n] > 0 ? rp[n] : 1));
  int64_t* rq = (int64_t*)malloc(sizeof(int64_t) * (size_t)(rp[n] > 0 ? rp[n] : 1));
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * nn);
  for (int32_t j = 0; j < n; ++j) fill[j] = rp[j];
  for (int32_t k = 0; k < n; ++k)            /* k ascending: lists come out sorted */
    for (int64_t q = lp[k] + 1; q < lp[k + 1]; ++q) {
      int64_t z = fill[li[q]]++;
      rk[z] = k;
      rq[z] = q;
    }
  /* etree heights (children before parents: parent[j] > j) */
  int32_t* height = (int32_t*)calloc(nn, sizeof(int32_t));
  int32_t maxh = 0;
  for (int32_t j = 0; j < n; ++j) {
    if (parent[j] >= 0 && height[parent[j]] < height[j] + 1) height[parent[j]] = height[j] + 1;
    if (height[j] > maxh) maxh = height[j];
  }
  int64_t* hp = (int64_t*)calloc((size_t)maxh + 2, sizeof(int64_t));
  for (int32_t j = 0; j < n; ++j) hp[height[j] + 1]++;
  for (int32_t h = 0; h <= maxh; ++h) hp[h + 1] += hp[h];
  int32_t* byh = (int32_t*)malloc(sizeof(int32_t) * nn);
  for (int32_t h = 0; h <= maxh; ++h) fill[h] = hp[h];
  for (int32_t j = 0; j < n; ++j) byh[fill[height[j]]++] = j;
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
  (void)nthreads;
  m->rp = rp; m->rk = rk; m->rq = rq; m->hp = hp; m->byh = byh;
  m->maxh = n > 0 ? maxh : -1;
  m->nt = nt;
  m->wall = (double*)calloc(nn * (size_t)nt, sizeof(double));
  m->first_bad = INT32_MAX;
  free(fill); free(height);
  return m;
}

int32_t orc_mt_max_height(void* h) { return ((orc_mt*)h)->maxh; }

/* The column of each position in height order and the start of every height */
/* (maxh + 2 offsets), for splitting the run by work.                          */
void orc_mt_schedule(void* h, int64_t* hp, int32_t* byh) {
  orc_mt* m = (orc_mt*)h;
  if (hp) memcpy(hp, m->hp, sizeof(int64_t) * (size_t)(m->maxh + 2));
  if (byh) memcpy(byh, m->byh, sizeof(int32_t) * (size_t)(m->hp[m->maxh + 1]));
}

void orc_mt_run(void* h, int32_t h0, int32_t h1) {
  orc_mt* m = (orc_mt*)h;
  orc_num* f = m->f;
  const int32_t n = f->n;
  const size_t nn = (size_t)(n > 0 ? n : 1);
  const int64_t* lp = f->lp;
  const int32_t* li = f->li;
  const int64_t *bcolptr = m->bcolptr, *rp = m->rp, *rq = m->rq, *hp = m->hp;
  const int32_t *browind = m->browind, *rk = m->rk, *byh = m->byh;
  const double* bvals = m->bvals;
  const int nt = m->nt;
  double* wall = m->wall;
  int32_t first_bad = m->first_bad;
  if (h1 > m->maxh + 1) h1 = m->maxh + 1;
  for (int32_t hh = h0 < 0 ? 0 : h0; hh < h1; ++hh) {
    if (hp[hh + 1] - hp[hh] >= nt) {
      /* many columns at this height: one column per thread at a time */
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 16) num_threads(nt) reduction(min : first_bad)
#endif
      for (int64_t z = hp[hh]; z < hp[hh + 1]; ++z) {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        double* w = wall + (size_t)tid * nn;
        int32_t j = byh[z];
        for (int64_t t = bcolptr[j]; t < bcolptr[j + 1]; ++t) w[browind[t]] += bvals[t];
        for (int64_t e = rp[j]; e < rp[j + 1]; ++e) {          /* cmod(j, k) */
          int32_t k = rk[e];
          int64_t q0 = rq[e];
          double ljk = f->lx[q0];
          for (int64_t q = q0; q < lp[k + 1]; ++q) w[li[q]] -= f->lx[q] * ljk;
        }
        double d = w[j];                                        /* cdiv(j) */
        if (!(d > 0.0) && j + 1 < first_bad) first_bad = j + 1;
        double ljj = sqrt(d);
        f->lx[lp[j]] = ljj;
        w[j] = 0.0;
        for (int64_t q = lp[j] + 1; q < lp[j + 1]; ++q) {
          f->lx[q] = w[li[q]] / ljj;
          w[li[q]] = 0.0;
        }
      }
    } else {
      /* few columns (the chains of the top separators): each column's cmod */
      /* terms are split over the threads in fixed contiguous ranges, every */
      /* thread sums its range into its own accumulator, and the            */
      /* accumulators are added over the column's pattern in thread order   */
      for (int64_t z = hp[hh]; z < hp[hh + 1]; ++z) {
        int32_t j = byh[z];
        int64_t e0 = rp[j], e1 = rp[j + 1];
#ifdef _OPENMP
#pragma omp parallel num_threads(nt)
#endif
        {
          int tid = 0, nth = 1;
#ifdef _OPENMP
          tid = omp_get_thread_num();
          nth = omp_get_num_threads();
#endif
          double* w = wall + (size_t)tid * nn;
          int64_t a = e0 + (e1 - e0) * tid / nth, b = e0 + (e1 - e0) * (tid + 1) / nth;
          for (int64_t e = a; e < b; ++e) {
            int32_t k = rk[e];
            int64_t q0 = rq[e];
            double ljk = f->lx[q0];
            for (int64_t q = q0; q < lp[k + 1]; ++q) w[li[q]] -= f->lx[q] * ljk;
          }
        }
        double* w0 = wall;
        for (int t = 1; t < nt; ++t) {
          double* wt = wall + (size_t)t * nn;
          for (int64_t q = lp[j]; q < lp[j + 1]; ++q) {
            w0[li[q]] += wt[li[q]];
            wt[li[q]] = 0.0;
          }
        }
        for (int64_t t = bcolptr[j]; t < bcolptr[j + 1]; ++t) w0[browind[t]] += bvals[t];
        double d = w0[j];
        if (!(d > 0.0) && j + 1 < first_bad) first_bad = j + 1;
        double ljj = sqrt(d);
        f->lx[lp[j]] = ljj;
        w0[j] = 0.0;
        for (int64_t q = lp[j] + 1; q < lp[j + 1]; ++q) {
          f->lx[q] = w0[li[q]] / ljj;
          w0[li[q]] = 0.0;
        }
      }
    }
  }
  m->first_bad = first_bad;
}

void* orc_mt_finish(void* h) {
  orc_mt* m = (orc_mt*)h;
  orc_num* f = m->f;
  f->info = m->first_bad == INT32_MAX ? 0 : m->first_bad;
  free(m->rp); free(m->rk); free(m->rq); free(m->hp); free(m->byh); free(m->wall); free(m);
  return f;
}

void* orc_factor_new_mt(int32_t n, const int64_t* bcolptr, const int32_t* browind, const double* bvals,
                        const int32_t* parent, const int64_t* lp, const int32_t* li, int32_t nthreads) {
  void* m = orc_mt_begin(n, bcolptr, browind, bvals, parent, lp, li, nthreads);
  orc_mt_run(m, 0, orc_mt_max_height(m) + 1);
  return orc_mt_finish(m);
}

int32_t orc_factor_info(void* h) { return ((orc_num*)h)->info; }
int64_t orc_factor_nnz(void* h) { orc_num* f = (orc_num*)h; return f->lp[f->n]; }
void orc_factor_get(void* h, int64_t* lp, int32_t* li, double* lx) {
  orc_num* f = (orc_num*)h;
  int64_t nnz = f->lp[f->n];
  if (lp) memcpy(lp, f->lp, sizeof(int64_t) * (size_t)(f->n + 1));
  if (li) memcpy(li, f->li, sizeof(int32_t) * (size_t)nnz);
  if (lx) memcpy(lx, f->lx, sizeof(double) * (size_t)nnz);
}
void orc_factor_free(void* h) {
  orc_num* f = (orc_num*)h;
  if (!f) return;
  free(f->lp); free(f->li); free(f->lx); free(f);
}

/* ------------------------------------------------------------------------ */
/* Triangular solves in the original ordering: x = P^T L^{-T} L^{-1} P b.    */
/* b and x are n x nrhs column-major; x may alias b.                         */
/* ------------------------------------------------------------------------ */
void orc_solve(int32_t n, const int64_t* lp, const int32_t* li, const double* lx,
               const int32_t* perm, int32_t nrhs, const double* b, double* x) {
  double* y = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int32_t r = 0; r < nrhs; ++r) {
    const double* br = b + (size_t)r * n;
    for (int32_t i = 0; i < n; ++i) y[i] = br[perm ? perm[i] : i];
    for (int32_t j = 0; j < n; ++j) {          /* L y = P b */
      y[j] /= lx[lp[j]];
      for (int64_t t = lp[j] + 1; t < lp[j + 1]; ++t) y[li[t]] -= lx[t] * y[j];
    }
    for (int32_t j = n - 1; j >= 0; --j) {     /* L^T z = y */
      double s = y[j];
      for (int64_t t = lp[j] + 1; t < lp[j + 1]; ++t) s -= lx[t] * y[li[t]];
      y[j] = s / lx[lp[j]];
    }
    double* xr = x + (size_t)r * n;
    for (int32_t i = 0; i < n; ++i) xr[perm ? perm[i] : i] = y[i];
  }
  free(y);
}

/* logdet A = 2 * sum_j log L_jj, summed in column order. */
double orc_logdet(int32_t n, const int64_t* lp, const double* lx) {
  double s = 0.0;
  for (int32_t j = 0; j < n; ++j) s += log(lx[lp[j]]);
  return 2.0 * s;
}

/* y = A x for symmetric A given by its lower CSC (original ordering). */
void orc_spmv(int32_t n, const int64_t* colptr, const int32_t* rowind, const double* vals,
              int32_t nrhs, const double* x, double* y) {
  for (int32_t r = 0; r < nrhs; ++r) {
    const double* xr = x + (size_t)r * n;
    double* yr = y + (size_t)r * n;
    for (int32_t i = 0; i < n; ++i) yr[i] = 0.0;
    for (int32_t j = 0; j < n; ++j)
      for (int64_t t = colptr[j]; t < colptr[j + 1]; ++t) {
        int32_t i = rowind[t];
        yr[i] += vals[t] * xr[j];
        if (i != j) yr[j] += vals[t] * xr[i];
      }
  }
}

/* Normwise backward error per right-hand side:
 * eta = ||b - A x||_inf / (||A||_inf ||x||_inf + ||b||_inf).                 */
void orc_backward_error(int32_t n, const int64_t* colptr, const int32_t* rowind, const double* vals,
                        int32_t nrhs, const double* b, const double* x, double* eta) {
  double* rs = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  for (int32_t j = 0; j < n; ++j)
    for (int64_t t = colptr[j]; t < colptr[j + 1]; ++t) {
      int32_t i = rowind[t];
      rs[i] += fabs(vals[t]);
      if (i != j) rs[j] += fabs(vals[t]);
    }
  double anorm = 0.0;
  for (int32_t i = 0; i < n; ++i) anorm = rs[i] > anorm ? rs[i] : anorm;
  double* ax = (double*)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
  for (int32_t r = 0; r < nrhs; ++r) {
    const double* xr = x + (size_t)r * n;
    const double* br = b + (size_t)r * n;
    orc_spmv(n, colptr, rowind, vals, 1, xr, ax);
    double rn = 0.0, xn = 0.0, bn = 0.0;
    for (int32_t i = 0; i < n; ++i) {
      double d = fabs(br[i] - ax[i]);
      rn = d > rn ? d : rn;
      xn = fabs(xr[i]) > xn ? fabs(xr[i]) : xn;
      bn = fabs(br[i]) > bn ? fabs(br[i]) : bn;
    }
    eta[r] = rn / (anorm * xn + bn);
  }
  free(ax); free(rs);
}

/* Factor residual ||B - L L^T||_F / ||B||_F for B = P A P^T (lower CSC) and a
 * given L (CSC, rows ascending, diagonal first). L L^T is formed column by
 * column of L: for k, every pair i >= j in struct(k) adds L_ik L_jk at (i, j).
 * Off-diagonal entries count twice in both Frobenius norms.                  */
double orc_factor_residual(int32_t n, const int64_t* bcolptr, const int32_t* browind, const double* bvals,
                           const int64_t* lp, const int32_t* li, const double* lx) {
  int64_t nnz = lp[n];
  double* m = (double*)calloc((size_t)(nnz > 0 ? nnz : 1), sizeof(double));
  int64_t* pos = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) pos[i] = -1;
  /* position of (i, j) inside column j of L: fill pos[] per column j on demand */
  /* (i, j) needs column j's map; process target columns j one at a time using */
  /* the row lists of L^T (which k have L_jk != 0).                            */
  int64_t* rcount = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
  for (int32_t k = 0; k < n; ++k)
    for (int64_t t = lp[k]; t < lp[k + 1]; ++t) rcount[li[t] + 1]++;
  for (int32_t i = 0; i < n; ++i) rcount[i + 1] += rcount[i];
  int64_t* rfill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) rfill[i] = rcount[i];
  int64_t* rent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1)); /* index t of L_jk */
  for (int32_t k = 0; k < n; ++k)
    for (int64_t t = lp[k]; t < lp[k + 1]; ++t) rent[rfill[li[t]]++] = t;
  int bad = 0;
  for (int32_t j = 0; j < n; ++j) {
    for (int64_t t = lp[j]; t < lp[j + 1]; ++t) pos[li[t]] = t;
    for (int64_t q = rcount[j]; q < rcount[j + 1]; ++q) {
      int64_t tj = rent[q];                   /* L_jk at tj in column k */
      int32_t k = 0;
      /* column k of entry tj: binary search lp */
      int32_t lo = 0, hi = n - 1;
      while (lo < hi) { int32_t mid = (lo + hi + 1) / 2; if (lp[mid] <= tj) lo = mid; else hi = mid - 1; }
      k = lo;
      double ljk = lx[tj];
      for (int64_t t = tj; t < lp[k + 1]; ++t) {
        int64_t p = pos[li[t]];
        if (p < 0) { bad = 1; continue; }
        m[p] += lx[t] * ljk;
      }
    }
    for (int64_t t = lp[j]; t < lp[j + 1]; ++t) pos[li[t]] = -1;
  }
  double num = 0.0, den = 0.0;
  for (int32_t j = 0; j < n; ++j) {
    for (int64_t t = lp[j]; t < lp[j + 1]; ++t) pos[li[t]] = t;
    for (int64_t t = bcolptr[j]; t < bcolptr[j + 1]; ++t) {
      int32_t i = browind[t];
      double w = (i == j) ? 1.0 : 2.0;
      den += w * bvals[t] * bvals[t];
      int64_t p = pos[i];
      if (p < 0) { bad = 1; continue; }
      m[p] -= bvals[t];
    }
    for (int64_t t = lp[j]; t < lp[j + 1]; ++t) {
      double w = (li[t] == j) ? 1.0 : 2.0;
      num += w * m[t] * m[t];
      pos[li[t]] = -1;
    }
  }
  free(m); free(pos); free(rcount); free(rfill); free(rent);
  if (bad) return -1.0;
  return sqrt(num) / sqrt(den);
}

/* Residual of selected columns: for each listed column j, the lower part
 * r_i = B_ij - sum_k L_ik L_jk (i >= j), returned as ||r||_2 / ||B_{j:n,j}||_2.
 * Row j of L (the k with L_jk != 0) comes from a transposed index built once. */
void orc_factor_residual_cols(int32_t n, const int64_t* bcolptr, const int32_t* browind,
                              const double* bvals, const int64_t* lp, const int32_t* li,
                              const double* lx, int32_t ncols, const int32_t* cols, double* out) {
  int64_t nnz = lp[n];
  int64_t* rcount = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
  for (int64_t t = 0; t < nnz; ++t) rcount[li[t] + 1]++;
  for (int32_t i = 0; i < n; ++i) rcount[i + 1] += rcount[i];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
  for (int32_t i = 0; i < n; ++i) fill[i] = rcount[i];
  int64_t* rent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  int32_t* rcol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  for (int32_t k = 0; k < n; ++k)
    for (int64_t t = lp[k]; t < lp[k + 1]; ++t) { rent[fill[li[t]]] = t; rcol[fill[li[t]]] = k; fill[li[t]]++; }
  double* w = (double*)calloc((size_t)(n > 0 ? n : 1), sizeof(double));
  for (int32_t q = 0; q < ncols; ++q) {
    int32_t j = cols[q];
    double bn = 0.0;
    for (int64_t t = bcolptr[j]; t < bcolptr[j + 1]; ++t) { w[browind[t]] += bvals[t]; bn += bvals[t] * bvals[t]; }
    for (int64_t e = rcount[j]; e < rcount[j + 1]; ++e) {
      int64_t tj = rent[e];
      int32_t k = rcol[e];
      double ljk = lx[tj];
      for (int64_t t = tj; t < lp[k + 1]; ++t) w[li[t]] -= lx[t] * ljk;
    }
    double rn = 0.0;
    for (int64_t e = rcount[j]; e < rcount[j + 1]; ++e) {
      int32_t k = rcol[e];
      for (int64_t t = rent[e]; t < lp[k + 1]; ++t) { rn += w[li[t]] * w[li[t]]; w[li[t]] = 0.0; }
    }
    for (int64_t t = bcolptr[j]; t < bcolptr[j + 1]; ++t) { rn += w[browind[t]] * w[browind[t]]; w[browind[t]] = 0.0; }
    out[q] = sqrt(rn) / sqrt(bn);
  }
  free(w); free(rcount); free(fill); free(rent); free(rcol);
}

/* Per-column parts of the factor residual ||B - L L^T||_F / ||B||_F (the same  */
/* quantity as orc_factor_residual): for column j, with r_i = B_ij -             */
/* sum_k L_ik L_jk over i >= j, num[j] = r_jj^2 + 2 sum_{i>j} r_i^2 and den[j] =  */
/* B_jj^2 + 2 sum_{i>j} B_ij^2 (off-diagonal entries count twice). Columns are   */
/* independent, so they run in parallel (one accumulator per thread); the      */
/* caller adds num and den in column order.                                    */
void orc_factor_residual_parts(int32_t n, const int64_t* bcolptr, const int32_t* browind, const double* bvals,
                               const int64_t* lp, const int32_t* li, const double* lx, int32_t nthreads,
                               double* num, double* den) {
  int64_t nnz = lp[n];
  size_t nn = (size_t)(n > 0 ? n : 1);
  int64_t* rcount = (int64_t*)calloc(nn + 1, sizeof(int64_t));
  for (int64_t t = 0; t < nnz; ++t) rcount[li[t] + 1]++;
  for (int32_t i = 0; i < n; ++i) rcount[i + 1] += rcount[i];
  int64_t* fill = (int64_t*)malloc(sizeof(int64_t) * nn);
  for (int32_t i = 0; i < n; ++i) fill[i] = rcount[i];
  int64_t* rent = (int64_t*)malloc(sizeof(int64_t) * (size_t)(nnz > 0 ? nnz : 1));
  int32_t* rcol = (int32_t*)malloc(sizeof(int32_t) * (size_t)(nnz > 0 ? nnz : 1));
  for (int32_t k = 0; k < n; ++k)
    for (int64_t t = lp[k]; t < lp[k + 1]; ++t) { rent[fill[li[t]]] = t; rcol[fill[li[t]]] = k; fill[li[t]]++; }
  int nt = 1;
#ifdef _OPENMP
  nt = nthreads > 0 ? nthreads : omp_get_max_threads();
#endif
  (void)nthreads;
  double* wall = (double*)calloc(nn * (size_t)nt, sizeof(double));
#ifdef _OPENMP
#pragma omp parallel for schedule(dynamic, 64) num_threads(nt)
#endif
  for (int32_t j = 0; j < n; ++j) {
    int tid = 0;
#ifdef _OPENMP
    tid = omp_get_thread_num();
#endif
    double* w = wall + (size_t)tid * nn;
    double bn = 0.0;
    for (int64_t t = bcolptr[j]; t < bcolptr[j + 1]; ++t) {
      w[browind[t]] += bvals[t];
      bn += (browind[t] == j ? 1.0 : 2.0) * bvals[t] * bvals[t];
    }
    for (int64_t e = rcount[j]; e < rcount[j + 1]; ++e) {
      int64_t tj = rent[e];
      int32_t k = rcol[e];
      double ljk = lx[tj];
      for (int64_t t = tj; t < lp[k + 1]; ++t) w[li[t]] -= lx[t] * ljk;
    }
    double rn = 0.0;
    for (int64_t e = rcount[j]; e < rcount[j + 1]; ++e) {
      int32_t k = rcol[e];
      for (int64_t t = rent[e]; t < lp[k + 1]; ++t) {
        int32_t i = li[t];
        rn += (i == j ? 1.0 : 2.0) * w[i] * w[i];
        w[i] = 0.0;
      }
    }
    for (int64_t t = bcolptr[j]; t < bcolptr[j + 1]; ++t) {
      int32_t i = browind[t];
      rn += (i == j ? 1.0 : 2.0) * w[i] * w[i];
      w[i] = 0.0;
    }
    num[j] = rn;
    den[j] = bn;
  }
  free(wall); free(rcount); free(fill); free(rent); free(rcol);
}

/* ------------------------------------------------------------------------ */
/* Selected inverse Z = B^{-1} on the pattern of L (column Takahashi          */
/* recurrence, B = L L^T). From B Z = I with Z symmetric, column by column    */
/* from the last one: for i in struct(j), i > j,                             */
/*   Z_ij = -sum_{k in struct(j), k > j} (L_kj / L_jj) Z_{ik}                 */
/* and Z_jj = 1 / L_jj^2 - sum_{k in struct(j), k > j} (L_kj / L_jj) Z_kj,    */
/* where Z_{ik} for i, k > j is an entry of an already computed column       */
/* (struct(j) is a clique of the filled graph, so it lies in pattern(L)).    */
/* zx has the layout of lx (lp/li).                                          */
/* ------------------------------------------------------------------------ */
static int64_t find_entry(const int64_t* lp, const int32_t* li, int32_t row, int32_t col) {
  int64_t lo = lp[col], hi = lp[col + 1] - 1;
  while (lo <= hi) {
    int64_t mid = (lo + hi) / 2;
    if (li[mid] == row) return mid;
    if (li[mid] < row) lo = mid + 1; else hi = mid - 1;
  }
  return -1;
}

int orc_selinv(int32_t n, const int64_t* lp, const int32_t* li, const double* lx, double* zx) {
  for (int32_t j = n - 1; j >= 0; --j) {
    const double ljj = lx[lp[j]];
    for (int64_t t = lp[j] + 1; t < lp[j + 1]; ++t) {
      const int32_t i = li[t];
      double s = 0.0;
      for (int64_t q = lp[j] + 1; q < lp[j + 1]; ++q) {
        const int32_t k = li[q];
        const int32_t r = i > k ? i : k, c = i > k ? k : i;
        const int64_t p = find_entry(lp, li, r, c);
        if (p < 0) return -1;
        s += (lx[q] / ljj) * zx[p];
      }
      zx[t] = -s;
    }
    double s = 0.0;
    for (int64_t q = lp[j] + 1; q < lp[j + 1]; ++q) s += (lx[q] / ljj) * zx[q];
    zx[lp[j]] = 1.0 / (ljj * ljj) - s;
  }
  return 0;
}
