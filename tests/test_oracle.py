"""Pins for the FP64 CPU oracle against facts fixed by the paper or by mathematics.

Each test checks the oracle against something other than itself: the worked
example of Fig. 1 / Fig. 2 (Sec. II), brute force by the fill-path theorem,
LAPACK (numpy) as a library, closed-form eigenvalues and determinants, and
exact counting.
"""
import math

import numpy as np
import pytest

import gridgen
import oracle
from golden_fig1 import load as load_fig1
from helpers import (brute_fill, csc_to_dense_lower, dense_from_lower, graph_from_lower,
                     lower_csc_from_dense, random_spd)


# --------------------------------------------------------------------------
# Fig. 1 / Fig. 2 worked example (integer, bit-exact)
# --------------------------------------------------------------------------

def _fig1_matrix(cols, drop=()):
    n = 15
    A = np.zeros((n, n))
    for j, rows in cols.items():
        for i in rows:
            if (i, j) in drop:
                continue
            A[i - 1, j - 1] = A[j - 1, i - 1] = -1.0
    A[np.diag_indices(n)] = 20.0
    return A


def _oracle_on_dense(A):
    n = A.shape[0]
    cp, ri, vx = lower_csc_from_dense(A)
    sym = oracle.Symbolic(n, cp, ri)
    return sym


def test_fig1_structure_etree_counts():
    g = load_fig1()
    sym = _oracle_on_dense(_fig1_matrix(g["cols"]))
    for j in range(1, 16):
        got = [int(i) + 1 for i in sym.li[sym.lp[j - 1]:sym.lp[j]]]
        assert got == [j] + g["cols"][j], j
    # etree by definition: parent(j) = smallest i > j with L_ij != 0
    parent = [(g["cols"][j][0] - 1) if g["cols"][j] else -1 for j in range(1, 16)]
    assert sym.parent.tolist() == parent
    assert sym.colcount.tolist() == [len(g["cols"][j]) + 1 for j in range(1, 16)]
    assert sym.nnz == 57
    assert sym.flops() == 239


def test_fig1_supernodes_tree_sizes():
    g = load_fig1()
    sym = _oracle_on_dense(_fig1_matrix(g["cols"]))
    ptr, sparent = sym.supernodes()
    names = ["J%d" % (k + 1) for k in range(len(ptr) - 1)]
    got = {names[k]: list(range(ptr[k] + 1, ptr[k + 1] + 1)) for k in range(len(ptr) - 1)}
    assert got == g["snodes"]
    edges = [(names[k], names[sparent[k]]) for k in range(len(names)) if sparent[k] >= 0]
    assert sorted(edges) == sorted(g["tree"])
    for J, (rows, ncols) in g["sizes"].items():
        k = names.index(J)
        f = ptr[k]
        assert (sym.colcount[f], ptr[k + 1] - ptr[k]) == (rows, ncols)
    # Fig. 2: the update matrix of J1 lives on struct(J1) minus J1's columns
    f, l = ptr[0], ptr[1]
    rows_j1 = [int(i) + 1 for i in sym.li[sym.lp[f]:sym.lp[f + 1]] if i >= l]
    assert rows_j1 == g["update"]["J1"]


def test_fig1_relind():
    g = load_fig1()
    sym = _oracle_on_dense(_fig1_matrix(g["cols"]))
    ptr, _ = sym.supernodes()
    rp, rt, ri = sym.relind(ptr)
    # recover (J, K) of every pair: J advances whenever K is not increasing
    pairs = {}
    ns = len(ptr) - 1
    J = 0
    p = 0
    # pairs are listed J ascending then K ascending; J owning pair p is found from
    # the row structure: recompute the touched ancestor list per J
    for Jn in range(ns):
        f, l = ptr[Jn], ptr[Jn + 1]
        rows = sym.li[sym.lp[f]:sym.lp[f + 1]]
        ks = []
        for i in rows:
            if i >= l:
                K = int(np.searchsorted(ptr, i, side="right") - 1)
                if K not in ks:
                    ks.append(K)
        for K in ks:
            assert rt[p] == K
            pairs[("J%d" % (Jn + 1), "J%d" % (K + 1))] = ri[rp[p]:rp[p + 1]].tolist()
            p += 1
    assert p == len(rt)
    for key, val in g["relind"].items():
        assert pairs[key] == val, key
    for J, targets in g["updates"].items():
        assert sorted(k for (a, k) in pairs if a == J) == sorted(targets)


def test_fig1_fill_from_sparser_matrix():
    """Drop every entry of A whose removal the fill-path theorem says is refilled;
    the oracle must still produce the L of Fig. 1."""
    g = load_fig1()
    drop = set()
    for j, rows in g["cols"].items():
        for i in rows:
            trial = drop | {(i, j)}
            A = _fig1_matrix(g["cols"], trial)
            cp, ri, _ = lower_csc_from_dense(A)
            st = brute_fill(15, graph_from_lower(15, cp, ri))
            if all([r + 1 for r in st[c - 1]] == g["cols"][c] for c in range(1, 16)):
                drop = trial
    assert len(drop) >= 5   # a genuinely sparser A
    sym = _oracle_on_dense(_fig1_matrix(g["cols"], drop))
    for j in range(1, 16):
        got = [int(i) + 1 for i in sym.li[sym.lp[j - 1] + 1:sym.lp[j]]]
        assert got == g["cols"][j]


# --------------------------------------------------------------------------
# brute force on tiny random graphs
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(12))
def test_symbolic_vs_fill_path_theorem(seed):
    rs = np.random.RandomState(100 + seed)
    n = int(rs.randint(5, 41))
    A, cp, ri, vx, perm = random_spd(n, rs.uniform(0.05, 0.25), seed)
    bp, bi, bx = oracle.permute(n, cp, ri, vx, perm)
    sym = oracle.Symbolic(n, bp, bi)
    brute = brute_fill(n, graph_from_lower(n, bp, bi))
    for j in range(n):
        assert sym.li[sym.lp[j]:sym.lp[j + 1]].tolist() == [j] + brute[j]
        assert sym.parent[j] == (brute[j][0] if brute[j] else -1)
    # supernodes: maximal runs of contiguous columns with equal structure
    ptr, _ = sym.supernodes()
    starts = [0] + [j for j in range(1, n) if brute[j - 1] != [j] + brute[j]]
    assert ptr[:-1].tolist() == starts
    # relind by a list search
    rp, rt, ri2 = sym.relind(ptr)
    p = 0
    for J in range(len(ptr) - 1):
        sJ = [ptr[J]] + brute[ptr[J]]
        sJ = sorted(set(range(ptr[J], ptr[J + 1])) | set(brute[ptr[J]]))
        ks = []
        for i in sJ:
            if i >= ptr[J + 1]:
                K = int(np.searchsorted(ptr, i, side="right") - 1)
                if K not in ks:
                    ks.append(K)
        for K in ks:
            sK = sorted(set(range(ptr[K], ptr[K + 1])) | set(brute[ptr[K]]))
            exp = [len(sK) - 1 - sK.index(i) for i in sJ if i in sK]
            assert rt[p] == K and ri2[rp[p]:rp[p + 1]].tolist() == exp
            p += 1
    assert p == len(rt)


@pytest.mark.parametrize("seed", range(8))
def test_numeric_pattern_equals_symbolic_and_dense(seed):
    rs = np.random.RandomState(200 + seed)
    n = int(rs.randint(10, 60))
    A, cp, ri, vx, perm = random_spd(n, rs.uniform(0.03, 0.15), 50 + seed)
    bp, bi, bx = oracle.permute(n, cp, ri, vx, perm)
    sym = oracle.Symbolic(n, bp, bi)
    fac = oracle.Factor(n, bp, bi, bx)
    assert fac.info == 0
    assert np.array_equal(sym.lp, fac.lp) and np.array_equal(sym.li, fac.li)
    P = np.eye(n)[perm]
    Ld = np.linalg.cholesky(P @ A @ P.T)
    dense_pattern = np.abs(Ld) > 0
    Lo = csc_to_dense_lower(n, fac.lp, fac.li, fac.lx)
    assert np.array_equal(dense_pattern, Lo != 0)


# --------------------------------------------------------------------------
# numeric values against LAPACK and closed forms
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(6))
def test_factor_solve_vs_lapack(seed):
    rs = np.random.RandomState(300 + seed)
    n = int(rs.randint(20, 201))
    A, cp, ri, vx, perm = random_spd(n, rs.uniform(0.01, 0.1), 70 + seed)
    bp, bi, bx = oracle.permute(n, cp, ri, vx, perm)
    fac = oracle.Factor(n, bp, bi, bx)
    P = np.eye(n)[perm]
    Ld = np.linalg.cholesky(P @ A @ P.T)
    Lo = csc_to_dense_lower(n, fac.lp, fac.li, fac.lx)
    assert np.max(np.abs(Lo - Ld)) <= 1e-13 * np.max(np.abs(Ld))
    b = rs.uniform(-1, 1, (n, 3))
    x = fac.solve(perm, b)
    xd = np.linalg.solve(A, b)
    assert np.max(np.abs(x - xd)) <= 1e-12 * np.max(np.abs(xd))
    sign, ld = np.linalg.slogdet(A)
    assert sign > 0 and abs(fac.logdet() - ld) <= 1e-12 * abs(ld) + 1e-12
    # residual and backward-error helpers against dense formulas
    B = P @ A @ P.T
    assert oracle.factor_residual(n, bp, bi, bx, fac.lp, fac.li, fac.lx) < 1e-15
    lx = fac.lx * (1.0 + rs.uniform(-1e-7, 1e-7, fac.lx.shape))   # well above rounding
    Lp = csc_to_dense_lower(n, fac.lp, fac.li, lx)
    res = oracle.factor_residual(n, bp, bi, bx, fac.lp, fac.li, lx)
    assert res == pytest.approx(np.linalg.norm(B - Lp @ Lp.T) / np.linalg.norm(B), rel=1e-8)
    assert np.all(oracle.backward_error(n, cp, ri, vx, b, x) < 1e-15)
    xp = x + rs.uniform(-1e-6, 1e-6, x.shape)      # residual well above rounding
    eta = oracle.backward_error(n, cp, ri, vx, b, xp)
    Ainf = np.abs(A).sum(axis=1).max()
    for r in range(3):
        exp = np.abs(b[:, r] - A @ xp[:, r]).max() / (Ainf * np.abs(xp[:, r]).max() + np.abs(b[:, r]).max())
        assert eta[r] == pytest.approx(exp, rel=1e-8)
    y = oracle.spmv(n, cp, ri, vx, b)
    assert np.allclose(y, A @ b, rtol=1e-14, atol=1e-14)


def test_residual_detects_a_wrong_factor():
    A, cp, ri, vx, perm = random_spd(40, 0.1, 9)
    bp, bi, bx = oracle.permute(40, cp, ri, vx, perm)
    fac = oracle.Factor(40, bp, bi, bx)
    assert oracle.factor_residual(40, bp, bi, bx, fac.lp, fac.li, fac.lx) < 1e-15
    lx = fac.lx.copy()
    lx[fac.lp[20]] *= 1.0 + 1e-6                 # one diagonal entry of L
    assert oracle.factor_residual(40, bp, bi, bx, fac.lp, fac.li, lx) > 1e-9


def test_logdet_2d_dirichlet_closed_form():
    """2D 64x64 Dirichlet 5-point + 1e-3: eigenvalues
    1e-3 + 4 sin^2(p pi / 2(k+1)) + 4 sin^2(q pi / 2(k+1)), p, q = 1..k."""
    k = 64
    p = gridgen.workload("2d64")
    ref = oracle.reference(p)
    s = 4 * np.sin(np.arange(1, k + 1) * np.pi / (2 * (k + 1))) ** 2
    exact = np.log(1e-3 + s[:, None] + s[None, :]).sum()
    assert abs(ref["fac"].logdet() - exact) <= 1e-12 * abs(exact)
    # cross-check under the nested-dissection reading (the counts of an
    # independent symbolic run): nnz(L) = 88,130 and sum c_j^2 = 3,717,076
    assert ref["sym"].nnz == 88130 and ref["sym"].flops() == 3717076


def test_logdet_3d_neumann_closed_form():
    """Constant-coefficient Neumann grid Laplacian + delta: eigenvalues
    delta + sum_d 4 sin^2(p_d pi / 2k), p_d = 0..k-1."""
    k, delta = 9, 1e-2
    p = gridgen.laplacian_neumann_varcoef((k, k, k), 1.0, 1.0, delta, seed=1)
    ref = oracle.reference(p)
    s = 4 * np.sin(np.arange(k) * np.pi / (2 * k)) ** 2
    lam = delta + s[:, None, None] + s[None, :, None] + s[None, None, :]
    exact = np.log(lam).sum()
    assert abs(ref["fac"].logdet() - exact) <= 1e-11 * abs(exact)


def test_logdet_tridiagonal_recurrence():
    """det of a tridiagonal SPD matrix by the three-term recurrence
    f_k = a_k f_{k-1} - b_{k-1}^2 f_{k-2}, tracked as ratios."""
    rs = np.random.RandomState(7)
    n = 300
    a = rs.uniform(2.5, 4.0, n)
    b = rs.uniform(-1.0, 1.0, n - 1)
    A = np.diag(a) + np.diag(b, -1) + np.diag(b, 1)
    cp, ri, vx = lower_csc_from_dense(A)
    fac = oracle.Factor(n, cp, ri, vx)
    r_prev, logdet = a[0], math.log(a[0])
    for k in range(1, n):
        r = a[k] - b[k - 1] ** 2 / r_prev       # r_k = f_k / f_{k-1}
        logdet += math.log(r)
        r_prev = r
    assert abs(fac.logdet() - logdet) <= 1e-12 * abs(logdet)


def test_flop_convention_counts_operations():
    """sum_j c_j^2 = #sqrt + #div + 2 * #multiply-add of column Cholesky on the
    structural nonzeros (counted in a plain instrumented loop)."""
    A, cp, ri, vx, perm = random_spd(35, 0.12, 11)
    bp, bi, bx = oracle.permute(35, cp, ri, vx, perm)
    sym = oracle.Symbolic(35, bp, bi)
    B = dense_from_lower(35, bp, bi, np.ones_like(bx))
    nz = B != 0
    n = 35
    ops = 0
    for j in range(n):                       # right-looking on the pattern only
        ops += 1                             # sqrt
        rows = [i for i in range(j + 1, n) if nz[i, j]]
        ops += len(rows)                     # divisions
        for c in rows:
            for r in rows:
                if r >= c:
                    nz[r, c] = True
                    ops += 2                 # multiply-add
    assert ops == sym.flops()


def test_manufactured_solution_and_backward_error():
    p = gridgen.workload("2d64")
    rs = np.random.RandomState(1)
    xs = rs.uniform(-1, 1, (p.n, 2))
    b = oracle.spmv(p.n, p["colptr"], p["rowind"], p["values"], xs)
    ref = oracle.reference(p, b)
    # kappa(A) < 2000 for this matrix (eigenvalues in [0.0046, 8.001])
    assert np.max(np.abs(ref["x"] - xs)) <= 2000 * 2.2e-16 * 50
    assert np.all(oracle.backward_error(p.n, p["colptr"], p["rowind"], p["values"], b, ref["x"]) < 1e-15)
    bp, bi, bx = ref["B"]
    f = ref["fac"]
    assert oracle.factor_residual(p.n, bp, bi, bx, f.lp, f.li, f.lx) <= 1e-13


def test_not_spd_reports_first_bad_pivot():
    A = np.diag([4.0, 3.0, 2.0, 1.0, 5.0, -1.0, 2.0])
    cp, ri, vx = lower_csc_from_dense(A)
    assert oracle.Factor(7, cp, ri, vx).info == 6
    B = np.array([[1.0, 2.0], [2.0, 1.0]])
    cp, ri, vx = lower_csc_from_dense(B)
    assert oracle.Factor(2, cp, ri, vx).info == 2


def test_permute_rejects_bad_perm():
    A, cp, ri, vx, perm = random_spd(10, 0.2, 1)
    bad = perm.copy(); bad[0] = bad[1]
    with pytest.raises(ValueError):
        oracle.permute(10, cp, ri, vx, bad)


def test_sampled_column_residual_matches_dense():
    A, cp, ri, vx, perm = random_spd(50, 0.1, 21)
    bp, bi, bx = oracle.permute(50, cp, ri, vx, perm)
    fac = oracle.Factor(50, bp, bi, bx)
    lx = fac.lx * (1.0 + np.random.RandomState(2).uniform(-1e-7, 1e-7, fac.lx.shape))
    Lp = csc_to_dense_lower(50, fac.lp, fac.li, lx)
    P = np.eye(50)[perm]
    B = P @ A @ P.T
    cols = np.array([0, 7, 23, 49])
    got = oracle.factor_residual_cols(50, bp, bi, bx, fac.lp, fac.li, lx, cols)
    R = B - Lp @ Lp.T
    for q, j in enumerate(cols):
        exp = np.linalg.norm(R[j:, j]) / np.linalg.norm(B[j:, j])
        assert got[q] == pytest.approx(exp, rel=1e-6)


# --------------------------------------------------------------------------
# selected inverse and gradients
# --------------------------------------------------------------------------

@pytest.mark.parametrize("seed", range(4))
def test_selected_inverse_vs_dense_inverse(seed):
    rs = np.random.RandomState(800 + seed)
    n = int(rs.randint(10, 120))
    A, cp, ri, vx, perm = random_spd(n, rs.uniform(0.03, 0.15), 90 + seed)
    bp, bi, bx = oracle.permute(n, cp, ri, vx, perm)
    fac = oracle.Factor(n, bp, bi, bx)
    zx = fac.selinv()
    P = np.eye(n)[perm]
    Zd = np.linalg.inv(P @ A @ P.T)
    Zsel = csc_to_dense_lower(n, fac.lp, fac.li, zx)
    mask = csc_to_dense_lower(n, fac.lp, fac.li, np.ones_like(zx)) != 0
    assert np.max(np.abs(Zsel[mask] - Zd[mask])) <= 1e-12 * np.max(np.abs(Zd))
    zA = oracle.inverse_on_pattern(dict(n=n, colptr=cp, rowind=ri), fac, perm)
    Ai = np.linalg.inv(A)
    cols = np.repeat(np.arange(n), np.diff(cp))
    assert np.allclose(zA, Ai[ri, cols], rtol=1e-12, atol=1e-14 * np.max(np.abs(Ai)))


def test_gradient_vs_central_differences():
    """d/da_ij of  w^T A^{-1} b + log det A  with a_ij and a_ji moved together."""
    rs = np.random.RandomState(3)
    n = 40
    A, cp, ri, vx, perm = random_spd(n, 0.1, 33)
    prob = dict(n=n, colptr=cp, rowind=ri, values=vx, perm=perm)
    b = rs.uniform(-1, 1, (n, 3))
    w = rs.normal(size=(n, 3))

    def loss(vals):
        bp, bi, bx = oracle.permute(n, cp, ri, vals, perm)
        f = oracle.Factor(n, bp, bi, bx)
        x = f.solve(perm, b)
        return float(np.sum(w * x)) + f.logdet()

    bp, bi, bx = oracle.permute(n, cp, ri, vx, perm)
    fac = oracle.Factor(n, bp, bi, bx)
    x = fac.solve(perm, b)
    g, xbar = oracle.gradient(prob, fac, w, x, 1.0)
    picks = rs.choice(len(vx), 20, replace=False)
    for t in picks:
        h = 1e-6 * abs(vx[t])
        vp = vx.copy(); vp[t] += h
        vm = vx.copy(); vm[t] -= h
        fd = (loss(vp) - loss(vm)) / (2 * h)
        assert abs(fd - g[t]) <= 1e-6 * max(1.0, abs(fd)), (t, fd, g[t])
    # d loss / d b = A^{-1} w
    assert np.allclose(xbar, np.linalg.solve(A, w), rtol=1e-10, atol=1e-12)
    # dense reference: G = -xbar x^T + A^{-1}, symmetrised onto the lower entries
    G = -xbar @ x.T + np.linalg.inv(A)
    cols = np.repeat(np.arange(n), np.diff(cp))
    dense = np.where(ri == cols, G[ri, cols], G[ri, cols] + G[cols, ri])
    assert np.allclose(g, dense, rtol=1e-9, atol=1e-12)


# --------------------------------------------------------------------------
# the multi-threaded timing variant of the oracle's numeric loops
# --------------------------------------------------------------------------

def _threaded_vs_serial(n, cp, ri, vx, perm, threads):
    bp, bi, bx = oracle.permute(n, cp, ri, vx, perm)
    a = oracle.Factor(n, bp, bi, bx)
    b = oracle.Factor(n, bp, bi, bx, threads=threads)
    assert a.info == b.info
    if a.info == 0:
        assert np.array_equal(a.lp, b.lp) and np.array_equal(a.li, b.li)
        scale = np.maximum.reduceat(np.abs(a.lx), a.lp[:-1]) if n else np.zeros(0)
        err = np.maximum.reduceat(np.abs(a.lx - b.lx), a.lp[:-1]) if n else np.zeros(0)
        # the cmod sums run in another order: rounding differences only, far
        # below what a dropped or misplaced term would cause
        assert np.all(err <= 1e-10 * scale)
        assert oracle.factor_residual(n, bp, bi, bx, b.lp, b.li, b.lx) <= 1e-13
    return a, b


@pytest.mark.parametrize("threads", [0, 3])
def test_threaded_factor_matches_serial(threads):
    for seed in (1, 2, 3):
        A, cp, ri, vx, p = random_spd(120, 0.04, seed)
        _threaded_vs_serial(120, cp, ri, vx, p, threads)
    g = gridgen.laplacian_neumann_varcoef((9, 8, 7), 1e-2, 1e2, 1e-3, seed=4)
    _threaded_vs_serial(g.n, g["colptr"], g["rowind"], g["values"], g["perm"], threads)
    q = gridgen.block_diagonal([gridgen.laplacian_2d_dirichlet(k) for k in (3, 11, 6)])
    _threaded_vs_serial(q.n, q["colptr"], q["rowind"], q["values"], q["perm"], threads)


def test_threaded_factor_reports_the_first_bad_pivot():
    # two independent failing columns at the same etree height: the smaller wins
    A = np.diag([4.0, -3.0, 2.0, 1.0, 5.0, -1.0, 2.0])
    cp, ri, vx = lower_csc_from_dense(A)
    _, b = _threaded_vs_serial(7, cp, ri, vx, None, 0)
    assert b.info == 2
    cp, ri, vx = lower_csc_from_dense(np.zeros((0, 0)))
    assert oracle.Factor(0, np.zeros(1, np.int64), np.zeros(0, np.int32), np.zeros(0), threads=0).info == 0


@pytest.mark.parametrize("threads", [0, 3])
def test_staged_factor_equals_one_piece_run(threads):
    """The timing form that runs the multi-threaded factor in pieces of
    elimination-tree heights gives the one-piece result bit for bit, for any
    split, and its per-height work adds up to the flop convention."""
    g = gridgen.laplacian_neumann_varcoef((10, 9, 8), 1e-2, 1e2, 1e-6, seed=6)
    bp, bi, bx = oracle.permute(g.n, g["colptr"], g["rowind"], g["values"], g["perm"])
    one = oracle.Factor(g.n, bp, bi, bx, threads=threads)
    rs = np.random.RandomState(threads)
    for trial in range(3):
        S = oracle.StagedFactor(g.n, bp, bi, bx, threads=threads)
        w = S.work()
        assert len(w) == S.max_height + 1
        assert w.sum() == S.sym.flops()
        cuts = np.unique(np.concatenate([[0, S.max_height + 1], rs.randint(0, S.max_height + 1, 4)]))
        for a, b in zip(cuts[:-1], cuts[1:]):
            S.run(a, b)
        f = S.finish()
        assert f.info == 0
        assert np.array_equal(f.lp, one.lp) and np.array_equal(f.li, one.li) and np.array_equal(f.lx, one.lx)


def test_residual_parts_match_dense_frobenius():
    """The column-parallel factor residual against the dense formula
    ||B - L L^T||_F / ||B||_F, on a perturbed factor (so that the residual is
    far above rounding), and its per-column values against dense columns."""
    A, cp, ri, vx, perm = random_spd(60, 0.1, 23)
    bp, bi, bx = oracle.permute(60, cp, ri, vx, perm)
    fac = oracle.Factor(60, bp, bi, bx)
    lx = fac.lx * (1.0 + np.random.RandomState(5).uniform(-1e-7, 1e-7, fac.lx.shape))
    Lp = csc_to_dense_lower(60, fac.lp, fac.li, lx)
    P = np.eye(60)[perm]
    B = P @ A @ P.T
    R = B - Lp @ Lp.T
    tot, cols = oracle.factor_residual_parts(60, bp, bi, bx, fac.lp, fac.li, lx, threads=3)
    assert tot == pytest.approx(np.linalg.norm(R) / np.linalg.norm(B), rel=1e-8)
    assert tot == pytest.approx(oracle.factor_residual(60, bp, bi, bx, fac.lp, fac.li, lx), rel=1e-8)
    w = np.ones(60); w[1:] = 2.0
    for j in (0, 11, 37, 59):
        rj = R[j:, j]; bj = B[j:, j]
        exp = np.sqrt(np.sum(w[: len(rj)] * rj ** 2) / np.sum(w[: len(bj)] * bj ** 2))
        assert cols[j] == pytest.approx(exp, rel=1e-6)
