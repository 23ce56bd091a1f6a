"""The C-ABI library: loads without a GPU, exports every declared symbol, validates
arguments, and its host symbolic analysis matches the oracle bit for bit."""
import os
import re

import numpy as np
import pytest

import gridgen
import oracle
from golden_fig1 import load as load_fig1
from helpers import lower_csc_from_dense, random_spd
from lib_fixture import ROOT, chol


def _declared():
    src = open(os.path.join(ROOT, "include", "chol.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(chol_[a-z_]+)\s*\(", src)))


def test_exports_every_declared_symbol():
    P = chol()
    names = _declared()
    assert "chol_analyze" in names and "chol_factor" in names and "chol_solve" in names
    for nm in names:
        assert hasattr(P.lib(), nm), nm
        assert nm in P.EXPORTED, nm


def test_update_mode_validation():
    P = chol()
    A = np.eye(3) * 2.0
    cp, ri, _ = lower_csc_from_dense(A)
    o = P.chol_default_options()
    assert o.update_mode == P.CHOL_UPDATE_RL
    o.update_mode = 2
    assert P.chol_analyze(3, cp, ri, None, o)[0] == -5
    o.update_mode = P.CHOL_UPDATE_RLB
    rc, h = P.chol_analyze(3, cp, ri, None, o)
    assert rc == 0
    P.chol_destroy(h)
    o.precision = P.CHOL_PREC_FP32          # RLB is binary64 only
    assert P.chol_analyze(3, cp, ri, None, o)[0] == -5
    o.precision = P.CHOL_PREC_FP64
    o.persistent = 1                        # ... and not in the persistent launch
    assert P.chol_analyze(3, cp, ri, None, o)[0] == -5


def test_strerror_and_defaults():
    P = chol()
    assert "success" in P.chol_strerror(0)
    assert "positive definite" in P.chol_strerror(5)
    assert "argument" in P.chol_strerror(-3)
    o = P.chol_default_options()
    assert (o.precision, o.small_max_cols, o.small_max_panel, o.block_cols) == (0, 64, 4096, 64)


def test_argument_validation():
    P = chol()
    A = np.array([[4.0, 1.0, 0.0], [1.0, 4.0, 1.0], [0.0, 1.0, 4.0]])
    cp, ri, vx = lower_csc_from_dense(A)
    assert P.chol_analyze(-1, cp, ri)[0] == -1
    bad = cp.copy(); bad[0] = 1
    assert P.chol_analyze(3, bad, ri)[0] == -2
    nodiag = ri.copy(); nodiag[0] = 1
    assert P.chol_analyze(3, cp, nodiag)[0] == -3
    unsorted = np.array([0, 2, 1, 1, 2], np.int32)
    assert P.chol_analyze(3, np.array([0, 3, 4, 5]), unsorted)[0] == -3
    assert P.chol_analyze(3, cp, ri, np.array([0, 0, 1]))[0] == -4
    o = P.chol_default_options(); o.block_cols = 128
    assert P.chol_analyze(3, cp, ri, None, o)[0] == -5
    rc, h = P.chol_analyze(3, cp, ri)
    assert rc == 0
    assert P.chol_solve(h, None, 1) == P.CHOL_ESTATE or P.chol_solve(h, 0, 1) in (-2, P.CHOL_ESTATE)
    assert P.chol_logdet(h)[0] == P.CHOL_ESTATE
    P.chol_destroy(h)
    rc, h = P.chol_analyze(0, np.zeros(1, np.int64), np.zeros(0, np.int32))
    assert rc == 0 and P.chol_get_info(h).nsuper == 0
    P.chol_destroy(h)


def _compare_symbolic(n, colptr, rowind, perm):
    P = chol()
    rc, h = P.chol_analyze(n, colptr, rowind, perm)
    assert rc == 0
    got = P.chol_get_symbolic(h)
    info = P.chol_get_info(h)
    P.chol_destroy(h)
    bp, bi, _ = oracle.permute(n, colptr, rowind, None, perm)
    sym = oracle.Symbolic(n, bp, bi)
    assert np.array_equal(got["parent"], sym.parent)
    assert np.array_equal(got["colcount"], sym.colcount)
    ptr, sparent = sym.supernodes()
    assert np.array_equal(got["snode_ptr"], ptr)
    assert np.array_equal(got["snode_parent"], sparent)
    # struct(J) = struct of its first column
    for J in range(len(ptr) - 1):
        f = ptr[J]
        assert np.array_equal(got["rows"][got["row_ptr"][J]:got["row_ptr"][J + 1]],
                              sym.li[sym.lp[f]:sym.lp[f + 1]])
    assert info.nnz_l == sym.nnz and info.flops == sym.flops()
    return got, sym, ptr


@pytest.mark.parametrize("seed", range(8))
def test_symbolic_bit_exact_random(seed):
    rs = np.random.RandomState(500 + seed)
    n = int(rs.randint(5, 120))
    A, cp, ri, vx, perm = random_spd(n, rs.uniform(0.02, 0.2), seed)
    got, sym, ptr = _compare_symbolic(n, cp, ri, perm)
    rp, rt, rv = sym.relind(ptr)
    assert np.array_equal(got["relind_ptr"], rp)
    assert np.array_equal(got["relind_target"], rt)
    assert np.array_equal(got["relind"], rv)


def test_symbolic_fig1_and_relind_golden():
    g = load_fig1()
    A = np.zeros((15, 15))
    for j, rows in g["cols"].items():
        for i in rows:
            A[i - 1, j - 1] = A[j - 1, i - 1] = -1.0
    A[np.diag_indices(15)] = 20.0
    cp, ri, _ = lower_csc_from_dense(A)
    got, sym, ptr = _compare_symbolic(15, cp, ri, None)
    rp, rt, rv = sym.relind(ptr)
    assert np.array_equal(got["relind"], rv)
    # J1 -> J3 pair is the first pair: [4 3 1] (definition reading of Sec. II-A)
    assert got["relind_target"][0] == 2 and got["relind"][:3].tolist() == [4, 3, 1]


@pytest.mark.parametrize("name", ["2d64", "3d10", "elast5", "batch"])
def test_symbolic_bit_exact_workloads(name):
    if name == "3d10":
        p = gridgen.laplacian_neumann_varcoef((10, 9, 11), 1e-2, 1e2, 1e-6, seed=9)
    elif name == "elast5":
        p = gridgen.elasticity_27pt(5)
    elif name == "batch":
        p = gridgen.block_diagonal(gridgen.batch_2d(count=6, kmin=4, kmax=12, seed=4))
    else:
        p = gridgen.workload(name)
    got, sym, ptr = _compare_symbolic(p.n, p["colptr"], p["rowind"], p["perm"])
    if p.n <= 4096:
        rp, rt, rv = sym.relind(ptr)
        assert np.array_equal(got["relind_ptr"], rp) and np.array_equal(got["relind"], rv)


@pytest.mark.parametrize("growth", [0.02, 0.1, 0.25, 1.0])
@pytest.mark.parametrize("case", ["2d20", "3d7", "rand"])
def test_relaxed_merging_matches_oracle(case, growth):
    """Sec. IV setup: the merged storage partition and the merged structures are
    those of the plain greedy restatement in oracle.merge."""
    from oracle.merge import merged_partition
    P = chol()
    if case == "2d20":
        p = gridgen.laplacian_2d_dirichlet(20)
    elif case == "3d7":
        p = gridgen.laplacian_neumann_varcoef((7, 6, 7), 1e-2, 1e2, 1e-6, seed=1)
    else:
        A, cp, ri, vx, perm = random_spd(150, 0.03, 77)
        p = dict(n=150, colptr=cp, rowind=ri, values=vx, perm=perm)
    o = P.chol_default_options()
    o.merge_growth = growth
    rc, h = P.chol_analyze(p["n"], p["colptr"], p["rowind"], p["perm"], o)
    assert rc == 0
    part = P.chol_get_partition(h)
    info = P.chol_get_info(h)
    canon = P.chol_get_symbolic(h)
    P.chol_destroy(h)
    bp, bi, _ = oracle.permute(p["n"], p["colptr"], p["rowind"], None, p["perm"])
    sym = oracle.Symbolic(p["n"], bp, bi)
    ptr, structs = merged_partition(sym, growth)
    assert np.array_equal(part["snode_ptr"], ptr)
    for J, st in enumerate(structs):
        assert part["rows"][part["row_ptr"][J]:part["row_ptr"][J + 1]].tolist() == st
    assert info.nnz_stored <= (1.0 + growth) * info.nnz_l
    # the canonical outputs do not change with merging
    assert np.array_equal(canon["snode_ptr"], sym.supernodes()[0])


def test_analyze_batch_validation_and_symbolic():
    P = chol()
    probs = gridgen.batch_2d(count=5, kmin=3, kmax=7, seed=4)
    bd = gridgen.block_diagonal(probs)
    offs = bd["meta"]["offsets"].astype(np.int32)
    rc, h = P.chol_analyze_batch(5, offs, bd["colptr"], bd["rowind"], bd["perm"])
    assert rc == 0
    info = P.chol_get_info(h)
    assert info.nsys == 5
    got = P.chol_get_symbolic(h)
    P.chol_destroy(h)
    bp, bi, _ = oracle.permute(bd.n, bd["colptr"], bd["rowind"], None, bd["perm"])
    sym = oracle.Symbolic(bd.n, bp, bi)
    assert np.array_equal(got["parent"], sym.parent)
    # a bad sys_ptr, an entry coupling two systems, a permutation across systems
    bad = offs.copy(); bad[2] = bad[1] - 1
    assert P.chol_analyze_batch(5, bad, bd["colptr"], bd["rowind"], bd["perm"])[0] == -2
    wrong = offs.copy(); wrong[1] += 1
    assert P.chol_analyze_batch(5, wrong, bd["colptr"], bd["rowind"], bd["perm"])[0] == -4
    perm = bd["perm"].copy(); perm[[0, offs[1]]] = perm[[offs[1], 0]]
    assert P.chol_analyze_batch(5, offs, bd["colptr"], bd["rowind"], perm)[0] == -4
