"""Mixed precision (scaled binary32 panels; SIMT, TF32 or BF16 tensor-core
updates) with binary64 iterative refinement, against the FP64 oracle.

The reduced-precision factor is stated as its error against the oracle's L
(per-column relative max error, bounded per mode); the refined solution must
reach the 1e-10 normwise backward error and agree with the oracle's x.
"""
import numpy as np
import pytest

import gridgen
import oracle
from gpu_util import colmajor, to_dev
from lib_fixture import chol

pytestmark = pytest.mark.gpu

MODES = {"fp32": 1, "tf32": 2, "bf16": 3}
# Backward error of the reduced-precision factor, ||P A P^T - L L^T||_F / ||A||_F
# (independent of the conditioning): the unit roundoff of the update operands
# (2^-24, 2^-11 truncation, 2^-9) times a modest growth factor.
RES_TOL = {"fp32": 1e-5, "tf32": 1e-2, "bf16": 5e-2}
# Per-column relative error of L itself, bounded only for the well-conditioned
# 2D grid (kappa < 2000); elsewhere it is reported (it scales with kappa).
L_TOL_2D = {"fp32": 1e-4, "tf32": 5e-2, "bf16": 2e-1}


def _run(problem, mode, b, merge=0.0, tau=1e-3, nb=64, small_rows=128, max_iter=200, static_pivot=0, extra=None):
    import torch
    P = chol()
    o = P.chol_default_options()
    for k, v in (extra or {}).items():
        setattr(o, k, v)
    o.precision = MODES[mode]
    o.merge_growth = merge
    o.pivot_tau = tau
    o.block_cols = nb
    o.small_max_rows = small_rows
    o.static_pivot = static_pivot
    rc, h = P.chol_analyze(problem["n"], problem["colptr"], problem["rowind"], problem["perm"], o)
    assert rc == 0, rc
    try:
        assert P.chol_factor(h, to_dev(problem["values"])) == 0
        info = P.chol_get_info(h)
        lp, li, lx = P.chol_get_factor(h)
        rc, ld = P.chol_logdet(h)
        assert rc == 0
        B = colmajor(b)
        X = torch.zeros_like(B)
        nrhs = b.shape[1]
        rc, iters, berr = P.chol_solve_refine(h, B, X, nrhs, 1e-10, max_iter)
        torch.cuda.synchronize()
        x = X.cpu().numpy()
        X0 = colmajor(b)
        assert P.chol_solve(h, X0, nrhs) == 0
        x0 = X0.cpu().numpy()
        stats = P.chol_get_stats(h)
    finally:
        P.chol_destroy(h)
    return dict(rc=rc, iters=iters, berr=berr, x=x, x0=x0, L=(lp, li, lx), logdet=ld, info=info, stats=stats)


def _check(problem, mode, nrhs=2, **kw):
    b = gridgen.rhs_uniform(problem["n"], nrhs, seed=11)
    ref = oracle.reference(problem, b)
    got = _run(problem, mode, b, **kw)
    f = ref["fac"]
    lp, li, lx = got["L"]
    assert np.array_equal(lp, f.lp) and np.array_equal(li, f.li)
    colmax = np.maximum.reduceat(np.abs(f.lx), f.lp[:-1])
    colerr = np.maximum.reduceat(np.abs(lx - f.lx), f.lp[:-1])
    factor_err = float(np.max(colerr / colmax))
    bp, bi, bx = ref["B"]
    fres = oracle.factor_residual(problem["n"], bp, bi, bx, lp, li, lx)
    print("mode=%s factor residual %.3e, max per-column L error %.3e, refine iters %d, perturbed %d"
          % (mode, fres, factor_err, got["iters"], got["info"].perturbed_pivots))
    if got["info"].perturbed_pivots == 0:     # static pivots perturb A on purpose
        assert fres <= RES_TOL[mode], fres
    assert got["rc"] == 0, (got["rc"], got["berr"], got["iters"])
    assert np.all(got["berr"] <= 1e-10)
    eta = oracle.backward_error(problem["n"], problem["colptr"], problem["rowind"], problem["values"], b, got["x"])
    assert np.all(eta <= 1e-10), eta
    rel = np.max(np.abs(got["x"] - ref["x"])) / np.max(np.abs(ref["x"]))
    return got, factor_err, rel, ref


@pytest.mark.parametrize("mode", list(MODES))
def test_2d64_mixed_refined(mode):
    got, ferr, rel, ref = _check(gridgen.workload("2d64"), mode)
    assert ferr <= L_TOL_2D[mode], ferr
    assert rel <= 1e-9
    assert abs(got["logdet"] - ref["fac"].logdet()) <= RES_TOL[mode] * abs(ref["fac"].logdet())


@pytest.mark.parametrize("mode", list(MODES))
@pytest.mark.parametrize("merge", [0.0, 0.1])
def test_3d_varcoef_mixed_refined(mode, merge):
    p = gridgen.laplacian_neumann_varcoef((16, 15, 14), 1e-2, 1e2, 1e-6, seed=8)
    # the shifted Neumann grid is nearly singular: bf16 updates can lose
    # definiteness there, so that mode runs with static pivoting
    got, ferr, rel, ref = _check(p, mode, nrhs=3, merge=merge, small_rows=32,
                                 static_pivot=1 if mode == "bf16" else 0)
    assert got["stats"]["panel"]["launches"] > 0 and got["stats"]["syrk"]["launches"] > 0


@pytest.mark.parametrize("mode", ["fp32", "tf32", "bf16"])
def test_elasticity_mixed_refined(mode):
    p = gridgen.elasticity_27pt(7, seed=3)
    _check(p, mode, nrhs=1, merge=0.05, small_rows=64)


def _dense_problem(n):
    from helpers import lower_csc_from_dense
    rs = np.random.RandomState(n)
    M = rs.normal(size=(n, n))
    A = M @ M.T + n * np.eye(n)
    cp, ri, vx = lower_csc_from_dense(A)
    return dict(n=n, colptr=cp, rowind=ri, values=vx, perm=np.arange(n, dtype=np.int32))


def _outer_launches(n, pairs):
    """Outer-update launches of one dense blocked supernode of n columns.
    Tensor-core modes (pairs): block b = 2p updates the next block's columns
    (K = 256) when there are any; block b = 2p + 1 updates the next pair's
    columns (K = 512, the pair) on the critical stream and, when there are
    columns beyond those, the rest on the side stream. binary32 SIMT tiles:
    every block updates the next block's columns, then the rest."""
    if pairs:
        return sum((n > 256 * (b + 1)) + (b % 2 == 1 and n > 256 * (b + 3)) for b in range((n + 255) // 256))
    return sum((n > 256 * (b + 1)) + (n > 256 * (b + 2)) for b in range((n + 255) // 256))


@pytest.mark.parametrize("n", [31, 32, 33, 64, 65, 100, 129, 255, 256, 257, 300, 520, 1100])
def test_fp32_blocked_diagonal_blocks_of_every_width(n):
    # the small-supernode kernel is off, so the whole matrix is one blocked
    # supernode: one panel launch per 256-column outer block (full and ragged
    # 64-column sub-blocks inside, 1 to 64 columns in the last one), and the
    # update of the columns right of each block
    got, ferr, rel, ref = _check(_dense_problem(n), "fp32", nrhs=2, extra=dict(small_max_cols=1, small_max_panel=1))
    assert got["info"].fp64_fallbacks == 0
    assert got["stats"]["panel"]["launches"] == (n + 255) // 256
    assert got["stats"]["gemm"]["launches"] == _outer_launches(n, pairs=False)
    assert ferr <= 1e-5, ferr


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
@pytest.mark.parametrize("n", [300, 520, 777, 1100])
def test_tensor_core_outer_updates_dense(mode, n):
    # several outer blocks: the tcgen05 updates of the columns right of each
    # pair of blocks (K = 256 after the first block, K = 512 after the second,
    # the columns the next panels need first, the rest on the side stream)
    got, ferr, rel, ref = _check(_dense_problem(n), mode, nrhs=2, extra=dict(small_max_cols=1, small_max_panel=1))
    assert got["stats"]["panel"]["launches"] == (n + 255) // 256
    assert got["stats"]["gemm"]["launches"] == _outer_launches(n, pairs=True)
    assert ferr <= (1e-2 if mode == "tf32" else 5e-2), ferr


def test_fp64_fallback_blocks_are_counted_and_exact():
    """tau close to 1 sends every blocked diagonal block through the binary64 redo."""
    p = gridgen.laplacian_neumann_varcoef((12, 12, 12), 1e-2, 1e2, 1e-6, seed=4)
    got, ferr, rel, ref = _check(p, "fp32", nrhs=1, tau=0.999, small_rows=16)
    assert got["info"].fp64_fallbacks > 0


def test_mixed_not_spd_reports_column():
    P = chol()
    p = gridgen.workload("2d64")
    vals = p["values"].copy()
    vals[p["colptr"][777]] = -1.0
    q = dict(p, values=vals)
    bp, bi, bx = oracle.permute(q["n"], q["colptr"], q["rowind"], q["values"], q["perm"])
    info = oracle.Factor(q["n"], bp, bi, bx).info
    for mode in MODES.values():
        o = P.chol_default_options()
        o.precision = mode
        rc, h = P.chol_analyze(q["n"], q["colptr"], q["rowind"], q["perm"], o)
        assert P.chol_factor(h, to_dev(q["values"])) == info
        P.chol_destroy(h)


def test_fp64_refine_is_one_solve():
    import torch
    P = chol()
    p = gridgen.workload("2d64")
    rc, h = P.chol_analyze(p["n"], p["colptr"], p["rowind"], p["perm"])
    assert P.chol_factor(h, to_dev(p["values"])) == 0
    b = gridgen.rhs_uniform(p["n"], 2, seed=3)
    B = colmajor(b)
    X = torch.zeros_like(B)
    rc, iters, berr = P.chol_solve_refine(h, B, X, 2, 1e-12, 5)
    P.chol_destroy(h)
    assert rc == 0 and iters == 0 and np.all(berr <= 1e-15)


def test_static_pivoting_bf16_3d_refines():
    """BF16 updates lose definiteness on the near-singular shifted Neumann grid;
    with static pivoting the factor completes (pivots raised to tau are counted)
    and refinement (conjugate gradients preconditioned by the factor) still
    reaches the 1e-10 backward error."""
    p = gridgen.laplacian_neumann_varcoef((20, 20, 20), 1e-2, 1e2, 1e-6, seed=2)
    b = gridgen.rhs_uniform(p["n"], 1, seed=2)
    import torch
    P = chol()
    o = P.chol_default_options()
    o.precision, o.merge_growth, o.static_pivot = 3, 0.1, 1
    rc, h = P.chol_analyze(p["n"], p["colptr"], p["rowind"], p["perm"], o)
    try:
        assert P.chol_factor(h, to_dev(p["values"])) == 0
        B = colmajor(b)
        X = torch.zeros_like(B)
        rc, iters, berr = P.chol_solve_refine(h, B, X, 1, 1e-10, 200)
        torch.cuda.synchronize()
        assert rc == 0, (rc, iters, berr)
        eta = oracle.backward_error(p["n"], p["colptr"], p["rowind"], p["values"], b, X.cpu().numpy())
        assert np.all(eta <= 1e-10)
    finally:
        P.chol_destroy(h)


@pytest.mark.parametrize("mode", ["tf32", "bf16"])
def test_elasticity_32_tensor_core_launch_shapes_and_unrefined_factor(mode):
    """3D 32^3 x 3-dof elasticity with the benchmark's options: the factor
    takes the tcgen05 update on both rings (2-stage, three CTAs per SM, for
    grids of at least two tiles per SM; 6-stage otherwise) and the outer
    updates right of every pair of outer blocks (K = 256 and 512). Before any refinement the
    low-precision factor's backward error on sampled columns is within the
    mode's bound, and refinement then reaches 1e-10 against the oracle's A."""
    import torch
    P = chol()
    p = gridgen.elasticity_27pt(32, seed=3)
    b = gridgen.rhs_uniform(p.n, 1, seed=4)
    o = P.chol_default_options()
    o.precision = MODES[mode]
    o.merge_growth = 0.1
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"], o)
    assert rc == 0
    try:
        assert P.chol_factor(h, to_dev(p["values"])) == 0
        info = P.chol_get_info(h)
        stats = P.chol_get_stats(h)
        print("%s: panel launches %d, tcgen05 launches shallow %d deep %d, outer updates %d, SYRK %d"
              % (mode, info.panel_launches, info.tc_launches_shallow, info.tc_launches_deep,
                 stats["gemm"]["launches"], stats["syrk"]["launches"]))
        assert info.tc_launches_shallow > 0 and info.tc_launches_deep > 0
        assert stats["gemm"]["launches"] > 0 and info.panel_launches == stats["panel"]["launches"] > 0
        lp, li, lx = P.chol_get_factor(h)
        bp, bi, bx = oracle.permute(p.n, p["colptr"], p["rowind"], p["values"], p["perm"])
        # the factor approximates D B D (D = diag(B)^-1/2, B = P A P^T): compare
        # D L against it, the residual the mode's bound is about
        d = 1.0 / np.sqrt(bx[bp[:-1]])
        bcol = np.repeat(np.arange(p.n), np.diff(bp))
        bxs = bx * d[bi] * d[bcol]
        lxs = lx * d[li]
        rs = np.random.RandomState(1)
        cols = np.unique(np.concatenate([rs.randint(0, p.n, 200), np.arange(p.n - 300, p.n)]))
        res = oracle.factor_residual_cols(p.n, bp, bi, bxs, lp, li, lxs, cols)
        print("%s: unrefined factor residual on %d columns: max %.3e" % (mode, len(cols), res.max()))
        assert np.all(res <= RES_TOL[mode]), res.max()
        B = colmajor(b)
        X = torch.zeros_like(B)
        rc, iters, berr = P.chol_solve_refine(h, B, X, 1, 1e-10, 100)
        torch.cuda.synchronize()
        assert rc == 0, (rc, iters, berr)
        eta = oracle.backward_error(p.n, p["colptr"], p["rowind"], p["values"], b, X.cpu().numpy())
        assert np.all(eta <= 1e-10), eta
    finally:
        P.chol_destroy(h)
