"""Selected inverse and the adjoint (gradients of sum w^T x + log det A with
respect to b and to A's stored entries), against the oracle, dense references
and central finite differences."""
import numpy as np
import pytest

import gridgen
import oracle
from gpu_util import colmajor, to_dev
from helpers import random_spd
from lib_fixture import chol

pytestmark = pytest.mark.gpu


def _opts(P, merge=0.0, small=(64, 4096, 128), nb=64):
    o = P.chol_default_options()
    o.merge_growth = merge
    o.small_max_cols, o.small_max_panel, o.small_max_rows = small
    o.block_cols = nb
    return o


def _selinv(p, o):
    import torch
    P = chol()
    rc, h = P.chol_analyze(p["n"], p["colptr"], p["rowind"], p["perm"], o)
    assert rc == 0
    assert P.chol_factor(h, to_dev(p["values"])) == 0
    z = torch.empty(len(p["rowind"]), dtype=torch.float64, device="cuda")
    assert P.chol_selected_inverse(h, z) == 0
    torch.cuda.synchronize()
    P.chol_destroy(h)
    return z.cpu().numpy()


@pytest.mark.parametrize("case,merge,small", [
    ("rand", 0.0, (64, 4096, 128)), ("2d64", 0.0, (64, 4096, 128)), ("2d64", 0.1, (2, 8, 8)),
    ("3d12", 0.05, (64, 4096, 128)), ("3d12", 0.5, (4, 64, 16)), ("dense", 0.0, (1, 1, 1))])
def test_selected_inverse_vs_oracle(case, merge, small):
    P = chol()
    if case == "rand":
        A, cp, ri, vx, perm = random_spd(300, 0.02, 5)
        p = dict(n=300, colptr=cp, rowind=ri, values=vx, perm=perm)
    elif case == "dense":
        rs = np.random.RandomState(2)
        M = rs.uniform(-1, 1, (230, 230))
        from helpers import lower_csc_from_dense
        cp, ri, vx = lower_csc_from_dense(M @ M.T + 230 * np.eye(230))
        p = dict(n=230, colptr=cp, rowind=ri, values=vx, perm=np.arange(230, dtype=np.int32))
    elif case == "2d64":
        p = gridgen.workload("2d64")
    else:
        p = gridgen.laplacian_neumann_varcoef((12, 12, 12), 1e-2, 1e2, 1e-2, seed=6)
    z = _selinv(p, _opts(P, merge, small))
    ref = oracle.reference(p)
    zr = oracle.inverse_on_pattern(p, ref["fac"], p["perm"])
    assert np.max(np.abs(z - zr)) <= 1e-10 * np.max(np.abs(zr)), np.max(np.abs(z - zr)) / np.max(np.abs(zr))


def test_adjoint_matches_oracle_gradient_16rhs():
    import torch
    P = chol()
    p = gridgen.laplacian_neumann_varcoef((11, 10, 12), 1e-2, 1e2, 1e-3, seed=5)
    b = gridgen.rhs_uniform(p["n"], 16, seed=5)
    w = gridgen.rhs_normal(p["n"], 16, seed=6)
    rc, h = P.chol_analyze(p["n"], p["colptr"], p["rowind"], p["perm"], _opts(P, 0.1))
    assert P.chol_factor(h, to_dev(p["values"])) == 0
    X = colmajor(b)
    assert P.chol_solve(h, X, 16) == 0
    W = colmajor(w)
    bbar = torch.empty_like(X)
    g = torch.empty(len(p["rowind"]), dtype=torch.float64, device="cuda")
    assert P.chol_adjoint(h, W, X, 16, 1.0, bbar, g) == 0
    torch.cuda.synchronize()
    P.chol_destroy(h)
    ref = oracle.reference(p)
    gr, xbr = oracle.gradient(p, ref["fac"], w, X.cpu().numpy(), 1.0)
    gg = g.cpu().numpy()
    assert np.max(np.abs(gg - gr)) <= 1e-9 * np.max(np.abs(gr))
    assert np.max(np.abs(bbar.cpu().numpy() - xbr)) <= 1e-10 * np.max(np.abs(xbr))


def _fd_check(p, merge=0.1, npick=64):
    """Autograd gradient of sum w^T x + log det A (16 RHS) against central
    differences at npick random stored entries (a_ij and a_ji moved together).

    The difference quotient is the fourth-order central stencil
    (8 (f(+h) - f(-h)) - (f(+2h) - f(-2h))) / 12h with h = 1e-3 |a_ij|; its
    rounding floor is about eps |f| / h, far below the gradient scale. The
    criterion is |g - fd| <= 1e-6 max(|fd|, G), G = the largest |fd| among
    the picks (relative 1e-6 on the scale of the gradient). dl/db is checked
    against A^{-1} w."""
    import torch
    P = chol()
    from paper_2409_14009_gb300.autograd import solve_logdet
    S = P.SparseCholesky(p["n"], p["colptr"], p["rowind"], p["perm"], _opts(P, merge))
    vals = to_dev(p["values"]).requires_grad_(True)
    b = to_dev(gridgen.rhs_uniform(p["n"], 16, seed=2)).requires_grad_(True)
    w = to_dev(gridgen.rhs_normal(p["n"], 16, seed=3))
    x, ld = solve_logdet(vals, b, S)
    loss = (w * x).sum() + ld
    gv, gb = torch.autograd.grad(loss, (vals, b))
    gv = gv.cpu().numpy()
    xb = S.solve(w).cpu().numpy()
    assert np.allclose(gb.cpu().numpy(), xb, rtol=1e-12, atol=1e-12 * np.abs(xb).max())

    base = p["values"]
    B = colmajor(gridgen.rhs_uniform(p["n"], 16, seed=2))
    wn = gridgen.rhs_normal(p["n"], 16, seed=3)

    def f(v):
        S.factor(to_dev(v))
        X = S.solve(B)
        return float(np.sum(wn * X.cpu().numpy())) + S.logdet()

    rs = np.random.RandomState(0)
    picks = rs.choice(len(base), npick, replace=False)
    fds = []
    for t in picks:
        hstep = 1e-3 * abs(base[t])
        fv = {}
        for k in (-2, -1, 1, 2):
            v = base.copy(); v[t] += k * hstep
            fv[k] = f(v)
        fds.append((8 * (fv[1] - fv[-1]) - (fv[2] - fv[-2])) / (12 * hstep))
    S.close()
    fds = np.array(fds)
    G = np.max(np.abs(fds))
    err = np.abs(gv[picks] - fds)
    tol = 1e-6 * np.maximum(np.abs(fds), G)
    rel = err / np.abs(fds)
    print("max |g - fd| / max(|fd|, G) = %.2e; per-entry relative: median %.2e, max %.2e"
          % (np.max(err / np.maximum(np.abs(fds), G)), np.median(rel), np.max(rel)))
    assert np.all(err <= tol), [(int(t), fd, g) for t, fd, g, e, tt in zip(picks, fds, gv[picks], err, tol) if e > tt][:5]


def test_autograd_and_central_differences_3d16():
    _fd_check(gridgen.laplacian_dirichlet_weighted((16, 16, 16), gridgen.SplitMix64(5), 1e-2, 1e2))


def test_autograd_and_central_differences_3d48_workload():
    """The differentiable-solve workload itself: 3D 48^3 7-point, n = 110,592."""
    _fd_check(gridgen.workload("3d48"))
