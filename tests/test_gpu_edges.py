"""GPU parity on degenerate and boundary inputs: the empty system, a 1 x 1
matrix, a diagonal matrix (every column its own root), a tridiagonal chain
(a supernodal tree as deep as the matrix), an arrowhead (every column updates
the last one), dense matrices at the 64- and 128-wide tile edges, a forest of
unequal components, and the mixed-precision path on the deep chain."""
import numpy as np
import pytest

import gridgen
from gpu_util import check_parity, colmajor, to_dev
from helpers import lower_csc_from_dense
from lib_fixture import chol

pytestmark = pytest.mark.gpu


def _prob(A, perm=None):
    cp, ri, vx = lower_csc_from_dense(A)
    n = A.shape[0]
    return dict(n=n, colptr=cp, rowind=ri, values=vx,
                perm=np.arange(n, dtype=np.int32) if perm is None else np.asarray(perm, np.int32))


def _opts(**kw):
    o = chol().chol_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


def test_empty_system():
    import torch
    P = chol()
    rc, h = P.chol_analyze(0, np.zeros(1, np.int64), np.zeros(0, np.int32), None, None)
    assert rc == 0
    try:
        st = torch.cuda.current_stream()
        assert P.chol_factor(h, torch.zeros(0, dtype=torch.float64, device="cuda"), st) == 0
        x = torch.zeros((0, 3), dtype=torch.float64, device="cuda")
        assert P.chol_solve(h, x, 3, st) == 0
        rc, ld = P.chol_logdet(h, st)
        assert rc == 0 and ld == 0.0
    finally:
        P.chol_destroy(h)


def test_one_by_one():
    p = _prob(np.array([[4.0]]))
    got, _ = check_parity(p, np.array([[2.0, -6.0]]))
    assert np.allclose(got["x"], [[0.5, -1.5]])
    assert abs(got["logdet"] - np.log(4.0)) < 1e-15


def test_diagonal_matrix_all_roots():
    rs = np.random.RandomState(1)
    A = np.diag(rs.uniform(0.5, 3.0, 500))
    got, _ = check_parity(_prob(A, rs.permutation(500)), rs.normal(size=(500, 4)))
    assert got["info"].nlevels == 1 and got["info"].nsuper == 500


@pytest.mark.parametrize("n", [300])
def test_tridiagonal_chain_deep_tree(n):
    # natural order: a path, so the supernodal tree is a chain about n deep
    A = np.diag(np.full(n, 2.5)) + np.diag(np.full(n - 1, -1.0), 1) + np.diag(np.full(n - 1, -1.0), -1)
    got, _ = check_parity(_prob(A), gridgen.rhs_normal(n, 2, seed=3))
    assert got["info"].nlevels >= n // 2


def test_arrowhead_star():
    n = 400
    rs = np.random.RandomState(2)
    A = np.diag(rs.uniform(5.0, 6.0, n))
    A[-1, :-1] = A[:-1, -1] = rs.uniform(-0.01, 0.01, n - 1)
    A[-1, -1] = 50.0
    check_parity(_prob(A), rs.normal(size=(n, 3)))


@pytest.mark.parametrize("n", [63, 64, 65, 127, 128, 129])
def test_dense_at_tile_edges(n):
    rs = np.random.RandomState(n)
    M = rs.normal(size=(n, n))
    A = M @ M.T + n * np.eye(n)
    # blocked path (small kernel off) so the 64-wide steps, the 128-row
    # tensor-core-sized tiles and their ragged ends are exercised
    check_parity(_prob(A), rs.normal(size=(n, 2)), _opts(small_max_cols=1, small_max_panel=1),
                 L_tol=1e-10, x_tol=1e-9)


def test_forest_of_unequal_components():
    probs = [gridgen.laplacian_2d_dirichlet(k) for k in (3, 17, 40, 9)]
    p = gridgen.block_diagonal(probs)
    check_parity(p, gridgen.rhs_uniform(p.n, 2, seed=5))


def test_mixed_precision_on_the_deep_chain():
    import torch
    P = chol()
    n = 257
    A = np.diag(np.full(n, 2.01)) + np.diag(np.full(n - 1, -1.0), 1) + np.diag(np.full(n - 1, -1.0), -1)
    p = _prob(A)
    rc, h = P.chol_analyze(n, p["colptr"], p["rowind"], p["perm"], _opts(precision=P.CHOL_PREC_FP32))
    assert rc == 0
    try:
        st = torch.cuda.current_stream()
        assert P.chol_factor(h, to_dev(p["values"]), st) == 0
        b = gridgen.rhs_uniform(n, 1, seed=9)
        B = colmajor(b)
        X = torch.zeros_like(B)
        rc, it, berr = P.chol_solve_refine(h, B, X, 1, 1e-12, 50)
        assert rc == 0 and berr[0] <= 1e-12
        x_ref = np.linalg.solve(A, b)
        assert np.max(np.abs(X.cpu().numpy() - x_ref)) <= 1e-9 * np.max(np.abs(x_ref))
    finally:
        P.chol_destroy(h)
