"""The nested dissection ordering (chol_order_nd), the irregular generator and
the Matrix Market reader, on the host: valid permutations on degenerate and
disconnected graphs, fill well below the natural ordering and close to the
geometric nested dissection on grids (which needs the coordinates the
ordering never sees), determinism, and lossless file round trips."""
import os

import numpy as np
import pytest

import gridgen
from helpers import lower_csc_from_dense
from lib_fixture import chol
from paper_2409_14009_gb300 import mmio


def _nnz_l(n, cp, ri, perm):
    P = chol()
    rc, h = P.chol_analyze(n, cp, ri, perm, None)
    assert rc == 0
    try:
        return P.chol_get_info(h).nnz_l
    finally:
        P.chol_destroy(h)


def _order(n, cp, ri):
    rc, perm = chol().chol_order_nd(n, cp, ri)
    assert rc == 0
    assert np.array_equal(np.sort(perm), np.arange(n))
    return perm


def _dense_pattern(A):
    cp, ri, _ = lower_csc_from_dense(A)
    return A.shape[0], cp, ri


def test_degenerate_graphs():
    assert chol().chol_order_nd(0, np.zeros(1, np.int64), np.zeros(0, np.int32))[0] == 0
    for A in (np.eye(1), np.eye(50),                                    # no edges
              np.ones((120, 120)),                                      # a clique
              np.eye(300) + np.eye(300, k=1) + np.eye(300, k=-1)):      # a path
        _order(*_dense_pattern(A))
    star = np.eye(200)
    star[0, :] = star[:, 0] = 1.0
    _order(*_dense_pattern(star))


def test_deterministic():
    q = gridgen.irregular_3d(9, seed=5)
    assert np.array_equal(_order(q.n, q["colptr"], q["rowind"]), _order(q.n, q["colptr"], q["rowind"]))


def test_deterministic_with_threads():
    # large enough for the two sides of the top splits to run on their own threads
    q = gridgen.irregular_3d(30, seed=2)
    first = _order(q.n, q["colptr"], q["rowind"])
    for _ in range(4):
        assert np.array_equal(first, _order(q.n, q["colptr"], q["rowind"]))


def test_rejects_bad_input():
    P = chol()
    cp = np.array([0, 2, 3], np.int64)
    assert P.chol_order_nd(-1, cp, np.zeros(3, np.int32))[0] == -1
    assert P.chol_order_nd(2, cp, np.array([0, 5, 1], np.int32))[0] == -3   # row out of range
    assert P.chol_order_nd(2, cp, np.array([0, 1, 0], np.int32))[0] == -3   # above the diagonal


def test_disconnected_components():
    probs = [gridgen.laplacian_2d_dirichlet(k) for k in (5, 11, 2, 17)]
    p = gridgen.block_diagonal(probs)
    perm = _order(p.n, p["colptr"], p["rowind"])
    assert _nnz_l(p.n, p["colptr"], p["rowind"], perm) <= 1.3 * _nnz_l(p.n, p["colptr"], p["rowind"], p["perm"])


@pytest.mark.parametrize("k", [40, 64])
def test_fill_on_2d_grid(k):
    p = gridgen.laplacian_2d_dirichlet(k)
    perm = _order(p.n, p["colptr"], p["rowind"])
    nd = _nnz_l(p.n, p["colptr"], p["rowind"], perm)
    natural = _nnz_l(p.n, p["colptr"], p["rowind"], np.arange(p.n, dtype=np.int32))
    geometric = _nnz_l(p.n, p["colptr"], p["rowind"], p["perm"])
    assert nd < 0.6 * natural
    assert nd <= 1.5 * geometric


def test_fill_on_3d_grid_and_irregular_pattern():
    p = gridgen.laplacian_neumann_varcoef((12, 12, 12), 1e-2, 1e2, 1e-3, seed=1)
    perm = _order(p.n, p["colptr"], p["rowind"])
    assert _nnz_l(p.n, p["colptr"], p["rowind"], perm) <= 1.6 * _nnz_l(p.n, p["colptr"], p["rowind"], p["perm"])
    # the irregular pattern (identity order as generated): well below the
    # natural fill, and no worse than the geometric dissection of its grid
    q = gridgen.irregular_3d(14)
    perm = _order(q.n, q["colptr"], q["rowind"])
    nd = _nnz_l(q.n, q["colptr"], q["rowind"], perm)
    assert nd < 0.5 * _nnz_l(q.n, q["colptr"], q["rowind"], q["perm"])
    assert nd <= 1.1 * _nnz_l(q.n, q["colptr"], q["rowind"], gridgen.nd_perm((14, 14, 14)).astype(np.int32))


def test_irregular_generator_is_spd_and_irregular():
    q = gridgen.irregular_3d(6, keep=0.35, seed=3)
    from helpers import dense_from_lower
    A = dense_from_lower(q.n, q["colptr"], q["rowind"], q["values"])
    assert np.allclose(A, A.T)
    assert np.linalg.eigvalsh(A).min() > 0
    deg = (np.abs(A) > 0).sum(axis=1) - 1
    assert deg.min() < deg.max()        # irregular degrees
    q2 = gridgen.irregular_3d(6, keep=0.35, seed=3)
    assert np.array_equal(q["values"], q2["values"])   # deterministic


def test_matrix_market_round_trip(tmp_path):
    p = gridgen.irregular_3d(5)
    f = os.path.join(tmp_path, "a.mtx")
    mmio.write_symmetric(f, p.n, p["colptr"], p["rowind"], p["values"])
    n, cp, ri, v = mmio.read_symmetric(f)
    assert n == p.n and np.array_equal(cp, p["colptr"]) and np.array_equal(ri, p["rowind"])
    assert np.array_equal(v, p["values"])
    # the same matrix given by its upper triangle, with a missing diagonal
    g = os.path.join(tmp_path, "b.mtx")
    with open(g, "w") as fh:
        fh.write("%%MatrixMarket matrix coordinate real symmetric\n% comment\n3 3 3\n")
        fh.write("1 1 4.0\n1 3 -1.0\n3 3 5.0\n")
    n, cp, ri, v = mmio.read_symmetric(g)
    assert n == 3 and list(cp) == [0, 2, 3, 4] and list(ri) == [0, 2, 1, 2]
    assert list(v) == [4.0, -1.0, 0.0, 5.0]
    h = os.path.join(tmp_path, "p.txt")
    np.savetxt(h, [3, 1, 2], fmt="%d")
    assert list(mmio.read_perm(h)) == [2, 0, 1]
    # general storage of a symmetric matrix: both triangles, the lower one kept
    with open(os.path.join(tmp_path, "g.mtx"), "w") as fh:
        fh.write("%%MatrixMarket matrix coordinate real general\n3 3 5\n")
        fh.write("1 1 4.0\n3 1 -1.0\n1 3 -1.0\n2 2 2.0\n3 3 5.0\n")
    n, cp, ri, v = mmio.read_symmetric(os.path.join(tmp_path, "g.mtx"))
    assert n == 3 and list(cp) == [0, 2, 3, 4] and list(ri) == [0, 2, 1, 2] and list(v) == [4.0, -1.0, 2.0, 5.0]
    for body in ("3 3 2\n1 1 1.0\n2 1 1.0\n", "3 3 3\n1 1 1.0\n2 1 1.0\n1 2 2.0\n"):
        with open(os.path.join(tmp_path, "c.mtx"), "w") as fh:   # not symmetric: pattern, then values
            fh.write("%%MatrixMarket matrix coordinate real general\n" + body)
        with pytest.raises(ValueError):
            mmio.read_symmetric(os.path.join(tmp_path, "c.mtx"))
    with open(os.path.join(tmp_path, "h.mtx"), "w") as fh:
        fh.write("%%MatrixMarket matrix coordinate real hermitian\n2 2 1\n1 1 1.0\n")
    with pytest.raises(ValueError):
        mmio.read_symmetric(os.path.join(tmp_path, "h.mtx"))
