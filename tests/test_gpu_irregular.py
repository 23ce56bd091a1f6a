"""GPU parity on irregular patterns: the random-edge 27-point matrix and a
forest of unequal irregular blocks, ordered by chol_order_nd (no coordinates),
in the RL and RLB update modes; the mixed-precision refinement on the same
pattern; and a Matrix Market file taken through the user-matrix command."""
import os

import numpy as np
import pytest

import gridgen
from gpu_util import check_parity
from lib_fixture import chol

pytestmark = pytest.mark.gpu


def _ordered(p):
    P = chol()
    rc, perm = P.chol_order_nd(p.n, p["colptr"], p["rowind"])
    assert rc == 0
    q = dict(n=p.n, colptr=p["colptr"], rowind=p["rowind"], values=p["values"], perm=perm)
    return q


def _opts(**kw):
    o = chol().chol_default_options()
    for k, v in kw.items():
        setattr(o, k, v)
    return o


@pytest.mark.parametrize("k,seed", [(11, 12), (14, 3)])
def test_irregular_nd_parity(k, seed):
    q = _ordered(gridgen.irregular_3d(k, seed=seed))
    got, _ = check_parity(q, gridgen.rhs_uniform(q["n"], 3, seed=k), L_tol=1e-11, x_tol=1e-10)
    assert got["info"].nsuper > 1


def test_irregular_nd_parity_rlb():
    P = chol()
    q = _ordered(gridgen.irregular_3d(13, seed=7))
    check_parity(q, gridgen.rhs_uniform(q["n"], 2, seed=2), _opts(update_mode=P.CHOL_UPDATE_RLB),
                 L_tol=1e-11, x_tol=1e-10)


def test_forest_of_irregular_blocks():
    p = gridgen.block_diagonal([gridgen.irregular_3d(k, seed=k) for k in (4, 9, 6)])
    check_parity(_ordered(p), gridgen.rhs_uniform(p.n, 2, seed=6), L_tol=1e-11, x_tol=1e-10)


def test_matrix_market_file_through_the_command(tmp_path):
    from paper_2409_14009_gb300 import mmio, run_matrix
    p = gridgen.irregular_3d(12, seed=4)
    f = os.path.join(tmp_path, "irr.mtx")
    mmio.write_symmetric(f, p.n, p["colptr"], p["rowind"], p["values"])
    out = run_matrix.main(["--mtx", f, "--reps", "1", "--nrhs", "2"])
    assert out["n"] == p.n and out["refine_rc"] == 0 and out["backward_error"] <= 1e-14
    out = run_matrix.main(["--mtx", f, "--reps", "1", "--precision", "fp32"])
    assert out["refine_rc"] == 0 and out["backward_error"] <= 1e-10 and out["refine_iterations"] >= 1
