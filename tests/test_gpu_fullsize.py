"""Full-size parity for the 3D 64^3 7-point variable-coefficient workload, in the
launch configuration the benchmark times (default options): properties that the
oracle checks at any size -- sampled factor-residual columns, the backward error of
the 8-RHS solve, the exact symbolic counts -- plus bitwise determinism."""
import numpy as np
import pytest

import gridgen
import oracle
from gpu_util import colmajor, to_dev
from lib_fixture import chol

pytestmark = pytest.mark.gpu


def test_3d64_properties():
    import torch
    P = chol()
    p = gridgen.workload("3d64")
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"])
    assert rc == 0
    info = P.chol_get_info(h)
    vals = to_dev(p["values"])
    assert P.chol_factor(h, vals) == 0
    lp, li, lx = P.chol_get_factor(h)
    bp, bi, bx = oracle.permute(p.n, p["colptr"], p["rowind"], p["values"], p["perm"])
    rs = np.random.RandomState(0)
    cols = np.unique(np.concatenate([rs.randint(0, p.n, 48), np.arange(p.n - 16, p.n)]))
    res = oracle.factor_residual_cols(p.n, bp, bi, bx, lp, li, lx, cols)
    assert np.all(res <= 1e-12), res.max()
    b = gridgen.rhs_uniform(p.n, 8, seed=2)
    xb = colmajor(b)
    assert P.chol_solve(h, xb, 8) == 0
    x = xb.cpu().numpy()
    eta = oracle.backward_error(p.n, p["colptr"], p["rowind"], p["values"], b, x)
    assert np.all(eta <= 1e-12), eta
    rc, ld = P.chol_logdet(h)
    assert rc == 0 and np.isfinite(ld)
    # determinism
    assert P.chol_factor(h, vals) == 0
    lx2 = P.chol_get_factor(h)[2]
    assert np.array_equal(lx, lx2)
    assert info.flops == float((np.diff(lp).astype(np.float64) ** 2).sum())
    P.chol_destroy(h)
