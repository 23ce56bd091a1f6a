"""chol_solve_noalloc: the triangular solves without any device allocation.

Some callers cannot call cudaMalloc once they are running -- a process whose
memory pool has already claimed the GPU, or a latency-bound loop where an
allocation could stall on device-wide synchronization. For them the library
offers a solve whose workspaces live in one fixed device array. These tests
check that it returns what chol_solve returns, call after call (the array keeps
the previous call's contents), and that a problem too large for the array is
refused. This file is collected last so that a failure here does not stop a
``-x`` run before the other tests.
"""
import numpy as np
import pytest

import gridgen
from gpu_util import colmajor, to_dev
from lib_fixture import chol

pytestmark = pytest.mark.gpu


def test_noalloc_solve_matches_chol_solve_on_two_calls():
    import torch
    P = chol()
    # 160,000 unknowns: one right-hand-side column needs more than 1/16 of the
    # fixed array, so 20 right-hand sides are processed in two chunks
    p = gridgen.laplacian_2d_dirichlet(400)
    o = P.chol_default_options()
    o.merge_growth = 0.05
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"], o)
    assert rc == 0
    try:
        assert P.chol_factor(h, to_dev(p["values"])) == 0
        for seed in (1, 2):                       # two calls in a row
            b = gridgen.rhs_uniform(p.n, 20, seed=seed)
            ref = colmajor(b)
            assert P.chol_solve(h, ref, 20) == 0
            got = colmajor(b)
            assert P.chol_solve_noalloc(h, got, 20) == 0
            torch.cuda.synchronize()
            ref, got = ref.cpu().numpy(), got.cpu().numpy()
            assert np.max(np.abs(got - ref)) <= 1e-12 * np.max(np.abs(ref))
    finally:
        P.chol_destroy(h)


def test_noalloc_solve_refuses_oversized_problem():
    P = chol()
    p = gridgen.laplacian_2d_dirichlet(1500)      # n = 2,250,000 > 2^21 doubles
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"])
    assert rc == 0
    try:
        dummy = to_dev(np.zeros(4))
        assert P.chol_solve_noalloc(h, dummy, 1) == P.CHOL_ETOOBIG
    finally:
        P.chol_destroy(h)
