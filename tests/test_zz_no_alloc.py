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
import oracle
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


def test_noalloc_first_solve_on_fresh_handle_single_rhs_vs_oracle():
    """The first solve of a new handle (the handle's own solve workspaces were
    never created) with one right-hand side, checked against the oracle's
    solution and by its backward error; then chol_solve gives the same x."""
    import torch
    P = chol()
    # Dirichlet-anchored (well conditioned), so x itself is compared tightly
    p = gridgen.laplacian_dirichlet_weighted((14, 13, 12), gridgen.SplitMix64(7), 1e-2, 1e2)
    b = gridgen.rhs_uniform(p.n, 1, seed=8)
    ref = oracle.reference(p, b)
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"])
    assert rc == 0
    try:
        assert P.chol_factor(h, to_dev(p["values"])) == 0
        got = colmajor(b[:, 0])
        assert P.chol_solve_noalloc(h, got, 1) == 0
        assert P.chol_check_waits(h) == 0
        x = got.cpu().numpy().reshape(-1, 1)
        eta = oracle.backward_error(p.n, p["colptr"], p["rowind"], p["values"], b, x)
        assert np.all(eta <= 1e-12), eta
        xr = ref["x"].reshape(-1, 1)
        assert np.max(np.abs(x - xr)) <= 1e-12 * np.max(np.abs(xr))
        again = colmajor(b[:, 0])
        assert P.chol_solve(h, again, 1) == 0
        torch.cuda.synchronize()
        assert np.array_equal(again.cpu().numpy().reshape(-1, 1), x)
    finally:
        P.chol_destroy(h)


@pytest.mark.parametrize("prec", ["fp32", "bf16"])
def test_noalloc_refuses_mixed_precision_handle(prec):
    P = chol()
    p = gridgen.laplacian_2d_dirichlet(24)
    o = P.chol_default_options()
    o.precision = P.CHOL_PREC_FP32 if prec == "fp32" else P.CHOL_PREC_BF16
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"], o)
    assert rc == 0
    try:
        assert P.chol_factor(h, to_dev(p["values"])) == 0
        x = colmajor(gridgen.rhs_uniform(p.n, 1, seed=1)[:, 0])
        assert P.chol_solve_noalloc(h, x, 1) == P.CHOL_ENOTSUP
    finally:
        P.chol_destroy(h)
