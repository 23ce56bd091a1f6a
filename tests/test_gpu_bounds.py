"""The bounds-checked build (-DCHOL_BOUNDS_CHECK): with an intact plan it gives
the normal build's factor bit for bit; with a plan damaged on the host before
the first factorization (a relind segment or task pointing outside its
supernodes, a value scatter position past the panels) the checks skip the
access and chol_factor returns CHOL_EBOUNDS with the failed check's code --
nothing faults, and the next handle factors normally."""
import ctypes as C

import numpy as np
import pytest

import gridgen
from gpu_util import to_dev
from lib_fixture import chol

pytestmark = pytest.mark.gpu

EXPECT = {1: 3, 2: 4, 3: 2, 4: 7, 5: 3}   # corruption kind -> bounds code (chol.h)


def _libs():
    P = chol()
    from paper_2409_14009_gb300 import build
    build.build(checked=True)
    return P, P.lib_checked()


def _analyze(P, L, p, precision=0):
    o = P.chol_default_options()
    o.precision = precision
    cp = np.ascontiguousarray(p["colptr"], np.int64)
    ri = np.ascontiguousarray(p["rowind"], np.int32)
    pm = np.ascontiguousarray(p["perm"], np.int32)
    h = C.c_void_p()
    rc = L.chol_analyze(int(p.n), cp.ctypes.data_as(C.c_void_p), ri.ctypes.data_as(C.c_void_p),
                        pm.ctypes.data_as(C.c_void_p), C.byref(o), C.byref(h))
    assert rc == 0
    return h


def _factor_l(P, L, h, vals):
    import torch
    rc = L.chol_factor(h, C.c_void_p(vals.data_ptr()), None)
    torch.cuda.synchronize()
    return rc


def _get_factor(P, L, h):
    info = P.chol_info()
    assert L.chol_get_info(h, C.byref(info)) == 0
    lx = np.zeros(max(info.nnz_l, 1))
    lp = np.zeros(info.n + 1, np.int64)
    li = np.zeros(max(info.nnz_l, 1), np.int32)
    assert L.chol_get_factor(h, lp.ctypes.data_as(C.c_void_p), li.ctypes.data_as(C.c_void_p),
                             lx.ctypes.data_as(C.c_void_p), None) == 0
    return lx[: info.nnz_l], info


@pytest.mark.parametrize("precision", [0, 3])
def test_checked_build_gives_the_normal_factor(precision):
    P, Lc = _libs()
    Ln = P.lib()
    # Dirichlet-anchored: positive definite in bf16 too (the shifted Neumann grid needs static pivoting)
    p = gridgen.laplacian_dirichlet_weighted((20, 19, 18), gridgen.SplitMix64(3), 1e-2, 1e2)
    vals = to_dev(p["values"])
    out = []
    for L in (Ln, Lc):
        h = _analyze(P, L, p, precision)
        try:
            assert _factor_l(P, L, h, vals) == 0
            lx, info = _get_factor(P, L, h)
            assert info.bounds_code == 0
            out.append(lx)
        finally:
            L.chol_destroy(h)
    assert np.array_equal(out[0], out[1])


@pytest.mark.parametrize("kind", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("precision", [0, 1])
def test_damaged_plan_is_caught_without_a_fault(kind, precision):
    P, Lc = _libs()
    # 3-dof elasticity: its levels have both CTA-sized and warp-sized assembly
    # tasks (on the 7-point grids every task is warp-sized)
    p = gridgen.elasticity_27pt(12, seed=3)
    vals = to_dev(p["values"])
    h = _analyze(P, Lc, p, precision)
    try:
        rc = Lc.chol_test_corrupt_plan(h, kind)
        assert rc == 0, rc
        assert _factor_l(P, Lc, h, vals) == P.CHOL_EBOUNDS
        info = P.chol_info()
        assert Lc.chol_get_info(h, C.byref(info)) == 0
        assert info.bounds_code == EXPECT[kind], info.bounds_code
        # the handle was not factored
        assert Lc.chol_logdet(h, C.byref(C.c_double()), None) == P.CHOL_ESTATE
    finally:
        Lc.chol_destroy(h)
    # the context is intact: a fresh handle factors normally
    h = _analyze(P, Lc, p, precision)
    try:
        assert _factor_l(P, Lc, h, vals) == 0
    finally:
        Lc.chol_destroy(h)


def test_corruption_entry_refuses_in_the_normal_build():
    P = chol()
    p = gridgen.laplacian_2d_dirichlet(12)
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"])
    assert rc == 0
    try:
        assert P.chol_test_corrupt_plan(h, 1) == P.CHOL_ENOTSUP
    finally:
        P.chol_destroy(h)
