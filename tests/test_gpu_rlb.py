"""The right-looking blocked update (RLB, Sec. II-B) against the oracle: the
update products are subtracted straight into the ancestors' panels (no update
workspace), so the factor must match the oracle and the RL factor to rounding
(not bit for bit: concurrent atomic adds reorder the additions)."""
import numpy as np
import pytest

import gridgen
import oracle
from gpu_util import check_parity, run, to_dev, colmajor
from helpers import lower_csc_from_dense, random_spd
from lib_fixture import chol

pytestmark = pytest.mark.gpu


def _opts(small_cols=64, small_panel=4096, nb=64, merge=0.0, small_rows=128):
    o = chol().chol_default_options()
    o.small_max_cols, o.small_max_panel, o.block_cols = small_cols, small_panel, nb
    o.merge_growth, o.small_max_rows = merge, small_rows
    o.update_mode = chol().CHOL_UPDATE_RLB
    return o


def test_rlb_2d64_default_and_no_workspace():
    p = gridgen.workload("2d64")
    got, _ = check_parity(p, gridgen.rhs_uniform(p.n, 2, seed=1), _opts())
    assert got["info"].update_doubles == 0
    assert got["stats"]["assemble"]["launches"] == 0


@pytest.mark.parametrize("forced", [(1, 1, 16), (4, 64, 8), (2, 32, 64), (8, 100, 32)])
def test_rlb_2d64_blocked(forced):
    p = gridgen.workload("2d64")
    got, _ = check_parity(p, gridgen.rhs_uniform(p.n, 3, seed=2), _opts(*forced))
    assert got["stats"]["syrk"]["launches"] > 0


@pytest.mark.parametrize("forced,merge", [(None, 0.0), ((4, 256, 32), 0.0), (None, 0.2)])
def test_rlb_3d_varcoef(forced, merge):
    p = gridgen.laplacian_neumann_varcoef((14, 13, 15), 1e-2, 1e2, 1e-6, seed=7)
    o = _opts(merge=merge) if forced is None else _opts(*forced, merge=merge)
    check_parity(p, gridgen.rhs_uniform(p.n, 4, seed=3), o, L_tol=1e-6, x_tol=1e-6)


@pytest.mark.parametrize("n,seed", [(150, 1), (300, 2)])
def test_rlb_random_spd(n, seed):
    A, cp, ri, vx, perm = random_spd(n, 0.05, seed)
    p = dict(n=n, colptr=cp, rowind=ri, values=vx, perm=perm)
    check_parity(p, np.random.RandomState(seed).normal(size=(n, 2)), _opts(2, 32, 32))


def test_rlb_elasticity_matches_rl():
    p = gridgen.elasticity_27pt(8, 1.0, 1e6, seed=3)
    o_rl = chol().chol_default_options()
    a = run(p, None, o_rl)
    r = run(p, None, _opts())
    assert a["rc"] == 0 and r["rc"] == 0
    la, lr = a["L"][2], r["L"][2]
    assert np.array_equal(a["L"][1], r["L"][1])
    colmax = np.maximum.reduceat(np.abs(la), a["L"][0][:-1])
    colerr = np.maximum.reduceat(np.abs(la - lr), a["L"][0][:-1])
    assert np.all(colerr <= 1e-11 * colmax)


def test_rlb_selected_inverse_matches_rl():
    # the adjoint gathers Z_RR into a workspace of its own on an RLB handle
    import torch
    P = chol()
    p = gridgen.laplacian_neumann_varcoef((10, 11, 9), 1e-2, 1e2, 1e-3, seed=4)
    zs = []
    for o in (chol().chol_default_options(), _opts()):
        rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"], o)
        assert rc == 0
        try:
            st = torch.cuda.current_stream()
            assert P.chol_factor(h, to_dev(p["values"]), st) == 0
            z = torch.zeros(len(p["rowind"]), dtype=torch.float64, device="cuda")
            assert P.chol_selected_inverse(h, z, st) == 0
            torch.cuda.synchronize()
            zs.append(z.cpu().numpy())
        finally:
            P.chol_destroy(h)
    assert np.max(np.abs(zs[0] - zs[1])) <= 1e-10 * np.max(np.abs(zs[0]))


def test_rlb_batch_with_large_small_panels_and_graph():
    # one-CTA supernodes with panels above the default 48 KB of shared memory,
    # direct launches and graph replay
    import torch
    P = chol()
    probs = gridgen.batch_2d(count=30, kmin=20, kmax=60, seed=11)
    bd = gridgen.block_diagonal(probs)
    offs = bd["meta"]["offsets"].astype(np.int32)
    b = gridgen.rhs_uniform(bd.n, 1, seed=2)
    ref = oracle.reference(bd, b)
    for graph in (0, 1):
        o = _opts(160, 24576, 64, small_rows=512)
        o.use_graph = graph
        rc, h = P.chol_analyze_batch(len(offs) - 1, offs, bd["colptr"], bd["rowind"], bd["perm"], o)
        assert rc == 0
        try:
            st = torch.cuda.current_stream()
            vals = to_dev(bd["values"])
            for _ in range(2):   # capture, then replay
                assert P.chol_factor(h, vals, st) == 0
            X = colmajor(b)
            assert P.chol_solve(h, X, 1, st) == 0
            torch.cuda.synchronize()
            x = X.cpu().numpy()
            assert np.max(np.abs(x - ref["x"])) <= 1e-10 * np.max(np.abs(ref["x"]))
        finally:
            P.chol_destroy(h)


def test_rlb_autotune_never_picks_the_persistent_kernel():
    # the persistent kernel reads the update workspace, which RLB does not have
    import torch
    P = chol()
    probs = gridgen.batch_2d(count=60, kmin=8, kmax=40, seed=5)
    bd = gridgen.block_diagonal(probs)
    offs = bd["meta"]["offsets"].astype(np.int32)
    o = _opts()
    o.update_mode = P.CHOL_UPDATE_RLB
    rc, h = P.chol_analyze_batch(len(offs) - 1, offs, bd["colptr"], bd["rowind"], bd["perm"], o)
    assert rc == 0
    try:
        vals = to_dev(bd["values"])
        assert P.chol_autotune(h, vals) == 0
        assert P.chol_get_info(h).launch_mode & 1 == 0
        b = gridgen.rhs_uniform(bd.n, 1, seed=4)
        X = colmajor(b)
        assert P.chol_factor(h, vals) == 0
        assert P.chol_solve(h, X, 1) == 0
        torch.cuda.synchronize()
        eta = oracle.backward_error(bd.n, bd["colptr"], bd["rowind"], bd["values"], b, X.cpu().numpy())
        assert eta[0] <= 1e-14
    finally:
        P.chol_destroy(h)
