"""GPU parity: the CUDA path (through the C ABI) against the FP64 oracle.

Integer/indexing results are compared bit-exact (the factor's pattern); FP64
values within 1e-12 (factor residual, solve backward error, per-column factor
entries, logdet). The forced-blocked options route small problems through the
blocked large-supernode kernels (POTRF/TRSM/GEMM/SYRK tiles) with ragged tiles.
"""
import numpy as np
import pytest

import gridgen
import oracle
from gpu_util import check_parity, colmajor, run
from helpers import lower_csc_from_dense, random_spd
from lib_fixture import chol

pytestmark = pytest.mark.gpu


def _opts(small_cols=64, small_panel=4096, nb=64, cap=0, merge=0.0, small_rows=128):
    o = chol().chol_default_options()
    o.small_max_cols, o.small_max_panel, o.block_cols, o.device_mem_cap = small_cols, small_panel, nb, cap
    o.merge_growth, o.small_max_rows = merge, small_rows
    return o


FORCED = [(1, 1, 16), (4, 64, 8), (2, 32, 64), (8, 100, 32)]


def _prob(A, perm=None):
    cp, ri, vx = lower_csc_from_dense(A)
    n = A.shape[0]
    return dict(n=n, colptr=cp, rowind=ri, values=vx,
                perm=np.arange(n, dtype=np.int32) if perm is None else perm)


def test_2d64_default():
    p = gridgen.workload("2d64")
    b = gridgen.rhs_uniform(p.n, 1, seed=1)
    got, _ = check_parity(p, b)
    assert got["stats"]["small"]["launches"] > 0


@pytest.mark.parametrize("forced", FORCED)
def test_2d64_forced_blocked(forced):
    p = gridgen.workload("2d64")
    b = gridgen.rhs_uniform(p.n, 3, seed=1)
    got, _ = check_parity(p, b, _opts(*forced))
    assert got["stats"]["gemm"]["launches"] > 0 and got["stats"]["trsm"]["launches"] > 0


@pytest.mark.parametrize("dims,forced", [((14, 13, 15), None), ((14, 13, 15), (4, 256, 32)),
                                         ((12, 12, 12), (1, 1, 64)), ((20, 20, 20), None)])
def test_3d_varcoef(dims, forced):
    p = gridgen.laplacian_neumann_varcoef(dims, 1e-2, 1e2, 1e-6, seed=7)
    b = gridgen.rhs_uniform(p.n, 8, seed=2)
    # kappa ~ 1e8 here: entries of L agree to ~kappa*u; the residual and the
    # backward error carry the 1e-12 criterion
    check_parity(p, b, None if forced is None else _opts(*forced), L_tol=1e-6, x_tol=1e-6)


def test_elasticity_small():
    p = gridgen.elasticity_27pt(6, seed=3)
    b = gridgen.rhs_uniform(p.n, 2, seed=3)
    check_parity(p, b, L_tol=1e-8, x_tol=1e-6)


def test_batch_block_diagonal():
    p = gridgen.block_diagonal(gridgen.batch_2d(count=40, kmin=4, kmax=24, seed=4))
    b = gridgen.rhs_uniform(p.n, 1, seed=4)
    check_parity(p, b, L_tol=1e-11, x_tol=1e-10)


@pytest.mark.parametrize("n,seed", [(1, 0), (2, 1), (37, 2), (150, 3), (257, 4)])
def test_random_spd(n, seed):
    A, cp, ri, vx, perm = random_spd(n, 0.08, 600 + seed)
    p = dict(n=n, colptr=cp, rowind=ri, values=vx, perm=perm)
    b = np.random.RandomState(seed).uniform(-1, 1, (n, 17))     # crosses the 16-column chunk
    check_parity(p, b)
    check_parity(p, b, _opts(2, 8, 8))


def test_dense_block_ragged():
    """A dense 200 x 200 SPD matrix: one supernode, many ragged blocked steps."""
    rs = np.random.RandomState(5)
    M = rs.uniform(-1, 1, (200, 200))
    A = M @ M.T + 200 * np.eye(200)
    p = _prob(A)
    for f in [(1, 1, 64), (1, 1, 24), (1, 1, 8)]:
        check_parity(p, rs.uniform(-1, 1, (200, 5)), _opts(*f))


def test_not_positive_definite_reports_column():
    p = gridgen.workload("2d64")
    vals = p["values"].copy()
    # make one diagonal entry negative (original index 777)
    diag_pos = p["colptr"][777]
    vals[diag_pos] = -1.0
    q = dict(p, values=vals)
    bp, bi, bx = oracle.permute(q["n"], q["colptr"], q["rowind"], q["values"], q["perm"])
    info = oracle.Factor(q["n"], bp, bi, bx).info
    assert info > 0
    assert run(q)["rc"] == info
    assert run(q, options=_opts(1, 1, 16))["rc"] == info


def test_deterministic_bitwise():
    p = gridgen.laplacian_neumann_varcoef((12, 11, 10), 1e-2, 1e2, 1e-6, seed=3)
    b = gridgen.rhs_uniform(p.n, 4, seed=3)
    a = run(p, b, _opts(4, 128, 32))
    c = run(p, b, _opts(4, 128, 32))
    assert np.array_equal(a["L"][2], c["L"][2]) and np.array_equal(a["x"], c["x"])
    assert a["logdet"] == c["logdet"]


def test_enomem_cap_and_state_errors():
    import torch
    P = chol()
    p = gridgen.workload("2d64")
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"], _opts(cap=4096))
    assert rc == 0
    vals = torch.as_tensor(p["values"], device="cuda")
    assert P.chol_factor(h, vals) == P.CHOL_ENOMEM
    b = torch.zeros(p.n, dtype=torch.float64, device="cuda")
    assert P.chol_solve(h, b, 1) == P.CHOL_ESTATE
    P.chol_destroy(h)
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"])
    assert P.chol_factor(h, vals) == 0
    assert P.chol_solve(h, b, 0) == 0
    assert P.chol_solve(h, b, -1) == -3
    P.chol_destroy(h)


def test_refactor_with_new_values():
    """Analyze once, factor twice with different values (handle reuse)."""
    p = gridgen.laplacian_neumann_varcoef((9, 9, 9), 1e-2, 1e2, 1e-6, seed=11)
    q = dict(p, values=p["values"] * 2.0)
    import torch
    P = chol()
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"])
    for prob in (p, q):
        assert P.chol_factor(h, torch.as_tensor(prob["values"], device="cuda")) == 0
        ref = oracle.reference(prob)
        rc, ld = P.chol_logdet(h)
        assert abs(ld - ref["fac"].logdet()) <= 1e-12 * abs(ld)
    P.chol_destroy(h)


@pytest.mark.parametrize("merge", [0.01, 0.05, 0.25, 1.0])
def test_relaxed_merging_parity(merge):
    """Merged storage partitions (explicit zeros) give the same factor on the
    canonical pattern and the same solution."""
    p = gridgen.laplacian_neumann_varcoef((16, 15, 14), 1e-2, 1e2, 1e-6, seed=8)
    b = gridgen.rhs_uniform(p.n, 8, seed=8)
    got, _ = check_parity(p, b, _opts(merge=merge), L_tol=1e-6, x_tol=1e-6)
    assert got["info"].nsuper_storage < got["info"].nsuper
    check_parity(gridgen.workload("2d64"), gridgen.rhs_uniform(4096, 2, seed=1), _opts(merge=merge, nb=32))


@pytest.mark.parametrize("nrhs", [5, 11, 17])
def test_solve_rhs_counts_and_chunks(nrhs):
    # 5 and 11: partial right-hand-side groups inside one chunk; 17: two chunks
    # (16 + 1). Forced blocked kernels give diagonal triangles of several 64-row
    # blocks, so the flag-ordered triangle solve runs with many blocks per level.
    p = gridgen.laplacian_neumann_varcoef((16, 15, 14), 1e-2, 1e2, 1e-3, seed=9)
    b = gridgen.rhs_normal(p.n, nrhs, seed=nrhs)
    check_parity(p, b, _opts(2, 64, 64, merge=0.2), L_tol=1e-8, x_tol=1e-8)


def test_solve_replays_from_a_cuda_graph():
    # the triangle launches keep their flag epoch on the device, so a captured
    # solve replays correctly with new right-hand sides
    import torch
    from gpu_util import colmajor, to_dev
    P = chol()
    p = gridgen.laplacian_neumann_varcoef((14, 14, 14), 1e-2, 1e2, 1e-3, seed=10)
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"], _opts(2, 64, 64))
    assert rc == 0
    try:
        st = torch.cuda.Stream()
        with torch.cuda.stream(st):
            vals = to_dev(p["values"])
            assert P.chol_factor(h, vals, st) == 0
            X = colmajor(gridgen.rhs_uniform(p.n, 2, seed=1))
            assert P.chol_solve(h, X, 2, st) == 0       # workspaces exist before capture
        st.synchronize()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g, stream=st):
            assert P.chol_solve(h, X, 2, st) == 0
        for seed in (2, 3, 4):
            b = gridgen.rhs_uniform(p.n, 2, seed=seed)
            X.copy_(colmajor(b))
            g.replay()
            torch.cuda.synchronize()
            x = X.cpu().numpy()
            ref = oracle.reference(p, b)
            assert np.max(np.abs(x - ref["x"])) <= 1e-8 * np.max(np.abs(ref["x"]))
    finally:
        P.chol_destroy(h)


def test_factor_solve_from_host_buffers_matches_device_path():
    """chol_factor_solve_host (values and right-hand sides in host memory,
    pinned or pageable) gives the device path's x and log det, and the oracle's."""
    import torch
    P = chol()
    # Dirichlet-anchored (well conditioned), so x itself is compared tightly
    p = gridgen.laplacian_dirichlet_weighted((13, 12, 11), gridgen.SplitMix64(9), 1e-2, 1e2)
    b = gridgen.rhs_uniform(p.n, 3, seed=10)
    ref = oracle.reference(p, b)
    rc, h = P.chol_analyze(p.n, p["colptr"], p["rowind"], p["perm"])
    assert rc == 0
    try:
        for pinned in (False, True):
            vals = torch.as_tensor(p["values"])
            bh = torch.as_tensor(np.ascontiguousarray(b.T))          # column-major n x 3
            xh = torch.zeros_like(bh)
            if pinned:
                vals, bh, xh = vals.pin_memory(), bh.pin_memory(), xh.pin_memory()
            rc, ld = P.chol_factor_solve_host(h, vals, bh, xh, 3)
            assert rc == 0
            x = xh.numpy().T
            eta = oracle.backward_error(p.n, p["colptr"], p["rowind"], p["values"], b, x)
            assert np.all(eta <= 1e-12), eta
            assert np.max(np.abs(x - ref["x"])) <= 1e-12 * np.max(np.abs(ref["x"]))
            assert abs(ld - ref["fac"].logdet()) <= 1e-12 * abs(ref["fac"].logdet())
        xd = colmajor(b)
        assert P.chol_solve(h, xd, 3) == 0
        torch.cuda.synchronize()
        assert np.array_equal(xd.cpu().numpy(), x)
        # x may alias b
        bh2 = torch.as_tensor(np.ascontiguousarray(b.T)).pin_memory()
        rc, _ = P.chol_factor_solve_host(h, torch.as_tensor(p["values"]), bh2, bh2, 3, want_logdet=False)
        assert rc == 0 and np.array_equal(bh2.numpy().T, x)
    finally:
        P.chol_destroy(h)
