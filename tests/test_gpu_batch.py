"""Batches of independent small SPD systems (2D weighted Laplacians of uneven
sizes): one block-diagonal analysis, level-by-level or persistent cooperative
execution, CUDA-graph replay, the launch autotuner, per-system logdet; FP64 and
binary32 (+ refinement), against the oracle system by system."""
import numpy as np
import pytest

import gridgen
import oracle
from gpu_util import colmajor, to_dev
from lib_fixture import chol

pytestmark = pytest.mark.gpu


def _batch(count=60, kmin=4, kmax=28, seed=4):
    probs = gridgen.batch_2d(count=count, kmin=kmin, kmax=kmax, seed=seed)
    return probs, gridgen.block_diagonal(probs)


def _opts(P, precision=0, persistent=0, graph=0):
    o = P.chol_default_options()
    o.precision, o.persistent, o.use_graph = precision, persistent, graph
    o.small_max_cols, o.small_max_panel, o.small_max_rows = 128, 16384, 512
    return o


def _run(P, bd, o, b):
    import torch
    offs = bd["meta"]["offsets"].astype(np.int32)
    rc, h = P.chol_analyze_batch(len(offs) - 1, offs, bd["colptr"], bd["rowind"], bd["perm"], o)
    assert rc == 0, rc
    info = P.chol_get_info(h)
    vals = to_dev(bd["values"])
    assert P.chol_factor(h, vals) == 0
    assert P.chol_factor(h, vals) == 0           # second call: graph replay when enabled
    lx = P.chol_get_factor(h)[2]
    X = colmajor(b)
    if o.precision == 0:
        assert P.chol_solve(h, X, b.shape[1]) == 0
        rcr = 0
    else:
        B = colmajor(b)
        rcr, iters, berr = P.chol_solve_refine(h, B, X, b.shape[1], 1e-10, 50)
    torch.cuda.synchronize()
    rc, lds = P.chol_logdet_batch(h, len(offs) - 1)
    assert rc == 0
    stats = P.chol_get_stats(h)
    P.chol_destroy(h)
    return dict(info=info, lx=lx, x=X.cpu().numpy(), logdet=lds, rc_refine=rcr, stats=stats)


@pytest.mark.parametrize("persistent,graph", [(0, 0), (1, 0), (0, 1), (1, 1)])
def test_batch_fp64_per_system(persistent, graph):
    P = chol()
    probs, bd = _batch()
    b = gridgen.rhs_uniform(bd.n, 1, seed=7)
    got = _run(P, bd, _opts(P, 0, persistent, graph), b)
    assert got["info"].nsys == len(probs) and got["info"].persistent_ok == 1
    offs = bd["meta"]["offsets"]
    for q, p in enumerate(probs):
        bq = b[offs[q]:offs[q + 1]]
        ref = oracle.reference(p, bq)
        xq = got["x"][offs[q]:offs[q + 1]]
        assert np.max(np.abs(xq - ref["x"])) <= 1e-11 * np.max(np.abs(ref["x"]))
        assert abs(got["logdet"][q] - ref["fac"].logdet()) <= 1e-12 * abs(ref["fac"].logdet())
    if persistent:
        assert got["stats"]["small"]["launches"] == 2        # one persistent launch per factorization
        assert got["stats"]["assemble"]["launches"] == 0


def test_batch_persistent_is_bitwise_identical():
    P = chol()
    probs, bd = _batch(count=40)
    b = gridgen.rhs_uniform(bd.n, 1, seed=8)
    a = _run(P, bd, _opts(P, 0, 0, 0), b)
    c = _run(P, bd, _opts(P, 0, 1, 1), b)
    assert np.array_equal(a["lx"], c["lx"]) and np.array_equal(a["x"], c["x"])


@pytest.mark.parametrize("persistent", [0, 1])
def test_batch_fp32_refined(persistent):
    P = chol()
    probs, bd = _batch(count=50, kmin=6, kmax=40, seed=9)
    b = gridgen.rhs_uniform(bd.n, 1, seed=9)
    got = _run(P, bd, _opts(P, 1, persistent, 1), b)
    assert got["rc_refine"] == 0
    eta = oracle.backward_error(bd.n, bd["colptr"], bd["rowind"], bd["values"], b, got["x"])
    assert eta[0] <= 1e-10
    offs = bd["meta"]["offsets"]
    for q, p in enumerate(probs[:10]):
        ref = oracle.reference(p)
        assert abs(got["logdet"][q] - ref["fac"].logdet()) <= 1e-5 * abs(ref["fac"].logdet())


def test_autotune_keeps_a_valid_configuration():
    import torch
    P = chol()
    probs, bd = _batch(count=80, kmin=8, kmax=48, seed=11)
    offs = bd["meta"]["offsets"].astype(np.int32)
    rc, h = P.chol_analyze_batch(len(offs) - 1, offs, bd["colptr"], bd["rowind"], bd["perm"], _opts(P))
    assert rc == 0
    vals = to_dev(bd["values"])
    assert P.chol_autotune(h, vals) == 0
    info = P.chol_get_info(h)
    assert info.persistent_threads in (128, 256)
    b = gridgen.rhs_uniform(bd.n, 1, seed=1)
    X = colmajor(b)
    assert P.chol_solve(h, X, 1) == 0
    torch.cuda.synchronize()
    eta = oracle.backward_error(bd.n, bd["colptr"], bd["rowind"], bd["values"], b, X.cpu().numpy())
    assert eta[0] <= 1e-14
    P.chol_destroy(h)


def test_batch_entry_points_match_the_oracle_per_system():
    # chol_factor_batch / chol_solve_batch on a batch handle, two right-hand sides
    import torch
    P = chol()
    probs, bd = _batch(count=40, kmin=4, kmax=24, seed=7)
    offs = bd["meta"]["offsets"].astype(np.int32)
    rc, h = P.chol_analyze_batch(len(offs) - 1, offs, bd["colptr"], bd["rowind"], bd["perm"], _opts(P))
    assert rc == 0
    try:
        b = gridgen.rhs_uniform(bd.n, 2, seed=3)
        assert P.chol_factor_batch(h, to_dev(bd["values"])) == 0
        X = colmajor(b)
        assert P.chol_solve_batch(h, X, 2) == 0
        torch.cuda.synchronize()
        x = X.cpu().numpy()
        for q, p in enumerate(probs[:8]):
            s0, s1 = int(offs[q]), int(offs[q + 1])
            ref = oracle.reference(p, b[s0:s1])
            assert np.max(np.abs(x[s0:s1] - ref["x"])) <= 1e-12 * max(1.0, np.max(np.abs(ref["x"])))
    finally:
        P.chol_destroy(h)


@pytest.mark.parametrize("persistent", [0, 1])
def test_batch_large_sides_at_bench_thresholds(persistent):
    """Systems with grid sides up to 96 (the top of the benchmark's range),
    with the benchmark's kernel-class thresholds (160 columns, 24,576 panel
    entries, 512 rows on the one-CTA kernel), graph replay: every system's x
    and log det against the oracle."""
    P = chol()
    probs, bd = _batch(count=16, kmin=80, kmax=96, seed=21)
    assert max(p["meta"]["k"] for p in probs) >= 90
    b = gridgen.rhs_uniform(bd.n, 1, seed=22)
    o = _opts(P, 0, persistent, 1)
    o.small_max_cols, o.small_max_panel, o.small_max_rows = 160, 24576, 512
    got = _run(P, bd, o, b)
    assert got["info"].persistent_ok == 1
    offs = bd["meta"]["offsets"]
    for q, p in enumerate(probs):
        bq = b[offs[q]:offs[q + 1]]
        ref = oracle.reference(p, bq)
        xq = got["x"][offs[q]:offs[q + 1]]
        assert np.max(np.abs(xq - ref["x"])) <= 1e-11 * np.max(np.abs(ref["x"]))
        assert abs(got["logdet"][q] - ref["fac"].logdet()) <= 1e-12 * abs(ref["fac"].logdet())


def test_tune_batch_searches_caches_and_keeps_parity(tmp_path):
    """chol_tune_batch: a search on a sample of the systems picks thresholds,
    merging and the launch configuration; the same pattern then comes from the
    cache file; the whole batch analyzed with the choice matches the oracle."""
    import torch
    P = chol()
    probs, bd = _batch(count=60, kmin=4, kmax=28, seed=31)
    offs = bd["meta"]["offsets"].astype(np.int32)
    vals = to_dev(bd["values"])
    cache = str(tmp_path / "tune.txt")
    rc, best, ms, hit = P.chol_tune_batch(len(offs) - 1, offs, bd["colptr"], bd["rowind"], bd["perm"], vals,
                                          sample_every=3, cache_path=cache)
    assert rc == 0 and not hit and ms > 0
    assert (best.small_max_cols, best.small_max_panel, best.small_max_rows) in (
        (64, 4096, 128), (128, 16384, 256), (160, 24576, 512))
    assert best.merge_growth in (0.0, 0.1, 0.25)
    rc2, best2, ms2, hit2 = P.chol_tune_batch(len(offs) - 1, offs, bd["colptr"], bd["rowind"], bd["perm"], vals,
                                              sample_every=3, cache_path=cache)
    assert rc2 == 0 and hit2
    assert (best2.small_max_cols, best2.merge_growth, best2.persistent, best2.use_graph) == \
        (best.small_max_cols, best.merge_growth, best.persistent, best.use_graph)
    b = gridgen.rhs_uniform(bd.n, 1, seed=32)
    got = _run(P, bd, best, b)
    for q, p in enumerate(probs):
        bq = b[offs[q]:offs[q + 1]]
        ref = oracle.reference(p, bq)
        xq = got["x"][offs[q]:offs[q + 1]]
        assert np.max(np.abs(xq - ref["x"])) <= 1e-11 * np.max(np.abs(ref["x"]))
        assert abs(got["logdet"][q] - ref["fac"].logdet()) <= 1e-12 * abs(ref["fac"].logdet())
