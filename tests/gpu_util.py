"""GPU-side helpers for the parity tests (run the library through its C ABI)."""
import numpy as np

import oracle
from lib_fixture import chol


def to_dev(a):
    import torch
    return torch.as_tensor(np.ascontiguousarray(a), device="cuda")


def colmajor(b):
    """n x nrhs host array -> column-major CUDA tensor."""
    import torch
    b = np.asarray(b, dtype=np.float64)
    if b.ndim == 1:
        return to_dev(b)
    return torch.as_tensor(np.ascontiguousarray(b.T), device="cuda").t()


def run(problem, b=None, options=None):
    """Factor (and solve) on the GPU. Returns dict with rc, L (csc), x, logdet, handle info."""
    import torch
    P = chol()
    rc, h = P.chol_analyze(problem["n"], problem["colptr"], problem["rowind"], problem["perm"], options)
    assert rc == 0, rc
    out = dict(info=P.chol_get_info(h))
    try:
        vals = to_dev(problem["values"])
        st = torch.cuda.current_stream()
        rc = P.chol_factor(h, vals, st)
        out["rc"] = rc
        if rc != 0:
            return out
        out["L"] = P.chol_get_factor(h, st)
        if b is not None:
            xb = colmajor(b)
            nrhs = 1 if np.ndim(b) == 1 else np.shape(b)[1]
            assert P.chol_solve(h, xb, nrhs, st) == 0
            torch.cuda.synchronize()
            out["x"] = xb.cpu().numpy()
        rc, ld = P.chol_logdet(h, st)
        assert rc == 0
        out["logdet"] = ld
        out["stats"] = P.chol_get_stats(h)
    finally:
        P.chol_destroy(h)
    return out


def check_parity(problem, b=None, options=None, L_tol=1e-12, x_tol=1e-12, ref=None):
    """GPU vs oracle: integer pattern bit-exact, L per column within L_tol of the
    column's max, residual and backward error <= 1e-12, x and logdet close."""
    n = problem["n"]
    if ref is None:
        ref = oracle.reference(problem, b)
    got = run(problem, b, options)
    assert got["rc"] == 0, got["rc"]
    lp, li, lx = got["L"]
    f = ref["fac"]
    assert np.array_equal(lp, f.lp) and np.array_equal(li, f.li)
    colmax = np.maximum.reduceat(np.abs(f.lx), f.lp[:-1]) if n else np.zeros(0)
    err = np.abs(lx - f.lx)
    colerr = np.maximum.reduceat(err, f.lp[:-1]) if n else np.zeros(0)
    assert np.all(colerr <= L_tol * colmax), float(np.max(colerr / colmax))
    bp, bi, bx = ref["B"]
    assert oracle.factor_residual(n, bp, bi, bx, lp, li, lx) <= 1e-12
    assert abs(got["logdet"] - f.logdet()) <= 1e-12 * max(1.0, abs(f.logdet()))
    if b is not None:
        x, xr = got["x"], ref["x"]
        eta = oracle.backward_error(n, problem["colptr"], problem["rowind"], problem["values"], b, x)
        assert np.all(eta <= 1e-12), eta
        scale = np.max(np.abs(xr)) if xr.size else 1.0
        assert np.max(np.abs(x - xr)) <= x_tol * scale
    return got, ref
