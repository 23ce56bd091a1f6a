"""Failure path of the solve's bounded waits, made on purpose without a fault.

The diagonal-triangle kernels of the solve hand 64-row blocks from CTA to CTA
(binary64 through flags, binary32 through tagged words), each wait bounded by
chol_options.wait_polls. With the testing
option test_unreachable_flags the dependent blocks wait for a flag value that
no block ever publishes, so every such wait runs out after a few thousand
polls; the kernel records it and returns, the context stays usable, and
chol_check_waits reports CHOL_ETIMEOUT once (then the record is clear).
"""
import numpy as np
import pytest

import oracle
from gpu_util import colmajor, to_dev
from helpers import lower_csc_from_dense
from lib_fixture import chol

pytestmark = pytest.mark.gpu


def _dense_spd(n, seed):
    rs = np.random.RandomState(seed)
    M = rs.uniform(-1, 1, (n, n))
    return M @ M.T + n * np.eye(n)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_unreachable_flag_wait_gives_up_and_is_reported(precision):
    """binary64: flags per block; binary32: tagged hand-off words per entry."""
    import torch
    P = chol()
    n = 200                                   # one supernode of 200 columns: 4 diagonal blocks
    A = _dense_spd(n, 3)
    cp, ri, vx = lower_csc_from_dense(A)
    b = np.random.RandomState(4).uniform(-1, 1, (n, 2))
    prec = P.CHOL_PREC_FP64 if precision == "fp64" else P.CHOL_PREC_FP32
    eta_max = 1e-14 if precision == "fp64" else 1e-6
    o = P.chol_default_options()
    o.precision = prec
    o.test_unreachable_flags = 1
    o.wait_polls = 4096
    rc, h = P.chol_analyze(n, cp, ri, None, o)
    assert rc == 0
    st = torch.cuda.current_stream()
    try:
        assert P.chol_factor(h, to_dev(vx), st) == 0
        x = colmajor(b)
        assert P.chol_solve(h, x, 2, st) == 0          # asynchronous: the wait runs out later
        assert P.chol_check_waits(h, st) == P.CHOL_ETIMEOUT
        assert P.chol_check_waits(h, st) == 0          # the record was cleared
        torch.cuda.synchronize()                       # the context is still usable
    finally:
        P.chol_destroy(h)
    # the same system without the option: every wait is met and x is right
    o.test_unreachable_flags = 0
    o.wait_polls = 0
    rc, h = P.chol_analyze(n, cp, ri, None, o)
    assert rc == 0
    try:
        assert P.chol_factor(h, to_dev(vx), st) == 0
        x = colmajor(b)
        assert P.chol_solve(h, x, 2, st) == 0
        assert P.chol_check_waits(h, st) == 0
        eta = oracle.backward_error(n, cp, ri, vx, b, x.cpu().numpy())
        assert np.all(eta <= eta_max), eta
    finally:
        P.chol_destroy(h)


def test_check_waits_needs_a_factor():
    P = chol()
    A = _dense_spd(8, 1)
    cp, ri, vx = lower_csc_from_dense(A)
    rc, h = P.chol_analyze(8, cp, ri)
    assert rc == 0
    try:
        assert P.chol_check_waits(h) == P.CHOL_ESTATE
    finally:
        P.chol_destroy(h)
