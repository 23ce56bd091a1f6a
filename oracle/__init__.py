"""FP64 CPU oracle for the sparse Cholesky hot path (TEST INFRASTRUCTURE).

Only the tests, ``__graft_entry__.smoke()`` and the benchmark's CPU-baseline
leg may import this package. It restates the definitions of "GPU Accelerated
Sparse Cholesky Factorization" (Karsavuran, Ng, Peyton) in the plainest
form, in ``oracle.c`` (symbolic and numeric parts, the selected inverse) and
in this module (the inverse on the pattern of A and the loss gradient), plus
``merge.py`` (relaxed supernode merging):

* ``permute``           B = P A P^T                           (Sec. II, problem)
* ``symbolic``          etree parent, column counts, struct(L) (Sec. II, etree
                        definition; fill by symbolic elimination)
* ``supernodes``        maximal supernode partition and tree  (Sec. II, Fig. 1)
* ``relind``            relative indices by definition        (Sec. II-A)
* ``factor``            left-looking column Cholesky (cmod/cdiv), FP64
* ``solve``             forward/backward substitution          (Sec. I)
* ``logdet``, ``spmv``, ``backward_error``, ``factor_residual``
* ``Factor.selinv``     Takahashi recurrence on the pattern of L (selected inverse)
* ``inverse_on_pattern``, ``gradient``  (A^{-1} on the pattern of A; dl/dA, dl/db)

It shares no code with the CUDA library.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

from . import build as _build

_lib = None


def lib():
    global _lib
    if _lib is None:
        path = _build.build()
        L = C.CDLL(path)
        P = C.c_void_p
        L.orc_permute.restype = C.c_int
        L.orc_permute.argtypes = [C.c_int32, P, P, P, P, P, P, P]
        L.orc_sym_new.restype = C.c_void_p
        L.orc_sym_new.argtypes = [C.c_int32, P, P]
        L.orc_sym_nnz.restype = C.c_int64
        L.orc_sym_nnz.argtypes = [P]
        L.orc_sym_get.argtypes = [P, P, P, P, P]
        L.orc_sym_free.argtypes = [P]
        L.orc_supernodes.restype = C.c_int32
        L.orc_supernodes.argtypes = [C.c_int32, P, P, P, P]
        L.orc_relind.argtypes = [C.c_int32, C.c_int32, P, P, P, P, P, P, P, P]
        L.orc_factor_new.restype = C.c_void_p
        L.orc_factor_new.argtypes = [C.c_int32, P, P, P]
        L.orc_factor_new_mt.restype = C.c_void_p
        L.orc_factor_new_mt.argtypes = [C.c_int32, P, P, P, P, P, P, C.c_int32]
        L.orc_mt_begin.restype = C.c_void_p
        L.orc_mt_begin.argtypes = [C.c_int32, P, P, P, P, P, P, C.c_int32]
        L.orc_mt_max_height.restype = C.c_int32
        L.orc_mt_max_height.argtypes = [P]
        L.orc_mt_schedule.restype = None
        L.orc_mt_schedule.argtypes = [P, P, P]
        L.orc_mt_run.restype = None
        L.orc_mt_run.argtypes = [P, C.c_int32, C.c_int32]
        L.orc_mt_finish.restype = C.c_void_p
        L.orc_mt_finish.argtypes = [P]
        L.orc_factor_residual_parts.restype = None
        L.orc_factor_residual_parts.argtypes = [C.c_int32, P, P, P, P, P, P, C.c_int32, P, P]
        L.orc_factor_info.restype = C.c_int32
        L.orc_factor_info.argtypes = [P]
        L.orc_factor_nnz.restype = C.c_int64
        L.orc_factor_nnz.argtypes = [P]
        L.orc_factor_get.argtypes = [P, P, P, P]
        L.orc_factor_free.argtypes = [P]
        L.orc_solve.argtypes = [C.c_int32, P, P, P, P, C.c_int32, P, P]
        L.orc_logdet.restype = C.c_double
        L.orc_logdet.argtypes = [C.c_int32, P, P]
        L.orc_spmv.argtypes = [C.c_int32, P, P, P, C.c_int32, P, P]
        L.orc_backward_error.argtypes = [C.c_int32, P, P, P, C.c_int32, P, P, P]
        L.orc_selinv.restype = C.c_int
        L.orc_selinv.argtypes = [C.c_int32, P, P, P, P]
        L.orc_factor_residual_cols.argtypes = [C.c_int32, P, P, P, P, P, P, C.c_int32, P, P]
        L.orc_factor_residual.restype = C.c_double
        L.orc_factor_residual.argtypes = [C.c_int32, P, P, P, P, P, P]
        _lib = L
    return _lib


def _p(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _c(a, dt):
    return np.ascontiguousarray(a, dtype=dt)


def permute(n, colptr, rowind, values, perm):
    """Lower CSC of B = P A P^T (perm new->old; None = identity)."""
    colptr = _c(colptr, np.int64); rowind = _c(rowind, np.int32)
    values = None if values is None else _c(values, np.float64)
    perm = None if perm is None else _c(perm, np.int32)
    nnz = int(colptr[n])
    bp = np.zeros(n + 1, np.int64); bi = np.zeros(max(nnz, 1), np.int32)
    bx = np.zeros(max(nnz, 1), np.float64)
    rc = lib().orc_permute(n, _p(colptr), _p(rowind), _p(values), _p(perm), _p(bp), _p(bi), _p(bx))
    if rc != 0:
        raise ValueError("perm is not a permutation")
    return bp, bi[:nnz], (bx[:nnz] if values is not None else None)


class Symbolic:
    """parent, colcount, lp, li (struct(L) column by column) of B = P A P^T."""

    def __init__(self, n, bcolptr, browind):
        bcolptr = _c(bcolptr, np.int64); browind = _c(browind, np.int32)
        h = lib().orc_sym_new(n, _p(bcolptr), _p(browind))
        try:
            nnz = lib().orc_sym_nnz(h)
            self.n = n
            self.parent = np.zeros(n, np.int32)
            self.colcount = np.zeros(n, np.int32)
            self.lp = np.zeros(n + 1, np.int64)
            self.li = np.zeros(max(nnz, 1), np.int32)
            lib().orc_sym_get(h, _p(self.parent), _p(self.colcount), _p(self.lp), _p(self.li))
            self.li = self.li[:nnz]
        finally:
            lib().orc_sym_free(h)

    @property
    def nnz(self):
        return int(self.lp[-1])

    def flops(self):
        """Factor flop count sum_j c_j^2 (c_j = nnz of column j incl. diagonal)."""
        c = self.colcount.astype(np.int64)
        return int((c * c).sum())

    def supernodes(self):
        ptr = np.zeros(self.n + 1, np.int32)
        sp = np.zeros(max(self.n, 1), np.int32)
        ns = lib().orc_supernodes(self.n, _p(self.parent), _p(self.colcount), _p(ptr), _p(sp))
        return ptr[: ns + 1].copy(), sp[:ns].copy()

    def relind(self, snode_ptr):
        """(relind_ptr, relind_target, relind) for every (J, touched ancestor K)."""
        ns = len(snode_ptr) - 1
        sptr = _c(snode_ptr, np.int32)
        npairs = C.c_int64(0); tot = C.c_int64(0)
        L = lib()
        L.orc_relind(self.n, ns, _p(sptr), _p(self.lp), _p(self.li), C.byref(npairs), C.byref(tot),
                     None, None, None)
        rp = np.zeros(npairs.value + 1, np.int64)
        rt = np.zeros(max(npairs.value, 1), np.int32)
        ri = np.zeros(max(tot.value, 1), np.int32)
        L.orc_relind(self.n, ns, _p(sptr), _p(self.lp), _p(self.li), C.byref(npairs), C.byref(tot),
                     _p(rp), _p(rt), _p(ri))
        return rp, rt[: npairs.value], ri[: tot.value]


class Factor:
    """Left-looking FP64 column Cholesky of B. info = 0 or j+1 (bad pivot at j).

    threads = 1: the serial loops, pattern found on the fly. threads != 1: the
    same cmod/cdiv loops in parallel over the columns of each elimination-tree
    height (0 = all cores), on the pattern of the symbolic factor; the result
    agrees with the serial one up to the order of the cmod sums.
    """

    def __init__(self, n, bcolptr, browind, bvals, threads=1, _handle=None):
        if _handle is not None:
            h = _handle
        elif threads == 1:
            bcolptr = _c(bcolptr, np.int64); browind = _c(browind, np.int32); bvals = _c(bvals, np.float64)
            h = lib().orc_factor_new(n, _p(bcolptr), _p(browind), _p(bvals))
        else:
            bcolptr = _c(bcolptr, np.int64); browind = _c(browind, np.int32); bvals = _c(bvals, np.float64)
            sym = Symbolic(n, bcolptr, browind)
            li = sym.li if sym.li.size else np.zeros(1, np.int32)
            h = lib().orc_factor_new_mt(n, _p(bcolptr), _p(browind), _p(bvals), _p(sym.parent), _p(sym.lp),
                                        _p(li), int(threads))
        try:
            self.n = n
            self.info = lib().orc_factor_info(h)
            nnz = lib().orc_factor_nnz(h)
            self.lp = np.zeros(n + 1, np.int64)
            self.li = np.zeros(max(nnz, 1), np.int32)
            self.lx = np.zeros(max(nnz, 1), np.float64)
            lib().orc_factor_get(h, _p(self.lp), _p(self.li), _p(self.lx))
            self.li = self.li[:nnz]; self.lx = self.lx[:nnz]
        finally:
            lib().orc_factor_free(h)

    def solve(self, perm, b):
        b = np.asfortranarray(b, dtype=np.float64)
        nrhs = 1 if b.ndim == 1 else b.shape[1]
        x = np.zeros_like(b, order="F")
        perm = None if perm is None else _c(perm, np.int32)
        lib().orc_solve(self.n, _p(self.lp), _p(self.li), _p(self.lx), _p(perm), nrhs, _p(b), _p(x))
        return x

    def logdet(self):
        return lib().orc_logdet(self.n, _p(self.lp), _p(self.lx))

    def selinv(self):
        """Z = (P A P^T)^{-1} on the pattern of L (same layout as lx)."""
        zx = np.zeros_like(self.lx)
        if lib().orc_selinv(self.n, _p(self.lp), _p(self.li), _p(self.lx), _p(zx)) != 0:
            raise ValueError("pattern of L is not closed")
        return zx

    def diag(self):
        return self.lx[self.lp[:-1]]


class StagedFactor:
    """The multi-threaded factor (Factor with threads != 1) run in pieces:
    run(h0, h1) factors the elimination-tree heights [h0, h1), in increasing
    order, each height once; finish() returns the Factor. The loops and their
    order are those of the one-piece run, so the result does not depend on
    how the heights are split. work() gives sum c_j^2 per height, for
    splitting by work."""

    def __init__(self, n, bcolptr, browind, bvals, threads=0, sym=None):
        self._keep = (_c(bcolptr, np.int64), _c(browind, np.int32), _c(bvals, np.float64))
        bcolptr, browind, bvals = self._keep
        self.n = n
        sym = sym if sym is not None else Symbolic(n, bcolptr, browind)
        self.sym = sym
        li = sym.li if sym.li.size else np.zeros(1, np.int32)
        self._li = li
        self.h = lib().orc_mt_begin(n, _p(bcolptr), _p(browind), _p(bvals), _p(sym.parent), _p(sym.lp),
                                    _p(li), int(threads))
        self.max_height = lib().orc_mt_max_height(self.h)

    def work(self):
        mh = self.max_height
        hp = np.zeros(mh + 2, np.int64)
        byh = np.zeros(max(self.n, 1), np.int32)
        lib().orc_mt_schedule(self.h, _p(hp), _p(byh))
        c2 = np.diff(self.sym.lp).astype(np.float64) ** 2
        return np.add.reduceat(c2[byh[: self.n]], hp[:-1]) if self.n else np.zeros(0)

    def run(self, h0, h1):
        lib().orc_mt_run(self.h, int(h0), int(h1))

    def finish(self):
        h, self.h = lib().orc_mt_finish(self.h), None
        return Factor(self.n, None, None, None, _handle=h)


def spmv(n, colptr, rowind, values, x):
    x = np.asfortranarray(x, dtype=np.float64)
    nrhs = 1 if x.ndim == 1 else x.shape[1]
    y = np.zeros_like(x, order="F")
    lib().orc_spmv(n, _p(_c(colptr, np.int64)), _p(_c(rowind, np.int32)), _p(_c(values, np.float64)),
                   nrhs, _p(x), _p(y))
    return y


def backward_error(n, colptr, rowind, values, b, x):
    """Per right-hand side eta = ||b-Ax||_inf / (||A||_inf ||x||_inf + ||b||_inf)."""
    b = np.asfortranarray(b, dtype=np.float64); x = np.asfortranarray(x, dtype=np.float64)
    nrhs = 1 if b.ndim == 1 else b.shape[1]
    eta = np.zeros(nrhs)
    lib().orc_backward_error(n, _p(_c(colptr, np.int64)), _p(_c(rowind, np.int32)),
                             _p(_c(values, np.float64)), nrhs, _p(b), _p(x), _p(eta))
    return eta


def factor_residual(n, bcolptr, browind, bvals, lp, li, lx):
    """||B - L L^T||_F / ||B||_F (B = P A P^T lower CSC, L in CSC)."""
    r = lib().orc_factor_residual(n, _p(_c(bcolptr, np.int64)), _p(_c(browind, np.int32)),
                                  _p(_c(bvals, np.float64)), _p(_c(lp, np.int64)),
                                  _p(_c(li, np.int32)), _p(_c(lx, np.float64)))
    if r < 0:
        raise ValueError("L L^T or B has an entry outside the pattern of L")
    return r


def factor_residual_parts(n, bcolptr, browind, bvals, lp, li, lx, threads=0):
    """(||B - L L^T||_F / ||B||_F, per-column residual ||r_j|| / ||B_j||) with
    the columns computed in parallel (the global value is the quantity of
    factor_residual; the column sums are added in column order)."""
    num = np.zeros(max(n, 1)); den = np.zeros(max(n, 1))
    lib().orc_factor_residual_parts(n, _p(_c(bcolptr, np.int64)), _p(_c(browind, np.int32)),
                                    _p(_c(bvals, np.float64)), _p(_c(lp, np.int64)), _p(_c(li, np.int32)),
                                    _p(_c(lx, np.float64)), int(threads), _p(num), _p(den))
    num, den = num[:n], den[:n]
    tot = float(np.sqrt(np.sum(num)) / np.sqrt(np.sum(den))) if n else 0.0
    return tot, np.sqrt(num / den)


def factor_residual_cols(n, bcolptr, browind, bvals, lp, li, lx, cols):
    """Per sampled column j: ||B_{j:,j} - (L L^T)_{j:,j}||_2 / ||B_{j:,j}||_2."""
    cols = _c(cols, np.int32)
    out = np.zeros(len(cols))
    lib().orc_factor_residual_cols(n, _p(_c(bcolptr, np.int64)), _p(_c(browind, np.int32)),
                                   _p(_c(bvals, np.float64)), _p(_c(lp, np.int64)), _p(_c(li, np.int32)),
                                   _p(_c(lx, np.float64)), len(cols), _p(cols), _p(out))
    return out


def inverse_on_pattern(problem, fac, perm):
    """(A^{-1})_ij for every entry (i, j) of A's lower CSC, from the selected inverse."""
    n = problem["n"]
    zx = fac.selinv()
    iperm = np.empty(n, np.int64)
    iperm[np.asarray(perm, np.int64)] = np.arange(n)
    colptr, rowind = problem["colptr"], problem["rowind"]
    out = np.zeros(len(rowind))
    for c in range(n):
        for t in range(colptr[c], colptr[c + 1]):
            a, b = iperm[rowind[t]], iperm[c]
            r, k = max(a, b), min(a, b)
            lo, hi = fac.lp[k], fac.lp[k + 1]
            pos = lo + np.searchsorted(fac.li[lo:hi], r)
            out[t] = zx[pos]
    return out


def gradient(problem, fac, w, x, logdet_weight=1.0):
    """Gradient of  sum_k w_k^T x_k + logdet_weight * log det A  (x = A^{-1} b)
    with respect to the stored lower entries of A (a_ij and a_ji move
    together) and with respect to b:
      xbar = A^{-1} w,  G = -xbar x^T + logdet_weight * A^{-1},
      g_ii = G_ii,  g_ij = G_ij + G_ji (i > j)."""
    n = problem["n"]
    perm = problem["perm"]
    w = np.asfortranarray(w, dtype=np.float64)
    x = np.asfortranarray(x, dtype=np.float64)
    xbar = fac.solve(perm, w)
    zA = inverse_on_pattern(problem, fac, perm) if logdet_weight != 0.0 else None
    colptr, rowind = problem["colptr"], problem["rowind"]
    cols = np.repeat(np.arange(n), np.diff(colptr))
    rows = np.asarray(rowind, np.int64)
    xb2 = xbar.reshape(n, -1)
    x2 = x.reshape(n, -1)
    g = -(np.einsum("tk,tk->t", xb2[rows], x2[cols]))
    off = rows != cols
    g[off] -= np.einsum("tk,tk->t", xb2[cols[off]], x2[rows[off]])
    if zA is not None:
        g += logdet_weight * np.where(off, 2.0, 1.0) * zA
    return g, xbar


def reference(problem, b=None, threads=1):
    """Run the whole oracle on a gridgen problem: returns a dict of results
    (threads != 1: the multi-threaded numeric factor, 0 = all cores)."""
    n = problem["n"]
    bp, bi, bx = permute(n, problem["colptr"], problem["rowind"], problem["values"], problem["perm"])
    sym = Symbolic(n, bp, bi)
    fac = Factor(n, bp, bi, bx, threads=threads)
    out = dict(B=(bp, bi, bx), sym=sym, fac=fac)
    if b is not None:
        out["x"] = fac.solve(problem["perm"], b)
    return out
