"""GB300 supernodal sparse Cholesky: thin Python binding of the C ABI (include/chol.h).

Every numeric step runs in the CUDA library ``_build/libchol.so``; this module
only marshals arguments (NumPy arrays for host data, raw device pointers and
CUDA streams for device data; PyTorch tensors are accepted for convenience).
Importing works without a GPU; loading the library fails loudly if it has not
been built (``python -m paper_2409_14009_gb300.build`` or ``__graft_entry__.build()``).
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libchol.so")

CHOL_OK = 0
CHOL_ENOMEM = -1001
CHOL_ECUDA = -1002
CHOL_ETIMEOUT = -1003
CHOL_ENOCONV = -1004
CHOL_ESTATE = -1005
CHOL_ENOTSUP = -1006
CHOL_ETOOBIG = -1007
CHOL_EBOUNDS = -1008
CHOL_PREC_FP64 = 0
CHOL_PREC_FP32 = 1
CHOL_PREC_TF32 = 2
CHOL_PREC_BF16 = 3
CHOL_UPDATE_RL = 0
CHOL_UPDATE_RLB = 1

EXPORTED = ["chol_default_options", "chol_analyze", "chol_factor", "chol_solve", "chol_solve_noalloc", "chol_check_waits", "chol_factor_solve_host", "chol_probe_fp64", "chol_tune_batch", "chol_test_corrupt_plan",
            "chol_solve_refine", "chol_logdet", "chol_analyze_batch", "chol_logdet_batch", "chol_autotune",
            "chol_factor_batch", "chol_solve_batch",
            "chol_selected_inverse", "chol_adjoint",
            "chol_get_info", "chol_get_symbolic", "chol_get_partition", "chol_get_factor", "chol_profile",
            "chol_get_stats", "chol_destroy", "chol_strerror", "chol_order_nd"]

KERNEL_CLASSES = ["scatter", "small", "potrf", "trsm", "gemm", "syrk", "assemble", "solve_diag",
                  "selinv_inv", "solve_fasm", "solve_bpanel", "selinv_gemm", "permute", "logdet",
                  "solve_gemv", "selinv_gather", "adjoint", "panel"]


class chol_options(C.Structure):
    _fields_ = [("precision", C.c_int32), ("small_max_cols", C.c_int32),
                ("small_max_panel", C.c_int32), ("block_cols", C.c_int32),
                ("device_mem_cap", C.c_int64), ("merge_growth", C.c_double),
                ("small_max_rows", C.c_int32), ("persistent", C.c_int32), ("pivot_tau", C.c_double),
                ("static_pivot", C.c_int32), ("use_graph", C.c_int32), ("update_mode", C.c_int32),
                ("wait_polls", C.c_int64), ("test_unreachable_flags", C.c_int32), ("reserved_opt", C.c_int32)]


class chol_info(C.Structure):
    _fields_ = [("n", C.c_int32), ("nsuper", C.c_int32), ("nlevels", C.c_int32),
                ("max_cols", C.c_int32), ("nnz_a", C.c_int64), ("nnz_l", C.c_int64),
                ("n_relind_pairs", C.c_int64), ("relind_len", C.c_int64),
                ("panel_doubles", C.c_int64), ("update_doubles", C.c_int64),
                ("flops", C.c_double), ("n_small", C.c_int32), ("n_large", C.c_int32),
                ("nsuper_storage", C.c_int32), ("reserved", C.c_int32), ("nnz_stored", C.c_int64),
                ("flops_stored", C.c_double), ("precision", C.c_int32), ("fp64_fallbacks", C.c_int32),
                ("perturbed_pivots", C.c_int32), ("nsys", C.c_int32), ("persistent_ok", C.c_int32),
                ("persistent_threads", C.c_int32), ("persistent_ctas_per_sm", C.c_int32),
                ("launch_mode", C.c_int32), ("tc_launches_shallow", C.c_int32), ("tc_launches_deep", C.c_int32),
                ("panel_launches", C.c_int32), ("bounds_code", C.c_int32)]


class chol_kernel_stat(C.Structure):
    _fields_ = [("launches", C.c_int64), ("flops", C.c_double), ("bytes", C.c_double),
                ("ms", C.c_double), ("timed", C.c_int64)]


class CholError(RuntimeError):
    def __init__(self, code, where=""):
        self.code = code
        super().__init__("%s: %d (%s)" % (where, code, chol_strerror(code)))


_lib = None
_lib_checked = None
LIB_CHECKED_PATH = os.path.join(_HERE, "_build_checked", "libchol.so")


def lib():
    """Load libchol.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is None:
        if not os.path.exists(LIB_PATH):
            raise ImportError("libchol.so is not built: run __graft_entry__.build()")
        _lib = _declare(C.CDLL(LIB_PATH))
    return _lib


def lib_checked():
    """The bounds-checked build (``build.build(checked=True)``), same C ABI; its
    handles are used with its own functions only."""
    global _lib_checked
    if _lib_checked is None:
        if not os.path.exists(LIB_CHECKED_PATH):
            raise ImportError("the bounds-checked library is not built: build.build(checked=True)")
        _lib_checked = _declare(C.CDLL(LIB_CHECKED_PATH))
    return _lib_checked


def _declare(L):
    """Argument and result types of every exported function."""
    if True:
        P = C.c_void_p
        L.chol_default_options.argtypes = [C.POINTER(chol_options)]
        L.chol_analyze.argtypes = [C.c_int32, P, P, P, C.POINTER(chol_options), C.POINTER(C.c_void_p)]
        L.chol_analyze.restype = C.c_int
        L.chol_factor.argtypes = [P, P, P]
        L.chol_factor.restype = C.c_int
        L.chol_solve.argtypes = [P, P, C.c_int32, P]
        L.chol_solve.restype = C.c_int
        L.chol_solve_noalloc.argtypes = [P, P, C.c_int32, P]
        L.chol_solve_noalloc.restype = C.c_int
        L.chol_check_waits.argtypes = [P, P]
        L.chol_check_waits.restype = C.c_int
        L.chol_tune_batch.argtypes = [C.c_int32, P, P, P, P, P, C.POINTER(chol_options), C.c_int32, C.c_char_p,
                                      C.POINTER(chol_options), C.POINTER(C.c_double), C.POINTER(C.c_int32), P]
        L.chol_tune_batch.restype = C.c_int
        L.chol_probe_fp64.argtypes = [C.c_int32, C.c_int32, C.POINTER(C.c_double), C.POINTER(C.c_double), P]
        L.chol_probe_fp64.restype = C.c_int
        L.chol_factor_solve_host.argtypes = [P, P, P, P, C.c_int32, C.POINTER(C.c_double), P]
        L.chol_factor_solve_host.restype = C.c_int
        L.chol_solve_refine.argtypes = [P, P, P, C.c_int32, C.c_double, C.c_int32,
                                        C.POINTER(C.c_int32), P, P]
        L.chol_solve_refine.restype = C.c_int
        L.chol_analyze_batch.argtypes = [C.c_int32, P, P, P, P, C.POINTER(chol_options), C.POINTER(C.c_void_p)]
        L.chol_analyze_batch.restype = C.c_int
        L.chol_logdet_batch.argtypes = [P, P, P]
        L.chol_logdet_batch.restype = C.c_int
        L.chol_factor_batch.argtypes = [P, P, P]
        L.chol_factor_batch.restype = C.c_int
        L.chol_solve_batch.argtypes = [P, P, C.c_int32, P]
        L.chol_solve_batch.restype = C.c_int
        L.chol_autotune.argtypes = [P, P, P]
        L.chol_autotune.restype = C.c_int
        L.chol_selected_inverse.argtypes = [P, P, P]
        L.chol_selected_inverse.restype = C.c_int
        L.chol_adjoint.argtypes = [P, P, P, C.c_int32, C.c_double, P, P, P]
        L.chol_adjoint.restype = C.c_int
        L.chol_logdet.argtypes = [P, C.POINTER(C.c_double), P]
        L.chol_logdet.restype = C.c_int
        L.chol_get_info.argtypes = [P, C.POINTER(chol_info)]
        L.chol_get_info.restype = C.c_int
        L.chol_get_symbolic.argtypes = [P] + [P] * 9
        L.chol_get_symbolic.restype = C.c_int
        L.chol_get_partition.argtypes = [P, P, P, P, P]
        L.chol_get_partition.restype = C.c_int
        L.chol_get_factor.argtypes = [P, P, P, P, P]
        L.chol_get_factor.restype = C.c_int
        L.chol_profile.argtypes = [P, C.c_uint32]
        L.chol_profile.restype = C.c_int
        L.chol_get_stats.argtypes = [P, C.POINTER(chol_kernel_stat), C.c_int32]
        L.chol_get_stats.restype = C.c_int
        L.chol_destroy.argtypes = [P]
        L.chol_destroy.restype = None
        L.chol_strerror.argtypes = [C.c_int]
        L.chol_strerror.restype = C.c_char_p
        L.chol_test_corrupt_plan.argtypes = [P, C.c_int32]
        L.chol_test_corrupt_plan.restype = C.c_int
    return L


def _np(a, dt):
    return None if a is None else np.ascontiguousarray(a, dtype=dt)


def _ptr(a):
    return None if a is None else a.ctypes.data_as(C.c_void_p)


def _dev_ptr(x):
    """Raw device pointer of a torch tensor or an int."""
    if x is None:
        return None
    if isinstance(x, int):
        return C.c_void_p(x)
    return C.c_void_p(x.data_ptr())


def _stream(s):
    if s is None:
        return None
    if isinstance(s, int):
        return C.c_void_p(s)
    return C.c_void_p(s.cuda_stream)


# ---- the C ABI, name for name -------------------------------------------------

def chol_default_options() -> chol_options:
    o = chol_options()
    lib().chol_default_options(C.byref(o))
    return o


def chol_analyze(n, colptr, rowind, perm=None, opt=None):
    """Returns (rc, handle)."""
    colptr = _np(colptr, np.int64); rowind = _np(rowind, np.int32); perm = _np(perm, np.int32)
    h = C.c_void_p()
    rc = lib().chol_analyze(int(n), _ptr(colptr), _ptr(rowind), _ptr(perm),
                            C.byref(opt) if opt is not None else None, C.byref(h))
    return rc, h


def chol_order_nd(n, colptr, rowind):
    """Nested dissection ordering of a lower-triangle CSC pattern: returns (rc, perm)."""
    colptr = _np(colptr, np.int64); rowind = _np(rowind, np.int32)
    perm = np.zeros(max(int(n), 1), np.int32)
    rc = lib().chol_order_nd(int(n), _ptr(colptr), _ptr(rowind), _ptr(perm))
    return rc, perm[: int(n)]


def chol_analyze_batch(count, sys_ptr, colptr, rowind, perm=None, opt=None):
    """Returns (rc, handle) for a block-diagonal batch of independent systems."""
    sys_ptr = _np(sys_ptr, np.int32); colptr = _np(colptr, np.int64)
    rowind = _np(rowind, np.int32); perm = _np(perm, np.int32)
    h = C.c_void_p()
    rc = lib().chol_analyze_batch(int(count), _ptr(sys_ptr), _ptr(colptr), _ptr(rowind), _ptr(perm),
                                  C.byref(opt) if opt is not None else None, C.byref(h))
    return rc, h


def chol_logdet_batch(h, count, stream=None):
    out = np.zeros(max(int(count), 1), np.float64)
    rc = lib().chol_logdet_batch(h, _ptr(out), _stream(stream))
    return rc, out[: int(count)]


def chol_factor_batch(h, values, stream=None) -> int:
    return lib().chol_factor_batch(h, _dev_ptr(values), _stream(stream))


def chol_solve_batch(h, b, nrhs, stream=None) -> int:
    return lib().chol_solve_batch(h, _dev_ptr(b), int(nrhs), _stream(stream))


def chol_autotune(h, values, stream=None) -> int:
    return lib().chol_autotune(h, _dev_ptr(values), _stream(stream))


def chol_factor(h, values, stream=None) -> int:
    return lib().chol_factor(h, _dev_ptr(values), _stream(stream))


def chol_solve(h, b, nrhs, stream=None) -> int:
    return lib().chol_solve(h, _dev_ptr(b), int(nrhs), _stream(stream))


def chol_solve_noalloc(h, b, nrhs, stream=None) -> int:
    """chol_solve whose workspaces come from a fixed device array (no allocation)."""
    return lib().chol_solve_noalloc(h, _dev_ptr(b), int(nrhs), _stream(stream))


def _host_ptr(a):
    """Address of host data: a NumPy array or a CPU torch tensor (pinned or not)."""
    if a is None:
        return None
    if isinstance(a, np.ndarray):
        return a.ctypes.data_as(C.c_void_p)
    return C.c_void_p(a.data_ptr())


def chol_factor_solve_host(h, values, b, x, nrhs, want_logdet=True, stream=None):
    """Factor + solve + log det from host buffers (values, b, x: host arrays).
    Returns (rc, logdet or None)."""
    ld = C.c_double(0.0)
    rc = lib().chol_factor_solve_host(h, _host_ptr(values), _host_ptr(b), _host_ptr(x), int(nrhs),
                                      C.byref(ld) if want_logdet else None, _stream(stream))
    return rc, (ld.value if want_logdet else None)


def chol_tune_batch(count, sys_ptr, colptr, rowind, perm, values, base=None, sample_every=10, cache_path=None,
                    stream=None):
    """Returns (rc, best chol_options, sample factor ms, from_cache)."""
    sys_ptr = _np(sys_ptr, np.int32); colptr = _np(colptr, np.int64)
    rowind = _np(rowind, np.int32); perm = _np(perm, np.int32)
    best = chol_options()
    ms = C.c_double(0.0)
    fc = C.c_int32(0)
    rc = lib().chol_tune_batch(int(count), _ptr(sys_ptr), _ptr(colptr), _ptr(rowind), _ptr(perm), _dev_ptr(values),
                               C.byref(base) if base is not None else None, int(sample_every),
                               cache_path.encode() if cache_path else None, C.byref(best), C.byref(ms),
                               C.byref(fc), _stream(stream))
    return rc, best, ms.value, bool(fc.value)


def chol_probe_fp64(kind=0, reps=5, stream=None):
    """Measured FP64 GFLOP/s of the current GPU: kind 0 = DFMA, 1 = DMMA.
    Returns (rc, gflops, SM GHz during the best run)."""
    g = C.c_double(0.0)
    ghz = C.c_double(0.0)
    rc = lib().chol_probe_fp64(int(kind), int(reps), C.byref(g), C.byref(ghz), _stream(stream))
    return rc, g.value, ghz.value


def chol_test_corrupt_plan(h, kind) -> int:
    """Damage the host plan of a fresh handle (bounds-checked build only, for tests)."""
    return lib().chol_test_corrupt_plan(h, int(kind))


def chol_check_waits(h, stream=None) -> int:
    """Synchronize `stream`; CHOL_ETIMEOUT if a solve's bounded wait gave up since the last check."""
    return lib().chol_check_waits(h, _stream(stream))


def chol_solve_refine(h, b, x, nrhs, tol=1e-10, max_iter=30, stream=None):
    """Returns (rc, iterations, backward errors per right-hand side)."""
    it = C.c_int32(0)
    berr = np.zeros(max(int(nrhs), 1), np.float64)
    rc = lib().chol_solve_refine(h, _dev_ptr(b), _dev_ptr(x), int(nrhs), float(tol), int(max_iter),
                                 C.byref(it), _ptr(berr), _stream(stream))
    return rc, it.value, berr[: int(nrhs)]


def chol_selected_inverse(h, zvals, stream=None) -> int:
    return lib().chol_selected_inverse(h, _dev_ptr(zvals), _stream(stream))


def chol_adjoint(h, w, x, nrhs, logdet_weight, bbar, grad, stream=None) -> int:
    return lib().chol_adjoint(h, _dev_ptr(w), _dev_ptr(x), int(nrhs), float(logdet_weight), _dev_ptr(bbar),
                              _dev_ptr(grad), _stream(stream))


def chol_logdet(h, stream=None):
    out = C.c_double(0.0)
    rc = lib().chol_logdet(h, C.byref(out), _stream(stream))
    return rc, out.value


def chol_get_info(h) -> chol_info:
    info = chol_info()
    rc = lib().chol_get_info(h, C.byref(info))
    if rc:
        raise CholError(rc, "chol_get_info")
    return info


def chol_get_symbolic(h) -> dict:
    info = chol_get_info(h)
    n, ns = info.n, info.nsuper
    out = dict(parent=np.zeros(n, np.int32), colcount=np.zeros(n, np.int32),
               snode_ptr=np.zeros(ns + 1, np.int32), snode_parent=np.zeros(ns, np.int32),
               row_ptr=np.zeros(ns + 1, np.int64), rows=np.zeros(info.nnz_l and 1, np.int32),
               relind_ptr=np.zeros(info.n_relind_pairs + 1, np.int64),
               relind_target=np.zeros(max(info.n_relind_pairs, 1), np.int32),
               relind=np.zeros(max(info.relind_len, 1), np.int32))
    # rows[] holds sum over supernodes of |struct(J)|: size it from a first call
    rc = lib().chol_get_symbolic(h, None, None, None, None, _ptr(out["row_ptr"]), None, None, None, None)
    if rc:
        raise CholError(rc, "chol_get_symbolic")
    out["rows"] = np.zeros(max(int(out["row_ptr"][-1]), 1), np.int32)
    rc = lib().chol_get_symbolic(h, *(_ptr(out[k]) for k in (
        "parent", "colcount", "snode_ptr", "snode_parent", "row_ptr", "rows", "relind_ptr",
        "relind_target", "relind")))
    if rc:
        raise CholError(rc, "chol_get_symbolic")
    out["rows"] = out["rows"][: int(out["row_ptr"][-1])]
    out["relind_target"] = out["relind_target"][: info.n_relind_pairs]
    out["relind"] = out["relind"][: info.relind_len]
    return out


def chol_get_partition(h) -> dict:
    """Storage partition used by the kernels (after relaxed merging, if enabled)."""
    info = chol_get_info(h)
    ns = info.nsuper_storage
    out = dict(snode_ptr=np.zeros(ns + 1, np.int32), snode_parent=np.zeros(max(ns, 1), np.int32),
               row_ptr=np.zeros(ns + 1, np.int64))
    rc = lib().chol_get_partition(h, _ptr(out["snode_ptr"]), _ptr(out["snode_parent"]),
                                  _ptr(out["row_ptr"]), None)
    if rc:
        raise CholError(rc, "chol_get_partition")
    out["rows"] = np.zeros(max(int(out["row_ptr"][-1]), 1), np.int32)
    lib().chol_get_partition(h, None, None, None, _ptr(out["rows"]))
    out["rows"] = out["rows"][: int(out["row_ptr"][-1])]
    out["snode_parent"] = out["snode_parent"][:ns]
    return out


def chol_get_factor(h, stream=None):
    info = chol_get_info(h)
    lp = np.zeros(info.n + 1, np.int64)
    li = np.zeros(max(info.nnz_l, 1), np.int32)
    lx = np.zeros(max(info.nnz_l, 1), np.float64)
    rc = lib().chol_get_factor(h, _ptr(lp), _ptr(li), _ptr(lx), _stream(stream))
    if rc:
        raise CholError(rc, "chol_get_factor")
    return lp, li[: info.nnz_l], lx[: info.nnz_l]


def chol_profile(h, timing_mask: int) -> int:
    return lib().chol_profile(h, int(timing_mask))


def chol_get_stats(h, reset: bool = False) -> dict:
    """{class name: dict(launches, flops, bytes, ms, timed)}."""
    arr = (chol_kernel_stat * len(KERNEL_CLASSES))()
    rc = lib().chol_get_stats(h, arr, 1 if reset else 0)
    if rc:
        raise CholError(rc, "chol_get_stats")
    return {nm: dict(launches=a.launches, flops=a.flops, bytes=a.bytes, ms=a.ms, timed=a.timed)
            for nm, a in zip(KERNEL_CLASSES, arr)}


def chol_destroy(h) -> None:
    lib().chol_destroy(h)


def chol_strerror(code) -> str:
    return lib().chol_strerror(int(code)).decode()


# ---- convenience wrapper over torch device memory ------------------------------

class SparseCholesky:
    """Analyze once, factor many times, solve many times (device-resident).

    ``values`` and right-hand sides are float64 CUDA tensors; the current
    torch stream is used unless one is given.
    """

    def __init__(self, n, colptr, rowind, perm=None, options: chol_options | None = None):
        rc, h = chol_analyze(n, colptr, rowind, perm, options)
        if rc:
            raise CholError(rc, "chol_analyze")
        self.h = h
        self.n = int(n)
        self.info = chol_get_info(h)

    def _st(self, stream):
        import torch
        return stream if stream is not None else torch.cuda.current_stream()

    def factor(self, values, stream=None):
        rc = chol_factor(self.h, values, self._st(stream))
        if rc:
            raise CholError(rc, "chol_factor")

    def solve_(self, b, stream=None):
        """In place: b (n x nrhs, column-major = a transposed contiguous tensor, or 1-D)."""
        nrhs = 1 if b.dim() == 1 else b.shape[1]
        if b.dim() == 2 and nrhs > 1 and b.stride() != (1, self.n):
            raise ValueError("b must be column-major (n x nrhs with strides (1, n))")
        rc = chol_solve(self.h, b, nrhs, self._st(stream))
        if rc:
            raise CholError(rc, "chol_solve")
        return b

    def solve(self, b, stream=None):
        """Returns a new column-major tensor; b is left untouched."""
        import torch
        if b.dim() == 2:
            x = torch.empty_strided(tuple(b.shape), (1, b.shape[0]), dtype=b.dtype, device=b.device)
            x.copy_(b)
        else:
            x = b.clone()
        return self.solve_(x, stream)

    def logdet(self, stream=None):
        rc, v = chol_logdet(self.h, self._st(stream))
        if rc:
            raise CholError(rc, "chol_logdet")
        return v

    def symbolic(self):
        return chol_get_symbolic(self.h)

    def factor_csc(self, stream=None):
        return chol_get_factor(self.h, self._st(stream))

    def close(self):
        if self.h:
            chol_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
