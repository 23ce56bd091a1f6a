"""Factor and solve a user-supplied sparse SPD matrix on the GPU.

    python -m paper_2409_14009_gb300.run_matrix --mtx A.mtx [--perm p.txt]
    python -m paper_2409_14009_gb300.run_matrix --irregular 40

The matrix comes from a Matrix Market file (coordinate, real or integer; symmetric
storage, or general storage of a symmetric matrix) or from
the synthetic irregular generator (a k^3-node 27-point pattern with random
edges dropped). Without --perm it is ordered by chol_order_nd (nested
dissection on the graph). Prints one JSON line: sizes, ordering, analysis and
factor times, factor GFLOP/s (symbolic flops sum_j c_j^2), the solve or
refinement time and the backward error of the solution of A x = b with
b ~ U(-1, 1). The CUDA library must already be built
(paper_2409_14009_gb300/build.py).
"""
import argparse
import json
import os
import sys
import time

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import paper_2409_14009_gb300 as P  # noqa: E402
from paper_2409_14009_gb300 import mmio  # noqa: E402

PRECISIONS = {"fp64": P.CHOL_PREC_FP64, "fp32": P.CHOL_PREC_FP32, "tf32": P.CHOL_PREC_TF32,
              "bf16": P.CHOL_PREC_BF16}


def main(argv=None):
    ap = argparse.ArgumentParser()
    src = ap.add_mutually_exclusive_group(required=True)
    src.add_argument("--mtx", help="Matrix Market file (coordinate; symmetric, or general holding a symmetric matrix)")
    src.add_argument("--irregular", type=int, help="synthetic irregular pattern on a k^3 grid of nodes")
    ap.add_argument("--perm", help="ordering file (new -> old, one index per line)")
    ap.add_argument("--precision", default="fp64", choices=sorted(PRECISIONS))
    ap.add_argument("--update", default="rl", choices=["rl", "rlb"])
    ap.add_argument("--merge", type=float, default=0.1)
    ap.add_argument("--nrhs", type=int, default=1)
    ap.add_argument("--reps", type=int, default=3)
    a = ap.parse_args(argv)
    if a.mtx:
        n, colptr, rowind, values = mmio.read_symmetric(a.mtx)
        name = os.path.basename(a.mtx)
    else:
        import gridgen
        g = gridgen.irregular_3d(a.irregular)
        n, colptr, rowind, values = g.n, g["colptr"], g["rowind"], g["values"]
        name = "irregular_3d(%d)" % a.irregular
    t0 = time.perf_counter()
    if a.perm:
        perm, ordering = mmio.read_perm(a.perm), "given"
    else:
        rc, perm = P.chol_order_nd(n, colptr, rowind)
        if rc:
            raise P.CholError(rc, "chol_order_nd")
        ordering = "nested dissection (chol_order_nd)"
    order_s = time.perf_counter() - t0
    o = P.chol_default_options()
    o.precision = PRECISIONS[a.precision]
    o.merge_growth = a.merge
    o.update_mode = P.CHOL_UPDATE_RLB if a.update == "rlb" else P.CHOL_UPDATE_RL
    t0 = time.perf_counter()
    S = P.SparseCholesky(n, colptr, rowind, perm, o)
    analyze_s = time.perf_counter() - t0
    info = S.info
    st = torch.cuda.current_stream()
    vals = torch.as_tensor(values, device="cuda")
    S.factor(vals)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    fms = []
    for _ in range(max(a.reps, 1)):
        e0.record(st)
        S.factor(vals)
        e1.record(st)
        torch.cuda.synchronize()
        fms.append(e0.elapsed_time(e1))
    rng = np.random.RandomState(1)
    b = rng.uniform(-1.0, 1.0, size=(a.nrhs, n))
    B = torch.as_tensor(b, device="cuda").t()
    X = torch.zeros_like(B)
    e0.record(st)
    rc, iters, berr = P.chol_solve_refine(S.h, B, X, a.nrhs, 1e-10 if a.precision != "fp64" else 1e-14, 60, st)
    e1.record(st)
    torch.cuda.synchronize()
    fm = float(np.median(fms))
    out = {"matrix": name, "n": int(n), "nnz_lower": int(len(rowind)), "ordering": ordering,
           "order_s": order_s, "analyze_s": analyze_s, "nnz_l": int(info.nnz_l), "flops": float(info.flops),
           "supernodes": int(info.nsuper_storage), "levels": int(info.nlevels), "precision": a.precision,
           "update": a.update, "factor_ms": fm, "factor_gflops": info.flops / (fm * 1e-3) / 1e9,
           "solve_ms": e0.elapsed_time(e1), "refine_rc": int(rc), "refine_iterations": int(iters),
           "backward_error": float(np.max(berr))}
    print(json.dumps(out))
    S.close()
    return out


if __name__ == "__main__":
    main()
