"""One factorization (and optionally one solve or one adjoint) of a named
synthetic workload, for running under a profiler.

    python -m paper_2409_14009_gb300.profile_case --grid elast:32 --precision bf16
    python -m paper_2409_14009_gb300.profile_case --grid neumann:48 --adjoint
    python -m paper_2409_14009_gb300.profile_case --batch 2000

Grids: ``neumann:k`` (7-point variable-coefficient k^3 Laplacian, Neumann,
shift 1e-6), ``dirichlet:k`` (7-point weighted k^3 Laplacian with Dirichlet
ghosts), ``elast:k`` (27-point 3-dof elasticity on a k^3 grid). The CUDA
library must already be built (``paper_2409_14009_gb300/build.py``).
"""
import argparse
import sys
import os

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))

import numpy as np  # noqa: E402
import torch  # noqa: E402

import gridgen  # noqa: E402
import paper_2409_14009_gb300 as P  # noqa: E402

PRECISIONS = {"fp64": P.CHOL_PREC_FP64, "fp32": P.CHOL_PREC_FP32, "tf32": P.CHOL_PREC_TF32,
              "bf16": P.CHOL_PREC_BF16}


def make(grid: str):
    kind, k = grid.split(":")
    k = int(k)
    if kind == "neumann":
        return gridgen.laplacian_neumann_varcoef((k, k, k), 1e-2, 1e2, 1e-6, seed=2)
    if kind == "dirichlet":
        return gridgen.laplacian_dirichlet_weighted((k, k, k), gridgen.SplitMix64(5), 1e-2, 1e2)
    if kind == "elast":
        return gridgen.elasticity_27pt(k, 1.0, 1e6, seed=3)
    raise SystemExit(f"unknown grid {grid}")


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--grid", default="neumann:48")
    ap.add_argument("--precision", default="fp64", choices=sorted(PRECISIONS))
    ap.add_argument("--merge", type=float, default=0.1)
    ap.add_argument("--block-cols", type=int, default=0, help="column block of the blocked path (0 = default)")
    ap.add_argument("--factors", type=int, default=1, help="factorizations to run")
    ap.add_argument("--nrhs", type=int, default=0, help="solve with this many right-hand sides")
    ap.add_argument("--adjoint", action="store_true", help="run one adjoint (selected inverse + gradient)")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead of --grid: this many independent 2D systems (sides U{16..96}), analysis options "
                         "from chol_tune_batch on every 10th system")
    ap.add_argument("--tuned", default="",
                    help="with --batch: skip the search and use 'cols,panel,rows,merge' (e.g. 128,16384,256,0.25)")
    ap.add_argument("--persistent", action="store_true",
                    help="with --batch --tuned: the persistent cooperative kernel instead of graph replay")
    ap.add_argument("--time", type=int, default=0,
                    help="time this many further factorizations (CUDA events), then one more with per-class events")
    a = ap.parse_args()
    o = P.chol_default_options()
    o.precision = PRECISIONS[a.precision]
    o.merge_growth = a.merge
    if a.block_cols:
        o.block_cols = a.block_cols
    if a.batch:
        probs = gridgen.batch_2d(count=a.batch)
        p = gridgen.block_diagonal(probs)
        offs = p["meta"]["offsets"].astype(np.int32)
        vals = torch.as_tensor(p["values"], device="cuda")
        if a.tuned:
            c, pn, r, m = a.tuned.split(",")
            o.small_max_cols, o.small_max_panel, o.small_max_rows, o.merge_growth = int(c), int(pn), int(r), float(m)
            o.use_graph, o.persistent = (0, 1) if a.persistent else (1, 0)
        else:
            rc, o, ms, _ = P.chol_tune_batch(len(offs) - 1, offs, p["colptr"], p["rowind"], p["perm"], vals, o, 10)
            if rc:
                raise P.CholError(rc, "chol_tune_batch")
        print(f"tuned: cols {o.small_max_cols} panel {o.small_max_panel} rows {o.small_max_rows} "
              f"merge {o.merge_growth} persistent {o.persistent} graph {o.use_graph}")
        rc, h = P.chol_analyze_batch(len(offs) - 1, offs, p["colptr"], p["rowind"], p["perm"], o)
        if rc:
            raise P.CholError(rc, "chol_analyze_batch")
        S = P.SparseCholesky.__new__(P.SparseCholesky)
        S.h, S.n, S.info = h, p.n, P.chol_get_info(h)
    else:
        p = make(a.grid)
        S = P.SparseCholesky(p.n, p["colptr"], p["rowind"], p["perm"], o)
        vals = torch.as_tensor(p["values"], device="cuda")
    for _ in range(a.factors):
        S.factor(vals)
    if a.nrhs:
        b = torch.as_tensor(gridgen.rhs_uniform(p.n, a.nrhs, seed=7), device="cuda")
        S.solve(b)
    if a.adjoint:
        b = torch.as_tensor(gridgen.rhs_uniform(p.n, 1, seed=7), device="cuda")
        x = S.solve(b)
        w = torch.ones_like(x)
        bbar = torch.empty_like(x)
        grad = torch.empty(len(p["rowind"]), dtype=torch.float64, device="cuda")
        rc = P.chol_adjoint(S.h, w, x, 1, 1.0, bbar, grad)
        if rc:
            raise P.CholError(rc, "chol_adjoint")
    if a.time:
        st = torch.cuda.current_stream()
        ms = []
        for _ in range(a.time):
            e0 = torch.cuda.Event(enable_timing=True); e1 = torch.cuda.Event(enable_timing=True)
            e0.record(st); S.factor(vals); e1.record(st); torch.cuda.synchronize()
            ms.append(e0.elapsed_time(e1))
        med = float(np.median(ms))
        print(f"factor: median {med:.3f} ms over {a.time} (min {min(ms):.3f}), {S.info.flops / med / 1e6:.1f} GFLOP/s")
        P.chol_profile(S.h, (1 << len(P.KERNEL_CLASSES)) - 1)
        P.chol_get_stats(S.h, reset=True)
        S.factor(vals)
        stats = P.chol_get_stats(S.h, reset=True)
        P.chol_profile(S.h, 0)
        for k, v in stats.items():
            if v["launches"]:
                print(f"  {k:14s} launches {v['launches']:6d}  event ms {v['ms']:9.3f}  flops {v['flops']:.3e}")
    torch.cuda.synchronize()
    print(f"ok n={p.n} flops={S.info.flops:.4g} panels={S.info.panel_doubles * (8 if a.precision == 'fp64' else 4) / 1e9:.3f} GB")


if __name__ == "__main__":
    main()
