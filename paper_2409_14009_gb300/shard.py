"""Sharding a batch of independent SPD systems over ranks (one GPU per rank).

The systems of a batch share nothing: each rank analyzes, factors and solves
its own share of them (chol_analyze_batch on the block-diagonal matrix of its
systems), and the only exchange is at the end, when every rank learns the
per-system status and log det of all systems (one all-gather of small
vectors). No device data crosses ranks.

Balance: the factorization of a 2D k x k grid under nested dissection costs
Theta(k^3) = Theta(n^1.5) flops, so the systems are assigned by a
longest-processing-time greedy on n^1.5: largest first, each to the rank with
the least assigned work so far (ties: the lower rank; equal sizes keep their
index order). The assignment is deterministic and depends only on the system
sizes and the number of ranks.
"""
from __future__ import annotations

import heapq

import numpy as np


def work_estimate(sizes) -> np.ndarray:
    """Relative factorization work of each system (n^1.5)."""
    return np.asarray(sizes, dtype=np.float64) ** 1.5


def partition_systems(sizes, world: int) -> list[np.ndarray]:
    """Indices of the systems each rank takes (ascending within a rank)."""
    if world < 1:
        raise ValueError("world must be >= 1")
    w = work_estimate(sizes)
    order = sorted(range(len(w)), key=lambda i: (-w[i], i))
    heap = [(0.0, r) for r in range(world)]
    parts = [[] for _ in range(world)]
    for i in order:
        load, r = heapq.heappop(heap)
        parts[r].append(i)
        heapq.heappush(heap, (load + w[i], r))
    return [np.array(sorted(p), dtype=np.int64) for p in parts]


def gather_results(dist, world: int, count: int, idx, logdets, status, device=None):
    """Every rank passes its systems' indices, log dets and statuses; every
    rank receives (logdet[count], status[count]) of the whole batch. One
    all-gather of fixed-size vectors (NaN / a sentinel where a rank has no
    entry), then each slot is taken from the rank that owns it."""
    import torch
    ld = torch.full((count,), float("nan"), dtype=torch.float64, device=device)
    st = torch.full((count,), -(2 ** 31) + 1, dtype=torch.int64, device=device)
    if len(idx):
        ii = torch.as_tensor(np.asarray(idx, np.int64), device=device)
        ld[ii] = torch.as_tensor(np.asarray(logdets, np.float64), device=device)
        st[ii] = torch.as_tensor(np.asarray(status, np.int64), device=device)
    if world == 1 or dist is None:
        return ld.cpu().numpy(), st.cpu().numpy()
    lds = [torch.empty_like(ld) for _ in range(world)]
    sts = [torch.empty_like(st) for _ in range(world)]
    dist.all_gather(lds, ld)
    dist.all_gather(sts, st)
    out_ld = torch.full_like(ld, float("nan"))
    out_st = torch.full_like(st, -(2 ** 31) + 1)
    for r in range(world):
        have = sts[r] != -(2 ** 31) + 1
        out_ld[have] = lds[r][have]
        out_st[have] = sts[r][have]
    return out_ld.cpu().numpy(), out_st.cpu().numpy()
