"""Pins of oracle/merge.py (relaxed supernode merging, Sec. IV setup).

merged_partition is the restatement the library's merging is checked against,
so it is pinned here against things it does not compute itself:

* Fig. 1 by hand. Of the six supernodes only J5 -> J6 has its parent next in
  column order; merging them stores 21 entries for 7 + 10, i.e. 4 explicit
  zeros (rows 12 and 13 of columns 10 and 11). The merged J4..J6, J3..J6,
  J2..J6 and J1..J6 then add 8, 15, 16 and 20 zeros (cumulative 4, 12, 27, 43,
  63 against nnz(L) = 57), so each budget below keeps a known prefix of that
  chain.
* A brute-force restatement on small random patterns: at every step it forms
  every admissible merge, counts the stored cells of the WHOLE resulting
  partition on a dense grid (not by the trapezoid formula, not as a
  difference), takes the smallest total (ties: the smaller first column) and
  ends when the total growth over nnz(L) would pass the budget. It also checks
  that every nonzero of L lies in a stored cell.
"""
import numpy as np
import pytest

import oracle
from golden_fig1 import load
from helpers import random_spd
from oracle.merge import merged_partition


def _fig1_symbolic():
    g = load()
    n = 15
    A = np.zeros((n, n))
    for j, rows in g["cols"].items():
        A[j - 1, j - 1] = 4.0 * n
        for i in rows:
            A[i - 1, j - 1] = A[j - 1, i - 1] = -1.0
    # the fill of Fig. 1 is already in this pattern (L's own pattern regenerates it)
    cp = [0]
    ri = []
    for j in range(n):
        ri += [i for i in range(j, n) if A[i, j] != 0.0]
        cp.append(len(ri))
    return oracle.Symbolic(n, np.array(cp, np.int64), np.array(ri, np.int32))


@pytest.mark.parametrize("growth,expect", [
    (0.05, [0, 2, 4, 7, 9, 11, 15]),      # 4 > 2.85: nothing merges
    (0.1, [0, 2, 4, 7, 9, 15]),           # J5+J6 (4 <= 5.7)
    (0.25, [0, 2, 4, 7, 15]),             # + J4 (12 <= 14.25); J3 would make 27
    (0.5, [0, 2, 4, 15]),                 # + J3 (27 <= 28.5); J2 would make 43
    (1.0, [0, 2, 15]),                    # + J2 (43 <= 57); J1 would make 63
    (1.2, [0, 15]),                       # everything (63 <= 68.4): one dense block
])
def test_fig1_merge_chain_by_hand(growth, expect):
    sym = _fig1_symbolic()
    assert sym.nnz == 57
    ptr, structs = merged_partition(sym, growth)
    assert ptr.tolist() == expect
    # the merged structures are contiguous ranges here (1-based {f..15} for a
    # block that reaches J6) or the canonical ones of Fig. 1
    canon = {(0, 2): [0, 1, 5, 6, 13], (2, 4): [2, 3, 7, 8, 12], (4, 7): [4, 5, 6, 12, 13, 14],
             (7, 9): [7, 8, 11, 12], (9, 11): [9, 10, 13, 14]}
    for k, st in enumerate(structs):
        f, l = int(ptr[k]), int(ptr[k + 1])
        assert st == (canon[(f, l)] if (f, l) in canon else list(range(f, 15)))


def _dense_pattern(sym):
    n = sym.n
    Lp = np.zeros((n, n), bool)
    for j in range(n):
        Lp[sym.li[sym.lp[j]:sym.lp[j + 1]], j] = True
    return Lp


def _stored_cells(Lp, groups):
    """Cells kept by a partition: for a group [f, l), every (i, j) with
    f <= j < l, i >= j and i in the union of the rows of its columns."""
    n = Lp.shape[0]
    keep = np.zeros((n, n), bool)
    for f, l in groups:
        rows = np.any(Lp[:, f:l], axis=1)
        for j in range(f, l):
            keep[j:, j] = rows[j:]
    return keep


def _brute_merge(sym, growth):
    Lp = _dense_pattern(sym)
    nnz = int(Lp.sum())
    ptr, _ = sym.supernodes()
    groups = [(int(ptr[k]), int(ptr[k + 1])) for k in range(len(ptr) - 1)]
    while True:
        cands = []
        for k in range(len(groups) - 1):
            (f, l), (f2, l2) = groups[k], groups[k + 1]
            p = int(sym.parent[l - 1])
            if not (f2 <= p < l2):
                continue
            trial = groups[:k] + [(f, l2)] + groups[k + 2:]
            cells = _stored_cells(Lp, trial)
            assert np.all(cells[Lp]), "a nonzero of L fell outside the stored cells"
            cands.append((int(cells.sum()), f, trial))
        if not cands:
            break
        total, _, trial = min(cands, key=lambda c: (c[0], c[1]))
        if total - nnz > growth * nnz:
            break
        groups = trial
    cells = _stored_cells(Lp, groups)
    structs = [sorted(np.nonzero(np.any(Lp[:, f:l], axis=1))[0].tolist()) for f, l in groups]
    return np.array([g[0] for g in groups] + [sym.n], np.int32), structs, int(cells.sum())


@pytest.mark.parametrize("seed", range(12))
@pytest.mark.parametrize("growth", [0.03, 0.1, 0.25, 0.6, 3.0])
def test_merge_matches_brute_force(seed, growth):
    n = 18 + 3 * seed
    A, cp, ri, vx, perm = random_spd(n, 0.12, 1000 + seed)
    bp, bi, _ = oracle.permute(n, cp, ri, None, perm)
    sym = oracle.Symbolic(n, bp, bi)
    ptr, structs = merged_partition(sym, growth)
    bptr, bstructs, stored = _brute_merge(sym, growth)
    assert ptr.tolist() == bptr.tolist()
    assert structs == bstructs
    assert stored - sym.nnz <= growth * sym.nnz


def test_brute_force_sees_ties_and_branching():
    """The random cases include steps with several admissible merges and steps
    where two of them add the same number of zeros, so the tie rule and the
    choice of the cheapest pair are exercised, not only chains."""
    ties = branching = 0
    for seed in range(12):
        n = 18 + 3 * seed
        A, cp, ri, vx, perm = random_spd(n, 0.12, 1000 + seed)
        bp, bi, _ = oracle.permute(n, cp, ri, None, perm)
        sym = oracle.Symbolic(n, bp, bi)
        Lp = _dense_pattern(sym)
        ptr, _ = sym.supernodes()
        groups = [(int(ptr[k]), int(ptr[k + 1])) for k in range(len(ptr) - 1)]
        costs = []
        for k in range(len(groups) - 1):
            (f, l), (f2, l2) = groups[k], groups[k + 1]
            if f2 <= int(sym.parent[l - 1]) < l2:
                trial = groups[:k] + [(f, l2)] + groups[k + 2:]
                costs.append(int(_stored_cells(Lp, trial).sum()))
        branching += len(costs) > 1
        ties += len(costs) != len(set(costs))
    assert branching >= 6 and ties >= 2, (branching, ties)
