"""Relaxed supernode merging, restated plainly (TEST INFRASTRUCTURE).

The experimental setup (Sec. IV) merges supernode pairs J and its parent p(J)
one after another, each time choosing the pair whose merge adds the least new
fill (explicit zeros), and stops when the cumulative growth of factor storage
would pass the budget (25% in the paper). Readings used here, since the paper
does not spell them out:

* only a parent that directly follows J in column order can be merged (the
  column ordering is never changed), so a merged supernode stays contiguous;
* "storage" counts the stored lower-trapezoid entries of every supernode
  (s columns, len rows: s*len - s*(s-1)/2), and the budget is a fraction of
  nnz(L);
* ties go to the pair whose J has the smaller first column; a merge that would
  take the cumulative growth past the budget ends the process.

The structure of a merged supernode is the union of the structures of its
columns, taken here directly from the oracle's column structures (so the
library's shortcut "J's columns + struct(parent)" is checked, not assumed).
This is a pure-Python O(nsuper^2) search, for small problems only.
"""
from __future__ import annotations

import numpy as np


def _stored(s, length):
    return s * length - s * (s - 1) // 2


def merged_partition(sym, growth):
    """sym: oracle.Symbolic. Returns (snode_ptr, structures) after merging."""
    ptr, _ = sym.supernodes()
    n = sym.n
    cols = [sym.li[sym.lp[j]:sym.lp[j + 1]] for j in range(n)]

    def struct_of(f, l):
        rows = set(range(f, l))
        for j in range(f, l):
            rows.update(int(i) for i in cols[j] if i >= l)
        return sorted(rows)

    groups = [(int(ptr[k]), int(ptr[k + 1])) for k in range(len(ptr) - 1)]   # [f, l)
    structs = [struct_of(f, l) for f, l in groups]
    budget = growth * sym.nnz
    total = 0
    while True:
        best = None
        for k in range(len(groups) - 1):
            (f, l), (f2, l2) = groups[k], groups[k + 1]
            if sym.parent[l - 1] < f2 or sym.parent[l - 1] >= l2:
                continue                       # the next supernode is not J's parent
            merged = struct_of(f, l2)
            cost = (_stored(l2 - f, len(merged)) - _stored(l - f, len(structs[k]))
                    - _stored(l2 - f2, len(structs[k + 1])))
            key = (cost, f)
            if best is None or key < best[0]:
                best = (key, k, merged)
        if best is None or total + best[0][0] > budget:
            break
        (cost, _), k, merged = best
        total += cost
        groups[k] = (groups[k][0], groups[k + 1][1])
        structs[k] = merged
        del groups[k + 1]
        del structs[k + 1]
    snode_ptr = np.array([g[0] for g in groups] + [n], dtype=np.int32)
    return snode_ptr, structs
