"""Small test helpers: random sparse SPD matrices and dense conversions."""
import numpy as np


def lower_csc_from_dense(A):
    n = A.shape[0]
    colptr = [0]
    rows, vals = [], []
    for j in range(n):
        nz = [i for i in range(j, n) if A[i, j] != 0.0 or i == j]
        rows.extend(nz)
        vals.extend(A[i, j] for i in nz)
        colptr.append(len(rows))
    return (np.array(colptr, np.int64), np.array(rows, np.int32), np.array(vals, np.float64))


def dense_from_lower(n, colptr, rowind, values):
    A = np.zeros((n, n))
    for j in range(n):
        for t in range(colptr[j], colptr[j + 1]):
            i = rowind[t]
            A[i, j] = values[t]
            A[j, i] = values[t]
    return A


def random_spd(n, density, seed, perm=True):
    """Strictly diagonally dominant random sparse SPD matrix (lower CSC) + perm."""
    rs = np.random.RandomState(seed)
    M = (rs.rand(n, n) < density)
    M = np.tril(M, -1)
    off = np.where(M, -rs.uniform(0.1, 1.0, (n, n)), 0.0)
    A = off + off.T
    A[np.diag_indices(n)] = np.abs(A).sum(axis=1) + rs.uniform(0.5, 1.5, n)
    cp, ri, vx = lower_csc_from_dense(A)
    p = rs.permutation(n).astype(np.int32) if perm else np.arange(n, dtype=np.int32)
    return A, cp, ri, vx, p


def graph_from_lower(n, colptr, rowind):
    adj = [set() for _ in range(n)]
    for j in range(n):
        for t in range(colptr[j], colptr[j + 1]):
            i = int(rowind[t])
            if i != j:
                adj[i].add(j); adj[j].add(i)
    return adj


def brute_fill(n, adj):
    """struct(j) minus j for every column, by the fill-path theorem:
    L_ij != 0 (i > j) iff G(A) has a path i..j whose inner vertices are < j."""
    out = []
    for j in range(n):
        seen = {j}
        stack = [j]
        while stack:
            v = stack.pop()
            for w in adj[v]:
                if w < j and w not in seen:
                    seen.add(w)
                    stack.append(w)
        rows = set()
        for v in seen:
            rows.update(w for w in adj[v] if w > j)
        out.append(sorted(rows))
    return out


def csc_to_dense_lower(n, lp, li, lx):
    L = np.zeros((n, n))
    for j in range(n):
        for t in range(lp[j], lp[j + 1]):
            L[li[t], j] = lx[t]
    return L
