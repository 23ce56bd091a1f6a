"""Matrix Market input for user-supplied matrices.

read_symmetric(path) reads a `%%MatrixMarket matrix coordinate real symmetric`
file (1-based entries of the lower or upper triangle), or a `general` file
holding both triangles of a symmetric matrix (the lower one is kept after a
check that every entry has its mirror with an equal value), and returns the
lower triangle in CSC form, as chol_analyze takes it: (n, colptr int64, rowind int32,
values float64), rows sorted within each column, duplicates summed, every
diagonal entry present (explicit zeros where the file has none).
read_perm(path) reads a permutation (one 0- or 1-based index per line; 1-based
if the smallest is 1), as new -> old.
write_symmetric(path, n, colptr, rowind, values) writes the same form back.
"""
import numpy as np


def read_symmetric(path):
    with open(path) as f:
        header = f.readline().strip().lower().split()
        if len(header) < 5 or header[0] != "%%matrixmarket" or header[1] != "matrix" or header[2] != "coordinate":
            raise ValueError("not a coordinate Matrix Market file: %s" % path)
        if header[3] not in ("real", "integer", "double"):
            raise ValueError("values must be real (got %s)" % header[3])
        if header[4] not in ("symmetric", "general"):
            raise ValueError("the matrix must be symmetric (got %s storage)" % header[4])
        general = header[4] == "general"
        line = f.readline()
        while line.startswith("%"):
            line = f.readline()
        m, n, nnz = (int(x) for x in line.split()[:3])
        if m != n:
            raise ValueError("matrix is not square")
        data = np.loadtxt(f, ndmin=2) if nnz > 0 else np.zeros((0, 3))
    if data.shape[0] != nnz:
        raise ValueError("expected %d entries, read %d" % (nnz, data.shape[0]))
    i = data[:, 0].astype(np.int64) - 1
    j = data[:, 1].astype(np.int64) - 1
    v = data[:, 2].astype(np.float64)
    if nnz and (i.min() < 0 or j.min() < 0 or i.max() >= n or j.max() >= n):
        raise ValueError("entry index out of range")
    if general:
        lo, up = i > j, i < j
        kl = np.sort(i[lo] * n + j[lo])
        ku = np.sort(j[up] * n + i[up])   # mirrored into the lower triangle
        if not np.array_equal(kl, ku):
            raise ValueError("general storage: the pattern is not symmetric")
        vl = v[lo][np.argsort(i[lo] * n + j[lo], kind="stable")]
        vu = v[up][np.argsort(j[up] * n + i[up], kind="stable")]
        if vl.size and np.max(np.abs(vl - vu)) > 1e-12 * max(1.0, float(np.max(np.abs(v)))):
            raise ValueError("general storage: the values are not symmetric")
        keep = i >= j
        i, j, v = i[keep], j[keep], v[keep]
    r = np.maximum(i, j)
    c = np.minimum(i, j)
    # every diagonal entry present
    r = np.concatenate([r, np.arange(n)])
    c = np.concatenate([c, np.arange(n)])
    v = np.concatenate([v, np.zeros(n)])
    key = c * n + r
    order = np.argsort(key, kind="stable")
    key, v = key[order], v[order]
    uniq, start = np.unique(key, return_index=True)
    vals = np.add.reduceat(v, start) if v.size else v
    cols = uniq // n
    rows = uniq % n
    colptr = np.zeros(n + 1, np.int64)
    np.add.at(colptr, cols + 1, 1)
    colptr = np.cumsum(colptr)
    return n, colptr, rows.astype(np.int32), vals


def read_perm(path):
    p = np.loadtxt(path, dtype=np.int64, ndmin=1)
    if p.size and p.min() == 1:
        p = p - 1
    return p.astype(np.int32)


def write_symmetric(path, n, colptr, rowind, values):
    with open(path, "w") as f:
        f.write("%%MatrixMarket matrix coordinate real symmetric\n")
        f.write("%d %d %d\n" % (n, n, len(rowind)))
        for j in range(n):
            for t in range(int(colptr[j]), int(colptr[j + 1])):
                f.write("%d %d %.17g\n" % (int(rowind[t]) + 1, j + 1, float(values[t])))
