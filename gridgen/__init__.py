"""Seeded synthetic inputs for the sparse Cholesky hot path.

This module only *generates inputs*: grid-graph SPD matrices in lower CSC form,
the geometric nested-dissection permutation, and right-hand sides. It holds none
of the factorization's arithmetic, and both the CPU oracle and the CUDA path
(tests, bench) draw their inputs from it.

Conventions (the paper is silent on all of them; they are readings stated in the
design notes):

* Grid nodes carry the natural index ``x + kx*(y + ky*z)``; for vector problems
  the degree of freedom is the fastest index (``dof + ndof*node``).
* Random numbers come from SplitMix64 (Steele, Lea, Flood, "Fast splittable
  pseudorandom number generators", OOPSLA 2014): ``state += 0x9E3779B97F4A7C15``
  then the two xor-shift-multiply rounds and a final xor-shift. A uniform double
  in [0,1) is ``(z >> 11) * 2**-53``. Draws are taken in "edge order" (node in
  natural order, then the direction loop of each generator).
* Log-uniform ``c = 10**(lo + (hi-lo)*u)``; N(0,1) by Box-Muller.
* Matrices are returned as the lower triangle (diagonal included) in CSC with
  0-based, ascending, unique row indices, ``colptr`` int64 and ``rowind`` int32.
* ``perm`` is new->old: row/column ``i`` of P A P^T is row/column ``perm[i]`` of A.
"""
from __future__ import annotations

import numpy as np

_GAMMA = np.uint64(0x9E3779B97F4A7C15)
_M1 = np.uint64(0xBF58476D1CE4E5B9)
_M2 = np.uint64(0x94D049BB133111EB)


class SplitMix64:
    """Counter-based SplitMix64 stream: draw ``m`` values at once."""

    def __init__(self, seed: int):
        self.state = np.uint64(seed & 0xFFFFFFFFFFFFFFFF)

    def next_u64(self, m: int) -> np.ndarray:
        with np.errstate(over="ignore"):
            k = np.arange(1, m + 1, dtype=np.uint64)
            z = self.state + k * _GAMMA
            self.state = self.state + np.uint64(m) * _GAMMA
            z = (z ^ (z >> np.uint64(30))) * _M1
            z = (z ^ (z >> np.uint64(27))) * _M2
            z = z ^ (z >> np.uint64(31))
        return z

    def uniform(self, m: int) -> np.ndarray:
        """m doubles uniform in [0, 1)."""
        return (self.next_u64(m) >> np.uint64(11)).astype(np.float64) * (2.0 ** -53)

    def log_uniform(self, m: int, lo: float, hi: float) -> np.ndarray:
        """10**U(log10 lo, log10 hi)."""
        a, b = np.log10(lo), np.log10(hi)
        return 10.0 ** (a + (b - a) * self.uniform(m))

    def normal(self, m: int) -> np.ndarray:
        """Box-Muller: pairs (u1,u2) -> sqrt(-2 ln(1-u1)) cos(2 pi u2), sin(...)."""
        h = (m + 1) // 2
        u = self.uniform(2 * h).reshape(h, 2)
        r = np.sqrt(-2.0 * np.log1p(-u[:, 0]))
        t = 2.0 * np.pi * u[:, 1]
        return np.stack([r * np.cos(t), r * np.sin(t)], axis=1).reshape(-1)[:m]


# ----------------------------------------------------------------------------
# geometric nested dissection
# ----------------------------------------------------------------------------

def _box_points_lex(lo, hi, dims):
    """Natural indices of the box [lo, hi) listed lexicographically, axis 0 slowest."""
    axes = [np.arange(lo[a], hi[a], dtype=np.int64) for a in range(len(dims))]
    grids = np.meshgrid(*axes, indexing="ij")  # axis 0 slowest in C order
    idx = np.zeros(grids[0].shape, dtype=np.int64)
    stride = 1
    for a in range(len(dims)):
        idx += grids[a] * stride
        stride *= dims[a]
    return idx.reshape(-1)


_ND_CACHE = {}


def nd_order(dims) -> np.ndarray:
    """Deterministic geometric nested dissection of a box grid.

    Returns the node order (new -> old node index). Rule: a box whose longest
    extent is <= 2 is emitted lexicographically (axis 0 slowest); otherwise the
    longest axis (ties: lowest axis index) is split at ``mid = lo + ext//2`` and
    the order is ND(low part), ND(high part), then the plane ``mid``.
    """
    dims = tuple(int(d) for d in dims)
    if dims in _ND_CACHE:
        return _ND_CACHE[dims].copy()
    out = []

    def rec(lo, hi):
        ext = [hi[a] - lo[a] for a in range(len(dims))]
        if min(ext) <= 0:
            return
        m = max(ext)
        if m <= 2:
            out.append(_box_points_lex(lo, hi, dims))
            return
        a = ext.index(m)
        mid = lo[a] + m // 2
        lo_hi = list(hi); lo_hi[a] = mid
        rec(lo, tuple(lo_hi))
        hi_lo = list(lo); hi_lo[a] = mid + 1
        rec(tuple(hi_lo), hi)
        plo = list(lo); plo[a] = mid
        phi = list(hi); phi[a] = mid + 1
        out.append(_box_points_lex(tuple(plo), tuple(phi), dims))
    rec(tuple(0 for _ in dims), dims)
    order = np.concatenate(out) if out else np.zeros(0, dtype=np.int64)
    assert order.size == int(np.prod(dims))
    _ND_CACHE[dims] = order
    return order.copy()


def nd_perm(dims, ndof: int = 1) -> np.ndarray:
    """new->old permutation of the matrix rows: ND node order, dof fastest."""
    order = nd_order(dims)
    if ndof == 1:
        return order.astype(np.int32)
    p = (order[:, None] * ndof + np.arange(ndof)[None, :]).reshape(-1)
    return p.astype(np.int32)


# ----------------------------------------------------------------------------
# assembly helpers (COO -> lower CSC)
# ----------------------------------------------------------------------------

def coo_to_lower_csc(n, rows, cols, vals):
    """Sum duplicates of a symmetric COO given by its lower entries (row >= col)."""
    rows = np.asarray(rows, dtype=np.int64)
    cols = np.asarray(cols, dtype=np.int64)
    vals = np.asarray(vals, dtype=np.float64)
    assert np.all(rows >= cols)
    key = cols * n + rows
    order = np.argsort(key, kind="stable")
    key = key[order]
    vals = vals[order]
    uniq, start = np.unique(key, return_index=True)
    summed = np.add.reduceat(vals, start) if vals.size else vals
    c = uniq // n
    r = uniq - c * n
    colptr = np.zeros(n + 1, dtype=np.int64)
    np.add.at(colptr, c + 1, 1)
    colptr = np.cumsum(colptr)
    return colptr, r.astype(np.int32), summed.astype(np.float64)


def _grid_coords(dims):
    n = int(np.prod(dims))
    idx = np.arange(n, dtype=np.int64)
    coords = []
    rem = idx
    for d in dims:
        coords.append(rem % d)
        rem = rem // d
    return idx, coords


def _offset_index(dims, coords, off):
    """Neighbour natural index for offset ``off`` (or -1 outside the grid)."""
    n = coords[0].size
    ok = np.ones(n, dtype=bool)
    nb = np.zeros(n, dtype=np.int64)
    stride = 1
    for a, d in enumerate(dims):
        c = coords[a] + off[a]
        ok &= (c >= 0) & (c < d)
        nb += c * stride
        stride *= d
    return np.where(ok, nb, -1)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

class Problem(dict):
    """n, colptr, rowind, values (lower CSC of A), perm (new->old), meta."""

    @property
    def n(self):
        return self["n"]


def laplacian_2d_dirichlet(k: int, shift: float = 1e-3) -> Problem:
    """5-point Dirichlet Laplacian on a k x k grid: diagonal 4+shift, neighbours -1."""
    dims = (k, k)
    n = k * k
    idx, coords = _grid_coords(dims)
    R, C, V = [idx], [idx], [np.full(n, 4.0 + shift)]
    for a in range(2):
        off = [0, 0]; off[a] = 1
        nb = _offset_index(dims, coords, off)
        m = nb >= 0
        R.append(nb[m]); C.append(idx[m]); V.append(np.full(int(m.sum()), -1.0))
    colptr, rowind, vals = coo_to_lower_csc(n, np.concatenate(R), np.concatenate(C), np.concatenate(V))
    return Problem(n=n, colptr=colptr, rowind=rowind, values=vals, perm=nd_perm(dims),
                   meta=dict(kind="laplacian_2d_dirichlet", k=k, shift=shift))


def laplacian_neumann_varcoef(dims, lo: float, hi: float, shift: float, seed: int) -> Problem:
    """Grid graph Laplacian with per-edge conductances log-uniform in [lo, hi].

    Edge order: node in natural order, then axis 0..d-1 towards the +1
    neighbour (edges leaving the grid do not exist). A_ij = -c_e,
    A_ii = sum of incident c_e + shift (Neumann graph Laplacian plus a shift).
    """
    dims = tuple(int(d) for d in dims)
    d = len(dims)
    n = int(np.prod(dims))
    idx, coords = _grid_coords(dims)
    nbs = []
    for a in range(d):
        off = [0] * d; off[a] = 1
        nbs.append(_offset_index(dims, coords, off))
    nb = np.stack(nbs, axis=1).reshape(-1)           # (node, axis) in edge order
    src = np.repeat(idx, d)
    m = nb >= 0
    rng = SplitMix64(seed)
    c = rng.log_uniform(int(m.sum()), lo, hi)
    i, j = nb[m], src[m]
    diag = np.full(n, shift)
    np.add.at(diag, i, c)
    np.add.at(diag, j, c)
    colptr, rowind, vals = coo_to_lower_csc(n, np.concatenate([idx, i]), np.concatenate([idx, j]),
                                            np.concatenate([diag, -c]))
    return Problem(n=n, colptr=colptr, rowind=rowind, values=vals, perm=nd_perm(dims),
                   meta=dict(kind="laplacian_neumann_varcoef", dims=dims, lo=lo, hi=hi,
                             shift=shift, seed=seed))


def _offsets_27():
    offs = []
    for dz in (-1, 0, 1):
        for dy in (-1, 0, 1):
            for dx in (-1, 0, 1):
                if (dx, dy, dz) != (0, 0, 0):
                    offs.append((dx, dy, dz))
    return offs


def _is_positive(off):
    """Lexicographically positive offset, comparing the slowest index (z) first."""
    for v in (off[2], off[1], off[0]):
        if v != 0:
            return v > 0
    return False


def elasticity_27pt(k: int, lo: float = 1.0, hi: float = 1e6, seed: int = 3) -> Problem:
    """3-dof-per-node 27-point SPD operator on a k^3 grid (elasticity-like blocks).

    For every 27-point edge e = (i, j) a conductance c_e is drawn log-uniform in
    [lo, hi] and the 3x3 block K_e = c_e (I + d_e d_e^T) (d_e the unit edge
    direction) enters A as (e_i - e_j)(e_i - e_j)^T (x) K_e. Edge order: node in
    natural order, then the 26 offsets in lexicographic order (dz slowest);
    an in-grid neighbour is drawn only from the lexicographically positive
    side; an offset leaving the grid is a Dirichlet ghost whose K_e is added to
    the node's diagonal block only. SPD by construction.
    """
    dims = (k, k, k)
    n_nodes = k ** 3
    idx, coords = _grid_coords(dims)
    offs = _offsets_27()
    nb_all = np.stack([_offset_index(dims, coords, o) for o in offs], axis=1)  # (node, 26)
    pos = np.array([_is_positive(o) for o in offs])
    draw = (nb_all < 0) | pos[None, :]             # which (node, offset) draw a c
    rng = SplitMix64(seed)
    c = np.zeros(nb_all.shape)
    c[draw] = rng.log_uniform(int(draw.sum()), lo, hi)  # row-major = edge order
    dirs = np.array(offs, dtype=np.float64)
    dirs /= np.linalg.norm(dirs, axis=1, keepdims=True)
    Kunit = np.eye(3)[None] + dirs[:, :, None] * dirs[:, None, :]   # (26, 3, 3)
    # diagonal blocks: sum over every incident edge (both ends) and ghosts
    D = np.zeros((n_nodes, 3, 3))
    ghost = nb_all < 0
    edge = (~ghost) & pos[None, :]
    for o in range(len(offs)):
        g = ghost[:, o]
        if g.any():
            D[g] += c[g, o][:, None, None] * Kunit[o]
        e = edge[:, o]
        if e.any():
            blk = c[e, o][:, None, None] * Kunit[o]
            D[e] += blk
            np.add.at(D, nb_all[e, o], blk)
    R, C, V = [], [], []
    # diagonal blocks (lower part)
    for p in range(3):
        for q in range(p + 1):
            R.append(idx * 3 + p); C.append(idx * 3 + q); V.append(D[:, p, q])
    # off-diagonal blocks -K_e between node i (src) and j (nb)
    for o in range(len(offs)):
        e = edge[:, o]
        if not e.any():
            continue
        i = idx[e]; j = nb_all[e, o]
        blk = -c[e, o][:, None, None] * Kunit[o]
        hi_n = np.maximum(i, j); lo_n = np.minimum(i, j)
        for p in range(3):
            for q in range(3):
                R.append(hi_n * 3 + p); C.append(lo_n * 3 + q); V.append(blk[:, p, q])
    n = 3 * n_nodes
    colptr, rowind, vals = coo_to_lower_csc(n, np.concatenate(R), np.concatenate(C), np.concatenate(V))
    return Problem(n=n, colptr=colptr, rowind=rowind, values=vals, perm=nd_perm(dims, 3),
                   meta=dict(kind="elasticity_27pt", k=k, lo=lo, hi=hi, seed=seed))


def irregular_3d(k: int, keep: float = 0.35, seed: int = 12, lo: float = 0.1, hi: float = 10.0,
                 shift: float = 1e-2) -> Problem:
    """A Laplacian with irregular structure on a k^3 grid of nodes: every
    27-point edge is kept with probability `keep` (one uniform draw per edge,
    edge order as in elasticity_27pt), a kept edge gets a weight log-uniform in
    [lo, hi], A_ii = sum of incident weights + shift (SPD). The pattern has no
    geometric ordering: perm is the identity (order it with chol_order_nd)."""
    dims = (k, k, k)
    n = k ** 3
    idx, coords = _grid_coords(dims)
    offs = _offsets_27()
    pos = np.array([_is_positive(o) for o in offs])
    nb = np.stack([_offset_index(dims, coords, o) for o in offs], axis=1)
    cand = (nb >= 0) & pos[None, :]
    rng = SplitMix64(seed)
    m = int(cand.sum())
    u = rng.uniform(m)
    w = rng.log_uniform(m, lo, hi)
    ii = np.broadcast_to(idx[:, None], nb.shape)[cand]
    jj = nb[cand]
    kept = u < keep
    ii, jj, w = ii[kept], jj[kept], w[kept]
    diag = np.full(n, shift)
    np.add.at(diag, ii, w)
    np.add.at(diag, jj, w)
    R = np.concatenate([idx, np.maximum(ii, jj)])
    C = np.concatenate([idx, np.minimum(ii, jj)])
    V = np.concatenate([diag, -w])
    colptr, rowind, vals = coo_to_lower_csc(n, R, C, V)
    return Problem(n=n, colptr=colptr, rowind=rowind, values=vals, perm=np.arange(n, dtype=np.int32),
                   meta=dict(kind="irregular_3d", k=k, keep=keep, seed=seed))


def laplacian_2d_dirichlet_weighted(k: int, rng: SplitMix64, lo: float = 0.1, hi: float = 10.0) -> Problem:
    """5-point Laplacian with log-uniform edge weights and Dirichlet ghost edges.

    Edge order: node in natural order, then (axis 0, -1), (axis 0, +1),
    (axis 1, -1), (axis 1, +1); an in-grid neighbour is drawn from its +1 side
    only, an out-of-grid neighbour is a ghost that adds its weight to A_ii.
    A_ii = sum of incident weights (ghosts included).
    """
    dims = (k, k)
    n = k * k
    idx, coords = _grid_coords(dims)
    offs = [(-1, 0), (1, 0), (0, -1), (0, 1)]
    nb_all = np.stack([_offset_index(dims, coords, o) for o in offs], axis=1)
    pos = np.array([False, True, False, True])
    draw = (nb_all < 0) | pos[None, :]
    w = np.zeros(nb_all.shape)
    w[draw] = rng.log_uniform(int(draw.sum()), lo, hi)
    diag = np.zeros(n)
    edge = (nb_all >= 0) & pos[None, :]
    diag += (w * (nb_all < 0)).sum(axis=1)
    R, C, V = [idx], [idx], []
    for o in range(4):
        e = edge[:, o]
        if not e.any():
            continue
        i = nb_all[e, o]; j = idx[e]
        diag[j] += w[e, o]
        np.add.at(diag, i, w[e, o])
        R.append(i); C.append(j); V.append(-w[e, o])
    V.insert(0, diag)
    colptr, rowind, vals = coo_to_lower_csc(n, np.concatenate(R), np.concatenate(C), np.concatenate(V))
    return Problem(n=n, colptr=colptr, rowind=rowind, values=vals, perm=nd_perm(dims),
                   meta=dict(kind="laplacian_2d_dirichlet_weighted", k=k, lo=lo, hi=hi))


def laplacian_dirichlet_weighted(dims, rng: SplitMix64, lo: float, hi: float) -> Problem:
    """Grid Laplacian (2D 5-point / 3D 7-point) with log-uniform conductances in
    [lo, hi] and Dirichlet ghost edges: edge order node in natural order, then
    for axis 0..d-1 the (-1, +1) neighbours; an in-grid neighbour is drawn from
    its +1 side only, an out-of-grid neighbour is a ghost whose conductance
    goes to A_ii only. A_ii = sum of incident conductances (ghosts included)."""
    dims = tuple(int(d) for d in dims)
    d = len(dims)
    n = int(np.prod(dims))
    idx, coords = _grid_coords(dims)
    offs = []
    for a in range(d):
        for sgn in (-1, 1):
            o = [0] * d
            o[a] = sgn
            offs.append(tuple(o))
    nb_all = np.stack([_offset_index(dims, coords, o) for o in offs], axis=1)
    pos = np.array([o[a] > 0 for o in offs for a in [next(i for i in range(d) if o[i] != 0)]])
    draw = (nb_all < 0) | pos[None, :]
    w = np.zeros(nb_all.shape)
    w[draw] = rng.log_uniform(int(draw.sum()), lo, hi)
    diag = (w * (nb_all < 0)).sum(axis=1)
    edge = (nb_all >= 0) & pos[None, :]
    R, C, V = [idx], [idx], []
    for o in range(len(offs)):
        e = edge[:, o]
        if not e.any():
            continue
        i = nb_all[e, o]; j = idx[e]
        diag[j] += w[e, o]
        np.add.at(diag, i, w[e, o])
        R.append(i); C.append(j); V.append(-w[e, o])
    V.insert(0, diag)
    colptr, rowind, vals = coo_to_lower_csc(n, np.concatenate(R), np.concatenate(C), np.concatenate(V))
    return Problem(n=n, colptr=colptr, rowind=rowind, values=vals, perm=nd_perm(dims),
                   meta=dict(kind="laplacian_dirichlet_weighted", dims=dims, lo=lo, hi=hi))


def batch_2d(count: int = 2000, kmin: int = 16, kmax: int = 96, seed: int = 4):
    """Independent weighted 2D Laplacians; side k_s ~ U{kmin..kmax} drawn first."""
    rng = SplitMix64(seed)
    ks = kmin + np.floor(rng.uniform(count) * (kmax - kmin + 1)).astype(np.int64)
    return [laplacian_2d_dirichlet_weighted(int(k), rng) for k in ks]


def block_diagonal(problems) -> Problem:
    """Concatenate independent problems into one block-diagonal system (perm too)."""
    offs = np.cumsum([0] + [p.n for p in problems])
    n = int(offs[-1])
    colptr = [np.zeros(1, dtype=np.int64)]
    rowind, vals, perm = [], [], []
    base = 0
    for o, p in zip(offs[:-1], problems):
        colptr.append(p["colptr"][1:] + base)
        base += int(p["colptr"][-1])
        rowind.append(p["rowind"].astype(np.int64) + o)
        vals.append(p["values"])
        perm.append(p["perm"].astype(np.int64) + o)
    return Problem(n=n, colptr=np.concatenate(colptr), rowind=np.concatenate(rowind).astype(np.int32),
                   values=np.concatenate(vals), perm=np.concatenate(perm).astype(np.int32),
                   meta=dict(kind="block_diagonal", count=len(problems), offsets=offs))


def rhs_uniform(n: int, nrhs: int, seed: int) -> np.ndarray:
    """n x nrhs column-major (Fortran order) right-hand sides, U(-1, 1)."""
    u = SplitMix64(seed).uniform(n * nrhs)
    return np.asfortranarray((2.0 * u - 1.0).reshape(nrhs, n).T)


def rhs_normal(n: int, nrhs: int, seed: int) -> np.ndarray:
    """n x nrhs column-major N(0, 1) draws (Box-Muller)."""
    z = SplitMix64(seed).normal(n * nrhs)
    return np.asfortranarray(z.reshape(nrhs, n).T)


# The five named workloads (sizes fixed; seed = index + 1).
def workload(name: str) -> Problem:
    if name == "2d64":
        return laplacian_2d_dirichlet(64)
    if name == "3d64":
        return laplacian_neumann_varcoef((64, 64, 64), 1e-2, 1e2, 1e-6, seed=2)
    if name == "elast48":
        return elasticity_27pt(48, 1.0, 1e6, seed=3)
    if name == "3d48":
        # the differentiable-solve workload: Dirichlet-anchored (ghost edges), so
        # finite differences of log det and w^T x are well posed
        return laplacian_dirichlet_weighted((48, 48, 48), SplitMix64(5), 1e-2, 1e2)
    raise KeyError(name)
