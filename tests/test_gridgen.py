"""Synthetic input generators: PRNG test vector, sizes, and the ND property."""
import numpy as np
import pytest

import gridgen


def test_splitmix64_reference_values():
    # SplitMix64 from state 0 (Steele, Lea, Flood 2014; Vigna's splitmix64.c)
    z = gridgen.SplitMix64(0).next_u64(3)
    assert [int(v) for v in z] == [0xE220A8397B1DCDAF, 0x6E789E6AA1B965F4, 0x06C45D188009454F]
    r = gridgen.SplitMix64(0)
    a = r.next_u64(2)
    b = r.next_u64(1)
    assert int(b[0]) == 0x06C45D188009454F      # stream continues across calls


def test_uniform_and_normal_ranges():
    u = gridgen.SplitMix64(5).uniform(10000)
    assert u.min() >= 0 and u.max() < 1 and abs(u.mean() - 0.5) < 0.02
    z = gridgen.SplitMix64(5).normal(20001)
    assert abs(z.mean()) < 0.03 and abs(z.std() - 1) < 0.03 and z.size == 20001


@pytest.mark.parametrize("dims", [(5, 5), (7, 3), (6, 5, 4), (1, 9), (3, 3, 3)])
def test_nd_order_is_permutation_with_separators(dims):
    order = gridgen.nd_order(dims)
    assert sorted(order.tolist()) == list(range(int(np.prod(dims))))


def test_nd_separator_property_2d():
    """The last block emitted for the whole box is the middle plane of the
    longest axis, and removing it disconnects the low and high halves."""
    k = 9
    order = gridgen.nd_order((k, k))
    sep = set(order[-k:].tolist())
    assert sep == {4 + k * y for y in range(k)}       # x = mid plane (axis 0, tie -> lowest)
    low = set(order[: (k * k - k) // 2].tolist())
    assert all((i % k) < 4 for i in low)


def test_workload_sizes():
    p = gridgen.workload("2d64")
    assert p.n == 4096 and int(p["colptr"][-1]) == 12160
    p = gridgen.laplacian_neumann_varcoef((8, 8, 8), 1e-2, 1e2, 1e-6, seed=2)
    # 7-point: n diagonal + 3*k^2*(k-1) edges
    assert int(p["colptr"][-1]) == 512 + 3 * 64 * 7
    e = gridgen.elasticity_27pt(4)
    A = np.zeros((e.n, e.n))
    for j in range(e.n):
        for t in range(e["colptr"][j], e["colptr"][j + 1]):
            A[e["rowind"][t], j] = A[j, e["rowind"][t]] = e["values"][t]
    assert np.linalg.eigvalsh(A).min() > 0          # SPD by construction


def test_batch_block_diagonal():
    probs = gridgen.batch_2d(count=5, kmin=3, kmax=6, seed=4)
    bd = gridgen.block_diagonal(probs)
    assert bd.n == sum(p.n for p in probs)
    assert sorted(bd["perm"].tolist()) == list(range(bd.n))
    assert all(3 <= p["meta"]["k"] <= 6 for p in probs)


def test_dirichlet_weighted_3d_is_spd_and_sized():
    p = gridgen.laplacian_dirichlet_weighted((4, 3, 5), gridgen.SplitMix64(1), 1e-2, 1e2)
    A = np.zeros((p.n, p.n))
    for j in range(p.n):
        for t in range(p["colptr"][j], p["colptr"][j + 1]):
            A[p["rowind"][t], j] = A[j, p["rowind"][t]] = p["values"][t]
    assert np.linalg.eigvalsh(A).min() > 0
    # 7-point: n diagonals + edges along each axis
    edges = (3 * 3 * 5) + (4 * 2 * 5) + (4 * 3 * 4)
    assert int(p["colptr"][-1]) == p.n + edges
    # row sums equal the ghost conductances (>= 0), strictly positive on the boundary
    rs = A.sum(axis=1)
    assert np.all(rs >= -1e-12) and rs[0] > 0
