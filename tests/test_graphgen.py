"""The seeded input generators (no method arithmetic): valid simple symmetric
CSR, determinism, and the intended size and shape of each workload."""
import numpy as np
import pytest

from paper_2112_06154_gb300 import graphgen as gg


def check_csr(rowptr, col):
    n = rowptr.size - 1
    assert rowptr[0] == 0 and rowptr[-1] == col.size
    assert (np.diff(rowptr) >= 0).all()
    src = np.repeat(np.arange(n), np.diff(rowptr))
    assert (src != col).all()  # no self loops
    for v in range(0, n, max(1, n // 50)):
        row = col[rowptr[v]:rowptr[v + 1]]
        assert (np.diff(row) > 0).all()  # sorted, no duplicates
    fwd = set(zip(src.tolist(), col.tolist()))
    assert all((b, a) in fwd for a, b in list(fwd)[:2000])  # symmetric


@pytest.mark.parametrize("make", [
    lambda s: gg.erdos_renyi(500, 2000, s),
    lambda s: gg.chung_lu(2000, 10, 2.5, 100, s),
    lambda s: gg.barabasi_albert(800, 3, s),
    lambda s: gg.grid(20, 30, 0.02, s),
    lambda s: gg.rmat(10, 8, 0.57, 0.19, 0.19, s),
    lambda s: gg.sbm_hierarchical(20000, s),
])
def test_generators_give_valid_deterministic_csr(make):
    a = make(5)
    b = make(5)
    check_csr(*a)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], b[1])


def test_sbm_hierarchical_edge_counts():
    # expected edges per block pair: pairs * 1e-6 i^2 (i <= j), block size n/10
    n = 100000
    rowptr, col = gg.sbm_hierarchical(n, 11)
    s = n // 10
    src = np.repeat(np.arange(n), np.diff(rowptr))
    upper = src < col
    bi, bj = src[upper] // s + 1, col[upper] // s + 1
    for i in (3, 7, 10):
        for j in (i, 10):
            pairs = s * (s - 1) // 2 if i == j else s * s
            mu = pairs * 1e-6 * i * i
            got = int(((bi == i) & (bj == j)).sum())
            assert abs(got - mu) < 5 * np.sqrt(mu) + 2, (i, j, got, mu)
    # no pair (i, j) with i > j exists by construction of the block order
    assert (bi <= bj).all()
