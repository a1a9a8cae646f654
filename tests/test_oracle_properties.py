"""Property-based checks of the oracle on random small graphs (hypothesis):
the invariants the paper fixes must hold on every graph, not only on the
fixed seeds of the pin tests."""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings, strategies as st  # noqa: E402

import oracle as O  # noqa: E402
from paper_2112_06154_gb300 import graphgen as gg  # noqa: E402


@st.composite
def small_graphs(draw):
    n = draw(st.integers(min_value=1, max_value=24))
    pairs = n * (n - 1) // 2
    m = draw(st.integers(min_value=0, max_value=min(pairs, 3 * n)))
    seed = draw(st.integers(min_value=0, max_value=10**6))
    if m == 0:
        return gg.csr_from_edges(n, np.empty(0, np.int64), np.empty(0, np.int64))
    return gg.erdos_renyi(n, m, seed)


SETTINGS = settings(max_examples=60, deadline=None)


@SETTINGS
@given(g=small_graphs(), h=st.integers(1, 3))
def test_hdegree_monotone_in_h_and_bounded(g, h):
    rowptr, col = g
    n = rowptr.size - 1
    a = O.hdegree_exact(rowptr, col, h)
    b = O.hdegree_exact(rowptr, col, h + 1)
    assert (a <= b).all() and (b <= max(n - 1, 0)).all()
    assert (O.hdegree_exact(rowptr, col, 1) == np.diff(rowptr)).all()


@SETTINGS
@given(g=small_graphs(), h=st.integers(1, 3), M=st.integers(1, 12), seed=st.integers(0, 99))
def test_bucket_peel_equals_sequential_and_prop44(g, h, M, seed):
    # R6: the bucket rounds give the sequential peel's core map (monotone d);
    # Prop. 4.4's second claim: min(c', M) = min(c, M)
    rowptr, col = g
    n = rowptr.size - 1
    r = O.ranks(n, seed)
    cb, _, _ = O.core_sampled(rowptr, col, r, h, M)
    cs, _, _ = O.core_sampled(rowptr, col, r, h, M, O.SEQUENTIAL)
    assert np.array_equal(cb, cs)
    ce, _, _ = O.core_exact(rowptr, col, h)
    ces, _, _ = O.core_exact(rowptr, col, h, O.SEQUENTIAL)
    assert np.array_equal(ce, ces)
    assert np.array_equal(np.minimum(cb.astype(np.int64), M), np.minimum(ce.astype(np.int64), M))


@SETTINGS
@given(g=small_graphs(), h=st.integers(1, 3), M=st.integers(1, 12), seed=st.integers(0, 99))
def test_estimate_definition_equals_level_recursion(g, h, M, seed):
    # Prop. 3.1 / Alg. 2 against Def. 4.1 on the ball, v first
    rowptr, col = g
    n = rowptr.size - 1
    r = O.ranks(n, seed)
    e1, k1, b1 = O.estimate_def(rowptr, col, r, h, M)
    e2, k2, b2 = O.estimate_dp(rowptr, col, r, h, M)
    assert np.array_equal(e1, e2) and np.array_equal(k1, k2) and np.array_equal(b1, b2)


@SETTINGS
@given(g=small_graphs(), h=st.integers(1, 3))
def test_dense_curve_identity(g, h):
    # Sec. 6: sum_v deg_h(v; X) = 2 |E_h(X)| on every candidate set of the exact peel
    rowptr, col = g
    n = rowptr.size - 1
    _, rnd, _ = O.core_exact(rowptr, col, h)
    rounds = int(rnd.max()) + 1 if n else 1
    total, size = O.dense_curve(rowptr, col, O.ranks(n, 1), h, 4, True, rnd, rounds)
    for q in range(rounds):
        alive = rnd >= q
        deg = O.hdegree_exact(rowptr, col, h, alive=alive)
        assert total[q] == int(deg[alive].sum()) and total[q] % 2 == 0
        assert size[q] == int(alive.sum())
