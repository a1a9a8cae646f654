"""EstDense (Alg. 7) on the GPU against the oracle: along a removal order, the
sum of d(v; X) over every candidate set X (deg_h or the estimate, all values
current for X), bit for bit.  The removal orders come from the oracle's own
peels, or are random permutations (one node per round: the paper's n
candidates)."""
from fractions import Fraction

import numpy as np
import pytest

import oracle as O
from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import khcore as K

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    K.load(build_if_missing=True)
    c = K.kh_ctx_create(0)
    yield c
    c.close()


def densest(total, size):
    best, val = -1, None
    for q in range(total.size):
        if size[q] == 0:
            continue
        f = Fraction(int(total[q]), int(size[q]))
        if val is None or f > val:
            best, val = q, f
    return best


def run_case(ctx, rowptr, col, h, M, exact, order, rounds, seed=7):
    n = rowptr.size - 1
    want_sum, want_size = O.dense_curve(rowptr, col, O.ranks(n, seed), h, M, exact, order, rounds)
    G = K.kh_graph_load_csr(ctx, rowptr, col)
    try:
        K.kh_set_h(G, h)
        K.kh_set_sampling(G, seed=seed, M=M)
        got_sum, got_size, best = K.kh_dense(G, exact, order, rounds)
        ro, replay_rounds, _ = K.kh_peel_info(G, True)
    finally:
        G.close()
    assert np.array_equal(got_size, want_size)
    assert np.array_equal(got_sum, want_sum)
    assert best == densest(want_sum, want_size)
    # the replay removed every node in its scheduled round
    assert np.array_equal(ro, order) and replay_rounds <= rounds
    return got_sum, got_size


GRAPHS = {
    "er2000": lambda: gg.erdos_renyi(2000, 8000, 1001),
    "cl1200": lambda: gg.chung_lu(1200, 10, 2.5, 120, 55),
    "ba1000": lambda: gg.barabasi_albert(1000, 4, 56),
    "grid": lambda: gg.grid(30, 40, 0.01, 57),
}


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("h", [1, 2, 3])
def test_dense_exact_along_exact_core(ctx, name, h):
    rowptr, col = GRAPHS[name]()
    _, rnd, _ = O.core_exact(rowptr, col, h)
    total, size = run_case(ctx, rowptr, col, h, 16, True, rnd, int(rnd.max()) + 1)
    # Sec. 6's identity: the whole graph's sum is twice its h-edge count, so
    # for h = 1 it is the number of adjacency entries
    if h == 1:
        assert total[0] == col.size


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("h,M", [(2, 16), (3, 24), (2, 535)])
def test_dense_sampled_along_sampled_core(ctx, name, h, M):
    rowptr, col = GRAPHS[name]()
    n = rowptr.size - 1
    _, rnd, _ = O.core_sampled(rowptr, col, O.ranks(n, 1), h, M)
    run_case(ctx, rowptr, col, h, M, False, rnd, int(rnd.max()) + 1)


@pytest.mark.parametrize("exact", [True, False])
def test_dense_one_node_per_round(ctx, exact):
    rowptr, col = gg.chung_lu(300, 8, 2.5, 60, 58)
    n = rowptr.size - 1
    order = np.random.default_rng(59).permutation(n).astype(np.int32)
    total, size = run_case(ctx, rowptr, col, 2, 12, exact, order, n)
    assert np.array_equal(size, np.arange(n, 0, -1))


def test_dense_rejects_bad_input(ctx):
    rowptr, col = gg.erdos_renyi(50, 100, 60)
    G = K.kh_graph_load_csr(ctx, rowptr, col)
    try:
        with pytest.raises(K.KhError):
            K.kh_dense(G, True, np.full(50, 4, np.int32), 3)
        with pytest.raises(K.KhError):
            K.kh_dense(G, True, np.zeros(50, np.int32), 0)
        # the context stays usable
        total, size, best = K.kh_dense(G, True, np.zeros(50, np.int32), 1)
        assert size[0] == 50 and best == 0
    finally:
        G.close()


@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("h,M,eps", [(2, 16, 0.5), (3, 24, 0.3), (2, 535, 0.5)])
def test_dense_pruned_along_sampled_core(ctx, name, h, M, eps):
    """The faster EstDense variant of Sec. 6 (nodes with c' < gamma k' removed
    first): sums, sizes, kept mask and the densest round equal the oracle's,
    exact and sampled, along the sampled core's order."""
    rowptr, col = GRAPHS[name]()
    n = rowptr.size - 1
    core, rnd, _ = O.core_sampled(rowptr, col, O.ranks(n, 1), h, M)
    rounds = int(rnd.max()) + 1
    for exact in (True, False):
        want_sum, want_size, want_keep = O.dense_curve_pruned(
            rowptr, col, O.ranks(n, 7), h, M, exact, rnd, rounds, core, eps)
        G = K.kh_graph_load_csr(ctx, rowptr, col)
        try:
            K.kh_set_h(G, h)
            K.kh_set_sampling(G, seed=7, M=M)
            got_sum, got_size, best, kept = K.kh_dense_pruned(G, exact, rnd, rounds, core, eps)
            ro, _, _ = K.kh_peel_info(G, True)
        finally:
            G.close()
        assert np.array_equal(kept, want_keep)
        assert np.array_equal(got_size, want_size)
        assert np.array_equal(got_sum, want_sum)
        assert best == densest(want_sum, want_size)
        assert (ro[kept == 0] == -1).all() and np.array_equal(ro[kept == 1], rnd[kept == 1])
