"""The peel's compaction: each time the alive node count halves, the peel
switches to a CSR of the alive nodes' alive neighbours and to a list of those
nodes (node ids unchanged).  Forced on at every size here, the exact and
sampled peels (ExactCore, Sec. 2; Core, Alg. 4), EstDense's replay (Alg. 7)
and a batch must give the oracle's core maps and removal rounds bit for bit,
and the same results as with compaction off."""
import numpy as np
import pytest

import oracle as O
from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import khcore as K

pytestmark = pytest.mark.gpu

GRAPHS = {
    "er": lambda: gg.erdos_renyi(2000, 8000, 1001),
    "ragged": lambda: gg.chung_lu(1037, 6, 2.2, 120, 7),
    "hubs": lambda: gg.with_hubs(12000, (9000, 5000), 77),
    "grid": lambda: gg.grid(40, 50, 0.01, 57),
}


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    K.load(build_if_missing=True)
    c = K.kh_ctx_create(0)
    yield c
    c.close()


def peel(ctx, rp, cl, h, M, sampled, mode):
    G = K.kh_graph_load_csr(ctx, rp, cl)
    try:
        K.kh_set_h(G, h)
        K.kh_set_sampling(G, seed=1, M=M)
        K.kh_set_variant(G, mode, op=K.KH_OP_PEEL_COMPACT)
        assert K.kh_get_variant(G, op=K.KH_OP_PEEL_COMPACT)[0] == mode
        core = K.kh_core_sampled(G) if sampled else K.kh_core_exact(G)
        ro, rounds, _ = K.kh_peel_info(G)
        # the graph's own CSR is back after the peel: a full pass still matches
        deg = K.kh_hdegree_exact(G)
        return core, ro, rounds, deg
    finally:
        G.close()


# (the oracle's exact peel of the hub graph at h = 3 takes too long for a test)
EXACT_CASES = [(g, h) for g in sorted(GRAPHS) for h in (1, 2, 3) if (g, h) != ("hubs", 3)]
SAMPLED_CASES = [(g, h, M) for g in sorted(GRAPHS) for h, M in ((2, 16), (3, 24), (4, 9), (2, 535))
                 if (g, h, M) != ("hubs", 2, 535)]


@pytest.mark.parametrize("name,h", EXACT_CASES)
def test_exact_peel_with_compaction(ctx, name, h):
    rp, cl = GRAPHS[name]()
    want, wround, steps = O.core_exact(rp, cl, h)
    core, ro, rounds, deg = peel(ctx, rp, cl, h, 16, False, K.KH_COMPACT_ALWAYS)
    assert np.array_equal(core, want) and np.array_equal(ro, wround) and rounds == steps
    assert np.array_equal(deg, O.hdegree_exact(rp, cl, h))


@pytest.mark.parametrize("name,h,M", SAMPLED_CASES)
def test_sampled_peel_with_compaction(ctx, name, h, M):
    rp, cl = GRAPHS[name]()
    r = O.ranks(rp.size - 1, 1)
    want, wround, steps = O.core_sampled(rp, cl, r, h, M)
    core, ro, rounds, _ = peel(ctx, rp, cl, h, M, True, K.KH_COMPACT_ALWAYS)
    assert np.array_equal(core, want) and np.array_equal(ro, wround) and rounds == steps
    off = peel(ctx, rp, cl, h, M, True, K.KH_COMPACT_OFF)
    assert np.array_equal(off[0], core) and np.array_equal(off[1], ro)


@pytest.mark.parametrize("exact", [True, False])
def test_dense_replay_with_compaction(ctx, exact):
    rp, cl = GRAPHS["hubs"]()
    n = rp.size - 1
    _, rnd, _ = O.core_exact(rp, cl, 2) if exact else O.core_sampled(rp, cl, O.ranks(n, 1), 2, 16)
    rounds = int(rnd.max()) + 1
    want_sum, want_size = O.dense_curve(rp, cl, O.ranks(n, 3), 2, 16, exact, rnd, rounds)
    G = K.kh_graph_load_csr(ctx, rp, cl)
    try:
        K.kh_set_h(G, 2)
        K.kh_set_sampling(G, seed=3, M=16)
        K.kh_set_variant(G, K.KH_COMPACT_ALWAYS, op=K.KH_OP_PEEL_COMPACT)
        got_sum, got_size, _ = K.kh_dense(G, exact, rnd, rounds)
    finally:
        G.close()
    assert np.array_equal(got_sum, want_sum) and np.array_equal(got_size, want_size)


def test_batch_with_compaction(ctx):
    graphs = [gg.barabasi_albert(n, m, 900 + i) for i, (n, m) in
              enumerate([(3000, 3), (500, 5), (1200, 4), (40, 3)])]
    hs = np.array([2, 3, 2, 4], np.int32)
    vo, rp, cl = gg.pack_batch(graphs)
    B = K.kh_graph_load_batch(ctx, vo, rp, cl, hs)
    try:
        K.kh_set_variant(B, K.KH_COMPACT_ALWAYS, op=K.KH_OP_PEEL_COMPACT)
        core = K.kh_core_sampled(B)
        ecore = None
        K.kh_set_h(B, 2)
        ecore = K.kh_core_exact(B)
    finally:
        B.close()
    for q, (grp, gcl) in enumerate(graphs):
        a, b = int(vo[q]), int(vo[q + 1])
        n = b - a
        M = O.budget_M(n, 0.5, 0.05)
        want, _, _ = O.core_sampled(grp, gcl, O.ranks(n, 1), int(hs[q]), M)
        assert np.array_equal(core[a:b], want), q
        assert np.array_equal(ecore[a:b], O.core_exact(grp, gcl, 2)[0]), q
