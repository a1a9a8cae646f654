"""GPU parity: the CUDA library (through the C ABI) against the CPU oracle.

All comparisons are bit-exact: every quantity of the path is an integer
(ranks, h-degrees, counts, levels, list sizes, estimates, core numbers).
"""
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


def load(ctx, g, h=2, seed=1, M=0):
    rp, cl = g
    G = K.kh_graph_load_csr(ctx, rp, cl)
    K.kh_set_h(G, h)
    K.kh_set_sampling(G, seed=seed, M=M)
    return G


ER = gg.erdos_renyi(2000, 8000, 1001)           # the small G(n=2000, m=8000) workload
CL20K = gg.chung_lu(20000, 20, 2.5, 500, 1102)   # Chung-Lu shaped like the 200k case, scaled down
RAGGED = gg.chung_lu(1037, 6, 2.2, 120, 7)       # n not a multiple of 32, isolated nodes


def test_ranks_match_oracle(ctx):
    for seed in [1, 7, 2**40 + 3]:
        G = load(ctx, ER, seed=seed)
        assert (K.kh_ranks(G) == O.ranks(2000, seed)).all()
        G.close()
    rp, cl = gg.grid(300, 400)
    G = load(ctx, (rp, cl), seed=5)
    assert (K.kh_ranks(G) == O.ranks(120000, 5)).all()
    G.close()


@pytest.mark.parametrize("h", [1, 2, 3, 4])
@pytest.mark.parametrize("graph", ["er", "ragged", "cl20k"])
def test_hdegree_exact(ctx, h, graph):
    g = {"er": ER, "ragged": RAGGED, "cl20k": CL20K}[graph]
    if graph == "cl20k" and h == 4:
        pytest.skip("oracle too slow")
    G = load(ctx, g, h=h)
    assert (K.kh_hdegree_exact(G) == O.hdegree_exact(*g, h)).all()
    G.close()


def test_hdegree_closed_forms(ctx):
    for g, h, want in [(gg.complete(40), 2, 39), (gg.cycle(101), 3, 6), (gg.star(300), 2, 300)]:
        G = load(ctx, g, h=h)
        assert (K.kh_hdegree_exact(G) == want).all()
        G.close()


def test_sampled_counts(ctx):
    for g, h in [(ER, 2), (RAGGED, 3), (CL20K, 2)]:
        G = load(ctx, g, h=h, seed=1)
        r = O.ranks(g[0].size - 1, 1)
        got = K.kh_sampled_counts(G, 0, 10)
        assert (got == O.fixed_counts(*g, r, h, 0, 10)).all()
        got = K.kh_sampled_counts(G, 3, 5)
        assert (got == O.fixed_counts(*g, r, h, 3, 5)).all()
        G.close()


@pytest.mark.parametrize("h", [1, 2, 3, 4])
@pytest.mark.parametrize("M", [1, 7, 16, 535])
def test_estimate_er(ctx, h, M):
    G = load(ctx, ER, h=h, M=M)
    est, lvl, bs = K.kh_estimate(G)
    r = O.ranks(2000, 1)
    we, wl, wb = O.estimate_dp(*ER, r, h, M)
    assert (lvl == wl).all()
    assert (bs == wb).all()
    assert (est == we).all()
    G.close()


@pytest.mark.parametrize("h", [2, 3])
def test_estimate_cl20k_default_budget(ctx, h):
    G = load(ctx, CL20K, h=h)
    M = K.kh_get_M(G)
    assert M == O.budget_M(20000, 0.5, 0.05)
    est, lvl, bs = K.kh_estimate(G)
    r = O.ranks(20000, 1)
    we, wl, wb = O.estimate_dp(*CL20K, r, h, M)
    assert (lvl == wl).all() and (bs == wb).all() and (est == we).all()
    G.close()


def test_estimate_small_budget_many_levels(ctx):
    G = load(ctx, CL20K, h=3, M=24)
    est, lvl, bs = K.kh_estimate(G)
    r = O.ranks(20000, 1)
    we, wl, wb = O.estimate_dp(*CL20K, r, 3, 24)
    assert (lvl == wl).all() and (bs == wb).all() and (est == we).all()
    G.close()


@pytest.mark.parametrize("h", [1, 2, 3])
@pytest.mark.parametrize("graph", ["er", "ragged"])
def test_core_exact(ctx, h, graph):
    g = {"er": ER, "ragged": RAGGED}[graph]
    G = load(ctx, g, h=h)
    core = K.kh_core_exact(G)
    want, wround, steps = O.core_exact(*g, h)
    assert (core == want).all()
    ro, rounds, updates = K.kh_peel_info(G)
    assert rounds == steps
    assert (ro == wround).all()
    G.close()


@pytest.mark.parametrize("h,M", [(1, 4), (2, 16), (3, 16), (2, 535), (4, 9)])
def test_core_sampled_er(ctx, h, M):
    G = load(ctx, ER, h=h, M=M)
    core = K.kh_core_sampled(G)
    r = O.ranks(2000, 1)
    want, wround, steps = O.core_sampled(*ER, r, h, M)
    assert (core == want).all()
    ro, rounds, _ = K.kh_peel_info(G)
    assert rounds == steps and (ro == wround).all()
    G.close()


@pytest.mark.parametrize("h", [2, 3])
def test_core_sampled_cl20k(ctx, h):
    G = load(ctx, CL20K, h=h, M=40)
    core = K.kh_core_sampled(G)
    r = O.ranks(20000, 1)
    want, _, _ = O.core_sampled(*CL20K, r, h, 40)
    assert (core == want).all()
    G.close()


def test_core_exact_cl20k_h2(ctx):
    G = load(ctx, CL20K, h=2)
    core = K.kh_core_exact(G)
    want, _, _ = O.core_exact(*CL20K, 2)
    assert (core == want).all()
    G.close()


def test_degenerate_graphs(ctx):
    # single node, two isolated nodes, one edge
    for rp, cl in [(np.array([0, 0]), np.array([], np.int32)),
                   (np.array([0, 0, 0]), np.array([], np.int32)),
                   (np.array([0, 1, 2]), np.array([1, 0], np.int32))]:
        G = load(ctx, (rp, cl), h=2, M=1)
        n = rp.size - 1
        assert (K.kh_hdegree_exact(G) == O.hdegree_exact(rp, cl, 2)).all()
        assert (K.kh_core_exact(G) == O.core_exact(rp, cl, 2)[0]).all()
        r = O.ranks(n, 1)
        assert (K.kh_core_sampled(G) == O.core_sampled(rp, cl, r, 2, 1)[0]).all()
        G.close()


def test_invalid_graphs_rejected_and_context_survives(ctx):
    bad = [
        (np.array([0, 1, 1]), np.array([1], np.int32)),          # missing reverse edge
        (np.array([0, 1, 2]), np.array([0, 1], np.int32)),       # self-loops
        (np.array([0, 2, 3, 4]), np.array([2, 1, 0, 0], np.int32)),  # unsorted row
        (np.array([0, 1, 2]), np.array([5, 0], np.int32)),       # id out of range
    ]
    for rp, cl in bad:
        with pytest.raises(K.KhError) as ei:
            K.kh_graph_load_csr(ctx, rp, cl)
        assert ei.value.code == K.KH_EGRAPH
    G = load(ctx, ER, h=2)
    assert (K.kh_hdegree_exact(G) == O.hdegree_exact(*ER, 2)).all()
    G.close()


def test_device_pointers_and_determinism(ctx):
    import torch
    rp, cl = CL20K
    G = K.kh_graph_load_csr(ctx, torch.from_numpy(rp).cuda(), torch.from_numpy(cl).cuda())
    K.kh_set_h(G, 2)
    K.kh_set_sampling(G, seed=1, M=40)
    out = torch.zeros(20000, dtype=torch.int64, device="cuda")
    K.kh_core_sampled(G, out)
    K.kh_sync(G)
    a = out.cpu().numpy().astype(np.uint64)
    b = K.kh_core_sampled(G)
    assert (a == b).all()
    deg = torch.zeros(20000, dtype=torch.int32, device="cuda")
    K.kh_hdegree_exact(G, deg)
    K.kh_sync(G)
    assert (deg.cpu().numpy() == O.hdegree_exact(rp, cl, 2)).all()
    G.close()


def test_parameter_errors(ctx):
    G = load(ctx, ER)
    for bad in [0, 17, -1]:
        with pytest.raises(K.KhError):
            K.kh_set_h(G, bad)
    with pytest.raises(K.KhError):
        K.kh_set_sampling(G, seed=1, M=20000)
    with pytest.raises(K.KhError):
        K.kh_set_sampling(G, seed=1, M=0, eps=0.0)
    with pytest.raises(K.KhError):
        K.kh_sampled_counts(G, 5, 2)
    G.close()


def test_profiled_rounds_match_graph_rounds(ctx):
    """Profiling launches rounds one by one; results must equal graph replay."""
    for sampled in (False, True):
        G = load(ctx, CL20K, h=2, M=40)
        fn = K.kh_core_sampled if sampled else K.kh_core_exact
        a = fn(G)
        _, ra, ua = K.kh_peel_info(G, False)
        K.kh_prof_enable(G, True)
        b = fn(G)
        _, rb, ub = K.kh_peel_info(G, False)
        assert (a == b).all() and ra == rb
        total_ms = 0.0
        for kind in range(K.KH_PROF_KINDS):
            ms, n, byt = K.kh_prof_read(G, kind)
            assert ms >= 0 and n >= 0 and byt >= 0
            total_ms += ms
        assert total_ms > 0
        bfs = K.kh_prof_read(G, K.KH_PROF_BFS)
        lvl = K.kh_prof_read(G, K.KH_PROF_LEVELU)
        assert (bfs[1] > 0) != sampled and (lvl[1] > 0) == sampled
        K.kh_prof_enable(G, False)
        G.close()


FAMILIES = {
    "ba": gg.barabasi_albert(1500, 4, 31),
    "grid_shortcuts": gg.grid(50, 60, 0.01, 32),
    "cl_dense": gg.chung_lu(1200, 25, 2.1, 300, 33),
    "rmat": gg.rmat(11, 8, 0.57, 0.19, 0.19, 34),
}


@pytest.mark.parametrize("family", sorted(FAMILIES))
@pytest.mark.parametrize("h", [2, 3])
def test_core_exact_families(ctx, family, h):
    g = FAMILIES[family]
    G = load(ctx, g, h=h)
    core = K.kh_core_exact(G)
    want, wround, steps = O.core_exact(*g, h)
    assert (core == want).all()
    ro, rounds, _ = K.kh_peel_info(G)
    assert rounds == steps and (ro == wround).all()
    G.close()


@pytest.mark.parametrize("family", sorted(FAMILIES))
@pytest.mark.parametrize("h,M", [(2, 20), (3, 12), (4, 30)])
def test_core_sampled_families(ctx, family, h, M):
    g = FAMILIES[family]
    n = g[0].size - 1
    G = load(ctx, g, h=h, M=M)
    core = K.kh_core_sampled(G)
    r = O.ranks(n, 1)
    want, wround, steps = O.core_sampled(*g, r, h, M)
    assert (core == want).all()
    ro, rounds, _ = K.kh_peel_info(G)
    assert rounds == steps and (ro == wround).all()
    G.close()


def _sparse_big():
    """n = 1,000,000 nodes (above the 819,200-node shared-memory bitmap limit,
    so the BFS keeps its visited set in global memory): a Chung-Lu component
    on the first 30,000 ids, the rest isolated."""
    rp0, cl0 = gg.chung_lu(30000, 12, 2.4, 400, 41)
    n = 1_000_000
    rp = np.concatenate([rp0, np.full(n - 30000, rp0[-1], dtype=np.int64)])
    return rp, cl0


def test_global_bitmap_bfs_and_peels(ctx):
    rp, cl = _sparse_big()
    for h in (2, 3):
        G = load(ctx, (rp, cl), h=h, M=30)
        deg = K.kh_hdegree_exact(G)
        want = O.hdegree_exact(rp, cl, h)
        assert (deg == want).all()
        cnt = K.kh_sampled_counts(G, 0, 4)
        r = O.ranks(rp.size - 1, 1)
        assert (cnt[:30000] == O.fixed_counts(rp[:30001], cl, r[:30000], h, 0, 4)).all()
        assert (cnt[30000:] == 0).all()
        if h == 2:
            core = K.kh_core_exact(G)
            assert (core[:30000] == O.core_exact(rp[:30001], cl, 2)[0]).all()
            assert (core[30000:] == 0).all()
        G.close()
