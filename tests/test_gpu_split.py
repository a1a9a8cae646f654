"""Nodes of more than 4096 neighbours: the level-union kernel splits them into
parts of 2048 neighbours whose trimmed partial sets are merged (exact by the
monotonicity of the trim level, Prop. 3.1).  Estimates (Alg. 1 after Alg. 2's
levels) and sampled cores (Alg. 4) on graphs with such hubs must equal the
oracle's bit for bit, including the lists' levels and sizes."""
import numpy as np
import pytest

import oracle as O
from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import khcore as K

pytestmark = pytest.mark.gpu
HUBS = (9000, 6000, 4500, 4100, 8193)


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    K.load(build_if_missing=True)
    c = K.kh_ctx_create(0)
    yield c
    c.close()


@pytest.fixture(scope="module")
def hub_graph():
    rp, cl = gg.with_hubs(12000, HUBS, 77)
    assert (np.diff(rp) > 4096).sum() == len(HUBS)
    return rp, cl


@pytest.mark.parametrize("h,M", [(2, 24), (3, 16), (4, 9), (2, 535), (3, 535)])
def test_split_estimates(ctx, hub_graph, h, M):
    rp, cl = hub_graph
    r = O.ranks(rp.size - 1, 1)
    want = O.estimate_dp(rp, cl, r, h, M)
    G = K.kh_graph_load_csr(ctx, rp, cl)
    try:
        K.kh_set_h(G, h)
        K.kh_set_sampling(G, seed=1, M=M)
        for _ in range(2):  # twice: the part counters are ready again after a pass
            got = K.kh_estimate(G)
            for x, y in zip(got, want):
                assert np.array_equal(x, y)
    finally:
        G.close()


@pytest.mark.parametrize("h,M", [(2, 24), (3, 16)])
def test_split_sampled_core(ctx, hub_graph, h, M):
    rp, cl = hub_graph
    r = O.ranks(rp.size - 1, 1)
    want, wround, steps = O.core_sampled(rp, cl, r, h, M)
    G = K.kh_graph_load_csr(ctx, rp, cl)
    try:
        K.kh_set_h(G, h)
        K.kh_set_sampling(G, seed=1, M=M)
        core = K.kh_core_sampled(G)
        ro, rounds, _ = K.kh_peel_info(G)
        assert np.array_equal(core, want)
        assert np.array_equal(ro, wround) and rounds == steps
    finally:
        G.close()
