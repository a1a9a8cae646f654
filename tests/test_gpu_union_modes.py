"""The schedules of the level >= 2 union (Alg. 2 with Alg. 5's trim):
barrier-separated steps, free-running warps, and free-running lane groups
(sized by the keys a list is expected to give, or an eighth of them).  All
must give the oracle's
estimates (levels and |B|) and sampled cores bit for bit, including split hubs,
small M (many trims and compactions) and refines that stop early."""
import numpy as np
import pytest

import oracle as O
from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import khcore as K

pytestmark = pytest.mark.gpu

GRAPHS = {
    "er": lambda: gg.erdos_renyi(2000, 8000, 1001),
    "cl20k": lambda: gg.chung_lu(20000, 20, 2.5, 500, 1102),
    "hubs": lambda: gg.with_hubs(12000, (9000, 6000, 4500), 77),
    "rmat12": lambda: gg.rmat(12, 16, 0.57, 0.19, 0.19, 5),
}
MODES = {"stepped": (K.KH_LEVELU_STEPPED, 0), "free": (K.KH_LEVELU_FREE, 0),
         "grouped": (K.KH_LEVELU_GROUPED, 0), "grouped8": (K.KH_LEVELU_GROUPED, 8)}


@pytest.fixture(scope="module")
def ctx():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    K.load(build_if_missing=True)
    c = K.kh_ctx_create(0)
    yield c
    c.close()


def graph(ctx, name, h, M, mode):
    rp, cl = GRAPHS[name]()
    G = K.kh_graph_load_csr(ctx, rp, cl)
    K.kh_set_h(G, h)
    K.kh_set_sampling(G, seed=1, M=M)
    K.kh_set_variant(G, MODES[mode][0], MODES[mode][1], op=K.KH_OP_LEVEL_UNION)
    return rp, cl, G


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("name", sorted(GRAPHS))
@pytest.mark.parametrize("h,M", [(2, 7), (3, 16), (4, 24), (3, 535)])
def test_estimates_per_union_schedule(ctx, mode, name, h, M):
    rp, cl, G = graph(ctx, name, h, M, mode)
    try:
        want = O.estimate_dp(rp, cl, O.ranks(rp.size - 1, 1), h, M)
        got = K.kh_estimate(G)
        for x, y in zip(got, want):
            assert np.array_equal(x, y)
    finally:
        G.close()


@pytest.mark.parametrize("mode", sorted(MODES))
@pytest.mark.parametrize("name,h,M", [("er", 2, 16), ("cl20k", 3, 24), ("hubs", 2, 24),
                                      ("hubs", 3, 16), ("rmat12", 3, 9)])
def test_cores_per_union_schedule(ctx, mode, name, h, M):
    rp, cl, G = graph(ctx, name, h, M, mode)
    try:
        want, wround, steps = O.core_sampled(rp, cl, O.ranks(rp.size - 1, 1), h, M)
        core = K.kh_core_sampled(G)
        ro, rounds, _ = K.kh_peel_info(G)
        assert np.array_equal(core, want) and np.array_equal(ro, wround) and rounds == steps
    finally:
        G.close()


@pytest.mark.parametrize("mode", ["stepped", "grouped"])
def test_largest_M_fits_and_matches(ctx, mode):
    # M = 12000 (the library's largest): the hash set takes 2^15 slots and
    # the kernel's shared memory must still fit; the 2-balls of the hubs of
    # this graph exceed M, so the union trims and compacts
    rp, cl, G = graph(ctx, "cl20k", 2, 12000, mode)
    try:
        want = O.estimate_dp(rp, cl, O.ranks(rp.size - 1, 1), 2, 12000)
        got = K.kh_estimate(G)
        for x, y in zip(got, want):
            assert np.array_equal(x, y)
        assert (want[1] > 0).any()  # some level above 0: the trim ran
    finally:
        G.close()
