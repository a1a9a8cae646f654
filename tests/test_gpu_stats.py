"""Work statistics and per-launch traces of a peel (kh_peel_stats,
kh_prof_trace): internally consistent, and the rank-filtered refreshes
never skip a list that changes (the sampled cores stay those of the oracle)."""
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


@pytest.mark.parametrize("h", [2, 3, 4])
def test_sampled_peel_stats(ctx, h):
    rowptr, col = gg.chung_lu(6000, 12, 2.5, 300, 77 + h)
    M = 24
    G = K.kh_graph_load_csr(ctx, rowptr, col)
    try:
        K.kh_set_h(G, h)
        K.kh_set_sampling(G, seed=5, M=M)
        K.kh_prof_enable(G, True)
        core = K.kh_core_sampled(G)
        ref, chg, stopped = K.kh_peel_stats(G)
        _, rounds, updates = K.kh_peel_info(G, False)
        # refreshes exist on every level below h, none on the lazy last level
        assert (chg <= ref).all()
        assert (ref[1:h] > 0).all() and (chg[1:h] > 0).all()
        assert ref[h:].sum() == 0
        # early-stopped refines leave a lower bound only: counted apart from updates
        assert stopped >= 0 and updates > 0
        ms, launches, alg = K.kh_prof_read(G, K.KH_PROF_LEVELU)
        trace = K.kh_prof_trace(G, K.KH_PROF_LEVELU)
        assert trace.size == launches > 0
        assert abs(float(trace.sum()) - ms) <= 1e-3 * max(ms, 1.0)
        # per-launch algorithmic bytes add up to the class counter
        tb = K.kh_prof_trace_bytes(G, K.KH_PROF_LEVELU)
        assert tb.size == launches and (tb != np.uint64(2**64 - 1)).all()
        assert int(tb.sum()) == int(alg)
        # the launch-by-launch (profiled) peel and the graph replay agree
        K.kh_prof_enable(G, False)
        assert (K.kh_core_sampled(G) == core).all()
        # refreshes below the last level do not depend on the lazy refines
        ref2, chg2, _ = K.kh_peel_stats(G)
        assert (ref2 == ref).all() and (chg2 == chg).all()
        r = O.ranks(rowptr.size - 1, 5)
        want, _, _ = O.core_sampled(rowptr, col, r, h, M)
        assert np.array_equal(core, want)
    finally:
        G.close()


def test_exact_peel_stops_early(ctx):
    rowptr, col = gg.chung_lu(6000, 12, 2.5, 300, 91)
    G = K.kh_graph_load_csr(ctx, rowptr, col)
    try:
        K.kh_set_h(G, 2)
        core = K.kh_core_exact(G)
        _, _, updates = K.kh_peel_info(G, False)
        ref, chg, stopped = K.kh_peel_stats(G)
        assert ref.sum() == 0 and chg.sum() == 0
        assert stopped > 0 and updates > 0
        want, _, _ = O.core_exact(rowptr, col, 2)
        assert np.array_equal(core, want)
    finally:
        G.close()
