"""Parity at the benchmark's full size (Chung-Lu n = 200,000, m ~ 2M).

The oracle cannot peel this graph in seconds, so the checks here are those
that hold at any size and that the oracle can evaluate one node at a time:
  * exact h-degrees, fixed-level counts and estimates of sampled nodes;
  * for sampled nodes v of a peel with core value c(v) removed in round r(v):
      d(v; X_r(v)) <= c(v)           (v was removed with d <= c), and
      d(v; {u : c(u) >= c(v)}) >= c(v)  (v belongs to the c(v)-core),
    with d the exact h-degree or the estimate, computed by the oracle on
    those node sets;
  * round values are consistent: c is nondecreasing in the round;
  * Prop. 4.4, second claim: min(c'(v), M) == min(c(v), M) between the
    sampled and the exact peel.
All comparisons are exact (integers).
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import khcore as K

pytestmark = pytest.mark.gpu

N = 200_000


@pytest.fixture(scope="module")
def setup():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    K.load(build_if_missing=True)
    ctx = K.kh_ctx_create(0)
    rp, cl = gg.chung_lu(N, 20, 2.5, 5000, 1002)
    G = K.kh_graph_load_csr(ctx, rp, cl)
    K.kh_set_sampling(G, seed=1, M=0, eps=0.5, delta=0.05)
    rng = np.random.default_rng(7)
    sample = np.unique(np.concatenate([rng.choice(N, 120, replace=False),
                                       np.argsort(np.diff(rp))[-8:]]))  # plus the hubs
    yield ctx, G, rp, cl, sample
    G.close()
    ctx.close()


def test_full_size_degrees_counts_estimates(setup):
    ctx, G, rp, cl, sample = setup
    r = O.ranks(N, 1)
    M = K.kh_get_M(G)
    assert M == 719
    for h in (2, 3):
        K.kh_set_h(G, h)
        deg = K.kh_hdegree_exact(G)
        assert (deg[sample] == O.hdegree_some(rp, cl, h, sample)).all()
        est, lvl, bs = K.kh_estimate(G)
        we, wl, wb = O.estimate_def_some(rp, cl, r, h, M, sample)
        assert (est[sample] == we).all() and (lvl[sample] == wl).all() and (bs[sample] == wb).all()
    K.kh_set_h(G, 2)
    cnt = K.kh_sampled_counts(G, 0, 10)
    for v in sample[:40]:
        ball = O.hball(rp, cl, int(v), 2)[1:]
        want = [(r[ball] >= j).sum() for j in range(11)]
        assert list(cnt[v]) == want


def certify(rp, cl, core, rnd, sample, dfun):
    """d(v; X_r(v)) <= c(v) <= d(v; S_c(v)) for sampled v; c nondecreasing in rounds."""
    order = np.argsort(rnd, kind="stable")
    assert (np.diff(core[order].astype(np.int64)) >= 0).all()
    for v in sample:
        xr = rnd >= rnd[v]
        assert dfun(v, xr) <= int(core[v])
        sk = core >= core[v]
        assert dfun(v, sk) >= int(core[v])


def test_full_size_exact_core_h2(setup):
    ctx, G, rp, cl, sample = setup
    K.kh_set_h(G, 2)
    core = K.kh_core_exact(G)
    rnd, rounds, _ = K.kh_peel_info(G)
    assert rnd.max() == rounds - 1
    certify(rp, cl, core, rnd, sample,
            lambda v, S: int(O.hdegree_some(rp, cl, 2, [v], alive=S)[0]))


@pytest.mark.parametrize("h", [2, 3])
def test_full_size_sampled_core(setup, h):
    ctx, G, rp, cl, sample = setup
    r = O.ranks(N, 1)
    M = K.kh_get_M(G)
    K.kh_set_h(G, h)
    core = K.kh_core_sampled(G)
    rnd, rounds, _ = K.kh_peel_info(G)
    assert rnd.max() == rounds - 1
    certify(rp, cl, core, rnd, sample[:60],
            lambda v, S: int(O.estimate_def_some(rp, cl, r, h, M, [v], alive=S)[0][0]))
    if h == 2:
        exact = K.kh_core_exact(G).astype(np.int64)
        assert (np.minimum(core.astype(np.int64), M) == np.minimum(exact, M)).all()
