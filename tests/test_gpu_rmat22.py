"""Parity on the R-MAT scale-22 workload (4.19M nodes, 64M edges).

Exact h-degrees at h = 2 (the BFS keeps its visited sets in global memory at
this size), adaptive estimates at h = 2, 3, 4, and the sampled (k,3)-core,
checked on sampled nodes one by one against the oracle, with the peel
certified by d(v; X_r(v)) <= c(v) <= d(v; {u : c(u) >= c(v)}).  Exact
integer comparisons throughout.
"""
import numpy as np
import pytest

import oracle as O
from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import khcore as K

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def rmat22():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    K.load(build_if_missing=True)
    rp, cl = gg.rmat(22, 16, 0.57, 0.19, 0.19, 1003)
    ctx = K.kh_ctx_create(0)
    G = K.kh_graph_load_csr(ctx, rp, cl)
    K.kh_set_sampling(G, seed=1, M=0, eps=0.5, delta=0.05)
    deg = np.diff(rp)
    rng = np.random.default_rng(11)
    nz = np.nonzero(deg > 0)[0]
    sample = np.unique(np.concatenate([rng.choice(nz, 12, replace=False), np.argsort(deg)[-2:]]))
    yield ctx, G, rp, cl, sample
    G.close()
    ctx.close()


def test_rmat22_exact_degrees_and_estimates(rmat22):
    ctx, G, rp, cl, sample = rmat22
    n = rp.size - 1
    r = O.ranks(n, 1)
    M = K.kh_get_M(G)
    assert M == O.budget_M(n, 0.5, 0.05) == 841
    K.kh_set_h(G, 2)
    deg = K.kh_hdegree_exact(G)
    assert (deg[sample] == O.hdegree_some(rp, cl, 2, sample)).all()
    for h in (2, 3, 4):
        K.kh_set_h(G, h)
        est, lvl, bs = K.kh_estimate(G)
        sub = sample if h < 4 else sample[:6]
        we, wl, wb = O.estimate_def_some(rp, cl, r, h, M, sub)
        assert (est[sub] == we).all() and (lvl[sub] == wl).all() and (bs[sub] == wb).all()


def test_rmat22_sampled_core_h3(rmat22):
    ctx, G, rp, cl, sample = rmat22
    n = rp.size - 1
    r = O.ranks(n, 1)
    M = K.kh_get_M(G)
    K.kh_set_h(G, 3)
    core = K.kh_core_sampled(G).astype(np.int64)
    rnd, rounds, _ = K.kh_peel_info(G)
    assert rnd.max() == rounds - 1
    order = np.argsort(rnd, kind="stable")
    assert (np.diff(core[order]) >= 0).all()
    for v in sample[:8]:
        xr = rnd >= rnd[v]
        assert int(O.estimate_def_some(rp, cl, r, 3, M, [v], alive=xr)[0][0]) <= core[v]
        sk = core >= core[v]
        assert int(O.estimate_def_some(rp, cl, r, 3, M, [v], alive=sk)[0][0]) >= core[v]
