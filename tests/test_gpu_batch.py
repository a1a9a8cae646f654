"""The batched form: many graphs packed in one CSR (kh_graph_load_batch).

Every per-node result of the batch must equal, bit for bit, the result of
loading that graph alone with the same h and M (each graph keeps its own
ranks, its own h and, by default, its own M from Eq. (buffer)).  This holds
because the h-neighbourhoods of a disjoint union never cross graphs and the
bucket peel yields the unique generalized core numbers whatever the order.
"""
import numpy as np
import pytest

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


def make_batch():
    graphs = [gg.barabasi_albert(300, 3, 1), gg.erdos_renyi(500, 2000, 2), gg.grid(20, 25, 0.02, 3),
              gg.chung_lu(800, 10, 2.3, 120, 4), gg.star(40), gg.complete(12),
              gg.barabasi_albert(1200, 5, 5), gg.path(30), gg.rmat(9, 8, .57, .19, .19, 6),
              gg.cycle(50), gg.barabasi_albert(150, 8, 7), gg.erdos_renyi(40, 0, 8)]
    hs = [2, 3, 4, 2, 1, 3, 4, 2, 3, 1, 2, 4]
    vtx_off, rp, cl = gg.pack_batch(graphs)
    return graphs, hs, vtx_off, rp, cl


def alone(ctx, g, h, M):
    G = K.kh_graph_load_csr(ctx, *g)
    K.kh_set_h(G, h)
    K.kh_set_sampling(G, seed=1, M=M)
    out = {"r": K.kh_ranks(G), "deg": K.kh_hdegree_exact(G), "cnt": K.kh_sampled_counts(G, 0, 5),
           "est": K.kh_estimate(G), "ce": K.kh_core_exact(G), "cs": K.kh_core_sampled(G)}
    G.close()
    return out


@pytest.mark.parametrize("uniform_M", [0, 9])
def test_batch_equals_graphs_alone(ctx, uniform_M):
    graphs, hs, vtx_off, rp, cl = make_batch()
    B = K.kh_graph_load_batch(ctx, vtx_off, rp, cl, hs)
    K.kh_set_sampling(B, seed=1, M=uniform_M)
    r = K.kh_ranks(B)
    deg = K.kh_hdegree_exact(B)
    cnt = K.kh_sampled_counts(B, 0, 5)
    est, lvl, bs = K.kh_estimate(B)
    ce = K.kh_core_exact(B)
    cs = K.kh_core_sampled(B)
    for q, (g, h) in enumerate(zip(graphs, hs)):
        a, b = vtx_off[q], vtx_off[q + 1]
        want = alone(ctx, g, h, uniform_M)
        assert (r[a:b] == want["r"]).all(), q
        assert (deg[a:b] == want["deg"]).all(), q
        assert (cnt[a:b] == want["cnt"]).all(), q
        assert (est[a:b] == want["est"][0]).all(), q
        assert (lvl[a:b] == want["est"][1]).all(), q
        assert (bs[a:b] == want["est"][2]).all(), q
        assert (ce[a:b] == want["ce"]).all(), q
        assert (cs[a:b] == want["cs"]).all(), q
    B.close()


def test_batch_rejects_edges_between_graphs(ctx):
    graphs, hs, vtx_off, rp, cl = make_batch()
    # join node 0 (graph 0) and the last node (last graph) by an edge
    from paper_2112_06154_gb300.graphgen import csr_from_edges
    n = int(vtx_off[-1])
    src = np.repeat(np.arange(n), np.diff(rp))
    keep = src < cl
    rp2, cl2 = csr_from_edges(n, np.concatenate([src[keep], [0]]), np.concatenate([cl[keep], [n - 1]]))
    with pytest.raises(K.KhError) as ei:
        K.kh_graph_load_batch(ctx, vtx_off, rp2, cl2, hs)
    assert ei.value.code == K.KH_EGRAPH


def test_batch_set_h_applies_to_every_graph(ctx):
    graphs, hs, vtx_off, rp, cl = make_batch()
    B = K.kh_graph_load_batch(ctx, vtx_off, rp, cl, hs)
    K.kh_set_h(B, 2)
    deg = K.kh_hdegree_exact(B)
    for q, g in enumerate(graphs):
        G = K.kh_graph_load_csr(ctx, *g)
        K.kh_set_h(G, 2)
        assert (deg[vtx_off[q]:vtx_off[q + 1]] == K.kh_hdegree_exact(G)).all()
        G.close()
    B.close()
