"""Full-size core maps, every node: a certificate that the library's core map
equals the unique (k,h)-core map, checked with the CPU oracle.

For a node function d(v; X) that never grows as X shrinks (deg_h: Sec. 2; the
estimate: Prop. 4.2), the core map c(v) = max{k : some set S containing v has
d(u; S) >= k for all u in S} is unique, and it is what the oracle's peels
compute (pinned on small graphs against the exhaustive subset definition).
Given the library's core map c' and removal rounds r', with X_r = {u : r'(u) >= r}
and S_k = {u : c'(u) >= k}, the checks
  (1) c' is constant within a round and nondecreasing in the round,
  (2) d(v; X_r'(v)) <= c'(v) for every node v  (v could leave when it did),
  (3) d(v; S_c'(v)) >= c'(v) for every node v  (S_k is a set of d >= k),
prove c' = c: (3) makes every S_k a witness, so c >= c'; for the other side
take a witness S* of c(v), its first-removed node u0 has
d(u0; X_r'(u0)) >= d(u0; S*) >= c(v), so by (2) and (1) c'(v) >= c'(u0) >= c(v).
The oracle evaluates d one node at a time on the node sets those checks name
(exact h-degrees by breadth-first search, the estimate by Def. 4.1); every
node of the graph is checked.  Large cases spread the node groups over a
process pool (spawn) of oracle workers.
"""
import multiprocessing as mp
import os

import numpy as np
import pytest

import oracle as O
from paper_2112_06154_gb300 import graphgen as gg
from paper_2112_06154_gb300 import khcore as K

pytestmark = pytest.mark.gpu
N = 200_000

_W = {}


def _init(h, M, exact, core, rnd):
    _W["g"] = gg.chung_lu(N, 20, 2.5, 5000, 1002)
    _W["r"] = O.ranks(N, 1)
    _W["h"], _W["M"], _W["exact"] = h, M, exact
    _W["core"], _W["rnd"] = core, rnd


def _d(vs, alive):
    rp, cl = _W["g"]
    if _W["exact"]:
        return O.hdegree_some(rp, cl, _W["h"], vs, alive=alive).astype(np.int64)
    return O.estimate_def_some(rp, cl, _W["r"], _W["h"], _W["M"], vs, alive=alive)[0].astype(np.int64)


def _check(task):
    """(2) for the nodes removed in round `key`, or (3) for the nodes of core `key`;
    returns the failing nodes (at most 5)."""
    kind, key, vs = task
    core, rnd = _W["core"], _W["rnd"]
    if kind == "removed":
        alive = (rnd >= key).astype(np.uint8)
        bad = _d(vs, alive) > core[vs]
    else:
        alive = (core >= key).astype(np.uint8)
        bad = _d(vs, alive) < core[vs]
    return [int(v) for v in vs[bad][:5]]


def certify(h, M, exact, core, rnd, jobs):
    core = np.asarray(core).astype(np.int64)
    rnd = np.asarray(rnd).astype(np.int64)
    assert (rnd >= 0).all()
    # (1) one value per round, nondecreasing in the round
    order = np.argsort(rnd, kind="stable")
    rs, cs = rnd[order], core[order]
    assert (np.diff(cs) >= 0).all()
    assert (cs[1:][rs[1:] == rs[:-1]] == cs[:-1][rs[1:] == rs[:-1]]).all()
    tasks = []
    for kind, key_of in (("removed", rnd), ("core", core)):
        o = np.argsort(key_of, kind="stable")
        keys, starts = np.unique(key_of[o], return_index=True)
        bounds = list(starts[1:]) + [o.size]
        for key, a, b in zip(keys, starts, bounds):
            vs = np.sort(o[a:b]).astype(np.int32)
            for c0 in range(0, vs.size, 512):
                tasks.append((kind, int(key), vs[c0:c0 + 512]))
    if jobs <= 1:
        _init(h, M, exact, core, rnd)
        bad = [x for t in tasks for x in _check(t)]
    else:
        ctx = mp.get_context("spawn")
        with ctx.Pool(jobs, initializer=_init, initargs=(h, M, exact, core, rnd)) as pool:
            bad = [x for res in pool.imap_unordered(_check, tasks, chunksize=4) for x in res]
    assert not bad, f"certificate fails at nodes {bad[:10]}"
    return len(tasks)


@pytest.fixture(scope="module")
def c2():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    K.load(build_if_missing=True)
    ctx = K.kh_ctx_create(0)
    rp, cl = gg.chung_lu(N, 20, 2.5, 5000, 1002)
    G = K.kh_graph_load_csr(ctx, rp, cl)
    K.kh_set_sampling(G, seed=1, M=0, eps=0.5, delta=0.05)
    yield G
    G.close()
    ctx.close()


def jobs():
    return max(1, min(16, (os.cpu_count() or 2) - 1))


def test_exact_core_h2_every_node(c2):
    K.kh_set_h(c2, 2)
    core = K.kh_core_exact(c2)
    rnd, _, _ = K.kh_peel_info(c2)
    certify(2, 0, True, core, rnd, jobs())


def test_sampled_core_h2_every_node_and_prop44(c2):
    M = K.kh_get_M(c2)
    K.kh_set_h(c2, 2)
    core = K.kh_core_sampled(c2)
    rnd, _, _ = K.kh_peel_info(c2)
    certify(2, M, False, core, rnd, jobs())
    # Prop. 4.4, second claim, against the (certified) exact core
    exact = K.kh_core_exact(c2).astype(np.int64)
    assert (np.minimum(core.astype(np.int64), M) == np.minimum(exact, M)).all()


def test_sampled_core_h3_every_node(c2):
    M = K.kh_get_M(c2)
    K.kh_set_h(c2, 3)
    core = K.kh_core_sampled(c2)
    rnd, _, _ = K.kh_peel_info(c2)
    certify(3, M, False, core, rnd, jobs())


def test_exact_core_h3_every_node(c2):
    M = K.kh_get_M(c2)
    K.kh_set_h(c2, 3)
    core = K.kh_core_exact(c2)
    rnd, _, _ = K.kh_peel_info(c2)
    certify(3, 0, True, core, rnd, jobs())
    # Prop. 4.4, second claim, between the two (k,3) peels
    K.kh_set_h(c2, 3)
    sampled = K.kh_core_sampled(c2).astype(np.int64)
    assert (np.minimum(sampled, M) == np.minimum(core.astype(np.int64), M)).all()
