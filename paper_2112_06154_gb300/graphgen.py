"""Seeded synthetic graph generators (inputs only).

Every generator returns a simple undirected graph as a symmetric CSR pair
``(rowptr int64[n+1], col int32[2m])`` with each row sorted ascending, no
self-loops and no duplicate edges.  This module holds none of the (k,h)-core
method's arithmetic: it only draws edges.  Both the CUDA path and the CPU
oracle read graphs made here, so the two never share anything else.

Workload shapes (stand-ins for the paper's SNAP/KONECT graphs, which are not
available offline):

* ``erdos_renyi(n, m)``: G(n, m), m distinct uniform edges.
* ``chung_lu(n, avg_deg, gamma, max_deg)``: power-law expected degrees
  w_i proportional to (i + i0)^(-1/(gamma-1)), scaled to ``avg_deg`` and capped at
  ``max_deg``; edges drawn with endpoints proportional to w, self-loops and
  duplicates dropped.
* ``rmat(scale, edge_factor, a, b, c)``: recursive-matrix edges, symmetrised,
  deduplicated, self-loops dropped, vertex ids permuted by a seeded permutation.
* ``barabasi_albert(n, m)``: preferential attachment (copy model), deduplicated.
* ``grid(a, b, shortcut_frac)``: a x b lattice plus random shortcut edges.
* ``with_hubs(n, hub_degrees)``: a Chung-Lu graph plus a few nodes of given
  (large) degree.
* closed-form graphs: complete, path, cycle, star, grid.
"""
from __future__ import annotations

import numpy as np

__all__ = [
    "csr_from_edges", "erdos_renyi", "chung_lu", "rmat", "barabasi_albert",
    "grid", "complete", "path", "cycle", "star", "random_small",
    "pack_batch", "graph_stats", "barabasi_albert_batch", "ba_batch_workload", "with_hubs",
]


def csr_from_edges(n: int, u: np.ndarray, v: np.ndarray):
    """Symmetric, sorted, deduplicated CSR from an undirected edge list."""
    u = np.asarray(u, dtype=np.int64)
    v = np.asarray(v, dtype=np.int64)
    keep = u != v
    u, v = u[keep], v[keep]
    lo = np.minimum(u, v)
    hi = np.maximum(u, v)
    key = lo * n + hi
    key.sort()
    if key.size:
        first = np.empty(key.size, dtype=bool)
        first[0] = True
        np.not_equal(key[1:], key[:-1], out=first[1:])
        key = key[first]
    lo = key // n
    hi = key - lo * n
    # both directions as one sorted key array: (src, dst) -> src * n + dst
    both = np.concatenate([key, hi * n + lo])
    both.sort()
    src = both // n
    dst = both - src * n
    counts = np.bincount(src, minlength=n).astype(np.int64)
    rowptr = np.zeros(n + 1, dtype=np.int64)
    np.cumsum(counts, out=rowptr[1:])
    return rowptr, dst.astype(np.int32)


def erdos_renyi(n: int, m: int, seed: int):
    """G(n, m): ``m`` distinct edges drawn uniformly without replacement."""
    rng = np.random.default_rng(seed)
    total = n * (n - 1) // 2
    if m > total:
        raise ValueError("m exceeds the number of vertex pairs")
    chosen = np.empty(0, dtype=np.int64)
    while chosen.size < m:
        need = m - chosen.size
        draw = rng.integers(0, total, size=int(need * 1.2) + 16, dtype=np.int64)
        chosen = np.unique(np.concatenate([chosen, draw]))
    chosen = rng.permutation(chosen)[:m]
    # decode pair index -> (i, j), i < j, row-major over the upper triangle
    i = (n - 2 - np.floor(np.sqrt(-8.0 * chosen + 4.0 * n * (n - 1) - 7) / 2.0 - 0.5)).astype(np.int64)
    j = chosen + i + 1 - n * (n - 1) // 2 + (n - i) * ((n - i) - 1) // 2
    return csr_from_edges(n, i, j)


def sbm_hierarchical(n: int, seed: int, blocks: int = 10, base: float = 1e-6):
    """Stochastic block model with `blocks` equal blocks C_1..C_b (block i holds
    nodes [(i-1) n/b, i n/b)); a pair in C_i x C_j, i <= j, is an edge with
    probability base * i^2 (the within-block probability uses i = j).  The
    number of edges of each block pair is binomial; the pairs are drawn
    uniformly and de-duplicated."""
    rng = np.random.default_rng(seed)
    bounds = [(q * n) // blocks for q in range(blocks + 1)]
    us, vs = [], []
    for i in range(1, blocks + 1):
        lo_i, hi_i = bounds[i - 1], bounds[i]
        for j in range(i, blocks + 1):
            lo_j, hi_j = bounds[j - 1], bounds[j]
            a, b = hi_i - lo_i, hi_j - lo_j
            pairs = a * (a - 1) // 2 if i == j else a * b
            if pairs <= 0:
                continue
            k = int(rng.binomial(pairs, min(1.0, base * i * i)))
            if k == 0:
                continue
            u = rng.integers(lo_i, hi_i, size=k, dtype=np.int64)
            v = rng.integers(lo_j, hi_j, size=k, dtype=np.int64)
            us.append(u)
            vs.append(v)
    if not us:
        return csr_from_edges(n, np.empty(0, np.int64), np.empty(0, np.int64))
    return csr_from_edges(n, np.concatenate(us), np.concatenate(vs))


def chung_lu(n: int, avg_deg: float, gamma: float, max_deg: int, seed: int):
    """Chung-Lu power-law graph with expected degrees w_i (see module doc)."""
    rng = np.random.default_rng(seed)
    idx = np.arange(n, dtype=np.float64)
    w = (idx + 10.0) ** (-1.0 / (gamma - 1.0))
    w = np.minimum(w * (avg_deg * n / w.sum()), max_deg)
    w *= avg_deg * n / w.sum()
    w = np.minimum(w, max_deg)
    m_draw = int(round(w.sum() / 2.0))
    p = w / w.sum()
    cdf = np.cumsum(p)
    cdf[-1] = 1.0
    u = np.searchsorted(cdf, rng.random(m_draw), side="right")
    v = np.searchsorted(cdf, rng.random(m_draw), side="right")
    np.minimum(u, n - 1, out=u)
    np.minimum(v, n - 1, out=v)
    perm = rng.permutation(n)
    return csr_from_edges(n, perm[u], perm[v])


def rmat(scale: int, edge_factor: int, a: float, b: float, c: float, seed: int):
    """R-MAT graph with 2^scale vertices and edge_factor * 2^scale edge draws.

    Each draw descends `scale` levels; at each level one uniform number picks
    quadrant a (0,0), b (0,1), c (1,0) or d (1,1), appending one bit to the
    row and column ids (most significant first)."""
    rng = np.random.default_rng(seed)
    n = 1 << scale
    m_draw = edge_factor * n
    u = np.empty(m_draw, dtype=np.int64)
    v = np.empty(m_draw, dtype=np.int64)
    ab = np.float32(a + b)
    abc = np.float32(a + b + c)
    a32 = np.float32(a)
    chunk = 1 << 24
    for s in range(0, m_draw, chunk):
        e = min(m_draw, s + chunk)
        uu = np.zeros(e - s, dtype=np.uint32)
        vv = np.zeros(e - s, dtype=np.uint32)
        for _ in range(scale):
            x = rng.random(e - s, dtype=np.float32)
            q = (x >= a32).astype(np.uint32)
            q += x >= ab
            q += x >= abc          # quadrant index 0..3 = a, b, c, d
            uu <<= 1
            uu |= q >> 1
            vv <<= 1
            vv |= q & 1
        u[s:e] = uu
        v[s:e] = vv
    perm = rng.permutation(n).astype(np.int64)
    return csr_from_edges(n, perm[u], perm[v])


def with_hubs(n: int, hub_degrees, seed: int, avg_deg: float = 6, gamma: float = 2.3,
              max_deg: int = 300):
    """A Chung-Lu graph (as in chung_lu) plus hub nodes: node ``10 * i + 5`` gets
    ``hub_degrees[i]`` extra neighbours drawn uniformly without replacement
    (duplicates with existing edges collapse)."""
    rp, cl = chung_lu(n, avg_deg, gamma, max_deg, seed)
    rng = np.random.default_rng(seed + 1)
    us = [np.repeat(np.arange(n, dtype=np.int64), np.diff(rp))]
    vs = [cl.astype(np.int64)]
    for i, k in enumerate(hub_degrees):
        us.append(np.full(int(k), 10 * i + 5, dtype=np.int64))
        vs.append(rng.choice(n, size=int(k), replace=False).astype(np.int64))
    return csr_from_edges(n, np.concatenate(us), np.concatenate(vs))


def barabasi_albert(n: int, m: int, seed: int):
    """Preferential attachment via the copy model.

    Vertex t >= m attaches ``m`` edges; each edge endpoint is a uniformly drawn
    entry of the endpoint list of all earlier edges (or a uniform earlier
    vertex for the seed clique), which selects targets with probability
    proportional to degree.  Duplicate targets collapse (dedup), so a vertex
    may end with fewer than ``m`` edges.
    """
    rng = np.random.default_rng(seed)
    if n <= m + 1:
        return complete(n)
    # seed: clique on vertices 0..m
    cu, cv = np.triu_indices(m + 1, k=1)
    n0 = cu.size
    t = np.arange(m + 1, n, dtype=np.int64)
    ne = (n - m - 1) * m
    src = np.repeat(t, m)
    # endpoint list: entries 2e, 2e+1 for edge e (seed edges first); a new
    # vertex draws among the endpoints of all edges created before it
    first_e_of_src = n0 + (src - (m + 1)) * m
    limit = 2 * first_e_of_src
    pick = (rng.random(ne) * limit).astype(np.int64)
    ends_u = np.concatenate([cu.astype(np.int64), src])
    # resolve picks by pointer jumping: even position -> source of the edge,
    # odd position -> target of the edge (which may itself be a pick)
    tgt = np.empty(n0 + ne, dtype=np.int64)
    tgt[:n0] = cv
    ptr = np.full(n0 + ne, -1, dtype=np.int64)
    is_odd = (pick & 1) == 1
    eid = pick >> 1
    direct = ~is_odd
    tgt_new = np.where(direct, ends_u[eid], -1)
    seed_ref = is_odd & (eid < n0)
    tgt_new = np.where(seed_ref, cv[np.minimum(eid, n0 - 1)], tgt_new)
    ptr_new = np.where(is_odd & (eid >= n0), eid, -1)
    tgt[n0:] = tgt_new
    ptr[n0:] = ptr_new
    for _ in range(64):
        pend = ptr >= 0
        if not pend.any():
            break
        idx = np.nonzero(pend)[0]
        p = ptr[idx]
        nxt = ptr[p]
        resolved = nxt < 0
        new_tgt = tgt[p]
        tgt[idx[resolved]] = new_tgt[resolved]
        ptr[idx] = nxt
    return csr_from_edges(n, ends_u, tgt)


def grid(a: int, b: int, shortcut_frac: float = 0.0, seed: int = 0):
    """a x b 4-neighbour lattice, plus round(shortcut_frac * m) random edges."""
    idx = np.arange(a * b, dtype=np.int64).reshape(a, b)
    u = np.concatenate([idx[:, :-1].ravel(), idx[:-1, :].ravel()])
    v = np.concatenate([idx[:, 1:].ravel(), idx[1:, :].ravel()])
    k = int(round(shortcut_frac * u.size))
    if k > 0:
        rng = np.random.default_rng(seed)
        su = rng.integers(0, a * b, size=k)
        sv = rng.integers(0, a * b, size=k)
        u = np.concatenate([u, su])
        v = np.concatenate([v, sv])
    return csr_from_edges(a * b, u, v)


def complete(n: int):
    u, v = np.triu_indices(n, k=1)
    return csr_from_edges(n, u, v)


def path(n: int):
    u = np.arange(n - 1)
    return csr_from_edges(n, u, u + 1)


def cycle(n: int):
    u = np.arange(n)
    return csr_from_edges(n, u, (u + 1) % n)


def star(leaves: int):
    return csr_from_edges(leaves + 1, np.zeros(leaves, dtype=np.int64), np.arange(1, leaves + 1))


def random_small(n: int, p: float, seed: int):
    """G(n, p) for tiny brute-force cases."""
    rng = np.random.default_rng(seed)
    u, v = np.triu_indices(n, k=1)
    keep = rng.random(u.size) < p
    return csr_from_edges(n, u[keep], v[keep])


def pack_batch(graphs):
    """Pack graphs into one offset-indexed CSR.

    Returns ``(vtx_off int64[g+1], rowptr int64[N+1], col int32[...])`` where
    graph ``i`` owns vertices ``vtx_off[i] .. vtx_off[i+1]-1`` and its column
    indices are global (shifted by ``vtx_off[i]``).
    """
    sizes = [int(rp.size - 1) for rp, _ in graphs]
    vtx_off = np.zeros(len(graphs) + 1, dtype=np.int64)
    np.cumsum(sizes, out=vtx_off[1:])
    rps = []
    cols = []
    base_e = 0
    for i, (rp, cl) in enumerate(graphs):
        rps.append(rp[:-1] + base_e)
        cols.append(cl.astype(np.int64) + vtx_off[i])
        base_e += int(rp[-1])
    rowptr = np.concatenate(rps + [np.array([base_e], dtype=np.int64)]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return vtx_off, rowptr, col


def graph_stats(rowptr, col):
    deg = np.diff(rowptr)
    return {
        "n": int(rowptr.size - 1),
        "m": int(col.size // 2),
        "max_deg": int(deg.max()) if deg.size else 0,
        "sum_deg2": int((deg.astype(np.int64) ** 2).sum()),
        "isolated": int((deg == 0).sum()),
    }


def barabasi_albert_batch(ns, ms, seed: int):
    """Many preferential-attachment graphs (copy model, as in barabasi_albert)
    drawn in one vectorised pass and packed as in pack_batch.

    Graph q has ns[q] > ms[q] + 1 nodes: a seed clique on ms[q] + 1 nodes, then
    every later node attaches ms[q] edges whose targets are uniformly drawn
    entries of the endpoint list of the graph's earlier edges.  Returns
    (vtx_off int64[g+1], rowptr int64[N+1], col int32[...])."""
    rng = np.random.default_rng(seed)
    ns = np.asarray(ns, dtype=np.int64)
    ms = np.asarray(ms, dtype=np.int64)
    if np.any(ns <= ms + 1):
        raise ValueError("every graph needs n > m + 1")
    G = ns.size
    vtx_off = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(ns, out=vtx_off[1:])
    e0 = ms * (ms + 1) // 2                       # seed-clique edges
    enew = (ns - ms - 1) * ms                     # attachment edges
    eq = e0 + enew
    ebase = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(eq, out=ebase[1:])
    etot = int(ebase[-1])
    src = np.empty(etot, dtype=np.int64)
    tgt = np.empty(etot, dtype=np.int64)
    ptr = np.full(etot, -1, dtype=np.int64)
    # seed cliques (graph-local ids shifted to global)
    for q in range(G):
        cu, cv = np.triu_indices(int(ms[q]) + 1, k=1)
        a = int(ebase[q])
        src[a:a + cu.size] = cu + vtx_off[q]
        tgt[a:a + cu.size] = cv + vtx_off[q]
    # attachment edges: graph, local node t, and the endpoint they copy
    gq = np.repeat(np.arange(G), enew)
    newbase = np.zeros(G + 1, dtype=np.int64)
    np.cumsum(enew, out=newbase[1:])
    idx = np.arange(int(newbase[-1]), dtype=np.int64) - newbase[gq]
    mq = ms[gq]
    t = mq + 1 + idx // mq
    eid = ebase[gq] + e0[gq] + idx                # global id of the edge itself
    src[eid] = vtx_off[gq] + t
    limit = 2 * (e0[gq] + (t - mq - 1) * mq)
    pick = (rng.random(idx.size) * limit).astype(np.int64)
    ref = ebase[gq] + (pick >> 1)                 # referenced (earlier) edge
    side = pick & 1
    direct = side == 0
    tgt[eid[direct]] = src[ref[direct]]
    seedref = (~direct) & ((pick >> 1) < e0[gq])
    tgt[eid[seedref]] = tgt[ref[seedref]]
    pend = (~direct) & ~seedref
    ptr[eid[pend]] = ref[pend]
    for _ in range(64):
        todo = np.nonzero(ptr >= 0)[0]
        if todo.size == 0:
            break
        p = ptr[todo]
        nxt = ptr[p]
        done = nxt < 0
        tgt[todo[done]] = tgt[p[done]]
        ptr[todo] = nxt
    n = int(vtx_off[-1])
    rowptr, col = csr_from_edges(n, src, tgt)
    return vtx_off, rowptr, col


def ba_batch_workload(num_graphs: int = 4096, seed: int = 1004, n_lo: int = 100, n_hi: int = 20000):
    """The batched workload: num_graphs preferential-attachment graphs with n
    log-uniform in [n_lo, n_hi], attachment m uniform in {3..8} and h uniform
    in {2, 3, 4}.  Returns (vtx_off, rowptr, col, h_per_graph)."""
    rng = np.random.default_rng(seed)
    ns = np.exp(rng.uniform(np.log(n_lo), np.log(n_hi), num_graphs)).round().astype(np.int64)
    ms = rng.integers(3, 9, num_graphs)
    hs = rng.integers(2, 5, num_graphs).astype(np.int32)
    vtx_off, rowptr, col = barabasi_albert_batch(ns, ms, seed + 1)
    return vtx_off, rowptr, col, hs
