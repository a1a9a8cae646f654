"""The exactness arguments behind the GPU refresh, checked as properties on
random graphs with the oracle and brute-force distances (no GPU).

Loss propagation (exact refresh): when a set R leaves X, a node x whose
nearest removed node is exactly h hops away keeps every path of at most h
edges except at its end, so deg_h(x; X \\ R) = deg_h(x; X) - |{u in R :
d_X(u, x) <= h}|, and a node farther than h from R keeps its h-degree.

Rank filter (sampled refresh): level i of v is the rank filter of the union
of its neighbours' level i-1 lists (Prop. 3.1, Alg. 2), so if v has no
removed neighbour and every changed neighbour list w has rho_w < k[v,i] - 1
(rho_w: the top rank among the members that left, or k_old[w] - 1 when the
level of w fell), then B[v,i] and k[v,i] do not change.

Bit-parallel 2-balls (sweeps of the exact 2-degree pass): with m1[u] = {j : u
in A(s_j)} for a batch of sources s_j, x is in N(s_j; 2) exactly when j is in
m1[x] | OR_{u in A(x)} m1[u]; and a filter with one bit per group of 4 node
ids, set for every group holding a node with m1 != {}, never drops an entry
that contributes."""
import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

import oracle as O
from paper_2112_06154_gb300 import graphgen as gg


def dist_matrix(rowptr, col, alive):
    n = rowptr.size - 1
    src = np.repeat(np.arange(n), np.diff(rowptr))
    keep = alive[src] & alive[col]
    A = csr_matrix((np.ones(keep.sum()), (src[keep], col[keep])), shape=(n, n))
    return shortest_path(A, unweighted=True, directed=False)


def graphs():
    yield gg.chung_lu(120, 6, 2.5, 25, 3)
    yield gg.erdos_renyi(90, 260, 4)
    yield gg.barabasi_albert(100, 3, 5)
    yield gg.grid(9, 11, 0.05, 6)


@pytest.mark.parametrize("h", [1, 2, 3])
def test_loss_propagation_is_exact(h):
    rng = np.random.default_rng(h)
    for rowptr, col in graphs():
        n = rowptr.size - 1
        alive = np.ones(n, bool)
        alive[rng.choice(n, n // 5, replace=False)] = False  # an earlier peel state X
        for _ in range(4):
            X = alive.copy()
            idx = np.nonzero(X)[0]
            R = rng.choice(idx, max(1, idx.size // 12), replace=False)
            Xn = X.copy()
            Xn[R] = False
            D = dist_matrix(rowptr, col, X)
            before = O.hdegree_exact(rowptr, col, h, alive=X)
            after = O.hdegree_exact(rowptr, col, h, alive=Xn)
            for x in np.nonzero(Xn)[0]:
                dR = D[R, x].min()
                if dR > h:
                    assert after[x] == before[x]
                elif dR == h:
                    lost = int((D[R, x] <= h).sum())
                    assert after[x] == before[x] - lost, (x, h)
            alive = Xn


def level_members(rowptr, col, r, i, k, alive, v):
    ball = O.hball(rowptr, col, int(v), i, alive=alive)
    return {int(u) for u in ball if r[u] >= k}


@pytest.mark.parametrize("h,M", [(2, 4), (3, 5), (3, 8)])
def test_rank_filter_never_skips_a_change(h, M):
    rng = np.random.default_rng(10 * h + M)
    for rowptr, col in graphs():
        n = rowptr.size - 1
        r = O.ranks(n, 7)
        X = np.ones(n, bool)
        for _ in range(3):
            idx = np.nonzero(X)[0]
            R = rng.choice(idx, max(1, idx.size // 15), replace=False)
            Xn = X.copy()
            Xn[R] = False
            _, _, _, _, lk_old = O.estimate_dp(rowptr, col, r, h, M, alive=X, levels=True)
            _, _, _, _, lk_new = O.estimate_dp(rowptr, col, r, h, M, alive=Xn, levels=True)
            adjR = np.zeros(n, bool)
            for u in R:
                adjR[col[rowptr[u]:rowptr[u + 1]]] = True
            for i in range(1, h + 1):
                old = {v: level_members(rowptr, col, r, i, lk_old[v, i - 1], X, v)
                       for v in np.nonzero(Xn)[0]}
                new = {v: level_members(rowptr, col, r, i, lk_new[v, i - 1], Xn, v)
                       for v in np.nonzero(Xn)[0]}
                if i == 1:
                    prev_rho = {}
                for v in np.nonzero(Xn)[0]:
                    changed = old[v] != new[v] or lk_old[v, i - 1] != lk_new[v, i - 1]
                    # a level never rises, and members enter only below the old level
                    assert lk_new[v, i - 1] <= lk_old[v, i - 1]
                    assert all(r[u] < lk_old[v, i - 1] for u in new[v] - old[v])
                    if not changed or adjR[v]:
                        continue
                    assert i >= 2, "a level-1 list changes only next to a removed node"
                    nbrs = [w for w in col[rowptr[v]:rowptr[v + 1]] if Xn[w]]
                    kv = int(lk_old[v, i - 1])
                    assert any(prev_rho.get(int(w), -2) >= kv - 1 for w in nbrs), (v, i)
                # rho of this level's changed lists, for the next level
                rho = {}
                for v in np.nonzero(Xn)[0]:
                    if old[v] == new[v] and lk_old[v, i - 1] == lk_new[v, i - 1]:
                        continue
                    left = [int(r[u]) for u in old[v] - new[v]]
                    t = max(left) if left else -1
                    if lk_new[v, i - 1] != lk_old[v, i - 1]:
                        t = max(t, int(lk_old[v, i - 1]) - 1)
                    rho[int(v)] = t
                prev_rho = rho
            X = Xn


def test_bit_parallel_two_balls_equal_the_definition():
    rng = np.random.default_rng(11)
    for rowptr, col in graphs():
        n = rowptr.size - 1
        deg = np.diff(rowptr)
        src_all = np.nonzero(deg > 0)[0]
        batch = rng.choice(src_all, min(40, src_all.size), replace=False)
        # m1 as Python ints (bit j per source), filter per 4-id group
        m1 = [0] * n
        for j, s_ in enumerate(batch):
            for u in col[rowptr[s_]:rowptr[s_ + 1]]:
                m1[u] |= 1 << j
        filt = np.zeros((n + 3) // 4, bool)
        for u in range(n):
            if m1[u]:
                filt[u >> 2] = True
        ball = [0] * n
        for x in range(n):
            if deg[x] == 0:
                continue
            b = m1[x]
            for u in col[rowptr[x]:rowptr[x + 1]]:
                if filt[u >> 2]:
                    b |= m1[u]
                else:
                    assert m1[u] == 0  # the filter only drops entries with no source bits
            ball[x] = b
        want = O.hdegree_exact(rowptr, col, 2)
        for j, s_ in enumerate(batch):
            members = sum(1 for x in range(n) if (ball[x] >> j) & 1)
            assert members - 1 == want[s_], (j, s_)
