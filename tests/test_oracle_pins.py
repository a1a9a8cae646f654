"""Pins of the CPU oracle against facts fixed outside the oracle itself.

Each test checks the oracle against one of: values the paper prints (Table 1's
M), a published generator test vector, hand-worked fixtures, brute force on
tiny graphs (scipy shortest paths, exhaustive subsets), closed forms,
textbook special cases (h = 1 k-cores; M >= n), and the paper's deterministic
propositions (Prop. 3.1, Prop. 4.2, the second claim of Prop. 4.4).
"""
import itertools

import numpy as np
import pytest
from scipy.sparse import csr_matrix
from scipy.sparse.csgraph import shortest_path

import oracle as O
from paper_2112_06154_gb300 import graphgen as gg
from tests.conftest import read_golden


# ---------------------------------------------------------------- helpers

def induced_dist(rowptr, col, alive):
    """All-pairs hop distances inside the induced subgraph (scipy)."""
    n = rowptr.size - 1
    alive = np.asarray(alive, dtype=bool)
    src = np.repeat(np.arange(n), np.diff(rowptr))
    keep = alive[src] & alive[col]
    A = csr_matrix((np.ones(keep.sum()), (src[keep], col[keep])), shape=(n, n))
    return shortest_path(A, unweighted=True, directed=False)


def brute_ball_sizes(rowptr, col, h, alive=None):
    n = rowptr.size - 1
    alive = np.ones(n, bool) if alive is None else np.asarray(alive, bool)
    D = induced_dist(rowptr, col, alive)
    out = np.zeros(n, dtype=np.int64)
    for v in range(n):
        if alive[v]:
            out[v] = int(((D[v] <= h) & alive).sum()) - 1
    return out


def textbook_kcore(rowptr, col):
    """Ordinary k-cores (h = 1) by repeated removal of a minimum-degree vertex
    (Seidman 1983; the O(m) bucket form is Batagelj-Zaversnik 2003)."""
    n = rowptr.size - 1
    cur = np.diff(rowptr).astype(np.int64)
    core = np.zeros(n, dtype=np.int64)
    alive = np.ones(n, bool)
    k = 0
    for _ in range(n):
        cand = np.where(alive)[0]
        v = cand[np.argmin(cur[cand])]
        k = max(k, cur[v])
        core[v] = k
        alive[v] = False
        for u in col[rowptr[v]:rowptr[v + 1]]:
            if alive[u]:
                cur[u] -= 1
    return core


def exhaustive_core(n, dfun):
    """c(v) = max over subsets S containing v of min_{u in S} d(u; S)."""
    best = np.zeros(n, dtype=np.int64)
    for mask in range(1, 1 << n):
        S = np.array([(mask >> i) & 1 for i in range(n)], dtype=bool)
        d = dfun(S)
        val = min(int(d[u]) for u in np.where(S)[0])
        for u in np.where(S)[0]:
            if val > best[u]:
                best[u] = val
    return best


def peel_to_kcore(n, dfun, k):
    """Largest set where every member has d >= k: delete violators until none."""
    S = np.ones(n, dtype=bool)
    while True:
        d = dfun(S)
        bad = S & (d < k)
        if not bad.any():
            return S
        S &= ~bad


# ---------------------------------------------------------------- ranks and M

def test_splitmix64_published_vector():
    want = np.array([int(r[0]) for r in read_golden("splitmix64_seed1234567.txt")], dtype=np.uint64)
    got = O.splitmix64_stream(1234567, len(want))
    assert (got == want).all()


def test_ranks_are_trailing_zeros_of_stream():
    stream = O.splitmix64_stream(7, 4096)
    r = O.ranks(4096, 7)
    for x, rr in zip(stream.tolist(), r.tolist()):
        tz = (x & -x).bit_length() - 1 if x else 64
        assert rr == min(tz, 31)


def test_rank_frequencies_geometric():
    n = 1 << 20
    r = O.ranks(n, 1)
    for j in range(0, 13):
        p = 2.0 ** -j
        cnt = int((r >= j).sum())
        sd = np.sqrt(n * p * (1 - p)) if j > 0 else 0.0
        assert abs(cnt - n * p) <= 5 * sd + 1e-9, (j, cnt, n * p)


def test_budget_M_matches_table1():
    for name, n, M in read_golden("table1_budget_M.txt"):
        assert O.budget_M(int(n), 0.5, 0.05) == int(M), name


# ---------------------------------------------------------------- h-degrees

@pytest.mark.parametrize("seed", range(6))
@pytest.mark.parametrize("h", [1, 2, 3, 4])
def test_hdegree_brute_force(seed, h):
    rp, cl = gg.random_small(14, 0.22, seed)
    rng = np.random.default_rng(seed + 100)
    for alive in [None, rng.random(14) < 0.7]:
        got = O.hdegree_exact(rp, cl, h, alive=alive)
        want = brute_ball_sizes(rp, cl, h, alive)
        if alive is not None:
            got = np.where(alive, got, 0)
        assert (got == want).all()


def test_hdegree_closed_forms():
    for n in [1, 2, 5, 9]:
        rp, cl = gg.complete(n)
        for h in [1, 2, 3]:
            assert (O.hdegree_exact(rp, cl, h) == n - 1).all()
    for n in [2, 3, 7, 12]:
        rp, cl = gg.path(n)
        for h in [1, 2, 3, 4]:
            i = np.arange(n)
            assert (O.hdegree_exact(rp, cl, h) == np.minimum(i, h) + np.minimum(n - 1 - i, h)).all()
    for n in [3, 5, 8, 11]:
        rp, cl = gg.cycle(n)
        for h in [1, 2, 3, 4]:
            assert (O.hdegree_exact(rp, cl, h) == min(2 * h, n - 1)).all()
    rp, cl = gg.star(6)
    assert list(O.hdegree_exact(rp, cl, 1)) == [6] + [1] * 6
    assert (O.hdegree_exact(rp, cl, 2) == 6).all()
    a, b = 5, 7
    rp, cl = gg.grid(a, b)
    for h in [1, 2, 3]:
        want = []
        for x in range(a):
            for y in range(b):
                cnt = sum(1 for dx in range(-h, h + 1) for dy in range(-h, h + 1)
                          if abs(dx) + abs(dy) <= h and 0 <= x + dx < a and 0 <= y + dy < b)
                want.append(cnt - 1)
        assert (O.hdegree_exact(rp, cl, h) == np.array(want)).all()


def test_fixed_counts_brute_force():
    rp, cl = gg.random_small(14, 0.3, 3)
    r = O.ranks(14, 11)
    D = induced_dist(rp, cl, np.ones(14, bool))
    for h in [1, 2, 3]:
        cnt = O.fixed_counts(rp, cl, r, h, 0, 6)
        assert (cnt[:, 0] == O.hdegree_exact(rp, cl, h)).all()
        for v in range(14):
            for j in range(7):
                want = sum(1 for u in range(14) if u != v and D[v, u] <= h and r[u] >= j)
                assert cnt[v, j] == want


# ---------------------------------------------------------------- the estimate

def test_estimate_hand_worked_star():
    rp, cl = gg.star(7)
    r = np.array([1, 0, 2, 1, 0, 3, 1, 0], dtype=np.uint8)
    for h, M, v, est, k, bs in read_golden("estimate_star7.txt"):
        h, M, v = int(h), int(M), int(v)
        for fn in (O.estimate_def, O.estimate_dp):
            e, kk, b = fn(rp, cl, r, h, M)
            assert (int(e[v]), int(kk[v]), int(b[v])) == (int(est), int(k), int(bs)), (fn.__name__, h, M, v)


def test_estimate_reduces_to_exact_when_M_ge_n():
    rp, cl = gg.chung_lu(3000, 8, 2.5, 300, 5)
    r = O.ranks(3000, 1)
    for h in [1, 2, 3]:
        e, k, b = O.estimate_dp(rp, cl, r, h, 3000)
        assert (k == 0).all()
        assert (e.astype(np.int64) == O.hdegree_exact(rp, cl, h)).all()


@pytest.mark.parametrize("h", [1, 2, 3, 4])
@pytest.mark.parametrize("M", [1, 2, 5, 16, 64])
def test_level_recursion_equals_definition(h, M):
    """Prop. 3.1 + Alg. 2 (lists) and Def. 4.1 (whole ball) agree."""
    rp, cl = gg.erdos_renyi(400, 1600, 21)
    r = O.ranks(400, 3)
    rng = np.random.default_rng(h * 100 + M)
    for alive in [None, rng.random(400) < 0.6]:
        a = O.estimate_def(rp, cl, r, h, M, alive=alive)
        b = O.estimate_dp(rp, cl, r, h, M, alive=alive)
        for x, y in zip(a, b):
            assert (x == y).all()


@pytest.mark.parametrize("h,M", [(1, 5), (2, 3), (3, 16), (4, 7)])
def test_level_by_level_ranges_equal_definition(h, M):
    """dp_level chained over levels and cut into node ranges gives Def. 4.1 on
    the whole ball (est, k, |B|), and each list is the rank filter of the ball
    at its level, in rank order (Prop. 3.1)."""
    rp, cl = gg.chung_lu(900, 9, 2.4, 120, 33)
    n = rp.size - 1
    r = O.ranks(n, 2)
    prev = None
    for i in range(1, h + 1):
        parts = [O.dp_level(rp, cl, r, i, M, prev, a, min(n, a + 97)) for a in range(0, n, 97)]
        k = np.concatenate([p[0] for p in parts])
        size = np.concatenate([p[1] for p in parts])
        est = np.concatenate([p[2] for p in parts])
        ids = np.concatenate([p[4] for p in parts])
        off = np.zeros(n + 1, np.int64)
        np.cumsum(size, out=off[1:])
        prev = (off, ids, k)
        we, wk, ws = O.estimate_def(rp, cl, r, i, M)
        assert (est == we).all() and (k == wk).all() and (size == ws).all()
        for v in (0, 17, 450, n - 1):
            ball = O.hball(rp, cl, v, i)
            want = sorted((u for u in ball if r[u] >= k[v]), key=lambda u: (-int(r[u]), u))
            assert list(ids[off[v]:off[v + 1]]) == want


def test_level_thresholds_monotone_prop31():
    """k[v,i] >= k[w,i-1] for w adjacent to v, and |B[v,i]| <= M (Prop. 3.1)."""
    rp, cl = gg.chung_lu(2000, 10, 2.3, 400, 4)
    r = O.ranks(2000, 5)
    h, M = 4, 12
    _, _, _, ls, lk = O.estimate_dp(rp, cl, r, h, M, levels=True)
    assert (ls <= M).all()
    src = np.repeat(np.arange(2000), np.diff(rp))
    for i in range(1, h):
        assert (lk[src, i] >= lk[cl, i - 1]).all()
        assert (lk[:, i] >= lk[:, i - 1]).all()


def test_estimate_monotone_under_removal_prop42():
    rp, cl = gg.erdos_renyi(300, 1500, 8)
    r = O.ranks(300, 9)
    rng = np.random.default_rng(0)
    alive = np.ones(300, bool)
    prev = O.estimate_def(rp, cl, r, 3, 8, alive=alive)[0]
    for _ in range(10):
        alive &= rng.random(300) < 0.85
        cur = O.estimate_def(rp, cl, r, 3, 8, alive=alive)[0]
        assert (cur[alive] <= prev[alive]).all()
        prev = cur


def test_estimate_thresholded_agrees_with_exact_below_M():
    """min(est, M) == min(deg_h, M): the deterministic core of Prop. 4.4's 2nd claim."""
    rp, cl = gg.chung_lu(3000, 12, 2.4, 500, 6)
    r = O.ranks(3000, 2)
    for h in [1, 2, 3]:
        for M in [4, 32, 200]:
            e = O.estimate_dp(rp, cl, r, h, M)[0].astype(np.int64)
            d = O.hdegree_exact(rp, cl, h).astype(np.int64)
            assert (np.minimum(e, M) == np.minimum(d, M)).all()


# ---------------------------------------------------------------- peeling

@pytest.mark.parametrize("seed", range(4))
@pytest.mark.parametrize("h", [1, 2, 3])
def test_exact_core_exhaustive(seed, h):
    n = 10
    rp, cl = gg.random_small(n, 0.3, 40 + seed)
    want = exhaustive_core(n, lambda S: brute_ball_sizes(rp, cl, h, S))
    got, _, _ = O.core_exact(rp, cl, h)
    assert (got == want).all()


@pytest.mark.parametrize("seed", range(3))
@pytest.mark.parametrize("h,M", [(1, 2), (2, 3), (3, 2)])
def test_sampled_core_exhaustive(seed, h, M):
    """Peel output equals max over subsets of min estimate (generalized cores)."""
    n = 10
    rp, cl = gg.random_small(n, 0.35, 70 + seed)
    r = O.ranks(n, seed + 1)
    want = exhaustive_core(n, lambda S: O.estimate_def(rp, cl, r, h, M, alive=S)[0].astype(np.int64))
    for mode in [0, O.SEQUENTIAL, O.DEFINITION, O.REFRESH_ALL]:
        got, _, _ = O.core_sampled(rp, cl, r, h, M, mode)
        assert (got.astype(np.int64) == want).all(), mode


def test_h1_equals_textbook_kcore():
    for seed in range(3):
        rp, cl = gg.chung_lu(1500, 9, 2.3, 200, seed)
        assert (O.core_exact(rp, cl, 1)[0] == textbook_kcore(rp, cl)).all()


def test_core_closed_forms():
    for n in [2, 6]:
        rp, cl = gg.complete(n)
        for h in [1, 2]:
            assert (O.core_exact(rp, cl, h)[0] == n - 1).all()
    for n in [4, 9]:
        rp, cl = gg.path(n)
        for h in [1, 2, 3]:
            assert (O.core_exact(rp, cl, h)[0] == min(h, n - 1)).all()
        rp, cl = gg.cycle(n)
        for h in [1, 2, 3]:
            assert (O.core_exact(rp, cl, h)[0] == min(2 * h, n - 1)).all()
    rp, cl = gg.star(5)
    assert (O.core_exact(rp, cl, 1)[0] == 1).all()
    assert (O.core_exact(rp, cl, 2)[0] == 5).all()
    rp, cl = gg.grid(4, 6)
    assert (O.core_exact(rp, cl, 1)[0] == 2).all()


@pytest.mark.parametrize("h", [1, 2, 3])
def test_core_level_sets_are_maximal_cores(h):
    """Each {c >= k} is the (k,h)-core obtained by deleting violators."""
    rp, cl = gg.chung_lu(500, 6, 2.5, 60, 12)
    n = 500
    core, _, _ = O.core_exact(rp, cl, h)
    dfun = lambda S: np.where(S, O.hdegree_exact(rp, cl, h, alive=S), 0)
    for k in sorted(set(core.tolist()))[::3] + [int(core.max())]:
        assert (peel_to_kcore(n, dfun, k) == (core >= k)).all()
    r = O.ranks(n, 4)
    M = 10
    cs, _, _ = O.core_sampled(rp, cl, r, h, M)
    dfun = lambda S: np.where(S, O.estimate_def(rp, cl, r, h, M, alive=S)[0].astype(np.int64), 0)
    for k in sorted(set(cs.tolist()))[::4] + [int(cs.max())]:
        assert (peel_to_kcore(n, dfun, k) == (cs >= k)).all()


def test_schedules_and_refresh_agree():
    rp, cl = gg.erdos_renyi(600, 3000, 2)
    r = O.ranks(600, 1)
    for h in [2, 3]:
        base, _, _ = O.core_exact(rp, cl, h)
        for mode in [O.SEQUENTIAL, O.REFRESH_ALL, O.SEQUENTIAL | O.REFRESH_ALL]:
            assert (O.core_exact(rp, cl, h, mode)[0] == base).all()
        for M in [8, 40]:
            sb, _, _ = O.core_sampled(rp, cl, r, h, M)
            for mode in [O.SEQUENTIAL, O.REFRESH_ALL, O.DEFINITION]:
                assert (O.core_sampled(rp, cl, r, h, M, mode)[0] == sb).all()


def test_core_monotone_in_h_and_prop44():
    rp, cl = gg.chung_lu(1200, 8, 2.4, 150, 3)
    r = O.ranks(1200, 1)
    prev_e = prev_s = None
    for h in [1, 2, 3]:
        ce = O.core_exact(rp, cl, h)[0].astype(np.int64)
        for M in [16, 100]:
            cs = O.core_sampled(rp, cl, r, h, M)[0].astype(np.int64)
            # Prop. 4.4, second claim: cores up to M are exact
            assert (np.minimum(cs, M) == np.minimum(ce, M)).all()
        cs = O.core_sampled(rp, cl, r, h, 16)[0].astype(np.int64)
        if prev_e is not None:
            assert (ce >= prev_e).all()
            assert (cs >= prev_s).all()
        prev_e, prev_s = ce, cs


def test_sampled_core_equals_exact_when_M_ge_n():
    rp, cl = gg.erdos_renyi(800, 3200, 5)
    r = O.ranks(800, 1)
    for h in [1, 2, 3]:
        assert (O.core_sampled(rp, cl, r, h, 800)[0].astype(np.int64) ==
                O.core_exact(rp, cl, h)[0]).all()


def test_round_of_is_consistent():
    """Removal rounds are nondecreasing in core value; within a round one value."""
    rp, cl = gg.erdos_renyi(500, 2500, 9)
    core, rnd, steps = O.core_exact(rp, cl, 2)
    assert rnd.max() == steps - 1
    order = np.argsort(rnd, kind="stable")
    assert (np.diff(core[order]) >= 0).all()
    for k in range(steps):
        vals = np.unique(core[rnd == k])
        assert vals.size == 1


# --------------------------------------------------------------- EstDense (Alg. 7)

def brute_pairs_within_h(rowptr, col, h, alive):
    """|E_h(X)|: unordered pairs of X joined by a path of at most h edges in G[X]."""
    D = induced_dist(rowptr, col, alive)
    idx = np.nonzero(alive)[0]
    sub = D[np.ix_(idx, idx)]
    return int(((sub <= h) & (sub > 0)).sum() // 2)


@pytest.mark.parametrize("h", [1, 2, 3])
def test_dense_curve_exact_counts_pairs(h):
    # the identity behind Alg. 7: sum_v deg_h(v; X) = 2 |E_h(X)|, on every candidate set
    rowptr, col = gg.erdos_renyi(40, 70, 31 + h)
    n = rowptr.size - 1
    r = O.ranks(n, 3)
    _, rnd, _ = O.core_exact(rowptr, col, h)
    rounds = int(rnd.max()) + 1
    total, size = O.dense_curve(rowptr, col, r, h, 8, True, rnd, rounds)
    for q in range(rounds):
        alive = rnd >= q
        assert size[q] == alive.sum()
        assert total[q] == 2 * brute_pairs_within_h(rowptr, col, h, alive)


def test_dense_curve_closed_forms():
    # K_n: every pair at distance 1, sum = n (n - 1); star with L leaves at h = 2:
    # every node reaches all others, sum = (L + 1) L
    for n in (2, 5, 9):
        rowptr, col = gg.complete(n)
        total, size = O.dense_curve(rowptr, col, O.ranks(n, 1), 1, 4, True, np.zeros(n, np.int32), 1)
        assert total[0] == n * (n - 1) and size[0] == n
    for L in (3, 7):
        rowptr, col = gg.star(L)
        n = L + 1
        total, _ = O.dense_curve(rowptr, col, O.ranks(n, 1), 2, 4, True, np.zeros(n, np.int32), 1)
        assert total[0] == (L + 1) * L


def test_dense_curve_sampled_is_exact_when_M_ge_n():
    rowptr, col = gg.erdos_renyi(60, 150, 41)
    n = rowptr.size - 1
    r = O.ranks(n, 9)
    _, rnd, _ = O.core_exact(rowptr, col, 2)
    rounds = int(rnd.max()) + 1
    ex, _ = O.dense_curve(rowptr, col, r, 2, n, True, rnd, rounds)
    sa, _ = O.dense_curve(rowptr, col, r, 2, n, False, rnd, rounds)
    assert np.array_equal(ex, sa)


def test_dense_curve_sampled_is_sum_of_definition_estimates():
    # sampled form: Def. 4.1 per node on X_q, summed; a schedule of one node per
    # round gives the paper's n candidates
    rowptr, col = gg.barabasi_albert(50, 3, 5)
    n = rowptr.size - 1
    r = O.ranks(n, 11)
    order = np.random.default_rng(2).permutation(n).astype(np.int32)
    total, size = O.dense_curve(rowptr, col, r, 2, 6, False, order, n)
    for q in (0, 7, 31, n - 1):
        alive = order >= q
        est, _, _ = O.estimate_def(rowptr, col, r, 2, 6, alive=alive)
        assert total[q] == int(est[alive].astype(np.uint64).sum())
        assert size[q] == n - q


@pytest.mark.parametrize("h,M,eps", [(1, 4, 0.5), (2, 5, 0.3), (2, 3, 0.5), (3, 6, 0.2)])
def test_dense_curve_pruned(h, M, eps):
    """The faster EstDense variant (Sec. 6): nodes with c'(v) < gamma k' are
    dropped first.  Kept set by its definition; exact sums are twice the
    brute-force pair counts inside each pruned candidate; along Core's own
    order the pruned candidates are the unpruned suffixes from the first
    round whose nodes all pass (c' only grows along Core's order)."""
    rowptr, col = gg.chung_lu(120, 6, 2.3, 25, 13 + h)
    n = rowptr.size - 1
    r = O.ranks(n, 4)
    core, rnd, _ = O.core_sampled(rowptr, col, r, h, M)
    rounds = int(rnd.max()) + 1
    gamma = (1 - eps) / (1 + eps)
    for exact in (True, False):
        total, size, keep = O.dense_curve_pruned(rowptr, col, r, h, M, exact, rnd, rounds, core, eps)
        want_keep = core.astype(np.float64) >= gamma * float(core.max())
        assert np.array_equal(keep.astype(bool), want_keep)
        full, fsize = O.dense_curve(rowptr, col, r, h, M, exact, rnd, rounds)
        q0 = int(rnd[want_keep].min())
        assert (rnd[~want_keep] < q0).all()
        assert np.array_equal(total[q0:], full[q0:]) and np.array_equal(size[q0:], fsize[q0:])
        assert (total[:q0] == full[q0]).all() and (size[:q0] == fsize[q0]).all()
        if exact:
            for q in range(rounds):
                alive = (rnd >= q) & want_keep
                assert size[q] == alive.sum()
                assert total[q] == 2 * brute_pairs_within_h(rowptr, col, h, alive)


def test_dense_curve_rejects_bad_schedules():
    rowptr, col = gg.erdos_renyi(10, 12, 1)
    with pytest.raises(Exception):
        O.dense_curve(rowptr, col, O.ranks(10, 1), 2, 4, True, np.full(10, 3, np.int32), 2)
