/*
 * khoracle.c -- CPU oracle for the distance-generalized (k,h)-core method of
 * Tatti, "Fast computation of distance-generalized cores using sampling".
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, single-threaded
 * statement of what the GPU library must compute.  Only the test-suite, the
 * smoke check and the benchmark's CPU-baseline leg may load it.  It shares no
 * code, header, table or helper with the CUDA library.
 *
 * Every routine follows one passage of the paper:
 *   kho_splitmix64_next   SplitMix64 (Steele, Lea, Flood 2014), the seeded
 *                         generator behind the geometric ranks r[v] (Sec. 3).
 *   kho_ranks             r[v] ~ geo(1/2) with P(r >= j) = 2^-j (Sec. 3, Alg. 4).
 *   kho_budget_M          M of Eq. (buffer), C = log(2n/delta) (Sec. 3).
 *   kho_hball             N(v; h, X): nodes reachable by an h-path inside X (Sec. 2).
 *   kho_hdegree_exact     deg_h(v; X) = |N(v; h, X)| - 1 (Sec. 2).
 *   kho_fixed_counts      |{u in N(v;h,X) \ {v} : r[u] >= j}|: Alg. 1 with the
 *                         level forced to j.
 *   kho_estimate_def      Def. 4.1 applied to the rank list of N(v;h,X), v first
 *                         (equal to Alg. 1's output, Sec. 4).
 *   kho_estimate_dp       B[v,i], k[v,i] by the naive Compute (Alg. 2) level by
 *                         level (Prop. 3.1), then Estimate (Alg. 1).
 *   kho_dp_level          the same Compute for one level and a range of nodes,
 *                         the previous level given as arrays (large graphs).
 *   kho_core_exact        ExactCore (Sec. 2): peel by smallest deg_h.
 *   kho_core_sampled      Core (Alg. 4) with naive Update (Alg. 3).
 *   kho_dense_curve       EstDense (Alg. 7, Sec. 6): along a removal order, the
 *                         sum of d(v; X) over each candidate set X.
 *   kho_dense_curve_pruned  the same after removing the nodes with
 *                         c'(v) < gamma k' (the faster variant of Sec. 6).
 *
 * Peeling schedule.  Both peels support two schedules that must give the same
 * core map because d(v; X) never grows when X shrinks (exact: N shrinks; sampled:
 * Prop. 4.2):
 *   sequential  one node per step, smallest d first (ties: k[v,h], then id),
 *               c = max(c, d[u]) -- Alg. 4's loop;
 *   bucket      c = max(c, min d); remove every alive v with d[v] <= c at once.
 * After a removal the oracle either recomputes every alive node ("refresh all")
 * or only the affected ones (exact: the h-ball of the removed set in the old
 * graph; sampled: Alg. 3's propagation of changed B/k level by level).
 *
 * Readings where the paper is silent or loose (each also listed in the design
 * notes): ranks are capped at 31 (ctz of a 64-bit word OR 2^31); M is used as
 * the integer floor(M) in Alg. 1 as well as in Alg. 2; an h-path has at most h
 * edges; ties inside a rank are ordered by node id.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define KHO_OK 0
#define KHO_ENOMEM -3
#define KHO_EINVAL -1

/* ------------------------------------------------------------------------ */
/* Ranks                                                                     */
/* ------------------------------------------------------------------------ */

/* One step of SplitMix64: advance the state by the golden-ratio increment and
 * return the finalised value (Steele, Lea, Flood, OOPSLA 2014). */
uint64_t kho_splitmix64_next(uint64_t *state)
{
    uint64_t z;
    *state = *state + 0x9E3779B97F4A7C15ULL;
    z = *state;
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}

/* r[u] = number of trailing zero bits of the u-th SplitMix64 output (seeded by
 * `seed`), capped at 31: P(r >= j) = 2^-j, the geometric(1/2) rank of Sec. 3. */
void kho_ranks(int64_t n, uint64_t seed, uint8_t *r)
{
    uint64_t state = seed;
    for (int64_t u = 0; u < n; u++) {
        uint64_t x = kho_splitmix64_next(&state);
        int tz = 0;
        while (tz < 31 && ((x >> tz) & 1ULL) == 0)
            tz++;
        r[u] = (uint8_t)tz;
    }
}

/* Eq. (buffer): M = 1 + 4(2+eps)/eps^2 (C + log 8), C = log(2n/delta), natural
 * logarithm, used as floor(M). */
int64_t kho_budget_M(int64_t n, double eps, double delta)
{
    double C = log(2.0 * (double)n / delta);
    double M = 1.0 + 4.0 * (2.0 + eps) / (eps * eps) * (C + log(8.0));
    return (int64_t)floor(M);
}

/* ------------------------------------------------------------------------ */
/* h-neighbourhoods                                                          */
/* ------------------------------------------------------------------------ */

static int is_alive(const uint8_t *alive, int64_t v)
{
    return alive == NULL || alive[v] != 0;
}

/* N(v; h, X) by breadth-first search inside X (alive nodes), at most h edges.
 * Writes the members (v first) to out[] and returns their number.  dist[] is
 * caller scratch of length n, all -1 on entry, and is restored to -1. */
int64_t kho_hball(int64_t n, const int64_t *rowptr, const int32_t *col,
                  const uint8_t *alive, int64_t v, int32_t h,
                  int32_t *out, int32_t *dist)
{
    (void)n;
    int64_t head = 0, tail = 0;
    if (!is_alive(alive, v))
        return 0;
    out[tail++] = (int32_t)v;
    dist[v] = 0;
    while (head < tail) {
        int32_t w = out[head++];
        if (dist[w] == h)
            continue;
        for (int64_t e = rowptr[w]; e < rowptr[w + 1]; e++) {
            int32_t u = col[e];
            if (!is_alive(alive, u) || dist[u] >= 0)
                continue;
            dist[u] = dist[w] + 1;
            out[tail++] = u;
        }
    }
    for (int64_t q = 0; q < tail; q++)
        dist[out[q]] = -1;
    return tail;
}

/* deg_h(v; X) = |N(v;h,X)| - 1 for alive v; 0 for removed v. */
int kho_hdegree_exact(int64_t n, const int64_t *rowptr, const int32_t *col,
                      const uint8_t *alive, int32_t h, int32_t *deg)
{
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!buf || !dist) {
        free(buf);
        free(dist);
        return KHO_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++)
        dist[i] = -1;
    for (int64_t v = 0; v < n; v++) {
        int64_t s = kho_hball(n, rowptr, col, alive, v, h, buf, dist);
        deg[v] = s > 0 ? (int32_t)(s - 1) : 0;
    }
    free(buf);
    free(dist);
    return KHO_OK;
}

/* cnt[v*(jhi-jlo+1) + (j-jlo)] = |{u in N(v;h,X), u != v : r[u] >= j}|. */
int kho_fixed_counts(int64_t n, const int64_t *rowptr, const int32_t *col,
                     const uint8_t *alive, const uint8_t *r, int32_t h,
                     int32_t jlo, int32_t jhi, int32_t *cnt)
{
    int32_t nj = jhi - jlo + 1;
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!buf || !dist) {
        free(buf);
        free(dist);
        return KHO_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++)
        dist[i] = -1;
    for (int64_t v = 0; v < n; v++) {
        int64_t s = kho_hball(n, rowptr, col, alive, v, h, buf, dist);
        for (int32_t j = jlo; j <= jhi; j++) {
            int32_t c = 0;
            for (int64_t q = 1; q < s; q++) /* q = 0 is v itself */
                if (r[buf[q]] >= j)
                    c++;
            cnt[v * nj + (j - jlo)] = c;
        }
    }
    free(buf);
    free(dist);
    return KHO_OK;
}

/* Def. 4.1 on a rank list x_1..x_d (x_1 belongs to v):
 * S_i = #{j : x_j >= i}, T_i = #{j >= 2 : x_j >= i}, k = min{i >= 0 : S_i <= M},
 * est = max(T_k 2^k, M 2^(k-1)) if k > 0 else T_k 2^k. */
static uint64_t def41(const uint8_t *x, int64_t d, int64_t M, uint8_t *k_out,
                      int32_t *s_out)
{
    int k = 0;
    int64_t S, T;
    for (;;) {
        S = 0;
        for (int64_t j = 0; j < d; j++)
            if (x[j] >= k)
                S++;
        if (S <= M)
            break;
        k++;
    }
    T = 0;
    for (int64_t j = 1; j < d; j++)
        if (x[j] >= k)
            T++;
    uint64_t est = (uint64_t)T << k;
    if (k > 0) {
        uint64_t floor_term = (uint64_t)M << (k - 1);
        if (floor_term > est)
            est = floor_term;
    }
    if (k_out)
        *k_out = (uint8_t)k;
    if (s_out)
        *s_out = (int32_t)S;
    return est;
}

/* Estimate of every alive node straight from Def. 4.1 on N(v;h,X):
 * est[v], the level k (= k[v,h]) and |B[v,h]| = S_k.  Removed nodes get 0. */
int kho_estimate_def(int64_t n, const int64_t *rowptr, const int32_t *col,
                     const uint8_t *alive, const uint8_t *r, int32_t h, int64_t M,
                     uint64_t *est, uint8_t *kap, int32_t *bsize)
{
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *x = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!buf || !dist || !x || M < 1) {
        free(buf);
        free(dist);
        free(x);
        return M < 1 ? KHO_EINVAL : KHO_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++)
        dist[i] = -1;
    for (int64_t v = 0; v < n; v++) {
        uint8_t k = 0;
        int32_t s = 0;
        uint64_t e = 0;
        int64_t d = kho_hball(n, rowptr, col, alive, v, h, buf, dist);
        if (d > 0) {
            for (int64_t q = 0; q < d; q++)
                x[q] = r[buf[q]];
            e = def41(x, d, M, &k, &s);
        }
        if (est)
            est[v] = e;
        if (kap)
            kap[v] = k;
        if (bsize)
            bsize[v] = s;
    }
    free(buf);
    free(dist);
    free(x);
    return KHO_OK;
}

/* ------------------------------------------------------------------------ */
/* Sampled lists B[v,i], k[v,i] (Sec. 3)                                     */
/* ------------------------------------------------------------------------ */

typedef struct {
    int32_t *ids;  /* members, sorted by rank descending, then id ascending */
    int32_t size;
    int32_t cap;
    uint8_t k;
} kho_list;

typedef struct {
    int64_t n;
    const int64_t *rowptr;
    const int32_t *col;
    const uint8_t *r;
    uint8_t *alive;
    int32_t h;
    int64_t M;
    kho_list *L;       /* L[(i-1)*n + v] holds B[v,i], i = 1..h */
    int32_t *tbuf;     /* scratch for T */
    int64_t tcap;
    int32_t *prev_ids; /* scratch copy of the old B for change detection */
} kho_dp;

static const uint8_t *g_sort_r; /* rank array used by the qsort comparator */

static int cmp_rank_desc_id_asc(const void *a, const void *b)
{
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    if (g_sort_r[x] != g_sort_r[y])
        return g_sort_r[x] > g_sort_r[y] ? -1 : 1;
    return (x > y) - (x < y);
}

static kho_list *dp_list(kho_dp *dp, int32_t i, int64_t v)
{
    return &dp->L[(int64_t)(i - 1) * dp->n + v];
}

/* Naive Compute(v, i) (Alg. 2): T = {v} union the B[w,i-1] of alive w in A(v),
 * sorted by rank; k = max k[w,i-1]; if |T| > M, k = max(k, r[t_(M+1)] + 1);
 * B[v,i] = {u in T : r[u] >= k}.  B[w,0] = {w}, k[w,0] = 0.
 * Returns 1 if B[v,i] or k[v,i] changed, 0 if not, <0 on error. */
static int dp_compute(kho_dp *dp, int32_t i, int64_t v)
{
    int64_t t = 0;
    int k = 0;
    const int64_t *rp = dp->rowptr;
    /* size bound for T */
    int64_t need = 1;
    for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
        int32_t w = dp->col[e];
        if (!dp->alive[w])
            continue;
        need += (i == 1) ? 1 : dp_list(dp, i - 1, w)->size;
    }
    if (need > dp->tcap) {
        int64_t nc = need * 2;
        int32_t *nb = (int32_t *)realloc(dp->tbuf, sizeof(int32_t) * (size_t)nc);
        if (!nb)
            return KHO_ENOMEM;
        dp->tbuf = nb;
        dp->tcap = nc;
    }
    dp->tbuf[t++] = (int32_t)v;
    for (int64_t e = rp[v]; e < rp[v + 1]; e++) {
        int32_t w = dp->col[e];
        if (!dp->alive[w])
            continue;
        if (i == 1) {
            dp->tbuf[t++] = w;
        } else {
            kho_list *bw = dp_list(dp, i - 1, w);
            memcpy(dp->tbuf + t, bw->ids, sizeof(int32_t) * (size_t)bw->size);
            t += bw->size;
            if (bw->k > k)
                k = bw->k;
        }
    }
    /* sort by rank and drop repeated nodes: T is a set */
    g_sort_r = dp->r;
    qsort(dp->tbuf, (size_t)t, sizeof(int32_t), cmp_rank_desc_id_asc);
    int64_t u = 0;
    for (int64_t q = 0; q < t; q++)
        if (u == 0 || dp->tbuf[q] != dp->tbuf[u - 1])
            dp->tbuf[u++] = dp->tbuf[q];
    t = u;
    if (t > dp->M) {
        int kk = dp->r[dp->tbuf[dp->M]] + 1; /* t_(M+1), 1-based */
        if (kk > k)
            k = kk;
    }
    kho_list *bv = dp_list(dp, i, v);
    int32_t old_size = bv->size;
    uint8_t old_k = bv->k;
    memcpy(dp->prev_ids, bv->ids, sizeof(int32_t) * (size_t)old_size);
    int32_t s = 0;
    for (int64_t q = 0; q < t; q++)
        if (dp->r[dp->tbuf[q]] >= k)
            s++;
    if (s > bv->cap) {
        int32_t *nb = (int32_t *)realloc(bv->ids, sizeof(int32_t) * (size_t)s);
        if (!nb)
            return KHO_ENOMEM;
        bv->ids = nb;
        bv->cap = s;
    }
    s = 0;
    for (int64_t q = 0; q < t; q++)
        if (dp->r[dp->tbuf[q]] >= k)
            bv->ids[s++] = dp->tbuf[q];
    bv->size = s;
    bv->k = (uint8_t)k;
    if (old_k != bv->k || old_size != s)
        return 1;
    return memcmp(dp->prev_ids, bv->ids, sizeof(int32_t) * (size_t)s) != 0;
}

/* Estimate(v) (Alg. 1): d = |B[v,h] \ {v}| 2^k; if k > 0, d = max(d, M 2^(k-1)). */
static uint64_t dp_estimate(kho_dp *dp, int64_t v)
{
    kho_list *b = dp_list(dp, dp->h, v);
    int64_t others = 0;
    for (int32_t q = 0; q < b->size; q++)
        if (b->ids[q] != v)
            others++;
    uint64_t d = (uint64_t)others << b->k;
    if (b->k > 0) {
        uint64_t f = (uint64_t)dp->M << (b->k - 1);
        if (f > d)
            d = f;
    }
    return d;
}

static void dp_free(kho_dp *dp)
{
    if (dp->L) {
        for (int64_t q = 0; q < (int64_t)dp->h * dp->n; q++)
            free(dp->L[q].ids);
    }
    free(dp->L);
    free(dp->tbuf);
    free(dp->prev_ids);
}

static int dp_init(kho_dp *dp, int64_t n, const int64_t *rowptr, const int32_t *col,
                   const uint8_t *r, uint8_t *alive, int32_t h, int64_t M)
{
    memset(dp, 0, sizeof(*dp));
    dp->n = n;
    dp->rowptr = rowptr;
    dp->col = col;
    dp->r = r;
    dp->alive = alive;
    dp->h = h;
    dp->M = M;
    dp->L = (kho_list *)calloc((size_t)((int64_t)h * n + 1), sizeof(kho_list));
    dp->tcap = 1024;
    dp->tbuf = (int32_t *)malloc(sizeof(int32_t) * (size_t)dp->tcap);
    dp->prev_ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(M + 1));
    if (!dp->L || !dp->tbuf || !dp->prev_ids) {
        dp_free(dp);
        return KHO_ENOMEM;
    }
    return KHO_OK;
}

/* All levels for all alive nodes (Alg. 4's set-up loop). */
static int dp_full(kho_dp *dp)
{
    for (int32_t i = 1; i <= dp->h; i++)
        for (int64_t v = 0; v < dp->n; v++) {
            if (!dp->alive[v])
                continue;
            int rc = dp_compute(dp, i, v);
            if (rc < 0)
                return rc;
        }
    return KHO_OK;
}

/* B/k via the level recursion (Prop. 3.1 + Alg. 2), then Alg. 1.
 * level_size / level_k (optional, n*h, row v*h + (i-1)) receive |B[v,i]|, k[v,i]. */
int kho_estimate_dp(int64_t n, const int64_t *rowptr, const int32_t *col,
                    const uint8_t *alive_in, const uint8_t *r, int32_t h, int64_t M,
                    uint64_t *est, uint8_t *kap, int32_t *bsize,
                    int32_t *level_size, uint8_t *level_k)
{
    if (M < 1 || h < 1)
        return KHO_EINVAL;
    uint8_t *alive = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!alive)
        return KHO_ENOMEM;
    for (int64_t v = 0; v < n; v++)
        alive[v] = is_alive(alive_in, v) ? 1 : 0;
    kho_dp dp;
    int rc = dp_init(&dp, n, rowptr, col, r, alive, h, M);
    if (rc == KHO_OK)
        rc = dp_full(&dp);
    if (rc == KHO_OK) {
        for (int64_t v = 0; v < n; v++) {
            kho_list *b = dp_list(&dp, h, v);
            if (est)
                est[v] = alive[v] ? dp_estimate(&dp, v) : 0;
            if (kap)
                kap[v] = alive[v] ? b->k : 0;
            if (bsize)
                bsize[v] = alive[v] ? b->size : 0;
            for (int32_t i = 1; i <= h; i++) {
                kho_list *bi = dp_list(&dp, i, v);
                if (level_size)
                    level_size[v * h + (i - 1)] = alive[v] ? bi->size : 0;
                if (level_k)
                    level_k[v * h + (i - 1)] = alive[v] ? bi->k : 0;
            }
        }
    }
    dp_free(&dp);
    free(alive);
    return rc;
}

/* One level of the list recursion for a range of nodes of the whole graph
 * (Prop. 3.1 with the naive Compute of Alg. 2), from the previous level's
 * lists of every node passed in as arrays, so that a large graph can be done
 * level by level and range by range.  Level i = 1 takes B[w,0] = {w} and
 * k[w,0] = 0 (prev_* unused); level i >= 2 reads B[w,i-1] at
 * prev_ids[prev_off[w] .. prev_off[w+1]) and k[w,i-1] = prev_k[w].
 * For v = v0 + q, q < v1 - v0:
 *   T = {v} union the B[w,i-1] of w in A(v), sorted by rank (descending, ties
 *   by id) without repeats; k = max of the k[w,i-1]; if |T| > M then
 *   k = max(k, r[t_(M+1)] + 1); B[v,i] = {u in T : r[u] >= k} (at most M
 *   members, written in T's order to out_ids[q*M ..]);
 *   out_k[q] = k, out_size[q] = |B[v,i]|, and out_est[q] = Alg. 1 on
 *   (B[v,i], k): |B[v,i] \ {v}| 2^k, raised to M 2^(k-1) when k > 0. */
int kho_dp_level(int64_t n, const int64_t *rowptr, const int32_t *col, const uint8_t *r,
                 int32_t i, int64_t M, const int64_t *prev_off, const int32_t *prev_ids,
                 const uint8_t *prev_k, int64_t v0, int64_t v1, uint8_t *out_k,
                 int32_t *out_size, int32_t *out_ids, uint64_t *out_est)
{
    (void)n;
    if (i < 1 || M < 1 || v0 < 0 || v1 < v0)
        return KHO_EINVAL;
    int64_t tcap = 1024;
    int32_t *t = (int32_t *)malloc(sizeof(int32_t) * (size_t)tcap);
    if (!t)
        return KHO_ENOMEM;
    for (int64_t v = v0; v < v1; v++) {
        int64_t q = v - v0;
        int64_t need = 1;
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
            int32_t w = col[e];
            need += (i == 1) ? 1 : prev_off[w + 1] - prev_off[w];
        }
        if (need > tcap) {
            int32_t *nt = (int32_t *)realloc(t, sizeof(int32_t) * (size_t)need);
            if (!nt) {
                free(t);
                return KHO_ENOMEM;
            }
            t = nt;
            tcap = need;
        }
        int64_t len = 0;
        int k = 0;
        t[len++] = (int32_t)v;
        for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++) {
            int32_t w = col[e];
            if (i == 1) {
                t[len++] = w;
            } else {
                for (int64_t p = prev_off[w]; p < prev_off[w + 1]; p++)
                    t[len++] = prev_ids[p];
                if (prev_k[w] > k)
                    k = prev_k[w];
            }
        }
        g_sort_r = r;
        qsort(t, (size_t)len, sizeof(int32_t), cmp_rank_desc_id_asc);
        int64_t u = 0;
        for (int64_t p = 0; p < len; p++)
            if (u == 0 || t[p] != t[u - 1])
                t[u++] = t[p];
        len = u;
        if (len > M) {
            int kk = r[t[M]] + 1; /* t_(M+1), 1-based */
            if (kk > k)
                k = kk;
        }
        int32_t size = 0, others = 0;
        for (int64_t p = 0; p < len; p++)
            if (r[t[p]] >= k) {
                out_ids[q * M + size] = t[p];
                size++;
                if (t[p] != (int32_t)v)
                    others++;
            }
        uint64_t d = (uint64_t)others << k;
        if (k > 0) {
            uint64_t f = (uint64_t)M << (k - 1);
            if (f > d)
                d = f;
        }
        out_k[q] = (uint8_t)k;
        out_size[q] = size;
        out_est[q] = d;
    }
    free(t);
    return KHO_OK;
}

/* ------------------------------------------------------------------------ */
/* Peeling                                                                   */
/* ------------------------------------------------------------------------ */

#define KHO_SEQUENTIAL 1u   /* one node per step (Alg. 4 loop) instead of buckets */
#define KHO_REFRESH_ALL 2u  /* recompute every alive node after each removal */
#define KHO_DEFINITION 4u   /* sampled: estimates from Def. 4.1 instead of the lists */

typedef struct {
    int32_t *items;
    int64_t size;
    uint8_t *mark;
} kho_set;

static void set_add(kho_set *s, int32_t v)
{
    if (!s->mark[v]) {
        s->mark[v] = 1;
        s->items[s->size++] = v;
    }
}

static void set_clear(kho_set *s)
{
    for (int64_t q = 0; q < s->size; q++)
        s->mark[s->items[q]] = 0;
    s->size = 0;
}

/* Alive nodes within h hops of the removed set R, measured in the graph before
 * the removal (alive_old = alive plus R).  Only these can change deg_h. */
static void affected_ball(int64_t n, const int64_t *rowptr, const int32_t *col,
                          const uint8_t *alive_old, const int32_t *R, int64_t nR,
                          int32_t h, int32_t *queue, int32_t *dist, kho_set *out)
{
    (void)n;
    int64_t head = 0, tail = 0;
    for (int64_t q = 0; q < nR; q++) {
        queue[tail++] = R[q];
        dist[R[q]] = 0;
    }
    while (head < tail) {
        int32_t w = queue[head++];
        if (dist[w] == h)
            continue;
        for (int64_t e = rowptr[w]; e < rowptr[w + 1]; e++) {
            int32_t u = col[e];
            if (!alive_old[u] || dist[u] >= 0)
                continue;
            dist[u] = dist[w] + 1;
            queue[tail++] = u;
        }
    }
    for (int64_t q = 0; q < tail; q++) {
        dist[queue[q]] = -1;
        if (q >= nR)
            set_add(out, queue[q]);
    }
}

/* ExactCore: peel by deg_h (Sec. 2).  core[v] = core number, round_of[v] =
 * index of the removal step (bucket round, or position in the sequential order).
 * Returns the number of steps, or <0 on error. */
int64_t kho_core_exact(int64_t n, const int64_t *rowptr, const int32_t *col,
                       int32_t h, uint32_t mode, int32_t *core, int32_t *round_of)
{
    if (h < 1)
        return KHO_EINVAL;
    size_t nn = (size_t)(n > 0 ? n : 1);
    uint8_t *alive = (uint8_t *)malloc(nn);
    uint8_t *alive_old = (uint8_t *)malloc(nn);
    int32_t *d = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *R = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *queue = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * nn);
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * nn);
    kho_set aff = {(int32_t *)malloc(sizeof(int32_t) * nn), 0, (uint8_t *)calloc(nn, 1)};
    int64_t steps = 0;
    if (!alive || !alive_old || !d || !R || !queue || !buf || !dist || !aff.items || !aff.mark) {
        steps = KHO_ENOMEM;
        goto out;
    }
    for (int64_t v = 0; v < n; v++) {
        alive[v] = 1;
        dist[v] = -1;
    }
    for (int64_t v = 0; v < n; v++)
        d[v] = (int32_t)(kho_hball(n, rowptr, col, alive, v, h, buf, dist) - 1);
    int64_t left = n;
    int32_t c = 0;
    while (left > 0) {
        int64_t nR = 0;
        if (mode & KHO_SEQUENTIAL) {
            int64_t best = -1;
            for (int64_t v = 0; v < n; v++)
                if (alive[v] && (best < 0 || d[v] < d[best]))
                    best = v;
            if (d[best] > c)
                c = d[best];
            R[nR++] = (int32_t)best;
        } else {
            int32_t mn = INT32_MAX;
            for (int64_t v = 0; v < n; v++)
                if (alive[v] && d[v] < mn)
                    mn = d[v];
            if (mn > c)
                c = mn;
            for (int64_t v = 0; v < n; v++)
                if (alive[v] && d[v] <= c)
                    R[nR++] = (int32_t)v;
        }
        memcpy(alive_old, alive, nn);
        for (int64_t q = 0; q < nR; q++) {
            core[R[q]] = c;
            if (round_of)
                round_of[R[q]] = (int32_t)steps;
            alive[R[q]] = 0;
        }
        left -= nR;
        steps++;
        if (mode & KHO_REFRESH_ALL) {
            for (int64_t v = 0; v < n; v++)
                if (alive[v])
                    d[v] = (int32_t)(kho_hball(n, rowptr, col, alive, v, h, buf, dist) - 1);
        } else {
            affected_ball(n, rowptr, col, alive_old, R, nR, h, queue, dist, &aff);
            for (int64_t q = 0; q < aff.size; q++) {
                int32_t v = aff.items[q];
                d[v] = (int32_t)(kho_hball(n, rowptr, col, alive, v, h, buf, dist) - 1);
            }
            set_clear(&aff);
        }
    }
out:
    free(alive);
    free(alive_old);
    free(d);
    free(R);
    free(queue);
    free(buf);
    free(dist);
    free(aff.items);
    free(aff.mark);
    return steps;
}

/* Core (Alg. 4) with the naive Update (Alg. 3).  core[v] = c'(v) (uint64,
 * estimates reach M 2^31).  Returns the number of steps, or <0 on error. */
int64_t kho_core_sampled(int64_t n, const int64_t *rowptr, const int32_t *col,
                         const uint8_t *r, int32_t h, int64_t M, uint32_t mode,
                         uint64_t *core, int32_t *round_of)
{
    if (h < 1 || M < 1)
        return KHO_EINVAL;
    size_t nn = (size_t)(n > 0 ? n : 1);
    uint8_t *alive = (uint8_t *)malloc(nn);
    uint64_t *d = (uint64_t *)malloc(sizeof(uint64_t) * nn);
    uint8_t *kh = (uint8_t *)malloc(nn);
    int32_t *R = (int32_t *)malloc(sizeof(int32_t) * nn);
    kho_set U = {(int32_t *)malloc(sizeof(int32_t) * nn), 0, (uint8_t *)calloc(nn, 1)};
    kho_set W = {(int32_t *)malloc(sizeof(int32_t) * nn), 0, (uint8_t *)calloc(nn, 1)};
    kho_dp dp;
    int have_dp = 0;
    int64_t steps = 0;
    if (!alive || !d || !kh || !R || !U.items || !U.mark || !W.items || !W.mark) {
        steps = KHO_ENOMEM;
        goto out;
    }
    for (int64_t v = 0; v < n; v++)
        alive[v] = 1;
    if (mode & KHO_DEFINITION) {
        int rc = kho_estimate_def(n, rowptr, col, alive, r, h, M, d, kh, NULL);
        if (rc < 0) {
            steps = rc;
            goto out;
        }
    } else {
        int rc = dp_init(&dp, n, rowptr, col, r, alive, h, M);
        if (rc < 0) {
            steps = rc;
            goto out;
        }
        have_dp = 1;
        rc = dp_full(&dp);
        if (rc < 0) {
            steps = rc;
            goto out;
        }
        for (int64_t v = 0; v < n; v++) {
            d[v] = dp_estimate(&dp, v);
            kh[v] = dp_list(&dp, h, v)->k;
        }
    }
    int64_t left = n;
    uint64_t c = 0;
    while (left > 0) {
        int64_t nR = 0;
        if (mode & KHO_SEQUENTIAL) {
            /* Alg. 4: argmin d, ties broken by k[v,h] (smaller first), then id */
            int64_t best = -1;
            for (int64_t v = 0; v < n; v++) {
                if (!alive[v])
                    continue;
                if (best < 0 || d[v] < d[best] || (d[v] == d[best] && kh[v] < kh[best]))
                    best = v;
            }
            if (d[best] > c)
                c = d[best];
            R[nR++] = (int32_t)best;
        } else {
            uint64_t mn = UINT64_MAX;
            for (int64_t v = 0; v < n; v++)
                if (alive[v] && d[v] < mn)
                    mn = d[v];
            if (mn > c)
                c = mn;
            for (int64_t v = 0; v < n; v++)
                if (alive[v] && d[v] <= c)
                    R[nR++] = (int32_t)v;
        }
        for (int64_t q = 0; q < nR; q++) {
            core[R[q]] = c;
            if (round_of)
                round_of[R[q]] = (int32_t)steps;
            alive[R[q]] = 0;
        }
        left -= nR;
        steps++;
        if (left == 0)
            break;
        if (mode & KHO_DEFINITION) {
            /* estimates from scratch on the new X (Def. 4.1) */
            int rc = kho_estimate_def(n, rowptr, col, alive, r, h, M, d, kh, NULL);
            if (rc < 0) {
                steps = rc;
                goto out;
            }
            continue;
        }
        if (mode & KHO_REFRESH_ALL) {
            int rc = dp_full(&dp);
            if (rc < 0) {
                steps = rc;
                goto out;
            }
            for (int64_t v = 0; v < n; v++)
                if (alive[v]) {
                    d[v] = dp_estimate(&dp, v);
                    kh[v] = dp_list(&dp, h, v)->k;
                }
            continue;
        }
        /* Alg. 3: at each level add the removed nodes' neighbours; recompute;
         * where B or k changed, queue the neighbours for the next level. */
        for (int32_t i = 1; i <= h; i++) {
            for (int64_t q = 0; q < nR; q++) {
                int32_t u = R[q];
                for (int64_t e = rowptr[u]; e < rowptr[u + 1]; e++)
                    if (alive[col[e]])
                        set_add(&U, col[e]);
            }
            for (int64_t q = 0; q < U.size; q++) {
                int32_t v = U.items[q];
                int rc = dp_compute(&dp, i, v);
                if (rc < 0) {
                    steps = rc;
                    goto out;
                }
                if (rc == 1 && i < h) {
                    for (int64_t e = rowptr[v]; e < rowptr[v + 1]; e++)
                        if (alive[col[e]])
                            set_add(&W, col[e]);
                }
                if (i == h) {
                    d[v] = dp_estimate(&dp, v);
                    kh[v] = dp_list(&dp, h, v)->k;
                }
            }
            set_clear(&U);
            /* U = W */
            for (int64_t q = 0; q < W.size; q++)
                set_add(&U, W.items[q]);
            set_clear(&W);
        }
        set_clear(&U);
    }
out:
    if (have_dp)
        dp_free(&dp);
    free(alive);
    free(d);
    free(kh);
    free(R);
    free(U.items);
    free(U.mark);
    free(W.items);
    free(W.mark);
    return steps;
}

/* ------------------------------------------------------------------------ */
/* Per-node versions for sampled checks on large graphs                      */
/* ------------------------------------------------------------------------ */

/* deg_h(v; X) for the nodes listed in vs[0..count). */
int kho_hdegree_some(int64_t n, const int64_t *rowptr, const int32_t *col,
                     const uint8_t *alive, int32_t h, const int32_t *vs, int64_t count,
                     int32_t *deg)
{
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    if (!buf || !dist) {
        free(buf);
        free(dist);
        return KHO_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++)
        dist[i] = -1;
    for (int64_t q = 0; q < count; q++) {
        int64_t s = kho_hball(n, rowptr, col, alive, vs[q], h, buf, dist);
        deg[q] = s > 0 ? (int32_t)(s - 1) : 0;
    }
    free(buf);
    free(dist);
    return KHO_OK;
}

/* Def. 4.1 estimate for the nodes listed in vs[0..count). */
int kho_estimate_def_some(int64_t n, const int64_t *rowptr, const int32_t *col,
                          const uint8_t *alive, const uint8_t *r, int32_t h, int64_t M,
                          const int32_t *vs, int64_t count,
                          uint64_t *est, uint8_t *kap, int32_t *bsize)
{
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *x = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!buf || !dist || !x || M < 1) {
        free(buf);
        free(dist);
        free(x);
        return M < 1 ? KHO_EINVAL : KHO_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++)
        dist[i] = -1;
    for (int64_t q = 0; q < count; q++) {
        uint8_t k = 0;
        int32_t s = 0;
        uint64_t e = 0;
        int64_t d = kho_hball(n, rowptr, col, alive, vs[q], h, buf, dist);
        if (d > 0) {
            for (int64_t j = 0; j < d; j++)
                x[j] = r[buf[j]];
            e = def41(x, d, M, &k, &s);
        }
        est[q] = e;
        if (kap)
            kap[q] = k;
        if (bsize)
            bsize[q] = s;
    }
    free(buf);
    free(dist);
    free(x);
    return KHO_OK;
}

/* ------------------------------------------------------------------------ */
/* EstDense (Alg. 7)                                                         */
/* ------------------------------------------------------------------------ */

/* Alg. 7 deletes the nodes in the order Core produced and, for every set X it
 * passes through, estimates the h-density |E_h(X)| / |X| from the identity
 * 2 |E_h(X)| = sum_{v in X} deg_h(v; X), with deg_h replaced by the estimate
 * of Alg. 1 in the sampled form.  The candidates here are the sets at the
 * boundaries of a removal order given by rounds: X_r = {v : round_of[v] >= r}
 * (one node per round gives the paper's n candidates).  For r in [0, rounds):
 * size[r] = |X_r| and sum[r] = sum over v in X_r of d(v; X_r), where d is
 * deg_h (exact != 0) or Def. 4.1 on the rank list of N(v; h, X_r), v first. */
static int dense_curve(int64_t n, const int64_t *rowptr, const int32_t *col, const uint8_t *r,
                       int32_t h, int64_t M, int32_t exact, const int32_t *round_of,
                       int32_t rounds, const uint8_t *keep, uint64_t *sum, int64_t *size);

int kho_dense_curve(int64_t n, const int64_t *rowptr, const int32_t *col, const uint8_t *r,
                    int32_t h, int64_t M, int32_t exact, const int32_t *round_of, int32_t rounds,
                    uint64_t *sum, int64_t *size)
{
    return dense_curve(n, rowptr, col, r, h, M, exact, round_of, rounds, NULL, sum, size);
}

/* The faster variant of EstDense used in the paper's experiments (Sec. 6,
 * after Prop. 6.2's proof): with k' = max_v c'(v) and gamma = (1 - eps) /
 * (1 + eps), every node with c'(v) < gamma k' is removed before EstDense runs,
 * so the candidates are X'_q = {v : c'(v) >= gamma k', round_of[v] >= q}.
 * The comparison is made in double precision: c'(v) >= gamma * k'.
 * keep_out (may be NULL) receives the kept-node mask. */
int kho_dense_curve_pruned(int64_t n, const int64_t *rowptr, const int32_t *col,
                           const uint8_t *r, int32_t h, int64_t M, int32_t exact,
                           const int32_t *round_of, int32_t rounds, const uint64_t *core,
                           double eps, uint64_t *sum, int64_t *size, uint8_t *keep_out)
{
    if (!(eps > 0.0) || !(eps < 1.0))
        return KHO_EINVAL;
    uint8_t *keep = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!keep)
        return KHO_ENOMEM;
    uint64_t kmax = 0;
    for (int64_t v = 0; v < n; v++)
        if (core[v] > kmax)
            kmax = core[v];
    double gamma = (1.0 - eps) / (1.0 + eps);
    double thr = gamma * (double)kmax;
    for (int64_t v = 0; v < n; v++)
        keep[v] = (double)core[v] >= thr ? 1 : 0;
    int rc = dense_curve(n, rowptr, col, r, h, M, exact, round_of, rounds, keep, sum, size);
    if (keep_out)
        memcpy(keep_out, keep, (size_t)n);
    free(keep);
    return rc;
}

static int dense_curve(int64_t n, const int64_t *rowptr, const int32_t *col, const uint8_t *r,
                       int32_t h, int64_t M, int32_t exact, const int32_t *round_of,
                       int32_t rounds, const uint8_t *keep, uint64_t *sum, int64_t *size)
{
    if (rounds < 0 || (!exact && M < 1))
        return KHO_EINVAL;
    for (int64_t v = 0; v < n; v++)
        if (round_of[v] < 0 || round_of[v] >= rounds)
            return KHO_EINVAL;
    int32_t *buf = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    int32_t *dist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    uint8_t *x = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    uint8_t *alive = (uint8_t *)malloc((size_t)(n > 0 ? n : 1));
    if (!buf || !dist || !x || !alive) {
        free(buf);
        free(dist);
        free(x);
        free(alive);
        return KHO_ENOMEM;
    }
    for (int64_t i = 0; i < n; i++)
        dist[i] = -1;
    for (int32_t q = 0; q < rounds; q++) {
        int64_t cnt = 0;
        uint64_t s = 0;
        for (int64_t v = 0; v < n; v++) {
            alive[v] = (round_of[v] >= q && (!keep || keep[v])) ? 1 : 0;
            cnt += alive[v];
        }
        for (int64_t v = 0; v < n; v++) {
            if (!alive[v])
                continue;
            int64_t d = kho_hball(n, rowptr, col, alive, v, h, buf, dist);
            if (exact) {
                s += d > 0 ? (uint64_t)(d - 1) : 0;
            } else if (d > 0) {
                uint8_t k = 0;
                int32_t bs = 0;
                for (int64_t j = 0; j < d; j++)
                    x[j] = r[buf[j]];
                s += def41(x, d, M, &k, &bs);
            }
        }
        sum[q] = s;
        size[q] = cnt;
    }
    free(buf);
    free(dist);
    free(x);
    free(alive);
    return KHO_OK;
}
