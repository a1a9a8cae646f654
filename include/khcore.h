/*
 * khcore.h -- C ABI of the GB300 (sm_103a) library for distance-generalized
 * (k,h)-cores, after Tatti, "Fast computation of distance-generalized cores
 * using sampling".
 *
 * Terms (paper, Sec. 2-3):
 *   N(v; h, X)   nodes reachable from v by a path of at most h edges inside the
 *                alive node set X; deg_h(v; X) = |N(v; h, X)| - 1.
 *   (k,h)-core   maximal node set whose members all have deg_h >= k inside it;
 *                the core number c(v) is the largest such k containing v.
 *   r[v]         geometric(1/2) rank, P(r >= j) = 2^-j (Sec. 3, Alg. 4).
 *   M            sample budget of Eq. (buffer).
 *   B[v,i],k[v,i]  nodes of N(v; i) with rank >= k[v,i], k[v,i] the smallest
 *                level leaving at most M of them (Sec. 3, Prop. 3.1).
 *   estimate     Alg. 1 / Def. 4.1: |B[v,h] \ {v}| 2^k, raised to M 2^(k-1)
 *                when k > 0.
 *
 * Conventions for every call:
 *   - Return 0 on success or a negative KH_E* code.  No call aborts, exits or
 *     traps; the text of the last error of a context is kh_last_error().
 *   - Graphs are simple and undirected, given as a symmetric CSR with int64
 *     row offsets and int32 column indices, each row strictly increasing, no
 *     self-loops.  Node ids must be below 2^27 (sampled lists pack the rank in
 *     the top 5 bits of a 32-bit key).
 *   - Output arrays are caller-allocated.  Without KH_DEVICE_PTR they are host
 *     memory and the call returns after the results are written.  With
 *     KH_DEVICE_PTR they are device memory of the context's device and the
 *     results are written by work enqueued on the context's stream (kh_sync
 *     waits): kh_ranks, kh_hdegree_exact and kh_sampled_counts only enqueue;
 *     kh_estimate waits for its device error word before returning; the peels
 *     (kh_core_*, kh_dense) read a small device state once per eight rounds
 *     to know when to stop, so they synchronize with the stream while they run
 *     and enqueue only the final copy.
 *   - Every result is a deterministic function of (graph, h, seed, M).
 *   - A context and its graphs must be used from one host thread at a time.
 */
#ifndef KHCORE_H
#define KHCORE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KH_OK 0
#define KH_EINVAL (-1)    /* bad argument (null pointer, h < 1, M < 1, ...) */
#define KH_EGRAPH (-2)    /* CSR not simple/symmetric/sorted, or ids >= 2^27 */
#define KH_ENOMEM (-3)    /* device or host allocation failed */
#define KH_ECUDA (-4)     /* a CUDA runtime call failed */
#define KH_ETIMEOUT (-5)  /* a bounded device loop gave up (peel round limit) */
#define KH_EINTERNAL (-6) /* a device-side bounds check fired */

#define KH_DEVICE_PTR 1u  /* pointer arguments are device memory */

typedef struct kh_ctx kh_ctx;
typedef struct kh_graph kh_graph;

/* Create a context on CUDA device `device`.  `cuda_stream` is a cudaStream_t
 * to run on, or NULL for a stream the library creates and owns.
 * *out receives the context; destroy it with kh_ctx_destroy. */
int kh_ctx_create(kh_ctx **out, int device, void *cuda_stream);
int kh_ctx_destroy(kh_ctx *ctx);

/* Text of the last error reported by a call on `ctx` (never NULL). */
const char *kh_last_error(kh_ctx *ctx);

/* Fault injection on the host (no counterpart in the paper; a test aid): the
 * k-th device allocation this context makes after the call fails with
 * KH_ENOMEM, once; k = 0 disarms.  A failed call leaves the graph and the
 * context usable: a later call allocates what is missing.  KH_EINVAL for a
 * NULL context or k < 0. */
int kh_debug_fail_alloc(kh_ctx *ctx, int64_t k);

/* Load a graph (Sec. 2: G = (V, E), n nodes, undirected).  rowptr has n+1
 * int64 entries, col has rowptr[n] int32 entries.  The library copies both
 * into device memory it owns; the caller keeps ownership of its arrays.
 * flags & KH_DEVICE_PTR: rowptr/col are device pointers.  The graph is
 * validated on the device: KH_EGRAPH if a row is unsorted or has duplicates,
 * a column is out of range or a self-loop, or an edge lacks its reverse. */
int kh_graph_load_csr(kh_ctx *ctx, int64_t n, const int64_t *rowptr, const int32_t *col,
                      uint32_t flags, kh_graph **out);
int kh_graph_free(kh_graph *g);

/* Load many graphs packed in one CSR as one batch (the batched form of the
 * decomposition; the paper processes one graph at a time).  Graph q owns
 * nodes vtx_off[q] .. vtx_off[q+1]-1 (vtx_off: int64[ngraphs+1], host memory,
 * vtx_off[0] = 0) and its column indices are global ids inside that range;
 * rowptr (int64[N+1]) and col follow kh_graph_load_csr (KH_DEVICE_PTR
 * applies to them).  h_per_graph (int32[ngraphs], host, may be NULL for h = 2)
 * sets each graph's h.  M is Eq. (buffer) of each graph's own node count
 * (eps 0.5, delta 0.05; kh_set_sampling with M_or_0 == 0 recomputes it per
 * graph, M_or_0 > 0 sets one M for all), and ranks use each node's id inside
 * its graph, so every result equals the result of loading that graph alone.
 * Results are per node of the batch (length N = vtx_off[ngraphs]).
 * kh_set_h on a batch replaces the per-graph h by one h for every graph.
 * KH_EGRAPH also when an edge joins two graphs. */
int kh_graph_load_batch(kh_ctx *ctx, int32_t ngraphs, const int64_t *vtx_off, const int64_t *rowptr,
                        const int32_t *col, const int32_t *h_per_graph, uint32_t flags,
                        kh_graph **out);

/* Before loading a graph (no counterpart in the paper; for callers that admit
 * work by device memory): the budget M in force for n nodes (M_or_0 > 0, else
 * Eq. (buffer) of eps and delta, as kh_set_sampling) into *M_out, and into
 * *bytes an upper bound of the device memory the library allocates for a
 * graph of n nodes and nnz adjacency entries and a sampled decomposition
 * (kh_core_sampled) at this h: the CSR, the per-node work arrays, the level
 * lists of levels 1..h-1, the split-part slots and the compaction buffers.
 * Either output may be NULL.  Host only: no device is touched.  KH_EINVAL for
 * negative sizes, h outside [1, 16], or M outside [1, 12000]. */
int kh_footprint(int64_t n, int64_t nnz, int32_t h, int64_t M_or_0, double eps, double delta,
                 int64_t *M_out, int64_t *bytes);

/* Number of nodes of a loaded graph. */
int kh_graph_n(kh_graph *g, int64_t *n);

/* Path length h >= 1 of h-neighbourhoods (Sec. 2; h = 1 gives ordinary
 * k-cores).  Default 2. */
int kh_set_h(kh_graph *g, int32_t h);

/* Sampling parameters (Sec. 3).  seed: SplitMix64 seed of the ranks r[v]
 * (r[v] = trailing zeros of the v-th output, capped at 31).  M_or_0 > 0 sets
 * M directly; M_or_0 == 0 sets M = floor(1 + 4(2+eps)/eps^2 (log(2n/delta) +
 * log 8)) (Eq. (buffer), natural log).  Requires eps > 0, 0 < delta < 1 when
 * M_or_0 == 0; M must lie in [1, 12000].  Default: seed 1, eps 0.5,
 * delta 0.05. */
int kh_set_sampling(kh_graph *g, uint64_t seed, int64_t M_or_0, double eps, double delta);

/* The budget M in force (for a batch with per-graph M: the largest). */
int kh_get_M(kh_graph *g, int64_t *M);

/* Ranks r[v], uint8[n] (Sec. 3; Alg. 4 first loop). */
int kh_ranks(kh_graph *g, uint8_t *r, uint32_t flags);

/* Exact h-degrees of the whole graph, deg[v] = |N(v; h, V)| - 1, int32[n]
 * (Sec. 2). */
int kh_hdegree_exact(kh_graph *g, int32_t *deg, uint32_t flags);

/* Fixed-level sampled counts of the whole graph: cnt[v*(j_hi-j_lo+1) +
 * (j-j_lo)] = |{u in N(v; h, V), u != v : r[u] >= j}|, int32, for
 * 0 <= j_lo <= j_hi <= 31.  cnt * 2^j is Alg. 1's estimate with the level
 * forced to j, i.e. sampling probability 2^-j; j = 0 gives deg_h. */
int kh_sampled_counts(kh_graph *g, int32_t j_lo, int32_t j_hi, int32_t *cnt, uint32_t flags);

/* Adaptive estimate of the whole graph (Alg. 1 after the level recursion
 * of Prop. 3.1 / Alg. 2): est uint64[n], level = k[v,h] uint8[n] (may be
 * NULL), bsize = |B[v,h]| int32[n] (may be NULL). */
int kh_estimate(kh_graph *g, uint64_t *est, uint8_t *level, int32_t *bsize, uint32_t flags);

/* ExactCore (Sec. 2): core[v] = c(v), int32[n], by bucket-synchronous peeling
 * (c = max(c, min deg_h); every alive v with deg_h <= c is removed at once),
 * which equals one-at-a-time peeling because deg_h never grows as nodes
 * leave.  After each round the h-ball of the removed nodes is recomputed. */
int kh_core_exact(kh_graph *g, int32_t *core, uint32_t flags);

/* Core (Alg. 4) with the estimate in place of deg_h: core[v] = c'(v),
 * uint64[n], bucket-synchronous as above (the estimate never grows as nodes
 * leave, Prop. 4.2); the lists are refreshed level by level where their
 * inputs changed (Alg. 3). */
int kh_core_sampled(kh_graph *g, uint64_t *core, uint32_t flags);

/* Statistics of the last kh_core_* call: round_of[v] (int32[n], may be NULL)
 * is the peeling round that removed v; *rounds the number of rounds;
 * *updates the number of completed node (re)computations of d, including the
 * initial pass and the exact decrements of the loss propagation (refines that
 * stopped early with a lower bound only are counted by kh_peel_stats).
 * Host pointers only. */
int kh_peel_info(kh_graph *g, int32_t *round_of, int64_t *rounds, int64_t *updates);

/* EstDense (Alg. 7, Sec. 6): replays a removal order and, at the start of
 * every round q, sums d(v; X_q) over X_q = {v : round_of[v] >= q}, where d is
 * deg_h (exact != 0) or the Alg. 1 estimate, every value current for X_q.
 * Since 2 |E_h(X)| = sum_v deg_h(v; X), sum[q] / (2 size[q]) estimates the
 * h-density |E_h(X_q)| / |X_q|.  round_of: host int32[n] with values in
 * [0, rounds), e.g. from kh_peel_info after kh_core_*; one node per round
 * gives the paper's n candidates.  Outputs (host, each may be NULL):
 * sum uint64[rounds], size int64[rounds] (|X_q|), *best = the q of largest
 * sum[q] / size[q] (ties: the smallest q; -1 when n = 0).  Uses the graph's
 * h and sampling parameters: the paper draws fresh ranks for Alg. 7, which a
 * caller gets with kh_set_sampling and another seed.  Afterwards kh_peel_info
 * and kh_peel_stats describe this replay.  KH_EINVAL for a batch, rounds
 * outside [1, n + 1] or a round_of value outside [0, rounds). */
int kh_dense(kh_graph *g, int32_t exact, const int32_t *round_of, int32_t rounds, uint64_t *sum,
             int64_t *size, int32_t *best);

/* The faster EstDense variant of Sec. 6 (after the proof of its guarantee):
 * with k' = max_v core[v] and gamma = (1 - eps) / (1 + eps), every node with
 * core[v] < gamma k' (compared in double precision) is removed before the
 * replay, so the candidates are X'_q = {v kept : round_of[v] >= q}; outputs
 * as kh_dense over those sets (size[q] = |X'_q|, a round with X'_q empty has
 * sum 0 and is never `best`).  core: host uint64[n], the sampled core map the
 * order came from (kh_core_sampled; an int32 exact core widened to uint64
 * also works); kept (host uint8[n], may be NULL) receives the kept-node mask.
 * KH_EINVAL as kh_dense, a NULL core, or eps outside (0, 1). */
int kh_dense_pruned(kh_graph *g, int32_t exact, const int32_t *round_of, int32_t rounds,
                    const uint64_t *core, double eps, uint64_t *sum, int64_t *size, int32_t *best,
                    uint8_t *kept);

/* Work statistics of the last kh_core_* call (no counterpart in the paper).
 * refreshed[i] / changed[i] (host int64[KH_MAX_H + 1], indexed by level i,
 * each may be NULL): level-i lists recomputed by the rounds' refresh passes
 * of kh_core_sampled, and how many of them came out different in size or
 * level; *stopped (may be NULL): lazy refines that ended early because the
 * partial ball or partial estimate already exceeded the round's threshold.
 * KH_EINVAL before any peeling. */
#define KH_MAX_H 16
int kh_peel_stats(kh_graph *g, int64_t *refreshed, int64_t *changed, int64_t *stopped);

/* Profiling of kernel classes (no counterpart in the paper; measurement aid).
 * kh_prof_enable(g, 1) resets the counters and brackets every later launch of
 * each kernel class with CUDA events on the context stream (peeling rounds
 * are then launched one by one instead of through a CUDA graph);
 * kh_prof_enable(g, 0) stops the brackets and keeps the counters.
 * kh_prof_read returns, for one class, the summed event time in ms, the number
 * of bracketed launches and the algorithmic bytes the class moved (counted on
 * the device: 8 + 4 deg per expanded vertex for the BFS, 4 per list key read
 * and written for the list kernels, plus per-node metadata). */
#define KH_PROF_BFS 0      /* exact h-degree / fixed-level count BFS */
#define KH_PROF_LEVEL1 1   /* level-1 lists (Alg. 2 at i = 1) */
#define KH_PROF_LEVELU 2   /* level >= 2 lists (Alg. 2 with Alg. 5's trim) */
#define KH_PROF_FRONTIER 3 /* removed-set balls and refresh work lists */
#define KH_PROF_PEEL 4     /* min / select / finish of each round */
#define KH_PROF_KINDS 5
int kh_prof_enable(kh_graph *g, int32_t on);
int kh_prof_read(kh_graph *g, int32_t kind, double *ms, int64_t *launches, double *alg_bytes);
/* Per-bracket event times of one class since kh_prof_enable(g, 1), in launch
 * order: the first min(cap, *count) go to ms (host float[cap]); *count is
 * the number recorded.  KH_EINVAL for a NULL count, a negative cap, or
 * cap > 0 with a NULL ms. */
int kh_prof_trace(kh_graph *g, int32_t kind, float *ms, int64_t cap, int64_t *count);
/* The algorithmic bytes of the same brackets, in the same order (the class's
 * device counter copied before and after each bracket; UINT64_MAX where the
 * copy was not made: more than 2^20 brackets between two reads, or no device
 * memory for the copies).  Same argument rules as kh_prof_trace. */
int kh_prof_trace_bytes(kh_graph *g, int32_t kind, uint64_t *bytes, int64_t cap, int64_t *count);

/* Number of CUDA kernels the library has launched for this graph since it was
 * loaded (kernels inside a replayed CUDA graph count one each per replay).
 * No counterpart in the paper; measurement aid. */
int kh_launch_count(kh_graph *g, int64_t *launches);

/* Exact h-degrees without allocating (the paper has no counterpart: this is
 * a deployment variant of kh_hdegree_exact).  For callers that cannot
 * allocate device memory -- a server whose device memory is owned by a pool
 * sized once at start-up, or a latency-bound caller that must not wait on the
 * allocator.
 * n, rowptr (int64[n+1]) and col (int32[rowptr[n]]) describe a graph that
 * kh_graph_load_csr would accept; it is not validated here, except that a
 * column id outside [0, n) is skipped instead of being visited (the degrees
 * are then meaningless; no error is reported).  All three arrays and deg
 * (int32[n], out: deg[v] = |N(v; h, V)| - 1) are device memory of the current
 * device.  cuda_stream is a cudaStream_t or NULL (legacy default stream); the
 * call only enqueues work on it.
 * Scratch lives in one fixed 64 MiB device array inside the library, which
 * every GPU that loads the library holds until the process exits; no call
 * allocates or frees memory.  Limits: 1 <= h <= 16 and n <= 819200 (the
 * visited set lives in shared memory); larger n returns KH_EINVAL.
 * The first call on a device looks the array up (cudaGetSymbolAddress) with
 * that device current; make that first call before any stream capture.  The
 * address is kept for the life of the process: after a cudaDeviceReset the
 * entry point must not be called again.  Every call shares the one array, so
 * calls that overlap on the GPU (on different streams, or from different
 * threads) race: serialise them. */
int kh_hdegree_exact_noalloc(int64_t n, const int64_t *rowptr, const int32_t *col, int32_t h,
                             int32_t *deg, void *cuda_stream);

/* Layout of the whole-graph exact h-degree pass at h = 2 (kh_hdegree_exact,
 * kh_sampled_counts; no counterpart in the paper: the schedule, not the
 * result).  KH_VAR_CTA: one CTA per source with a visited bitmap of all n
 * nodes in shared memory (only while n <= 819200); KH_VAR_SLICED: (source,
 * slice) work items, the id range cut into `slices` ranges whose visited
 * bitmap fits in shared memory, `threads` per CTA (128, 256, 512 or 1024).
 * KH_VAR_AUTO (default): the library's autotuner times the candidate layouts
 * on a sample of the graph's sources at the first such call and keeps the
 * fastest; with the environment variable KH_TUNE_FILE naming a text file, the
 * choice is also recorded there per graph shape class (device SM count, log2
 * n, log2 nnz, log2 of max degree over mean degree) and reused by later
 * processes.  Every layout returns the same degrees.  kh_set_variant forces
 * a layout (KH_EINVAL for an unknown op or variant, KH_VAR_CTA with n too
 * large, or slices outside [the shared-memory minimum, min(1024, n)]);
 * kh_get_variant returns the layout in force, tuning first if needed, and the
 * sample time in ms it was chosen with (0 when forced or read from a file). */
#define KH_OP_HDEG2 0
#define KH_VAR_AUTO 0
#define KH_VAR_CTA 1
#define KH_VAR_SLICED 2
/* KH_VAR_SLICED_SMALL: as KH_VAR_SLICED for sources whose 2-hop work (the sum
 * of their neighbours' degrees) is at least 511; the others take one warp
 * each with a private hash set of their 2-ball in shared memory. */
#define KH_VAR_SLICED_SMALL 3
/* KH_OP_PEEL_COMPACT: the peels (kh_core_*, kh_dense*) switch, each time the
 * alive node count has halved, to a CSR that keeps only the neighbours alive
 * at that moment (node ids unchanged; results unchanged).  KH_VAR_AUTO: for
 * graphs of at least 65536 nodes; KH_COMPACT_OFF: never; KH_COMPACT_ALWAYS:
 * at any size.  slices and threads are ignored. */
#define KH_OP_PEEL_COMPACT 1
#define KH_COMPACT_OFF 1
#define KH_COMPACT_ALWAYS 2
/* KH_OP_LEVEL_UNION: how the level >= 2 list union (Alg. 2 with Alg. 5's
 * trim) schedules a node's lists over the warps of its CTA.
 * KH_LEVELU_STEPPED: barrier-separated steps, the trim once per step;
 * KH_LEVELU_FREE: warps claim lists and trim from their own view of the rank
 * counts, meeting only to compact the hash set;
 * KH_LEVELU_GROUPED: as free, with groups of 32, 16, ..., 1 lanes claiming
 * lists in place of whole warps: per node, the fewest lanes whose step of
 * 4 keys a lane covers the keys a list is expected to give at or above the
 * starting level (sum of |B[w]| 2^(k[w] - t) over the lists, over their
 * number); with slices = d > 1 (a power of two up to 64) a group covers 1/d
 * of those keys (0: the default).  KH_VAR_AUTO: grouped.  The lists are the
 * same every way. */
#define KH_OP_LEVEL_UNION 2
#define KH_LEVELU_STEPPED 1
#define KH_LEVELU_FREE 2
#define KH_LEVELU_GROUPED 3
/* KH_OP_HDEG2_SWEEP: the whole-graph exact 2-degrees (kh_hdegree_exact at
 * h = 2 with a sliced layout) may hand the sources of largest 2-hop work
 * (sum of their neighbours' degrees) to bit-parallel sweeps: one pass over
 * every row per batch of 128 sources, with 128-bit source masks per node.
 * KH_VAR_AUTO: the tuner decides the threshold; KH_SWEEP_OFF: never;
 * KH_SWEEP_FROM: the sources of work >= 2^slices - 1 (slices in [1, 48)).
 * kh_get_variant with this op reports KH_SWEEP_OFF or KH_SWEEP_FROM and the
 * bin in *slices.  The degrees are the same every way. */
#define KH_OP_HDEG2_SWEEP 3
#define KH_SWEEP_OFF 1
#define KH_SWEEP_FROM 2
int kh_set_variant(kh_graph *g, int32_t op, int32_t variant, int32_t slices, int32_t threads);
int kh_get_variant(kh_graph *g, int32_t op, int32_t *variant, int32_t *slices, int32_t *threads,
                   double *tuned_ms);

/* Wait for all work enqueued on the graph's context stream. */
int kh_sync(kh_graph *g);

#ifdef __cplusplus
}
#endif

#endif /* KHCORE_H */
