// kh_peel.cu -- bucket-synchronous peeling (ExactCore of Sec. 2; Core, Alg. 4).
//
// Round r on the alive set X (all device-resident):
//   1. minval = min_{v in X} d[v]                         (k_min_alive)
//   2. c = max(c, minval); R = {v in X : d[v] <= c};
//      core[v] = c, alive[v] = 2 for v in R               (k_select)
//   3. refresh d on X \ R where it can have changed:
//      exact:   nodes within h hops of R in the old graph (k_ball_hop x h),
//               then a bounded BFS per such node;
//      sampled: level i = 1..h recomputes the alive neighbours of R and of the
//               nodes whose (|B|, k) changed at level i-1 (Alg. 3).
//   4. alive[R] = 0; the last block advances the state          (k_finish)
// Removing every node with d <= c at once gives the same core map as Alg. 4's
// one-at-a-time loop because d(v; X) never grows as X shrinks (deg_h by
// inclusion of neighbourhoods; the estimate by Prop. 4.2): every node of R
// would still have d <= c when its turn came.
//
// Exact mode applies the paper's early stop (Sec. 5): once c >= |X| - 1 every
// remaining node has deg_h <= |X| - 1 <= c, so all get core c in the next
// round; the refresh of this round is then skipped.
//
// Lazy last level.  A node whose h-neighbourhood may have changed is only
// marked stale: its last value stays as an upper bound (d never grows as X
// shrinks) and it carries a lower bound lb (exact: max(deg_X(v), max_w
// deg_X(w)); sampled: Alg. 1 on its own level-(h-1) list, a sub-list of
// N(v; h) with v first, so Prop. 4.2 applies).  Each round first takes
// U = min over alive d (upper bounds), recomputes every stale node with
// lb <= T = max(c, U), and only then takes the minimum and the removal set:
// the true minimum is at most U <= T, every skipped node has d >= lb > T,
// so the minimum is attained by a fresh node and no skipped node can have
// d <= c' = max(c, min) <= T.  The result is the same core map, with the
// expensive recomputations of high-degree nodes deferred until c nears them
// (the lower-bound pruning of the exact baselines, and the paper's lazy
// initialisation, Sec. 5).
//
// A round reads every size it needs from device memory, so one captured CUDA
// graph holds kRoundsPerGraph rounds; rounds that start with no alive node do
// nothing.  The host replays the graph and reads the state once per replay.
#include <cstring>
#include <vector>

#include "kh_internal.cuh"

namespace kh {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kPeelThreads = 256;
constexpr int kRoundsPerGraph = 8;

// Per-graph peel state (a single graph has one entry; a batch one per graph,
// so each graph peels with its own c exactly as it would alone):
//   c[g]   core value reached so far,
//   mu[g]  this round's minimum of d over the alive nodes, fresh or not
//          (the lazy refine threshold is max(c, mu)),
//   mn[g]  the same minimum over the fresh nodes only,
//   mr[g]  the minimum of the values the round's refine completed.
// The round's minimum of d after the refine is min(mn, mr): a node attaining
// mu is fresh, or stale with lb <= d = mu and so refined to a value <= mu;
// every node left stale has d >= lb > max(c, mu).
struct PeelState {
    unsigned long long* c;
    unsigned long long* mn;
    unsigned long long* mu;
    unsigned long long* mr;
    int32_t* left;       // alive nodes per graph (batches: per-graph early stop)
    const int32_t* gid;  // graph of each node; nullptr for a single graph
};

__device__ __forceinline__ int graph_of(const PeelState& p, int64_t v) {
    return p.gid ? p.gid[v] : 0;
}

__device__ __forceinline__ unsigned long long round_min(const PeelState& p, int g) {
    return p.mn[g] < p.mr[g] ? p.mn[g] : p.mr[g];
}

__device__ __forceinline__ unsigned long long umin(unsigned long long a, unsigned long long b) {
    return a < b ? a : b;
}

// Round start: the minimum of d over the alive nodes into mu[graph] and over
// the fresh ones into mn[graph].  A single graph reduces per block; a batch
// takes one atomic per node that improves its graph's current minimum (read
// first, so most nodes need none).
template <typename T>
__global__ void k_min_alive(const uint8_t* __restrict__ alive, const uint8_t* __restrict__ fresh,
                            const T* __restrict__ d, int64_t n, const int32_t* __restrict__ vl,
                            DevState* st, unsigned long long* mu, unsigned long long* mn,
                            const int32_t* __restrict__ gid) {
    if (st->n_alive == 0) return;
    unsigned long long m = ~0ull, mf = ~0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t v = vl ? vl[i] : i;
        if (alive[v] == 1) {
            const unsigned long long x = (unsigned long long)d[v];
            const bool fr = fresh[v] != 0;
            if (gid) {
                const int g = gid[v];
                if (x < *(volatile unsigned long long*)(mu + g)) atomicMin(mu + g, x);
                if (fr && x < *(volatile unsigned long long*)(mn + g)) atomicMin(mn + g, x);
            } else {
                m = umin(m, x);
                if (fr) mf = umin(mf, x);
            }
        }
    }
    if (gid) return;
    for (int off = 16; off > 0; off >>= 1) {
        m = umin(m, __shfl_down_sync(kFull, m, off));
        mf = umin(mf, __shfl_down_sync(kFull, mf, off));
    }
    __shared__ unsigned long long s_m[kPeelThreads / 32], s_f[kPeelThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) {
        s_m[warp] = m;
        s_f[warp] = mf;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w) {
            m = umin(m, s_m[w]);
            mf = umin(mf, s_f[w]);
        }
        if (m != ~0ull) atomicMin(mu, m);
        if (mf != ~0ull) atomicMin(mn, mf);
        if (blockIdx.x == 0) atomicAdd(&st->bytes[kProfPeel], (unsigned long long)n * (2 + sizeof(T)));
    }
}

struct LbArgs {
    const unsigned long long* lb;  // lower bounds of stale nodes
};

__device__ __forceinline__ unsigned long long lower_bound(const LbArgs& a, int v) { return a.lb[v]; }

__global__ void k_min_lb(const uint8_t* __restrict__ alive, const uint8_t* __restrict__ fresh,
                         int64_t n, LbArgs a, DevState* st, PeelState p) {
    if (st->n_alive == 0) return;
    unsigned long long m = ~0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (alive[v] == 1 && !fresh[v]) {
            const unsigned long long x = lower_bound(a, (int)v);
            if (p.gid) {
                const int g = p.gid[v];
                if (x < *(volatile unsigned long long*)(p.mu + g)) atomicMin(p.mu + g, x);
            } else if (x < m) {
                m = x;
            }
        }
    if (p.gid) return;
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_down_sync(kFull, m, off);
        if (o < m) m = o;
    }
    if ((threadIdx.x & 31) == 0 && m != ~0ull) atomicMin(p.mu, m);
}

// Stale nodes with lb <= T = max(c, U) join the refine list and become fresh
// (their value is recomputed right after, before anything reads it).  A stale
// node whose upper bound is already <= c leaves in this round whatever its
// exact value (c' = max(c, min) >= c >= d), so it is not refined; its upper
// bound joins the round minimum (mr), which keeps that minimum <= c and so
// c' = c, as the exact values would (the true minimum is <= its bound <= c).
// The replay of a given order (dense) needs every value and skips nothing.
template <typename T>
__global__ void k_collect(const uint8_t* __restrict__ alive, uint8_t* __restrict__ fresh, int64_t n,
                          const int32_t* __restrict__ vl, LbArgs a, const T* __restrict__ d,
                          int keep_all, DevState* st, PeelState p, int32_t* __restrict__ out) {
    if (st->n_alive == 0) return;
    const int lane = threadIdx.x & 31;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nround = (n + 31) & ~(int64_t)31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nround; i += stride) {
        bool due = false;
        const int64_t v = i < n ? (vl ? vl[i] : i) : 0;
        if (i < n && alive[v] == 1 && !fresh[v]) {
            const int g = graph_of(p, v);
            const unsigned long long ub = (unsigned long long)d[v];
            if (!keep_all && ub <= p.c[g]) {
                atomicMin(p.mr + g, ub);  // removed this round: no refine needed
            } else {
                const unsigned long long T = p.c[g] > p.mu[g] ? p.c[g] : p.mu[g];
                due = lower_bound(a, (int)v) <= T;
            }
        }
        const uint32_t m = __ballot_sync(kFull, due);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&st->nQ, __popc(m));
        base = __shfl_sync(kFull, base, 0);
        if (due) {
            out[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)v;
            fresh[v] = 1;
        }
    }
}

// Alive degrees and "no upper bound yet".  A start from a subset (alive[v]
// from the caller) counts only alive neighbours; a start from the whole graph
// (all alive) takes the row length.
__global__ void k_init_exact(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             const uint8_t* __restrict__ alive, int subset, int64_t n,
                             int32_t* __restrict__ degX, int32_t* __restrict__ d) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        int32_t dx = (int32_t)(rowptr[v + 1] - rowptr[v]);
        if (subset) {
            dx = 0;
            for (int64_t k = rowptr[v]; k < rowptr[v + 1]; ++k) dx += alive[col[k]] == 1;
        }
        degX[v] = dx;
        d[v] = 0x7fffffff;  // no upper bound known yet
    }
}

// Start from the kept nodes only: alive[v] = keep[v], removed ones in deadbm.
// Nodes that are not kept get no removal round (-1).
__global__ void k_init_keep(const uint8_t* __restrict__ keep, int64_t n, uint8_t* __restrict__ alive,
                            uint32_t* __restrict__ deadbm, int32_t* __restrict__ round_of) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        alive[v] = keep[v] ? 1 : 0;
        if (!keep[v]) {
            atomicOr(deadbm + (v >> 5), 1u << (v & 31));
            round_of[v] = -1;
        }
    }
}

template <typename T, typename C>
__global__ void k_select(uint8_t* __restrict__ alive, const T* __restrict__ d, int64_t n,
                         const int32_t* __restrict__ vl, DevState* st, PeelState p,
                         C* __restrict__ core, int32_t* __restrict__ round_of,
                         int32_t* __restrict__ R, int32_t* __restrict__ seen) {
    if (st->n_alive == 0) return;
    const int round = st->round;
    const int lane = threadIdx.x & 31;
    int keep = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nround = (n + 31) & ~(int64_t)31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nround; i += stride) {
        bool rm = false;
        const int64_t v = i < n ? (vl ? vl[i] : i) : 0;
        if (i < n && alive[v] == 1) {
            const int g = graph_of(p, v);
            const unsigned long long m = round_min(p, g);
            const unsigned long long c = p.c[g] > m ? p.c[g] : m;
            if ((unsigned long long)d[v] <= c) {
                rm = true;
                if (p.gid) atomicSub(p.left + g, 1);
                core[v] = (C)c;
                round_of[v] = round;
                alive[v] = 2;
                seen[v] = round * kPhaseStride;
            } else {
                ++keep;
            }
        }
        const uint32_t m = __ballot_sync(kFull, rm);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&st->nR, __popc(m));
        base = __shfl_sync(kFull, base, 0);
        if (rm) R[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)v;
    }
    for (int off = 16; off > 0; off >>= 1) keep += __shfl_down_sync(kFull, keep, off);
    if (lane == 0 && keep) atomicAdd(&st->n_alive_next, keep);
    if (blockIdx.x == 0 && threadIdx.x == 0)
        atomicAdd(&st->bytes[kProfPeel], (unsigned long long)n * (1 + sizeof(T)));
}

// Exact mode early stop: when c >= |X_new| - 1 every remaining node gets core
// c in round `round + 1`.  Every block evaluates the condition; block 0
// records it for the kernels that follow (they skip the refresh).
template <typename C>
__global__ void k_assign_rest(uint8_t* __restrict__ alive, int64_t n, const int32_t* __restrict__ vl,
                              DevState* st, PeelState p, C* __restrict__ core,
                              int32_t* __restrict__ round_of) {
    if (st->n_alive == 0) return;
    // single graphs only (a batch has no global early stop)
    const unsigned long long m = round_min(p, 0);
    const unsigned long long c = p.c[0] > m ? p.c[0] : m;
    const int left = st->n_alive_next;
    const bool early = left > 0 && c + 1 >= (unsigned long long)left;
    if (blockIdx.x == 0 && threadIdx.x == 0) st->early = early ? 1 : 0;
    if (!early) return;
    const int round = st->round + 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t v = vl ? vl[i] : i;
        if (alive[v] == 1) {
            core[v] = (C)c;
            round_of[v] = round;
            alive[v] = 0;
        }
    }
}

// Batches: the early stop of each graph on its own (c_g >= |X_g| - 1 after
// this round's removal).  Finished graphs' nodes leave at once, so the
// refresh that follows never reaches them.
template <typename C>
__global__ void k_assign_rest_batch(uint8_t* __restrict__ alive, int64_t n,
                                    const int32_t* __restrict__ vl, DevState* st, PeelState p,
                                    C* __restrict__ core, int32_t* __restrict__ round_of) {
    if (st->n_alive == 0) return;
    const int round = st->round + 1;
    int gone = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t v = vl ? vl[i] : i;
        if (alive[v] == 1) {
            const int g = p.gid[v];
            const unsigned long long m = round_min(p, g);
            const unsigned long long c = p.c[g] > m ? p.c[g] : m;
            const int left = *(volatile int32_t*)(p.left + g);
            if (left > 0 && c + 1 >= (unsigned long long)left) {
                core[v] = (C)c;
                round_of[v] = round;
                alive[v] = 0;
                ++gone;
            }
        }
    }
    for (int off = 16; off > 0; off >>= 1) gone += __shfl_down_sync(kFull, gone, off);
    if ((threadIdx.x & 31) == 0 && gone) atomicSub(&st->n_alive_next, gone);
}

// Ends a round: removed nodes leave (alive = 0, dead bitmap bit set); the
// last block to finish advances the state and zeroes the per-round counters.
__global__ void k_finish(uint8_t* __restrict__ alive, const int32_t* __restrict__ R, DevState* st,
                         uint32_t* __restrict__ deadbm, PeelState p, int64_t ngraphs) {
    __shared__ int s_last;
    const int nR = st->nR;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nR; i += stride) {
        const int v = R[i];
        alive[v] = 0;
        atomicOr(deadbm + (v >> 5), 1u << (v & 31));
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        s_last = atomicAdd(&st->done, 1) == (int)gridDim.x - 1;
    }
    __syncthreads();
    if (!s_last) return;
    __threadfence();
    for (int i = threadIdx.x; i < kRcCount; i += blockDim.x) st->rc[i] = 0;
    // every graph: c = max(c, this round's minimum); minima reset
    for (int64_t q = threadIdx.x; q < ngraphs; q += blockDim.x) {
        const unsigned long long m = round_min(p, (int)q);
        if (m != ~0ull && m > p.c[q]) p.c[q] = m;
        p.mn[q] = ~0ull;
        p.mr[q] = ~0ull;
        p.mu[q] = ~0ull;
    }
    if (threadIdx.x == 0) {
        if (st->n_alive != 0) {
            st->round += st->early ? 2 : 1;
            st->n_alive = st->early ? 0 : st->n_alive_next;
        }
        st->n_alive_next = 0;
        st->nR = 0;
        st->nQ = 0;
        st->early = 0;
        st->done = 0;
    }
}

// EstDense: the round's candidate set X is the alive set with every value
// current; its sum of d goes to dsum[round].
template <typename T>
__global__ void k_dense_sum(const uint8_t* __restrict__ alive, const T* __restrict__ d, int64_t n,
                            const int32_t* __restrict__ vl, const DevState* __restrict__ st,
                            unsigned long long* __restrict__ dsum, int64_t cap) {
    if (st->n_alive == 0) return;
    const int round = st->round;
    if (round >= cap) return;
    unsigned long long s = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride) {
        const int64_t v = vl ? vl[i] : i;
        if (alive[v] == 1) s += (unsigned long long)d[v];
    }
    for (int off = 16; off > 0; off >>= 1) s += __shfl_down_sync(kFull, s, off);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(dsum + round, s);
}

// EstDense: the nodes whose scheduled round has come leave (the removal order
// is given, not chosen by d).
__global__ void k_select_sched(uint8_t* __restrict__ alive, const int32_t* __restrict__ sched,
                               int64_t n, const int32_t* __restrict__ vl, DevState* st,
                               int32_t* __restrict__ R, int32_t* __restrict__ seen,
                               int32_t* __restrict__ round_of) {
    if (st->n_alive == 0) return;
    const int round = st->round;
    const int lane = threadIdx.x & 31;
    int keep = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nround = (n + 31) & ~(int64_t)31;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nround; i += stride) {
        bool rm = false;
        const int64_t v = i < n ? (vl ? vl[i] : i) : 0;
        if (i < n && alive[v] == 1) {
            if (sched[v] <= round) {
                rm = true;
                round_of[v] = round;
                alive[v] = 2;
                seen[v] = round * kPhaseStride;
            } else {
                ++keep;
            }
        }
        const uint32_t m = __ballot_sync(kFull, rm);
        int base = 0;
        if (lane == 0 && m) base = atomicAdd(&st->nR, __popc(m));
        base = __shfl_sync(kFull, base, 0);
        if (rm) R[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)v;
    }
    for (int off = 16; off > 0; off >>= 1) keep += __shfl_down_sync(kFull, keep, off);
    if (lane == 0 && keep) atomicAdd(&st->n_alive_next, keep);
}

// ---- compaction of the peel's graph ----------------------------------------
// As nodes leave, rows still list them.  Once the alive count has halved since
// the last compaction, the peel switches to a CSR that keeps, for every node,
// only the neighbours alive at that moment, and to the list of those nodes for
// its whole-node scans.  Every peel kernel filters rows by alive (1: alive, 2:
// removed this round, 0: removed earlier) and only ever needs neighbours with
// alive != 0, all of which were alive at the last compaction, so the kept rows
// serve the rest of the peel unchanged; node ids stay the same.

constexpr int kScanThreads = 256;
constexpr int kScanPer = 8;
constexpr int kScanTile = kScanThreads * kScanPer;

// Exclusive scan of one tile of `in` into `out`; the tile's total to sums[tile].
__global__ void k_scan_tiles(const int64_t* __restrict__ in, int64_t n, int64_t* __restrict__ out,
                             int64_t* __restrict__ sums) {
    __shared__ int64_t s_w[kScanThreads / 32];
    const int64_t base = (int64_t)blockIdx.x * kScanTile + (int64_t)threadIdx.x * kScanPer;
    int64_t x[kScanPer];
    int64_t t = 0;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        x[j] = base + j < n ? in[base + j] : 0;
        t += x[j];
    }
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    int64_t inc = t;  // inclusive warp scan of the thread totals
    for (int off = 1; off < 32; off <<= 1) {
        const int64_t y = __shfl_up_sync(kFull, inc, off);
        if (lane >= off) inc += y;
    }
    if (lane == 31) s_w[warp] = inc;
    __syncthreads();
    int64_t before = 0;
    for (int w = 0; w < warp; ++w) before += s_w[w];
    int64_t run = before + inc - t;
#pragma unroll
    for (int j = 0; j < kScanPer; ++j) {
        if (base + j < n) out[base + j] = run;
        run += x[j];
    }
    if (threadIdx.x == kScanThreads - 1) sums[blockIdx.x] = before + inc;
}

// Exclusive scan of the tile totals (one block, in chunks with a carry).
__global__ void k_scan_sums(int64_t* __restrict__ sums, int64_t tiles) {
    __shared__ int64_t s_w[kScanThreads / 32];
    __shared__ int64_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    for (int64_t c0 = 0; c0 < tiles; c0 += kScanThreads) {
        const int64_t i = c0 + threadIdx.x;
        const int64_t x = i < tiles ? sums[i] : 0;
        int64_t inc = x;
        for (int off = 1; off < 32; off <<= 1) {
            const int64_t y = __shfl_up_sync(kFull, inc, off);
            if (lane >= off) inc += y;
        }
        if (lane == 31) s_w[warp] = inc;
        __syncthreads();
        int64_t before = s_carry;
        for (int w = 0; w < warp; ++w) before += s_w[w];
        if (i < tiles) sums[i] = before + inc - x;
        __syncthreads();
        if (threadIdx.x == kScanThreads - 1) s_carry = before + inc;
        __syncthreads();
    }
}

__global__ void k_scan_add(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ sums) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += stride)
        out[i] += sums[i / kScanTile];
}

// Per listed alive node: its alive neighbours and itself (flag), warp per node.
__global__ void k_compact_count(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const uint8_t* __restrict__ alive, const int32_t* __restrict__ vl,
                                int64_t vn, int64_t* __restrict__ cnt, int64_t* __restrict__ flag) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < vn; i += nw) {
        const int64_t v = vl ? vl[i] : i;
        if (alive[v] != 1) continue;
        int64_t c = 0;
        for (int64_t k = rowptr[v] + lane; k < rowptr[v + 1]; k += 32) c += alive[col[k]] == 1;
        for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(kFull, c, off);
        if (lane == 0) {
            cnt[v] = c;
            flag[v] = 1;
        }
    }
}

// Write each listed alive node's alive neighbours (in row order) and the node
// itself into the new CSR and list.
__global__ void k_compact_fill(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                               const uint8_t* __restrict__ alive, const int32_t* __restrict__ vl,
                               int64_t vn, const int64_t* __restrict__ nrow,
                               const int64_t* __restrict__ pos, int32_t* __restrict__ ncol,
                               int32_t* __restrict__ nlist) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < vn; i += nw) {
        const int64_t v = vl ? vl[i] : i;
        if (alive[v] != 1) continue;
        int64_t out = nrow[v];
        for (int64_t k0 = rowptr[v]; k0 < rowptr[v + 1]; k0 += 32) {
            const int64_t k = k0 + lane;
            int32_t u = 0;
            bool keep = false;
            if (k < rowptr[v + 1]) {
                u = col[k];
                keep = alive[u] == 1;
            }
            const uint32_t m = __ballot_sync(kFull, keep);
            if (keep) ncol[out + __popc(m & ((1u << lane) - 1u))] = u;
            out += __popc(m);
        }
        if (lane == 0) nlist[pos[v]] = (int32_t)v;
    }
}

// Exclusive scan of n values (n + 1 outputs would need in[n] = 0).
int scan_i64(Graph& g, const int64_t* in, int64_t n, int64_t* out, int64_t* sums, cudaStream_t s) {
    const int64_t tiles = (n + kScanTile - 1) / kScanTile;
    if (tiles == 0) return KH_OK;
    k_scan_tiles<<<(int)tiles, kScanThreads, 0, s>>>(in, n, out, sums);
    k_scan_sums<<<1, kScanThreads, 0, s>>>(sums, tiles);
    k_scan_add<<<g.ctx->sm_count * 4, 256, 0, s>>>(out, n, sums);
    count_launch(g, 3);
    return KH_OK;
}

// Rebuild the peel's CSR and node list from the alive nodes (between rounds).
int compact_peel(Graph& g, cudaStream_t s) {
    const size_t n1 = (size_t)g.n + 1;
    int rc;
    if (!g.cp_tmp) {
        if ((rc = alloc_bytes(g.ctx, (void**)&g.cp_tmp, sizeof(int64_t) * 2 * n1, "compaction counts")))
            return rc;
        if ((rc = alloc_bytes(g.ctx, (void**)&g.cp_sums,
                              sizeof(int64_t) * (2 * (n1 / kScanTile) + 4), "compaction sums")))
            return rc;
    }
    const int nb = g.cp_cur ^ 1;  // the buffer set not in use
    if (!g.cp_row[nb]) {
        if ((rc = alloc_bytes(g.ctx, (void**)&g.cp_row[nb], sizeof(int64_t) * n1, "compacted rowptr")))
            return rc;
        if ((rc = alloc_bytes(g.ctx, (void**)&g.cp_list[nb], sizeof(int32_t) * n1, "compacted list")))
            return rc;
    }
    int64_t* cnt = g.cp_tmp;
    int64_t* flag = g.cp_tmp + n1;
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.cp_tmp, 0, sizeof(int64_t) * 2 * n1, s));
    const int grid = g.ctx->sm_count * 8;
    k_compact_count<<<grid, 256, 0, s>>>(g.rowptr, g.col, g.alive, g.vlist, g.vcount, cnt, flag);
    count_launch(g, 1);
    int64_t* pos = g.cp_tmp + n1;  // scanned in place over the flags
    if ((rc = scan_i64(g, cnt, (int64_t)n1, g.cp_row[nb], g.cp_sums, s))) return rc;
    if ((rc = scan_i64(g, flag, (int64_t)n1, pos, g.cp_sums + (n1 / kScanTile) + 2, s))) return rc;
    int64_t tot[2] = {0, 0};
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(&tot[0], g.cp_row[nb] + g.n, sizeof(int64_t),
                                       cudaMemcpyDeviceToHost, s));
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(&tot[1], pos + g.n, sizeof(int64_t), cudaMemcpyDeviceToHost, s));
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
    if (g.cp_col_cap[nb] < tot[0]) {
        if (g.cp_col[nb]) cudaFree(g.cp_col[nb]);
        g.cp_col[nb] = nullptr;
        g.cp_col_cap[nb] = 0;
        if ((rc = alloc_bytes(g.ctx, (void**)&g.cp_col[nb], sizeof(int32_t) * (size_t)(tot[0] > 0 ? tot[0] : 1),
                              "compacted col")))
            return rc;
        g.cp_col_cap[nb] = tot[0];
    }
    k_compact_fill<<<grid, 256, 0, s>>>(g.rowptr, g.col, g.alive, g.vlist, g.vcount, g.cp_row[nb], pos,
                                        g.cp_col[nb], g.cp_list[nb]);
    count_launch(g, 1);
    KH_CUDA_TRY(g.ctx, cudaGetLastError());
    g.rowptr = g.cp_row[nb];
    g.col = g.cp_col[nb];
    g.vlist = g.cp_list[nb];
    g.vcount = tot[1];
    g.cp_cur = nb;
    return KH_OK;
}

int peel_grid(const Graph& g) {
    int64_t grid = (g.vcount + kPeelThreads - 1) / kPeelThreads;
    const int64_t gmax = (int64_t)g.ctx->sm_count * 4;
    if (grid > gmax) grid = gmax;
    return (int)(grid < 1 ? 1 : grid);
}

LbArgs lb_args(const Graph& g) {
    LbArgs a;
    a.lb = g.lb64;
    return a;
}

PeelState peel_state(const Graph& g) {
    PeelState p;
    p.c = g.pc;
    p.mn = g.pmn;
    p.mr = g.pmr;
    p.mu = g.pmu;
    p.left = g.pleft;
    p.gid = g.gid;
    return p;
}

int64_t peel_graphs(const Graph& g) { return g.gid ? g.ngraphs : 1; }

// Recompute the last level of the refine list (stale nodes with lb <= T).
int refine(Graph& g, bool sampled, cudaStream_t s) {
    const int grid = peel_grid(g);
    const LbArgs la = lb_args(g);
    prof_begin(g, kProfPeel, s);
    if (sampled)
        k_collect<unsigned long long><<<grid, kPeelThreads, 0, s>>>(
            g.alive, g.fresh, g.vcount, g.vlist, la, g.d64, g.dense ? 1 : 0, g.state, peel_state(g),
            g.listB);
    else
        k_collect<int32_t><<<grid, kPeelThreads, 0, s>>>(g.alive, g.fresh, g.vcount, g.vlist, la,
                                                         g.d32, g.dense ? 1 : 0, g.state,
                                                         peel_state(g), g.listB);
    count_launch(g, 1);
    prof_end(g, kProfPeel, s);
    if (sampled) return launch_level(g, g.h, g.listB, &g.state->nQ, 0, 0, s, 2);
    return launch_hdeg(g, g.listB, &g.state->nQ, 0, g.d32, nullptr, 0, 0, s,
                       &g.state->rc[kRcBfs], !g.dense);
}

// Start of a peel: levels below h in full (sampled), every node stale with its
// lower bound, then the nodes of smallest lower bound get exact values.
int start_peel(Graph& g, bool sampled, cudaStream_t s) {
    const int grid = peel_grid(g);
    int rc = KH_OK;
    if (sampled) {
        // every list below each node's last level; the last level itself stays lazy
        for (int i = 1; i < g.hmax && rc == KH_OK; ++i)
            rc = launch_level(g, i, nullptr, nullptr, g.n, 0, s, 0, 1);
        if (rc) return rc;
        KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.d64, 0xff, sizeof(unsigned long long) * (size_t)g.n, s));
        launch_stale_sampled(g, nullptr, nullptr, s);
    } else {
        k_init_exact<<<grid, kPeelThreads, 0, s>>>(g.rowptr, g.col, g.alive, g.start_keep ? 1 : 0,
                                                   g.n, g.degX, g.d32);
        count_launch(g, 1);
        launch_stale_exact(g, nullptr, nullptr, s);
    }
    const LbArgs la = lb_args(g);
    k_min_lb<<<grid, kPeelThreads, 0, s>>>(g.alive, g.fresh, g.n, la, g.state, peel_state(g));
    count_launch(g, 1);
    rc = refine(g, sampled, s);
    if (rc) return rc;
    // the bootstrap used the per-round counters: zero them for round 0
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.state->rc, 0, sizeof(int) * kRcCount, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(&g.state->nQ, 0, sizeof(int), s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.pmu, 0xff, sizeof(unsigned long long) * peel_graphs(g), s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.pmn, 0xff, sizeof(unsigned long long) * peel_graphs(g), s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.pmr, 0xff, sizeof(unsigned long long) * peel_graphs(g), s));
    return KH_OK;
}

// The second half of a round: the refresh of the nodes the removal set R
// affects, then the end of the round.
int refresh_and_finish(Graph& g, bool sampled, cudaStream_t s) {
    const int grid = peel_grid(g);
    const PeelState ps = peel_state(g);
    int rc = KH_OK;
    if (!sampled) {
        // the ball of R in the old graph: alive degrees drop (hop 1), the
        // nodes within h-1 hops become stale with new lower bounds ...
        const int hops = g.hmax > 2 ? g.hmax - 1 : 1;
        for (int hop = 1; hop <= hops; ++hop) launch_ball_hop(g, hop, s);
        launch_stale_exact(g, g.listW, &g.state->rc[kRcW], s);
        // ... and the nodes exactly h hops away lose exactly the removed nodes
        // within h hops: their values (and bounds) are decremented in place
        rc = launch_hdeg(g, g.listR, &g.state->nR, 0, g.d32, nullptr, 0, 0, s,
                         &g.state->rc[kRcLossWork], false, true);
        if (rc) return rc;
        launch_apply_loss(g, s);
    } else {
        int* rcs = g.state->rc;
        for (int i = 1; i <= g.hmax && rc == KH_OK; ++i) {
            // level i candidates: A(R), plus A(nodes whose level i-1 changed)
            launch_mark_neighbours(g, g.listR, &g.state->nR, i >= 2 ? g.listC[(i - 1) & 1] : nullptr,
                                   rcs + kRcC + i - 1, i, rcs + kRcW + i, s);
            // nodes with more levels recompute level i (tracking changes) ...
            if (i < g.hmax) rc = launch_level(g, i, g.listW, rcs + kRcW + i, 0, 1, s, 1);
            // ... nodes whose last level is i become stale (lazy refine)
            if (i >= g.hmin) launch_stale_sampled(g, g.listW, rcs + kRcW + i, s, i);
        }
        if (rc) return rc;
    }
    prof_begin(g, kProfPeel, s);
    k_finish<<<grid, kPeelThreads, 0, s>>>(g.alive, g.listR, g.state, g.deadbm, ps, peel_graphs(g));
    count_launch(g, 1);
    prof_end(g, kProfPeel, s);
    return KH_OK;
}

// One peeling round, entirely stream-ordered (capturable).
int launch_round(Graph& g, bool sampled, cudaStream_t s) {
    const int grid = peel_grid(g);
    int rc = KH_OK;
    if (g.dense) {
        // EstDense: the threshold stays infinite (no round minimum is taken),
        // so every stale node is recomputed in full before the sum is taken
        rc = refine(g, sampled, s);
        if (rc) return rc;
        prof_begin(g, kProfPeel, s);
        if (sampled)
            k_dense_sum<unsigned long long><<<grid, kPeelThreads, 0, s>>>(
                g.alive, g.d64, g.vcount, g.vlist, g.state, g.dsum, g.n + 1);
        else
            k_dense_sum<int32_t><<<grid, kPeelThreads, 0, s>>>(g.alive, g.d32, g.vcount, g.vlist,
                                                               g.state, g.dsum, g.n + 1);
        k_select_sched<<<grid, kPeelThreads, 0, s>>>(g.alive, g.sched, g.vcount, g.vlist, g.state,
                                                     g.listR, g.seen, g.round_of);
        count_launch(g, 2);
        prof_end(g, kProfPeel, s);
        return refresh_and_finish(g, sampled, s);
    }
    // U = min of the upper bounds (and of the fresh values); refine stale
    // nodes with lb <= max(c, U); the refine folds its results into mr
    prof_begin(g, kProfPeel, s);
    if (sampled)
        k_min_alive<unsigned long long><<<grid, kPeelThreads, 0, s>>>(
            g.alive, g.fresh, g.d64, g.vcount, g.vlist, g.state, g.pmu, g.pmn, g.gid);
    else
        k_min_alive<int32_t><<<grid, kPeelThreads, 0, s>>>(g.alive, g.fresh, g.d32, g.vcount, g.vlist,
                                                           g.state, g.pmu, g.pmn, g.gid);
    count_launch(g, 1);
    prof_end(g, kProfPeel, s);
    rc = refine(g, sampled, s);
    if (rc) return rc;
    prof_begin(g, kProfPeel, s);
    const PeelState ps = peel_state(g);
    if (sampled) {
        k_select<unsigned long long, unsigned long long><<<grid, kPeelThreads, 0, s>>>(
            g.alive, g.d64, g.vcount, g.vlist, g.state, ps, g.core64, g.round_of, g.listR, g.seen);
        count_launch(g, 1);
    } else {
        k_select<int32_t, int32_t><<<grid, kPeelThreads, 0, s>>>(
            g.alive, g.d32, g.vcount, g.vlist, g.state, ps, g.core32, g.round_of, g.listR, g.seen);
        count_launch(g, 1);
        if (!g.gid)  // the early stop of Sec. 5
            k_assign_rest<int32_t><<<grid, kPeelThreads, 0, s>>>(g.alive, g.vcount, g.vlist, g.state,
                                                                 ps, g.core32, g.round_of);
        else  // the same, graph by graph
            k_assign_rest_batch<int32_t><<<grid, kPeelThreads, 0, s>>>(g.alive, g.vcount, g.vlist,
                                                                       g.state, ps, g.core32,
                                                                       g.round_of);
        count_launch(g, 1);
    }
    prof_end(g, kProfPeel, s);
    return refresh_and_finish(g, sampled, s);
}

int check_state_err(Graph& g, const DevState& hs) {
    if (hs.err)
        return set_error(g.ctx, KH_EINTERNAL, "device check failed (flags 0x%x)", hs.err);
    return KH_OK;
}

// Capture kRoundsPerGraph rounds into an executable graph (cached per shape).
int round_graph(Graph& g, bool sampled, cudaStream_t s, cudaGraphExec_t* out) {
    // everything a captured launch bakes in: mode, h, M, slot size, scratch, batch tables
    const int key[10] = {(sampled ? 1 : 0) | (g.dense ? 2 : 0), g.h, (int)g.M, (int)g.cap,
                         (int)g.scratch_ctas, (int)(reinterpret_cast<uintptr_t>(g.hv) >> 4),
                         (int)(reinterpret_cast<uintptr_t>(g.Mv) >> 4), g.hmin,
                         (int)(reinterpret_cast<uintptr_t>(g.rowptr) >> 4), (int)g.vcount};
    if (g.round_exec && memcmp(key, g.round_exec_key, sizeof(key)) == 0) {
        *out = g.round_exec;
        return KH_OK;
    }
    if (g.round_exec) {
        cudaGraphExecDestroy(g.round_exec);
        g.round_exec = nullptr;
    }
    cudaGraph_t graph = nullptr;
    KH_CUDA_TRY(g.ctx, cudaStreamBeginCapture(s, cudaStreamCaptureModeRelaxed));
    int rc = KH_OK;
    const int64_t before = g.launches;
    for (int r = 0; r < kRoundsPerGraph && rc == KH_OK; ++r) rc = launch_round(g, sampled, s);
    g.round_exec_kernels = g.launches - before;  // captured, not yet run
    g.launches = before;
    cudaError_t e = cudaStreamEndCapture(s, &graph);
    if (rc) {
        if (graph) cudaGraphDestroy(graph);
        return rc;
    }
    if (e != cudaSuccess) return check_cuda(g.ctx, e, "cudaStreamEndCapture");
    e = cudaGraphInstantiate(&g.round_exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) {
        g.round_exec = nullptr;
        return check_cuda(g.ctx, e, "cudaGraphInstantiate");
    }
    memcpy(g.round_exec_key, key, sizeof(key));
    *out = g.round_exec;
    return KH_OK;
}

}  // namespace

int run_estimate_all(Graph& g) {
    cudaStream_t s = g.ctx->stream;
    int rc = ensure_work(g);
    if (rc) return rc;
    rc = ensure_lists(g);
    if (rc) return rc;
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.alive, 1, (size_t)g.n, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(&g.state->err, 0, sizeof(int), s));
    for (int i = 1; i <= g.hmax && rc == KH_OK; ++i)
        rc = launch_level(g, i, nullptr, nullptr, g.n, 0, s, 0, 0);
    if (rc) return rc;
    int err = 0;
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(&err, &g.state->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
    if (err) return set_error(g.ctx, KH_EINTERNAL, "device check failed (flags 0x%x)", err);
    return KH_OK;
}

// The peel's CSR and node list are the graph's own outside a peel.
struct PeelView {
    Graph& g;
    explicit PeelView(Graph& gg) : g(gg) {
        g.orig_rowptr = g.rowptr;
        g.orig_col = g.col;
        g.vlist = nullptr;
        g.vcount = g.n;
    }
    ~PeelView() {
        g.rowptr = g.orig_rowptr;
        g.col = g.orig_col;
        g.vlist = nullptr;
        g.vcount = g.n;
    }
};

constexpr int64_t kCompactMinAlive = 65536;  // automatic compaction only for larger graphs

int run_core(Graph& g, bool sampled, void* out_core, int32_t* round_of_host, bool out_dev) {
    (void)round_of_host;
    cudaStream_t s = g.ctx->stream;
    PeelView view(g);
    int rc = ensure_work(g);
    if (rc) return rc;
    if (sampled) {
        rc = ensure_lists(g);
        if (rc) return rc;
    }
    g.have_rounds = false;
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.alive, 1, (size_t)g.n, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.seen, 0xff, sizeof(int32_t) * (size_t)g.n, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.deadbm, 0, ((size_t)(g.n + 127) / 128) * 16, s));
    if (g.start_keep && g.n > 0) {
        k_init_keep<<<peel_grid(g), kPeelThreads, 0, s>>>(g.keep, g.n, g.alive, g.deadbm, g.round_of);
        count_launch(g, 1);
    }
    if (!sampled) KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.loss, 0, sizeof(int32_t) * (size_t)g.n, s));
    DevState init;
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(&init, g.state, sizeof(init), cudaMemcpyDeviceToHost, s));
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
    unsigned long long keep_bytes[kProfKinds];
    memcpy(keep_bytes, init.bytes, sizeof(keep_bytes));
    memset(&init, 0, sizeof(init));
    memcpy(init.bytes, keep_bytes, sizeof(keep_bytes));  // profiling counters accumulate
    init.minval = ~0ull;
    init.minU = ~0ull;
    init.n_alive = (int)(g.start_keep ? g.start_alive : g.n);
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(g.state, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));  // `init` is a host stack object
    const size_t pbytes = sizeof(unsigned long long) * (size_t)peel_graphs(g);
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.pc, 0, pbytes, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.pmn, 0xff, pbytes, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.pmr, 0xff, pbytes, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.pmu, 0xff, pbytes, s));
    if (g.gid) {
        // alive nodes per graph start at the graph sizes
        std::vector<int32_t> sizes((size_t)g.ngraphs);
        for (int64_t q = 0; q < g.ngraphs; ++q)
            sizes[(size_t)q] = (int32_t)((*g.h_vtx_off)[q + 1] - (*g.h_vtx_off)[q]);
        KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(g.pleft, sizes.data(), sizeof(int32_t) * sizes.size(),
                                           cudaMemcpyHostToDevice, s));
        KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));  // `sizes` is a host vector
    }
    rc = start_peel(g, sampled, s);
    if (rc) return rc;
    // the BFS scratch must exist before capture (its allocation may synchronize)
    DevState hs;
    int64_t launches = 0;
    cudaGraphExec_t exec = nullptr;
    const bool use_graph = !g.prof_on;
    if (use_graph) {
        rc = round_graph(g, sampled, s, &exec);
        if (rc) return rc;
    }
    int64_t compact_at = g.start_keep ? g.start_alive : g.n;  // alive count at the last compaction
    for (;;) {
        NvtxRange nvtx_range(use_graph ? "peel rounds (graph replay)" : "peel round");
        if (use_graph) {
            KH_CUDA_TRY(g.ctx, cudaGraphLaunch(exec, s));
            launches += kRoundsPerGraph;
            count_launch(g, g.round_exec_kernels);
        } else {
            rc = launch_round(g, sampled, s);
            if (rc) return rc;
            launches += 1;
        }
        KH_CUDA_TRY(g.ctx, cudaGetLastError());
        KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(&hs, g.state, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
        rc = check_state_err(g, hs);
        if (rc) return rc;
        if (hs.n_alive == 0) break;
        const bool may = g.compact_mode == KH_COMPACT_ALWAYS ||
                         (g.compact_mode == KH_VAR_AUTO && compact_at >= kCompactMinAlive);
        if (may && 2 * (int64_t)hs.n_alive <= compact_at) {
            NvtxRange nvtx_compact("peel compaction");
            rc = compact_peel(g, s);
            if (rc) return rc;
            compact_at = hs.n_alive;
            if (use_graph) {
                rc = round_graph(g, sampled, s, &exec);  // the launches changed: capture again
                if (rc) return rc;
            }
        }
        if (launches > g.n + 2 + kRoundsPerGraph)
            return set_error(g.ctx, KH_ETIMEOUT, "peeling did not finish within n+1 rounds");
    }
    g.last_rounds = hs.round;
    g.last_updates = (int64_t)hs.updates;
    for (int i = 0; i <= kMaxH; ++i) {
        g.last_lvl_work[i] = (int64_t)hs.lvl_work[i];
        g.last_lvl_changed[i] = (int64_t)hs.lvl_changed[i];
    }
    g.last_stopped = (int64_t)hs.stopped;
    g.have_rounds = true;
    const size_t bytes = (size_t)g.n * (sampled ? sizeof(unsigned long long) : sizeof(int32_t));
    const void* src = sampled ? (const void*)g.core64 : (const void*)g.core32;
    if (g.n > 0 && out_core)
        KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(out_core, src, bytes,
                                           out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!out_dev) KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
    return KH_OK;
}

}  // namespace kh
