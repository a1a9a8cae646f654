// kh_exact.cu -- ranks, CSR validation, exact h-degrees, removed-set balls.
//
// Exact h-degree (Sec. 2): deg_h(v; X) = |N(v; h, X)| - 1, N taken inside the
// alive set X.  One CTA runs one bounded breadth-first search at a time and
// takes the next source from a global counter (dynamic scheduling over a
// persistent grid).  The visited set is a bitmap of n bits, in shared memory
// when it fits (cleared with vector stores between sources) or else in a
// per-CTA global scratch slice (cleared by walking the visit queue).  Each
// frontier is expanded warp-per-vertex; vertices of degree >= kHeavyDeg (and a
// lone frontier vertex) are expanded by the whole CTA.  New vertices are
// appended to the CTA's queue with one warp-aggregated atomic per warp step.
#include <atomic>
#include <cstdio>
#include <cstring>

#include "kh_internal.cuh"

namespace kh {

namespace {

constexpr int kBfsThreads = 256;
constexpr int kHeavyDeg = 128;
constexpr int kMaxHeavy = 64;
constexpr uint32_t kFull = 0xffffffffu;

// SplitMix64 output function (Steele, Lea, Flood 2014).  The u-th output of a
// generator seeded with s is mix(s + (u + 1) * golden), so each rank is
// computed independently from its counter.
__device__ __forceinline__ uint64_t splitmix_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
    return z ^ (z >> 31);
}

// In a batch of graphs a node's counter is its id inside its own graph, so
// each graph gets the ranks it would get alone.
__global__ void k_ranks(uint8_t* __restrict__ r, int64_t n, uint64_t seed,
                        const int32_t* __restrict__ gid, const int64_t* __restrict__ vtx_off) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t u = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; u < n; u += stride) {
        const int64_t local = gid ? u - vtx_off[gid[u]] : u;
        const uint64_t x = splitmix_mix(seed + (uint64_t)(local + 1) * 0x9E3779B97F4A7C15ull);
        // trailing zeros, capped at 31: geometric(1/2) rank of Sec. 3
        r[u] = (uint8_t)(__ffsll((long long)(x | (1ull << 31))) - 1);
    }
}

// One warp per row: rows strictly increasing, ids in range, no self-loops,
// and every edge (u, v) has its reverse (binary search in row v).
__global__ void k_validate(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           int64_t n, int64_t nnz, int* err, const int32_t* __restrict__ gid) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t u = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; u < n; u += nw) {
        const int64_t b = rowptr[u], e = rowptr[u + 1];
        if (b < 0 || e < b || e > nnz) {
            if (lane == 0) atomicOr(err, kErrGraph);
            continue;
        }
        for (int64_t k = b + lane; k < e; k += 32) {
            const int32_t v = col[k];
            bool bad = v < 0 || (int64_t)v >= n || v == (int32_t)u;
            if (!bad && gid && gid[v] != gid[u]) bad = true;  // batch: no edge between graphs
            if (!bad && k > b && col[k - 1] >= v) bad = true;
            int64_t lo = 0, hi = -1;
            if (!bad) {
                lo = rowptr[v];
                hi = rowptr[v + 1] - 1;
                if (lo < 0 || hi >= nnz || hi < lo - 1) bad = true;
            }
            if (!bad) {
                bool found = false;
                while (lo <= hi) {
                    const int64_t mid = (lo + hi) >> 1;
                    const int32_t x = col[mid];
                    if (x == (int32_t)u) { found = true; break; }
                    if (x < (int32_t)u) lo = mid + 1; else hi = mid - 1;
                }
                bad = !found;
            }
            if (bad) atomicOr(err, kErrGraph);
        }
    }
}

struct BfsArgs {
    const int64_t* rowptr;
    const int32_t* col;
    const uint8_t* alive;
    const uint8_t* rank;
    int64_t n;
    int h;
    int words;                 // bitmap words
    const int32_t* worklist;   // nullptr: sources 0..count_static-1
    const int* d_count;
    int64_t count_static;
    int32_t* deg;
    int32_t* cnt;              // fixed-level counts (RANKS only)
    int jlo, nj;
    int32_t* queues;           // per-CTA queue, qcap entries each
    int64_t qcap;
    uint32_t* gbitmaps;        // per-CTA bitmaps (global mode)
    int* work_ctr;
    int* err;
    unsigned long long* updates;
    unsigned long long* bytes;  // algorithmic bytes: 8 + 4 deg per expanded vertex, 4 per result
    const int* skip;            // nonzero: the exact early stop fired, nothing to do
    const uint32_t* deadbm;     // removed-node bitmap (shared-memory mode): seeds the visited set
    // batches: graph of each node, first node of each graph, per-node h; the
    // visited bitmap is indexed by the id inside the source's graph
    const int32_t* gid;
    const int64_t* vtx_off;
    const uint8_t* hv;
    // early stop of the lazy refine (nullptr: every ball is completed)
    const unsigned long long* stop_c;
    const unsigned long long* stop_mu;
    unsigned long long* lb;
    uint8_t* fresh;
    unsigned long long* stopped;  // early-stop count
    unsigned long long* min_done;  // refine: per-graph minimum of the completed values
    // loss mode (nullptr: off): per-node loss counters and their list, the
    // ball stamps of the round and where the round index lives
    int32_t* loss;
    int32_t* loss_list;
    int* n_loss;
    const int32_t* seen;
    const int* round;
};

// Loss mode: u was first reached at the source's last hop.  Unless u is within
// h-1 hops of the removed set (stamped by the ball hops and made stale), every
// path of at most h edges from u avoids the removed nodes except at its end,
// so u's h-ball loses exactly the removed nodes within h hops: count this one.
__device__ __forceinline__ void loss_mark(const BfsArgs& a, int32_t u) {
    if (a.alive[u] != 1) return;
    if (a.seen[u] == (*a.round) * kPhaseStride) return;
    if (atomicAdd(a.loss + u, 1) == 0) {
        const int p = atomicAdd(a.n_loss, 1);
        if (p < a.n) a.loss_list[p] = u;
    }
}

// Visit neighbour u of a frontier vertex (all 32 lanes call this together;
// `valid` false for lanes past the end of the row).
template <bool RANKS, bool SEEDED, bool ALLALIVE = false>
__device__ __forceinline__ void visit(const BfsArgs& a, uint32_t* bm, int32_t* q, int* s_qtail,
                                      int* s_hist, bool valid, int32_t u, bool push, bool last,
                                      int lane,
                                      int& my, int32_t base) {
    bool isnew = false;
    // ALLALIVE (the allocation-free entry point, whose graph is not validated):
    // an id outside [0, n) is skipped, never used as a bitmap index
    if (ALLALIVE && valid && (uint32_t)u >= (uint32_t)a.n) {
        valid = false;
        atomicOr(a.err, kErrGraph);
    }
    // seeded: removed nodes already have their bit set, no alive lookup needed;
    // ALLALIVE: the whole graph, no alive array at all
    if (valid && (SEEDED || ALLALIVE || a.alive[u] == 1)) {
        const int32_t lu = u - base;
        const uint32_t bit = 1u << (lu & 31);
        uint32_t* wp = bm + (lu >> 5);
        if (!(*(volatile uint32_t*)wp & bit)) {
            const uint32_t old = atomicOr(wp, bit);
            isnew = !(old & bit);
        }
    }
    if (isnew) {
        ++my;
        if (RANKS) atomicAdd(&s_hist[a.rank[u]], 1);
        if (last && a.loss) loss_mark(a, u);
    }
    if (push) {
        const uint32_t nm = __ballot_sync(kFull, isnew);
        if (nm) {
            const int leader = __ffs(nm) - 1;
            int base = 0;
            if (lane == leader) base = atomicAdd(s_qtail, __popc(nm));
            base = __shfl_sync(kFull, base, leader);
            if (isnew) {
                const int pos = base + __popc(nm & ((1u << lane) - 1u));
                if (pos < a.qcap) q[pos] = u;
                else atomicOr(a.err, kErrQueue);
            }
        }
    }
}

// Add the lanes' new-vertex counts to the source's shared count (early stop).
__device__ __forceinline__ void fold_count(int& my, int* s_count, int lane) {
    int x = my;
    for (int off = 16; off > 0; off >>= 1) x += __shfl_down_sync(kFull, x, off);
    if (lane == 0 && x) atomicAdd(s_count, x);
    my = 0;
}

// Expand the row [b, e): lanes take 32 consecutive entries, each warp step
// issues four independent row loads before visiting (memory-level parallelism).
template <bool RANKS, bool SEEDED, bool ALLALIVE = false>
__device__ __forceinline__ void expand_row(const BfsArgs& a, uint32_t* bm, int32_t* q, int* s_qtail,
                                           int* s_hist, int64_t b, int64_t e, int64_t first,
                                           int64_t stride, bool push, bool last, int lane, int& my,
                                           int32_t base) {
    for (int64_t k0 = b + first; k0 < e; k0 += stride) {
        int32_t u[4];
        bool val[4];
#pragma unroll
        for (int qq = 0; qq < 4; ++qq) {
            const int64_t k = k0 + qq * 32 + lane;
            val[qq] = k < e;
            u[qq] = val[qq] ? __ldg(a.col + k) : 0;
        }
#pragma unroll
        for (int qq = 0; qq < 4; ++qq)
            visit<RANKS, SEEDED, ALLALIVE>(a, bm, q, s_qtail, s_hist, val[qq], u[qq], push, last, lane, my,
                                           base);
    }
}

template <bool RANKS, bool SMEM, bool ALLALIVE = false>
__global__ void __launch_bounds__(kBfsThreads) k_hdeg(BfsArgs a) {
    extern __shared__ __align__(16) uint32_t s_bm_dyn[];
    __shared__ int s_src, s_qtail, s_count, s_nheavy, s_stop;
    __shared__ unsigned long long s_T;
    __shared__ int s_hist[32];
    __shared__ int s_heavy[kMaxHeavy];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    uint32_t* bm = SMEM ? s_bm_dyn : a.gbitmaps + (size_t)blockIdx.x * (size_t)a.words;
    int32_t* q = a.queues + (size_t)blockIdx.x * (size_t)a.qcap;
    const int64_t total = (a.skip && *a.skip) ? 0 : (a.worklist ? (int64_t)(*a.d_count) : a.count_static);
    if (total == 0) return;
    unsigned long long my_bytes = 0;

    const bool seeded = SMEM && a.deadbm != nullptr && a.gid == nullptr;
    if (!seeded) {
        for (int i = tid; i < a.words; i += blockDim.x) bm[i] = 0u;
        __syncthreads();
    }

    for (;;) {
        if (tid == 0) s_src = atomicAdd(a.work_ctr, 1);
        __syncthreads();
        const int64_t idx = s_src;
        if (idx >= total) break;
        const int v = a.worklist ? a.worklist[idx] : (int)idx;
        // loss mode starts from the round's removed nodes (alive == 2)
        if (!ALLALIVE && (a.loss ? a.alive[v] == 0 : a.alive[v] != 1)) {
            if (tid == 0 && !a.loss) a.deg[v] = 0;
            if (RANKS && tid < a.nj) a.cnt[(size_t)v * a.nj + tid] = 0;
            __syncthreads();
            continue;
        }
        if (seeded) {
            // visited set := removed nodes (vector copy of the dead bitmap)
            const uint4* src = reinterpret_cast<const uint4*>(a.deadbm);
            uint4* dst = reinterpret_cast<uint4*>(bm);
            const int w4 = a.words >> 2;
            for (int i = tid; i < w4; i += blockDim.x) dst[i] = __ldg(src + i);
            for (int i = (w4 << 2) + tid; i < a.words; i += blockDim.x) bm[i] = __ldg(a.deadbm + i);
            __syncthreads();
        }
        const int32_t base = a.gid ? (int32_t)a.vtx_off[a.gid[v]] : 0;
        const int hsrc = a.hv ? (int)a.hv[v] : a.h;
        if (tid == 0) {
            q[0] = v;
            s_qtail = 1;
            s_count = 0;
            s_stop = 0;
            unsigned long long T = ~0ull;
            if (a.stop_c) {
                const int g = a.gid ? a.gid[v] : 0;
                T = stop_level(a.stop_c[g] > a.stop_mu[g] ? a.stop_c[g] : a.stop_mu[g]);
            }
            s_T = T;
            bm[(v - base) >> 5] |= 1u << ((v - base) & 31);
        }
        if (RANKS && tid < 32) s_hist[tid] = 0;
        __syncthreads();
        int fs = 0, fe = 1, my = 0;
        // early stop: rows fold their new vertices into s_count as they finish;
        // once it passes T the remaining rows are skipped (the visited set is a
        // subset of the ball, so the count is a lower bound of deg_h)
        const bool can_stop = s_T != ~0ull;
        const unsigned long long T = s_T;
        for (int d = 0; d < hsrc; ++d) {
            // vertices found at distance d+1 are queued if they will be expanded,
            // or, in global-bitmap mode, so the bitmap can be cleared by a walk
            const bool push = (d + 1 < hsrc) || !SMEM;
            const bool last = d + 1 == hsrc;
            if (tid == 0) s_nheavy = 0;
            __syncthreads();
            const bool single = (fe - fs) == 1;
            for (int i = fs + warp; i < fe; i += nwarps) {
                if (can_stop) {
                    int cnow = 0;
                    if (lane == 0) cnow = *(volatile int*)&s_count;
                    if ((unsigned long long)__shfl_sync(kFull, cnow, 0) > T) {
                        if (lane == 0) s_stop = 1;
                        break;
                    }
                }
                const int w = q[i];
                const int64_t b = a.rowptr[w], e = a.rowptr[w + 1];
                if (lane == 0) my_bytes += 8ull + 4ull * (unsigned long long)(e - b);
                if (single || e - b >= kHeavyDeg) {
                    int slot = 0;
                    if (lane == 0) slot = atomicAdd(&s_nheavy, 1);
                    slot = __shfl_sync(kFull, slot, 0);
                    if (slot < kMaxHeavy) {
                        if (lane == 0) s_heavy[slot] = w;
                        continue;
                    }
                }
                if (seeded)
                    expand_row<RANKS, true>(a, bm, q, &s_qtail, s_hist, b, e, 0, 128, push, last, lane, my,
                                            base);
                else
                    expand_row<RANKS, false, ALLALIVE>(a, bm, q, &s_qtail, s_hist, b, e, 0, 128, push,
                                                       last, lane, my, base);
                if (can_stop) fold_count(my, &s_count, lane);
            }
            __syncthreads();
            const int nh = min(s_nheavy, kMaxHeavy);
            for (int hi = 0; hi < nh; ++hi) {
                if (can_stop) {
                    fold_count(my, &s_count, lane);
                    int cnow = 0;
                    if (lane == 0) cnow = *(volatile int*)&s_count;
                    if ((unsigned long long)__shfl_sync(kFull, cnow, 0) > T) {
                        if (lane == 0) s_stop = 1;
                        break;
                    }
                }
                const int w = s_heavy[hi];
                const int64_t b = a.rowptr[w], e = a.rowptr[w + 1];
                if (seeded)
                    expand_row<RANKS, true>(a, bm, q, &s_qtail, s_hist, b, e, warp * 128,
                                            4 * blockDim.x, push, last, lane, my, base);
                else
                    expand_row<RANKS, false, ALLALIVE>(a, bm, q, &s_qtail, s_hist, b, e, warp * 128,
                                                       4 * blockDim.x, push, last, lane, my, base);
            }
            __syncthreads();
            if (s_stop) break;  // d(v) > T: the rest of the ball is not needed
            fs = fe;
            fe = min(s_qtail, (int)a.qcap);
            if (fs >= fe) break;  // nothing new: the ball is complete
        }
        // reduce the count of newly visited vertices
        for (int off = 16; off > 0; off >>= 1) my += __shfl_down_sync(kFull, my, off);
        if (lane == 0 && my) atomicAdd(&s_count, my);
        __syncthreads();
        if (tid == 0 && !a.loss) {
            if (s_stop) {
                // v stays stale: its upper bound is kept, its lower bound raised
                a.lb[v] = (unsigned long long)s_count;
                a.fresh[v] = 0;
                atomicAdd(a.stopped, 1ull);
            } else {
                // a completed ball is one h-degree update; a stopped one is not
                a.deg[v] = s_count;
                if (a.min_done)
                    atomicMin(a.min_done + (a.gid ? a.gid[v] : 0), (unsigned long long)s_count);
                atomicAdd(a.updates, 1ull);
            }
            my_bytes += 4ull + (RANKS ? 4ull * (unsigned long long)a.nj : 0ull);
        }
        if (RANKS && tid < a.nj) {
            int c = 0;
            for (int j = a.jlo + tid; j < 32; ++j) c += s_hist[j];
            a.cnt[(size_t)v * a.nj + tid] = c;
        }
        // clear the visited set for the next source (seeded sets are re-copied)
        if (seeded) {
        } else if (SMEM) {
            uint4* b4 = reinterpret_cast<uint4*>(bm);
            const int w4 = a.words >> 2;
            for (int i = tid; i < w4; i += blockDim.x) b4[i] = make_uint4(0u, 0u, 0u, 0u);
            for (int i = (w4 << 2) + tid; i < a.words; i += blockDim.x) bm[i] = 0u;
        } else {
            const int qt = min(s_qtail, (int)a.qcap);
            for (int i = tid; i < qt; i += blockDim.x) bm[(q[i] - base) >> 5] = 0u;
        }
        __syncthreads();
    }
    for (int off = 16; off > 0; off >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, off);
    if (lane == 0 && my_bytes) atomicAdd(a.bytes, my_bytes);
}

constexpr int kWarpRowX = 2048;   // longer rows are done by the whole block
constexpr int kBlockHeavyX = 64;

// One entry of a ball hop (all lanes of the warp together): u = col[k], when
// k < e, is stamped at its first visit of the round, joins the next frontier if
// a further hop below its h follows and, when alive, the stale list; hop 1 also
// lowers the alive degree of R's alive neighbours.
__device__ __forceinline__ void ball_entry(const int32_t* __restrict__ col,
                                           const uint8_t* __restrict__ alive,
                                           int32_t* __restrict__ seen, int32_t* __restrict__ fout,
                                           int* nfout, int32_t* __restrict__ wl, int* nwl,
                                           int h_all, int64_t cap, int32_t* __restrict__ degX,
                                           const uint8_t* __restrict__ hv, int hop, int stamp,
                                           int64_t k, int64_t e, int lane) {
    bool isnew = false;
    int32_t u = 0;
    uint8_t au = 0;
    int hu = h_all;
    if (k < e) {
        u = col[k];
        au = alive[u];
        if (hv) hu = (int)hv[u];  // batches: the h of u's graph
        // hop 1 scans each removed node's row once: alive neighbours lose a degree
        if (degX && au == 1) atomicSub(degX + u, 1);
        if (au != 0 && hop < hu && *(volatile int32_t*)(seen + u) != stamp)
            isnew = atomicExch(seen + u, stamp) != stamp;
    }
    const bool to_f = isnew && hop + 1 < hu;
    const bool to_w = isnew && au == 1;
    const uint32_t m1 = __ballot_sync(kFull, to_f);
    const uint32_t m2 = __ballot_sync(kFull, to_w);
    if (!(m1 | m2)) return;
    int b1 = 0, b2 = 0;
    if (lane == 0) {
        if (m1) b1 = atomicAdd(nfout, __popc(m1));
        if (m2) b2 = atomicAdd(nwl, __popc(m2));
    }
    b1 = __shfl_sync(kFull, b1, 0);
    b2 = __shfl_sync(kFull, b2, 0);
    const uint32_t lower = (1u << lane) - 1u;
    if (to_f) {
        const int p = b1 + __popc(m1 & lower);
        if (p < cap) fout[p] = u;
    }
    if (to_w) {
        const int p = b2 + __popc(m2 & lower);
        if (p < cap) wl[p] = u;
    }
}

// One hop of the ball around the removed set R in the OLD graph (alive != 0),
// for hops 1 .. h-1: every newly reached vertex is stamped, joins the next
// frontier (if a further hop below h follows) and, when it is still alive
// (alive == 1), the stale list.  Hop 1 also lowers the alive degrees of R's
// neighbours (with h = 1 it stamps nothing).  Nodes exactly h hops from R are
// handled by the loss BFS instead.  One warp per frontier vertex; rows longer
// than kWarpRowX are gathered per block and spread over all its warps.
__global__ void k_ball_hop(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                           const uint8_t* __restrict__ alive, int32_t* __restrict__ seen,
                           const int32_t* __restrict__ fin, const int* __restrict__ nfin,
                           int32_t* __restrict__ fout, int* nfout, int32_t* __restrict__ wl, int* nwl,
                           const DevState* __restrict__ st, int h_all, int64_t cap,
                           unsigned long long* bytes, int32_t* __restrict__ degX,
                           const uint8_t* __restrict__ hv, int hop) {
    if (st->early) return;
    __shared__ int s_heavy[kBlockHeavyX];
    __shared__ int s_nheavy;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int nin = *nfin;
    const int stamp = st->round * kPhaseStride;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_bytes = 0;
    if (threadIdx.x == 0) s_nheavy = 0;
    __syncthreads();
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nin; i += nw) {
        const int w = fin[i];
        const int64_t b = rowptr[w], e = rowptr[w + 1];
        if (e - b > kWarpRowX) {
            int slot = 0;
            if (lane == 0) slot = atomicAdd(&s_nheavy, 1);
            slot = __shfl_sync(kFull, slot, 0);
            if (slot < kBlockHeavyX) {
                if (lane == 0) s_heavy[slot] = w;
                continue;
            }
        }
        if (lane == 0) my_bytes += 12ull + 4ull * (unsigned long long)(e - b);
        for (int64_t k0 = b; k0 < e; k0 += 32)
            ball_entry(col, alive, seen, fout, nfout, wl, nwl, h_all, cap, degX, hv, hop, stamp,
                       k0 + lane, e, lane);
    }
    __syncthreads();
    const int nh = min(s_nheavy, kBlockHeavyX);
    for (int j = 0; j < nh; ++j) {
        const int w = s_heavy[j];
        const int64_t b = rowptr[w], e = rowptr[w + 1];
        if (threadIdx.x == 0) my_bytes += 12ull + 4ull * (unsigned long long)(e - b);
        for (int64_t k0 = b + warp * 32; k0 < e; k0 += blockDim.x)
            ball_entry(col, alive, seen, fout, nfout, wl, nwl, h_all, cap, degX, hv, hop, stamp,
                       k0 + lane, e, lane);
    }
    for (int off = 16; off > 0; off >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, off);
    if (lane == 0 && my_bytes) atomicAdd(bytes, my_bytes);
}

// Mark nodes stale and give each the lower bound max(deg_X(v), max_w deg_X(w))
// of deg_h(v; X), h >= 2: N(v; h) contains N(w; 1) for every alive neighbour w.
// The bound only depends on the 2-ball of v, which the h-ball refresh covers.
// One warp per node; rows longer than kWarpRowX go to the whole block.
// (A row longer than kStaleScanX takes the neighbour term from its neighbour
// of largest degree alone while that one is alive: still a lower bound.)
constexpr int kStaleScanX = 64;

__global__ void k_stale_exact(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const uint8_t* __restrict__ alive, const int32_t* __restrict__ degX,
                              const int32_t* __restrict__ list, const int* __restrict__ nlist,
                              int64_t n, uint8_t* __restrict__ fresh,
                              unsigned long long* __restrict__ lb, const DevState* __restrict__ st,
                              unsigned long long* bytes, int h_all, const uint8_t* __restrict__ hv,
                              const int32_t* __restrict__ bestnb) {
    if (st->early) return;
    __shared__ int s_max[kBfsThreads / 32];
    __shared__ int s_heavy[kBlockHeavyX];
    __shared__ int s_nheavy;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t cnt = list ? (int64_t)(*nlist) : n;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_bytes = 0;
    if (threadIdx.x == 0) s_nheavy = 0;
    __syncthreads();
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < cnt; i += nw) {
        const int v = list ? list[i] : (int)i;
        if (alive[v] != 1) continue;  // warp-uniform
        const int h = hv ? (int)hv[v] : h_all;
        const int64_t b = rowptr[v], e = rowptr[v + 1];
        if (bestnb && h >= 2 && e - b > kStaleScanX && alive[bestnb[v]] == 1) {
            if (lane == 0) {
                lb[v] = (unsigned long long)max(degX[bestnb[v]], degX[v]);
                fresh[v] = 0;
                my_bytes += 8ull + 5ull + 13ull;
            }
            continue;
        }
        if (h >= 2 && e - b > kWarpRowX) {
            int slot = 0;
            if (lane == 0) slot = atomicAdd(&s_nheavy, 1);
            slot = __shfl_sync(kFull, slot, 0);
            if (slot < kBlockHeavyX) {
                if (lane == 0) s_heavy[slot] = v;
                continue;
            }
        }
        int m = 0;
        if (h >= 2) {
            for (int64_t k = b + lane; k < e; k += 32) {
                const int32_t w = col[k];
                if (alive[w] == 1) m = max(m, degX[w]);
            }
            for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_down_sync(kFull, m, off));
        }
        if (lane == 0) {
            // h = 1: deg_1 = deg_X(v) itself; the neighbour term needs h >= 2
            lb[v] = (unsigned long long)max(m, degX[v]);
            fresh[v] = 0;
            my_bytes += 8ull + 5ull * (unsigned long long)(e - b) + 13ull;
        }
    }
    __syncthreads();
    const int nh = min(s_nheavy, kBlockHeavyX);
    for (int j = 0; j < nh; ++j) {
        const int v = s_heavy[j];
        const int64_t b = rowptr[v], e = rowptr[v + 1];
        int m = 0;
        for (int64_t k = b + threadIdx.x; k < e; k += blockDim.x) {
            const int32_t w = col[k];
            if (alive[w] == 1) m = max(m, degX[w]);
        }
        for (int off = 16; off > 0; off >>= 1) m = max(m, __shfl_down_sync(kFull, m, off));
        if (lane == 0) s_max[warp] = m;
        __syncthreads();
        if (threadIdx.x == 0) {
            for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = max(m, s_max[w]);
            lb[v] = (unsigned long long)max(m, degX[v]);
            fresh[v] = 0;
            my_bytes += 8ull + 5ull * (unsigned long long)(e - b) + 13ull;
        }
        __syncthreads();
    }
    for (int off = 16; off > 0; off >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, off);
    if (lane == 0 && my_bytes) atomicAdd(bytes, my_bytes);
}

// The nodes the loss BFS reached keep their state: d (exact when fresh, an
// upper bound when stale) and the stale lower bound both drop by the loss.
// Each is one h-degree update (an incremental recomputation).
__global__ void k_apply_loss(const int32_t* __restrict__ list, const int* __restrict__ nlist,
                             int32_t* __restrict__ loss, int32_t* __restrict__ d,
                             const uint8_t* __restrict__ fresh, unsigned long long* __restrict__ lb,
                             DevState* __restrict__ st, int64_t cap) {
    if (st->early) return;
    const int cnt = (int)min((int64_t)*nlist, cap);
    if (blockIdx.x == 0 && threadIdx.x == 0 && cnt > 0) {
        atomicAdd(&st->updates, (unsigned long long)cnt);
        atomicAdd(&st->bytes[kProfFrontier], 21ull * (unsigned long long)cnt);
    }
    for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < cnt; i += gridDim.x * blockDim.x) {
        const int v = list[i];
        const int l = loss[v];
        loss[v] = 0;
        d[v] -= l;
        if (!fresh[v]) {
            const unsigned long long x = lb[v];
            lb[v] = x > (unsigned long long)l ? x - (unsigned long long)l : 0ull;
        }
    }
}

// The neighbour of largest degree of each node (ties: the smaller id; -1 for
// an isolated node), one warp per node.
__global__ void k_best_nb(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                          int64_t n, int32_t* __restrict__ best) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
        long long key = -1;  // (degree << 32) | (0x7fffffff - id): max picks largest degree, smallest id
        for (int64_t k = rowptr[v] + lane; k < rowptr[v + 1]; k += 32) {
            const int32_t w = col[k];
            const long long kk = ((long long)(rowptr[w + 1] - rowptr[w]) << 32) | (long long)(0x7fffffff - w);
            key = key > kk ? key : kk;
        }
        for (int off = 16; off > 0; off >>= 1) {
            const long long o = __shfl_down_sync(kFull, key, off);
            key = key > o ? key : o;
        }
        if (lane == 0) best[v] = key < 0 ? -1 : (int32_t)(0x7fffffff - (int32_t)(key & 0x7fffffff));
    }
}

int pick_grid(int sm, int per_sm, int64_t work) {
    int64_t g = (int64_t)sm * per_sm;
    if (work < g) g = work;
    return (int)(g < 1 ? 1 : g);
}

}  // namespace

int ensure_bestnb(Graph& g, cudaStream_t s) {
    if (g.bestnb || g.n == 0) return KH_OK;
    int rc = alloc_bytes(g.ctx, (void**)&g.bestnb, sizeof(int32_t) * (size_t)g.n, "best neighbours");
    if (rc) return rc;
    k_best_nb<<<pick_grid(g.ctx->sm_count, 8, (g.n * 32 + 255) / 256), 256, 0, s>>>(g.rowptr, g.col,
                                                                                   g.n, g.bestnb);
    count_launch(g, 1);
    return KH_OK;
}

void launch_ranks(const Graph& g, cudaStream_t s) {
    if (g.n == 0) return;
    const int grid = pick_grid(g.ctx->sm_count, 4, (g.n + 255) / 256);
    k_ranks<<<grid, 256, 0, s>>>(g.rank, g.n, g.seed, g.gid, g.vtx_off);
    count_launch(const_cast<Graph&>(g), 1);
}

void launch_validate(const Graph& g, int* d_err, cudaStream_t s) {
    if (g.n == 0) return;
    const int grid = pick_grid(g.ctx->sm_count, 8, (g.n * 32 + 255) / 256);
    k_validate<<<grid, 256, 0, s>>>(g.rowptr, g.col, g.n, g.nnz, d_err, g.gid);
    count_launch(const_cast<Graph&>(g), 1);
}

int launch_hdeg(Graph& g, const int* worklist, const int* d_count, int64_t count_static,
                int32_t* deg, int32_t* cnt, int jlo, int nj, cudaStream_t s, int* round_ctr,
                bool early_stop, bool loss) {
    if (g.n == 0) return KH_OK;
    if (!worklist && count_static == 0) return KH_OK;
    // batches index the visited bitmap inside the source's graph
    const int64_t domain = g.gid ? g.max_gn : g.n;
    const int words = (int)((domain + 31) / 32);
    const int64_t words_padded = ((int64_t)words + 3) & ~(int64_t)3;
    const bool smem = words_padded * 4 <= kSmemBitmapMax;
    const size_t dyn = smem ? (size_t)words_padded * 4 : 0;
    void (*kern)(BfsArgs);
    if (cnt) kern = smem ? k_hdeg<true, true> : k_hdeg<true, false>;
    else kern = smem ? k_hdeg<false, true> : k_hdeg<false, false>;
    if (smem) {
        cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kSmemBitmapMax);
        if (e != cudaSuccess) return check_cuda(g.ctx, e, "cudaFuncSetAttribute(k_hdeg)");
    }
    int per_sm = 0;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBfsThreads, dyn);
    if (e != cudaSuccess) return check_cuda(g.ctx, e, "occupancy(k_hdeg)");
    if (per_sm < 1) per_sm = 1;
    if (!smem && per_sm > 2) per_sm = 2;  // global bitmaps: bound the scratch
    int64_t work = worklist ? g.n : count_static;
    const int grid = pick_grid(g.ctx->sm_count, per_sm, work);
    int rc = ensure_bfs_scratch(g, grid, !smem);
    if (rc) return rc;
    BfsArgs a{};
    a.rowptr = g.rowptr;
    a.col = g.col;
    a.alive = g.alive;
    a.rank = g.rank;
    a.n = g.n;
    a.h = g.h;
    a.words = words;
    a.worklist = worklist;
    a.d_count = d_count;
    a.count_static = count_static;
    a.deg = deg;
    a.cnt = cnt;
    a.jlo = jlo;
    a.nj = nj;
    a.queues = g.queues;
    a.qcap = domain;  // matches the per-CTA queue allocation of ensure_bfs_scratch
    a.gbitmaps = g.gbitmaps;
    a.work_ctr = round_ctr ? round_ctr : &g.state->work_ctr[0];
    a.err = &g.state->err;
    a.updates = &g.state->updates;
    a.bytes = &g.state->bytes[kProfBfs];
    a.skip = worklist ? &g.state->early : nullptr;
    a.deadbm = g.deadbm;
    a.gid = g.gid;
    a.vtx_off = g.vtx_off;
    a.hv = g.hv;
    const bool stop = early_stop && !cnt && !loss;
    a.min_done = (stop && !g.dense) ? g.pmr : nullptr;
    if (loss) {
        a.loss = g.loss;
        a.loss_list = g.listL;
        a.n_loss = &g.state->rc[kRcLossCount];
        a.seen = g.seen;
        a.round = &g.state->round;
    }
    a.stop_c = stop ? g.pc : nullptr;
    a.stop_mu = stop ? g.pmu : nullptr;
    a.lb = g.lb64;
    a.fresh = g.fresh;
    a.stopped = &g.state->stopped;
    if (!round_ctr) {
        e = cudaMemsetAsync(a.work_ctr, 0, sizeof(int), s);
        if (e != cudaSuccess) return check_cuda(g.ctx, e, "memset work_ctr");
    }
    prof_begin(g, kProfBfs, s);
    kern<<<grid, kBfsThreads, dyn, s>>>(a);
    count_launch(g, 1);
    prof_end(g, kProfBfs, s);
    return KH_OK;
}

void launch_ball_hop(Graph& g, int hop, cudaStream_t s) {
    // hop 1 starts from R; hop k >= 2 from the frontier written by hop k-1
    const int32_t* fin = hop == 1 ? g.listR : (hop & 1 ? g.listB : g.listA);
    const int* nfin = hop == 1 ? &g.state->nR : &g.state->rc[kRcF + hop - 1];
    int32_t* fout = hop & 1 ? g.listA : g.listB;
    int* nfout = &g.state->rc[kRcF + hop];
    const int grid = g.ctx->sm_count * 8;
    prof_begin(g, kProfFrontier, s);
    k_ball_hop<<<grid, 256, 0, s>>>(g.rowptr, g.col, g.alive, g.seen, fin, nfin, fout, nfout,
                                    g.listW, &g.state->rc[kRcW], g.state, g.h, g.n,
                                    &g.state->bytes[kProfFrontier], hop == 1 ? g.degX : nullptr,
                                    g.hv, hop);
    count_launch(g, 1);
    prof_end(g, kProfFrontier, s);
}

void launch_apply_loss(Graph& g, cudaStream_t s) {
    const int grid = g.ctx->sm_count * 4;
    prof_begin(g, kProfFrontier, s);
    k_apply_loss<<<grid, 256, 0, s>>>(g.listL, &g.state->rc[kRcLossCount], g.loss, g.d32, g.fresh,
                                      g.lb64, g.state, g.n);
    count_launch(g, 1);
    prof_end(g, kProfFrontier, s);
}

void launch_stale_exact(Graph& g, const int* list, const int* d_count, cudaStream_t s) {
    if (g.n == 0) return;
    const int grid = g.ctx->sm_count * 8;
    prof_begin(g, kProfFrontier, s);
    k_stale_exact<<<grid, kBfsThreads, 0, s>>>(g.rowptr, g.col, g.alive, g.degX, list, d_count, g.n,
                                       g.fresh, g.lb64, g.state, &g.state->bytes[kProfFrontier],
                                       g.h, g.hv, g.bestnb);
    count_launch(g, 1);
    prof_end(g, kProfFrontier, s);
}

// ---------------------------------------------------------------------------
// Exact h-degrees without any allocation
//
// Some callers cannot allocate device memory: a serving process whose device
// memory is carved up once at start-up by its own pool, or a real-time caller
// that must not block on the allocator.  This
// variant of the BFS kernel runs on caller-owned inputs and outputs and keeps
// its scratch (work counter and the per-CTA BFS queues) in one file-scope
// device array of fixed size, which every GPU that loads the library holds
// until the process exits.
// ---------------------------------------------------------------------------
namespace {
constexpr int64_t kNoAllocScratchInts = (int64_t)16 << 20;  // 64 MiB per device
constexpr int64_t kNoAllocHeaderInts = 64;                  // counters, 256-byte aligned
constexpr int kNoAllocMaxDevices = 64;
// the shared-memory visited bitmap bounds n: words * 4 <= kSmemBitmapMax
constexpr int64_t kNoAllocMaxN = (kSmemBitmapMax / 4) * 32;

static __device__ __align__(256) int32_t g_noalloc_scratch[kNoAllocScratchInts];
// host-side: the device address of g_noalloc_scratch on each device, looked
// up once per device (the symbol itself is only a host stand-in); atomic, as
// two host threads may make their first call on a device at the same time
std::atomic<int32_t*> g_noalloc_addr[kNoAllocMaxDevices] = {};
}  // namespace

}  // namespace kh

extern "C" int kh_hdegree_exact_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col,
                                        int32_t h, int32_t* deg, void* cuda_stream) {
    using namespace kh;
    if (n < 0 || h < 1 || h > kMaxH) return KH_EINVAL;
    if (n > kNoAllocMaxN) return KH_EINVAL;
    if (n == 0) return KH_OK;
    if (!rowptr || !col || !deg) return KH_EINVAL;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) {
        cudaGetLastError();
        return KH_ECUDA;
    }
    if (dev < 0 || dev >= kNoAllocMaxDevices) return KH_EINVAL;
    int32_t* base = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!base) {
        // first call on this device (with it current): find the array's address
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) {
            cudaGetLastError();
            return KH_ECUDA;
        }
        base = (int32_t*)p;  // every thread finds the same address
        g_noalloc_addr[dev].store(base, std::memory_order_release);
    }
    cudaStream_t s = (cudaStream_t)cuda_stream;
    int sm = 0;
    if (cudaDeviceGetAttribute(&sm, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) {
        cudaGetLastError();
        return KH_ECUDA;
    }
    const int words = (int)((n + 31) / 32);
    const size_t dyn = (size_t)((((int64_t)words + 3) & ~(int64_t)3) * 4);
    void (*kern)(BfsArgs) = k_hdeg<false, true, true>;
    if (cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemBitmapMax) !=
        cudaSuccess) {
        cudaGetLastError();
        return KH_ECUDA;
    }
    int per_sm = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kBfsThreads, dyn) != cudaSuccess) {
        cudaGetLastError();
        return KH_ECUDA;
    }
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)sm * per_sm;
    const int64_t fit = (kNoAllocScratchInts - kNoAllocHeaderInts) / n;  // queues of n entries
    if (grid > fit) grid = fit;
    if (grid > n) grid = n;
    BfsArgs a{};
    memset(&a, 0, sizeof(a));
    a.rowptr = rowptr;
    a.col = col;
    a.n = n;
    a.h = h;
    a.words = words;
    a.count_static = n;
    a.deg = deg;
    a.queues = base + kNoAllocHeaderInts;
    a.qcap = n;
    a.work_ctr = base;
    a.err = base + 1;
    a.updates = reinterpret_cast<unsigned long long*>(base + 4);
    a.bytes = reinterpret_cast<unsigned long long*>(base + 6);
    // the counters must start at zero; the queues need no clearing
    if (cudaMemsetAsync(base, 0, kNoAllocHeaderInts * sizeof(int32_t), s) != cudaSuccess) {
        cudaGetLastError();
        return KH_ECUDA;
    }
    kern<<<(int)grid, kBfsThreads, dyn, s>>>(a);
    if (cudaGetLastError() != cudaSuccess) return KH_ECUDA;
    return KH_OK;
}
