// kh_sampled.cu -- the level recursion of the sampled lists B[v,i], k[v,i].
//
// Prop. 3.1: B[v,i] is the rank filter of T = {v} U B[w,i-1] (w alive
// neighbours of v) at level k[v,i] >= max_w k[w,i-1], and Alg. 2 picks the
// smallest level leaving at most M members.  Because N(w; i-1) is inside
// N(v; i), the result equals {u in N(v;i,X) : r[u] >= kappa} with kappa the
// smallest level whose rank-filtered N(v;i,X) has at most M members, so B and
// k depend only on the alive set, the ranks and M.
//
// Level 1 (T = {v} plus alive neighbours, no repeats): one warp per node, a
// 32-bin rank histogram, kappa from its suffix sums, a second pass writes the
// members grouped by rank.
//
// Levels >= 2: one CTA per node with an open-addressing hash set of packed keys
// (r << 27 | id) in shared memory.  Warps stream the neighbours' lists
// (coalesced 32-key chunks).  A running threshold t starts at max_w k[w,i-1];
// keys below t are skipped, and because each list is grouped by rank from the
// highest, a warp stops reading a list at its first key below t.  After every
// chunk step the CTA raises t to the smallest level whose count of distinct
// keys is <= M (Alg. 5's trim), and compacts the set when dead entries pile
// up.  The last level only needs |B[v,h]| and k[v,h] for the estimate of
// Alg. 1, so it writes no list.
//
// A node's (|B|, k) pair changes exactly when B[v,i] or k[v,i] changes: with k
// fixed, the new list is a subset of the old one (nodes only leave), so equal
// sizes mean equal sets.  Changed nodes drive the next level's refresh (Alg. 3).
#include "kh_internal.cuh"

namespace kh {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr uint32_t kEmpty = 0xffffffffu;
constexpr int kL1Threads = 256;
constexpr int kLuThreads = 256;

struct LevelArgs {
    const int64_t* rowptr;
    const int32_t* col;
    const uint8_t* alive;
    const uint8_t* rank;
    int64_t n;
    int level;                 // level to compute; 0: each node's last level h(v)
    int h;                     // h of every node when hv is nullptr
    const uint8_t* hv;         // per-node h (batches)
    int skip_last;             // leave a node's last level to the lazy refine
    int64_t M;                 // M of every node when Mv is nullptr
    const int32_t* Mv;         // per-node M (batches)
    int64_t cap;
    uint32_t* keys;            // level i lists at keys + (i-1) n cap
    int32_t* lsz;              // |B[v,i]| at lsz + (i-1) n
    uint8_t* lk;               // k[v,i] at lk + (i-1) n
    uint8_t* ltop;             // highest rank in B[v,i] at ltop + (i-1) n, stored levels only
    unsigned long long* est;   // estimate (at a node's last level)
    const int32_t* worklist;
    const int* d_count;
    int64_t count_static;
    int track;
    int group_lists;           // free union: lane groups per list (0: a warp per list)
    int group_div;             // grouped: a group covers 1/group_div of the expected keys
    int32_t* changed;
    int* n_changed;
    int32_t* heavy;            // level 1: nodes of degree > kL1Heavy, for the CTA kernel
    int* n_heavy;
    int* work_ctr;
    int* err;
    unsigned long long* updates;
    unsigned long long* bytes;
    // Early stop of the lazy refine: a node whose partial estimate already
    // exceeds T = max(c, mu) of its graph cannot leave in this round, so it
    // stays stale with that value as its lower bound (nullptr: no early stop).
    const unsigned long long* stop_c;
    const unsigned long long* stop_mu;
    const int32_t* gid;
    unsigned long long* lb;
    uint8_t* fresh;
    // work statistics (indexed by level) and early-stop count
    unsigned long long* lvl_work;
    unsigned long long* lvl_changed;
    unsigned long long* stopped;
    int8_t* rho;  // tracked passes: top rank of each changed list's changes
    unsigned long long* min_done;  // refine: per-graph minimum of the completed values
    // split heavy nodes (k_levelU): partial sets of cap keys per part slot,
    // their sizes and levels, parts finished per split node (at its first
    // slot), each heavy node's first slot, the part items (part_cap 0: no split)
    uint32_t* part_keys;
    int32_t* part_size;
    uint8_t* part_t;
    int32_t* part_done;
    int32_t* part_stop;             // per split node: some part stopped early (refine)
    unsigned long long* part_lb;    // per split node: the largest partial estimate above T
    int32_t* split_first;
    int32_t* sub_v;
    int32_t* sub_j;
    int* n_sub;
    int64_t part_cap;
};

constexpr int kL1Heavy = 512;
// k_levelU splits nodes of more than kSplitDeg neighbours into parts of
// kSplitChunk neighbours each
constexpr int kSplitDeg = 4096;
constexpr int kSplitChunk = 2048;

// What one node computes in this launch: its level, whether that is its last
// level h(v) (estimate) or an intermediate one (list), its M, and where its
// inputs (level - 1) and outputs live.
struct NodeLevel {
    int lvl;
    bool last;
    bool skip;
    int64_t M;
    const uint32_t* keys_in;
    uint32_t* keys_out;
    const int32_t* lsz_in;
    const uint8_t* lk_in;
    const uint8_t* ltop_in;
    int32_t* lsz_out;
    uint8_t* lk_out;
    uint8_t* ltop_out;  // nullptr at a node's last level (no list is stored)
};

__device__ __forceinline__ NodeLevel node_level(const LevelArgs& a, int v) {
    NodeLevel nl;
    const int hvv = a.hv ? (int)a.hv[v] : a.h;
    nl.lvl = a.level ? a.level : hvv;
    nl.last = nl.lvl == hvv;
    nl.skip = nl.lvl > hvv || (nl.last && a.skip_last);
    nl.M = a.Mv ? (int64_t)a.Mv[v] : a.M;
    const size_t nn = (size_t)a.n, lc = nn * (size_t)a.cap;
    const int L = nl.lvl;
    nl.keys_in = L >= 2 ? a.keys + (size_t)(L - 2) * lc : nullptr;
    nl.keys_out = (!nl.last && a.keys) ? a.keys + (size_t)(L - 1) * lc : nullptr;
    nl.lsz_in = L >= 2 ? a.lsz + (size_t)(L - 2) * nn : nullptr;
    nl.lk_in = L >= 2 ? a.lk + (size_t)(L - 2) * nn : nullptr;
    nl.ltop_in = L >= 2 ? a.ltop + (size_t)(L - 2) * nn : nullptr;
    nl.lsz_out = a.lsz + (size_t)(L - 1) * nn;
    nl.lk_out = a.lk + (size_t)(L - 1) * nn;
    nl.ltop_out = (!nl.last && a.ltop) ? a.ltop + (size_t)(L - 1) * nn : nullptr;
    return nl;
}

__device__ __forceinline__ unsigned long long estimate_of(int S, int kappa, int rv, int64_t M) {
    // Alg. 1: d = |B[v,h] \ {v}| 2^k; if k > 0, d = max(d, M 2^(k-1))
    const int T = S - (rv >= kappa ? 1 : 0);
    unsigned long long d = (unsigned long long)T << kappa;
    if (kappa > 0) {
        const unsigned long long f = (unsigned long long)M << (kappa - 1);
        if (f > d) d = f;
    }
    return d;
}

__device__ __forceinline__ void record_change(const LevelArgs& a, const NodeLevel& nl, int v, int S,
                                              int kappa) {
    const int old_s = nl.lsz_out[v];
    const int old_k = nl.lk_out[v];
    nl.lsz_out[v] = S;
    nl.lk_out[v] = (uint8_t)kappa;
    if (a.track) atomicAdd(a.lvl_work + nl.lvl, 1ull);
    if (a.track && (old_s != S || old_k != kappa)) {
        atomicAdd(a.lvl_changed + nl.lvl, 1ull);
        const int p = atomicAdd(a.n_changed, 1);
        if (p < a.n) a.changed[p] = v;
    }
}

// rho of a tracked list about to be rewritten with (S, kappa): -2 when it is
// unchanged (same size and level imply the same members, as the level never
// rises and a list only gains members below its old level), else the highest
// rank among the members that left and, if the level fell, old level - 1 (the
// members that entered rank below the old level).  At level 1 the members that
// leave are exactly the removed ones.  Warp-wide; every lane gets the result.
__device__ __forceinline__ int level1_rho_warp(const LevelArgs& a, const NodeLevel& nl, int v,
                                               int S, int kappa, int lane) {
    const int old_s = nl.lsz_out[v], old_k = nl.lk_out[v];
    if (old_s == S && old_k == kappa) return -2;
    int r = kappa != old_k ? old_k - 1 : -1;
    const uint32_t* old = nl.keys_out + (size_t)v * (size_t)a.cap;
    const int m = min(old_s, (int)a.cap);
    for (int p = lane; p < m; p += 32) {
        const uint32_t key = old[p];
        if (a.alive[key & kIdMask] != 1) r = max(r, (int)(key >> kIdBits));
    }
    for (int off = 16; off > 0; off >>= 1) r = max(r, __shfl_xor_sync(kFull, r, off));
    return r;
}

// Bytes a node's level-1 computation must move: row offsets, the row, the
// neighbours' ranks, and the list it writes with its size and level.
__device__ __forceinline__ unsigned long long level1_bytes(int64_t deg, int S, int last) {
    return 8ull + 5ull * (unsigned long long)deg + (last ? 8ull : 4ull * (unsigned long long)S) + 5ull;
}

__global__ void __launch_bounds__(kL1Threads) k_level1(LevelArgs a) {
    __shared__ int s_hist[kL1Threads / 32][32];
    const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
    int* hist = s_hist[wib];
    const int64_t total = a.worklist ? (int64_t)(*a.d_count) : a.count_static;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_bytes = 0;
    for (int64_t idx = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; idx < total; idx += nw) {
        const int v = a.worklist ? a.worklist[idx] : (int)idx;
        if (a.alive[v] != 1) continue;
        const NodeLevel nl = node_level(a, v);
        if (nl.skip || nl.lvl != 1) continue;
        const int64_t b = a.rowptr[v], e = a.rowptr[v + 1];
        if (e - b > kL1Heavy) {
            if (lane == 0) {
                const int p = atomicAdd(a.n_heavy, 1);
                if (p < a.n) a.heavy[p] = v;
            }
            continue;
        }
        hist[lane] = 0;
        __syncwarp();
        for (int64_t k0 = b; k0 < e; k0 += 32) {
            const int64_t k = k0 + lane;
            if (k < e) {
                const int32_t u = a.col[k];
                if (a.alive[u] == 1) atomicAdd(&hist[a.rank[u]], 1);
            }
        }
        const int rv = a.rank[v];
        if (lane == 0) atomicAdd(&hist[rv], 1);
        __syncwarp();
        // S_j = #{u in T : r[u] >= j}, lane j holds S_j
        int S = hist[lane];
        for (int off = 1; off < 32; off <<= 1) {
            const int t = __shfl_down_sync(kFull, S, off);
            if (lane + off < 32) S += t;
        }
        const uint32_t over = __ballot_sync(kFull, S > nl.M);
        const int kappa = over ? 32 - __clz(over) : 0;
        const int Sk = __shfl_sync(kFull, S, kappa & 31);
        const int Skap = kappa < 32 ? Sk : 0;
        const uint32_t nz = __ballot_sync(kFull, S > 0);
        const int top = nz ? 31 - __clz(nz) : 0;  // highest rank present
        if (lane == 0) my_bytes += level1_bytes(e - b, Skap, nl.last);
        if (nl.last) {
            if (lane == 0) {
                const unsigned long long e = estimate_of(Skap, kappa, rv, nl.M);
                a.est[v] = e;
                if (a.min_done) atomicMin(a.min_done + (a.gid ? a.gid[v] : 0), e);
                record_change(a, nl, v, Skap, kappa);
                atomicAdd(a.updates, 1ull);
            }
            continue;
        }
        if (a.track) {
            // rho: the old list is read before it is overwritten
            const int r = level1_rho_warp(a, nl, v, Skap, kappa, lane);
            if (lane == 0 && r > -2) a.rho[v] = (int8_t)r;
        }
        // members grouped by rank, highest first: rank j starts at S_{j+1}
        const int above = __shfl_down_sync(kFull, S, 1);
        __syncwarp();
        hist[lane] = lane < 31 ? above : 0;
        __syncwarp();
        uint32_t* out = nl.keys_out + (size_t)v * (size_t)a.cap;
        for (int64_t k0 = b; k0 < e; k0 += 32) {
            const int64_t k = k0 + lane;
            if (k < e) {
                const int32_t u = a.col[k];
                if (a.alive[u] == 1) {
                    const int r = a.rank[u];
                    if (r >= kappa) {
                        const int p = atomicAdd(&hist[r], 1);
                        if (p < a.cap) out[p] = ((uint32_t)r << kIdBits) | (uint32_t)u;
                        else atomicOr(a.err, kErrList);
                    }
                }
            }
        }
        if (lane == 0) {
            if (rv >= kappa) {
                const int p = atomicAdd(&hist[rv], 1);
                if (p < a.cap) out[p] = ((uint32_t)rv << kIdBits) | (uint32_t)v;
                else atomicOr(a.err, kErrList);
            }
            if (nl.ltop_out) nl.ltop_out[v] = (uint8_t)top;
            record_change(a, nl, v, Skap, kappa);
        }
        __syncwarp();
    }
    for (int off = 16; off > 0; off >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, off);
    if (lane == 0 && my_bytes) atomicAdd(a.bytes, my_bytes);
}

// Level 1 for the nodes of degree > kL1Heavy deferred by k_level1: one CTA per node.
__global__ void __launch_bounds__(kL1Threads) k_level1_heavy(LevelArgs a) {
    __shared__ int s_hist[32];
    __shared__ int s_kappa, s_S, s_top;
    const int tid = threadIdx.x, lane = tid & 31;
    const int nh = *a.n_heavy;
    for (int idx = blockIdx.x; idx < nh; idx += gridDim.x) {
        const int v = a.heavy[idx];
        const NodeLevel nl = node_level(a, v);  // deferred by k_level1: level 1, not skipped
        if (tid < 32) s_hist[tid] = 0;
        __syncthreads();
        const int64_t b = a.rowptr[v], e = a.rowptr[v + 1];
        for (int64_t k = b + tid; k < e; k += blockDim.x) {
            const int32_t u = a.col[k];
            if (a.alive[u] == 1) atomicAdd(&s_hist[a.rank[u]], 1);
        }
        const int rv = a.rank[v];
        if (tid == 0) atomicAdd(&s_hist[rv], 1);
        __syncthreads();
        if (tid < 32) {
            int S = s_hist[lane];
            for (int off = 1; off < 32; off <<= 1) {
                const int t = __shfl_down_sync(kFull, S, off);
                if (lane + off < 32) S += t;
            }
            const uint32_t over = __ballot_sync(kFull, S > nl.M);
            const int kappa = over ? 32 - __clz(over) : 0;
            const int Sk = __shfl_sync(kFull, S, kappa & 31);
            const int above = __shfl_down_sync(kFull, S, 1);
            const uint32_t nz = __ballot_sync(kFull, S > 0);
            s_hist[lane] = lane < 31 ? above : 0;
            if (lane == 0) {
                s_kappa = kappa;
                s_S = kappa < 32 ? Sk : 0;
                s_top = nz ? 31 - __clz(nz) : 0;
            }
        }
        __syncthreads();
        const int kappa = s_kappa, Skap = s_S;
        if (nl.last) {
            if (tid == 0) {
                const unsigned long long e = estimate_of(Skap, kappa, rv, nl.M);
                a.est[v] = e;
                if (a.min_done) atomicMin(a.min_done + (a.gid ? a.gid[v] : 0), e);
                record_change(a, nl, v, Skap, kappa);
                atomicAdd(a.updates, 1ull);
                atomicAdd(a.bytes, level1_bytes(e - b, Skap, 1));
            }
        } else {
            if (a.track && tid < 32) {
                // rho (one warp); the old list is read before it is overwritten
                const int r = level1_rho_warp(a, nl, v, Skap, kappa, lane);
                if (lane == 0 && r > -2) a.rho[v] = (int8_t)r;
            }
            __syncthreads();
            uint32_t* out = nl.keys_out + (size_t)v * (size_t)a.cap;
            for (int64_t k = b + tid; k < e; k += blockDim.x) {
                const int32_t u = a.col[k];
                if (a.alive[u] == 1) {
                    const int r = a.rank[u];
                    if (r >= kappa) {
                        const int p = atomicAdd(&s_hist[r], 1);
                        if (p < a.cap) out[p] = ((uint32_t)r << kIdBits) | (uint32_t)u;
                        else atomicOr(a.err, kErrList);
                    }
                }
            }
            if (tid == 0) {
                if (rv >= kappa) {
                    const int p = atomicAdd(&s_hist[rv], 1);
                    if (p < a.cap) out[p] = ((uint32_t)rv << kIdBits) | (uint32_t)v;
                    else atomicOr(a.err, kErrList);
                }
                if (nl.ltop_out) nl.ltop_out[v] = (uint8_t)s_top;
                record_change(a, nl, v, Skap, kappa);
                atomicAdd(a.bytes, level1_bytes(e - b, Skap, 0));
            }
        }
        __syncthreads();
    }
}

// A flag another CTA of this launch may set (read past the L1 cache).
__device__ __forceinline__ int ld_acquire(const int32_t* p) {
    return *(volatile const int32_t*)p;
}

// Insert `key` into the shared hash set; returns its slot if it was not
// there, -1 if it was (or the probe limit was reached).
__device__ __forceinline__ int set_insert(uint32_t* tab, int lg, uint32_t key, int* err) {
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t s = ((key & kIdMask) * 0x9E3779B1u) >> (32 - lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        // most keys of a union are repeats: a plain read settles them without an atomic
        const uint32_t cur = *(volatile uint32_t*)(tab + s);
        if (cur == key) return -1;
        if (cur == kEmpty) {
            const uint32_t prev = atomicCAS(tab + s, kEmpty, key);
            if (prev == kEmpty) return (int)s;
            if (prev == key) return -1;
        }
        s = (s + 1u) & mask;
    }
    atomicOr(err, kErrProbe);
    return -1;
}

// Whether `key` is in the shared hash set (linear probing, no deletions
// between rebuilds).
__device__ __forceinline__ bool set_contains(const uint32_t* tab, int lg, uint32_t key) {
    const uint32_t mask = (1u << lg) - 1u;
    uint32_t s = ((key & kIdMask) * 0x9E3779B1u) >> (32 - lg);
    for (uint32_t probe = 0; probe <= mask; ++probe) {
        const uint32_t x = tab[s];
        if (x == key) return true;
        if (x == kEmpty) return false;
        s = (s + 1u) & mask;
    }
    return false;
}

// Grouped union: a lane group's step covers 1/kGroupDivDefault of the keys a
// list is expected to give (the rest take further steps).
constexpr int kGroupDivDefault = 1;

// Keys one thread loads per step (one 16-byte vector); a warp's chunk.
constexpr int kKeysPerLane = 4;
constexpr int kChunkKeys = 32 * kKeysPerLane;
// Nodes up to this degree use the flat (list, chunk) schedule of k_levelU.
constexpr int kFlatMax = kLuThreads;

// Shared memory of k_levelU for a table of 2^lg slots: keys, the compaction
// stage (scap keys: a compaction keeps the keys at or above the level trimmed
// from the complete counts, at most M), and the list of used slots (16-bit
// indices; a set holds at most half its slots plus what the warps insert
// before they stop for a compaction, under 2048).
__host__ __device__ __forceinline__ int levelU_used_cap(int hcap) { return (hcap >> 1) + 2048; }

int levelU_stage_cap(int lg, int64_t M) {
    const int64_t half = (int64_t)1 << (lg - 1);
    const int64_t need = (M + 64 + 3) & ~(int64_t)3;
    return (int)(need < half ? need : half);
}

size_t levelU_smem(int lg, int scap) {
    const size_t hcap = (size_t)1 << lg;
    return hcap * 4 + (size_t)scap * 4 + (size_t)levelU_used_cap((int)hcap) * 2;
}

// Drop the keys below t from the hash set: empty their slots, re-insert the
// rest (all threads of the CTA).
__device__ __forceinline__ void compact_set(uint32_t* tab, uint32_t* stage, uint16_t* used, int lg,
                                            int scap, int ucap, int tc, int* s_nused,
                                            int* s_nstage, int* err) {
    const int tid = threadIdx.x;
    const int nu = min(*s_nused, ucap);
    if (tid == 0) *s_nstage = 0;
    __syncthreads();
    for (int i = tid; i < nu; i += blockDim.x) {
        const int slot = used[i];
        const uint32_t key = tab[slot];
        tab[slot] = kEmpty;
        if ((int)(key >> kIdBits) >= tc) {
            const int p = atomicAdd(s_nstage, 1);
            if (p < scap) stage[p] = key;
            else atomicOr(err, kErrProbe);
        }
    }
    __syncthreads();
    if (tid == 0) *s_nused = 0;
    __syncthreads();
    const int ns = min(*s_nstage, scap);
    for (int i = tid; i < ns; i += blockDim.x) {
        const int slot = set_insert(tab, lg, stage[i], err);
        if (slot >= 0) used[atomicAdd(s_nused, 1)] = (uint16_t)slot;
    }
    __syncthreads();
}

// The warp's view of the union's rank counts: lane j gets S_j = #{distinct
// keys inserted so far with rank >= j}.  Read while other warps insert, the
// counts are those of a subset of the union (each rank class read at one
// moment), so every level derived from them is at most the final one and the
// partial estimate is at most the final estimate (Prop. 4.2).
__device__ __forceinline__ int snapshot_counts(const int* s_hist, int lane) {
    int S = *(volatile const int*)(s_hist + lane);
    for (int off = 1; off < 32; off <<= 1) {
        const int x = __shfl_down_sync(kFull, S, off);
        if (lane + off < 32) S += x;
    }
    return S;
}

// The union of free-running warps (k_levelU<true>): the warps' lanes form
// groups of G (G = 32: a warp per list); each group claims whole lists from a
// shared counter and reads its list 4 G keys per step (four keys per lane)
// until a key below the running level t shows (lists are grouped by rank,
// highest first).  After every step the warp raises t from its snapshot of
// the rank counts (Alg. 5's trim) and, in a refine, tests the partial
// estimate against T.  The CTA meets at a barrier only to compact the set
// (once it holds more than half its slots: at most one step per warp and one
// more from each other warp follow before they stop, so the set never fills)
// and at the end, where warp 0 trims from the complete counts.  Small groups
// suit many lists that each give a few keys above t: a warp step then covers
// 32 / G lists instead of one.
// Returns true when the refine stopped early (s_part holds the bound).
__device__ __forceinline__ bool free_union(const LevelArgs& a, const NodeLevel& nl, uint32_t* tab,
                                        uint32_t* stage, uint16_t* used, int lg, int hcap,
                                        int scap, int ucap,
                                        int* s_hist, int* s_t, int* s_nused, int* s_nstage,
                                        int* s_exit, unsigned long long* s_part, int* s_item,
                                        int* s_creq, unsigned long long T, int vin, bool can_stop,
                                        int mode, int first, int64_t b, int l0, int L, int rv,
                                        int G, unsigned long long& my_bytes) {
    const int tid = threadIdx.x, lane = tid & 31;
    if (tid == 0) {
        *s_item = 0;
        *s_creq = 0;
    }
    __syncthreads();
    // this group's open list (kept across a compaction): index (-1: none,
    // -2: the last claim found no list left), position, size
    int cli = -1, cpos = 0, csz = 0;
    const uint32_t* clp = nullptr;
    // every step claims a list or reads 4 keys of one: a bound on the steps
    // that no correct run reaches (past it: error flag, and the union ends)
    const long long cap64 = (long long)L * ((long long)a.cap / 4 + 2) + 4096;
    int steps_left = cap64 < 0x7fffffffLL ? (int)cap64 : 0x7fffffff;
    for (;;) {
        for (;;) {
            // one read for the whole warp: lanes that saw the flags at different
            // moments would leave the loop apart and stall the warp's shuffles
            int stop = 0;
            if (lane == 0) stop = *(volatile int*)s_creq | *(volatile int*)s_exit;
            if (__shfl_sync(kFull, stop, 0)) break;
            if (--steps_left < 0) {
                if (lane == 0) {
                    atomicOr(a.err, kErrLoop);
                    atomicCAS(s_exit, 0, 3);
                }
                break;
            }
            // groups without an open list claim the next lists (a list that
            // turns out dead, or with nothing at or above t, is passed over)
            for (int tries = 0; tries < 4; ++tries) {
                const bool need = cli == -1;
                const uint32_t nb = __ballot_sync(kFull, need && (lane & (G - 1)) == 0);
                if (!nb) break;
                const int lead = __ffs(nb) - 1;
                int base = 0;
                if (lane == lead) base = atomicAdd(s_item, __popc(nb));
                base = __shfl_sync(kFull, base, lead);
                int c = base + __popc(nb & ((1u << lane) - 1u)), sz = 0, w = -1;
                if (need && (lane & (G - 1)) == 0 && c < L) {
                    if (mode == 2) {
                        sz = __ldcg(a.part_size + first + c);
                    } else {
                        w = a.col[b + l0 + c];
                        // a list whose highest rank is below t has nothing to give
                        if (a.alive[w] == 1 && (int)nl.ltop_in[w] >= *(volatile int*)s_t)
                            sz = min(nl.lsz_in[w], (int)a.cap);
                    }
                }
                const int src = lane & ~(G - 1);
                c = __shfl_sync(kFull, c, src);
                sz = __shfl_sync(kFull, sz, src);
                w = __shfl_sync(kFull, w, src);
                if (need) {
                    if (c >= L) {
                        cli = -2;
                    } else if (sz > 0) {
                        cli = l0 + c;
                        cpos = 0;
                        csz = sz;
                        clp = mode == 2 ? a.part_keys + (size_t)(first + c) * (size_t)a.cap
                                        : nl.keys_in + (size_t)w * (size_t)a.cap;
                    }
                }
            }
            if (__all_sync(kFull, cli == -2)) break;
            const int t = *(volatile int*)s_t;
            bool below = false;
            const int p = cpos + (lane & (G - 1)) * kKeysPerLane;
            if (cli >= 0 && p < csz) {
                const uint4 k4 = mode == 2 ? __ldcg(reinterpret_cast<const uint4*>(clp + p))
                                           : *reinterpret_cast<const uint4*>(clp + p);
                const uint32_t kk[4] = {k4.x, k4.y, k4.z, k4.w};
                if (mode != 2) my_bytes += 4ull * (unsigned long long)min(kKeysPerLane, csz - p);
#pragma unroll
                for (int q = 0; q < kKeysPerLane; ++q) {
                    if (p + q < csz) {
                        const uint32_t key = kk[q];
                        const int r = (int)(key >> kIdBits);
                        if (r >= t) {
                            const int slot = set_insert(tab, lg, key, a.err);
                            if (slot >= 0) {
                                const int u = atomicAdd(s_nused, 1);
                                if (u < ucap) used[u] = (uint16_t)slot;
                                else atomicOr(a.err, kErrProbe);
                                atomicAdd(&s_hist[r], 1);
                            }
                        } else {
                            below = true;
                        }
                    }
                }
            }
            // ranks only fall along a list: after a key below t the rest is below t
            const uint32_t bal = __ballot_sync(kFull, below);
            if (cli >= 0) {
                const uint32_t gmask = G == 32 ? kFull : (((1u << G) - 1u) << (lane & ~(G - 1)));
                cpos += kKeysPerLane * G;
                if ((bal & gmask) || cpos >= csz) cli = -1;
            }
            // trim from this warp's snapshot; the early-stop test in a refine
            const int S = snapshot_counts(s_hist, lane);
            const uint32_t over = __ballot_sync(kFull, S > nl.M);
            const int pmax = over ? 31 - __clz(over) : -1;
            if (lane == 0 && pmax + 1 > t) atomicMax(s_t, pmax + 1);
            if (can_stop) {
                const int Sp = S + ((!vin && rv >= lane) ? 1 : 0);
                const uint32_t fits = __ballot_sync(kFull, Sp <= nl.M);
                const int k = fits ? __ffs(fits) - 1 : 32;
                const int Sk = __shfl_sync(kFull, Sp, k & 31);
                const unsigned long long pe = estimate_of(k < 32 ? Sk : 0, k, rv, nl.M);
                if (lane == 0 && pe > T) {
                    atomicMax(s_part, pe);
                    atomicCAS(s_exit, 0, 1);
                }
                // a part stops too once another part of the node has shown d(v) > T
                if (mode == 1 && lane == 0 && ld_acquire(a.part_stop + first)) atomicCAS(s_exit, 0, 2);
            }
            if (lane == 0 && *(volatile int*)s_nused > (hcap >> 1)) *(volatile int*)s_creq = 1;
        }
        __syncthreads();
        if (*(volatile int*)s_exit) return true;
        if (!*(volatile int*)s_creq) break;  // every list claimed and read
        // compaction: trim from the complete counts first, then drop keys below t
        if (tid < 32) {
            const int S = snapshot_counts(s_hist, lane);
            const uint32_t over = __ballot_sync(kFull, S > nl.M);
            const int pmax = over ? 31 - __clz(over) : -1;
            if (lane == 0 && pmax + 1 > *s_t) *s_t = pmax + 1;
        }
        __syncthreads();
        compact_set(tab, stage, used, lg, scap, ucap, *s_t, s_nused, s_nstage, a.err);
        if (tid == 0) *s_creq = 0;
        __syncthreads();
    }
    // the level from the complete counts
    if (tid < 32) {
        const int S = snapshot_counts(s_hist, lane);
        const uint32_t over = __ballot_sync(kFull, S > nl.M);
        const int pmax = over ? 31 - __clz(over) : -1;
        if (lane == 0 && pmax + 1 > *s_t) *s_t = pmax + 1;
    }
    __syncthreads();
    return false;
}

// Heavy nodes (degree > kSplitDeg) are split: part j unions the lists of
// neighbours [j kSplitChunk, (j+1) kSplitChunk) into its own trimmed partial
// set, and the CTA that finishes a node's last part merges the partial sets.
// The merge is exact: a part's level t_p (max of its neighbours' k[w,i-1] and
// its own trim) is at most the node's final level kappa, because adding lists
// only raises the counts S_j; so every member of B[v,i] (rank >= kappa) is in
// some partial set, and for j >= t* = max_p t_p the counts S_j of the union of
// the partial sets equal those of the full union.  The merge therefore runs the
// same running-threshold union over the partial sets from t = t*.
// FREE: the union's warps run free instead of in barrier-separated steps (see
// the FREE branch below); both give the same lists.
template <bool FREE>
__global__ void __launch_bounds__(kLuThreads, 6) k_levelU(LevelArgs a, int lg, int scap) {
    extern __shared__ __align__(16) uint32_t s_dyn[];
    const int hcap = 1 << lg;
    const int ucap = levelU_used_cap(hcap);
    uint32_t* tab = s_dyn;
    uint32_t* stage = s_dyn + hcap;                                         // scap keys
    uint16_t* used = reinterpret_cast<uint16_t*>(s_dyn + hcap + scap);      // ucap slots
    __shared__ int s_hist[32];
    __shared__ int s_src, s_t, s_nused, s_nstage, s_compact;
    __shared__ int s_vin, s_exit;                // own key in the table; early stop taken
    __shared__ int s_rho, s_last;
    __shared__ int s_item, s_creq;              // free mode: list claims; compaction request
    __shared__ float s_ex;                      // grouped free mode: expected keys x 2^t
    __shared__ unsigned long long s_T, s_part;  // early-stop threshold; partial estimate
    // flat mode (degree <= kFlatMax): per neighbour list its node, size, first
    // chunk index (exclusive prefix of 128-key chunk counts) and the first
    // chunk that showed a key below t (INT_MAX while none has)
    __shared__ int32_t s_w[kFlatMax];
    __shared__ int32_t s_sz[kFlatMax];
    __shared__ int32_t s_off[kFlatMax];
    __shared__ int32_t s_dead[kFlatMax];
    __shared__ int s_wsum[kLuThreads / 32];
    __shared__ int s_total;
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    const int nwarps = kLuThreads / 32;
    const int64_t total = a.worklist ? (int64_t)(*a.d_count) : a.count_static;
    const int64_t nsub = a.n_sub ? min((int64_t)(*a.n_sub), a.part_cap) : 0;
    if (total + nsub == 0) return;
    unsigned long long my_bytes = 0;
    // the table starts empty once per launch; every node leaves it empty again
    for (int i = tid; i < hcap; i += blockDim.x) tab[i] = kEmpty;
    for (;;) {
        if (tid == 0) s_src = atomicAdd(a.work_ctr, 1);
        __syncthreads();
        const int64_t idx = s_src;
        if (idx >= total + nsub) break;
        // mode 0: a whole node; 1: one part of a split node (2: its merge)
        int v, mode = 0, part = 0;
        if (idx < total) {
            v = a.worklist ? a.worklist[idx] : (int)idx;
        } else {
            v = a.sub_v[idx - total];
            part = a.sub_j[idx - total];
            mode = 1;
        }
        if (v < 0) {  // a part the plan could not place
            __syncthreads();
            continue;
        }
        const NodeLevel nl = node_level(a, v);
        const int64_t b = a.rowptr[v], e = a.rowptr[v + 1];
        const int deg = (int)(e - b);
        // a heavy node is done by its parts (k_split_plan gave it slots)
        if (a.alive[v] != 1 || nl.skip || nl.lvl < 2 ||
            (mode == 0 && a.part_cap > 0 && deg > kSplitDeg)) {
            __syncthreads();
            continue;
        }
        const int rv = a.rank[v];
        const int first = mode ? a.split_first[v] : -1;
        const int nparts = (deg + kSplitChunk - 1) / kSplitChunk;
        for (;;) {  // a node's last part continues as its merge (mode 2)
            // lists: neighbours [l0, l1) (modes 0, 1) or partial sets [0, nparts) (mode 2)
            const int l0 = mode == 1 ? part * kSplitChunk : 0;
            const int l1 = mode == 0 ? deg : (mode == 1 ? min(deg, l0 + kSplitChunk) : nparts);
            const int L = l1 - l0;
            if (tid < 32) s_hist[tid] = 0;
            if (tid == 0) {
                s_t = 0;
                s_ex = 0.f;
                s_nused = 0;
                s_vin = 0;
                s_exit = 0;
                s_part = 0;
                unsigned long long T = ~0ull;
                if (a.stop_c && nl.last && mode != 2) {
                    const int g = a.gid ? a.gid[v] : 0;
                    T = stop_level(a.stop_c[g] > a.stop_mu[g] ? a.stop_c[g] : a.stop_mu[g]);
                }
                s_T = T;
            }
            __syncthreads();
            const bool can_stop = s_T != ~0ull;
            // t starts at max k[w,i-1] over alive neighbours (Prop. 3.1), or at
            // the largest level of the partial sets (merge)
            // (grouped free union) also sum |B[w]| 2^k[w]: over 2^t it is the
            // expected number of keys at or above t (ranks halve per level)
            int myk = 0;
            float ex = 0.f;
            for (int li = l0 + tid; li < l1; li += blockDim.x) {
                int k = 0, sz = 0;
                if (mode == 2) {
                    k = (int)__ldcg(a.part_t + first + li);
                    sz = FREE && a.group_lists ? __ldcg(a.part_size + first + li) : 0;
                } else {
                    const int32_t w = a.col[b + li];
                    if (a.alive[w] == 1) {
                        k = (int)nl.lk_in[w];
                        sz = FREE && a.group_lists ? min(nl.lsz_in[w], (int)a.cap) : 0;
                    }
                }
                myk = max(myk, k);
                ex += (float)sz * (float)(1u << (k & 31));
            }
            for (int off = 16; off > 0; off >>= 1) {
                myk = max(myk, __shfl_down_sync(kFull, myk, off));
                ex += __shfl_down_sync(kFull, ex, off);
            }
            if (lane == 0 && myk) atomicMax(&s_t, myk);
            if (lane == 0 && ex > 0.f) atomicAdd(&s_ex, ex);
            __syncthreads();
            if (tid == 0 && rv >= s_t) {
                const int slot = set_insert(tab, lg, ((uint32_t)rv << kIdBits) | (uint32_t)v, a.err);
                if (slot >= 0) {
                    used[s_nused++] = (uint16_t)slot;
                    s_hist[rv] += 1;
                    s_vin = 1;
                }
            }
            __syncthreads();
            bool stopped = false;
            if constexpr (FREE) {
                // lanes per list: a warp, or (grouped) the fewest whose step of
                // 4 G keys covers the keys a list is expected to give at or
                // above the starting level
                int G = 32;
                if (a.group_lists) {
                    const float per = s_ex / (float)(1u << (s_t & 31)) / (float)(L > 0 ? L : 1);
                    while (G > 1 && (float)(kKeysPerLane * (G >> 1) * a.group_div) >= per) G >>= 1;
                }
                stopped = free_union(a, nl, tab, stage, used, lg, hcap, scap, ucap, s_hist, &s_t,
                                     &s_nused,
                                     &s_nstage, &s_exit, &s_part, &s_item, &s_creq, s_T, s_vin,
                                     can_stop, mode, first, b, l0, L, rv, G, my_bytes);
            } else {
            // Flat mode, whole nodes of degree <= kFlatMax: every (list, 128-key
            // chunk) pair is one work item, warps take items in order, one per
            // step, so long and short lists balance; a list is dropped once a
            // chunk shows a key below t.
            const bool flat = mode == 0 && deg <= kFlatMax;
            if (flat) {
                int cnt = 0;
                const int t0 = s_t;
                if (tid < deg) {
                    const int32_t w = a.col[b + tid];
                    int sz = 0;
                    // a list whose highest rank is below t has nothing to give
                    if (a.alive[w] == 1 && (int)nl.ltop_in[w] >= t0) sz = min(nl.lsz_in[w], (int)a.cap);
                    s_w[tid] = w;
                    s_sz[tid] = sz;
                    s_dead[tid] = INT_MAX;
                    cnt = (sz + kChunkKeys - 1) / kChunkKeys;
                }
                int inc = cnt;  // block-wide exclusive scan of the chunk counts
                for (int off = 1; off < 32; off <<= 1) {
                    const int x = __shfl_up_sync(kFull, inc, off);
                    if (lane >= off) inc += x;
                }
                if (lane == 31) s_wsum[warp] = inc;
                __syncthreads();
                int before = 0;
                for (int w2 = 0; w2 < warp; ++w2) before += s_wsum[w2];
                if (tid < deg) s_off[tid] = before + inc - cnt;
                if (tid == kLuThreads - 1) s_total = before + inc;
                __syncthreads();
            }
            int fbase = 0;  // flat mode: first item of this step
            // Grouped mode: G lanes share one list and read G*4 consecutive keys
            // per step; G shrinks as the number of lists grows, so that many
            // lists are open at once (hubs: one lane per list)
            int G = 32;
            while (G > 1 && (kLuThreads / G) < L) G >>= 1;
            const int ngroups = kLuThreads / G;
            const int gid = tid / G, gl = tid % G;
            const uint32_t gmask = (G == 32) ? kFull : (((1u << G) - 1u) << (lane & ~(G - 1)));
            const int step = kKeysPerLane * G;
            int li = l0 + gid;  // list index of this group's current list
            int pos = 0;
            bool any = true;
            while (any) {
                const int t = *(volatile int*)&s_t;
                if (flat) {
                    const int c = fbase + warp;
                    if (c < s_total) {
                        int lo = 0, hi = deg - 1;  // last list whose first chunk is <= c
                        while (lo < hi) {
                            const int mid = (lo + hi + 1) >> 1;
                            if (s_off[mid] <= c) lo = mid;
                            else hi = mid - 1;
                        }
                        // chunks after one with a key below t hold only keys below t;
                        // warps of one step run unordered, so an earlier chunk of the
                        // same list is still read even when a later one was seen first
                        if (c <= __shfl_sync(kFull, s_dead[lo], 0)) {
                            const int sz = s_sz[lo];
                            const int p = (c - s_off[lo]) * kChunkKeys + lane * kKeysPerLane;
                            bool below = false;
                            if (p < sz) {
                                const uint4 k4 = *reinterpret_cast<const uint4*>(
                                    nl.keys_in + (size_t)s_w[lo] * (size_t)a.cap + p);
                                const uint32_t kk[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
                                for (int q = 0; q < kKeysPerLane; ++q) {
                                    if (p + q < sz) {
                                        const uint32_t key = kk[q];
                                        const int r = (int)(key >> kIdBits);
                                        my_bytes += 4;
                                        if (r >= t) {
                                            const int slot = set_insert(tab, lg, key, a.err);
                                            if (slot >= 0) {
                                                const int u = atomicAdd(&s_nused, 1);
                                                if (u < ucap) used[u] = (uint16_t)slot;
                                                else atomicOr(a.err, kErrProbe);
                                                atomicAdd(&s_hist[r], 1);
                                            }
                                        } else {
                                            below = true;
                                        }
                                    }
                                }
                            }
                            // ranks only fall along a list: the rest of it is below t
                            if (__any_sync(kFull, below) && lane == 0) atomicMin(&s_dead[lo], c);
                        }
                    }
                    fbase += nwarps;
                }
                // advance to a list with keys left (group-uniform)
                const uint32_t* lp = nullptr;
                int sz = 0;
                while (!flat && li < l1) {
                    if (mode == 2) {
                        sz = __ldcg(a.part_size + first + li);
                        lp = a.part_keys + (size_t)(first + li) * (size_t)a.cap;
                        if (sz > pos) break;
                    } else {
                        const int32_t w = a.col[b + li];
                        if (a.alive[w] == 1 && (int)nl.ltop_in[w] >= t) {
                            sz = min(nl.lsz_in[w], (int)a.cap);
                            lp = nl.keys_in + (size_t)w * (size_t)a.cap;
                            if (sz > pos) break;
                        }
                    }
                    li += ngroups;
                    pos = 0;
                }
                bool below = false;
                if (!flat && li < l1) {
                    const int p = pos + gl * kKeysPerLane;
                    if (p < sz) {
                        const uint4 k4 = mode == 2 ? __ldcg(reinterpret_cast<const uint4*>(lp + p))
                                                   : *reinterpret_cast<const uint4*>(lp + p);
                        const uint32_t kk[4] = {k4.x, k4.y, k4.z, k4.w};
#pragma unroll
                        for (int q = 0; q < kKeysPerLane; ++q) {
                            if (p + q < sz) {
                                const uint32_t key = kk[q];
                                const int r = (int)(key >> kIdBits);
                                if (mode != 2) my_bytes += 4;
                                if (r >= t) {
                                    const int slot = set_insert(tab, lg, key, a.err);
                                    if (slot >= 0) {
                                        const int u = atomicAdd(&s_nused, 1);
                                        if (u < ucap) used[u] = (uint16_t)slot;
                                        else atomicOr(a.err, kErrProbe);
                                        atomicAdd(&s_hist[r], 1);
                                    }
                                } else {
                                    below = true;
                                }
                            }
                        }
                    }
                }
                const uint32_t bal = __ballot_sync(kFull, below);
                if (!flat && li < l1) {
                    if ((bal & gmask) || pos + step >= sz) {
                        li += ngroups;
                        pos = 0;
                    } else {
                        pos += step;
                    }
                }
                any = __syncthreads_or(flat ? fbase < s_total : li < l1);
                if (warp == 0) {
                    // smallest level >= t with at most M distinct members (Alg. 5's
                    // trim): lane j holds S_j = #{distinct keys with rank >= j}
                    int S = s_hist[lane];
                    for (int off = 1; off < 32; off <<= 1) {
                        const int x = __shfl_down_sync(kFull, S, off);
                        if (lane + off < 32) S += x;
                    }
                    const uint32_t over = __ballot_sync(kFull, S > nl.M);
                    const int pmax = over ? 31 - __clz(over) : -1;
                    if (can_stop) {
                        // Def. 4.1 on the keys inserted so far plus v itself: a subset
                        // of N(v;h) led by v, so by Prop. 4.2 at most the final estimate
                        const int Sp = S + ((!s_vin && rv >= lane) ? 1 : 0);
                        const uint32_t fits = __ballot_sync(kFull, Sp <= nl.M);
                        const int k = fits ? __ffs(fits) - 1 : 32;
                        const int Sk = __shfl_sync(kFull, Sp, k & 31);
                        const unsigned long long pe = estimate_of(k < 32 ? Sk : 0, k, rv, nl.M);
                        if (lane == 0 && pe > s_T) {
                            s_exit = 1;
                            s_part = pe;
                        }
                        // a part stops too once another part of the node has
                        // shown d(v) > T
                        if (mode == 1 && lane == 0 && !s_exit && ld_acquire(a.part_stop + first))
                            s_exit = 2;
                    }
                    if (lane == 0) {
                        const int told = s_t;
                        s_t = max(told, pmax + 1);
                        s_compact = s_nused > (hcap >> 1);
                        s_nstage = 0;
                    }
                }
                __syncthreads();
                if (s_exit && any) {  // (with every list read, finish: the exact value is kept)
                    stopped = true;
                    break;
                }
                if (s_compact) {
                    // drop keys below t: empty their slots, re-insert the rest
                    const int tc = s_t, nu = min(s_nused, ucap);
                    for (int i = tid; i < nu; i += blockDim.x) {
                        const int slot = used[i];
                        const uint32_t key = tab[slot];
                        tab[slot] = kEmpty;
                        if ((int)(key >> kIdBits) >= tc) {
                            const int p = atomicAdd(&s_nstage, 1);
                            if (p < scap) stage[p] = key;
                            else atomicOr(a.err, kErrProbe);
                        }
                    }
                    __syncthreads();
                    if (tid == 0) s_nused = 0;
                    __syncthreads();
                    const int ns = min(s_nstage, scap);
                    for (int i = tid; i < ns; i += blockDim.x) {
                        const int slot = set_insert(tab, lg, stage[i], a.err);
                        if (slot >= 0) used[atomicAdd(&s_nused, 1)] = (uint16_t)slot;
                    }
                    __syncthreads();
                }
            }
            }  // stepped union
            if (stopped) {
                // d(v) > T: v stays stale, its lower bound raised to the partial estimate
                const int nu = min(s_nused, ucap);
                for (int i = tid; i < nu; i += blockDim.x) tab[used[i]] = kEmpty;
                if (mode == 0) {
                    if (tid == 0) {
                        a.lb[v] = s_part;
                        a.fresh[v] = 0;
                        atomicAdd(a.stopped, 1ull);  // a lower bound only: not an update
                        my_bytes += 8ull + 10ull * (unsigned long long)deg + 9ull;
                    }
                    break;
                }
                // a part: its partial set (a sub-multiset of N(v; h) led by v)
                // already estimates above T; the node's last part finishes it
                if (tid == 0) {
                    if (s_exit == 1) atomicMax(a.part_lb + first, s_part);
                    a.part_stop[first] = 1;
                }
            }
            const int kappa = s_t;
            const int nu = min(s_nused, ucap);
            int S = 0;
            for (int j = kappa; j < 32; ++j) S += s_hist[j];
            __syncthreads();
            if (mode == 1 && stopped) {
                if (tid == 0) my_bytes += 10ull * (unsigned long long)L;
            } else if (mode == 1) {
                // this part's trimmed set, grouped by rank (highest first), and its level
                if (tid < 32) {
                    int above = 0;
                    for (int j = tid + 1; j < 32; ++j) above += s_hist[j];
                    __syncwarp();  // every lane has read before any lane writes
                    s_hist[tid] = above;
                }
                __syncthreads();
                uint32_t* out = a.part_keys + (size_t)(first + part) * (size_t)a.cap;
                for (int i = tid; i < nu; i += blockDim.x) {
                    const int slot = used[i];
                    const uint32_t key = tab[slot];
                    tab[slot] = kEmpty;
                    const int r = (int)(key >> kIdBits);
                    if (r >= kappa) {
                        const int p = atomicAdd(&s_hist[r], 1);
                        if (p < a.cap) out[p] = key;
                        else atomicOr(a.err, kErrList);
                    }
                }
                if (tid == 0) {
                    a.part_size[first + part] = S;
                    a.part_t[first + part] = (uint8_t)kappa;
                    my_bytes += 10ull * (unsigned long long)L;
                }
            }
            if (mode == 1) {
                __threadfence();
                __syncthreads();
                if (tid == 0) s_last = atomicAdd(a.part_done + first, 1) == nparts - 1;
                __syncthreads();
                if (!s_last) break;
                __threadfence();  // the other parts' sets are visible from here on
                if (__ldcg(a.part_stop + first)) {
                    // some part showed d(v) > T: v stays stale with that lower bound
                    if (tid == 0) {
                        a.lb[v] = __ldcg(a.part_lb + first);
                        a.fresh[v] = 0;
                        atomicAdd(a.stopped, 1ull);
                        a.part_stop[first] = 0;
                        a.part_lb[first] = 0;
                        a.part_done[first] = 0;
                    }
                    break;
                }
                mode = 2;
                continue;
            }
            if (tid == 0) my_bytes += 8ull + 5ull + (mode == 0 ? 10ull * (unsigned long long)deg : 0ull);
            if (nl.last) {
                if (tid == 0) {
                    const unsigned long long est = estimate_of(S, kappa, rv, nl.M);
                    a.est[v] = est;
                    if (a.min_done) atomicMin(a.min_done + (a.gid ? a.gid[v] : 0), est);
                    record_change(a, nl, v, S, kappa);
                    atomicAdd(a.updates, 1ull);
                    my_bytes += 8;
                }
                for (int i = tid; i < nu; i += blockDim.x) tab[used[i]] = kEmpty;
            } else {
                if (a.track) {
                    // rho (see level1_rho_warp): an old member left iff its key is
                    // not in the new union, where every key of rank >= kappa is kept
                    const int old_s = nl.lsz_out[v], old_k = nl.lk_out[v];
                    if (old_s != S || old_k != kappa) {
                        if (tid == 0) s_rho = kappa != old_k ? old_k - 1 : -1;
                        __syncthreads();
                        const uint32_t* old = nl.keys_out + (size_t)v * (size_t)a.cap;
                        const int m = min(old_s, (int)a.cap);
                        int r = -1;
                        for (int p = tid; p < m; p += blockDim.x) {
                            const uint32_t key = old[p];
                            if (!set_contains(tab, lg, key)) r = max(r, (int)(key >> kIdBits));
                        }
                        for (int off = 16; off > 0; off >>= 1) r = max(r, __shfl_xor_sync(kFull, r, off));
                        if (lane == 0 && r >= 0) atomicMax(&s_rho, r);
                        __syncthreads();  // the old list is read before it is overwritten
                        if (tid == 0) a.rho[v] = (int8_t)s_rho;
                    }
                }
                // write members grouped by rank, highest first, emptying the table
                if (tid < 32) {
                    const uint32_t nz = __ballot_sync(kFull, tid >= kappa && s_hist[tid] > 0);
                    if (tid == 0 && nl.ltop_out) nl.ltop_out[v] = (uint8_t)(nz ? 31 - __clz(nz) : 0);
                    __syncwarp();
                    int above = 0;
                    for (int j = tid + 1; j < 32; ++j) above += s_hist[j];
                    __syncwarp();
                    s_hist[tid] = above;  // start offset of rank tid
                }
                __syncthreads();
                uint32_t* out = nl.keys_out + (size_t)v * (size_t)a.cap;
                for (int i = tid; i < nu; i += blockDim.x) {
                    const int slot = used[i];
                    const uint32_t key = tab[slot];
                    tab[slot] = kEmpty;
                    const int r = (int)(key >> kIdBits);
                    if (r >= kappa) {
                        const int p = atomicAdd(&s_hist[r], 1);
                        if (p < a.cap) out[p] = key;
                        else atomicOr(a.err, kErrList);
                    }
                }
                if (tid == 0) {
                    record_change(a, nl, v, S, kappa);
                    my_bytes += 4ull * (unsigned long long)S;
                }
            }
            if (mode == 2 && tid == 0) a.part_done[first] = 0;  // ready for the next launch
            break;
        }
        __syncthreads();
    }
    for (int off = 16; off > 0; off >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, off);
    if (lane == 0 && my_bytes) atomicAdd(a.bytes, my_bytes);
}

// Plan the split of the heavy nodes of a level pass: every listed node that
// computes a level >= 2 and has more than kSplitDeg neighbours gets
// ceil(deg / kSplitChunk) consecutive part slots and part items.
__global__ void k_split_plan(LevelArgs a) {
    const int64_t total = a.worklist ? (int64_t)(*a.d_count) : a.count_static;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; idx < total; idx += stride) {
        const int v = a.worklist ? a.worklist[idx] : (int)idx;
        const int64_t deg = a.rowptr[v + 1] - a.rowptr[v];
        if (deg <= kSplitDeg || a.alive[v] != 1) continue;
        const NodeLevel nl = node_level(a, v);
        if (nl.skip || nl.lvl < 2) continue;
        const int P = (int)((deg + kSplitChunk - 1) / kSplitChunk);
        const int base = atomicAdd(a.n_sub, P);
        if ((int64_t)base + P <= a.part_cap) {
            for (int j = 0; j < P; ++j) {
                a.sub_v[base + j] = v;
                a.sub_j[base + j] = j;
            }
            a.split_first[v] = base;
        } else {
            // cannot happen: part_cap covers every heavy node of the graph at once
            for (int64_t j = base; j < a.part_cap && j < (int64_t)base + P; ++j) a.sub_v[j] = -1;
            atomicOr(a.err, kErrList);
        }
    }
}

// Rank filter for the neighbours of changed lists.  Level i of u is the
// rank filter (Prop. 3.1) of the union of its neighbours' level i-1 lists at
// k[u,i]; if every change of a neighbour's list (members that left, or members
// that entered below its old level) ranks below k[u,i] - 1, the counts S_j for
// j >= k[u,i] - 1, the level and the members are all unchanged.  The test needs
// k[u,i] for the current node set: intermediate levels always have it, a last
// level only while u is fresh.
struct MarkFilter {
    const int8_t* rho;    // nullptr: no filter
    const uint8_t* lk;    // k[u, phase]
    const uint8_t* hv;    // per-node h (batches) or nullptr
    int h;
    const uint8_t* fresh;
};

__device__ __forceinline__ bool level_may_change(const MarkFilter& f, int u, int rw, int level) {
    const int hu = f.hv ? (int)f.hv[u] : f.h;
    const bool known = level < hu || (level == hu && f.fresh[u]);
    return !known || rw >= (int)f.lk[u] - 1;
}

// Alive neighbours of the listed nodes (two lists, the second optional and
// rank-filtered) join the work list once per stamp (round, phase).  One CTA
// per listed node.
// (The CTA-wide path of the row kernels below: rows longer than kWarpRow are
// gathered per block and done by all its warps after the warp-per-node pass.)
constexpr int kWarpRow = 2048;
constexpr int kBlockHeavy = 64;

__device__ __forceinline__ unsigned long long umax64(unsigned long long a, unsigned long long b) {
    return a > b ? a : b;
}

// Visit entries [k0 + lane, ...) of a listed node's row: mark each alive
// neighbour that passes the filter once per stamp and append it to wl.
__device__ __forceinline__ void mark_entry(const int32_t* __restrict__ col,
                                           const uint8_t* __restrict__ alive,
                                           int32_t* __restrict__ seen, int32_t* __restrict__ wl,
                                           int* nwl, int64_t cap, const MarkFilter& f, bool filt,
                                           int rw, int phase, int stamp, int64_t k, int64_t e,
                                           int lane) {
    bool isnew = false;
    int32_t u = 0;
    if (k < e) {
        u = col[k];
        if (alive[u] == 1 && (!filt || level_may_change(f, u, rw, phase)) &&
            *(volatile int32_t*)(seen + u) != stamp)
            isnew = atomicExch(seen + u, stamp) != stamp;
    }
    const uint32_t m = __ballot_sync(kFull, isnew);
    if (!m) return;
    int base = 0;
    if (lane == 0) base = atomicAdd(nwl, __popc(m));
    base = __shfl_sync(kFull, base, 0);
    if (isnew) {
        const int p = base + __popc(m & ((1u << lane) - 1u));
        if (p < cap) wl[p] = u;
    }
}

__global__ void k_mark_nbrs(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                            const uint8_t* __restrict__ alive, int32_t* __restrict__ seen,
                            const int32_t* __restrict__ list1, const int* __restrict__ nlist1,
                            const int32_t* __restrict__ list2, const int* __restrict__ nlist2,
                            int32_t* __restrict__ wl, int* nwl, const DevState* __restrict__ st,
                            int phase, int64_t cap, unsigned long long* bytes, MarkFilter f) {
    __shared__ int s_heavy[kBlockHeavy];
    __shared__ int s_nheavy;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int n1 = *nlist1;
    const int nin = n1 + (list2 ? *nlist2 : 0);
    const int stamp = st->round * kPhaseStride + phase;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_bytes = 0;
    if (threadIdx.x == 0) s_nheavy = 0;
    __syncthreads();
    // one warp per listed node; rows longer than kWarpRow go to the block afterwards
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < nin; i += nw) {
        const int w = i < n1 ? list1[i] : list2[i - n1];
        const int64_t b = rowptr[w], e = rowptr[w + 1];
        if (e - b > kWarpRow) {
            int slot = 0;
            if (lane == 0) slot = atomicAdd(&s_nheavy, 1);
            slot = __shfl_sync(kFull, slot, 0);
            if (slot < kBlockHeavy) {
                if (lane == 0) s_heavy[slot] = (int)i;
                continue;
            }
        }
        const bool filt = f.rho != nullptr && i >= n1;
        const int rw = filt ? (int)f.rho[w] : 0;
        if (lane == 0) my_bytes += 12ull + 4ull * (unsigned long long)(e - b);
        for (int64_t k0 = b; k0 < e; k0 += 32)
            mark_entry(col, alive, seen, wl, nwl, cap, f, filt, rw, phase, stamp, k0 + lane, e, lane);
    }
    __syncthreads();
    const int nh = min(s_nheavy, kBlockHeavy);
    for (int j = 0; j < nh; ++j) {
        const int i = s_heavy[j];
        const int w = i < n1 ? list1[i] : list2[i - n1];
        const bool filt = f.rho != nullptr && i >= n1;
        const int rw = filt ? (int)f.rho[w] : 0;
        const int64_t b = rowptr[w], e = rowptr[w + 1];
        if (threadIdx.x == 0) my_bytes += 12ull + 4ull * (unsigned long long)(e - b);
        for (int64_t k0 = b + warp * 32; k0 < e; k0 += blockDim.x)
            mark_entry(col, alive, seen, wl, nwl, cap, f, filt, rw, phase, stamp, k0 + lane, e, lane);
    }
    for (int off = 16; off > 0; off >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, off);
    if (lane == 0 && my_bytes) atomicAdd(bytes, my_bytes);
}

// Alg. 1 on a level list of size S and level kappa, with the node of rank
// r_first counted first (it is a member of the list's neighbourhood).
__device__ __forceinline__ unsigned long long est_first(int S, int kappa, int r_first, int64_t M) {
    const int T = S - (r_first >= kappa ? 1 : 0);
    unsigned long long d = (unsigned long long)T << kappa;
    if (kappa > 0) {
        const unsigned long long f = (unsigned long long)M << (kappa - 1);
        if (f > d) d = f;
    }
    return d;
}

// Mark nodes stale at the last level h and give each a lower bound of its
// estimate: N(v; h-1) and, for every alive neighbour w, N(w; h-1) (which
// contains v) are inside N(v; h); Alg. 1 on either with v's rank first is at
// most the estimate of N(v; h) (Prop. 4.2).  Only the level-(h-1) sizes and
// levels are read.  One CTA per node.
// Batches: a node's h and M come from its graph, and only nodes whose last
// level is `only_h` (when nonzero) are marked.
// A row longer than kStaleScan takes its neighbour term from the neighbour
// of largest degree alone (bestnb) while that neighbour is alive: any alive
// neighbour w gives a sub-multiset N(w; h-1) of N(v; h) led by v, so one
// neighbour's term is still a lower bound, at O(1) cost instead of O(deg).
constexpr int kStaleScan = 64;

__global__ void k_stale_sampled(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const uint8_t* __restrict__ alive, const uint8_t* __restrict__ rank,
                                const int32_t* __restrict__ lsz, const uint8_t* __restrict__ lk,
                                int h_all, const uint8_t* __restrict__ hv, int64_t M_all,
                                const int32_t* __restrict__ Mv, int only_h,
                                const int32_t* __restrict__ list, const int* __restrict__ nlist,
                                int64_t n, uint8_t* __restrict__ fresh,
                                unsigned long long* __restrict__ lb, unsigned long long* bytes,
                                const int32_t* __restrict__ bestnb) {
    __shared__ unsigned long long s_max[kLuThreads / 32];
    __shared__ int s_heavy[kBlockHeavy];
    __shared__ int s_nheavy;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const int64_t cnt = list ? (int64_t)(*nlist) : n;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_bytes = 0;
    if (threadIdx.x == 0) s_nheavy = 0;
    __syncthreads();
    // one warp per node; rows longer than kWarpRow go to the block afterwards
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < cnt; i += nw) {
        const int v = list ? list[i] : (int)i;
        if (alive[v] != 1) continue;  // warp-uniform
        const int h = hv ? (int)hv[v] : h_all;
        if (only_h && h != only_h) continue;
        const int64_t b = rowptr[v], e = rowptr[v + 1];
        if (bestnb && h >= 2 && e - b > kStaleScan) {
            const int w = bestnb[v];
            if (alive[w] == 1) {  // warp-uniform
                if (lane == 0) {
                    const int64_t M = Mv ? (int64_t)Mv[v] : M_all;
                    const size_t off = (size_t)(h - 2) * (size_t)n;
                    const int rv = rank[v];
                    lb[v] = umax64(est_first(lsz[off + v], lk[off + v], rv, M),
                                   est_first(lsz[off + w], lk[off + w], rv, M));
                    fresh[v] = 0;
                    my_bytes += 29ull + 9ull;
                }
                continue;
            }
        }
        if (e - b > kWarpRow) {
            int slot = 0;
            if (lane == 0) slot = atomicAdd(&s_nheavy, 1);
            slot = __shfl_sync(kFull, slot, 0);
            if (slot < kBlockHeavy) {
                if (lane == 0) s_heavy[slot] = v;
                continue;
            }
        }
        const int64_t M = Mv ? (int64_t)Mv[v] : M_all;
        const int32_t* lsz_prev = h >= 2 ? lsz + (size_t)(h - 2) * (size_t)n : nullptr;
        const uint8_t* lk_prev = h >= 2 ? lk + (size_t)(h - 2) * (size_t)n : nullptr;
        unsigned long long m = 0;
        if (lsz_prev) {
            const int rv = rank[v];
            for (int64_t k = b + lane; k < e; k += 32) {
                const int32_t w = col[k];
                if (alive[w] == 1) m = umax64(m, est_first(lsz_prev[w], lk_prev[w], rv, M));
            }
            for (int off = 16; off > 0; off >>= 1) m = umax64(m, __shfl_down_sync(kFull, m, off));
            m = umax64(m, est_first(lsz_prev[v], lk_prev[v], rv, M));
        }
        if (lane == 0) {
            lb[v] = m;
            fresh[v] = 0;
            my_bytes += 29ull + 9ull * (unsigned long long)(e - b);
        }
    }
    __syncthreads();
    const int nh = min(s_nheavy, kBlockHeavy);
    for (int j = 0; j < nh; ++j) {
        const int v = s_heavy[j];
        const int h = hv ? (int)hv[v] : h_all;
        const int64_t M = Mv ? (int64_t)Mv[v] : M_all;
        const int32_t* lsz_prev = h >= 2 ? lsz + (size_t)(h - 2) * (size_t)n : nullptr;
        const uint8_t* lk_prev = h >= 2 ? lk + (size_t)(h - 2) * (size_t)n : nullptr;
        unsigned long long m = 0;
        const int64_t b = rowptr[v], e = rowptr[v + 1];
        if (lsz_prev) {
            const int rv = rank[v];
            for (int64_t k = b + threadIdx.x; k < e; k += blockDim.x) {
                const int32_t w = col[k];
                if (alive[w] == 1) m = umax64(m, est_first(lsz_prev[w], lk_prev[w], rv, M));
            }
            for (int off = 16; off > 0; off >>= 1) m = umax64(m, __shfl_down_sync(kFull, m, off));
            if (lane == 0) s_max[warp] = m;
            __syncthreads();
            if (threadIdx.x == 0) {
                for (int w = 1; w < (int)(blockDim.x >> 5); ++w) m = umax64(m, s_max[w]);
                m = umax64(m, est_first(lsz_prev[v], lk_prev[v], rv, M));
            }
        }
        if (threadIdx.x == 0) {
            lb[v] = m;
            fresh[v] = 0;
            my_bytes += 29ull + 9ull * (unsigned long long)(e - b);
        }
        __syncthreads();
    }
    for (int off = 16; off > 0; off >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, off);
    if (lane == 0 && my_bytes) atomicAdd(bytes, my_bytes);
}

}  // namespace

namespace {
// Part slots a whole-graph level pass needs: ceil(deg / kSplitChunk) per node
// of degree above kSplitDeg.
__global__ void k_count_parts(const int64_t* __restrict__ rowptr, int64_t n,
                              unsigned long long* out) {
    unsigned long long c = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int64_t deg = rowptr[v + 1] - rowptr[v];
        if (deg > kSplitDeg) c += (unsigned long long)((deg + kSplitChunk - 1) / kSplitChunk);
    }
    for (int off = 16; off > 0; off >>= 1) c += __shfl_down_sync(kFull, c, off);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(out, c);
}
}  // namespace

int ensure_split(Graph& g) {
    cudaStream_t s = g.ctx->stream;
    if (!g.split_planned) {
        unsigned long long* d = nullptr;
        unsigned long long parts = 0;
        KH_CUDA_TRY(g.ctx, cudaMallocAsync((void**)&d, sizeof(unsigned long long), s));
        cudaError_t e = cudaMemsetAsync(d, 0, sizeof(unsigned long long), s);
        if (e == cudaSuccess && g.n > 0) {
            k_count_parts<<<g.ctx->sm_count * 4, 256, 0, s>>>(g.rowptr, g.n, d);
            count_launch(g, 1);
        }
        if (e == cudaSuccess) e = cudaMemcpyAsync(&parts, d, sizeof(parts), cudaMemcpyDeviceToHost, s);
        if (e == cudaSuccess) e = cudaStreamSynchronize(s);
        cudaFreeAsync(d, s);
        if (e != cudaSuccess) return check_cuda(g.ctx, e, "count split parts");
        g.part_cap = (int64_t)parts;
        g.split_planned = true;
    }
    if (g.part_cap == 0) return KH_OK;
    if (g.part_keys && g.part_cap_keys < g.cap) {
        KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
        cudaFree(g.part_keys);
        g.part_keys = nullptr;
    }
    int rc;
    if (!g.part_keys) {
        if ((rc = alloc_bytes(g.ctx, (void**)&g.part_keys,
                              sizeof(uint32_t) * (size_t)g.part_cap * (size_t)g.cap, "split part keys")))
            return rc;
        g.part_cap_keys = g.cap;
    }
    const size_t pc = (size_t)g.part_cap;
    if (!g.part_done) {
        if ((rc = alloc_bytes(g.ctx, (void**)&g.part_done, sizeof(int32_t) * pc, "split part counters")))
            return rc;
        KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.part_done, 0, sizeof(int32_t) * pc, s));
    }
    if (!g.part_stop) {
        if ((rc = alloc_bytes(g.ctx, (void**)&g.part_stop, sizeof(int32_t) * pc, "split stop flags")))
            return rc;
        KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.part_stop, 0, sizeof(int32_t) * pc, s));
    }
    if (!g.part_lb) {
        if ((rc = alloc_bytes(g.ctx, (void**)&g.part_lb, sizeof(unsigned long long) * pc,
                              "split lower bounds")))
            return rc;
        KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.part_lb, 0, sizeof(unsigned long long) * pc, s));
    }
    if (!g.part_size && (rc = alloc_bytes(g.ctx, (void**)&g.part_size, sizeof(int32_t) * pc, "split part sizes")))
        return rc;
    if (!g.part_t && (rc = alloc_bytes(g.ctx, (void**)&g.part_t, pc, "split part levels"))) return rc;
    if (!g.sub_v && (rc = alloc_bytes(g.ctx, (void**)&g.sub_v, sizeof(int32_t) * pc, "split part nodes")))
        return rc;
    if (!g.sub_j && (rc = alloc_bytes(g.ctx, (void**)&g.sub_j, sizeof(int32_t) * pc, "split part indices")))
        return rc;
    if (!g.split_first &&
        (rc = alloc_bytes(g.ctx, (void**)&g.split_first, sizeof(int32_t) * (size_t)g.n, "split first slots")))
        return rc;
    return KH_OK;
}

int table_lg(int64_t M) {
    // capacity >= 2 (M + keys inserted per step) rounded up to a power of two
    int lg = 10;
    while ((int64_t(1) << lg) < 2 * (M + (int64_t)kKeysPerLane * kLuThreads)) ++lg;
    return lg;
}

int launch_level(Graph& g, int level, const int* worklist, const int* d_count,
                 int64_t count_static, int track, cudaStream_t s, int round_mode, int skip_last) {
    if (g.n == 0) return KH_OK;
    if (!worklist && count_static == 0) return KH_OK;
    LevelArgs a{};
    a.rowptr = g.rowptr;
    a.col = g.col;
    a.alive = g.alive;
    a.rank = g.rank;
    a.n = g.n;
    a.level = round_mode == 2 ? 0 : level;  // the refine computes each node's last level
    a.h = g.h;
    a.hv = g.hv;
    a.skip_last = skip_last < 0 ? (round_mode == 1 ? 1 : 0) : skip_last;
    a.M = g.M;
    a.Mv = g.Mv;
    a.cap = g.cap;
    a.keys = g.keys;
    a.lsz = g.lsz;
    a.lk = g.lk;
    a.ltop = g.ltop;
    a.est = g.d64;
    a.worklist = worklist;
    a.d_count = d_count;
    a.count_static = count_static;
    a.track = track;
    a.changed = g.listC[level & 1];
    a.heavy = g.listH;
    a.err = &g.state->err;
    a.updates = &g.state->updates;
    const bool stop = round_mode == 2;
    a.stop_c = stop ? g.pc : nullptr;
    a.stop_mu = stop ? g.pmu : nullptr;
    a.gid = g.gid;
    a.lb = g.lb64;
    a.fresh = g.fresh;
    a.rho = g.rho;
    a.min_done = (round_mode == 2 && !g.dense) ? g.pmr : nullptr;
    a.lvl_work = g.state->lvl_work;
    a.lvl_changed = g.state->lvl_changed;
    a.stopped = &g.state->stopped;
    int* rc = g.state->rc;
    if (round_mode == 1) {
        a.n_changed = rc + kRcC + level;
        a.n_heavy = rc + kRcLevelHeavy + level;
        a.work_ctr = rc + kRcLevelWork + level;
        a.n_sub = rc + kRcSub + level;
    } else if (round_mode == 2) {
        a.n_changed = rc + kRcC + 0;  // unused: the refine does not track changes
        a.n_heavy = rc + kRcRefineHeavy;
        a.work_ctr = rc + kRcRefineWork;
        a.n_sub = rc + kRcSub + 0;
    } else {
        a.n_changed = &g.state->nC[level & 1];
        a.n_heavy = &g.state->nH;
        a.work_ctr = &g.state->work_ctr[1];
        a.n_sub = &g.state->nSub;
    }
    a.part_cap = g.part_cap;
    a.part_keys = g.part_keys;
    a.part_size = g.part_size;
    a.part_t = g.part_t;
    a.part_done = g.part_done;
    a.part_stop = g.part_stop;
    a.part_lb = g.part_lb;
    a.split_first = g.split_first;
    a.sub_v = g.sub_v;
    a.sub_j = g.sub_j;
    cudaError_t e;
    if (track && round_mode == 0) {
        e = cudaMemsetAsync(a.n_changed, 0, sizeof(int), s);
        if (e != cudaSuccess) return check_cuda(g.ctx, e, "memset n_changed");
    }
    const int64_t work = worklist ? g.n : count_static;
    // which kernels can have nodes to do: level 1 (warp per node) and/or >= 2 (CTA per node)
    const bool want1 = round_mode == 2 ? g.hmin == 1 : level == 1;
    const bool wantU = round_mode == 2 ? g.hmax >= 2 : level >= 2;
    if (want1) {
        a.bytes = &g.state->bytes[kProfLevel1];
        if (round_mode == 0) {
            e = cudaMemsetAsync(a.n_heavy, 0, sizeof(int), s);
            if (e != cudaSuccess) return check_cuda(g.ctx, e, "memset n_heavy");
        }
        int64_t grid = (work + (kL1Threads / 32) - 1) / (kL1Threads / 32);
        const int64_t gmax = (int64_t)g.ctx->sm_count * 8;
        if (grid > gmax) grid = gmax;
        if (grid < 1) grid = 1;
        prof_begin(g, kProfLevel1, s);
        k_level1<<<(int)grid, kL1Threads, 0, s>>>(a);
        k_level1_heavy<<<g.ctx->sm_count * 2, kL1Threads, 0, s>>>(a);
        count_launch(g, 2);
        prof_end(g, kProfLevel1, s);
    }
    if (!wantU) return KH_OK;
    a.bytes = &g.state->bytes[kProfLevelU];
    const int lg = table_lg(g.M);
    const int scap = levelU_stage_cap(lg, g.M);
    const size_t dyn = levelU_smem(lg, scap);
    // free-running lane groups unless another schedule is asked for (grouped
    // is the fastest, or within 2%, on every measured workload)
    void (*kern)(LevelArgs, int, int) =
        g.levelu_mode == KH_LEVELU_STEPPED ? k_levelU<false> : k_levelU<true>;
    a.group_lists = g.levelu_mode == KH_LEVELU_FREE ? 0 : 1;
    a.group_div = g.levelu_div > 0 ? g.levelu_div : kGroupDivDefault;
    // the largest table any graph can ask for (M up to kMaxM)
    const int lg_max = table_lg(kMaxM);
    e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)levelU_smem(lg_max, levelU_stage_cap(lg_max, kMaxM)));
    if (e != cudaSuccess) return check_cuda(g.ctx, e, "cudaFuncSetAttribute(k_levelU)");
    int per_sm = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kLuThreads, dyn);
    if (e != cudaSuccess) return check_cuda(g.ctx, e, "occupancy(k_levelU)");
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)g.ctx->sm_count * per_sm;
    if (work < grid) grid = work;
    if (grid < 1) grid = 1;
    if (round_mode == 0) {
        e = cudaMemsetAsync(a.work_ctr, 0, sizeof(int), s);
        if (e != cudaSuccess) return check_cuda(g.ctx, e, "memset work_ctr");
        if (g.part_cap > 0) {
            e = cudaMemsetAsync(a.n_sub, 0, sizeof(int), s);
            if (e != cudaSuccess) return check_cuda(g.ctx, e, "memset n_sub");
        }
    }
    prof_begin(g, kProfLevelU, s);
    if (g.part_cap > 0) {
        k_split_plan<<<g.ctx->sm_count * 2, 256, 0, s>>>(a);
        count_launch(g, 1);
        // parts need CTAs of their own beyond the node count
        const int64_t cap = (int64_t)g.ctx->sm_count * per_sm;
        grid = cap;
    } else {
        a.n_sub = nullptr;
    }
    kern<<<(int)grid, kLuThreads, dyn, s>>>(a, lg, scap);
    count_launch(g, 1);
    prof_end(g, kProfLevelU, s);
    return KH_OK;
}

void launch_mark_neighbours(Graph& g, const int* list1, const int* cnt1, const int* list2,
                            const int* cnt2, int phase, int* out_count, cudaStream_t s) {
    const int grid = g.ctx->sm_count * 8;
    prof_begin(g, kProfFrontier, s);
    MarkFilter f{};
    if (list2) {
        f.rho = g.rho;
        f.lk = g.lk + (size_t)(phase - 1) * (size_t)g.n;
        f.hv = g.hv;
        f.h = g.h;
        f.fresh = g.fresh;
    }
    k_mark_nbrs<<<grid, 256, 0, s>>>(g.rowptr, g.col, g.alive, g.seen, list1, cnt1, list2, cnt2,
                                     g.listW, out_count, g.state, phase, g.n,
                                     &g.state->bytes[kProfFrontier], f);
    count_launch(g, 1);
    prof_end(g, kProfFrontier, s);
}

// lvl_out[v] = k[v, h(v)], bs_out[v] = |B[v, h(v)]| (each node's last level)
__global__ void k_gather_last(int64_t n, int h_all, const uint8_t* __restrict__ hv,
                              const int32_t* __restrict__ lsz, const uint8_t* __restrict__ lk,
                              uint8_t* __restrict__ lvl_out, int32_t* __restrict__ bs_out) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int h = hv ? (int)hv[v] : h_all;
        const size_t at = (size_t)(h - 1) * (size_t)n + (size_t)v;
        if (lvl_out) lvl_out[v] = lk[at];
        if (bs_out) bs_out[v] = lsz[at];
    }
}

void launch_gather_last(Graph& g, uint8_t* lvl_out, int32_t* bs_out, cudaStream_t s) {
    if (g.n == 0) return;
    k_gather_last<<<g.ctx->sm_count * 4, 256, 0, s>>>(g.n, g.h, g.hv, g.lsz, g.lk, lvl_out, bs_out);
    count_launch(g, 1);
}

void launch_stale_sampled(Graph& g, const int* list, const int* d_count, cudaStream_t s, int only_h) {
    if (g.n == 0) return;
    const int grid = g.ctx->sm_count * 8;
    prof_begin(g, kProfFrontier, s);
    k_stale_sampled<<<grid, kLuThreads, 0, s>>>(g.rowptr, g.col, g.alive, g.rank, g.lsz, g.lk, g.h,
                                                g.hv, g.M, g.Mv, only_h, list, d_count, g.n,
                                                g.fresh, g.lb64, &g.state->bytes[kProfFrontier],
                                                g.bestnb);
    count_launch(g, 1);
    prof_end(g, kProfFrontier, s);
}

}  // namespace kh
