// kh_internal.cuh -- internal declarations of the (k,h)-core CUDA library.
//
// Device data layout of one graph (all arrays in HBM, owned by kh_graph):
//   rowptr   int64[n+1], col int32[nnz]      symmetric CSR, rows sorted
//   rank     uint8[n]                          r[v] (Sec. 3)
//   alive    uint8[n]                          1 alive, 2 removed in the current
//                                              peeling round (still part of the
//                                              old graph), 0 removed earlier
//   keys     uint32[(h-1) * n * cap]           B[v,i] for levels i = 1..h-1, one
//                                              fixed slot of cap >= M keys per
//                                              (level, node); key = r << 27 | id,
//                                              grouped by rank, highest first
//   lsz      int32[h * n], lk uint8[h * n]     |B[v,i]| and k[v,i], i = 1..h
//   d32 / d64                                  deg_h (exact) or estimate (sampled)
//   seen     int32[n]                          stamp array for frontier dedup
//   lists    int32[n] x 4                      removed set, frontiers, work lists
//   state    kh_dev_state                      round counters (device resident)
//   scratch  per-CTA BFS queues (and bitmaps when n is too large for shared memory)
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <vector>

#include "../../include/khcore.h"
#include <nvtx3/nvToolsExt.h>

namespace kh {

constexpr int kRankBits = 5;
constexpr int kIdBits = 27;
constexpr uint32_t kIdMask = (1u << kIdBits) - 1u;
constexpr int kMaxM = 12000;
constexpr int kMaxH = 16;
constexpr int kPhaseStride = 32;  // stamp = round * kPhaseStride + phase
// Shared-memory visited bitmap limit per CTA (bytes); larger n uses global scratch.
constexpr int64_t kSmemBitmapMax = 100 * 1024;

// Dynamic shared memory the sliced 2-degree kernel may use per CTA (bytes).
constexpr int64_t kSmem2Max = 220 * 1024;
// Kernels whose dynamic shared memory depends on the graph set their
// maximum-dynamic-shared-memory attribute to the largest size they can ever
// use (a constant), not to the size of the launch at hand: contexts on other
// host threads (the server's slots) launch the same kernels concurrently, and
// a smaller value set by one between another's setting and its launch would
// make that launch fail.

// Error bits written by device-side checks.
constexpr int kErrQueue = 1;   // BFS queue overflow
constexpr int kErrProbe = 2;   // hash probe limit reached
constexpr int kErrList = 4;    // list larger than its slot
constexpr int kErrGraph = 8;   // CSR validation failure
constexpr int kErrLoop = 16;   // a work loop ran past its iteration bound
constexpr int64_t kProfSnapCap = 1 << 21;  // byte snapshots kept between two reads
constexpr int kOrderBinsMax = 48;  // log2 bins of a source's 2-hop work (order2)
constexpr int kSweepMinBin = 16;   // smallest work bin the tuner offers to the sweeps

// Kernel classes for the profiling counters (kh_prof_read kinds).
constexpr int kProfBfs = 0;       // exact h-degree / fixed-level count BFS
constexpr int kProfLevel1 = 1;    // level-1 lists
constexpr int kProfLevelU = 2;    // level >= 2 lists (hashed union)
constexpr int kProfFrontier = 3;  // removed-set ball hops, neighbour marking
constexpr int kProfPeel = 4;      // min, select, finish, advance
constexpr int kProfKinds = 5;

// Per-round counters: every launch inside a peeling round has its own slot,
// and the last block of the round's final kernel zeroes them all, so a round
// needs no memset nodes.
constexpr int kRcBfs = 0;          // refine BFS work counter
constexpr int kRcRefineWork = 1;   // refine last-level list work counter
constexpr int kRcRefineHeavy = 2;  // refine level-1 heavy count (h = 1)
constexpr int kRcLevelWork = 3;    // + i: refresh level i work counter, i = 1..kMaxH
constexpr int kRcLevelHeavy = 20;  // + i: refresh level i heavy count
constexpr int kRcW = 37;           // + i: work list of level i (0: exact affected nodes)
constexpr int kRcF = 54;           // + hop: frontier written by that hop (exact)
constexpr int kRcC = 71;           // + i: changed nodes at level i
constexpr int kRcLossWork = 88;    // exact refresh: loss-BFS work counter
constexpr int kRcLossCount = 89;   // exact refresh: nodes with a loss this round
constexpr int kRcSub = 90;         // + i: split-part items of level i (0: the refine)
constexpr int kRcCount = 107;

struct DevState {
    unsigned long long c;        // current core value (max of round minima)
    unsigned long long minval;   // min d over alive nodes in this round
    int round;                   // current round index
    int n_alive;                 // alive nodes at the start of the round
    int n_alive_next;            // alive nodes after this round's removal
    int nR;                      // |R| removed this round
    int nC[2];                   // changed-list sizes (standalone level passes)
    int work_ctr[4];             // dynamic scheduling counters
    unsigned long long updates;  // node recomputations
    unsigned long long bytes[kProfKinds];  // algorithmic bytes per kernel class
    int err;                     // kErr* bits
    int early;                   // exact early stop taken this round
    int nH;                      // heavy nodes deferred by the level-1 kernel
    int nQ;                      // refine list size (stale nodes due this round)
    unsigned long long minU;     // min of the upper bounds d over alive nodes
    int rc[kRcCount];            // per-round counters (kRc*)
    int done;                    // blocks of the round's final kernel that finished
    // peel work statistics: list recomputations and changes per level in the
    // rounds' refresh passes, refines stopped early
    unsigned long long lvl_work[kMaxH + 1];
    unsigned long long lvl_changed[kMaxH + 1];
    unsigned long long stopped;
    int tune_count;              // sample size of an autotuner measurement
    int nSub;                    // split-part items (standalone level passes)
};

struct Graph;

// The lazy refine decides whether d(v) <= T = max(c, U) and may stop once a
// partial value (a lower bound of d(v)) exceeds it.  It runs on until the
// partial value exceeds kStopSlack * T instead: the node's new lower bound then
// stays above the rising threshold for longer, so a node whose value is far
// above T is refined O(log) times instead of once per round (any lower bound
// above T gives the same removal decision).
constexpr unsigned long long kStopSlack = 2;
__host__ __device__ __forceinline__ unsigned long long stop_level(unsigned long long T) {
    return T >= (~0ull) / kStopSlack ? ~0ull : T * kStopSlack;
}

// A launch layout of the whole-graph exact 2-degree pass (kh_tune.cu):
// variant KH_VAR_CTA or KH_VAR_SLICED (KH_VAR_AUTO: not chosen yet), the
// sliced kernel's slice count and CTA size, and the sample time it took.
struct TuneChoice {
    int variant;
    int slices;
    int threads;
    double ms;
    int sweep_bin;  // sources with 2-hop work >= 2^sweep_bin go to the bit-parallel sweeps (0: none)
};

// NVTX range for profilers and tracers (a no-op unless a tool is attached).
struct NvtxRange {
    explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
    ~NvtxRange() { nvtxRangePop(); }
    NvtxRange(const NvtxRange&) = delete;
    NvtxRange& operator=(const NvtxRange&) = delete;
};

// ---- launchers (kh_exact.cu) -------------------------------------------------
void launch_ranks(const Graph& g, cudaStream_t s);
// each node's neighbour of largest degree (computed once per graph, before a peel)
int ensure_bestnb(Graph& g, cudaStream_t s);
void launch_validate(const Graph& g, int* d_err, cudaStream_t s);
// exact h-degrees of `count` nodes (worklist == nullptr: nodes 0..n-1) into deg32;
// when cnt != nullptr also the fixed-level counts for j in [jlo, jlo+nj).
// early_stop (the peel's lazy refine): a source whose partial ball already
// holds more than T = max(c, mu) of its graph stops and stays stale with that
// count as its lower bound.
// loss (the peel's exact refresh): sources are the removed nodes of the round;
// every alive node first reached at the source's last hop and not within h-1
// hops of the removed set (ball stamp) gains one in loss[] instead of a degree.
int launch_hdeg(Graph& g, const int* worklist, const int* d_count, int64_t count_static,
                int32_t* deg, int32_t* cnt, int jlo, int nj, cudaStream_t s,
                int* round_ctr = nullptr, bool early_stop = false, bool loss = false);
// d and (stale nodes) lb drop by loss[] for the listed nodes; loss[] is cleared
void launch_apply_loss(Graph& g, cudaStream_t s);
// one hop of the removed set's ball in the old graph (exact refresh)
void launch_ball_hop(Graph& g, int hop, cudaStream_t s);
// exact mode: mark the nodes of `list` (nullptr: all) stale and set their
// lower bound max(deg_X(v), max_w deg_X(w)) <= deg_h(v; X) for h >= 2
void launch_stale_exact(Graph& g, const int* list, const int* d_count, cudaStream_t s);

// ---- launchers (kh_hdeg2.cu) -------------------------------------------------
// exact 2-degrees (and fixed-level counts when cnt != nullptr) of every node
// with a sliced shared-memory visited set: `slices` node ranges, `threads` per
// CTA, sources from `order` (nsrc of them).  init: deg (and cnt) are set to
// their starting values first (every node); otherwise they must hold them.
int launch_hdeg2_slice(Graph& g, int32_t* deg, int32_t* cnt, int jlo, int nj, cudaStream_t s,
                       int slices, int threads, const int32_t* order, int64_t nsrc, bool init);
// the sources of the sliced kernel, longest 2-hop work first (cached per graph)
int ensure_order2(Graph& g, cudaStream_t s);
size_t hdeg2_smem(int64_t width);
// sources of order2 whose 2-hop work is too large for the warp-per-source
// kernel (they come first in order2), and that kernel for the rest
int64_t hdeg2_small_split(const Graph& g);
// sources of order2 whose 2-hop work is at least 2^bin (they come first)
int64_t hdeg2_sources_from_bin(const Graph& g, int bin);
// exact 2-degrees of `count` sources by bit-parallel sweeps of 128 sources
int run_sweeps(Graph& g, int32_t* deg, const int32_t* src, int64_t count, cudaStream_t s);
int launch_hdeg2_small(Graph& g, int32_t* deg, int32_t* cnt, int jlo, int nj, cudaStream_t s,
                       const int32_t* order, int64_t count);
// kh_tune.cu: the layout of the 2-degree pass for this graph (tuned once), and
// the whole-graph exact h-degree / fixed-level count pass through it
int choose_hdeg2(Graph& g, cudaStream_t s, TuneChoice* out);
int run_hdeg_full(Graph& g, int32_t* deg, int32_t* cnt, int jlo, int nj, cudaStream_t s);
int64_t hdeg2_width(int64_t n, int slices);
int hdeg2_min_slices(int64_t n);

// ---- launchers (kh_sampled.cu) -----------------------------------------------
// level i of the list recursion for `count` nodes (worklist == nullptr: all);
// track != 0 records nodes whose (|B|, k) changed into the changed list.
// round_mode 0: standalone (counters zeroed with memsets); 1: refresh of
// level `level` inside a round; 2: refine of the last level inside a round
// (per-round counters, no memsets).
int launch_level(Graph& g, int level, const int* worklist, const int* d_count,
                 int64_t count_static, int track, cudaStream_t s, int round_mode = 0,
                 int skip_last = -1);
// alive neighbours of the nodes in list1 and list2 (may be nullptr) join the
// work list listW (count *out_count), deduplicated by stamp phase
// A(list1) and the part of A(list2) whose level `phase` can have changed
// (rank filter on rho) join the work list.
void launch_mark_neighbours(Graph& g, const int* list1, const int* cnt1, const int* list2,
                            const int* cnt2, int phase, int* out_count, cudaStream_t s);
// sampled mode: mark the nodes of `list` (nullptr: all) stale at the last
// level with a lower bound of their estimate
void launch_stale_sampled(Graph& g, const int* list, const int* d_count, cudaStream_t s,
                          int only_h = 0);
// each node's last-level k and |B| into device arrays (either may be nullptr)
void launch_gather_last(Graph& g, uint8_t* lvl_out, int32_t* bs_out, cudaStream_t s);

// ---- launchers (kh_peel.cu) --------------------------------------------------
int run_core(Graph& g, bool sampled, void* out_core, int32_t* round_of_host, bool out_dev);
// EstDense (Alg. 7): replay of a removal order with eager refresh; per round,
// the sum of d over the alive set (host outputs)
int run_dense(Graph& g, bool sampled, const int32_t* round_of, int32_t rounds, uint64_t* sum,
              int64_t* size, int32_t* best);
int run_estimate_all(Graph& g);

}  // namespace kh

struct kh_ctx {
    int device;
    cudaStream_t stream;
    bool own_stream;
    int sm_count;
    char err[512];
    // fault injection on the host: the fail_alloc_at-th device allocation from
    // the arming call fails with KH_ENOMEM (0: off)
    int64_t fail_alloc_at;
    int64_t alloc_count;
};

namespace kh {
struct Graph {
    kh_ctx* ctx;
    int64_t n;
    int64_t nnz;
    int h;
    uint64_t seed;
    int64_t M;
    int64_t cap;            // list slot capacity (>= M, multiple of 4)
    bool ranks_valid;
    bool lists_valid;       // lists hold the full-graph recursion for (h, M, seed)
    int64_t *rowptr;
    int32_t *col;
    uint8_t *rank;
    uint8_t *alive;
    uint32_t *keys;
    uint8_t *ltop;          // highest rank of each stored list (levels 1..h-1)
    int64_t keys_levels;    // allocated levels in keys
    int32_t *lsz;
    uint8_t *lk;
    int64_t lvl_alloc;      // allocated levels in lsz/lk
    int32_t *d32;
    unsigned long long *d64;
    int32_t *core32;
    unsigned long long *core64;
    int32_t *round_of;
    int32_t *seen;
    int32_t *listR;
    int32_t *listA;
    int32_t *listB;
    int32_t *listW;
    int32_t *listC[2];
    DevState *state;
    // BFS scratch
    int32_t *queues;
    uint32_t *gbitmaps;
    int64_t scratch_ctas;
    int32_t *listH;         // heavy nodes deferred by the level-1 warp kernel
    // batches of graphs packed in one CSR (all nullptr for a single graph)
    int32_t *gid;           // graph of each node
    int64_t *vtx_off;       // first node of each graph, ngraphs + 1 entries
    uint8_t *hv;            // per-node h (nullptr: g.h for every node)
    int32_t *Mv;            // per-node M (nullptr: g.M for every node)
    int64_t ngraphs;
    int64_t max_gn;         // largest graph of the batch
    // per graph: c, round-start minimum over fresh nodes, refine threshold,
    // minimum of the values the round's refine completed
    unsigned long long *pc, *pmn, *pmu, *pmr;
    int32_t *pleft;         // per-graph alive count (batches)
    int hmin, hmax;         // range of h over the nodes
    std::vector<int64_t>* h_vtx_off;  // host copy of vtx_off (per-graph M)
    std::vector<int32_t>* h_hgraph;   // host copy of the per-graph h
    // lazy refinement of the last level: fresh[v] = d[v] is exact for the
    // current alive set; otherwise d[v] is an upper bound (d never grows as
    // nodes leave) and lb64[v] (exact mode) a lower bound
    uint8_t *fresh;
    // rho[v]: highest rank among the elements that left or entered v's list in
    // the level just recomputed (-1: none); filters the next level's refresh
    int8_t *rho;
    uint32_t *deadbm;       // bitmap of removed nodes (n bits), seeds BFS visited sets
    int32_t *degX;          // alive degree (exact mode)
    unsigned long long *lb64;
    // exact refresh: loss[v] = removed nodes within h hops of a node exactly
    // h hops from the removed set (zero between rounds), listed in listL
    int32_t *loss;
    int32_t *listL;
    // last peel statistics
    int64_t last_rounds;
    int64_t last_updates;
    int64_t last_lvl_work[kMaxH + 1];
    int64_t last_lvl_changed[kMaxH + 1];
    int64_t last_stopped;
    bool have_rounds;
    // EstDense replay: the removal order (round per node), per-round sums of d
    bool dense;
    // the pruned EstDense replay starts from the kept nodes only (keep[v] != 0)
    bool start_keep;
    int64_t start_alive;
    uint8_t* keep;
    int32_t* sched;
    unsigned long long* dsum;
    // profiling: CUDA events around every launch of a kernel class
    bool prof_on;
    std::vector<cudaEvent_t>* ev_pool;
    std::vector<int>* prof_kind;
    std::vector<cudaEvent_t>* prof_ev;  // pairs (start, stop)
    double prof_ms[kProfKinds];
    int64_t prof_launches[kProfKinds];
    std::vector<float>* prof_trace[kProfKinds];  // per-bracket ms, in launch order
    // per-bracket algorithmic bytes: the class counter copied before and after
    // each bracket into prof_snap (device; prof_snapi: first slot or -1)
    unsigned long long* prof_snap;
    int64_t prof_nsnap;
    std::vector<int64_t>* prof_snapi;
    std::vector<unsigned long long>* prof_btrace[kProfKinds];
    // cached CUDA graph of a batch of peeling rounds
    cudaGraphExec_t round_exec;
    int round_exec_key[10];
    int64_t round_exec_kernels;  // kernels in one replay of round_exec
    // kernels launched on behalf of this graph (graph replays count their nodes)
    int64_t launches;
    // level passes: part slots of split heavy nodes (part_cap slots of cap
    // keys; 0 when the graph has no node above the split degree)
    int64_t part_cap;
    int64_t part_cap_keys;  // cap the slots were sized for
    uint32_t *part_keys;
    int32_t *part_size;
    uint8_t *part_t;
    int32_t *part_done;
    int32_t *part_stop;
    unsigned long long *part_lb;
    int32_t *split_first;
    int32_t *sub_v;
    int32_t *sub_j;
    bool split_planned;     // part_cap computed for this graph
    // the peel's view of the graph (kh_peel.cu): rowptr/col above are switched
    // to a compacted CSR of the nodes alive at the last compaction, and the
    // whole-node scans run over vlist (vcount nodes; nullptr: all n); the
    // graph's own arrays are kept in orig_* and restored when the peel ends
    int64_t *orig_rowptr;
    int32_t *orig_col;
    const int32_t *vlist;
    int64_t vcount;
    int compact_mode;       // KH_VAR_AUTO, KH_COMPACT_OFF or KH_COMPACT_ALWAYS
    int levelu_mode;        // KH_VAR_AUTO (grouped), KH_LEVELU_STEPPED, _FREE or _GROUPED
    int levelu_div;         // grouped: coverage divisor (0: the default)
    int cp_cur;             // buffer set in use (0 or 1)
    int64_t *cp_row[2];
    int32_t *cp_col[2];
    int64_t cp_col_cap[2];
    int32_t *cp_list[2];
    int64_t *cp_tmp;        // counts and flags, 2 (n + 1)
    int64_t *cp_sums;       // scan tile totals
    // sliced 2-degree kernel: sources longest first (non-isolated nodes only)
    int32_t *order2;
    int64_t nsrc2;
    int64_t order2_hist[48];  // sources per log2 bin of 2-hop work (order2 is by descending bin)
    // bit-parallel 2-degree sweeps: source bits of the batch per node (128 per
    // node), node index among the rows longer than the sweep's head (or -1),
    // those rows' tail pieces and their partial ORs, per-bit ball counts
    uint32_t* sw_m1;
    uint32_t* sw_filter;      // one bit per 4 nodes: some of them has source bits in m1
    int32_t* sw_hpos;
    int32_t* sw_piece_h;
    int32_t* sw_piece_off;
    int32_t* sw_hnode;
    uint32_t* sw_bh;
    unsigned int* sw_cnt;
    int64_t sw_nheavy, sw_npieces;
    int sw_force;             // forced sweep threshold bin (0: tuner; -1: no sweeps)
    // each node's neighbour of largest degree (-1: none), for cheap stale bounds
    int32_t *bestnb;
    // the 2-degree pass layout: forced by kh_set_variant, or chosen by the tuner
    TuneChoice force_hdeg2;
    TuneChoice tuned_hdeg2;
};
}  // namespace kh

struct kh_graph {
    kh::Graph g;
};

namespace kh {
// Utility: set the context error text; returns code.
int set_error(kh_ctx* ctx, int code, const char* fmt, ...);
// Ensure the per-graph work arrays exist (idempotent).
int ensure_work(Graph& g);
int ensure_lists(Graph& g);
// part slots for the split heavy nodes of the level passes (kh_sampled.cu)
int ensure_split(Graph& g);
int ensure_bfs_scratch(Graph& g, int64_t ctas, bool bitmaps);
// A device allocation through the context's fault-injection counter.
int alloc_bytes(kh_ctx* ctx, void** p, size_t bytes, const char* what);
int check_cuda(kh_ctx* ctx, cudaError_t e, const char* what);
inline void count_launch(Graph& g, int64_t k) { g.launches += k; }
// Profiling brackets around a launch (no-ops unless profiling is enabled).
void prof_begin(Graph& g, int kind, cudaStream_t s);
void prof_end(Graph& g, int kind, cudaStream_t s);
}  // namespace kh

#define KH_CUDA_TRY(ctx, expr)                                  \
    do {                                                        \
        cudaError_t _e = (expr);                                \
        if (_e != cudaSuccess) return kh::check_cuda((ctx), _e, #expr); \
    } while (0)
