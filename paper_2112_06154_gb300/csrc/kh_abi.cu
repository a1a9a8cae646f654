// kh_abi.cu -- the extern "C" entry points declared in include/khcore.h:
// contexts, graph loading and validation, parameters, and the calls that run
// the exact and sampled paths.  Every device array of a graph is allocated
// here once and reused across calls.
#include <algorithm>
#include <cmath>
#include <vector>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "kh_internal.cuh"

namespace kh {

int set_error(kh_ctx* ctx, int code, const char* fmt, ...) {
    if (ctx) {
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(ctx->err, sizeof(ctx->err), fmt, ap);
        va_end(ap);
    }
    return code;
}

int check_cuda(kh_ctx* ctx, cudaError_t e, const char* what) {
    const int code = (e == cudaErrorMemoryAllocation) ? KH_ENOMEM : KH_ECUDA;
    cudaGetLastError();  // clear a sticky-free error so the context stays usable
    return set_error(ctx, code, "%s: %s", what, cudaGetErrorString(e));
}

template <typename T>
static int dalloc(kh_ctx* ctx, T** p, size_t count, const char* what) {
    if (*p) return KH_OK;
    if (ctx->fail_alloc_at > 0 && ++ctx->alloc_count == ctx->fail_alloc_at) {
        ctx->fail_alloc_at = 0;  // one failure per arming
        return set_error(ctx, KH_ENOMEM, "%s: injected allocation failure", what);
    }
    if (count == 0) count = 1;
    cudaError_t e = cudaMalloc((void**)p, count * sizeof(T));
    if (e != cudaSuccess) {
        *p = nullptr;
        return check_cuda(ctx, e, what);
    }
    return KH_OK;
}

int alloc_bytes(kh_ctx* ctx, void** p, size_t bytes, const char* what) {
    return dalloc(ctx, reinterpret_cast<uint8_t**>(p), bytes, what);
}

template <typename T>
static void dfree(T** p) {
    if (*p) cudaFree(*p);
    *p = nullptr;
}

int ensure_work(Graph& g) {
    const size_t n = (size_t)g.n;
    int rc;
    if ((rc = dalloc(g.ctx, &g.alive, n, "alive"))) return rc;
    if ((rc = dalloc(g.ctx, &g.d32, n, "d32"))) return rc;
    if ((rc = dalloc(g.ctx, &g.d64, n, "d64"))) return rc;
    if ((rc = dalloc(g.ctx, &g.core32, n, "core32"))) return rc;
    if ((rc = dalloc(g.ctx, &g.core64, n, "core64"))) return rc;
    if ((rc = dalloc(g.ctx, &g.round_of, n, "round_of"))) return rc;
    if ((rc = dalloc(g.ctx, &g.seen, n, "seen"))) return rc;
    if ((rc = dalloc(g.ctx, &g.listR, n, "listR"))) return rc;
    if ((rc = dalloc(g.ctx, &g.listA, n, "listA"))) return rc;
    if ((rc = dalloc(g.ctx, &g.listB, n, "listB"))) return rc;
    if ((rc = dalloc(g.ctx, &g.listW, n, "listW"))) return rc;
    if ((rc = dalloc(g.ctx, &g.listC[0], n, "listC0"))) return rc;
    if ((rc = dalloc(g.ctx, &g.listC[1], n, "listC1"))) return rc;
    if ((rc = dalloc(g.ctx, &g.listH, n, "listH"))) return rc;
    if ((rc = dalloc(g.ctx, &g.fresh, n, "fresh"))) return rc;
    if ((rc = dalloc(g.ctx, &g.deadbm, ((n + 127) / 128) * 4, "deadbm"))) return rc;
    if ((rc = dalloc(g.ctx, &g.degX, n, "degX"))) return rc;
    if ((rc = dalloc(g.ctx, &g.lb64, n, "lb64"))) return rc;
    if (!g.loss) {
        if ((rc = dalloc(g.ctx, &g.loss, n, "loss"))) return rc;
        KH_CUDA_TRY(g.ctx, cudaMemset(g.loss, 0, sizeof(int32_t) * (n ? n : 1)));
    }
    if ((rc = dalloc(g.ctx, &g.listL, n, "listL"))) return rc;
    if ((rc = ensure_bestnb(g, g.ctx->stream))) return rc;
    const size_t ng = (size_t)(g.gid ? g.ngraphs : 1);
    if ((rc = dalloc(g.ctx, &g.pc, ng, "per-graph c"))) return rc;
    if ((rc = dalloc(g.ctx, &g.pmn, ng, "per-graph minimum"))) return rc;
    if ((rc = dalloc(g.ctx, &g.pmr, ng, "per-graph refined minimum"))) return rc;
    if ((rc = dalloc(g.ctx, &g.pmu, ng, "per-graph threshold"))) return rc;
    if ((rc = dalloc(g.ctx, &g.pleft, ng, "per-graph alive count"))) return rc;
    return KH_OK;
}

static cudaEvent_t pool_event(Graph& g) {
    if (!g.ev_pool) g.ev_pool = new std::vector<cudaEvent_t>();
    if (!g.ev_pool->empty()) {
        cudaEvent_t e = g.ev_pool->back();
        g.ev_pool->pop_back();
        return e;
    }
    cudaEvent_t e = nullptr;
    if (cudaEventCreate(&e) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return e;
}

void prof_begin(Graph& g, int kind, cudaStream_t s) {
    if (!g.prof_on) return;
    if (g.prof_ev->size() % 2 == 1) {
        // a bracket left open (its launch returned an error before prof_end): drop it
        g.ev_pool->push_back(g.prof_ev->back());
        g.prof_ev->pop_back();
        g.prof_kind->pop_back();
        g.prof_snapi->pop_back();
    }
    cudaEvent_t e = pool_event(g);
    if (!e) return;
    int64_t si = -1;
    if (g.prof_snap && g.prof_nsnap + 2 <= kProfSnapCap &&
        cudaMemcpyAsync(g.prof_snap + g.prof_nsnap, &g.state->bytes[kind], sizeof(unsigned long long),
                        cudaMemcpyDeviceToDevice, s) == cudaSuccess) {
        si = g.prof_nsnap;
        g.prof_nsnap += 2;
    }
    cudaEventRecord(e, s);
    g.prof_kind->push_back(kind);
    g.prof_ev->push_back(e);
    g.prof_snapi->push_back(si);
}

void prof_end(Graph& g, int kind, cudaStream_t s) {
    if (!g.prof_on) return;
    if (g.prof_ev->size() != 2 * g.prof_kind->size() - 1) return;  // its begin was not recorded
    cudaEvent_t e = pool_event(g);
    if (!e) {
        // drop the open bracket
        g.ev_pool->push_back(g.prof_ev->back());
        g.prof_ev->pop_back();
        g.prof_kind->pop_back();
        g.prof_snapi->pop_back();
        return;
    }
    cudaEventRecord(e, s);
    g.prof_ev->push_back(e);
    const int64_t si = g.prof_snapi->back();
    if (si >= 0 && cudaMemcpyAsync(g.prof_snap + si + 1, &g.state->bytes[kind], sizeof(unsigned long long),
                                   cudaMemcpyDeviceToDevice, s) != cudaSuccess)
        g.prof_snapi->back() = -1;
}

// Fold recorded event pairs into the per-kind totals (synchronizes the stream).
static int prof_collect(Graph& g) {
    if (!g.prof_ev || g.prof_ev->empty()) return KH_OK;
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(g.ctx->stream));
    const size_t pairs = g.prof_kind->size();
    std::vector<unsigned long long> snap((size_t)g.prof_nsnap);
    if (g.prof_nsnap > 0)
        KH_CUDA_TRY(g.ctx, cudaMemcpy(snap.data(), g.prof_snap, sizeof(unsigned long long) * snap.size(),
                                      cudaMemcpyDeviceToHost));
    for (size_t i = 0; i < pairs && 2 * i + 1 < g.prof_ev->size(); ++i) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, (*g.prof_ev)[2 * i], (*g.prof_ev)[2 * i + 1]) == cudaSuccess) {
            const int k = (*g.prof_kind)[i];
            g.prof_ms[k] += ms;
            g.prof_launches[k] += 1;
            if (!g.prof_trace[k]) g.prof_trace[k] = new std::vector<float>();
            g.prof_trace[k]->push_back(ms);
            // bytes of the bracket (~0: not recorded)
            const int64_t si = (*g.prof_snapi)[i];
            if (!g.prof_btrace[k]) g.prof_btrace[k] = new std::vector<unsigned long long>();
            g.prof_btrace[k]->push_back(si >= 0 ? snap[(size_t)si + 1] - snap[(size_t)si] : ~0ull);
        } else {
            cudaGetLastError();
        }
    }
    for (cudaEvent_t e : *g.prof_ev) g.ev_pool->push_back(e);
    g.prof_ev->clear();
    g.prof_kind->clear();
    g.prof_snapi->clear();
    g.prof_nsnap = 0;
    return KH_OK;
}

int ensure_lists(Graph& g) {
    // lists for levels 1..hmax-1, sizes/levels for 1..hmax
    const int64_t need_keys = (int64_t)(g.hmax - 1) * g.n * g.cap;
    if (g.keys && g.keys_levels * g.n * g.cap < need_keys) {
        dfree(&g.keys);
        dfree(&g.ltop);
    }
    if (g.lsz && g.lvl_alloc < g.hmax) {
        dfree(&g.lsz);
        dfree(&g.lk);
    }
    int rc;
    if (need_keys > 0) {
        if ((rc = dalloc(g.ctx, &g.keys, (size_t)need_keys, "sample lists"))) return rc;
        if ((rc = dalloc(g.ctx, &g.ltop, (size_t)(g.hmax - 1) * (size_t)g.n, "list top ranks")))
            return rc;
        g.keys_levels = g.hmax - 1;
    }
    if (!g.lsz) g.lvl_alloc = g.hmax;
    if ((rc = dalloc(g.ctx, &g.lsz, (size_t)g.lvl_alloc * g.n, "list sizes"))) return rc;
    if ((rc = dalloc(g.ctx, &g.lk, (size_t)g.lvl_alloc * g.n, "list levels"))) return rc;
    if ((rc = dalloc(g.ctx, &g.rho, (size_t)g.n, "list change ranks"))) return rc;
    if ((rc = ensure_split(g))) return rc;
    if (!g.ranks_valid) {
        launch_ranks(g, g.ctx->stream);
        g.ranks_valid = true;
    }
    return KH_OK;
}

int ensure_bfs_scratch(Graph& g, int64_t ctas, bool bitmaps) {
    if (g.queues && g.scratch_ctas >= ctas && (!bitmaps || g.gbitmaps)) return KH_OK;
    // enlarging: wait for in-flight users of the old scratch first
    if (g.queues || g.gbitmaps) {
        cudaError_t e = cudaStreamSynchronize(g.ctx->stream);
        if (e != cudaSuccess) return check_cuda(g.ctx, e, "sync before scratch resize");
    }
    dfree(&g.queues);
    dfree(&g.gbitmaps);
    int rc;
    // a batch's BFS stays inside one graph: queues and bitmaps span its largest graph
    const int64_t domain = g.gid ? g.max_gn : g.n;
    if ((rc = dalloc(g.ctx, &g.queues, (size_t)ctas * (size_t)domain, "BFS queues"))) return rc;
    if (bitmaps) {
        const size_t words = (size_t)((domain + 31) / 32);
        if ((rc = dalloc(g.ctx, &g.gbitmaps, (size_t)ctas * words, "BFS bitmaps"))) return rc;
    }
    g.scratch_ctas = ctas;
    return KH_OK;
}

static int64_t budget_M(int64_t n, double eps, double delta) {
    // Eq. (buffer): M = 1 + 4(2 + eps)/eps^2 (C + log 8), C = log(2n/delta)
    const double C = std::log(2.0 * (double)n / delta);
    const double m = std::floor(1.0 + 4.0 * (2.0 + eps) / (eps * eps) * (C + std::log(8.0)));
    // a tiny eps overflows the double range: saturate (the caller's range check rejects it)
    if (!(m < 9.0e18)) return INT64_MAX;
    return (int64_t)m;
}

static void free_graph_arrays(Graph& g) {
    dfree(&g.rowptr);
    dfree(&g.col);
    dfree(&g.rank);
    dfree(&g.alive);
    dfree(&g.keys);
    dfree(&g.ltop);
    dfree(&g.lsz);
    dfree(&g.lk);
    dfree(&g.d32);
    dfree(&g.d64);
    dfree(&g.core32);
    dfree(&g.core64);
    dfree(&g.round_of);
    dfree(&g.seen);
    dfree(&g.listR);
    dfree(&g.listA);
    dfree(&g.listB);
    dfree(&g.listW);
    dfree(&g.listC[0]);
    dfree(&g.listC[1]);
    dfree(&g.state);
    dfree(&g.queues);
    dfree(&g.gbitmaps);
    dfree(&g.listH);
    dfree(&g.fresh);
    dfree(&g.rho);
    dfree(&g.loss);
    dfree(&g.listL);
    dfree(&g.sched);
    dfree(&g.keep);
    dfree(&g.dsum);
    dfree(&g.deadbm);
    dfree(&g.gid);
    dfree(&g.vtx_off);
    dfree(&g.pc);
    dfree(&g.pmn);
    dfree(&g.pmr);
    dfree(&g.pmu);
    dfree(&g.pleft);
    dfree(&g.hv);
    dfree(&g.Mv);
    delete g.h_vtx_off;
    g.h_vtx_off = nullptr;
    delete g.h_hgraph;
    g.h_hgraph = nullptr;
    dfree(&g.degX);
    dfree(&g.lb64);
    dfree(&g.order2);
    dfree(&g.sw_m1);
    dfree(&g.sw_filter);
    dfree(&g.sw_hpos);
    dfree(&g.sw_piece_h);
    dfree(&g.sw_piece_off);
    dfree(&g.sw_hnode);
    dfree(&g.sw_bh);
    dfree(&g.sw_cnt);
    dfree(&g.bestnb);
    for (int b = 0; b < 2; ++b) {
        dfree(&g.cp_row[b]);
        dfree(&g.cp_col[b]);
        dfree(&g.cp_list[b]);
        g.cp_col_cap[b] = 0;
    }
    dfree(&g.cp_tmp);
    dfree(&g.cp_sums);
    dfree(&g.part_keys);
    dfree(&g.part_size);
    dfree(&g.part_t);
    dfree(&g.part_done);
    dfree(&g.part_stop);
    dfree(&g.part_lb);
    dfree(&g.split_first);
    dfree(&g.sub_v);
    dfree(&g.sub_j);
    if (g.round_exec) cudaGraphExecDestroy(g.round_exec);
    g.round_exec = nullptr;
    if (g.ev_pool) {
        for (cudaEvent_t e : *g.ev_pool) cudaEventDestroy(e);
        delete g.ev_pool;
        g.ev_pool = nullptr;
    }
    if (g.prof_ev) {
        for (cudaEvent_t e : *g.prof_ev) cudaEventDestroy(e);
        delete g.prof_ev;
        g.prof_ev = nullptr;
    }
    delete g.prof_kind;
    g.prof_kind = nullptr;
    delete g.prof_snapi;
    g.prof_snapi = nullptr;
    if (g.prof_snap) cudaFree(g.prof_snap);
    g.prof_snap = nullptr;
    for (int k = 0; k < kProfKinds; ++k) {
        delete g.prof_trace[k];
        g.prof_trace[k] = nullptr;
        delete g.prof_btrace[k];
        g.prof_btrace[k] = nullptr;
    }
}

static int set_M(Graph& g, int64_t M) {
    if (M < 1 || M > kMaxM)
        return set_error(g.ctx, KH_EINVAL, "M = %lld outside [1, %d]", (long long)M, kMaxM);
    if (M != g.M) {
        g.M = M;
        const int64_t cap = (M + 3) & ~(int64_t)3;
        if (cap > g.cap) dfree(&g.keys);
        if (cap > g.cap) g.cap = cap;
    }
    return KH_OK;
}

static int copy_out(Graph& g, void* dst, const void* src, size_t bytes, uint32_t flags) {
    cudaStream_t s = g.ctx->stream;
    if (bytes == 0) return KH_OK;
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(dst, src, bytes,
                                       (flags & KH_DEVICE_PTR) ? cudaMemcpyDeviceToDevice
                                                               : cudaMemcpyDeviceToHost, s));
    if (!(flags & KH_DEVICE_PTR)) KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
    return KH_OK;
}

static int finish_check(Graph& g) {
    int err = 0;
    cudaStream_t s = g.ctx->stream;
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(&err, &g.state->err, sizeof(int), cudaMemcpyDeviceToHost, s));
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
    if (err) return set_error(g.ctx, KH_EINTERNAL, "device check failed (flags 0x%x)", err);
    return KH_OK;
}

}  // namespace kh

using kh::Graph;

extern "C" {

int kh_ctx_create(kh_ctx** out, int device, void* cuda_stream) {
    if (!out) return KH_EINVAL;
    *out = nullptr;
    kh_ctx* c = (kh_ctx*)calloc(1, sizeof(kh_ctx));
    if (!c) return KH_ENOMEM;
    c->device = device;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->sm_count, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) {
        if (cuda_stream) {
            c->stream = (cudaStream_t)cuda_stream;
            c->own_stream = false;
        } else {
            e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
            c->own_stream = true;
        }
    }
    if (e != cudaSuccess) {
        free(c);
        cudaGetLastError();
        return e == cudaErrorMemoryAllocation ? KH_ENOMEM : KH_ECUDA;
    }
    *out = c;
    return KH_OK;
}

int kh_ctx_destroy(kh_ctx* ctx) {
    if (!ctx) return KH_EINVAL;
    cudaSetDevice(ctx->device);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
    free(ctx);
    return KH_OK;
}

int kh_debug_fail_alloc(kh_ctx* ctx, int64_t k) {
    if (!ctx || k < 0) return KH_EINVAL;
    ctx->fail_alloc_at = k;
    ctx->alloc_count = 0;
    return KH_OK;
}

const char* kh_last_error(kh_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->err;
}

namespace kh {
// Shared by kh_graph_load_csr and kh_graph_load_batch: copy and validate the
// CSR; host_gid (batches) makes the validation reject edges between graphs.
static int load_graph(kh_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col,
                      uint32_t flags, const int32_t* host_gid, kh_graph** out) {
    if (!ctx || !out) return KH_EINVAL;
    *out = nullptr;
    if (n < 0 || (n > 0 && (!rowptr))) return kh::set_error(ctx, KH_EINVAL, "bad n or rowptr");
    if (n > (int64_t)kh::kIdMask)
        return kh::set_error(ctx, KH_EGRAPH, "n = %lld exceeds 2^27 - 1 node ids", (long long)n);
    cudaError_t ce = cudaSetDevice(ctx->device);
    if (ce != cudaSuccess) return kh::check_cuda(ctx, ce, "cudaSetDevice");
    const bool dev = (flags & KH_DEVICE_PTR) != 0;
    cudaStream_t s = ctx->stream;
    int64_t ends[2] = {0, 0};
    if (n > 0) {
        if (dev) {
            ce = cudaMemcpyAsync(&ends[0], rowptr, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess)
                ce = cudaMemcpyAsync(&ends[1], rowptr + n, sizeof(int64_t), cudaMemcpyDeviceToHost, s);
            if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
            if (ce != cudaSuccess) return kh::check_cuda(ctx, ce, "read rowptr ends");
        } else {
            ends[0] = rowptr[0];
            ends[1] = rowptr[n];
        }
    }
    const int64_t nnz = ends[1];
    if (ends[0] != 0 || nnz < 0 || nnz > ((int64_t)1 << 40))
        return kh::set_error(ctx, KH_EGRAPH, "rowptr must start at 0 and end at nnz >= 0");
    if (nnz > 0 && !col) return kh::set_error(ctx, KH_EINVAL, "null col");
    kh_graph* G = (kh_graph*)calloc(1, sizeof(kh_graph));
    if (!G) return KH_ENOMEM;
    Graph& g = G->g;
    g.ctx = ctx;
    g.n = n;
    g.nnz = nnz;
    g.h = 2;
    g.hmin = g.hmax = 2;
    g.seed = 1;
    g.M = 0;
    g.cap = 0;
    int rc = KH_OK;
    if ((rc = kh::dalloc(ctx, &g.rowptr, (size_t)n + 1, "rowptr")) ||
        (rc = kh::dalloc(ctx, &g.col, (size_t)nnz, "col")) ||
        (rc = kh::dalloc(ctx, &g.rank, (size_t)n, "rank")) ||
        (rc = kh::dalloc(ctx, &g.state, 1, "state")) ||
        (host_gid && (rc = kh::dalloc(ctx, &g.gid, (size_t)n, "graph ids")))) {
        kh::free_graph_arrays(g);
        free(G);
        return rc;
    }
    const cudaMemcpyKind kind = dev ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    ce = cudaMemcpyAsync(g.rowptr, rowptr, sizeof(int64_t) * (size_t)(n + 1), kind, s);
    if (ce == cudaSuccess && nnz > 0)
        ce = cudaMemcpyAsync(g.col, col, sizeof(int32_t) * (size_t)nnz, kind, s);
    if (ce == cudaSuccess) ce = cudaMemsetAsync(g.state, 0, sizeof(kh::DevState), s);
    if (ce == cudaSuccess && host_gid && n > 0)
        ce = cudaMemcpyAsync(g.gid, host_gid, sizeof(int32_t) * (size_t)n, cudaMemcpyHostToDevice, s);
    if (ce != cudaSuccess) {
        rc = kh::check_cuda(ctx, ce, "copy CSR");
        kh::free_graph_arrays(g);
        free(G);
        return rc;
    }
    // row offsets must be nondecreasing: checked by the validation kernel
    // (a decreasing pair is flagged there), together with sorted rows,
    // in-range ids, no self-loops and symmetry
    kh::launch_validate(g, &g.state->err, s);
    int err = 0;
    ce = cudaMemcpyAsync(&err, &g.state->err, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (ce == cudaSuccess) ce = cudaStreamSynchronize(s);
    if (ce != cudaSuccess) {
        rc = kh::check_cuda(ctx, ce, "validate CSR");
        kh::free_graph_arrays(g);
        free(G);
        return rc;
    }
    if (err) {
        kh::free_graph_arrays(g);
        free(G);
        return kh::set_error(ctx, KH_EGRAPH,
                             host_gid ? "batch is not a simple symmetric CSR with sorted rows and "
                                        "no edge between graphs"
                                      : "graph is not a simple symmetric CSR with sorted rows");
    }
    rc = kh::set_M(g, kh::budget_M(n > 0 ? n : 1, 0.5, 0.05));
    if (rc) {
        kh::free_graph_arrays(g);
        free(G);
        return rc;
    }
    *out = G;
    return KH_OK;
}
}  // namespace kh

int kh_graph_load_csr(kh_ctx* ctx, int64_t n, const int64_t* rowptr, const int32_t* col,
                      uint32_t flags, kh_graph** out) {
    kh::NvtxRange nvtx_range("kh_graph_load_csr");
    return kh::load_graph(ctx, n, rowptr, col, flags, nullptr, out);
}

int kh_graph_load_batch(kh_ctx* ctx, int32_t ngraphs, const int64_t* vtx_off, const int64_t* rowptr,
                        const int32_t* col, const int32_t* h_per_graph, uint32_t flags,
                        kh_graph** out) {
    kh::NvtxRange nvtx_range("kh_graph_load_batch");
    if (!ctx || !out || ngraphs < 1 || !vtx_off) return KH_EINVAL;
    *out = nullptr;
    if (vtx_off[0] != 0) return kh::set_error(ctx, KH_EINVAL, "vtx_off[0] must be 0");
    int64_t max_gn = 0;
    int hmin = kh::kMaxH, hmax = 1;
    for (int32_t q = 0; q < ngraphs; ++q) {
        const int64_t gn = vtx_off[q + 1] - vtx_off[q];
        if (gn < 0) return kh::set_error(ctx, KH_EINVAL, "vtx_off must be nondecreasing");
        if (gn > max_gn) max_gn = gn;
        const int hq = h_per_graph ? h_per_graph[q] : 2;
        if (hq < 1 || hq > kh::kMaxH)
            return kh::set_error(ctx, KH_EINVAL, "graph %d: h = %d outside [1, %d]", q, hq, kh::kMaxH);
        hmin = std::min(hmin, hq);
        hmax = std::max(hmax, hq);
    }
    const int64_t n = vtx_off[ngraphs];
    if (n > (int64_t)kh::kIdMask)
        return kh::set_error(ctx, KH_EGRAPH, "n = %lld exceeds 2^27 - 1 node ids", (long long)n);
    std::vector<int32_t> gid((size_t)n);
    std::vector<uint8_t> hv((size_t)n);
    for (int32_t q = 0; q < ngraphs; ++q)
        for (int64_t v = vtx_off[q]; v < vtx_off[q + 1]; ++v) {
            gid[(size_t)v] = q;
            hv[(size_t)v] = (uint8_t)(h_per_graph ? h_per_graph[q] : 2);
        }
    kh_graph* G = nullptr;
    int rc = kh::load_graph(ctx, n, rowptr, col, flags, gid.data(), &G);
    if (rc) return rc;
    Graph& g = G->g;
    g.ngraphs = ngraphs;
    g.max_gn = max_gn;
    g.h = hmax;
    g.hmin = hmin;
    g.hmax = hmax;
    g.h_vtx_off = new std::vector<int64_t>(vtx_off, vtx_off + ngraphs + 1);
    if ((rc = kh::dalloc(ctx, &g.vtx_off, (size_t)ngraphs + 1, "vtx_off")) ||
        (rc = kh::dalloc(ctx, &g.hv, (size_t)n, "per-node h"))) {
        kh_graph_free(G);
        return rc;
    }
    cudaError_t ce = cudaMemcpy(g.vtx_off, vtx_off, sizeof(int64_t) * (size_t)(ngraphs + 1),
                                cudaMemcpyHostToDevice);
    if (ce == cudaSuccess && n > 0) ce = cudaMemcpy(g.hv, hv.data(), (size_t)n, cudaMemcpyHostToDevice);
    if (ce != cudaSuccess) {
        rc = kh::check_cuda(ctx, ce, "copy batch tables");
        kh_graph_free(G);
        return rc;
    }
    rc = kh_set_sampling(G, 1, 0, 0.5, 0.05);  // per-graph M from each graph's n
    if (rc) {
        kh_graph_free(G);
        return rc;
    }
    *out = G;
    return KH_OK;
}

int kh_graph_free(kh_graph* G) {
    if (!G) return KH_EINVAL;
    cudaSetDevice(G->g.ctx->device);
    cudaStreamSynchronize(G->g.ctx->stream);
    kh::free_graph_arrays(G->g);
    free(G);
    return KH_OK;
}

int kh_footprint(int64_t n, int64_t nnz, int32_t h, int64_t M_or_0, double eps, double delta,
                 int64_t* M_out, int64_t* bytes) {
    if (n < 0 || nnz < 0 || h < 1 || h > kh::kMaxH || M_or_0 < 0) return KH_EINVAL;
    int64_t M = M_or_0;
    if (M == 0) {
        if (!(eps > 0.0) || !(delta > 0.0) || !(delta < 1.0) || !std::isfinite(eps)) return KH_EINVAL;
        M = kh::budget_M(n > 0 ? n : 1, eps, delta);
    }
    if (M < 1 || M > kh::kMaxM) return KH_EINVAL;
    if (M_out) *M_out = M;
    if (!bytes) return KH_OK;
    const int64_t cap = (M + 3) & ~(int64_t)3;
    // the graph: CSR, ranks, state
    int64_t b = 8 * (n + 1) + 4 * nnz + n + (int64_t)sizeof(kh::DevState);
    // per-node work arrays of ensure_work (alive, d, core, rounds, stamps, seven
    // node lists, fresh, degrees, bounds, loss and its list, best neighbours,
    // removed-node bitmap)
    b += n * (1 + 4 + 8 + 4 + 8 + 4 + 4 + 7 * 4 + 1 + 4 + 8 + 4 + 4 + 4) + n / 8 + 64;
    // level lists 1..h-1 (cap keys per node and level), sizes and levels of
    // 1..h, change ranks, top ranks
    b += (int64_t)(h - 1) * n * cap * 4 + (int64_t)h * n * 5 + n + (int64_t)(h - 1) * n;
    // split parts of heavy nodes: at most nnz / 1365 slots (ceil(deg/2048) <=
    // deg/1365 for deg > 4096), each cap keys plus counters
    const int64_t parts = nnz / 1365;
    b += parts * (cap * 4 + 29) + 4 * n;
    // the peel's compaction buffers (graphs of at least 65536 nodes)
    if (n >= 65536) b += 2 * 8 * (n + 1) + 2 * 4 * nnz + 2 * 4 * (n + 1) + 16 * (n + 1) + 64 * 1024;
    *bytes = b + (1 << 20);
    return KH_OK;
}

int kh_graph_n(kh_graph* G, int64_t* n) {
    if (!G || !n) return KH_EINVAL;
    *n = G->g.n;
    return KH_OK;
}

int kh_set_h(kh_graph* G, int32_t h) {
    if (!G) return KH_EINVAL;
    if (h < 1 || h > kh::kMaxH) return kh::set_error(G->g.ctx, KH_EINVAL, "h = %d outside [1, %d]", h, kh::kMaxH);
    Graph& g = G->g;
    cudaSetDevice(g.ctx->device);
    if (g.hv) {  // a batch: one h for every graph from now on
        cudaStreamSynchronize(g.ctx->stream);
        kh::dfree(&g.hv);
    }
    g.h = g.hmin = g.hmax = h;
    return KH_OK;
}

int kh_set_sampling(kh_graph* G, uint64_t seed, int64_t M_or_0, double eps, double delta) {
    if (!G) return KH_EINVAL;
    Graph& g = G->g;
    int64_t M = M_or_0;
    if (M_or_0 < 0) return kh::set_error(g.ctx, KH_EINVAL, "M must be >= 0");
    if (M_or_0 == 0) {
        if (!(eps > 0.0) || !(delta > 0.0) || !(delta < 1.0) || !std::isfinite(eps))
            return kh::set_error(g.ctx, KH_EINVAL, "need eps > 0 and 0 < delta < 1");
        M = kh::budget_M(g.n > 0 ? g.n : 1, eps, delta);
    }
    cudaSetDevice(g.ctx->device);
    if (g.h_vtx_off) {
        // a batch: M of Eq. (buffer) from each graph's own n, or one M for all
        cudaStreamSynchronize(g.ctx->stream);
        kh::dfree(&g.Mv);
        if (M_or_0 == 0) {
            const std::vector<int64_t>& off = *g.h_vtx_off;
            std::vector<int32_t> mv((size_t)g.n);
            int64_t mmax = 1;
            for (size_t q = 0; q + 1 < off.size(); ++q) {
                const int64_t gn = off[q + 1] - off[q];
                const int64_t Mg = kh::budget_M(gn > 0 ? gn : 1, eps, delta);
                if (Mg < 1 || Mg > kh::kMaxM)
                    return kh::set_error(g.ctx, KH_EINVAL, "graph %zu: M = %lld outside [1, %d]", q,
                                         (long long)Mg, kh::kMaxM);
                if (Mg > mmax) mmax = Mg;
                for (int64_t v = off[q]; v < off[q + 1]; ++v) mv[(size_t)v] = (int32_t)Mg;
            }
            int rc0 = kh::dalloc(g.ctx, &g.Mv, (size_t)g.n, "per-node M");
            if (rc0) return rc0;
            if (g.n > 0)
                KH_CUDA_TRY(g.ctx, cudaMemcpy(g.Mv, mv.data(), sizeof(int32_t) * (size_t)g.n,
                                              cudaMemcpyHostToDevice));
            M = mmax;  // sizes the list slots and hash tables
        }
    }
    int rc = kh::set_M(g, M);
    if (rc) return rc;
    if (seed != g.seed) {
        g.seed = seed;
        g.ranks_valid = false;
    }
    return KH_OK;
}

int kh_get_M(kh_graph* G, int64_t* M) {
    if (!G || !M) return KH_EINVAL;
    *M = G->g.M;
    return KH_OK;
}

int kh_ranks(kh_graph* G, uint8_t* r, uint32_t flags) {
    if (!G || (!r && G->g.n > 0)) return KH_EINVAL;
    Graph& g = G->g;
    cudaSetDevice(g.ctx->device);
    if (!g.ranks_valid) {
        kh::launch_ranks(g, g.ctx->stream);
        g.ranks_valid = true;
    }
    KH_CUDA_TRY(g.ctx, cudaGetLastError());
    return kh::copy_out(g, r, g.rank, (size_t)g.n, flags);
}

int kh_hdegree_exact(kh_graph* G, int32_t* deg, uint32_t flags) {
    kh::NvtxRange nvtx_range("kh_hdegree_exact");
    if (!G || (!deg && G->g.n > 0)) return KH_EINVAL;
    Graph& g = G->g;
    cudaSetDevice(g.ctx->device);
    cudaStream_t s = g.ctx->stream;
    int rc = kh::ensure_work(g);
    if (rc) return rc;
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.alive, 1, (size_t)g.n, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.deadbm, 0, ((size_t)(g.n + 127) / 128) * 16, s));
    rc = kh::run_hdeg_full(g, g.d32, nullptr, 0, 0, s);
    if (rc) return rc;
    KH_CUDA_TRY(g.ctx, cudaGetLastError());
    rc = kh::copy_out(g, deg, g.d32, sizeof(int32_t) * (size_t)g.n, flags);
    if (rc) return rc;
    return (flags & KH_DEVICE_PTR) ? KH_OK : kh::finish_check(g);
}

int kh_sampled_counts(kh_graph* G, int32_t j_lo, int32_t j_hi, int32_t* cnt, uint32_t flags) {
    kh::NvtxRange nvtx_range("kh_sampled_counts");
    if (!G || (!cnt && G->g.n > 0)) return KH_EINVAL;
    Graph& g = G->g;
    if (j_lo < 0 || j_hi > 31 || j_lo > j_hi)
        return kh::set_error(g.ctx, KH_EINVAL, "need 0 <= j_lo <= j_hi <= 31");
    cudaSetDevice(g.ctx->device);
    cudaStream_t s = g.ctx->stream;
    int rc = kh::ensure_work(g);
    if (rc) return rc;
    if (!g.ranks_valid) {
        kh::launch_ranks(g, s);
        g.ranks_valid = true;
    }
    const int nj = j_hi - j_lo + 1;
    int32_t* dcnt = nullptr;
    if (flags & KH_DEVICE_PTR) {
        dcnt = cnt;
    } else if (g.n > 0) {
        KH_CUDA_TRY(g.ctx, cudaMallocAsync((void**)&dcnt, sizeof(int32_t) * (size_t)g.n * nj, s));
    }
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.alive, 1, (size_t)g.n, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.deadbm, 0, ((size_t)(g.n + 127) / 128) * 16, s));
    rc = kh::run_hdeg_full(g, g.d32, dcnt, j_lo, nj, s);
    if (rc == KH_OK && !(flags & KH_DEVICE_PTR) && g.n > 0) {
        rc = kh::copy_out(g, cnt, dcnt, sizeof(int32_t) * (size_t)g.n * nj, 0);
    }
    if (dcnt && !(flags & KH_DEVICE_PTR)) cudaFreeAsync(dcnt, s);
    if (rc) return rc;
    KH_CUDA_TRY(g.ctx, cudaGetLastError());
    return (flags & KH_DEVICE_PTR) ? KH_OK : kh::finish_check(g);
}

int kh_estimate(kh_graph* G, uint64_t* est, uint8_t* level, int32_t* bsize, uint32_t flags) {
    kh::NvtxRange nvtx_range("kh_estimate");
    if (!G || (!est && G->g.n > 0)) return KH_EINVAL;
    Graph& g = G->g;
    cudaSetDevice(g.ctx->device);
    int rc = kh::run_estimate_all(g);
    if (rc) return rc;
    // each node's last level (h of its graph) into scratch, then out
    uint8_t* lvl_tmp = reinterpret_cast<uint8_t*>(g.listB);
    int32_t* bs_tmp = g.listA;
    kh::launch_gather_last(g, lvl_tmp, bs_tmp, g.ctx->stream);
    KH_CUDA_TRY(g.ctx, cudaGetLastError());
    rc = kh::copy_out(g, est, g.d64, sizeof(uint64_t) * (size_t)g.n, flags);
    if (!rc && level) rc = kh::copy_out(g, level, lvl_tmp, (size_t)g.n, flags);
    if (!rc && bsize) rc = kh::copy_out(g, bsize, bs_tmp, sizeof(int32_t) * (size_t)g.n, flags);
    return rc;
}

int kh_core_exact(kh_graph* G, int32_t* core, uint32_t flags) {
    kh::NvtxRange nvtx_range("kh_core_exact");
    if (!G || (!core && G->g.n > 0)) return KH_EINVAL;
    cudaSetDevice(G->g.ctx->device);
    return kh::run_core(G->g, false, core, nullptr, (flags & KH_DEVICE_PTR) != 0);
}

int kh_core_sampled(kh_graph* G, uint64_t* core, uint32_t flags) {
    kh::NvtxRange nvtx_range("kh_core_sampled");
    if (!G || (!core && G->g.n > 0)) return KH_EINVAL;
    cudaSetDevice(G->g.ctx->device);
    return kh::run_core(G->g, true, core, nullptr, (flags & KH_DEVICE_PTR) != 0);
}

int kh_peel_info(kh_graph* G, int32_t* round_of, int64_t* rounds, int64_t* updates) {
    if (!G) return KH_EINVAL;
    Graph& g = G->g;
    if (!g.have_rounds) return kh::set_error(g.ctx, KH_EINVAL, "no peeling has run on this graph");
    if (rounds) *rounds = g.last_rounds;
    if (updates) *updates = g.last_updates;
    if (round_of && g.n > 0) {
        cudaSetDevice(g.ctx->device);
        return kh::copy_out(g, round_of, g.round_of, sizeof(int32_t) * (size_t)g.n, 0);
    }
    return KH_OK;
}

namespace kh {
// EstDense replay of a removal order (Alg. 7); keep (host, may be nullptr):
// nodes outside it are removed before the replay starts (the pruned variant).
static int dense_common(Graph& g, int32_t exact, const int32_t* round_of, int32_t rounds,
                        const uint8_t* keep, uint64_t* sum, int64_t* size, int32_t* best) {
    if (g.gid) return set_error(g.ctx, KH_EINVAL, "kh_dense takes a single graph, not a batch");
    if (rounds < 1 || (int64_t)rounds > g.n + 1)
        return set_error(g.ctx, KH_EINVAL, "rounds must be in [1, n + 1]");
    std::vector<int64_t> left((size_t)rounds + 1, 0);
    for (int64_t v = 0; v < g.n; ++v) {
        const int32_t r = round_of[v];
        if (r < 0 || r >= rounds) return set_error(g.ctx, KH_EINVAL, "round_of[%lld] = %d outside [0, rounds)", (long long)v, r);
        if (!keep || keep[v]) left[(size_t)r] += 1;
    }
    for (int32_t q = rounds - 1; q >= 0; --q) left[(size_t)q] += left[(size_t)q + 1];  // |X_q|
    cudaSetDevice(g.ctx->device);
    int rc = ensure_work(g);
    if (rc) return rc;
    if ((rc = dalloc(g.ctx, &g.sched, (size_t)g.n, "removal order"))) return rc;
    if ((rc = dalloc(g.ctx, &g.dsum, (size_t)g.n + 1, "per-round sums"))) return rc;
    if (keep && (rc = dalloc(g.ctx, &g.keep, (size_t)g.n, "kept nodes"))) return rc;
    if (g.n > 0)
        KH_CUDA_TRY(g.ctx, cudaMemcpy(g.sched, round_of, sizeof(int32_t) * (size_t)g.n, cudaMemcpyHostToDevice));
    if (keep && g.n > 0)
        KH_CUDA_TRY(g.ctx, cudaMemcpy(g.keep, keep, (size_t)g.n, cudaMemcpyHostToDevice));
    KH_CUDA_TRY(g.ctx, cudaMemset(g.dsum, 0, sizeof(unsigned long long) * ((size_t)g.n + 1)));
    g.dense = true;
    g.start_keep = keep != nullptr;
    g.start_alive = keep ? left[0] : g.n;
    rc = run_core(g, exact == 0, nullptr, nullptr, false);
    g.dense = false;
    g.start_keep = false;
    if (rc) return rc;
    std::vector<unsigned long long> s((size_t)rounds);
    KH_CUDA_TRY(g.ctx, cudaMemcpy(s.data(), g.dsum, sizeof(unsigned long long) * (size_t)rounds, cudaMemcpyDeviceToHost));
    int32_t arg = -1;
    for (int32_t q = 0; q < rounds; ++q) {
        if (sum) sum[q] = (uint64_t)s[(size_t)q];
        if (size) size[q] = left[(size_t)q];
        if (left[(size_t)q] == 0) continue;
        // densest: largest sum / size, compared exactly; ties keep the earlier (larger) set
        if (arg < 0 || (unsigned __int128)s[(size_t)q] * (unsigned __int128)left[(size_t)arg] >
                           (unsigned __int128)s[(size_t)arg] * (unsigned __int128)left[(size_t)q])
            arg = q;
    }
    if (best) *best = arg;
    return KH_OK;
}
}  // namespace kh

int kh_dense(kh_graph* G, int32_t exact, const int32_t* round_of, int32_t rounds, uint64_t* sum,
             int64_t* size, int32_t* best) {
    kh::NvtxRange nvtx_range("kh_dense");
    if (!G || !round_of) return KH_EINVAL;
    return kh::dense_common(G->g, exact, round_of, rounds, nullptr, sum, size, best);
}

int kh_dense_pruned(kh_graph* G, int32_t exact, const int32_t* round_of, int32_t rounds,
                    const uint64_t* core, double eps, uint64_t* sum, int64_t* size, int32_t* best,
                    uint8_t* kept) {
    kh::NvtxRange nvtx_range("kh_dense_pruned");
    if (!G || !round_of || !core) return KH_EINVAL;
    Graph& g = G->g;
    if (!(eps > 0.0) || !(eps < 1.0)) return kh::set_error(g.ctx, KH_EINVAL, "need 0 < eps < 1");
    // Sec. 6: drop every node with c'(v) < gamma k', gamma = (1 - eps) / (1 + eps),
    // k' = max c' (compared in double precision)
    uint64_t kmax = 0;
    for (int64_t v = 0; v < g.n; ++v) kmax = core[v] > kmax ? core[v] : kmax;
    const double thr = (1.0 - eps) / (1.0 + eps) * (double)kmax;
    std::vector<uint8_t> keep((size_t)(g.n > 0 ? g.n : 1));
    for (int64_t v = 0; v < g.n; ++v) keep[(size_t)v] = (double)core[v] >= thr ? 1 : 0;
    if (kept && g.n > 0) memcpy(kept, keep.data(), (size_t)g.n);
    return kh::dense_common(g, exact, round_of, rounds, keep.data(), sum, size, best);
}

int kh_peel_stats(kh_graph* G, int64_t* refreshed, int64_t* changed, int64_t* stopped) {
    if (!G) return KH_EINVAL;
    Graph& g = G->g;
    if (!g.have_rounds) return kh::set_error(g.ctx, KH_EINVAL, "no peeling has run on this graph");
    for (int i = 0; i <= kh::kMaxH; ++i) {
        if (refreshed) refreshed[i] = g.last_lvl_work[i];
        if (changed) changed[i] = g.last_lvl_changed[i];
    }
    if (stopped) *stopped = g.last_stopped;
    return KH_OK;
}

int kh_prof_enable(kh_graph* G, int32_t on) {
    if (!G) return KH_EINVAL;
    Graph& g = G->g;
    cudaSetDevice(g.ctx->device);
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(g.ctx->stream));
    if (!g.prof_ev) g.prof_ev = new std::vector<cudaEvent_t>();
    if (!g.prof_kind) g.prof_kind = new std::vector<int>();
    if (!g.prof_snapi) g.prof_snapi = new std::vector<int64_t>();
    if (!g.ev_pool) g.ev_pool = new std::vector<cudaEvent_t>();
    for (cudaEvent_t e : *g.prof_ev) g.ev_pool->push_back(e);
    g.prof_ev->clear();
    g.prof_kind->clear();
    g.prof_snapi->clear();
    g.prof_nsnap = 0;
    // the byte snapshots are optional: without their buffer the byte trace reads ~0
    if (on && !g.prof_snap &&
        cudaMalloc((void**)&g.prof_snap, sizeof(unsigned long long) * (size_t)kh::kProfSnapCap) !=
            cudaSuccess) {
        cudaGetLastError();
        g.prof_snap = nullptr;
    }
    for (int k = 0; k < kh::kProfKinds; ++k) {
        g.prof_ms[k] = 0.0;
        g.prof_launches[k] = 0;
        if (g.prof_trace[k]) g.prof_trace[k]->clear();
        if (g.prof_btrace[k]) g.prof_btrace[k]->clear();
    }
    KH_CUDA_TRY(g.ctx, cudaMemset(g.state->bytes, 0, sizeof(g.state->bytes)));
    g.prof_on = on != 0;
    return KH_OK;
}

int kh_prof_read(kh_graph* G, int32_t kind, double* ms, int64_t* launches, double* alg_bytes) {
    if (!G) return KH_EINVAL;
    Graph& g = G->g;
    if (kind < 0 || kind >= kh::kProfKinds) return kh::set_error(g.ctx, KH_EINVAL, "bad profiling kind");
    cudaSetDevice(g.ctx->device);
    int rc = kh::prof_collect(g);
    if (rc) return rc;
    unsigned long long b = 0;
    KH_CUDA_TRY(g.ctx, cudaMemcpy(&b, &g.state->bytes[kind], sizeof(b), cudaMemcpyDeviceToHost));
    if (ms) *ms = g.prof_ms[kind];
    if (launches) *launches = g.prof_launches[kind];
    if (alg_bytes) *alg_bytes = (double)b;
    return KH_OK;
}

int kh_prof_trace(kh_graph* G, int32_t kind, float* ms, int64_t cap, int64_t* count) {
    if (!G || !count || cap < 0 || (cap > 0 && !ms)) return KH_EINVAL;
    Graph& g = G->g;
    if (kind < 0 || kind >= kh::kProfKinds) return kh::set_error(g.ctx, KH_EINVAL, "bad profiling kind");
    cudaSetDevice(g.ctx->device);
    int rc = kh::prof_collect(g);
    if (rc) return rc;
    const std::vector<float>* t = g.prof_trace[kind];
    const int64_t total = t ? (int64_t)t->size() : 0;
    for (int64_t i = 0; i < total && i < cap; ++i) ms[i] = (*t)[(size_t)i];
    *count = total;
    return KH_OK;
}

int kh_prof_trace_bytes(kh_graph* G, int32_t kind, uint64_t* bytes, int64_t cap, int64_t* count) {
    if (!G || !count || cap < 0 || (cap > 0 && !bytes)) return KH_EINVAL;
    Graph& g = G->g;
    if (kind < 0 || kind >= kh::kProfKinds) return kh::set_error(g.ctx, KH_EINVAL, "bad profiling kind");
    cudaSetDevice(g.ctx->device);
    int rc = kh::prof_collect(g);
    if (rc) return rc;
    const std::vector<unsigned long long>* t = g.prof_btrace[kind];
    const int64_t total = t ? (int64_t)t->size() : 0;
    for (int64_t i = 0; i < total && i < cap; ++i) bytes[i] = (uint64_t)(*t)[(size_t)i];
    *count = total;
    return KH_OK;
}

int kh_launch_count(kh_graph* G, int64_t* launches) {
    if (!G || !launches) return KH_EINVAL;
    *launches = G->g.launches;
    return KH_OK;
}

int kh_sync(kh_graph* G) {
    if (!G) return KH_EINVAL;
    cudaSetDevice(G->g.ctx->device);
    KH_CUDA_TRY(G->g.ctx, cudaStreamSynchronize(G->g.ctx->stream));
    return KH_OK;
}

}  // extern "C"
