// kh_tune.cu -- the autotuner of the exact h-degree pass, and the dispatch of
// the whole-graph exact h-degree / fixed-level count calls.
//
// Three kernels compute deg_2 of every node (Sec. 2) with different visited-set
// layouts:
//   KH_VAR_CTA     k_hdeg: one CTA per source, a visited bitmap of all n nodes
//                  in shared memory (only while n bits fit), cleared per source;
//   KH_VAR_SLICED  k_hdeg2_slice: (source, slice) items, a bitmap of one slice
//                  of the id range, cleared through the words the item set;
//   KH_VAR_SLICED_SMALL  the same for sources of large 2-hop work, and
//                  k_hdeg2_small (a warp and a private hash set per source)
//                  for the rest.
// The sliced kernel has two launch parameters: the number of slices S (at
// least what shared memory requires) and the CTA size.  With a sliced layout
// the sources of the largest 2-hop work may go to the bit-parallel sweeps
// (k_sweep_*: 128 sources per pass over the rows), from a work threshold.
// The tuner times every layout candidate on the same sample of sources (every
// k-th source of the longest-first order, so every size class is represented)
// with CUDA events on the context stream, keeps the fastest, then prices the
// sweep thresholds (sweeps times a measured sweep, plus the sliced layout on
// the rest of the sample), and records the choice in a table keyed by the
// graph's shape class (device SMs, log2 n, log2 nnz, log2 of max degree / mean
// degree).  With the environment variable KH_TUNE_FILE set, the table is read
// from and appended to that text file, so a later process on a graph of the
// same class skips the measurement.  The choice changes the schedule only:
// every candidate computes the same degrees.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include "kh_internal.cuh"

namespace kh {

namespace {

struct TableRow {
    std::string key;
    int variant, slices, threads;
    double ms;
    int sweep_bin;
};

std::mutex g_table_mu;
std::vector<TableRow>* g_table = nullptr;
bool g_table_loaded = false;

int ilog2(double x) { return x <= 1.0 ? 0 : (int)std::floor(std::log2(x)); }

std::string shape_key(const Graph& g, int64_t max_deg) {
    const double avg = g.n > 0 ? (double)g.nnz / (double)g.n : 0.0;
    char buf[160];
    snprintf(buf, sizeof(buf), "hdeg2 sm%d n%d e%d s%d", g.ctx->sm_count, ilog2((double)g.n),
             ilog2((double)g.nnz), ilog2(avg > 0 ? (double)max_deg / avg : 1.0));
    return buf;
}

void load_table_locked() {
    if (g_table_loaded) return;
    g_table_loaded = true;
    g_table = new std::vector<TableRow>();
    const char* path = getenv("KH_TUNE_FILE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "r");
    if (!f) return;
    char line[512];
    while (fgets(line, sizeof(line), f)) {
        // key words ... | variant slices threads ms [sweep_bin]
        char* bar = strchr(line, '|');
        if (!bar || line[0] == '#') continue;
        *bar = 0;
        TableRow r;
        r.key = line;
        r.sweep_bin = 0;
        while (!r.key.empty() && r.key.back() == ' ') r.key.pop_back();
        if (sscanf(bar + 1, "%d %d %d %lf %d", &r.variant, &r.slices, &r.threads, &r.ms, &r.sweep_bin) >= 4)
            g_table->push_back(r);
    }
    fclose(f);
}

bool table_find(const std::string& key, TuneChoice* out) {
    std::lock_guard<std::mutex> lk(g_table_mu);
    load_table_locked();
    for (auto it = g_table->rbegin(); it != g_table->rend(); ++it)
        if (it->key == key) {
            out->variant = it->variant;
            out->slices = it->slices;
            out->threads = it->threads;
            out->ms = it->ms;
            out->sweep_bin = it->sweep_bin;
            return true;
        }
    return false;
}

void table_add(const std::string& key, const TuneChoice& c) {
    std::lock_guard<std::mutex> lk(g_table_mu);
    load_table_locked();
    g_table->push_back({key, c.variant, c.slices, c.threads, c.ms, c.sweep_bin});
    const char* path = getenv("KH_TUNE_FILE");
    if (!path || !*path) return;
    FILE* f = fopen(path, "a");
    if (!f) return;
    fprintf(f, "%s | %d %d %d %.4f %d\n", key.c_str(), c.variant, c.slices, c.threads, c.ms, c.sweep_bin);
    fclose(f);
}

bool cta_fits(const Graph& g) {
    const int64_t words = (g.n + 31) / 32;
    return ((words + 3) & ~(int64_t)3) * 4 <= kSmemBitmapMax;
}

__global__ void k_stride_sample(const int32_t* __restrict__ order, int64_t nsrc, int64_t stride,
                                int32_t* __restrict__ out, int* count) {
    const int64_t m = (nsrc + stride - 1) / stride;
    const int64_t step = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < m; i += step)
        out[i] = order[i * stride];
    if (blockIdx.x == 0 && threadIdx.x == 0) *count = (int)m;
}

// The sliced layout over `order` (nsrc sources, the first nbig of them too
// large for the warp-per-source kernel): KH_VAR_SLICED_SMALL hands the rest
// to that kernel.
int run_sliced(Graph& g, const TuneChoice& c, int32_t* deg, int32_t* cnt, int jlo, int nj,
               cudaStream_t s, const int32_t* order, int64_t nsrc, int64_t nbig) {
    if (c.variant != KH_VAR_SLICED_SMALL)
        return launch_hdeg2_slice(g, deg, cnt, jlo, nj, s, c.slices, c.threads, order, nsrc, true);
    int rc = launch_hdeg2_slice(g, deg, cnt, jlo, nj, s, c.slices, c.threads, order, nbig, true);
    if (rc) return rc;
    return launch_hdeg2_small(g, deg, cnt, jlo, nj, s, order + nbig, nsrc - nbig);
}

// One candidate on the sample; returns its event time in ms (negative: failed).
double time_candidate(Graph& g, const TuneChoice& c, const int32_t* sample, const int* d_count,
                      int64_t m, int32_t* scratch, cudaStream_t s, int64_t sample_big) {
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) {
        cudaGetLastError();
        if (e0) cudaEventDestroy(e0);
        return -1.0;
    }
    double best = -1.0;
    for (int rep = 0; rep < 2; ++rep) {  // the first run warms caches and loads the module
        cudaEventRecord(e0, s);
        int rc;
        if (c.variant == KH_VAR_CTA)
            rc = launch_hdeg(g, sample, d_count, 0, scratch, nullptr, 0, 0, s);
        else
            rc = run_sliced(g, c, scratch, nullptr, 0, 0, s, sample, m, sample_big);
        cudaEventRecord(e1, s);
        if (rc != KH_OK || cudaEventSynchronize(e1) != cudaSuccess) {
            cudaGetLastError();
            best = -1.0;
            break;
        }
        float ms = 0.f;
        cudaEventElapsedTime(&ms, e0, e1);
        best = ms;
    }
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    return best;
}

}  // namespace

int choose_hdeg2(Graph& g, cudaStream_t s, TuneChoice* out) {
    if (g.force_hdeg2.variant != KH_VAR_AUTO) {
        *out = g.force_hdeg2;
        return KH_OK;
    }
    if (g.tuned_hdeg2.variant != KH_VAR_AUTO) {
        *out = g.tuned_hdeg2;
        return KH_OK;
    }
    int rc = ensure_order2(g, s);
    if (rc) return rc;
    // the graph's shape class (needs the largest degree: one read of rowptr)
    int64_t max_deg = 0;
    {
        std::vector<int64_t> rp((size_t)g.n + 1);
        KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(rp.data(), g.rowptr, sizeof(int64_t) * rp.size(),
                                           cudaMemcpyDeviceToHost, s));
        KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
        for (int64_t v = 0; v < g.n; ++v) max_deg = std::max(max_deg, rp[(size_t)v + 1] - rp[(size_t)v]);
    }
    const std::string key = shape_key(g, max_deg);
    TuneChoice c{};
    if (table_find(key, &c) && (c.variant != KH_VAR_CTA || cta_fits(g))) {
        g.tuned_hdeg2 = c;
        *out = c;
        return KH_OK;
    }
    std::vector<TuneChoice> cand;
    if (cta_fits(g)) cand.push_back({KH_VAR_CTA, 0, 256, 0.0});
    const int s0 = hdeg2_min_slices(g.n);
    int slist[4] = {s0, s0 + 1, 2 * s0, 4 * s0};
    for (int si = 0; si < 4; ++si) {
        if (si > 0 && slist[si] == slist[si - 1]) continue;
        if (slist[si] > 64) continue;
        for (int t : {256, 512, 1024}) {
            cand.push_back({KH_VAR_SLICED, slist[si], t, 0.0});
            cand.push_back({KH_VAR_SLICED_SMALL, slist[si], t, 0.0});
        }
    }
    // sample: every stride-th source of the longest-first order
    const int64_t stride = g.nsrc2 > 65536 ? 32 : 1;
    const int64_t m = (g.nsrc2 + stride - 1) / stride;
    // the stride sample keeps order2's order: its first sample_big sources are big
    const int64_t big = hdeg2_small_split(g);
    const int64_t sample_big = (big + stride - 1) / stride;
    int32_t* sample = g.listB;   // scratch (ensure_work holds n entries)
    int32_t* scratch = g.listA;
    int* d_count = &g.state->tune_count;
    if (m > 0) {
        k_stride_sample<<<g.ctx->sm_count, 256, 0, s>>>(g.order2, g.nsrc2, stride, sample, d_count);
        count_launch(g, 1);
    }
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.alive, 1, (size_t)g.n, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.deadbm, 0, ((size_t)(g.n + 127) / 128) * 16, s));
    const int64_t launches_before = g.launches;
    TuneChoice best{};
    best.ms = 1e30;
    for (TuneChoice& t : cand) {
        if (m == 0) break;
        const double ms = time_candidate(g, t, sample, d_count, m, scratch, s, sample_big);
        t.ms = ms;
        if (ms >= 0.0 && ms < best.ms) best = t;
    }
    if (best.variant == KH_VAR_AUTO) {
        // nothing measured (no sources): any valid layout does
        best = cta_fits(g) ? TuneChoice{KH_VAR_CTA, 0, 256, 0.0, 0}
                           : TuneChoice{KH_VAR_SLICED, s0, 1024, 0.0, 0};
    }
    // Bit-parallel sweeps for the sources of 2-hop work >= 2^b - 1, the
    // sliced layout for the rest: the number of sweeps times the time of the
    // middle sweep of the range (a sweep's cost hardly depends on its batch,
    // except for the first few, whose sources' own rows are the longest),
    // plus the sliced layout's time on the sample's remaining sources scaled
    // by the stride, against the sliced layout alone on the whole sample,
    // likewise scaled.
    // (only where the whole pass takes 20 ms or more, and only for a predicted
    // gain of 5%: on small graphs the sample times are too short to rank them)
    best.sweep_bin = 0;
    if (best.variant != KH_VAR_CTA && m > 0 && hdeg2_sources_from_bin(g, kSweepMinBin) > 0 &&
        best.ms * (double)stride >= 20.0) {
        auto time_sweep = [&](int64_t first, int64_t nb) -> double {
            cudaEvent_t e0 = nullptr, e1 = nullptr;
            double t = -1.0;
            if (cudaEventCreate(&e0) == cudaSuccess && cudaEventCreate(&e1) == cudaSuccess) {
                for (int rep = 0; rep < 2; ++rep) {  // the first run also builds the sweep arrays
                    cudaEventRecord(e0, s);
                    const int rc2 = run_sweeps(g, scratch, g.order2 + first, nb, s);
                    cudaEventRecord(e1, s);
                    float ms = 0.f;
                    if (rc2 != KH_OK || cudaEventSynchronize(e1) != cudaSuccess ||
                        cudaEventElapsedTime(&ms, e0, e1) != cudaSuccess) {
                        cudaGetLastError();
                        t = -1.0;
                        break;
                    }
                    t = ms;
                }
            } else {
                cudaGetLastError();
            }
            if (e0) cudaEventDestroy(e0);
            if (e1) cudaEventDestroy(e1);
            return t;
        };
        const double t_warm = time_sweep(0, std::min<int64_t>(g.nsrc2, 128));  // builds the arrays
        const double t_none = best.ms * (double)stride;
        double t_best = 0.95 * t_none;
        for (int bin = kOrderBinsMax - 1; t_warm >= 0.0 && bin >= kSweepMinBin; --bin) {
            const int64_t nsw = hdeg2_sources_from_bin(g, bin);
            if (nsw == 0) continue;
            if (nsw >= g.nsrc2) break;
            const int64_t sbig = (nsw + stride - 1) / stride;  // sample entries that are swept
            if (sbig >= m) break;
            const int64_t nb_mid = std::min<int64_t>(nsw, 128);
            const int64_t mid = ((nsw / 2) / 128) * 128;
            const double t_mid = time_sweep(mid + nb_mid <= nsw ? mid : nsw - nb_mid, nb_mid);
            if (t_mid < 0.0) break;
            TuneChoice rest = best;
            const double t_rest = time_candidate(g, rest, sample + sbig, d_count, m - sbig, scratch, s,
                                                 sample_big > sbig ? sample_big - sbig : 0);
            if (t_rest < 0.0) break;
            const double t = (double)((nsw + 127) / 128) * t_mid + t_rest * (double)stride;
            if (t < t_best) {
                t_best = t;
                best.sweep_bin = bin;
            }
        }
    }
    g.launches = launches_before;  // tuning launches are not the caller's work
    g.tuned_hdeg2 = best;
    table_add(key, best);
    *out = best;
    return KH_OK;
}

int run_hdeg_full(Graph& g, int32_t* deg, int32_t* cnt, int jlo, int nj, cudaStream_t s) {
    if (g.h == 2 && !g.gid && g.n > 0) {
        TuneChoice c{};
        int rc = choose_hdeg2(g, s, &c);
        if (rc) return rc;
        if (c.variant == KH_VAR_SLICED || c.variant == KH_VAR_SLICED_SMALL) {
            rc = ensure_order2(g, s);
            if (rc) return rc;
            // the sources of largest 2-hop work go to the bit-parallel sweeps
            // (2-degrees only: the fixed-level counts stay with the sliced kernel)
            int bin = g.sw_force != 0 ? g.sw_force : c.sweep_bin;
            if (cnt || bin < 0) bin = 0;
            int64_t nsw = bin > 0 ? hdeg2_sources_from_bin(g, bin) : 0;
            const int64_t big = hdeg2_small_split(g);
            rc = run_sliced(g, c, deg, cnt, jlo, nj, s, g.order2 + nsw, g.nsrc2 - nsw,
                            big > nsw ? big - nsw : 0);
            if (rc || nsw == 0) return rc;
            return run_sweeps(g, deg, g.order2, nsw, s);
        }
    }
    return launch_hdeg(g, nullptr, nullptr, g.n, deg, cnt, jlo, nj, s);
}

}  // namespace kh

extern "C" int kh_set_variant(kh_graph* G, int32_t op, int32_t variant, int32_t slices,
                              int32_t threads) {
    if (!G) return KH_EINVAL;
    kh::Graph& g = G->g;
    if (op == KH_OP_PEEL_COMPACT) {
        if (variant != KH_VAR_AUTO && variant != KH_COMPACT_OFF && variant != KH_COMPACT_ALWAYS)
            return kh::set_error(g.ctx, KH_EINVAL, "unknown compaction setting %d", variant);
        g.compact_mode = variant;
        return KH_OK;
    }
    if (op == KH_OP_LEVEL_UNION) {
        if (variant != KH_VAR_AUTO && variant != KH_LEVELU_STEPPED && variant != KH_LEVELU_FREE &&
            variant != KH_LEVELU_GROUPED)
            return kh::set_error(g.ctx, KH_EINVAL, "unknown union schedule %d", variant);
        if (slices < 0 || slices > 64 || (slices & (slices - 1)))
            return kh::set_error(g.ctx, KH_EINVAL, "group divisor %d: 0 or a power of two up to 64",
                                 slices);
        g.levelu_mode = variant;
        g.levelu_div = slices;
        return KH_OK;
    }
    if (op == KH_OP_HDEG2_SWEEP) {
        if (variant == KH_VAR_AUTO) {
            g.sw_force = 0;
        } else if (variant == KH_SWEEP_OFF) {
            g.sw_force = -1;
        } else if (variant == KH_SWEEP_FROM) {
            if (slices < 1 || slices >= kh::kOrderBinsMax)
                return kh::set_error(g.ctx, KH_EINVAL, "sweep work bin %d outside [1, %d)", slices,
                                     kh::kOrderBinsMax);
            g.sw_force = slices;
        } else {
            return kh::set_error(g.ctx, KH_EINVAL, "unknown sweep setting %d", variant);
        }
        return KH_OK;
    }
    if (op != KH_OP_HDEG2) return kh::set_error(g.ctx, KH_EINVAL, "unknown operation %d", op);
    if (variant == KH_VAR_AUTO) {
        g.force_hdeg2 = kh::TuneChoice{};
        return KH_OK;
    }
    if (variant == KH_VAR_CTA) {
        const int64_t words = (g.n + 31) / 32;
        if (((words + 3) & ~(int64_t)3) * 4 > kh::kSmemBitmapMax)
            return kh::set_error(g.ctx, KH_EINVAL, "n too large for the one-CTA-per-source layout");
        g.force_hdeg2 = kh::TuneChoice{KH_VAR_CTA, 0, 256, 0.0};
        return KH_OK;
    }
    if (variant != KH_VAR_SLICED && variant != KH_VAR_SLICED_SMALL)
        return kh::set_error(g.ctx, KH_EINVAL, "unknown variant %d", variant);
    if (threads != 128 && threads != 256 && threads != 512 && threads != 1024)
        return kh::set_error(g.ctx, KH_EINVAL, "threads must be 128, 256, 512 or 1024");
    if (slices < kh::hdeg2_min_slices(g.n) || slices > 1024 || (g.n > 0 && slices > g.n))
        return kh::set_error(g.ctx, KH_EINVAL, "slices must lie in [%d, min(1024, n)]",
                             kh::hdeg2_min_slices(g.n));
    g.force_hdeg2 = kh::TuneChoice{variant, slices, threads, 0.0};
    return KH_OK;
}

extern "C" int kh_get_variant(kh_graph* G, int32_t op, int32_t* variant, int32_t* slices,
                              int32_t* threads, double* tuned_ms) {
    if (!G) return KH_EINVAL;
    kh::Graph& g = G->g;
    if (op == KH_OP_PEEL_COMPACT || op == KH_OP_LEVEL_UNION) {
        if (variant) *variant = op == KH_OP_PEEL_COMPACT ? g.compact_mode : g.levelu_mode;
        if (slices) *slices = op == KH_OP_LEVEL_UNION ? g.levelu_div : 0;
        if (threads) *threads = 0;
        if (tuned_ms) *tuned_ms = 0.0;
        return KH_OK;
    }
    const bool sweep_op = op == KH_OP_HDEG2_SWEEP;
    if (sweep_op) op = KH_OP_HDEG2;
    if (op != KH_OP_HDEG2) return kh::set_error(g.ctx, KH_EINVAL, "unknown operation %d", op);
    cudaSetDevice(g.ctx->device);
    kh::TuneChoice c{};
    int rc = kh::ensure_work(g);
    if (rc) return rc;
    if (!g.ranks_valid) {
        kh::launch_ranks(g, g.ctx->stream);
        g.ranks_valid = true;
    }
    rc = kh::choose_hdeg2(g, g.ctx->stream, &c);
    if (rc) return rc;
    if (sweep_op) {
        // the sweep setting in force: off, or the work bin it starts from
        const int bin = g.sw_force != 0 ? g.sw_force : c.sweep_bin;
        if (variant) *variant = bin > 0 ? KH_SWEEP_FROM : KH_SWEEP_OFF;
        if (slices) *slices = bin > 0 ? bin : 0;
        if (threads) *threads = 0;
        if (tuned_ms) *tuned_ms = c.ms;
        return KH_OK;
    }
    if (variant) *variant = c.variant;
    if (slices) *slices = c.slices;
    if (threads) *threads = c.threads;
    if (tuned_ms) *tuned_ms = c.ms;
    return KH_OK;
}
