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
//   4. alive[R] = 0, counters advance                      (k_finish, k_advance)
// Removing every node with d <= c at once gives the same core map as Alg. 4's
// one-at-a-time loop because d(v; X) never grows as X shrinks (deg_h by
// inclusion of neighbourhoods; the estimate by Prop. 4.2): every node of R
// would still have d <= c when its turn came.
//
// Exact mode applies the paper's early stop (Sec. 5): once c >= |X| - 1 every
// remaining node has deg_h <= |X| - 1 <= c, so all get core c in the next round.
#include <cstring>

#include "kh_internal.cuh"

namespace kh {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kPeelThreads = 256;

template <typename T>
__global__ void k_min_alive(const uint8_t* __restrict__ alive, const T* __restrict__ d, int64_t n,
                            DevState* st) {
    unsigned long long m = ~0ull;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (alive[v] == 1) {
            const unsigned long long x = (unsigned long long)d[v];
            if (x < m) m = x;
        }
    for (int off = 16; off > 0; off >>= 1) {
        const unsigned long long o = __shfl_down_sync(kFull, m, off);
        if (o < m) m = o;
    }
    __shared__ unsigned long long s_m[kPeelThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (lane == 0) s_m[warp] = m;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int w = 1; w < (int)(blockDim.x >> 5); ++w)
            if (s_m[w] < m) m = s_m[w];
        if (m != ~0ull) atomicMin(&st->minval, m);
    }
}

template <typename T, typename C>
__global__ void k_select(uint8_t* __restrict__ alive, const T* __restrict__ d, int64_t n,
                         DevState* st, C* __restrict__ core, int32_t* __restrict__ round_of,
                         int32_t* __restrict__ R, int32_t* __restrict__ seen) {
    const unsigned long long c = st->c > st->minval ? st->c : st->minval;
    const int round = st->round;
    const int lane = threadIdx.x & 31;
    int keep = 0;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int64_t nround = (n + 31) & ~(int64_t)31;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < nround; v += stride) {
        bool rm = false;
        if (v < n && alive[v] == 1) {
            if ((unsigned long long)d[v] <= c) {
                rm = true;
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
}

// Early stop: every remaining node gets core c in round `round + 1`.
template <typename C>
__global__ void k_assign_rest(uint8_t* __restrict__ alive, int64_t n, const DevState* st,
                              C* __restrict__ core, int32_t* __restrict__ round_of) {
    const unsigned long long c = st->c > st->minval ? st->c : st->minval;
    const int round = st->round + 1;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride)
        if (alive[v] == 1) {
            core[v] = (C)c;
            round_of[v] = round;
            alive[v] = 0;
        }
}

__global__ void k_finish(uint8_t* __restrict__ alive, const int32_t* __restrict__ R,
                         const DevState* st) {
    const int nR = st->nR;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < nR; i += stride)
        alive[R[i]] = 0;
}

__global__ void k_advance(DevState* st) {
    if (st->minval > st->c && st->minval != ~0ull) st->c = st->minval;
    st->minval = ~0ull;
    st->round += 1;
    st->n_alive = st->n_alive_next;
    st->n_alive_next = 0;
    st->nR = 0;
    st->nW = 0;
    st->nF[0] = st->nF[1] = 0;
}

int peel_grid(const Graph& g) {
    int64_t grid = (g.n + kPeelThreads - 1) / kPeelThreads;
    const int64_t gmax = (int64_t)g.ctx->sm_count * 4;
    if (grid > gmax) grid = gmax;
    return (int)(grid < 1 ? 1 : grid);
}

// Full-graph pass: every alive node gets d (exact deg_h or the estimate).
int full_pass(Graph& g, bool sampled, cudaStream_t s) {
    if (!sampled) return launch_hdeg(g, nullptr, nullptr, g.n, g.d32, nullptr, 0, 0, s);
    for (int i = 1; i <= g.h; ++i) {
        int rc = launch_level(g, i, nullptr, nullptr, g.n, 0, s);
        if (rc) return rc;
    }
    return KH_OK;
}

int refresh(Graph& g, bool sampled, cudaStream_t s) {
    if (!sampled) {
        for (int hop = 1; hop <= g.h; ++hop) launch_ball_hop(g, hop, s);
        return launch_hdeg(g, g.listW, &g.state->nW, 0, g.d32, nullptr, 0, 0, s);
    }
    for (int i = 1; i <= g.h; ++i) {
        cudaMemsetAsync(&g.state->nW, 0, sizeof(int), s);
        launch_mark_neighbours(g, g.listR, &g.state->nR, i, s);
        if (i >= 2) launch_mark_neighbours(g, g.listC[(i - 1) & 1], &g.state->nC[(i - 1) & 1], i, s);
        int rc = launch_level(g, i, g.listW, &g.state->nW, 0, i < g.h ? 1 : 0, s);
        if (rc) return rc;
    }
    return KH_OK;
}

int check_state_err(Graph& g, const DevState& hs) {
    if (hs.err)
        return set_error(g.ctx, KH_EINTERNAL, "device check failed (flags 0x%x)", hs.err);
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
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.state, 0, sizeof(DevState), s));
    rc = full_pass(g, true, s);
    if (rc) return rc;
    DevState hs;
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(&hs, g.state, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
    return check_state_err(g, hs);
}

int run_core(Graph& g, bool sampled, void* out_core, int32_t* round_of_host, bool out_dev) {
    (void)round_of_host;
    cudaStream_t s = g.ctx->stream;
    int rc = ensure_work(g);
    if (rc) return rc;
    if (sampled) {
        rc = ensure_lists(g);
        if (rc) return rc;
    }
    g.have_rounds = false;
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.alive, 1, (size_t)g.n, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.seen, 0xff, sizeof(int32_t) * (size_t)g.n, s));
    DevState init;
    memset(&init, 0, sizeof(init));
    init.minval = ~0ull;
    init.n_alive = (int)g.n;
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(g.state, &init, sizeof(init), cudaMemcpyHostToDevice, s));
    rc = full_pass(g, sampled, s);
    if (rc) return rc;
    const int grid = peel_grid(g);
    DevState hs;
    int64_t rounds = 0;
    int64_t alive_left = g.n;
    while (alive_left > 0) {
        if (rounds > g.n + 1)
            return set_error(g.ctx, KH_ETIMEOUT, "peeling did not finish within n+1 rounds");
        if (sampled) {
            k_min_alive<unsigned long long><<<grid, kPeelThreads, 0, s>>>(g.alive, g.d64, g.n, g.state);
            k_select<unsigned long long, unsigned long long><<<grid, kPeelThreads, 0, s>>>(
                g.alive, g.d64, g.n, g.state, g.core64, g.round_of, g.listR, g.seen);
        } else {
            k_min_alive<int32_t><<<grid, kPeelThreads, 0, s>>>(g.alive, g.d32, g.n, g.state);
            k_select<int32_t, int32_t><<<grid, kPeelThreads, 0, s>>>(
                g.alive, g.d32, g.n, g.state, g.core32, g.round_of, g.listR, g.seen);
        }
        KH_CUDA_TRY(g.ctx, cudaGetLastError());
        KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(&hs, g.state, sizeof(DevState), cudaMemcpyDeviceToHost, s));
        KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
        rc = check_state_err(g, hs);
        if (rc) return rc;
        const unsigned long long c = hs.c > hs.minval ? hs.c : hs.minval;
        alive_left = hs.n_alive_next;
        ++rounds;
        if (alive_left > 0 && !sampled && c + 1 >= (unsigned long long)alive_left) {
            k_assign_rest<int32_t><<<grid, kPeelThreads, 0, s>>>(g.alive, g.n, g.state, g.core32,
                                                                 g.round_of);
            ++rounds;
            alive_left = 0;
        } else if (alive_left > 0) {
            rc = refresh(g, sampled, s);
            if (rc) return rc;
        }
        k_finish<<<grid, kPeelThreads, 0, s>>>(g.alive, g.listR, g.state);
        k_advance<<<1, 1, 0, s>>>(g.state);
        KH_CUDA_TRY(g.ctx, cudaGetLastError());
    }
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(&hs, g.state, sizeof(DevState), cudaMemcpyDeviceToHost, s));
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
    rc = check_state_err(g, hs);
    if (rc) return rc;
    g.last_rounds = rounds;
    g.last_updates = (int64_t)hs.updates;
    g.have_rounds = true;
    const size_t bytes = (size_t)g.n * (sampled ? sizeof(unsigned long long) : sizeof(int32_t));
    const void* src = sampled ? (const void*)g.core64 : (const void*)g.core32;
    if (g.n > 0)
        KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(out_core, src, bytes,
                                           out_dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s));
    if (!out_dev) KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
    return KH_OK;
}

}  // namespace kh
