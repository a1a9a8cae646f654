// kh_hdeg2.cu -- exact 2-degrees of a whole graph with sliced shared-memory
// visited sets (graphs whose n-bit visited set does not fit in shared memory).
//
// Sec. 2: deg_2(v) = |N(v; 2)| - 1 with N(v; 2) = {v} U A(v) U (U_{w in A(v)} A(w)).
// For a node with at least one neighbour, v itself lies in A(w) for every w in
// A(v) (the graph is symmetric), so N(v; 2) is the union of the rows of v and
// of its neighbours.  The node range [0, n) is cut into S slices of `width`
// ids; one work item is (source v, slice s): a CTA marks, in a shared-memory
// bitmap of `width` bits, every member of those rows that falls in slice s
// (each row is sorted, so its part inside the slice is found by two searches)
// and adds the number of newly set bits to deg[v].  Each row entry is read
// once over the S items of a source, so the items of one source move the
// algorithmic bytes of one BFS.
//
// Sources are processed in decreasing order of their 2-hop work sum_{w in
// A(v)} deg(w) (longest first), so the large balls of hubs start early and the
// small ones fill the tail.  Isolated nodes (deg_2 = 0) are not items.
//
// The bitmap is cleared between items through the list of words the item set
// first (when it fits), otherwise with vector stores over the whole slice.
#include "kh_internal.cuh"

namespace kh {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kMaxHeavy2 = 128;      // rows expanded by the whole CTA per item
constexpr int kHeavyRow2 = 512;      // a row part this long goes to the whole CTA
constexpr int kTouchCap = 4096;      // words cleared one by one (else full clear)
constexpr int kOrderBins = 48;       // log2 bins of the 2-hop work

struct Slice2Args {
    const int64_t* rowptr;
    const int32_t* col;
    const uint8_t* rank;
    int64_t n;
    int nslices;
    int64_t width;        // nodes per slice (multiple of 128)
    const int32_t* order;  // sources, longest first
    int64_t nsrc;
    int32_t* deg;          // += marked nodes per item (starts at -1 / 0)
    int32_t* cnt;          // fixed-level counts (RANKS), += per item
    int jlo, nj;
    int* work_ctr;
    int* err;
    unsigned long long* updates;
    unsigned long long* bytes;
};

// First position p in [b, e) with col[p] >= key (e if none); the whole warp
// calls it and every lane gets the answer.  Each step samples 32 evenly spaced
// entries and keeps the gap where the sorted row crosses key.
__device__ __forceinline__ int64_t warp_lower_bound(const int32_t* __restrict__ col, int64_t b,
                                                    int64_t e, int32_t key, int lane) {
    // 32-bit offsets from b (a row has fewer than 2^31 entries)
    const int32_t* __restrict__ r = col + b;
    int lo = 0, hi = (int)(e - b);  // answer in [lo, hi]
    while (hi - lo > 32) {
        const int step = (hi - lo + 31) >> 5;
        const int p = lo + lane * step;
        const bool below = p < hi && __ldg(r + p) < key;
        const int c = __popc(__ballot_sync(kFull, below));
        // positions lo + j*step, j < c, hold keys below `key`
        const int nlo = c > 0 ? lo + (c - 1) * step + 1 : lo;
        const int nhi = lo + c * step;
        lo = nlo;
        hi = nhi < hi ? nhi : hi;
    }
    const int p = lo + lane;
    const bool below = p < hi && __ldg(r + p) < key;
    return b + lo + __popc(__ballot_sync(kFull, below));
}

// Mark u (in the slice) in the bitmap; count it and remember its word when it
// is the word's first bit.  All 32 lanes call this together.
template <bool RANKS>
__device__ __forceinline__ void mark(const Slice2Args& a, uint32_t* bm, int32_t* touch,
                                     int* s_ntouch, int* s_hist, bool valid, int32_t lu,
                                     int32_t u, int lane, int& my) {
    bool fresh_word = false;
    int word = 0;
    if (valid) {
        word = lu >> 5;
        const uint32_t bit = 1u << (lu & 31);
        if (!(*(volatile uint32_t*)(bm + word) & bit)) {
            const uint32_t old = atomicOr(bm + word, bit);
            if (!(old & bit)) {
                ++my;
                if (RANKS) atomicAdd(&s_hist[a.rank[u]], 1);
                fresh_word = old == 0u;
            }
        }
    }
    const uint32_t fm = __ballot_sync(kFull, fresh_word);
    if (fm) {
        const int leader = __ffs(fm) - 1;
        int base = 0;
        if (lane == leader) base = atomicAdd(s_ntouch, __popc(fm));
        base = __shfl_sync(kFull, base, leader);
        if (fresh_word) {
            const int p = base + __popc(fm & ((1u << lane) - 1u));
            if (p < kTouchCap) touch[p] = word;
        }
    }
}

// Mark the entries [ps, pe) of col, lanes take 32 consecutive entries and
// each step issues four independent loads per lane.
template <bool RANKS>
__device__ __forceinline__ void mark_range(const Slice2Args& a, uint32_t* bm, int32_t* touch,
                                           int* s_ntouch, int* s_hist, int64_t ps, int64_t pe,
                                           int64_t first, int64_t stride, int32_t lo, int lane,
                                           int& my) {
    // 32-bit offsets from the part's start (a row has fewer than 2^31 entries)
    const int32_t* __restrict__ base = a.col + ps;
    const int len = (int)(pe - ps);
    for (int k0 = (int)first; k0 < len; k0 += (int)stride) {
        int32_t u[4];
        bool val[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int k = k0 + q * 32 + lane;
            val[q] = k < len;
            u[q] = val[q] ? __ldg(base + k) : lo;
        }
#pragma unroll
        for (int q = 0; q < 4; ++q)
            mark<RANKS>(a, bm, touch, s_ntouch, s_hist, val[q], u[q] - lo, u[q], lane, my);
    }
}

template <bool RANKS>
__global__ void k_hdeg2_slice(Slice2Args a) {
    extern __shared__ __align__(16) uint32_t s_dyn[];
    const int words = (int)(a.width >> 5);
    uint32_t* bm = s_dyn;
    int32_t* touch = reinterpret_cast<int32_t*>(s_dyn + words);
    __shared__ int s_item, s_ntouch, s_nheavy, s_count, s_row;
    __shared__ int64_t s_hb[kMaxHeavy2], s_he[kMaxHeavy2];
    __shared__ int s_hist[32];
    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5, nwarps = blockDim.x >> 5;
    const int64_t total = a.nsrc * a.nslices;
    unsigned long long my_bytes = 0;
    {
        uint4* b4 = reinterpret_cast<uint4*>(bm);
        for (int i = tid; i < (words >> 2); i += blockDim.x) b4[i] = make_uint4(0u, 0u, 0u, 0u);
    }
    __syncthreads();
    for (;;) {
        if (tid == 0) {
            s_item = atomicAdd(a.work_ctr, 1);
            s_ntouch = 0;
            s_nheavy = 0;
            s_row = 0;
            s_count = 0;
        }
        if (RANKS && tid < 32) s_hist[tid] = 0;
        __syncthreads();
        const int64_t item = s_item;
        if (item >= total) break;
        const int v = a.order[item / a.nslices];
        const int sl = (int)(item % a.nslices);
        const int32_t lo = (int32_t)((int64_t)sl * a.width);
        const int64_t hi64 = (int64_t)lo + a.width;
        const int32_t hi = (int32_t)(hi64 < a.n ? hi64 : a.n);
        const int64_t vb = a.rowptr[v], ve = a.rowptr[v + 1];
        const int64_t deg = ve - vb;
        int my = 0;
        // rows: v's own (i == deg) and each neighbour's (i < deg), claimed by
        // the warps one at a time (row lengths vary widely)
        for (;;) {
            int64_t i = 0;
            if (lane == 0) i = atomicAdd(&s_row, 1);
            i = __shfl_sync(kFull, i, 0);
            if (i > deg) break;
            const int32_t x = i < deg ? __ldg(a.col + vb + i) : v;
            const int64_t rb = a.rowptr[x], re = a.rowptr[x + 1];
            const int64_t ps = lo > 0 ? warp_lower_bound(a.col, rb, re, lo, lane) : rb;
            const int64_t pe = hi < a.n ? warp_lower_bound(a.col, ps, re, hi, lane) : re;
            if (lane == 0) my_bytes += (sl == 0 ? 8ull : 0ull) + 4ull * (unsigned long long)(pe - ps);
            if (pe - ps >= kHeavyRow2) {
                int slot = 0;
                if (lane == 0) slot = atomicAdd(&s_nheavy, 1);
                slot = __shfl_sync(kFull, slot, 0);
                if (slot < kMaxHeavy2) {
                    if (lane == 0) {
                        s_hb[slot] = ps;
                        s_he[slot] = pe;
                    }
                    continue;
                }
            }
            mark_range<RANKS>(a, bm, touch, &s_ntouch, s_hist, ps, pe, 0, 128, lo, lane, my);
        }
        __syncthreads();
        const int nh = min(s_nheavy, kMaxHeavy2);
        for (int j = 0; j < nh; ++j)
            mark_range<RANKS>(a, bm, touch, &s_ntouch, s_hist, s_hb[j], s_he[j], (int64_t)warp * 128,
                              (int64_t)nwarps * 128, lo, lane, my);
        for (int off = 16; off > 0; off >>= 1) my += __shfl_down_sync(kFull, my, off);
        if (lane == 0 && my) atomicAdd(&s_count, my);
        __syncthreads();
        if (tid == 0) {
            if (s_count) atomicAdd(a.deg + v, s_count);
            if (sl == 0) {
                atomicAdd(a.updates, 1ull);
                my_bytes += 4ull + (RANKS ? 4ull * (unsigned long long)a.nj : 0ull);
            }
        }
        if (RANKS && tid < a.nj) {
            int c = 0;
            for (int j = a.jlo + tid; j < 32; ++j) c += s_hist[j];
            if (c) atomicAdd(a.cnt + (size_t)v * a.nj + tid, c);
        }
        // clear what this item set
        const int nt = s_ntouch;
        if (nt <= kTouchCap) {
            for (int i = tid; i < nt; i += blockDim.x) bm[touch[i]] = 0u;
        } else {
            uint4* b4 = reinterpret_cast<uint4*>(bm);
            for (int i = tid; i < (words >> 2); i += blockDim.x) b4[i] = make_uint4(0u, 0u, 0u, 0u);
        }
        __syncthreads();
    }
    for (int off = 16; off > 0; off >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, off);
    if (lane == 0 && my_bytes) atomicAdd(a.bytes, my_bytes);
}

// Sources of small 2-hop work (bin < kSmallBin: work < 2^kSmallBin, so at most
// 2 (2^kSmallBin - 1) row entries in all) take one warp each, without slices:
// the warp dedupes its source's 2-ball in a private open-addressing set of
// kSmallSlots node ids in shared memory (load at most one half), cleared with
// vector stores afterwards.  This spares the per-item cost of S slice items
// for the many small balls of a power-law graph.
constexpr int kSmallBin = 9;
constexpr int kSmallSlots = 2048;
constexpr int kSmallWarps = 8;
constexpr uint32_t kIdEmpty = 0xffffffffu;

template <bool RANKS>
__global__ void __launch_bounds__(kSmallWarps * 32)
    k_hdeg2_small(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                  const uint8_t* __restrict__ rank, const int32_t* __restrict__ order,
                  int64_t count, int32_t* __restrict__ deg, int32_t* __restrict__ cnt, int jlo,
                  int nj, unsigned long long* updates, unsigned long long* bytes) {
    extern __shared__ __align__(16) uint32_t s_tab_all[];
    __shared__ int s_hist_all[kSmallWarps][32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    uint32_t* tab = s_tab_all + (size_t)warp * kSmallSlots;
    int* hist = s_hist_all[warp];
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    unsigned long long my_bytes = 0, my_upd = 0;
    {
        uint4* t4 = reinterpret_cast<uint4*>(tab);
        for (int i = lane; i < kSmallSlots / 4; i += 32) t4[i] = make_uint4(kIdEmpty, kIdEmpty, kIdEmpty, kIdEmpty);
    }
    __syncwarp();
    for (int64_t i = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; i < count; i += nw) {
        const int v = order[i];
        if (RANKS) hist[lane] = 0;
        __syncwarp();
        const int64_t vb = rowptr[v], ve = rowptr[v + 1];
        const int64_t dv = ve - vb;
        int my = 0;
        // rows: v's own (r == dv) and each neighbour's
        for (int64_t r = 0; r <= dv; ++r) {
            const int32_t x = r < dv ? __ldg(col + vb + r) : v;
            const int64_t rb = rowptr[x], re = rowptr[x + 1];
            if (lane == 0) my_bytes += 8ull + 4ull * (unsigned long long)(re - rb);
            for (int64_t k = rb + lane; k < re; k += 32) {
                const uint32_t u = (uint32_t)__ldg(col + k);
                uint32_t slot = (u * 0x9E3779B1u) >> (32 - 11);  // 2^11 = kSmallSlots
                for (int probe = 0; probe < kSmallSlots; ++probe) {
                    const uint32_t cur = *(volatile uint32_t*)(tab + slot);
                    if (cur == u) break;
                    if (cur == kIdEmpty) {
                        const uint32_t prev = atomicCAS(tab + slot, kIdEmpty, u);
                        if (prev == kIdEmpty) {
                            ++my;
                            if (RANKS) atomicAdd(&hist[rank[u]], 1);
                            break;
                        }
                        if (prev == u) break;
                    }
                    slot = (slot + 1u) & (kSmallSlots - 1);
                }
            }
        }
        for (int off = 16; off > 0; off >>= 1) my += __shfl_down_sync(kFull, my, off);
        __syncwarp();
        if (lane == 0) {
            deg[v] = my - 1;  // the ball holds v itself (by symmetry, in each neighbour's row)
            ++my_upd;
            my_bytes += 4ull + (RANKS ? 4ull * (unsigned long long)nj : 0ull);
        }
        if (RANKS && lane < nj) {
            int c = 0;
            for (int j = jlo + lane; j < 32; ++j) c += hist[j];
            cnt[(size_t)v * nj + lane] = c - (rank[v] >= jlo + lane ? 1 : 0);
        }
        uint4* t4 = reinterpret_cast<uint4*>(tab);
        for (int q = lane; q < kSmallSlots / 4; q += 32) t4[q] = make_uint4(kIdEmpty, kIdEmpty, kIdEmpty, kIdEmpty);
        __syncwarp();
    }
    for (int off = 16; off > 0; off >>= 1) my_bytes += __shfl_down_sync(kFull, my_bytes, off);
    if (lane == 0 && my_bytes) atomicAdd(bytes, my_bytes);
    if (lane == 0 && my_upd) atomicAdd(updates, my_upd);
}

// 2-hop work of each node and its log2 bin (isolated nodes: bin -1).
__global__ void k_order_bins(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                             int64_t n, int8_t* __restrict__ bin, int* __restrict__ hist) {
    __shared__ int s_h[kOrderBins];
    for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x) s_h[i] = 0;
    __syncthreads();
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t v = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; v < n; v += nw) {
        const int64_t b = rowptr[v], e = rowptr[v + 1];
        unsigned long long w = 0;
        for (int64_t k = b + lane; k < e; k += 32) {
            const int32_t x = col[k];
            w += (unsigned long long)(rowptr[x + 1] - rowptr[x]);
        }
        for (int off = 16; off > 0; off >>= 1) w += __shfl_down_sync(kFull, w, off);
        if (lane == 0) {
            int bb = -1;
            if (e > b) {
                bb = 63 - __clzll((long long)(w + 1));
                if (bb >= kOrderBins) bb = kOrderBins - 1;
                atomicAdd(&s_h[bb], 1);
            }
            bin[v] = (int8_t)bb;
        }
    }
    __syncthreads();
    for (int i = threadIdx.x; i < kOrderBins; i += blockDim.x)
        if (s_h[i]) atomicAdd(hist + i, s_h[i]);
}

// Scatter the non-isolated nodes by bin, largest bin first; hist holds each
// bin's start (exclusive prefix in descending bin order) and is advanced.
__global__ void k_order_scatter(const int8_t* __restrict__ bin, int64_t n, int* __restrict__ pos,
                                int32_t* __restrict__ order) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const int b = bin[v];
        if (b >= 0) order[atomicAdd(pos + b, 1)] = (int32_t)v;
    }
}

// deg[v] starts at -1 for a node with a neighbour (v is counted in its own
// ball), 0 for an isolated node; the counts start at minus v's own rank test.
__global__ void k_init2(const int64_t* __restrict__ rowptr, const uint8_t* __restrict__ rank,
                        int64_t n, int32_t* __restrict__ deg, int32_t* __restrict__ cnt, int jlo,
                        int nj) {
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t v = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; v < n; v += stride) {
        const bool iso = rowptr[v + 1] == rowptr[v];
        deg[v] = iso ? 0 : -1;
        if (cnt) {
            const int rv = rank[v];
            for (int j = 0; j < nj; ++j) cnt[(size_t)v * nj + j] = (!iso && rv >= jlo + j) ? -1 : 0;
        }
    }
}

}  // namespace

size_t hdeg2_smem(int64_t width) { return (size_t)(width / 8) + (size_t)kTouchCap * 4; }

int64_t hdeg2_width(int64_t n, int slices) {
    int64_t w = (n + slices - 1) / slices;
    return (w + 127) & ~(int64_t)127;
}

int hdeg2_min_slices(int64_t n) {
    int s = 1;
    while (hdeg2_smem(hdeg2_width(n, s)) > (size_t)kSmem2Max) ++s;
    return s;
}

int ensure_order2(Graph& g, cudaStream_t s) {
    if (g.order2) return KH_OK;
    int8_t* bin = nullptr;
    int* hist = nullptr;
    int rc = alloc_bytes(g.ctx, (void**)&g.order2, sizeof(int32_t) * (size_t)(g.n > 0 ? g.n : 1),
                         "source order");
    if (rc) return rc;
    cudaError_t e = cudaMallocAsync((void**)&bin, (size_t)(g.n > 0 ? g.n : 1), s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&hist, sizeof(int) * kOrderBins, s);
    if (e == cudaSuccess) e = cudaMemsetAsync(hist, 0, sizeof(int) * kOrderBins, s);
    if (e != cudaSuccess) {
        if (bin) cudaFreeAsync(bin, s);
        if (hist) cudaFreeAsync(hist, s);
        cudaFree(g.order2);
        g.order2 = nullptr;
        return check_cuda(g.ctx, e, "source order");
    }
    const int grid = g.ctx->sm_count * 8;
    k_order_bins<<<grid, 256, 0, s>>>(g.rowptr, g.col, g.n, bin, hist);
    int h[kOrderBins];
    e = cudaMemcpyAsync(h, hist, sizeof(h), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e == cudaSuccess) {
        // starts in descending bin order
        int pos[kOrderBins];
        int64_t acc = 0;
        for (int b = kOrderBins - 1; b >= 0; --b) {
            pos[b] = (int)acc;
            acc += h[b];
        }
        g.nsrc2 = acc;
        for (int b = 0; b < kOrderBins; ++b) g.order2_hist[b] = h[b];
        e = cudaMemcpyAsync(hist, pos, sizeof(pos), cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) {
            k_order_scatter<<<grid, 256, 0, s>>>(bin, g.n, hist, g.order2);
            e = cudaStreamSynchronize(s);  // `pos` is a host stack array
        }
    }
    cudaFreeAsync(bin, s);
    cudaFreeAsync(hist, s);
    count_launch(g, 2);
    if (e != cudaSuccess) {
        cudaFree(g.order2);
        g.order2 = nullptr;
        return check_cuda(g.ctx, e, "source order");
    }
    return KH_OK;
}

int64_t hdeg2_small_split(const Graph& g) {
    int64_t big = 0;
    for (int b = kSmallBin; b < kOrderBins; ++b) big += g.order2_hist[b];
    return big;
}

int launch_hdeg2_small(Graph& g, int32_t* deg, int32_t* cnt, int jlo, int nj, cudaStream_t s,
                       const int32_t* order, int64_t count) {
    if (count <= 0) return KH_OK;
    void (*kern)(const int64_t*, const int32_t*, const uint8_t*, const int32_t*, int64_t, int32_t*,
                 int32_t*, int, int, unsigned long long*, unsigned long long*) =
        cnt ? k_hdeg2_small<true> : k_hdeg2_small<false>;
    const size_t dyn = (size_t)kSmallWarps * kSmallSlots * 4;
    KH_CUDA_TRY(g.ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = 0;
    KH_CUDA_TRY(g.ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, kSmallWarps * 32, dyn));
    if (per_sm < 1) per_sm = 1;
    int64_t grid = (int64_t)g.ctx->sm_count * per_sm;
    const int64_t need = (count + kSmallWarps - 1) / kSmallWarps;
    if (grid > need) grid = need;
    prof_begin(g, kProfBfs, s);
    kern<<<(int)grid, kSmallWarps * 32, dyn, s>>>(g.rowptr, g.col, g.rank, order, count, deg, cnt, jlo,
                                                   nj, &g.state->updates, &g.state->bytes[kProfBfs]);
    count_launch(g, 1);
    prof_end(g, kProfBfs, s);
    return KH_OK;
}

int launch_hdeg2_slice(Graph& g, int32_t* deg, int32_t* cnt, int jlo, int nj, cudaStream_t s,
                       int slices, int threads, const int32_t* order, int64_t nsrc, bool init) {
    if (g.n == 0) return KH_OK;
    const int64_t width = hdeg2_width(g.n, slices);
    const size_t dyn = hdeg2_smem(width);
    if (dyn > (size_t)kSmem2Max) return set_error(g.ctx, KH_EINVAL, "slice too wide for shared memory");
    void (*kern)(Slice2Args) = cnt ? k_hdeg2_slice<true> : k_hdeg2_slice<false>;
    KH_CUDA_TRY(g.ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn));
    int per_sm = 0;
    KH_CUDA_TRY(g.ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kern, threads, dyn));
    if (per_sm < 1) return set_error(g.ctx, KH_EINVAL, "slice kernel does not fit on an SM");
    int64_t grid = (int64_t)g.ctx->sm_count * per_sm;
    const int64_t items = nsrc * slices;
    if (grid > items) grid = items;
    if (grid < 1) grid = 1;
    if (init) {
        k_init2<<<g.ctx->sm_count * 4, 256, 0, s>>>(g.rowptr, g.rank, g.n, deg, cnt, jlo, nj);
        count_launch(g, 1);
    }
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(&g.state->work_ctr[2], 0, sizeof(int), s));
    if (items == 0) return KH_OK;
    Slice2Args a{};
    a.rowptr = g.rowptr;
    a.col = g.col;
    a.rank = g.rank;
    a.n = g.n;
    a.nslices = slices;
    a.width = width;
    a.order = order;
    a.nsrc = nsrc;
    a.deg = deg;
    a.cnt = cnt;
    a.jlo = jlo;
    a.nj = nj;
    a.work_ctr = &g.state->work_ctr[2];
    a.err = &g.state->err;
    a.updates = &g.state->updates;
    a.bytes = &g.state->bytes[kProfBfs];
    prof_begin(g, kProfBfs, s);
    kern<<<(int)grid, threads, dyn, s>>>(a);
    count_launch(g, 1);
    prof_end(g, kProfBfs, s);
    return KH_OK;
}

}  // namespace kh
