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
//
// Two more kernels serve the same pass: sources of small 2-hop work on one
// warp each with a private hash set (k_hdeg2_small), and, for the sources of
// the largest 2-hop work, bit-parallel sweeps of 128 sources at a time
// (k_sweep_*; see the comment above them).
#include <vector>

#include "kh_internal.cuh"

namespace kh {

namespace {

constexpr uint32_t kFull = 0xffffffffu;
constexpr int kMaxHeavy2 = 128;      // rows expanded by the whole CTA per item
constexpr int kHeavyRow2 = 512;      // a row part this long goes to the whole CTA
constexpr int kTouchCap = 4096;      // words cleared one by one (else full clear)
constexpr int kOrderBins = kOrderBinsMax;  // log2 bins of the 2-hop work

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

// ---- bit-parallel sweeps for the sources of largest 2-hop work ----
// For a batch of up to 128 sources s_j, m1[u] holds bit j when u is a
// neighbour of s_j.  A node x lies in N(s_j; 2) exactly when bit j is set in
// m1[x] | OR_{u in A(x)} m1[u] (x = s_j itself through any neighbour u, as s_j
// is in A(u)).  One sweep over all rows thus gives the 2-balls of 128 sources:
// it reads each row once (2m column ids and 2m 16-byte gathers from m1, which
// stays in L2), where the per-source union reads sum_{w in A(s_j)} deg(w)
// entries for each source.  It pays off for sources whose 2-hop work exceeds
// about one pass over the graph per batch.  A filter of one bit per 4 nodes
// (some of them has source bits), held in shared memory by the count kernel,
// skips the gathers of entries that cannot contribute: for batches of
// mid-size sources half of all entries or more.
constexpr int kSweepSrc = 128;
constexpr int kSweepHead = 64;     // row entries the count kernel reads itself (8 per lane)
constexpr int kSweepPiece = 2048;  // entries per tail piece of a longer row
constexpr int kSweepPlanes = 8;    // carry-save counter planes: 255 additions between flushes

// Set (clear = 0) or zero (clear = 1) the batch's source bits on the
// neighbours of its sources, one CTA per source (the largest sources' rows
// hold up to the maximum degree); the setting pass also counts each source's
// algorithmic bytes (those of one 2-hop search).
__global__ void k_sweep_scatter(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                                const int32_t* __restrict__ src, int nb, uint32_t* __restrict__ m1,
                                uint32_t* __restrict__ filter, int clear, unsigned long long* bytes) {
    const int j = blockIdx.x;
    if (j >= nb) return;
    const int v = src[j];
    const int64_t b = rowptr[v], e = rowptr[v + 1];
    unsigned long long my = 0;
    for (int64_t k = b + threadIdx.x; k < e; k += blockDim.x) {
        const int32_t u = __ldg(col + k);
        if (clear) {
            reinterpret_cast<uint4*>(m1)[u] = make_uint4(0u, 0u, 0u, 0u);
            filter[u >> 7] = 0u;
        } else {
            atomicOr(m1 + 4 * (size_t)u + (j >> 5), 1u << (j & 31));
            atomicOr(filter + (u >> 7), 1u << ((u >> 2) & 31));
            my += 8ull + 4ull * (unsigned long long)(rowptr[u + 1] - rowptr[u]);
        }
    }
    if (clear) return;
    if (threadIdx.x == 0) my += 8ull + 4ull * (unsigned long long)(e - b) + 4ull;
    for (int off = 16; off > 0; off >>= 1) my += __shfl_down_sync(kFull, my, off);
    if ((threadIdx.x & 31) == 0 && my) atomicAdd(bytes, my);
}

__device__ __forceinline__ void or4(uint4& a, const uint4 b) {
    a.x |= b.x;
    a.y |= b.y;
    a.z |= b.z;
    a.w |= b.w;
}

// Rows longer than kSweepHead: the OR of m1 over each tail piece of
// kSweepPiece entries, into that row's partial word bh (zeroed per sweep).
__global__ void k_sweep_tails(const int64_t* __restrict__ rowptr, const int32_t* __restrict__ col,
                              const int32_t* __restrict__ hnode, const int32_t* __restrict__ piece_h,
                              const int32_t* __restrict__ piece_off, int64_t npieces,
                              const uint4* __restrict__ m1, const uint32_t* __restrict__ filter,
                              uint32_t* __restrict__ bh) {
    const int lane = threadIdx.x & 31;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t p = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5; p < npieces; p += nw) {
        const int h = piece_h[p];
        const int x = hnode[h];
        const int64_t b = rowptr[x] + piece_off[p];
        const int64_t re = rowptr[x + 1];
        const int64_t e = b + kSweepPiece < re ? b + kSweepPiece : re;
        uint4 acc = make_uint4(0u, 0u, 0u, 0u);
        for (int64_t k = b + lane; k < e; k += 32) {
            const int32_t u = __ldg(col + k);
            if ((__ldg(filter + (u >> 7)) >> ((u >> 2) & 31)) & 1u) or4(acc, __ldg(m1 + u));
        }
        for (int off = 16; off > 0; off >>= 1) {
            acc.x |= __shfl_xor_sync(kFull, acc.x, off);
            acc.y |= __shfl_xor_sync(kFull, acc.y, off);
            acc.z |= __shfl_xor_sync(kFull, acc.z, off);
            acc.w |= __shfl_xor_sync(kFull, acc.w, off);
        }
        if (lane < 4) {
            const uint32_t w = lane == 0 ? acc.x : lane == 1 ? acc.y : lane == 2 ? acc.z : acc.w;
            if (w) atomicOr(bh + 4 * (size_t)h + lane, w);
        }
    }
}

// Add the counts held in carry-save planes (bit `bit` of plane p is worth
// 2^p) to the block's per-source counters; lane gl of a group owns bits
// [16 gl, 16 gl + 16) of the ball word.
__device__ __forceinline__ void sweep_flush(uint32_t (&c)[kSweepPlanes], unsigned int* s_cnt, int gl) {
#pragma unroll
    for (int bit = 0; bit < 16; ++bit) {
        unsigned int v = 0;
#pragma unroll
        for (int p = 0; p < kSweepPlanes; ++p) v |= ((c[p] >> bit) & 1u) << p;
        if (v) atomicAdd(&s_cnt[16 * gl + bit], v);
    }
#pragma unroll
    for (int p = 0; p < kSweepPlanes; ++p) c[p] = 0u;
}

// Ball words of every node (groups of 8 lanes per node, four nodes per warp
// step; a row's first kSweepHead entries here, the rest from bh) and the
// number of nodes in each source's ball (per-lane carry-save counters of 16
// source bits, flushed every 255 nodes).  With use_filter the filter's
// fwords words are first copied to shared memory.
__global__ void __launch_bounds__(1024) k_sweep_count(const int64_t* __restrict__ rowptr,
                                                      const int32_t* __restrict__ col, int64_t n,
                                                      const uint4* __restrict__ m1,
                                                      const uint32_t* __restrict__ filter,
                                                      int use_filter, int fwords,
                                                      const int32_t* __restrict__ hpos,
                                                      const uint4* __restrict__ bh,
                                                      unsigned int* __restrict__ cnt) {
    extern __shared__ __align__(16) uint32_t s_filter[];
    __shared__ unsigned int s_cnt[kSweepSrc];
    for (int i = threadIdx.x; i < kSweepSrc; i += blockDim.x) s_cnt[i] = 0u;
    if (use_filter) {
        const uint4* f4 = reinterpret_cast<const uint4*>(filter);
        uint4* s4 = reinterpret_cast<uint4*>(s_filter);
        for (int i = threadIdx.x; i < (fwords >> 2); i += blockDim.x) s4[i] = f4[i];
    }
    __syncthreads();
    const int lane = threadIdx.x & 31, g = lane >> 3, gl = lane & 7;
    const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    uint32_t c[kSweepPlanes];
#pragma unroll
    for (int p = 0; p < kSweepPlanes; ++p) c[p] = 0u;
    int adds = 0;
    // the loop bound is the same for the whole warp (the shuffles need every lane)
    for (int64_t x0 = (((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5) * 4; x0 < n; x0 += nw * 4) {
        const int64_t x = x0 + g;
        uint4 acc = make_uint4(0u, 0u, 0u, 0u);
        if (x < n) {
            const int64_t b = rowptr[x], e = rowptr[x + 1];
            if (e > b) {
                if (gl == 0) acc = m1[x];
                const int64_t he = e - b > kSweepHead ? b + kSweepHead : e;
                if (use_filter) {
                    for (int64_t k = b + gl; k < he; k += 8) {
                        const int32_t u = __ldg(col + k);
                        if ((s_filter[u >> 7] >> ((u >> 2) & 31)) & 1u) or4(acc, __ldg(m1 + u));
                    }
                } else {
                    for (int64_t k = b + gl; k < he; k += 8) or4(acc, __ldg(m1 + __ldg(col + k)));
                }
                if (gl == 1 && e - b > kSweepHead) or4(acc, bh[hpos[x]]);
            }
        }
        for (int off = 1; off < 8; off <<= 1) {
            acc.x |= __shfl_xor_sync(kFull, acc.x, off);
            acc.y |= __shfl_xor_sync(kFull, acc.y, off);
            acc.z |= __shfl_xor_sync(kFull, acc.z, off);
            acc.w |= __shfl_xor_sync(kFull, acc.w, off);
        }
        const int wi = gl >> 1;
        const uint32_t word = wi == 0 ? acc.x : wi == 1 ? acc.y : wi == 2 ? acc.z : acc.w;
        uint32_t carry = (gl & 1) ? (word >> 16) : (word & 0xffffu);
#pragma unroll
        for (int p = 0; p < kSweepPlanes; ++p) {
            const uint32_t t = c[p] & carry;
            c[p] ^= carry;
            carry = t;
        }
        if (++adds == (1 << kSweepPlanes) - 1) {
            sweep_flush(c, s_cnt, gl);
            adds = 0;
        }
    }
    sweep_flush(c, s_cnt, gl);
    __syncthreads();
    for (int i = threadIdx.x; i < kSweepSrc; i += blockDim.x)
        if (s_cnt[i]) atomicAdd(cnt + i, s_cnt[i]);
}

// deg_2 of the batch's sources (the ball holds the source itself); the
// counters are zeroed for the next sweep.
__global__ void k_sweep_finish(const int32_t* __restrict__ src, int nb, unsigned int* __restrict__ cnt,
                               int32_t* __restrict__ deg, unsigned long long* updates) {
    const int j = threadIdx.x;
    if (j < nb) deg[src[j]] = (int32_t)cnt[j] - 1;
    if (j < kSweepSrc) cnt[j] = 0u;
    if (j == 0) atomicAdd(updates, (unsigned long long)nb);
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

int64_t hdeg2_sources_from_bin(const Graph& g, int bin) {
    int64_t c = 0;
    for (int b = bin < 0 ? 0 : bin; b < kOrderBins; ++b) c += g.order2_hist[b];
    return c;
}

// The sweep's per-graph arrays: m1 (zeroed), the rows longer than kSweepHead
// and their tail pieces, the counters.
static int ensure_sweep(Graph& g, cudaStream_t s) {
    if (g.sw_m1) return KH_OK;
    const size_t n = (size_t)(g.n > 0 ? g.n : 1);
    std::vector<int64_t> rp((size_t)g.n + 1);
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(rp.data(), g.rowptr, sizeof(int64_t) * rp.size(),
                                       cudaMemcpyDeviceToHost, s));
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));
    std::vector<int32_t> hpos(n, -1), hnode, piece_h, piece_off;
    for (int64_t x = 0; x < g.n; ++x) {
        const int64_t d = rp[(size_t)x + 1] - rp[(size_t)x];
        if (d <= kSweepHead) continue;
        const int h = (int)hnode.size();
        hpos[(size_t)x] = h;
        hnode.push_back((int32_t)x);
        for (int64_t off = kSweepHead; off < d; off += kSweepPiece) {
            piece_h.push_back(h);
            piece_off.push_back((int32_t)off);
        }
    }
    const size_t nh = hnode.size() > 0 ? hnode.size() : 1;
    const size_t np = piece_h.size() > 0 ? piece_h.size() : 1;
    int rc;
    const size_t fw = ((n + 127) / 128 + 3) & ~(size_t)3;  // filter words, a multiple of 4
    if ((rc = alloc_bytes(g.ctx, (void**)&g.sw_m1, 16 * n, "sweep source bits")) ||
        (rc = alloc_bytes(g.ctx, (void**)&g.sw_filter, 4 * fw, "sweep filter")) ||
        (rc = alloc_bytes(g.ctx, (void**)&g.sw_hpos, 4 * n, "sweep row index")) ||
        (rc = alloc_bytes(g.ctx, (void**)&g.sw_hnode, 4 * nh, "sweep long rows")) ||
        (rc = alloc_bytes(g.ctx, (void**)&g.sw_bh, 16 * nh, "sweep tail words")) ||
        (rc = alloc_bytes(g.ctx, (void**)&g.sw_piece_h, 4 * np, "sweep pieces")) ||
        (rc = alloc_bytes(g.ctx, (void**)&g.sw_piece_off, 4 * np, "sweep pieces")) ||
        (rc = alloc_bytes(g.ctx, (void**)&g.sw_cnt, 4 * kSweepSrc, "sweep counts"))) {
        cudaFree(g.sw_m1); cudaFree(g.sw_filter); cudaFree(g.sw_hpos); cudaFree(g.sw_hnode); cudaFree(g.sw_bh);
        cudaFree(g.sw_piece_h); cudaFree(g.sw_piece_off); cudaFree(g.sw_cnt);
        g.sw_m1 = nullptr; g.sw_filter = nullptr; g.sw_hpos = nullptr; g.sw_hnode = nullptr; g.sw_bh = nullptr;
        g.sw_piece_h = nullptr; g.sw_piece_off = nullptr; g.sw_cnt = nullptr;
        return rc;
    }
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.sw_m1, 0, 16 * n, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.sw_filter, 0, 4 * fw, s));
    KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.sw_cnt, 0, 4 * kSweepSrc, s));
    KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(g.sw_hpos, hpos.data(), 4 * n, cudaMemcpyHostToDevice, s));
    if (!hnode.empty()) {
        KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(g.sw_hnode, hnode.data(), 4 * hnode.size(),
                                           cudaMemcpyHostToDevice, s));
        KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(g.sw_piece_h, piece_h.data(), 4 * piece_h.size(),
                                           cudaMemcpyHostToDevice, s));
        KH_CUDA_TRY(g.ctx, cudaMemcpyAsync(g.sw_piece_off, piece_off.data(), 4 * piece_off.size(),
                                           cudaMemcpyHostToDevice, s));
    }
    KH_CUDA_TRY(g.ctx, cudaStreamSynchronize(s));  // host vectors go out of scope
    g.sw_nheavy = (int64_t)hnode.size();
    g.sw_npieces = (int64_t)piece_h.size();
    return KH_OK;
}

int run_sweeps(Graph& g, int32_t* deg, const int32_t* src, int64_t count, cudaStream_t s) {
    if (count <= 0) return KH_OK;
    int rc = ensure_sweep(g, s);
    if (rc) return rc;
    // the filter in shared memory while it fits (n up to 7.2M nodes)
    const size_t n1 = (size_t)(g.n > 0 ? g.n : 1);
    const int fwords = (int)(((n1 + 127) / 128 + 3) & ~(size_t)3);
    const size_t fsm = (size_t)fwords * 4;
    const int use_filter = fsm <= (size_t)kSmem2Max ? 1 : 0;
    const size_t dyn = use_filter ? fsm : 0;
    KH_CUDA_TRY(g.ctx, cudaFuncSetAttribute(k_sweep_count, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kSmem2Max));
    int per_sm = 0;
    KH_CUDA_TRY(g.ctx, cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_sweep_count, 1024, dyn));
    if (per_sm < 1) return set_error(g.ctx, KH_EINVAL, "sweep kernel does not fit on an SM");
    const int cgrid = g.ctx->sm_count * per_sm;
    int64_t tgrid = (g.sw_npieces + 7) / 8;
    if (tgrid > (int64_t)g.ctx->sm_count * 8) tgrid = (int64_t)g.ctx->sm_count * 8;
    if (tgrid < 1) tgrid = 1;
    prof_begin(g, kProfBfs, s);
    int64_t sweeps = 0;
    for (int64_t b0 = 0; b0 < count; b0 += kSweepSrc, ++sweeps) {
        const int nb = (int)(count - b0 < kSweepSrc ? count - b0 : kSweepSrc);
        const int sgrid = nb;
        k_sweep_scatter<<<sgrid, 256, 0, s>>>(g.rowptr, g.col, src + b0, nb, g.sw_m1, g.sw_filter, 0,
                                              &g.state->bytes[kProfBfs]);
        if (g.sw_npieces > 0) {
            KH_CUDA_TRY(g.ctx, cudaMemsetAsync(g.sw_bh, 0, 16 * (size_t)g.sw_nheavy, s));
            k_sweep_tails<<<(int)tgrid, 256, 0, s>>>(g.rowptr, g.col, g.sw_hnode, g.sw_piece_h,
                                                     g.sw_piece_off, g.sw_npieces,
                                                     reinterpret_cast<const uint4*>(g.sw_m1), g.sw_filter,
                                                     g.sw_bh);
        }
        k_sweep_count<<<cgrid, 1024, dyn, s>>>(g.rowptr, g.col, g.n, reinterpret_cast<const uint4*>(g.sw_m1),
                                               g.sw_filter, use_filter, fwords, g.sw_hpos,
                                               reinterpret_cast<const uint4*>(g.sw_bh), g.sw_cnt);
        k_sweep_finish<<<1, kSweepSrc, 0, s>>>(src + b0, nb, g.sw_cnt, deg, &g.state->updates);
        k_sweep_scatter<<<sgrid, 256, 0, s>>>(g.rowptr, g.col, src + b0, nb, g.sw_m1, g.sw_filter, 1,
                                              nullptr);
    }
    count_launch(g, sweeps * (g.sw_npieces > 0 ? 5 : 4));
    prof_end(g, kProfBfs, s);
    KH_CUDA_TRY(g.ctx, cudaGetLastError());
    return KH_OK;
}

int launch_hdeg2_slice(Graph& g, int32_t* deg, int32_t* cnt, int jlo, int nj, cudaStream_t s,
                       int slices, int threads, const int32_t* order, int64_t nsrc, bool init) {
    if (g.n == 0) return KH_OK;
    const int64_t width = hdeg2_width(g.n, slices);
    const size_t dyn = hdeg2_smem(width);
    if (dyn > (size_t)kSmem2Max) return set_error(g.ctx, KH_EINVAL, "slice too wide for shared memory");
    void (*kern)(Slice2Args) = cnt ? k_hdeg2_slice<true> : k_hdeg2_slice<false>;
    KH_CUDA_TRY(g.ctx, cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                            (int)kSmem2Max));
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
