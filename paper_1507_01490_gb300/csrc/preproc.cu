// Preprocessing kernels (Algorithm 1's PreProcessing and the degree order):
//   * CSR validation and 64->32-bit offset narrowing,
//   * connected components for r(v) on undirected graphs (Section 2.2),
//   * the processing order: decreasing degree, ties by increasing id
//     (Section 2.1), as a stable LSD radix sort on the degree key,
//   * scan and radix-sort primitives also used by the SCC pass.
#include <cstdio>
#include <cuda_runtime.h>

#include "internal.h"

namespace bcm {

static inline int blocks_for(size_t n, int threads, int cap = 152 * 32) {
    size_t b = (n + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > (size_t)cap) b = cap;
    return (int)b;
}

// ------------------------------------------------------------ validation
__global__ void k_validate(const uint64_t* rp, const uint32_t* col, uint32_t n, uint64_t m, int* err) {
    size_t tid = blockIdx.x * (size_t)blockDim.x + threadIdx.x;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    if (tid == 0 && (rp[0] != 0 || rp[n] != m)) atomicOr(err, DEV_ERR_INVALID_CSR);
    for (size_t i = tid; i < n; i += stride)
        if (rp[i] > rp[i + 1]) atomicOr(err, DEV_ERR_INVALID_CSR);
    for (size_t e = tid; e < m; e += stride)
        if (col[e] >= n) atomicOr(err, DEV_ERR_INVALID_CSR);
}

// *not_simple |= 1 if some row is not strictly increasing or holds its own
// vertex (a repeated arc or a self-loop).  Two balanced passes: per row,
// mark where it starts and look for its own vertex by binary search (valid
// when the row is sorted, which the second pass checks); per arc, compare it
// with the arc before unless a row starts there.
__global__ void k_simple_rows(const uint32_t* rp, const uint32_t* col, uint32_t n, uint32_t* starts,
                              int* not_simple) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += stride) {
        uint32_t lo = rp[u], hi = rp[u + 1];
        if (lo == hi) continue;
        atomicOr(&starts[lo >> 5], 1u << (lo & 31));
        while (lo < hi) {
            const uint32_t mid = lo + (hi - lo) / 2;
            const uint32_t c = col[mid];
            if (c == u) { atomicOr(not_simple, 1); break; }
            if (c < u) lo = mid + 1; else hi = mid;
        }
    }
}

__global__ void k_simple_arcs(const uint32_t* col, uint64_t m, const uint32_t* starts, int* not_simple) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    bool bad = false;
    for (size_t e = blockIdx.x * (size_t)blockDim.x + threadIdx.x + 1; e < m; e += stride)
        bad = bad || (!((starts[e >> 5] >> (e & 31)) & 1u) && col[e - 1] >= col[e]);
    if (__any_sync(0xffffffffu, bad) && (threadIdx.x & 31) == 0) atomicOr(not_simple, 1);
}

size_t simple_check_scratch_bytes(uint64_t m) { return (((size_t)m + 31) / 32 * 4 + 255) & ~(size_t)255; }

int launch_simple_check(const uint32_t* rp32, const uint32_t* col, uint32_t n, uint64_t m, int* not_simple,
                        void* scratch, cudaStream_t s) {
    if (n == 0 || m == 0) return 0;
    uint32_t* starts = (uint32_t*)scratch;
    cudaMemsetAsync(starts, 0, ((size_t)m + 31) / 32 * 4, s);
    k_simple_rows<<<blocks_for(n, 256), 256, 0, s>>>(rp32, col, n, starts, not_simple);
    k_simple_arcs<<<blocks_for(m, 256), 256, 0, s>>>(col, m, starts, not_simple);
    note_launch(2);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_validate(const uint64_t* rp64, const uint32_t* col, uint32_t n, uint64_t m, int* err,
                    cudaStream_t s) {
    k_validate<<<blocks_for(m > n ? m : n, 256), 256, 0, s>>>(rp64, col, n, m, err);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__global__ void k_narrow(const uint64_t* rp64, uint32_t* rp32, size_t cnt) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < cnt; i += stride)
        rp32[i] = (uint32_t)rp64[i];
}

int launch_narrow_offsets(const uint64_t* rp64, uint32_t* rp32, uint32_t n, cudaStream_t s) {
    k_narrow<<<blocks_for((size_t)n + 1, 256), 256, 0, s>>>(rp64, rp32, (size_t)n + 1);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------- connected components
// Union-find with roots hooked under smaller roots, so every parent pointer
// points to a smaller id and each component's root is its smallest vertex.
__device__ __forceinline__ uint32_t uf_find(uint32_t* parent, uint32_t x) {
    for (;;) {
        // vertex 0 is a root for good (nothing is smaller): its entry, where
        // most walks would end, is never read
        if (x == 0) return 0;
        uint32_t p = vload(&parent[x]);
        if (p == x || p == 0) return p;
        uint32_t gp = vload(&parent[p]);
        if (gp != p) vstore(&parent[x], gp);   // path halving; gp is still an ancestor
        x = gp;
    }
}

__global__ void k_uf_init(uint32_t* parent, uint32_t* size, uint32_t n) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        parent[v] = (uint32_t)v;
        size[v] = 0;
    }
}

__device__ __forceinline__ void uf_union(uint32_t* parent, uint32_t a, uint32_t b, int* err) {
    for (int it = 0;; ++it) {
        if (it > (1 << 20)) { atomicOr(err, DEV_ERR_RETRY_LIMIT); return; }
        a = uf_find(parent, a);
        b = uf_find(parent, b);
        if (a == b) return;
        uint32_t hi = a > b ? a : b, lo = a > b ? b : a;
        if (atomicCAS(&parent[hi], hi, lo) == hi) return;
    }
}

// Components after Afforest (Sutton, Ben-Nun, Barak, IPDPS 2018): link every
// vertex to its first kLink neighbours, compress, take the most frequent
// component of a sample as the giant one, then link the remaining arcs only
// of vertices outside it.  For a symmetric arc set a skipped arc (u,w) of a
// giant-component u is either linked from w's side or joins two vertices
// already in the giant set, so the components are exact.
constexpr uint32_t kLink = 2;
// A sampled arc to a vertex of more than kHubDeg arcs is not linked while
// sampling but with the other arcs afterwards: thousands of rows sample the
// same hub, and their atomics and walks on its entry serialise; once the
// giant component exists the hub points straight at its root.
#ifndef BCM_CC_HUB_DEG
#define BCM_CC_HUB_DEG 64
#endif
constexpr uint32_t kHubDeg = BCM_CC_HUB_DEG;   // 0: every sampled arc is linked while sampling

__device__ __forceinline__ bool sampled(const uint32_t* rp, uint32_t w, uint32_t pos) {
    return pos < kLink && (kHubDeg == 0 || rp[w + 1] - rp[w] <= kHubDeg);
}

__global__ void k_uf_link_first(const uint32_t* rp, const uint32_t* col, uint32_t n, uint32_t* parent, int* err) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t u = blockIdx.x * (size_t)blockDim.x + threadIdx.x; u < n; u += stride) {
        uint32_t beg = rp[u], end = rp[u + 1];
        for (uint32_t e = beg; e < end && e < beg + kLink; ++e)
            if (sampled(rp, col[e], e - beg)) uf_union(parent, (uint32_t)u, col[e], err);
    }
}

__global__ void k_uf_flatten(uint32_t* parent, uint32_t n) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += stride)
        parent[v] = uf_find(parent, (uint32_t)v);
}

// The giant component after sampling, as Afforest finds it: the most
// frequent root among 1024 vertices spread evenly over the ids (one block
// of 1024 threads: sort the roots in shared memory, take the longest run).
// best gets (run length << 32 | ~root), the form k_uf_link_rest reads.
__global__ void __launch_bounds__(1024) k_uf_giant_sample(const uint32_t* parent, uint32_t n,
                                                           unsigned long long* best) {
    __shared__ uint32_t s_r[1024];
    __shared__ unsigned long long s_best;
    const uint32_t i = threadIdx.x;
    if (i == 0) s_best = 0;
    s_r[i] = vload(&parent[(uint32_t)(((unsigned long long)i * n) >> 10)]);   // flattened: the root
    __syncthreads();
    for (uint32_t k = 2; k <= 1024; k <<= 1) {          // bitonic sort, ascending
        for (uint32_t j = k >> 1; j > 0; j >>= 1) {
            const uint32_t l = i ^ j;
            if (l > i) {
                const uint32_t a = s_r[i], b = s_r[l];
                if (((i & k) == 0) == (a > b)) { s_r[i] = b; s_r[l] = a; }
            }
            __syncthreads();
        }
    }
    if (i == 0 || s_r[i] != s_r[i - 1]) {               // a run starts here
        uint32_t e = i + 1;
        while (e < 1024 && s_r[e] == s_r[i]) ++e;
        atomicMax(&s_best, ((unsigned long long)(e - i) << 32) | (0xffffffffull - s_r[i]));
    }
    __syncthreads();
    if (i == 0) *best = s_best;
}

// One warp per vertex outside the giant component: link its arcs that
// sampling left (beyond the first kLink, and the sampled ones to hubs).
__global__ void k_uf_link_rest(const uint32_t* rp, const uint32_t* col, uint32_t n, uint32_t* parent,
                               const unsigned long long* best, int* err) {
    // the giant component's root (the sampled one, or the component of
    // the vertex best names), found once per block (every thread walking to
    // it would read the same words a million times)
    __shared__ uint32_t s_giant;
    if (threadIdx.x == 0) s_giant = uf_find(parent, 0xffffffffu - (uint32_t)(*best & 0xffffffffull));
    __syncthreads();
    const uint32_t giant = s_giant;
    const uint32_t lane = threadIdx.x & 31;
    size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
    size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    for (size_t u = warp; u < n; u += nwarps) {
        uint32_t beg = rp[u], end = rp[u + 1];
        if (kHubDeg == 0 && end - beg <= kLink) continue;
        // after k_uf_flatten every vertex points at its root: one load tells
        // a giant vertex (roots only change by later links, which keep a
        // giant vertex in the giant component)
        if (vload(&parent[u]) == giant || uf_find(parent, (uint32_t)u) == giant) continue;
        for (uint32_t e = beg + lane; e < end; e += 32)
            if (!sampled(rp, col[e], e - beg)) uf_union(parent, (uint32_t)u, col[e], err);
    }
}

// Final roots and component sizes; lanes holding the same root add their
// count with one atomic (most vertices share the giant component's root).
__global__ void k_uf_compress_count(uint32_t* parent, uint32_t* size, uint32_t n) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t v0 = (blockIdx.x * (size_t)blockDim.x) + (threadIdx.x & ~31u); v0 < n; v0 += stride) {
        size_t v = v0 + (threadIdx.x & 31);
        uint32_t r = v < n ? uf_find(parent, (uint32_t)v) : 0xffffffffu;
        uint32_t peers = __match_any_sync(0xffffffffu, r);
        if (r != 0xffffffffu && (threadIdx.x & 31) == (uint32_t)(__ffs(peers) - 1))
            atomicAdd(&size[r], (uint32_t)__popc(peers));
    }
}

// ------------------------------------------------------------------ scan
// Exclusive scan in tiles of SCAN_TILE: tile sums, a one-block scan of the
// sums (chunked, any length), then each tile rescans with its offset.
constexpr int SCAN_THREADS = 256;
constexpr int SCAN_ITEMS = 8;
constexpr int SCAN_TILE = SCAN_THREADS * SCAN_ITEMS;

__global__ void k_uf_reach(uint32_t* parent, const uint32_t* size, uint32_t n, uint32_t* xlo, uint32_t* xhi) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t v0 = (blockIdx.x * (size_t)blockDim.x) + (threadIdx.x & ~31u); v0 < n; v0 += stride) {
        const size_t v = v0 + (threadIdx.x & 31);
        const uint32_t r = v < n ? uf_find(parent, (uint32_t)v) : 0xffffffffu;
        // lanes of one component read its size once (most share the giant one)
        const uint32_t peers = __match_any_sync(0xffffffffu, r);
        const int first = __ffs(peers) - 1;
        uint32_t sz = 0;
        if (r != 0xffffffffu && (threadIdx.x & 31) == (uint32_t)first) sz = size[r];
        sz = __shfl_sync(0xffffffffu, sz, first);
        if (v < n) {
            parent[v] = r;
            xlo[v] = sz;
            xhi[v] = sz;
        }
    }
}

int launch_cc_reach(const uint32_t* rp, const uint32_t* col, uint32_t n, uint32_t* parent,
                    uint32_t* size, uint32_t* xlo, uint32_t* xhi, int* err, cudaStream_t s) {
    if (n == 0) return 0;
    int b = blocks_for(n, 256);
    unsigned long long* best = (unsigned long long*)(size + (((size_t)n + 63) & ~(size_t)63));
    cudaMemsetAsync(best, 0, sizeof(unsigned long long), s);
    k_uf_init<<<b, 256, 0, s>>>(parent, size, n);
    k_uf_link_first<<<b, 256, 0, s>>>(rp, col, n, parent, err);
    k_uf_flatten<<<b, 256, 0, s>>>(parent, n);
    k_uf_giant_sample<<<1, 1024, 0, s>>>(parent, n, best);
    k_uf_link_rest<<<blocks_for((size_t)n * 32, 256), 256, 0, s>>>(rp, col, n, parent, best, err);
    k_uf_compress_count<<<b, 256, 0, s>>>(parent, size, n);
    k_uf_reach<<<b, 256, 0, s>>>(parent, size, n, xlo, xhi);
    note_launch(7);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

__device__ __forceinline__ uint32_t block_exclusive_scan(uint32_t v, uint32_t* total) {
    __shared__ uint32_t s_warp[32];
    __shared__ uint32_t s_total;
    const uint32_t lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    uint32_t incl = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (uint32_t)o) incl += t;
    }
    if (lane == 31) s_warp[wid] = incl;
    __syncthreads();
    if (wid == 0) {
        uint32_t nw = blockDim.x >> 5;
        uint32_t x = lane < nw ? s_warp[lane] : 0;
        uint32_t xi = x;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t t = __shfl_up_sync(0xffffffffu, xi, o);
            if (lane >= (uint32_t)o) xi += t;
        }
        if (lane < nw) s_warp[lane] = xi - x;
        if (lane == nw - 1) s_total = xi;
    }
    __syncthreads();
    uint32_t res = s_warp[wid] + incl - v;
    *total = s_total;
    __syncthreads();
    return res;
}

__global__ void k_scan_tiles(const uint32_t* in, size_t count, uint32_t* tile_sum) {
    size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
    uint32_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i)
        if (base + i < count) s += in[base + i];
    uint32_t tot;
    block_exclusive_scan(s, &tot);
    if (threadIdx.x == 0) tile_sum[blockIdx.x] = tot;
}

__global__ void k_scan_sums(uint32_t* sums, size_t nt, uint32_t* total) {
    __shared__ uint32_t s_carry;
    if (threadIdx.x == 0) s_carry = 0;
    __syncthreads();
    for (size_t c = 0; c < nt; c += SCAN_TILE) {
        size_t base = c + (size_t)threadIdx.x * SCAN_ITEMS;
        uint32_t v[SCAN_ITEMS], s = 0;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            v[i] = (base + i < nt) ? sums[base + i] : 0;
            s += v[i];
        }
        uint32_t tot;
        uint32_t off = block_exclusive_scan(s, &tot) + s_carry;
#pragma unroll
        for (int i = 0; i < SCAN_ITEMS; ++i) {
            if (base + i < nt) sums[base + i] = off;
            off += v[i];
        }
        __syncthreads();
        if (threadIdx.x == 0) s_carry += tot;
        __syncthreads();
    }
    if (threadIdx.x == 0 && total) *total = s_carry;
}

__global__ void k_scan_apply(const uint32_t* in, uint32_t* out, size_t count, const uint32_t* tile_off) {
    size_t base = (size_t)blockIdx.x * SCAN_TILE + (size_t)threadIdx.x * SCAN_ITEMS;
    uint32_t v[SCAN_ITEMS], s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        v[i] = (base + i < count) ? in[base + i] : 0;
        s += v[i];
    }
    uint32_t tot;
    uint32_t off = block_exclusive_scan(s, &tot) + tile_off[blockIdx.x];
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; ++i) {
        if (base + i < count) out[base + i] = off;
        off += v[i];
    }
}

size_t scan_scratch_bytes(size_t count) {
    size_t nt = (count + SCAN_TILE - 1) / SCAN_TILE;
    return ((nt + 1) * sizeof(uint32_t) + 255) & ~(size_t)255;
}

int exclusive_scan_u32(const uint32_t* in, uint32_t* out, size_t count, uint32_t* total_dev,
                       void* scratch, cudaStream_t s) {
    if (count == 0) {
        if (total_dev) cudaMemsetAsync(total_dev, 0, sizeof(uint32_t), s);
        return cudaGetLastError() == cudaSuccess ? 0 : -1;
    }
    size_t nt = (count + SCAN_TILE - 1) / SCAN_TILE;
    uint32_t* sums = (uint32_t*)scratch;
    k_scan_tiles<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, count, sums);
    k_scan_sums<<<1, SCAN_THREADS, 0, s>>>(sums, nt, total_dev);
    k_scan_apply<<<(unsigned)nt, SCAN_THREADS, 0, s>>>(in, out, count, sums);
    note_launch(3);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// ------------------------------------------------------------ radix sort
// Stable LSD radix sort, 8-bit digits, tiles of RADIX_TILE elements.  Per
// pass: per-tile digit histograms (digit-major), one exclusive scan, then a
// stable scatter in which element order inside a tile is (round, warp, lane).
constexpr int RADIX_THREADS = 256;
constexpr int RADIX_ITEMS = 8;
constexpr int RADIX_TILE = RADIX_THREADS * RADIX_ITEMS;

template <typename K>
__global__ void k_radix_hist(const K* keys, size_t count, int shift, uint32_t* hist, uint32_t ntiles) {
    __shared__ uint32_t h[256];
    h[threadIdx.x] = 0;
    __syncthreads();
    size_t base = (size_t)blockIdx.x * RADIX_TILE;
#pragma unroll
    for (int r = 0; r < RADIX_ITEMS; ++r) {
        size_t i = base + (size_t)r * RADIX_THREADS + threadIdx.x;
        if (i < count) atomicAdd(&h[(uint32_t)(keys[i] >> shift) & 255u], 1u);
    }
    __syncthreads();
    hist[(size_t)threadIdx.x * ntiles + blockIdx.x] = h[threadIdx.x];
}

template <typename K, bool HAS_V>
__global__ void k_radix_scatter(const K* kin, const uint32_t* vin, K* kout, uint32_t* vout, size_t count,
                                int shift, const uint32_t* offs, uint32_t ntiles) {
    __shared__ uint32_t s_run[256];
    __shared__ uint32_t s_w[RADIX_THREADS / 32][256];
    const uint32_t wid = threadIdx.x >> 5;
    s_run[threadIdx.x] = offs[(size_t)threadIdx.x * ntiles + blockIdx.x];
    size_t base = (size_t)blockIdx.x * RADIX_TILE;
    for (int r = 0; r < RADIX_ITEMS; ++r) {
        for (int w = 0; w < RADIX_THREADS / 32; ++w) s_w[w][threadIdx.x] = 0;
        __syncthreads();
        size_t i = base + (size_t)r * RADIX_THREADS + threadIdx.x;
        bool valid = i < count;
        K key = valid ? kin[i] : (K)0;
        uint32_t val = (HAS_V && valid) ? vin[i] : 0u;
        uint32_t dg = valid ? ((uint32_t)(key >> shift) & 255u) : 256u;
        uint32_t peers = __match_any_sync(0xffffffffu, dg);
        uint32_t rank = __popc(peers & lanemask_lt());
        if (valid && rank == 0) s_w[wid][dg] = __popc(peers);
        __syncthreads();
        {   // per digit: prefix over warps, then advance the running offset
            uint32_t d = threadIdx.x, run = s_run[d];
            for (int w = 0; w < RADIX_THREADS / 32; ++w) {
                uint32_t c = s_w[w][d];
                s_w[w][d] = run;
                run += c;
            }
            s_run[d] = run;
        }
        __syncthreads();
        if (valid) {
            uint32_t pos = s_w[wid][dg] + rank;
            kout[pos] = key;
            if (HAS_V) vout[pos] = val;
        }
        __syncthreads();
    }
}

size_t radix_scratch_bytes(size_t count) {
    size_t nt = (count + RADIX_TILE - 1) / RADIX_TILE;
    if (nt == 0) nt = 1;
    return 256 * nt * sizeof(uint32_t) + scan_scratch_bytes(256 * nt) + 256;
}

template <typename K, bool HAS_V>
static int radix_sort_impl(K* keys, uint32_t* vals, K* ktmp, uint32_t* vtmp, size_t count, int bits,
                           void* scratch, cudaStream_t s, bool* in_tmp) {
    *in_tmp = false;
    if (count <= 1 || bits <= 0) return 0;
    uint32_t ntiles = (uint32_t)((count + RADIX_TILE - 1) / RADIX_TILE);
    uint32_t* hist = (uint32_t*)scratch;
    void* scan_scr = (char*)scratch + ((256 * (size_t)ntiles * sizeof(uint32_t) + 255) & ~(size_t)255);
    K* ka = keys; K* kb = ktmp;
    uint32_t* va = vals; uint32_t* vb = vtmp;
    for (int shift = 0; shift < bits; shift += 8) {
        k_radix_hist<K><<<ntiles, RADIX_THREADS, 0, s>>>(ka, count, shift, hist, ntiles);
        note_launch();
        if (exclusive_scan_u32(hist, hist, 256 * (size_t)ntiles, nullptr, scan_scr, s)) return -1;
        k_radix_scatter<K, HAS_V><<<ntiles, RADIX_THREADS, 0, s>>>(ka, va, kb, vb, count, shift, hist, ntiles);
        note_launch();
        K* t = ka; ka = kb; kb = t;
        uint32_t* tv = va; va = vb; vb = tv;
        *in_tmp = !*in_tmp;
    }
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int radix_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                         size_t count, int bits, void* scratch, cudaStream_t s, bool* result_in_tmp) {
    return radix_sort_impl<uint32_t, true>(keys, vals, keys_tmp, vals_tmp, count, bits, scratch, s,
                                           result_in_tmp);
}

int radix_sort_u64(uint64_t* keys, uint64_t* keys_tmp, size_t count, int bits, void* scratch,
                   cudaStream_t s, bool* result_in_tmp) {
    return radix_sort_impl<uint64_t, false>((uint64_t*)keys, nullptr, (uint64_t*)keys_tmp, nullptr,
                                            count, bits, scratch, s, result_in_tmp);
}

// ---------------------------------------------------------- degree order
__global__ void k_max_degree(const uint32_t* rp, uint32_t n, uint32_t* out) {
    uint32_t best = 0;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        uint32_t d = rp[v + 1] - rp[v];
        best = d > best ? d : best;
    }
    best = __reduce_max_sync(0xffffffffu, best);
    // then across the block's warps: one atomic per block on the one word
    __shared__ uint32_t s_b[32];
    if ((threadIdx.x & 31) == 0) s_b[threadIdx.x >> 5] = best;
    __syncthreads();
    if (threadIdx.x == 0) {
        for (unsigned w = 1; w < blockDim.x / 32; ++w) best = s_b[w] > best ? s_b[w] : best;
        atomicMax(out, best);
    }
}

__global__ void k_degree_keys(const uint32_t* rp, uint32_t n, const uint32_t* maxdeg, uint32_t* keys,
                              uint32_t* vals) {
    uint32_t md = *maxdeg;
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += stride) {
        keys[v] = md - (rp[v + 1] - rp[v]);   // larger degree -> smaller key
        vals[v] = (uint32_t)v;                 // ids ascending: ties keep id order
    }
}

size_t degree_order_scratch_bytes(uint32_t n) {
    size_t a = ((size_t)n * sizeof(uint32_t) + 255) & ~(size_t)255;
    return 3 * a + radix_scratch_bytes(n) + 256;
}

// order[] = vertices by (degree desc, id asc); degree = CSR row length.
int launch_degree_order(const uint32_t* rp, uint32_t n, uint32_t* order, void* scratch,
                        size_t scratch_bytes, cudaStream_t s, uint32_t* max_degree) {
    if (n == 0) return 0;
    if (scratch_bytes < degree_order_scratch_bytes(n)) return -1;
    size_t a = ((size_t)n * sizeof(uint32_t) + 255) & ~(size_t)255;
    char* p = (char*)scratch;
    uint32_t* keys = (uint32_t*)p;
    uint32_t* ktmp = (uint32_t*)(p + a);
    uint32_t* vtmp = (uint32_t*)(p + 2 * a);
    uint32_t* d_max = (uint32_t*)(p + 3 * a);
    void* rscr = p + 3 * a + 256;
    cudaMemsetAsync(d_max, 0, sizeof(uint32_t), s);
    k_max_degree<<<blocks_for(n, 256, 152 * 4), 256, 0, s>>>(rp, n, d_max);
    k_degree_keys<<<blocks_for(n, 256), 256, 0, s>>>(rp, n, d_max, keys, order);
    note_launch(2);
    uint32_t maxdeg = 0;
    if (cudaMemcpyAsync(&maxdeg, d_max, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    if (max_degree) *max_degree = maxdeg;
    int bits = 0;
    while (bits < 32 && (maxdeg >> bits)) ++bits;
    bool in_tmp = false;
    if (radix_sort_pairs_u32(keys, order, ktmp, vtmp, n, bits, rscr, s, &in_tmp)) return -1;
    if (in_tmp) cudaMemcpyAsync(order, vtmp, (size_t)n * sizeof(uint32_t), cudaMemcpyDeviceToDevice, s);
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace bcm
