// The C-ABI of include/bcm.h: graph handles, preprocessing, the wave
// kernels' workspace and launch sequence, and error reporting.
#include <algorithm>
#include <array>
#include <atomic>
#include <chrono>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <vector>

#include <cuda_runtime.h>

#include "bcm.h"
#include "internal.h"

namespace bcm {

static std::atomic<uint64_t> g_launches{0};
void note_launch(int count) { g_launches.fetch_add((uint64_t)count, std::memory_order_relaxed); }

static thread_local std::string t_err;

void set_error_message(const char* msg) { t_err = msg; }

static bcm_status fail(bcm_status st, const char* fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    t_err = buf;
    return st;
}

static bcm_status cuda_fail(cudaError_t e, const char* what) {
    if (e == cudaErrorMemoryAllocation) {
        cudaGetLastError();
        return fail(BCM_ERR_OOM, "%s: %s", what, cudaGetErrorString(e));
    }
    return fail(BCM_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CU(call, what)                                  \
    do {                                                \
        cudaError_t e_ = (call);                        \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

// ---------------------------------------------------------- workspaces
// The slot region of the wave kernels is large (44 n W bytes per CTA) and
// must start zeroed; every successful run leaves it zeroed again.  Clean
// regions are kept here for reuse instead of being freed and re-zeroed.
// A region is only known to be zero under the slot layout it was last used
// with (vertex count, words per vertex, CTA count): frontier lists and logs
// of one layout overlap the bit arrays of another.
struct Layout {
    uint32_t n = 0, W = 0, blocks = 0, entries = 0;   // entries: the vertex tables', or the sparse queues'
    bool sparse = false;
    bool operator==(const Layout& o) const {
        return n == o.n && W == o.W && blocks == o.blocks && entries == o.entries && sparse == o.sparse;
    }
};
struct Region { int dev; void* ptr; size_t bytes; Layout layout; };
static std::mutex g_region_mu;
static std::vector<Region> g_regions;
static size_t g_cached_bytes = 0;
static const size_t kCacheCap = 96ull << 30;   // clean regions kept for reuse, at most

static void buf_drop_cache(int dev);

static void regions_drop_cache(int dev) {
    std::vector<Region> drop;
    {
        std::lock_guard<std::mutex> lk(g_region_mu);
        for (size_t i = 0; i < g_regions.size();)
            if (g_regions[i].dev == dev) {
                drop.push_back(g_regions[i]);
                g_cached_bytes -= g_regions[i].bytes;
                g_regions.erase(g_regions.begin() + i);
            } else {
                ++i;
            }
    }
    for (auto& r : drop) cudaFree(r.ptr);
}

static bcm_status region_acquire(size_t bytes, const Layout& lay, cudaStream_t s, Region* out) {
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(g_region_mu);
        int best = -1;
        for (size_t i = 0; i < g_regions.size(); ++i) {
            const Region& r = g_regions[i];
            if (r.dev != dev || r.bytes < bytes) continue;
            // a much larger region stays for a run that needs it: a small run
            // holding it would hide that memory from the caller's accounting
            // (bcm_workspace_bytes)
            if (r.bytes > 2 * bytes + (64ull << 20)) continue;
            // prefer a region already zero under this layout, then the smallest
            if (best < 0 || (r.layout == lay && !(g_regions[best].layout == lay)) ||
                ((r.layout == lay) == (g_regions[best].layout == lay) && r.bytes < g_regions[best].bytes))
                best = (int)i;
        }
        if (best >= 0) {
            *out = g_regions[best];
            g_cached_bytes -= g_regions[best].bytes;
            g_regions.erase(g_regions.begin() + best);
        }
    }
    if (out->ptr) {
        if (!(out->layout == lay)) {
            // only the layout's own bytes must be zero; the rest is unused under it
            CU(cudaMemsetAsync(out->ptr, 0, bytes, s), "workspace clear");
            out->layout = lay;
        }
        return BCM_OK;
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        // drop the cached regions and buffers of this device and retry once
        cudaGetLastError();
        regions_drop_cache(dev);
        buf_drop_cache(dev);
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return cuda_fail(e, "workspace allocation");
    }
    CU(cudaMemsetAsync(p, 0, bytes, s), "workspace clear");
    *out = Region{dev, p, bytes, lay};
    return BCM_OK;
}

static void region_release(Region& r, bool clean) {
    if (!r.ptr) return;
    bool kept = false;
    if (clean) {
        std::lock_guard<std::mutex> lk(g_region_mu);
        if (g_cached_bytes + r.bytes <= kCacheCap) {
            g_regions.push_back(r);
            g_cached_bytes += r.bytes;
            kept = true;
        }
    }
    if (!kept) cudaFree(r.ptr);
    r.ptr = nullptr;
    r.bytes = 0;
    r.layout = Layout{};
}

// ------------------------------------------------------------ buffers
// Device buffers of graphs and runs (CSR copies, preprocessing arrays and
// scratch, source lists, outputs) come from a cache of freed buffers: a
// caller that creates and releases a graph per request (or per benchmark
// step) then pays no cudaMalloc / cudaFree -- the latter synchronises the
// device.  A cached buffer is reused for a request of at least half its size.
struct Buf { int dev; void* ptr; size_t bytes; };
static std::mutex g_buf_mu;
static std::vector<Buf> g_bufs;                 // free
static std::vector<Buf> g_live;                 // handed out
static size_t g_buf_cached = 0;
static const size_t kBufCap = 16ull << 30;

static void buf_drop_cache(int dev) {
    std::vector<Buf> drop;
    {
        std::lock_guard<std::mutex> lk(g_buf_mu);
        for (size_t i = 0; i < g_bufs.size();)
            if (g_bufs[i].dev == dev) {
                drop.push_back(g_bufs[i]);
                g_buf_cached -= g_bufs[i].bytes;
                g_bufs.erase(g_bufs.begin() + i);
            } else {
                ++i;
            }
    }
    for (auto& b : drop) cudaFree(b.ptr);
}

static void regions_drop_cache(int dev);

static cudaError_t buf_get(void** out, size_t bytes) {
    int dev = 0;
    cudaGetDevice(&dev);
    if (bytes == 0) bytes = 256;
    {
        std::lock_guard<std::mutex> lk(g_buf_mu);
        int best = -1;
        for (size_t i = 0; i < g_bufs.size(); ++i) {
            const Buf& b = g_bufs[i];
            if (b.dev != dev || b.bytes < bytes || b.bytes > 2 * bytes + (1u << 20)) continue;
            if (best < 0 || b.bytes < g_bufs[best].bytes) best = (int)i;
        }
        if (best >= 0) {
            Buf b = g_bufs[best];
            g_buf_cached -= b.bytes;
            g_bufs.erase(g_bufs.begin() + best);
            g_live.push_back(b);
            *out = b.ptr;
            return cudaSuccess;
        }
    }
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e != cudaSuccess) {
        cudaGetLastError();
        buf_drop_cache(dev);
        regions_drop_cache(dev);
        e = cudaMalloc(&p, bytes);
        if (e != cudaSuccess) return e;
    }
    std::lock_guard<std::mutex> lk(g_buf_mu);
    g_live.push_back(Buf{dev, p, bytes});
    *out = p;
    return cudaSuccess;
}

static void buf_put(void* p) {
    if (!p) return;
    Buf b{0, nullptr, 0};
    bool free_it = false;
    {
        std::lock_guard<std::mutex> lk(g_buf_mu);
        for (size_t i = 0; i < g_live.size(); ++i)
            if (g_live[i].ptr == p) {
                b = g_live[i];
                g_live[i] = g_live.back();
                g_live.pop_back();
                break;
            }
        if (!b.ptr) return;   // not from the pool
        if (g_buf_cached + b.bytes <= kBufCap) {
            g_bufs.push_back(b);
            g_buf_cached += b.bytes;
        } else {
            free_it = true;
        }
    }
    if (free_it) cudaFree(b.ptr);
}

template <class T>
static cudaError_t buf_get_t(T** out, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = buf_get(&p, bytes);
    *out = (T*)p;
    return e;
}

// Pinned host blocks and event sets of runs, reused across graphs.
struct HostBlock;
static std::mutex g_pool_mu;
static std::vector<void*> g_pinned_free;
struct RunRes {                 // per-graph CUDA objects, reused across graphs
    int dev;
    std::array<cudaEvent_t, 7> ev; // run timing (5), preprocessing fork and join (2)
    cudaStream_t aux;              // helper stream of preprocessing
};
static std::vector<RunRes> g_res_free;

// Small per-run state of the wave kernels (all zeroed before a run).
struct Aux {
    uint32_t topk_id[1024];
    u64 topk_f[1024];
    uint32_t topk_r[1024];
    uint32_t topk_count;
    uint32_t lock;
    uint32_t head;
    int err;
    Threshold thr;
    Threshold ext;        // key offered by bcm_topk_offer (written by the host while the run goes on)
    Threshold snap;       // the threshold all blocks of a grid-wide or plain launch cut with
    unsigned long long stats[ST_COUNT];        // per-CTA wave kernel
    unsigned long long seed_stats[ST_COUNT];   // seed wave / plain kernel
    GridBarrier bar;
    uint32_t gcnt[2 * kCntParity];
    uint32_t glist_n[2];
    uint32_t glog_n;
    uint32_t gchunk[2];
    unsigned long long garc[2];
    HeavyEntry gheavy[2048];
    uint32_t gheavy_n;
    uint32_t trace_n;
    uint32_t defer_n;     // sources handed back by per-CTA waves
    uint32_t head2;       // queue head of the grid-wide pass over them
    uint32_t surv_n;      // sources the prefilter could not stop
    uint32_t head3;       // queue head of the per-CTA waves over them
};

// Host side of a run in flight: pinned memory the run's counters are copied
// into, read once the run's last event has completed.
struct HostBlock {
    int err;
    uint32_t topk_count;
    uint32_t trace_n;
    int not_simple;            // preprocessing: the simple-graph check
    unsigned long long stats[ST_COUNT];        // per-CTA wave kernel
    unsigned long long seed_stats[ST_COUNT];   // grid-wide or plain kernel
    // bcm_topk_threshold / bcm_topk_offer staging (helper stream)
    u64 rd_seq[2];
    Threshold rd;
    u64 wr_seq[2];             // odd, then even
    Threshold wr;
};

constexpr uint32_t kTraceCap = 1u << 16;   // trace records kept per run

}  // namespace bcm

using namespace bcm;

struct bcm_graph {
    uint32_t n = 0;
    uint64_t m = 0;
    int directed = 0;
    uint32_t flags = 0;            // bcm_graph_create flags
    cudaStream_t stream = nullptr;
    int dev = 0;
    uint32_t* d_rp = nullptr;
    uint32_t* d_col = nullptr;
    uint32_t* d_order = nullptr;
    uint32_t* d_xlo = nullptr;
    uint32_t* d_xhi = nullptr;
    uint32_t* d_comp = nullptr;    // component / SCC label, smallest-member order
    uint32_t* d_rrp = nullptr;     // directed: in-arcs CSR
    uint32_t* d_rcol = nullptr;
    uint32_t n_comp = 0;
    bool labels_ready = false;     // d_comp holds labels (else component roots)
    bool simple = false;           // rows strictly increasing, no self-loops (found by preprocessing):
                                   // level 1 of every BFS is then known from degrees alone (the prefilter)
    bool preprocessed = false;
    uint32_t max_deg = 0;          // largest row length (found by preprocessing)
    Aux* d_aux = nullptr;
    uint32_t* d_plain = nullptr;   // stamps [n], two vertex queues [2n]
    unsigned long long* d_far = nullptr;   // exhaustive outputs [n]
    uint32_t* d_reach = nullptr;
    Region slots{0, nullptr, 0, Layout{}};
    int sms = 0;
    // the run started by bcm_topk_start (or a synchronous call) until finished
    struct Pending {
        bool active = false;
        bool exhaustive = false;
        bool plain = false;
        bool sparse = false;      // the per-CTA phase ran k_sparse
        uint32_t kk = 0;          // entries the top-k must hold
        uint32_t flags = 0;
        uint64_t l0 = 0;          // launch counter at the start
        double pms = 0;           // preprocessing time of this call
        std::chrono::steady_clock::time_point t0;
    } pend;
    // start, first grid pass done, per-CTA pass done, deferred grid pass done, copies done;
    // then the fork and join of preprocessing's helper stream
    cudaEvent_t ev[7] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
    cudaStream_t aux = nullptr;
    uint32_t* d_defer = nullptr;   // [n] sources deferred by per-CTA waves
    uint32_t* d_shard = nullptr;   // [n] this shard's sources, in degree order
    uint32_t* d_surv = nullptr;    // [n] sources left for the per-CTA waves by the prefilter
    HostBlock* h = nullptr;        // pinned
    unsigned long long* d_trace = nullptr;   // kTraceCap records of 4 words
    uint32_t trace_n = 0;          // records of the last finished traced run
    // threshold exchange (bcm_topk_threshold / bcm_topk_offer), guarded by xmu: they may run on
    // another thread while a run is pending
    std::mutex xmu;
    cudaEvent_t ev_x = nullptr;    // the run's state is cleared (recorded at its start)
    bool offered = false;          // the pending run was given a key
    bcm_key best{0, 0, 0, 0};      // the best key given to it
    uint64_t xseq = 0;             // sequence count of the run's offered-key record
};

namespace {

constexpr uint64_t kDefaultLimitNs = 20ull * 1000 * 1000 * 1000;

struct Cfg {
    int W, threads, blocks, grid_W, grid_blocks;
    uint32_t pull_div;
    uint64_t heavy_words;
    uint64_t defer_words;
    uint32_t shard_index, shard_count;
    uint64_t limit_ns;
    uint32_t flags;
    uint32_t cta_entries, tab_shift;   // per-CTA vertex tables (WaveParams)
    bool sparse;                       // per-CTA phase: one source per CTA (k_sparse)
    uint32_t sparse_qcap;
};

// Entries of a hashed per-CTA vertex table by default: n/8 rounded up to a
// power of two, within [2^16, 2^21].  A per-CTA wave runs after the
// grid-wide waves and the prefilter and reaches a small part of the graph
// before it completes, is cut, or turns wide enough to be deferred anyway
// (Chung-Lu n = 2^20 leaves no source to the per-CTA waves at all), so a
// table of n/8 entries stands in for n records per CTA.  A table too small
// defers waves by the hundred thousand, measured on Barabasi-Albert graphs
// (k = 10): n = 2^21 with 2^16 entries deferred 258,176 sources (611 ms
// against 75 ms dense), with 2^17 none (88 ms, 2.0 GB of slots against
// 26.5 GB); n = 2^20 with 2^16 entries took 162 ms against 33 ms dense.
constexpr uint32_t kCtaTableMin = 1u << 16, kCtaTableMax = 1u << 21;
uint32_t default_cta_table(uint32_t n) {
    uint32_t t = kCtaTableMin;
    while (t < kCtaTableMax && (uint64_t)t * 8 < n) t <<= 1;
    return t;
}

// One source per CTA (k_sparse) by default on undirected graphs whose
// largest degree is at most this: lattices, meshes, road-like graphs, where
// the sources of a wave (consecutive in the degree order) have BFS spheres
// that share almost no vertex at any level, and bit lanes would carry one
// live bit per word.  A hub is reached by every source's search and makes
// lanes share frontiers, so graphs with hubs keep the bit-lane waves.
constexpr uint32_t kSparseMaxDeg = 8;
// Entries of each of its vertex queues where a longer frontier can be
// deferred to the grid-wide pass (else n).
constexpr uint32_t kSparseQcap = 1u << 18;

bcm_status resolve(bcm_graph* g, const bcm_options* opt, Cfg* c) {
    bcm_options o{};
    if (opt) o = *opt;
    c->flags = o.flags;
    if ((o.flags & BCM_SPARSE) && (o.flags & BCM_NO_SPARSE))
        return fail(BCM_ERR_INVALID, "BCM_SPARSE and BCM_NO_SPARSE exclude each other");
    uint32_t lanes = o.lanes ? o.lanes : 64;
    if (lanes != 64 && lanes != 128 && lanes != 256)
        return fail(BCM_ERR_UNSUPPORTED, "lanes must be 64, 128 or 256 (got %u)", lanes);
    c->W = (int)(lanes / 64);
    // one source per CTA: asked for, or by default on undirected graphs
    // without hubs (kSparseMaxDeg)
    c->sparse = !(o.flags & BCM_GRID_ONLY) &&
                ((o.flags & BCM_SPARSE) || (!(o.flags & BCM_NO_SPARSE) && !g->directed && g->n >= 4096 &&
                                            g->max_deg <= kSparseMaxDeg));
    // its default block is 256 threads: on damaged grids 512 threads took
    // 3.4 s against 2.5 s at 512^2, 128 threads 25.7 s against 23.6 s at
    // 1024^2 (it also runs 128)
    c->threads = o.threads ? (int)o.threads : (c->sparse ? 256 : 512);
    if (c->sparse) {
        if (c->threads != 128 && c->threads != 256 && c->threads != 512 && c->threads != 1024)
            return fail(BCM_ERR_UNSUPPORTED, "threads must be 128, 256, 512 or 1024 (got %u)", o.threads);
    } else {
        if (c->threads != 256 && c->threads != 512 && c->threads != 1024)
            return fail(BCM_ERR_UNSUPPORTED, "threads must be 256, 512 or 1024 (got %u)", o.threads);
        if (c->threads < 64 * c->W)
            return fail(BCM_ERR_UNSUPPORTED, "threads (%d) must be >= lanes (%u)", c->threads, lanes);
    }
    const int per_threads = c->threads < 256 ? 256 : c->threads;   // the wave kernel's shape (not run)
    int per = cta_blocks_per_sm(c->W, per_threads < 64 * c->W ? 64 * c->W : per_threads);
    if (per < 1) return fail(BCM_ERR_CUDA, "wave kernel does not fit on an SM");
    int maxb = per * g->sms;
    // default: every CTA that fits, but no more than there are waves of
    // sources (a small graph then holds a small workspace)
    uint64_t waves = ((uint64_t)g->n + 64 * c->W - 1) / (64 * c->W);
    c->blocks = o.blocks ? (int)o.blocks : (waves < (uint64_t)maxb ? (int)(waves ? waves : 1) : maxb);
    if (c->blocks > maxb) c->blocks = maxb;
    c->limit_ns = o.wait_limit_ns ? o.wait_limit_ns : kDefaultLimitNs;
    uint32_t glanes = o.grid_lanes ? o.grid_lanes : 128;
    if (glanes != 64 && glanes != 128 && glanes != 256)
        return fail(BCM_ERR_UNSUPPORTED, "grid_lanes must be 64, 128 or 256 (got %u)", glanes);
    c->grid_W = (int)(glanes / 64);
    int gb = max_coop_blocks(0, c->grid_W, 512);
    if (gb < 1) return fail(BCM_ERR_CUDA, "grid wave kernel does not fit on an SM");
    c->grid_blocks = gb;
    c->heavy_words = o.heavy_words ? o.heavy_words : (uint64_t)gb * 16 * 4;   // 4 words per warp and level
    c->pull_div = (c->flags & BCM_NO_PULL) ? 0u : o.pull_div;   // 0: per-mode default below
    c->defer_words = (c->flags & BCM_NO_DEFER) ? 0 : (o.defer_words ? o.defer_words : c->heavy_words);
    // per-CTA vertex tables: hashed where a wave that fills its table can be
    // handed to the grid-wide pass (deferral on, and a graph larger than the
    // table), else dense
    if (o.cta_table && o.cta_table < g->n && (o.cta_table < 1024 || (o.cta_table & (o.cta_table - 1))))
        return fail(BCM_ERR_UNSUPPORTED, "cta_table must be a power of two >= 1024, or >= n (got %u)", o.cta_table);
    const uint32_t tab = o.cta_table ? o.cta_table : default_cta_table(g->n);
    const bool can_defer = !(c->flags & (BCM_CTA_ONLY | BCM_GRID_ONLY)) && c->defer_words &&
                           (uint64_t)g->n * c->W >= c->defer_words;
    if (can_defer && tab < g->n) {
        c->cta_entries = tab;
        c->tab_shift = 1 + (uint32_t)__builtin_clz(tab);   // 32 - log2(tab)
    } else {
        c->cta_entries = g->n;
        c->tab_shift = 0;
    }
    // one source per CTA: its queues are bounded only where an overflowing
    // source can be deferred
    const bool sparse_defer = !(c->flags & (BCM_CTA_ONLY | BCM_GRID_ONLY)) && c->defer_words;
    c->sparse_qcap = (sparse_defer && g->n > kSparseQcap) ? kSparseQcap : g->n;
    if (c->sparse) {
        const int sper = sparse_blocks_per_sm(c->threads);
        if (sper < 1) return fail(BCM_ERR_CUDA, "one-source kernel does not fit on an SM");
        const int smax = sper * g->sms;
        c->blocks = o.blocks ? (int)o.blocks : (g->n < (uint32_t)smax ? (int)(g->n ? g->n : 1) : smax);
        if (c->blocks > smax) c->blocks = smax;
    }
    c->shard_count = o.shard_count > 1 ? o.shard_count : 1;
    c->shard_index = o.shard_count > 1 ? o.shard_index : 0;
    if (c->shard_index >= c->shard_count)
        return fail(BCM_ERR_INVALID, "shard_index %u is not below shard_count %u", o.shard_index, o.shard_count);
    if ((c->flags & BCM_CTA_ONLY) && (c->flags & BCM_GRID_ONLY))
        return fail(BCM_ERR_INVALID, "BCM_CTA_ONLY and BCM_GRID_ONLY exclude each other");
    return BCM_OK;
}

// CTA slots first, then one slot (4 words per vertex) for the grid-wide waves.
size_t cta_slot_stride(bcm_graph* g, const Cfg& c) {
    return c.sparse ? sparse_slot_bytes(g->n, c.sparse_qcap) : slot_bytes(c.cta_entries, c.W);
}
size_t cta_region_bytes(bcm_graph* g, const Cfg& c) { return (size_t)c.blocks * cta_slot_stride(g, c); }
size_t region_bytes(bcm_graph* g, const Cfg& c) {
    return cta_region_bytes(g, c) + slot_bytes(g->n, 4);
}
Layout region_layout(bcm_graph* g, const Cfg& c) {
    Layout l;
    l.n = g->n;
    l.W = (uint32_t)c.W;
    l.blocks = (uint32_t)c.blocks;
    l.entries = c.sparse ? c.sparse_qcap : c.cta_entries;
    l.sparse = c.sparse;
    return l;
}

bcm_status ensure_aux(bcm_graph* g) {
    if (g->d_aux) return BCM_OK;
    CU(buf_get_t(&g->d_aux, sizeof(Aux)), "aux allocation");
    return BCM_OK;
}

bcm_status ensure_slots(bcm_graph* g, const Cfg& c) {
    size_t bytes = region_bytes(g, c);
    Layout lay = region_layout(g, c);
    if (g->slots.ptr && g->slots.bytes >= bytes) {
        if (!(g->slots.layout == lay)) {
            CU(cudaMemsetAsync(g->slots.ptr, 0, bytes, g->stream), "workspace clear");
            g->slots.layout = lay;
        }
        return BCM_OK;
    }
    region_release(g->slots, true);
    return region_acquire(bytes, lay, g->stream, &g->slots);
}

bcm_status check_dev_err(int err) {
    if (err == 0) return BCM_OK;
    if (err & (DEV_ERR_BARRIER_TIMEOUT | DEV_ERR_LOCK_TIMEOUT))
        return fail(BCM_ERR_TIMEOUT, "an in-kernel wait ran past its limit (device error bits 0x%x)", err);
    if (err & DEV_ERR_INVALID_CSR) return fail(BCM_ERR_INVALID, "malformed CSR (device check 0x%x)", err);
    if (err & DEV_ERR_TABLE_FULL)
        return fail(BCM_ERR_CUDA, "a per-CTA wave filled its vertex table with no grid-wide pass to take it "
                                  "(device error bits 0x%x)", err);
    return fail(BCM_ERR_CUDA, "device error bits 0x%x", err);
}

double ms_since(std::chrono::steady_clock::time_point t0) {
    return std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
}

// ------------------------------------------------------ preprocessing
bcm_status ensure_run_state(bcm_graph* g, bool trace);

bcm_status preprocess(bcm_graph* g, double* ms) {
    if (g->preprocessed) return BCM_OK;
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    // timed with the graph's run events (no run is pending before preprocessing)
    bcm_status est = ensure_run_state(g, false);
    if (est) return est;
    cudaEvent_t e0 = g->ev[0], e1 = g->ev[1];
    CU(cudaEventRecord(e0, s), "event record");
    size_t nb = ((size_t)n * sizeof(uint32_t) + 255) & ~(size_t)255;
    size_t scratch = 2 * nb + degree_order_scratch_bytes(n) + scan_scratch_bytes((size_t)n + 1) + 1024;
    if (g->directed) {
        size_t sc = scc_scratch_bytes(n, g->m);
        if (sc > scratch) scratch = sc;
    }
    if (!g->d_order) {
        CU(buf_get_t(&g->d_order, nb * 4), "preprocess allocation");
        g->d_xlo = (uint32_t*)((char*)g->d_order + nb);
        g->d_xhi = (uint32_t*)((char*)g->d_order + 2 * nb);
        g->d_comp = (uint32_t*)((char*)g->d_order + 3 * nb);
    }
    char* d_scr = nullptr;
    CU(buf_get_t(&d_scr, scratch), "preprocess scratch");
    int* d_err = (int*)(d_scr + scratch - 256);
    // the degree order and the simple-graph check do not depend on the
    // components: they run on the helper stream meanwhile, with their own
    // scratch, and are joined below
    const size_t dos = (degree_order_scratch_bytes(n) + 255) & ~(size_t)255;
    const size_t scs = simple_check_scratch_bytes(g->m);
    char* d_scr2 = nullptr;
    if (buf_get_t(&d_scr2, dos + scs + 256) != cudaSuccess) {
        buf_put(d_scr);
        return fail(BCM_ERR_OOM, "preprocess scratch");
    }
    int* d_simple = (int*)(d_scr2 + dos + scs);
    bcm_status st = BCM_OK;
    int herr = 0;
    bool forked = false;
    do {
        if (cudaMemsetAsync(d_err, 0, sizeof(int), s) != cudaSuccess) { st = fail(BCM_ERR_CUDA, "memset"); break; }
        if (n == 0) break;
        if (cudaEventRecord(g->ev[5], s) != cudaSuccess || cudaStreamWaitEvent(g->aux, g->ev[5], 0) != cudaSuccess) {
            st = fail(BCM_ERR_CUDA, "stream fork");
            break;
        }
        forked = true;
        if (cudaMemsetAsync(d_simple, 0, sizeof(int), g->aux) != cudaSuccess ||
            launch_degree_order(g->d_rp, n, g->d_order, d_scr2, dos, g->aux, &g->max_deg) ||
            launch_simple_check(g->d_rp, g->d_col, n, g->m, d_simple, d_scr2 + dos, g->aux) ||
            cudaMemcpyAsync(&g->h->not_simple, d_simple, sizeof(int), cudaMemcpyDeviceToHost, g->aux) != cudaSuccess) {
            st = fail(BCM_ERR_CUDA, "degree order: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        if (!g->directed) {
            uint32_t* parent = g->d_comp;
            uint32_t* size = (uint32_t*)d_scr;
            if (launch_cc_reach(g->d_rp, g->d_col, n, parent, size, g->d_xlo, g->d_xhi, d_err, s)) {
                st = fail(BCM_ERR_CUDA, "component kernels: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            // d_comp now holds each vertex's component root (its smallest
            // vertex); bcm_scc_bounds turns roots into labels when asked
            g->labels_ready = false;
        } else {
            uint32_t nscc = 0;
            if (!g->d_rrp) {
                if (buf_get_t(&g->d_rrp, ((size_t)n + 1) * 4) != cudaSuccess ||
                    buf_get_t(&g->d_rcol, (g->m ? g->m : 1) * 4) != cudaSuccess) {
                    st = fail(BCM_ERR_OOM, "in-arc CSR allocation");
                    break;
                }
            }
            if (launch_reverse_csr(g->d_rp, g->d_col, n, g->m, g->d_rrp, g->d_rcol, d_scr, scratch - 1024, s)) {
                st = fail(BCM_ERR_CUDA, "in-arc CSR: %s", cudaGetErrorString(cudaGetLastError()));
                break;
            }
            int rc = launch_scc_bounds(g->d_rp, g->d_col, g->d_rrp, g->d_rcol, n, g->m, g->d_comp, g->d_xlo,
                                       g->d_xhi, &nscc, !(g->flags & BCM_PLAIN_BOUNDS), d_scr, scratch - 1024,
                                       d_err, s);
            if (rc == -2) { st = fail(BCM_ERR_UNSUPPORTED, "directed preprocessing is not available"); break; }
            if (rc) { st = fail(BCM_ERR_CUDA, "SCC kernels: %s", cudaGetErrorString(cudaGetLastError())); break; }
            g->n_comp = nscc;
            g->labels_ready = true;
        }
        if (cudaMemcpyAsync(&herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) {
            st = fail(BCM_ERR_CUDA, "copy");
            break;
        }
    } while (0);
    if (forked) {   // join the helper stream
        cudaEventRecord(g->ev[6], g->aux);
        cudaStreamWaitEvent(s, g->ev[6], 0);
    }
    cudaEventRecord(e1, s);
    cudaError_t se = cudaStreamSynchronize(s);
    if (forked) cudaStreamSynchronize(g->aux);
    buf_put(d_scr);
    buf_put(d_scr2);
    if (forked) g->simple = g->h->not_simple == 0;
    float t = 0;
    cudaEventElapsedTime(&t, e0, e1);
    if (st != BCM_OK) return st;
    if (se != cudaSuccess) return cuda_fail(se, "preprocessing");
    if (herr) return check_dev_err(herr);
    g->preprocessed = true;
    if (ms) *ms += t;
    return BCM_OK;
}

// Undirected graphs: component roots -> labels ordered by smallest member
// (a root is its component's smallest vertex, so the label is the root's rank
// among roots).
bcm_status ensure_labels(bcm_graph* g) {
    if (g->labels_ready || g->n == 0) { g->labels_ready = true; return BCM_OK; }
    cudaStream_t s = g->stream;
    const uint32_t n = g->n;
    size_t nb = ((size_t)n * sizeof(uint32_t) + 255) & ~(size_t)255;
    size_t bytes = nb + scan_scratch_bytes(n) + 512;
    char* d_scr = nullptr;
    CU(buf_get_t(&d_scr, bytes), "label scratch");
    uint32_t* flags = (uint32_t*)d_scr;
    uint32_t* total = (uint32_t*)(d_scr + bytes - 256);
    bcm_status st = BCM_OK;
    if (launch_root_flags(g->d_comp, n, flags, s) || exclusive_scan_u32(flags, flags, n, total, d_scr + nb, s) ||
        launch_relabel(g->d_comp, flags, n, s))
        st = fail(BCM_ERR_CUDA, "component labels");
    if (st == BCM_OK &&
        cudaMemcpyAsync(&g->n_comp, total, sizeof(uint32_t), cudaMemcpyDeviceToHost, s) != cudaSuccess)
        st = fail(BCM_ERR_CUDA, "copy");
    cudaError_t e = cudaStreamSynchronize(s);
    buf_put(d_scr);
    if (st) return st;
    if (e != cudaSuccess) return cuda_fail(e, "component labels");
    g->labels_ready = true;
    return BCM_OK;
}

WaveParams base_params(bcm_graph* g, const Cfg& c) {
    WaveParams p;
    memset(&p, 0, sizeof(p));
    p.g.n = g->n;
    p.g.m = g->m;
    p.g.rp = g->d_rp;
    p.g.col = g->d_col;
    p.g.order = g->d_order;
    p.g.xlo = g->d_xlo;
    p.g.xhi = g->d_xhi;
    p.g.rrp = g->directed ? g->d_rrp : g->d_rp;
    p.g.rcol = g->directed ? g->d_rcol : g->d_col;
    p.footnote = (!g->directed && !(c.flags & BCM_NO_FOOTNOTE)) ? 1u : 0u;
    Aux* a = g->d_aux;
    p.sources = g->d_order;
    p.head = &a->head;
    p.n_end = g->n;
    p.topk.id = a->topk_id;
    p.topk.f = a->topk_f;
    p.topk.r = a->topk_r;
    p.topk.count = &a->topk_count;
    p.topk.lock = &a->lock;
    p.topk.thr = &a->thr;
    p.topk.ext = &a->ext;
    p.snap = &a->snap;
    p.slot_base = (char*)g->slots.ptr;
    p.slot_stride = cta_slot_stride(g, c);
    p.sparse_qcap = c.sparse_qcap;
    p.cta_entries = c.cta_entries;
    p.tab_shift = c.tab_shift;
    p.tab_limit = c.cta_entries / 2;
    p.seed_base = (char*)g->slots.ptr + cta_region_bytes(g, c);
    p.stats = a->stats;
    p.err = &a->err;
    p.lock_limit_ns = c.limit_ns;
    p.barrier_limit_ns = c.limit_ns;
    p.bar = &a->bar;
    p.gcnt = a->gcnt;
    p.glist_n = a->glist_n;
    p.glog_n = &a->glog_n;
    p.gchunk = a->gchunk;
    p.garc = a->garc;
    p.gheavy = a->gheavy;
    p.gheavy_n = &a->gheavy_n;
    p.gheavy_cap = 2048;
    return p;
}

// Algorithmic bytes of the per-CTA wave kernel, from its counters: the words
// it must move at minimum (word granularity, no cache or sector effects).
//   started source            20 B  order entry, row_ptr pair, x_lo/x_hi
//   frontier word expanded    28 B  list entry, F word read and clear, row_ptr pair
//     (of a pulled level)     12 B  list entry, F word clear (its reads are the arcs')
//   (arc, frontier word)      12 B  col entry, vis word
//   new frontier word         32 B  vis and F-next atomics, row_ptr pair, list and log entries
//   cleared word              28 B  log entry, vis/F/F' stores
uint64_t wave_alg_bytes(const unsigned long long* w, uint64_t sources) {
    return 20ull * sources + 28ull * (w[ST_ENTRIES] - w[ST_PULLENTRIES]) + 12ull * w[ST_PULLENTRIES] +
           12ull * w[ST_ARCWORDS] + 32ull * w[ST_DISCWORDS] + 28ull * w[ST_CLEARED];
}

// The one-source kernel's (its counters count vertices, arcs and bitmap words):
//   source started            20 B  order entry, row_ptr pair, x_lo/x_hi
//   frontier vertex expanded  12 B  queue entry, row_ptr pair
//   arc scanned                8 B  col entry, the target's bitmap word
//   vertex discovered         16 B  bitmap atomicOr, row_ptr pair, queue entry
//   cleared bitmap word       12 B  log entry written and read, the word cleared
uint64_t sparse_alg_bytes(const unsigned long long* w, uint64_t sources) {
    return 20ull * sources + 12ull * w[ST_ENTRIES] + 8ull * w[ST_ARCWORDS] + 16ull * w[ST_DISCWORDS] +
           12ull * w[ST_CLEARED];
}

void fill_stats(bcm_stats* s, const unsigned long long* st, uint64_t launches, double kms, double pms, double tms) {
    if (!s) return;
    s->m_vis = st[ST_MVIS];
    s->visits = st[ST_DISC];
    s->completed = st[ST_COMPLETED];
    s->cut = st[ST_CUT];
    s->waves = st[ST_WAVES];
    s->levels = st[ST_LEVELS];
    s->max_level = st[ST_MAXLEVEL];
    s->frontier_words = st[ST_ENTRIES];
    s->arc_words = st[ST_ARCWORDS];
    s->new_words = st[ST_DISCWORDS];
    s->cleared_words = st[ST_CLEARED];
    s->deferred = st[ST_DEFERRED];
    s->launches = launches;
    s->kernel_ms = kms;
    s->preprocess_ms = pms;
    s->total_ms = tms;
}

// Times and counters of a finished run.
struct RunTimes {
    double kernel_ms = 0, seed_ms = 0, wave_ms = 0;
    unsigned long long grid[ST_COUNT] = {0};
};

bcm_status copy_out(void* dst, const void* src, size_t bytes, bool dev, cudaStream_t s);

// Sources of one shard: the degree order's positions in every
// count-th chunk of kShardChunk, starting with chunk `index`.
constexpr uint32_t kShardChunk = 64;

__global__ void k_shard_sources(const uint32_t* order, uint32_t n_local, uint32_t index, uint32_t count,
                                uint32_t* out) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < n_local; i += stride) {
        const size_t pos = ((i / kShardChunk) * count + index) * kShardChunk + i % kShardChunk;
        out[i] = order[pos];
    }
}

// Positions of the degree order that fall to shard `index` of `count`.
uint32_t shard_size(uint32_t n, uint32_t index, uint32_t count) {
    const uint64_t C = kShardChunk, round = C * count;
    const uint64_t rem = n % round, lo = (uint64_t)index * C;
    uint64_t r = (n / round) * C;
    if (rem > lo) r += (rem - lo < C ? rem - lo : C);
    return (uint32_t)r;
}

bcm_status ensure_run_state(bcm_graph* g, bool trace) {
    if (!g->ev[0] || !g->h) {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (!g->ev[0])
            for (size_t i = 0; i < g_res_free.size(); ++i)
                if (g_res_free[i].dev == g->dev) {
                    for (int j = 0; j < 7; ++j) g->ev[j] = g_res_free[i].ev[j];
                    g->aux = g_res_free[i].aux;
                    g_res_free.erase(g_res_free.begin() + i);
                    break;
                }
        if (!g->h && !g_pinned_free.empty()) {
            g->h = (HostBlock*)g_pinned_free.back();
            g_pinned_free.pop_back();
        }
    }
    for (int i = 0; i < 7; ++i)
        if (!g->ev[i]) CU(cudaEventCreateWithFlags(&g->ev[i], i < 5 ? cudaEventDefault : cudaEventDisableTiming), "event");
    if (!g->aux) CU(cudaStreamCreateWithFlags(&g->aux, cudaStreamNonBlocking), "stream");
    if (!g->h) CU(cudaMallocHost(&g->h, sizeof(HostBlock)), "pinned host allocation");
    if (trace && !g->d_trace) CU(buf_get_t(&g->d_trace, (size_t)kTraceCap * 4 * sizeof(u64)), "trace allocation");
    return BCM_OK;
}

// Enqueues one run of the wave kernels on the graph's stream and the copies
// of its results and counters, and returns without waiting.  exhaustive:
// every source, no cut, outputs o_far/o_reach (n entries); else top-k with
// outputs o_ids/o_far/o_reach (min(k, n) entries).
bcm_status start_run(bcm_graph* g, const Cfg& c, uint32_t k, bool exhaustive, void* o_ids, void* o_far,
                     void* o_reach) {
    cudaStream_t s = g->stream;
    const bool trace = (c.flags & BCM_TRACE) != 0;
    bcm_status st = ensure_aux(g);
    if (st) return st;
    if ((st = ensure_run_state(g, trace))) return st;
    const bool plain = !exhaustive && (c.flags & BCM_PLAIN);
    if (!plain && (st = ensure_slots(g, c))) return st;
    if (exhaustive && !g->d_far) {
        CU(buf_get_t(&g->d_far, (size_t)g->n * sizeof(uint64_t) + 256), "output allocation");
        CU(buf_get_t(&g->d_reach, (size_t)g->n * sizeof(uint32_t) + 256), "output allocation");
    }
    if (plain && !g->d_plain)
        CU(buf_get_t(&g->d_plain, (size_t)g->n * 3 * sizeof(uint32_t) + 256), "plain buffers");
    CU(cudaMemsetAsync(g->d_aux, 0, sizeof(Aux), s), "aux clear");
    // ids of entries a run does not fill (a shard run with an offered key may hold fewer than k)
    CU(cudaMemsetAsync(g->d_aux->topk_id, 0xff, sizeof(g->d_aux->topk_id), s), "aux clear");
    {
        std::lock_guard<std::mutex> lk(g->xmu);
        if (!g->ev_x) CU(cudaEventCreateWithFlags(&g->ev_x, cudaEventDisableTiming), "event");
        CU(cudaEventRecord(g->ev_x, s), "event record");
        g->offered = false;
        g->best = bcm_key{0, 0, 0, 0};
        g->xseq = 0;
    }
    WaveParams p = base_params(g, c);
    p.exhaustive = exhaustive ? 1u : 0u;
    p.topk.k = k;
    uint32_t n_src = g->n;   // sources this run takes
    if (!exhaustive && c.shard_count > 1) {
        n_src = shard_size(g->n, c.shard_index, c.shard_count);
        if (!g->d_shard) CU(buf_get_t(&g->d_shard, (size_t)g->n * sizeof(uint32_t)), "shard list allocation");
        if (n_src) {
            unsigned blocks = (n_src + 255) / 256 < 4864 ? (n_src + 255) / 256 : 4864;
            k_shard_sources<<<blocks, 256, 0, s>>>(g->d_order, n_src, c.shard_index, c.shard_count, g->d_shard);
            note_launch();
            CU(cudaGetLastError(), "shard list kernel");
        }
        p.sources = g->d_shard;
        p.n_end = n_src;
    }
    p.out_far = g->d_far;
    p.out_reach = g->d_reach;
    if (trace) {
        p.trace = g->d_trace;
        p.trace_cap = kTraceCap;
        p.trace_n = &g->d_aux->trace_n;
        p.trace_lanes = (c.flags & BCM_TRACE_LANES) ? 1u : 0u;
    }
    p.nocut = (!exhaustive && (c.flags & BCM_NO_CUT)) ? 1u : 0u;
    p.all_pull = ((c.flags & BCM_ALL_PULL) && !(c.flags & BCM_NO_PULL)) ? 1u : 0u;
    CU(cudaEventRecord(g->ev[0], s), "event record");
    int rc = 0;
    p.stats = g->d_aux->seed_stats;
    if (plain) {
        CU(cudaMemsetAsync(g->d_plain, 0, (size_t)g->n * sizeof(uint32_t), s), "stamp clear");
        int blocks = max_coop_blocks(1, 1, 256);
        int want = g->sms;   // one 256-thread CTA per SM
        if (blocks > want) blocks = want;
        for (uint32_t it = 0; it < g->n && rc == 0; ++it)
            rc = launch_plain_source(p, it, g->d_plain, g->d_plain + g->n, blocks, 256, s);
        cudaEventRecord(g->ev[1], s);
    } else {
        // grid-wide waves while they are heavy (every wave for exhaustive
        // runs), then per-CTA waves from wherever the grid kernel left head.
        // A top-k run on a graph with fewer (vertex, word) pairs than the
        // heavy threshold cannot have a heavy wave and skips the grid kernel.
        const bool grid = !(c.flags & BCM_CTA_ONLY) &&
                          ((c.flags & BCM_GRID_ONLY) ||
                           (!c.sparse && (exhaustive || (uint64_t)g->n * c.grid_W >= c.heavy_words)));
        // a per-CTA wave whose frontier grows to defer_words words hands its
        // sources to a second grid-wide pass (only where one can follow, and
        // only if a frontier that wide is possible)
        // (one source per CTA: a source whose frontier outgrows its queue,
        // in exhaustive runs too)
        const bool defer = c.sparse ? (!(c.flags & (BCM_CTA_ONLY | BCM_GRID_ONLY)) && c.defer_words &&
                                       c.sparse_qcap < g->n)
                                    : (!exhaustive && !(c.flags & (BCM_CTA_ONLY | BCM_GRID_ONLY)) && c.defer_words &&
                                       (uint64_t)g->n * c.W >= c.defer_words);
        if (defer) {
            if (!g->d_defer) CU(buf_get_t(&g->d_defer, (size_t)g->n * sizeof(uint32_t)), "defer list allocation");
            p.defer_words = (uint32_t)(c.defer_words < 0xffffffffull ? c.defer_words : 0xffffffffull);
            p.defer_n = &g->d_aux->defer_n;
            p.defer_src = g->d_defer;
        }
        if (grid) {
            p.max_grid_waves = 0xffffffffu;
            p.heavy_words = (exhaustive || (c.flags & BCM_GRID_ONLY)) ? 0 : c.heavy_words;
            // default measured per level on the Chung-Lu and R-MAT workloads:
            // pull wins once the frontier's out-arcs reach about n*W/32
            p.pull_div = (c.flags & BCM_NO_PULL) ? 0u : (c.pull_div ? c.pull_div : 32u);
            rc = launch_grid_waves(p, c.grid_W, c.grid_blocks, 512, s);
        }
        p.stats = g->d_aux->stats;
        // a graph too small for grid-wide waves: one CTA first runs the
        // first wave alone (the highest-degree sources), so the threshold
        // exists before the other waves start (otherwise they all start at
        // once, and none of them can be stopped)
        const bool seed = !grid && rc == 0 && !exhaustive && !c.sparse &&
                          !(c.flags & (BCM_CTA_ONLY | BCM_NO_PREFILTER));
        if (seed) {
            WaveParams ps = p;
            ps.max_cta_waves = 1;
            rc = launch_cta_waves(ps, c.W, 1, c.threads, s);
        }
        cudaEventRecord(g->ev[1], s);
        WaveParams pc = p;
        // on a simple graph, the sources the grid (or the seed wave) left are
        // first tested at levels 0 and 1 from degrees alone; the waves take
        // the rest
        const bool prefilter = (grid || seed) && rc == 0 && g->simple &&
                               !(c.flags & (BCM_NO_PREFILTER | BCM_GRID_ONLY | BCM_NO_CUT));
        if (prefilter) {
            if (!g->d_surv) {
                cudaError_t e = buf_get_t(&g->d_surv, (size_t)g->n * sizeof(uint32_t));
                if (e != cudaSuccess) { cudaStreamSynchronize(s); return cuda_fail(e, "prefilter list allocation"); }
            }
            rc = launch_prefilter(p, g->d_surv, &g->d_aux->surv_n, s);
            pc.sources = g->d_surv;
            pc.head = &g->d_aux->head3;
            pc.n_end = 0;
            pc.n_end_dev = &g->d_aux->surv_n;
        }
        if (rc == 0)
            rc = c.sparse ? launch_sparse(pc, c.blocks, c.threads, s) : launch_cta_waves(pc, c.W, c.blocks, c.threads, s);
        cudaEventRecord(g->ev[2], s);
        if (defer && rc == 0) {
            // the deferred sources, on the grid kernel, every wave
            WaveParams q = p;
            q.sources = g->d_defer;
            q.head = &g->d_aux->head2;
            q.n_end = 0;
            q.n_end_dev = &g->d_aux->defer_n;
            q.max_grid_waves = 0xffffffffu;
            q.heavy_words = 0;
            q.defer_words = 0;
            q.pull_div = (c.flags & BCM_NO_PULL) ? 0u : (c.pull_div ? c.pull_div : 32u);
            q.stats = g->d_aux->seed_stats;
            rc = launch_grid_waves(q, c.grid_W, c.grid_blocks, 512, s);
        }
    }
    if (plain) cudaEventRecord(g->ev[2], s);
    cudaEventRecord(g->ev[3], s);
    if (rc) {
        cudaStreamSynchronize(s);
        return fail(BCM_ERR_CUDA, "wave kernel launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    }
    Aux* a = g->d_aux;
    HostBlock* h = g->h;
    CU(cudaMemcpyAsync(&h->err, &a->err, sizeof(int), cudaMemcpyDeviceToHost, s), "copy");
    CU(cudaMemcpyAsync(&h->topk_count, &a->topk_count, sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "copy");
    CU(cudaMemcpyAsync(&h->trace_n, &a->trace_n, sizeof(uint32_t), cudaMemcpyDeviceToHost, s), "copy");
    CU(cudaMemcpyAsync(h->stats, a->stats, sizeof(h->stats), cudaMemcpyDeviceToHost, s), "copy");
    CU(cudaMemcpyAsync(h->seed_stats, a->seed_stats, sizeof(h->seed_stats), cudaMemcpyDeviceToHost, s), "copy");
    const bool dev = (c.flags & BCM_OUT_DEVICE) != 0;
    if (exhaustive) {
        if ((st = copy_out(o_far, g->d_far, (size_t)g->n * sizeof(uint64_t), dev, s))) return st;
        if ((st = copy_out(o_reach, g->d_reach, (size_t)g->n * sizeof(uint32_t), dev, s))) return st;
    } else {
        const uint32_t kk = k < n_src ? k : n_src;
        if ((st = copy_out(o_ids, a->topk_id, kk * sizeof(uint32_t), dev, s))) return st;
        if ((st = copy_out(o_far, a->topk_f, kk * sizeof(uint64_t), dev, s))) return st;
        if ((st = copy_out(o_reach, a->topk_r, kk * sizeof(uint32_t), dev, s))) return st;
    }
    CU(cudaEventRecord(g->ev[4], s), "event record");
    g->pend.active = true;
    g->pend.exhaustive = exhaustive;
    g->pend.plain = plain;
    g->pend.sparse = !plain && c.sparse;
    g->pend.kk = k < n_src ? k : n_src;
    g->pend.flags = c.flags;
    return BCM_OK;
}

// Completes the pending run: BCM_ERR_PENDING if !wait and it has not
// finished, else its outcome, with its counters in sv (both kernels),
// wv (per-CTA kernel) and rt.
bcm_status finish_run(bcm_graph* g, bool wait, unsigned long long* sv, unsigned long long* wv, RunTimes* rt) {
    if (!g->pend.active) return fail(BCM_ERR_INVALID, "no run is pending on this graph");
    if (!wait) {
        cudaError_t q = cudaEventQuery(g->ev[4]);
        if (q == cudaErrorNotReady) return BCM_ERR_PENDING;
        if (q != cudaSuccess) {
            std::lock_guard<std::mutex> lk(g->xmu);
            g->pend.active = false;
            return cuda_fail(q, "wave kernels");
        }
    }
    cudaError_t se = cudaEventSynchronize(g->ev[4]);
    bool offered = false;
    {
        std::lock_guard<std::mutex> lk(g->xmu);
        g->pend.active = false;
        offered = g->offered;
    }
    if (se != cudaSuccess) return cuda_fail(se, "wave kernels");
    const HostBlock* h = g->h;
    float t = 0, t01 = 0, t12 = 0, t23 = 0;
    cudaEventElapsedTime(&t, g->ev[0], g->ev[3]);
    cudaEventElapsedTime(&t01, g->ev[0], g->ev[1]);
    cudaEventElapsedTime(&t12, g->ev[1], g->ev[2]);
    cudaEventElapsedTime(&t23, g->ev[2], g->ev[3]);
    const float t0m = t01 + t23, tm1 = t12;
    for (int i = 0; i < ST_COUNT; ++i) {
        wv[i] = h->stats[i];
        sv[i] = (i == ST_MAXLEVEL) ? (h->stats[i] > h->seed_stats[i] ? h->stats[i] : h->seed_stats[i])
                                   : h->stats[i] + h->seed_stats[i];
        rt->grid[i] = h->seed_stats[i];
    }
    rt->kernel_ms = t;
    rt->seed_ms = t0m;
    rt->wave_ms = tm1;
    g->trace_n = (g->pend.flags & BCM_TRACE) ? h->trace_n : 0;
    if (h->err) {
        // a timed-out run may leave words set: do not reuse the region
        region_release(g->slots, false);
        return check_dev_err(h->err);
    }
    // with an offered key a shard keeps only sources that rank before it: fewer entries are fine
    if (!g->pend.exhaustive && (offered ? h->topk_count > g->pend.kk : h->topk_count != g->pend.kk))
        return fail(BCM_ERR_CUDA, "top-k holds %u entries, expected %u", h->topk_count, g->pend.kk);
    return BCM_OK;
}

void fill_run_stats(bcm_stats* stats, bcm_graph* g, const unsigned long long* sv, const unsigned long long* wv,
                    const RunTimes& rt) {
    if (!stats) return;
    fill_stats(stats, sv, g_launches.load() - g->pend.l0, rt.kernel_ms, g->pend.pms, ms_since(g->pend.t0));
    const bool plain = g->pend.plain;
    stats->seed_ms = rt.seed_ms;
    stats->wave_ms = rt.wave_ms;
    stats->wave_bytes = plain ? 0
                      : g->pend.sparse ? sparse_alg_bytes(wv, wv[ST_WAVES])
                                       : wave_alg_bytes(wv, wv[ST_COMPLETED] + wv[ST_CUT]);
    stats->sparse = g->pend.sparse ? wv[ST_WAVES] : 0;
    stats->grid_waves = rt.grid[ST_WAVES];
    stats->grid_levels = rt.grid[ST_LEVELS];
    stats->grid_bytes = plain ? 0 : wave_alg_bytes(rt.grid, rt.grid[ST_COMPLETED] + rt.grid[ST_CUT]);
}

bcm_status copy_out(void* dst, const void* src, size_t bytes, bool dev, cudaStream_t s) {
    CU(cudaMemcpyAsync(dst, src, bytes, dev ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, s), "output copy");
    return BCM_OK;
}

}  // namespace

// ------------------------------------------------ symmetric-pairs check
namespace bcm {
__global__ void k_check_symmetric(const uint32_t* rp, const uint32_t* col, uint32_t n, int* bad) {
    size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
    size_t nw = ((size_t)gridDim.x * blockDim.x) >> 5;
    uint32_t lane = threadIdx.x & 31;
    for (size_t u = warp; u < n; u += nw) {
        for (uint32_t e = rp[u] + lane; e < rp[u + 1]; e += 32) {
            uint32_t w = col[e];
            if (e + 1 < rp[u + 1] && col[e + 1] < w) { atomicOr(bad, 2); continue; }   // rows must be sorted
            uint32_t lo = rp[w], hi = rp[w + 1];
            while (lo < hi) {
                uint32_t mid = lo + (hi - lo) / 2;
                if (col[mid] < u) lo = mid + 1; else hi = mid;
            }
            if (lo >= rp[w + 1] || col[lo] != u) atomicOr(bad, 1);
        }
    }
}

__global__ void k_root_flags(const uint32_t* parent, uint32_t n, uint32_t* flags) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += stride)
        flags[v] = parent[v] == v ? 1u : 0u;
}

__global__ void k_relabel(uint32_t* parent, const uint32_t* rank, uint32_t n) {
    size_t stride = (size_t)gridDim.x * blockDim.x;
    for (size_t v = blockIdx.x * (size_t)blockDim.x + threadIdx.x; v < n; v += stride)
        parent[v] = rank[parent[v]];
}

int launch_root_flags(const uint32_t* parent, uint32_t n, uint32_t* flags, cudaStream_t s) {
    k_root_flags<<<(n + 255) / 256 < 4864 ? (n + 255) / 256 : 4864, 256, 0, s>>>(parent, n, flags);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// parent[v] holds a root id; rank[root] its label.  Roots are relabelled
// last, after every vertex read them, by a second pass.
int launch_relabel(uint32_t* parent, const uint32_t* rank, uint32_t n, cudaStream_t s) {
    // rank[] is the exclusive scan of the root flags; parent[v] = rank[parent[v]]
    // is safe in one pass because rank is a separate array.
    k_relabel<<<(n + 255) / 256 < 4864 ? (n + 255) / 256 : 4864, 256, 0, s>>>(parent, rank, n);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace bcm

// ================================================================= C-ABI
extern "C" {

const char* bcm_last_error(void) { return t_err.c_str(); }

uint64_t bcm_launch_count(void) { return g_launches.load(); }

bcm_status bcm_graph_create(const uint64_t* row_ptr, const uint32_t* col, uint32_t n, uint64_t m, int directed,
                            int ptr_on_device, void* stream, uint32_t flags, bcm_graph_t* out) {
    t_err.clear();
    if (!out) return fail(BCM_ERR_INVALID, "out is NULL");
    *out = nullptr;
    if (!row_ptr || (m > 0 && !col)) return fail(BCM_ERR_INVALID, "row_ptr/col is NULL");
    if (n >= (1u << 30)) return fail(BCM_ERR_UNSUPPORTED, "n = %u: at most 2^30 - 1 vertices", n);
    if (m >= (1ull << 32)) return fail(BCM_ERR_UNSUPPORTED, "m = %llu: fewer than 2^32 arcs", (unsigned long long)m);
    bcm_graph* g = new (std::nothrow) bcm_graph();
    if (!g) return fail(BCM_ERR_OOM, "host allocation");
    g->n = n;
    g->m = m;
    g->directed = directed ? 1 : 0;
    g->flags = flags;
    g->stream = (cudaStream_t)stream;
    cudaGetDevice(&g->dev);
    cudaDeviceGetAttribute(&g->sms, cudaDevAttrMultiProcessorCount, g->dev);
    cudaStream_t s = g->stream;
    bcm_status st = BCM_OK;
    uint64_t* d_rp64 = nullptr;
    int* d_err = nullptr;
    do {
        cudaError_t e;
        if ((e = buf_get_t(&g->d_rp, ((size_t)n + 1) * sizeof(uint32_t))) != cudaSuccess) { st = cuda_fail(e, "graph allocation"); break; }
        if ((e = buf_get_t(&g->d_col, (m ? m : 1) * sizeof(uint32_t))) != cudaSuccess) { st = cuda_fail(e, "graph allocation"); break; }
        if ((e = buf_get_t(&d_rp64, ((size_t)n + 1) * sizeof(uint64_t) + sizeof(int) * 4)) != cudaSuccess) { st = cuda_fail(e, "graph allocation"); break; }
        d_err = (int*)(d_rp64 + n + 1);
        cudaMemcpyKind kind = ptr_on_device ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
        if ((e = cudaMemcpyAsync(d_rp64, row_ptr, ((size_t)n + 1) * sizeof(uint64_t), kind, s)) != cudaSuccess) { st = cuda_fail(e, "row_ptr copy"); break; }
        if (m && (e = cudaMemcpyAsync(g->d_col, col, m * sizeof(uint32_t), kind, s)) != cudaSuccess) { st = cuda_fail(e, "col copy"); break; }
        if ((e = cudaMemsetAsync(d_err, 0, 4 * sizeof(int), s)) != cudaSuccess) { st = cuda_fail(e, "memset"); break; }
        if (launch_validate(d_rp64, g->d_col, n, m, d_err, s) || launch_narrow_offsets(d_rp64, g->d_rp, n, s)) {
            st = fail(BCM_ERR_CUDA, "validation kernels: %s", cudaGetErrorString(cudaGetLastError()));
            break;
        }
        int herr[4] = {0, 0, 0, 0};
        if ((e = cudaMemcpyAsync(herr, d_err, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) { st = cuda_fail(e, "copy"); break; }
        if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { st = cuda_fail(e, "graph upload"); break; }
        if (herr[0]) { st = fail(BCM_ERR_INVALID, "malformed CSR: row_ptr must rise from 0 to m and every col < n"); break; }

        if (!directed && (flags & BCM_CHECK_SYMMETRIC) && n > 0) {
            if ((e = cudaMemsetAsync(d_err + 1, 0, sizeof(int), s)) != cudaSuccess) { st = cuda_fail(e, "memset"); break; }
            unsigned blocks = (unsigned)(((size_t)n * 32 + 255) / 256);
            if (blocks > 4864) blocks = 4864;
            k_check_symmetric<<<blocks, 256, 0, s>>>(g->d_rp, g->d_col, n, d_err + 1);
            note_launch();
            if ((e = cudaMemcpyAsync(&herr[1], d_err + 1, sizeof(int), cudaMemcpyDeviceToHost, s)) != cudaSuccess) { st = cuda_fail(e, "copy"); break; }
            if ((e = cudaStreamSynchronize(s)) != cudaSuccess) { st = cuda_fail(e, "symmetry check"); break; }
            if (herr[1] & 2) { st = fail(BCM_ERR_INVALID, "the symmetry check needs every row sorted"); break; }
            if (herr[1] & 1) { st = fail(BCM_ERR_NOT_SYMMETRIC, "undirected graph has an arc (u,w) without (w,u)"); break; }
        }
    } while (0);
    if (d_rp64) buf_put(d_rp64);
    if (st != BCM_OK) {
        bcm_graph_destroy(g);
        return st;
    }
    *out = g;
    return BCM_OK;
}

bcm_status bcm_graph_destroy(bcm_graph_t g) {
    if (!g) return BCM_OK;
    if (g->stream) cudaStreamSynchronize(g->stream);
    else cudaDeviceSynchronize();
    for (void* b : {(void*)g->d_rp, (void*)g->d_col, (void*)g->d_order, (void*)g->d_aux, (void*)g->d_plain,
                    (void*)g->d_far, (void*)g->d_reach, (void*)g->d_rrp, (void*)g->d_rcol, (void*)g->d_trace,
                    (void*)g->d_defer, (void*)g->d_shard, (void*)g->d_surv})
        buf_put(b);
    {
        std::lock_guard<std::mutex> lk(g_pool_mu);
        if (g->ev[0]) {
            RunRes r;
            r.dev = g->dev;
            for (int i = 0; i < 7; ++i) r.ev[i] = g->ev[i];
            r.aux = g->aux;
            g_res_free.push_back(r);
        }
        if (g->h) g_pinned_free.push_back(g->h);
    }
    // a run that was started and never finished may not have left the region clean
    region_release(g->slots, !g->pend.active);
    if (g->ev_x) cudaEventDestroy(g->ev_x);
    delete g;
    return BCM_OK;
}

bcm_status bcm_preprocess(bcm_graph_t g, uint32_t* order, uint32_t* x_lo, uint32_t* x_hi, int out_on_device) {
    t_err.clear();
    if (!g) return fail(BCM_ERR_INVALID, "graph is NULL");
    bcm_status st = preprocess(g, nullptr);
    if (st) return st;
    size_t b = (size_t)g->n * sizeof(uint32_t);
    if (b) {
        if (order && (st = copy_out(order, g->d_order, b, out_on_device, g->stream))) return st;
        if (x_lo && (st = copy_out(x_lo, g->d_xlo, b, out_on_device, g->stream))) return st;
        if (x_hi && (st = copy_out(x_hi, g->d_xhi, b, out_on_device, g->stream))) return st;
    }
    CU(cudaStreamSynchronize(g->stream), "copy");
    return BCM_OK;
}

bcm_status bcm_scc_bounds(bcm_graph_t g, uint32_t* comp, uint32_t* alpha, uint32_t* omega, uint32_t* n_scc,
                          int out_on_device) {
    t_err.clear();
    if (!g) return fail(BCM_ERR_INVALID, "graph is NULL");
    bcm_status st = preprocess(g, nullptr);
    if (st) return st;
    if ((st = ensure_labels(g))) return st;
    size_t b = (size_t)g->n * sizeof(uint32_t);
    if (b) {
        if (comp && (st = copy_out(comp, g->d_comp, b, out_on_device, g->stream))) return st;
        if (alpha && (st = copy_out(alpha, g->d_xlo, b, out_on_device, g->stream))) return st;
        if (omega && (st = copy_out(omega, g->d_xhi, b, out_on_device, g->stream))) return st;
    }
    CU(cudaStreamSynchronize(g->stream), "copy");
    if (n_scc) {
        if (out_on_device) CU(cudaMemcpy(n_scc, &g->n_comp, sizeof(uint32_t), cudaMemcpyHostToDevice), "copy");
        else *n_scc = g->n_comp;
    }
    return BCM_OK;
}

bcm_status bcm_topk_start(bcm_graph_t g, uint32_t k, const bcm_options* opt, uint32_t* ids, uint64_t* farness,
                          uint32_t* reach) {
    t_err.clear();
    auto t0 = std::chrono::steady_clock::now();
    uint64_t l0 = g_launches.load();
    if (!g) return fail(BCM_ERR_INVALID, "graph is NULL");
    if (g->pend.active) return fail(BCM_ERR_INVALID, "a run on this graph has not been finished");
    if (k < 1 || k > 1024) return fail(BCM_ERR_INVALID, "k = %u: must be in 1..1024", k);
    if (!ids || !farness || !reach) return fail(BCM_ERR_INVALID, "output pointer is NULL");
    double pms = 0;
    bcm_status st = preprocess(g, &pms);
    if (st) return st;
    Cfg c;
    if ((st = resolve(g, opt, &c))) return st;
    if (g->n > 0) {
        if ((st = start_run(g, c, k, false, ids, farness, reach))) return st;
    } else {
        // nothing to run: the empty result is complete at once
        if ((st = ensure_run_state(g, false))) return st;
        memset(g->h, 0, sizeof(HostBlock));
        for (int i = 0; i < 5; ++i) CU(cudaEventRecord(g->ev[i], g->stream), "event record");
        g->pend.active = true;
        g->pend.exhaustive = false;
        g->pend.plain = false;
        g->pend.sparse = false;
        g->pend.kk = 0;
        g->pend.flags = 0;
    }
    g->pend.l0 = l0;
    g->pend.pms = pms;
    g->pend.t0 = t0;
    return BCM_OK;
}

bcm_status bcm_topk_finish(bcm_graph_t g, int wait, bcm_stats* stats) {
    t_err.clear();
    if (!g) return fail(BCM_ERR_INVALID, "graph is NULL");
    unsigned long long sv[ST_COUNT] = {0}, wv[ST_COUNT] = {0};
    RunTimes rt;
    bcm_status st = finish_run(g, wait != 0, sv, wv, &rt);
    if (st == BCM_ERR_PENDING) return st;
    if (st == BCM_OK) fill_run_stats(stats, g, sv, wv, rt);
    return st;
}

bcm_status bcm_topk(bcm_graph_t g, uint32_t k, const bcm_options* opt, uint32_t* ids, uint64_t* farness,
                    uint32_t* reach, bcm_stats* stats) {
    bcm_status st = bcm_topk_start(g, k, opt, ids, farness, reach);
    if (st) return st;
    return bcm_topk_finish(g, 1, stats);
}

namespace {
bool key_before(const bcm_key& a, const bcm_key& b) {
    const unsigned __int128 l = (unsigned __int128)a.N * b.F, r = (unsigned __int128)b.N * a.F;
    if (l != r) return l > r;
    return a.id < b.id;
}
}  // namespace

bcm_status bcm_topk_threshold(bcm_graph_t g, bcm_key* out) {
    t_err.clear();
    if (!g || !out) return fail(BCM_ERR_INVALID, "a pointer argument is NULL");
    std::lock_guard<std::mutex> lk(g->xmu);
    *out = bcm_key{0, 0, 0, 0};
    if (!g->d_aux || !g->ev_x || !g->aux || !g->h) return BCM_OK;   // no run yet
    CU(cudaStreamWaitEvent(g->aux, g->ev_x, 0), "stream wait");
    HostBlock* h = g->h;
    const Aux* a = g->d_aux;
    // the record's sequence count, its fields, the count again: a snapshot is
    // consistent when both counts are equal and even (no write in between)
    for (int tries = 0; tries < 64; ++tries) {
        CU(cudaMemcpyAsync(&h->rd_seq[0], &a->thr.seq, sizeof(u64), cudaMemcpyDeviceToHost, g->aux), "copy");
        CU(cudaMemcpyAsync(&h->rd, &a->thr, sizeof(Threshold), cudaMemcpyDeviceToHost, g->aux), "copy");
        CU(cudaMemcpyAsync(&h->rd_seq[1], &a->thr.seq, sizeof(u64), cudaMemcpyDeviceToHost, g->aux), "copy");
        CU(cudaStreamSynchronize(g->aux), "threshold copy");
        if (h->rd_seq[0] == h->rd_seq[1] && !(h->rd_seq[0] & 1) && h->rd.seq == h->rd_seq[0]) {
            if (h->rd.valid) *out = bcm_key{h->rd.N, h->rd.F, h->rd.id, 1};
            return BCM_OK;
        }
    }
    return BCM_OK;   // no consistent snapshot: no key (always safe)
}

bcm_status bcm_topk_offer(bcm_graph_t g, const bcm_key* key) {
    t_err.clear();
    if (!g || !key) return fail(BCM_ERR_INVALID, "a pointer argument is NULL");
    std::lock_guard<std::mutex> lk(g->xmu);
    if (!g->pend.active || g->pend.exhaustive) return fail(BCM_ERR_INVALID, "no top-k run is pending on this graph");
    if (!key->valid) return BCM_OK;
    if (key->F == 0 || (key->N == 0 && key->F != 1))
        return fail(BCM_ERR_INVALID, "a key is (N, F) = ((r-1)^2, f) with f > 0, or (0, 1)");
    if (g->best.valid && !key_before(*key, g->best)) return BCM_OK;   // not stronger than what the run has
    HostBlock* h = g->h;
    Aux* a = g->d_aux;
    h->wr_seq[0] = g->xseq + 1;     // odd: write in progress
    h->wr_seq[1] = g->xseq + 2;     // even: consistent
    h->wr.seq = h->wr_seq[0];
    h->wr.N = key->N;
    h->wr.F = key->F;
    h->wr.id = key->id;
    h->wr.valid = 1;
    CU(cudaStreamWaitEvent(g->aux, g->ev_x, 0), "stream wait");
    CU(cudaMemcpyAsync(&a->ext.seq, &h->wr_seq[0], sizeof(u64), cudaMemcpyHostToDevice, g->aux), "copy");
    CU(cudaMemcpyAsync(&a->ext, &h->wr, sizeof(Threshold), cudaMemcpyHostToDevice, g->aux), "copy");
    CU(cudaMemcpyAsync(&a->ext.seq, &h->wr_seq[1], sizeof(u64), cudaMemcpyHostToDevice, g->aux), "copy");
    CU(cudaStreamSynchronize(g->aux), "offer copy");
    g->xseq += 2;
    g->best = *key;
    g->offered = true;
    return BCM_OK;
}

bcm_status bcm_farness_all(bcm_graph_t g, const bcm_options* opt, uint64_t* farness, uint32_t* reach,
                           bcm_stats* stats) {
    t_err.clear();
    auto t0 = std::chrono::steady_clock::now();
    uint64_t l0 = g_launches.load();
    if (!g) return fail(BCM_ERR_INVALID, "graph is NULL");
    if (g->pend.active) return fail(BCM_ERR_INVALID, "a run on this graph has not been finished");
    if (!farness || !reach) return fail(BCM_ERR_INVALID, "output pointer is NULL");
    double pms = 0;
    bcm_status st = preprocess(g, &pms);
    if (st) return st;
    Cfg c;
    if ((st = resolve(g, opt, &c))) return st;
    unsigned long long sv[ST_COUNT] = {0}, wv[ST_COUNT] = {0};
    RunTimes rt;
    if (g->n > 0) {
        if ((st = start_run(g, c, 0, true, nullptr, farness, reach))) return st;
        g->pend.l0 = l0;
        g->pend.pms = pms;
        g->pend.t0 = t0;
        if ((st = finish_run(g, true, sv, wv, &rt))) return st;
        fill_run_stats(stats, g, sv, wv, rt);
    } else if (stats) {
        g->pend.l0 = l0;
        g->pend.pms = pms;
        g->pend.t0 = t0;
        g->pend.plain = false;
        fill_run_stats(stats, g, sv, wv, rt);
    }
    return BCM_OK;
}

bcm_status bcm_trace(bcm_graph_t g, uint64_t* records, uint32_t cap, uint32_t* count) {
    t_err.clear();
    if (!g) return fail(BCM_ERR_INVALID, "graph is NULL");
    if (g->pend.active) return fail(BCM_ERR_INVALID, "a run on this graph has not been finished");
    if (!count || (cap && !records)) return fail(BCM_ERR_INVALID, "output pointer is NULL");
    *count = g->trace_n;
    uint32_t have = g->trace_n < kTraceCap ? g->trace_n : kTraceCap;
    uint32_t nrec = have < cap ? have : cap;
    if (nrec && g->d_trace) {
        CU(cudaMemcpyAsync(records, g->d_trace, (size_t)nrec * 4 * sizeof(u64), cudaMemcpyDeviceToHost, g->stream),
           "trace copy");
        CU(cudaStreamSynchronize(g->stream), "trace copy");
    }
    return BCM_OK;
}

bcm_status bcm_graph_trim(bcm_graph_t g) {
    t_err.clear();
    if (!g) return fail(BCM_ERR_INVALID, "graph is NULL");
    if (g->pend.active) return fail(BCM_ERR_INVALID, "a run on this graph has not been finished");
    CU(g->stream ? cudaStreamSynchronize(g->stream) : cudaDeviceSynchronize(), "synchronize");
    region_release(g->slots, true);
    for (void* b : {(void*)g->d_plain, (void*)g->d_far, (void*)g->d_reach, (void*)g->d_trace, (void*)g->d_defer,
                    (void*)g->d_shard, (void*)g->d_surv})
        buf_put(b);
    g->d_surv = nullptr;
    g->d_defer = nullptr;
    g->d_shard = nullptr;
    g->d_plain = nullptr;
    g->d_far = nullptr;
    g->d_reach = nullptr;
    g->d_trace = nullptr;
    g->trace_n = 0;
    return BCM_OK;
}

bcm_status bcm_topk_merge(const uint32_t* ids, const uint64_t* farness, const uint32_t* reach, uint32_t count,
                          uint32_t k, uint32_t* out_ids, uint64_t* out_far, uint32_t* out_reach,
                          uint32_t* written) {
    t_err.clear();
    if (k == 0) return fail(BCM_ERR_INVALID, "k must be at least 1");
    if (!written || (count && (!ids || !farness || !reach)) || !out_ids || !out_far || !out_reach)
        return fail(BCM_ERR_INVALID, "a pointer argument is NULL");
    std::vector<uint32_t> idx;
    try {
        idx.resize(count);
    } catch (...) {
        return fail(BCM_ERR_OOM, "host allocation");
    }
    uint32_t used = 0;
    for (uint32_t i = 0; i < count; ++i)
        if (ids[i] != 0xffffffffu) idx[used++] = i;   // padding of a shard list that holds fewer than k
    idx.resize(used);
    // (N, F) = ((r-1)^2, f), or (0, 1) when r <= 1; a before b iff
    // N_a F_b > N_b F_a, or equal and id_a < id_b
    auto key = [&](uint32_t i, unsigned __int128& N, unsigned __int128& F) {
        if (reach[i] <= 1) { N = 0; F = 1; return; }
        const uint64_t r1 = reach[i] - 1;
        N = (unsigned __int128)r1 * r1;
        F = farness[i];
    };
    auto before = [&](uint32_t a, uint32_t b) {
        unsigned __int128 Na, Fa, Nb, Fb;
        key(a, Na, Fa);
        key(b, Nb, Fb);
        // N < 2^60 and F < 2^62, so the products fit in 128 bits
        const unsigned __int128 l = Na * Fb, r = Nb * Fa;
        if (l != r) return l > r;
        return ids[a] < ids[b];
    };
    const uint32_t w = k < used ? k : used;
    std::partial_sort(idx.begin(), idx.begin() + w, idx.end(), before);
    for (uint32_t i = 0; i < w; ++i) {
        out_ids[i] = ids[idx[i]];
        out_far[i] = farness[idx[i]];
        out_reach[i] = reach[idx[i]];
    }
    *written = w;
    return BCM_OK;
}

// --------------------------------------------------------------- batches
struct bcm_batch {
    cudaGraphExec_t exec = nullptr;
    cudaStream_t stream = nullptr;
    std::vector<bcm_graph*> graphs;
    std::vector<uint32_t> kk;     // entries each run must hold
};

static bcm_status batch_fail(bcm_batch* b, bcm_status st) {
    if (b) {
        if (b->exec) cudaGraphExecDestroy(b->exec);
        delete b;
    }
    return st;
}

bcm_status bcm_batch_create(bcm_graph_t* graphs, uint32_t count, const uint32_t* k, const bcm_options* opt,
                            void* stream, uint32_t* const* ids, uint64_t* const* farness, uint32_t* const* reach,
                            bcm_batch_t* out) {
    t_err.clear();
    if (!out || !graphs || !k || !ids || !farness || !reach || count == 0)
        return fail(BCM_ERR_INVALID, "a pointer argument is NULL or count is 0");
    *out = nullptr;
    bcm_options o{};
    if (opt) o = *opt;
    if (!(o.flags & BCM_OUT_DEVICE)) return fail(BCM_ERR_INVALID, "batch outputs must be device memory (BCM_OUT_DEVICE)");
    if (o.flags & (BCM_PLAIN | BCM_TRACE | BCM_GRID_ONLY) || o.shard_count > 1)
        return fail(BCM_ERR_UNSUPPORTED, "plain, traced, grid-only and sharded runs cannot be batched");
    bcm_batch* b = new (std::nothrow) bcm_batch();
    if (!b) return fail(BCM_ERR_OOM, "host allocation");
    b->stream = (cudaStream_t)stream;
    std::vector<Cfg> cfg(count);
    // every run once, outside the capture: preprocessing, workspaces and
    // buffers are allocated here, and each run is checked
    for (uint32_t i = 0; i < count; ++i) {
        bcm_graph* g = graphs[i];
        if (!g || !ids[i] || !farness[i] || !reach[i]) {
            fail(BCM_ERR_INVALID, "graph or output %u is NULL", i);
            return batch_fail(b, BCM_ERR_INVALID);
        }
        if (g->pend.active) {
            fail(BCM_ERR_INVALID, "graph %u has a run that has not been finished", i);
            return batch_fail(b, BCM_ERR_INVALID);
        }
        if (k[i] < 1 || k[i] > 1024) {
            fail(BCM_ERR_INVALID, "k[%u] = %u: must be in 1..1024", i, k[i]);
            return batch_fail(b, BCM_ERR_INVALID);
        }
        bcm_status st = preprocess(g, nullptr);
        if (st) return batch_fail(b, st);
        if ((st = resolve(g, &o, &cfg[i]))) return batch_fail(b, st);
        // the batch holds no cooperative launch: only graphs below the
        // grid-wide threshold, whose runs are a seed wave, the prefilter and
        // per-CTA waves
        if ((uint64_t)g->n * cfg[i].grid_W >= cfg[i].heavy_words || g->n == 0) {
            fail(BCM_ERR_UNSUPPORTED, "graph %u (n = %u) is too large (or empty) for a batch; use bcm_topk", i, g->n);
            return batch_fail(b, BCM_ERR_UNSUPPORTED);
        }
        cudaStream_t keep = g->stream;
        g->stream = b->stream;
        unsigned long long sv[ST_COUNT], wv[ST_COUNT];
        RunTimes rt;
        st = start_run(g, cfg[i], k[i], false, ids[i], farness[i], reach[i]);
        if (st == BCM_OK) st = finish_run(g, true, sv, wv, &rt);
        g->stream = keep;
        if (st) return batch_fail(b, st);
        b->graphs.push_back(g);
        b->kk.push_back(k[i] < g->n ? k[i] : g->n);
    }
    // record the runs on kBatchBranches parallel branches (graph i on branch
    // i mod kBatchBranches): streams forked from the batch stream by an event
    // and joined back, so the recorded graph runs independent graphs at once
    constexpr uint32_t kBatchBranches = 16;
    const uint32_t nbr = count < kBatchBranches ? count : kBatchBranches;
    std::vector<cudaStream_t> br(nbr, nullptr);
    std::vector<cudaEvent_t> ev(nbr + 1, nullptr);
    bcm_status st = BCM_OK;
    for (uint32_t j = 0; j < nbr && st == BCM_OK; ++j)
        if (cudaStreamCreateWithFlags(&br[j], cudaStreamNonBlocking) != cudaSuccess) st = fail(BCM_ERR_CUDA, "stream");
    for (uint32_t j = 0; j <= nbr && st == BCM_OK; ++j)
        if (cudaEventCreateWithFlags(&ev[j], cudaEventDisableTiming) != cudaSuccess) st = fail(BCM_ERR_CUDA, "event");
    cudaError_t e = cudaSuccess;
    if (st == BCM_OK) {
        e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) st = cuda_fail(e, "stream capture");
    }
    const bool capturing = st == BCM_OK;
    if (capturing) {
        cudaEventRecord(ev[nbr], b->stream);                 // fork
        for (uint32_t j = 0; j < nbr; ++j) cudaStreamWaitEvent(br[j], ev[nbr], 0);
    }
    for (uint32_t i = 0; i < count && st == BCM_OK; ++i) {
        bcm_graph* g = graphs[i];
        cudaStream_t keep = g->stream;
        g->stream = br[i % nbr];
        st = start_run(g, cfg[i], k[i], false, ids[i], farness[i], reach[i]);
        g->pend.active = false;   // recorded, not running
        g->stream = keep;
    }
    if (capturing) {
        for (uint32_t j = 0; j < nbr; ++j) {                // join
            cudaEventRecord(ev[j], br[j]);
            cudaStreamWaitEvent(b->stream, ev[j], 0);
        }
    }
    cudaGraph_t graph = nullptr;
    if (capturing) e = cudaStreamEndCapture(b->stream, &graph);
    if (st == BCM_OK && e != cudaSuccess) st = cuda_fail(e, "stream capture");
    if (st == BCM_OK) {
        e = cudaGraphInstantiate(&b->exec, graph, 0);
        if (e != cudaSuccess) st = cuda_fail(e, "graph instantiation");
    }
    if (graph) cudaGraphDestroy(graph);
    for (auto x : br)
        if (x) cudaStreamDestroy(x);
    for (auto x : ev)
        if (x) cudaEventDestroy(x);
    if (st) return batch_fail(b, st);
    *out = b;
    return BCM_OK;
}

bcm_status bcm_batch_run(bcm_batch_t b, int wait) {
    t_err.clear();
    if (!b) return fail(BCM_ERR_INVALID, "batch is NULL");
    CU(cudaGraphLaunch(b->exec, b->stream), "graph launch");
    if (!wait) return BCM_OK;
    CU(cudaStreamSynchronize(b->stream), "batch run");
    for (size_t i = 0; i < b->graphs.size(); ++i) {
        const HostBlock* h = b->graphs[i]->h;
        if (h->err) {
            region_release(b->graphs[i]->slots, false);
            bcm_status st = check_dev_err(h->err);
            return fail(st, "graph %zu of the batch: %s", i, t_err.c_str());
        }
        if (h->topk_count != b->kk[i])
            return fail(BCM_ERR_CUDA, "graph %zu of the batch: top-k holds %u entries, expected %u", i, h->topk_count,
                        b->kk[i]);
    }
    return BCM_OK;
}

bcm_status bcm_batch_destroy(bcm_batch_t b) {
    if (!b) return BCM_OK;
    if (b->stream) cudaStreamSynchronize(b->stream);
    if (b->exec) cudaGraphExecDestroy(b->exec);
    delete b;
    return BCM_OK;
}

uint64_t bcm_workspace_bytes(bcm_graph_t g, const bcm_options* opt) {
    if (!g) return 0;
    if (!g->preprocessed && preprocess(g, nullptr) != BCM_OK) return 0;   // the default kernels depend on it
    Cfg c;
    if (resolve(g, opt, &c)) return 0;
    return (uint64_t)region_bytes(g, c) + sizeof(Aux) + (uint64_t)g->n * 12;
}

}  // extern "C"
