// Internal interfaces between the library's translation units (not part of
// the C-ABI).  Kernels are launched only through the functions declared here.
#pragma once
#include <cstddef>
#include <cstdint>
#include <cuda_runtime.h>

#include "common.cuh"

namespace bcm {

// Counters accumulated by the wave kernels, in this order.
enum Stat {
    ST_MVIS = 0,        // arcs scanned, counted per source (Section 3.1's m_vis)
    ST_DISC,            // (source, vertex) discoveries
    ST_COMPLETED,       // sources whose BFS ran to the end
    ST_CUT,             // sources stopped by the bound
    ST_WAVES,           // waves run
    ST_LEVELS,          // levels expanded, summed over waves
    ST_MAXLEVEL,        // deepest level reached
    ST_ENTRIES,         // frontier words expanded (level >= 1)
    ST_ARCWORDS,        // (arc, frontier word) pairs scanned
    ST_DISCWORDS,       // frontier words created (first discovery in a level)
    ST_CLEARED,         // vertex words cleared at wave ends
    ST_DEFERRED,        // sources a per-CTA wave handed to the grid-wide pass
    ST_PULLENTRIES,     // frontier words of pulled levels (also in ST_ENTRIES)
    ST_COUNT
};

// The graph as the kernels see it.  Offsets are narrowed to 32 bits (m < 2^32).
struct GraphDev {
    uint32_t n;
    uint64_t m;
    const uint32_t* rp;      // [n+1]
    const uint32_t* col;     // [m]
    const uint32_t* order;   // [n] vertices by (degree desc, id asc)
    const uint32_t* xlo;     // [n] r(v) (undirected) or alpha(v)
    const uint32_t* xhi;     // [n] r(v) (undirected) or omega(v)
    const uint32_t* rrp;     // in-arcs CSR (the graph itself when undirected)
    const uint32_t* rcol;
};

// Per-slot working memory of one MS-BFS wave with W words (64W sources) per
// vertex, for n vertices (or table entries).  Word index of (entry v, word g)
// is v*W + g; each word has a 32-byte record (vis, key, F[0], F[1]), then two
// frontier lists and a clear log of 4-byte word indices.
constexpr size_t slot_bytes(uint32_t n, int W) {
    size_t nw = (size_t)n * W;
    size_t b = nw * (4 * sizeof(uint64_t) + 3 * sizeof(uint32_t));
    return (b + 255) & ~(size_t)255;
}

// One-source-per-CTA slot (k_sparse): a visited bitmap of one bit per vertex,
// the log of its words that became non-zero, then two queues of qcap
// entries each (a frontier vertex's first arc and degree, 8 bytes).
__host__ __device__ constexpr size_t al256(size_t b) { return (b + 255) & ~(size_t)255; }
__host__ __device__ constexpr size_t sparse_bitmap_bytes(uint32_t n) { return al256(((size_t)n + 31) / 32 * sizeof(uint32_t)); }
__host__ __device__ constexpr size_t sparse_slot_bytes(uint32_t n, uint32_t qcap) {
    return 2 * sparse_bitmap_bytes(n) + 2 * al256((size_t)qcap * 2 * sizeof(uint32_t));
}

// The grid kernel's per-lane level counters are summed in kCntCopies copies
// (block b adds into copy b % kCntCopies, and every block sums the copies
// after the barrier): 304 blocks adding into one set of 512 words made the
// adds queue on a few cache lines.
constexpr uint32_t kCntCopies = 16;
constexpr uint32_t kCntParity = kCntCopies * 512;   // u32 per level parity

// A frontier word whose vertex has many out-arcs, queued so that every warp
// can take a share of its arcs.
struct HeavyEntry {
    unsigned long long F;   // live frontier lanes of the word
    uint32_t beg, deg;      // the vertex's arcs
    uint32_t g, pad;        // word group
};

struct WaveParams {
    GraphDev g;
    uint32_t footnote;       // undirected: gamma~ uses deg(u)-1 for d >= 1
    uint32_t exhaustive;     // 1: no cut, write farness/reach of every source
    const uint32_t* sources; // the source queue: the degree order, or the deferred sources
    uint32_t* head;          // next position in `sources` (atomic)
    uint32_t n_end;          // sources are sources[*head .. n_end)
    TopK topk;
    unsigned long long* out_far;   // exhaustive outputs, indexed by vertex id
    uint32_t* out_reach;
    char* slot_base;         // CTA i: slot_base + i * slot_stride
    size_t slot_stride;
    // per-CTA slots: vertex tables of cta_entries entries (cta_entries = n
    // and tab_shift = 0: dense, vertex x is entry x; else hashed, cta_entries
    // = 2^(32 - tab_shift), and a wave making more than tab_limit entries is
    // given up and deferred)
    uint32_t cta_entries;
    uint32_t tab_shift;
    uint32_t tab_limit;
    // one-source-per-CTA kernel: entries of each vertex queue (a longer
    // frontier defers the source)
    uint32_t sparse_qcap;
    char* seed_base;         // the grid kernel's own slot (4 words per vertex)
    unsigned long long* stats;   // [ST_COUNT]
    int* err;
    unsigned long long lock_limit_ns;
    unsigned long long barrier_limit_ns;
    // grid-wide (seed / plain) kernels only
    GridBarrier* bar;
    uint32_t* gcnt;          // [2][kCntCopies][2][256] per-lane level counters (gamma, degree sum) by
                             // level parity, in copies that blocks add into by blockIdx % kCntCopies
    uint32_t* glist_n;       // [2] frontier list sizes
    uint32_t* glog_n;        // [1] cleared-word log size
    uint32_t* gchunk;        // [2] chunk counters of the frontier lists
    unsigned long long* garc; // [2] out-arcs of the frontier lists' words
    HeavyEntry* gheavy;      // heavy entries of the level being pushed
    uint32_t* gheavy_n;
    uint32_t gheavy_cap;
    uint32_t max_grid_waves;  // grid kernel: at most this many waves
    uint64_t heavy_words;   // grid kernel: a wave with fewer frontier words in total is light
    uint32_t pull_div;      // grid kernel: pull a level whose frontier words have >= n*W/pull_div out-arcs (0: never)
    uint32_t all_pull;      // grid kernel: pull every level after the first (a check of the pull path)
    // per-CTA kernel: a wave about to expand a level of at least defer_words
    // words, or of at least 8 * defer_words out-arcs, is given up and its
    // live sources appended to defer_src (0: never)
    uint32_t defer_words;
    uint32_t* defer_n;
    uint32_t* defer_src;
    // per-CTA kernel: each CTA stops after this many waves (0: when the queue is empty)
    uint32_t max_cta_waves;
    // when set, the sources end at *n_end_dev (read at launch)
    const uint32_t* n_end_dev;
    // optional trace: records of 4 u64 (layout in include/bcm.h, bcm_trace), NULL when off
    unsigned long long* trace;
    uint32_t trace_cap;      // records
    uint32_t* trace_n;       // records written (may exceed trace_cap; the excess is dropped)
    uint32_t trace_lanes;    // also record every lane's level state and end (needs trace)
    uint32_t nocut;          // top-k runs: never stop a source (every BFS runs to its end)
    Threshold* snap;         // grid-wide and plain kernels: the threshold all blocks cut with (see store_snapshot)
};

// Trace record kinds (bits 60..63 of a record's second word).
enum TraceKind { TR_GRID_LEVEL = 0, TR_GRID_WAVE = 1, TR_CTA_WAVE = 2, TR_LANE_LEVEL = 3, TR_LANE_END = 4 };

// ---- preproc.cu
int launch_validate(const uint64_t* rp64, const uint32_t* col, uint32_t n, uint64_t m, int* err,
                    cudaStream_t s);
int launch_narrow_offsets(const uint64_t* rp64, uint32_t* rp32, uint32_t n, cudaStream_t s);
// *not_simple |= 1 unless every row is strictly increasing and free of its own vertex
// (scratch: simple_check_scratch_bytes(m))
size_t simple_check_scratch_bytes(uint64_t m);
int launch_simple_check(const uint32_t* rp32, const uint32_t* col, uint32_t n, uint64_t m, int* not_simple,
                        void* scratch, cudaStream_t s);
int launch_cc_reach(const uint32_t* rp, const uint32_t* col, uint32_t n, uint32_t* parent,
                    uint32_t* size, uint32_t* xlo, uint32_t* xhi, int* err, cudaStream_t s);
int launch_degree_order(const uint32_t* rp, uint32_t n, uint32_t* order, void* scratch,
                        size_t scratch_bytes, cudaStream_t s, uint32_t* max_degree = nullptr);
size_t degree_order_scratch_bytes(uint32_t n);
// stable LSD radix sort of (key, value) pairs on the low `bits` of the key
size_t radix_scratch_bytes(size_t count);
int radix_sort_pairs_u32(uint32_t* keys, uint32_t* vals, uint32_t* keys_tmp, uint32_t* vals_tmp,
                         size_t count, int bits, void* scratch, cudaStream_t s, bool* result_in_tmp);
int radix_sort_u64(uint64_t* keys, uint64_t* keys_tmp, size_t count, int bits, void* scratch,
                   cudaStream_t s, bool* result_in_tmp);
// exclusive scan of u32 counts into u32 offsets (out may alias in); returns total via *total_dev
size_t scan_scratch_bytes(size_t count);
int exclusive_scan_u32(const uint32_t* in, uint32_t* out, size_t count, uint32_t* total_dev,
                       void* scratch, cudaStream_t s);

// component labels: flags[v] = (parent[v] == v); parent[v] = rank[parent[v]]
int launch_root_flags(const uint32_t* parent, uint32_t n, uint32_t* flags, cudaStream_t s);
int launch_relabel(uint32_t* parent, const uint32_t* rank, uint32_t n, cudaStream_t s);

// ---- scc.cu
struct SccResult { uint32_t n_scc; };
size_t scc_scratch_bytes(uint32_t n, uint64_t m);
int launch_reverse_csr(const uint32_t* rp, const uint32_t* col, uint32_t n, uint64_t m, uint32_t* rrp,
                       uint32_t* rcol, void* scratch, size_t scratch_bytes, cudaStream_t s);
int launch_scc_bounds(const uint32_t* rp, const uint32_t* col, const uint32_t* rrp, const uint32_t* rcol,
                      uint32_t n, uint64_t m, uint32_t* comp, uint32_t* xlo, uint32_t* xhi, uint32_t* n_scc_host,
                      int refine, void* scratch, size_t scratch_bytes, int* err, cudaStream_t s);

// ---- msbfs.cu
int launch_grid_waves(const WaveParams& p, int W, int blocks, int threads, cudaStream_t s);
int launch_cta_waves(const WaveParams& p, int W, int blocks, int threads, cudaStream_t s);
// level-0/1 stopping rule for sources p.sources[*p.head .. p.n_end) of a simple graph;
// the sources it cannot stop are appended to out (count in *out_n)
int launch_prefilter(const WaveParams& p, uint32_t* out, uint32_t* out_n, cudaStream_t s);
int launch_plain_source(const WaveParams& p, uint32_t it, uint32_t* stamp, uint32_t* lists,
                        int blocks, int threads, cudaStream_t s);

int max_coop_blocks(int kind, int W, int threads);   // kind 0 grid waves, 1 plain
int cta_blocks_per_sm(int W, int threads);
// one source per CTA (high-diameter graphs): sources p.sources[*p.head .. n_end)
int launch_sparse(const WaveParams& p, int blocks, int threads, cudaStream_t s);
int sparse_blocks_per_sm(int threads);

// launch bookkeeping (api.cu)
void note_launch(int count = 1);
// sets the calling thread's bcm_last_error() message (api.cu)
void set_error_message(const char* msg);

}  // namespace bcm
