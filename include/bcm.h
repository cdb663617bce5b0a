/*
 * libbcm -- exact top-k closeness centrality on one GPU.
 *
 * Method: Borassi, Crescenzi, Marino, "Fast and Simple Computation of Top-k
 * Closeness Centralities" (arXiv 1507.01490), called BCM below.
 *
 *   closeness   c(v) = (r(v)-1)^2 / ((n-1) f(v))                 (Section 1)
 *               r(v) = |R(v)|, the vertices reachable from v (v included);
 *               f(v) = sum of d(v,w) over R(v), the farness.
 *   ranking     by c(v) descending, equal values by vertex id ascending;
 *               r(v) = 1 gives c(v) = 0.
 *   BCM         Algorithm 1: vertices in decreasing degree order (outdeg on
 *               digraphs, equal degrees by id), each one's BFS cut by
 *               BFSCut (Algorithm 2) once Lemma 1's farness lower bound
 *               (Lemma 2's for digraphs, with the alpha/omega bounds of
 *               Section 2.3) shows it cannot enter the current top-k.
 *
 * Results are exact: farness is an integer, every comparison is done in
 * 128-bit integer arithmetic, and the top-k is the one the textbook
 * algorithm (one BFS per vertex) returns.
 *
 * Conventions
 *   - Graphs are CSR: row_ptr[n+1] (uint64), col[m] (uint32).  Undirected
 *     graphs store both arcs of every edge (m counts arcs).  Self-loops and
 *     repeated arcs are accepted; they change no distance.  Supported sizes:
 *     n < 2^30 and m < 2^32.
 *   - The caller owns every array it passes; the library copies inputs and
 *     writes outputs into caller-allocated memory.  Output pointers are host
 *     memory unless BCM_OUT_DEVICE is set (then they are device memory on the
 *     current device).
 *   - Calls are synchronous: they return after the work on the graph's
 *     stream has finished, except bcm_topk_start, which returns once the
 *     run is enqueued (bcm_topk_finish completes it).
 *   - Every function returns a bcm_status; on failure bcm_last_error()
 *     returns a message for the calling thread.  No C++ exception crosses
 *     this interface.
 *   - A handle must not be used by two threads at once.
 *   - Every wait inside a kernel (grid barrier, top-k lock) has a time
 *     limit; when one runs out the call returns BCM_ERR_TIMEOUT and the
 *     CUDA context stays usable.
 */
#ifndef BCM_H
#define BCM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct bcm_graph* bcm_graph_t;

typedef enum {
    BCM_OK = 0,
    BCM_ERR_INVALID = 1,        /* bad argument or malformed CSR */
    BCM_ERR_NOT_SYMMETRIC = 2,  /* undirected graph whose arcs are not paired */
    BCM_ERR_OOM = 3,            /* device memory exhausted */
    BCM_ERR_CUDA = 4,           /* a CUDA call failed (message has the CUDA error) */
    BCM_ERR_TIMEOUT = 5,        /* a bounded in-kernel wait ran out */
    BCM_ERR_UNSUPPORTED = 6,    /* size or option outside the supported range */
    BCM_ERR_PENDING = 7         /* bcm_topk_finish(wait = 0): the run has not finished yet */
} bcm_status;

/* bcm_options.flags */
#define BCM_OUT_DEVICE    0x1u  /* output pointers are device memory */
#define BCM_NO_FOOTNOTE   0x2u  /* undirected: bound gamma_{d+1} by sum of deg(u), not deg(u)-1
                                   (the footnote of Section 2.2 tightens; results are the same) */
#define BCM_PLAIN         0x4u  /* bcm_topk: one source per kernel launch (comparison baseline) */
#define BCM_CTA_ONLY      0x8u  /* run every wave on the per-CTA kernel (no grid-wide waves) */
#define BCM_CHECK_SYMMETRIC 0x10u /* bcm_graph_create: verify undirected arcs are paired */
#define BCM_GRID_ONLY     0x20u /* run every wave on the grid-wide kernel */
#define BCM_NO_PULL       0x40u /* grid-wide waves expand every level by push */
#define BCM_PLAIN_BOUNDS  0x80u /* bcm_graph_create, digraphs: alpha/omega from the plain programme of
                                   Section 2.3, without its biggest-SCC refinement (results are the same) */
#define BCM_TRACE         0x100u /* record the run's trace (read it with bcm_trace) */
#define BCM_NO_DEFER      0x200u /* per-CTA waves never hand their sources to the grid-wide pass */
#define BCM_NO_PREFILTER  0x400u /* no level-0/1 prefilter before the per-CTA waves (it runs on simple
                                    graphs -- sorted rows, no repeated arc, no self-loop -- after the
                                    grid-wide waves; results are the same) */
#define BCM_NO_CUT        0x800u /* bcm_topk: no source is ever stopped by the bound, every BFS runs to its
                                    end (Algorithm 1 without BFSCut is the textbook algorithm of Section
                                    2.1); the top-k is the same -- a check of the cut, not a fast path */
#define BCM_TRACE_LANES   0x1000u /* with BCM_TRACE: also record every lane's state at every level and how
                                     it ended (record kinds 3 and 4 of bcm_trace); meant for small graphs */
#define BCM_ALL_PULL      0x2000u /* grid-wide waves expand every level after the first by pull (a check of
                                     the pull path; results are the same) */
#define BCM_SPARSE        0x4000u /* one source per CTA instead of bit-lane waves: a visited bitmap and
                                     vertex queues (for graphs whose sources' searches share no frontier).
                                     The default on undirected graphs of n >= 4096 and largest degree <= 8
                                     (lattices, meshes); with it there are no grid-wide waves unless
                                     BCM_GRID_ONLY.  Results are the same */
#define BCM_NO_SPARSE     0x8000u /* bit-lane waves whatever the graph */

/* Sources are taken from the degree order in waves.  Waves run first on a
 * grid-wide kernel (all CTAs on one wave) while they are heavy, then on a
 * per-CTA kernel (each CTA its own wave).  A grid wave is narrow when its
 * frontiers averaged fewer than heavy_words (vertex, 64-lane word) entries
 * per level; the first narrow one ends the grid phase (a graph whose
 * n * grid_lanes/64 is below heavy_words has no heavy wave, and its top-k
 * runs skip the grid kernel).  A per-CTA wave that turns out wide after all
 * is stopped and its sources run again on the grid kernel after the
 * per-CTA phase (see defer_words).  Exhaustive runs stay on the grid
 * kernel (with BCM_SPARSE, on the one-source kernel).  Levels of grid waves
 * run by push (each frontier vertex
 * sets its lanes' bits in its out-neighbours) or, when the frontier's arcs
 * are a large share of the graph's, by pull (each vertex with lanes still
 * to reach gathers them from its in-neighbours' frontier bits, with no
 * atomics). */
typedef struct {
    uint32_t lanes;           /* sources per per-CTA wave: 64, 128 or 256; 0 = 64 */
    uint32_t grid_lanes;      /* sources per grid-wide wave: 64, 128 or 256; 0 = 128 */
    uint32_t flags;           /* BCM_* flags above */
    uint32_t blocks;          /* CTAs of the per-CTA kernel; 0 = all that fit on the GPU, at most
                                 one per wave of sources (ceil(n / lanes)).  Each holds a slot of
                                 44 E lanes/64 bytes, E its table's entries (cta_table); with the
                                 one-source kernel (BCM_SPARSE) 8 ceil(n/32) + 16 Q bytes, Q =
                                 min(n, 2^18) where an overflowing source can be deferred, else n */
    uint32_t threads;         /* threads per CTA of the per-CTA kernel: 256, 512 or 1024; 0 = 512
                                 (the one-source kernel, BCM_SPARSE: also 128; 0 = 256) */
    uint32_t heavy_words;     /* see above; 0 = default (4 per warp of the grid) */
    uint32_t pull_div;        /* a grid-wave level is expanded by pull when the out-arcs of its
                                 frontier's (vertex, word) entries number at least n*W/pull_div
                                 (W = grid_lanes/64; 0 = default, 32) and at least a quarter of the
                                 pull's estimated cost, n/4 + (n - n_min) m/n, n_min the fewest vertices
                                 a live source has reached (so a lattice's thin frontiers stay push) */
    uint32_t defer_words;     /* a per-CTA wave about to expand a level of this many words (or of 8x
                                 as many out-arcs) stops and hands its live sources to a second
                                 grid-wide pass, which runs them from the start; 0 = default
                                 (heavy_words) */
    uint64_t wait_limit_ns;   /* limit of every in-kernel wait; 0 = default (20 s) */
    uint32_t shard_index;     /* bcm_topk over one shard of the sources (several GPUs, one graph):  */
    uint32_t shard_count;     /* the positions p of the degree order with (p / 64) % shard_count ==
                                 shard_index; the result is that shard's own top-k, min(k, shard
                                 size) entries, and bcm_topk_merge of every shard's lists is the
                                 graph's top-k.  shard_count 0 or 1 = every source */
    uint32_t cta_table;       /* entries of a per-CTA wave's vertex table.  Where the per-CTA
                                 waves can defer (top-k runs, no BCM_CTA_ONLY / BCM_GRID_ONLY /
                                 BCM_NO_DEFER) and n is larger, the table is hashed with this many
                                 entries (a power of two >= 1024; 0 = default, n/8 rounded up to a
                                 power of two within [65536, 2^21]), and a wave
                                 that makes more than half as many entries is deferred like a wide
                                 one; otherwise (or with a value >= n) it is dense, n entries.
                                 Results are the same either way */
} bcm_options;

typedef struct {
    uint64_t m_vis;           /* arcs scanned, counted once per source scanning them
                                 (Section 3.1's visited arcs) */
    uint64_t visits;          /* (source, vertex) pairs reached */
    uint64_t completed;       /* sources whose BFS ran to the end */
    uint64_t cut;             /* sources stopped by the bound */
    uint64_t waves;           /* waves (groups of sources expanded together) */
    uint64_t levels;          /* BFS levels expanded, summed over waves */
    uint64_t max_level;       /* deepest level expanded */
    uint64_t frontier_words;  /* (vertex, 64-lane word) frontier entries expanded */
    uint64_t arc_words;       /* (arc, frontier word) pairs scanned */
    uint64_t new_words;       /* frontier words created */
    uint64_t cleared_words;   /* words reset between waves */
    uint64_t launches;        /* kernels this call launched */
    double   kernel_ms;       /* device time of the BFS kernels (CUDA events) */
    double   preprocess_ms;   /* device time of preprocessing done by this call */
    double   total_ms;        /* wall time of the call */
    double   seed_ms;         /* device time of the grid-wide waves (or of the plain launches) */
    double   wave_ms;         /* device time of the per-CTA wave kernel (or of the one-source kernel) */
    uint64_t wave_bytes;      /* algorithmic bytes the per-CTA wave kernel moved: 20 per source
                                 started, 28 per frontier word, 12 per (arc, frontier word), 32 per
                                 new frontier word, 28 per cleared word; the one-source kernel: 20 per
                                 source, 12 per frontier vertex, 8 per arc, 16 per discovered vertex,
                                 12 per cleared bitmap word */
    uint64_t grid_waves;      /* waves run by the grid-wide kernel */
    uint64_t grid_levels;     /* levels those waves expanded */
    uint64_t grid_bytes;      /* algorithmic bytes of the grid-wide kernel (same unit costs) */
    uint64_t deferred;        /* sources per-CTA waves handed to the grid-wide pass */
    uint64_t sparse;          /* sources the one-source-per-CTA kernel ran (BCM_SPARSE), else 0 */
} bcm_stats;

/*
 * bcm_graph_create -- copy a CSR graph to the device and validate it.
 *   row_ptr, col : CSR arrays (host memory, or device memory if
 *                  ptr_on_device != 0).  Not retained.
 *   n, m         : vertex and arc counts.
 *   directed     : 0 = undirected (both arcs of each edge present), 1 = directed.
 *   stream       : cudaStream_t used for all work on this graph (NULL = legacy default).
 *   flags        : BCM_CHECK_SYMMETRIC, BCM_PLAIN_BOUNDS, or 0.
 *   out          : receives the handle; release it with bcm_graph_destroy.
 * Errors: BCM_ERR_INVALID (NULL pointer, row_ptr not monotone from 0 to m,
 * a column >= n), BCM_ERR_NOT_SYMMETRIC, BCM_ERR_UNSUPPORTED (n >= 2^30 or
 * m >= 2^32), BCM_ERR_OOM, BCM_ERR_CUDA.  Preprocessing (Algorithm 1's
 * PreProcessing and the degree order) runs lazily on first use.
 */
bcm_status bcm_graph_create(const uint64_t* row_ptr, const uint32_t* col, uint32_t n, uint64_t m,
                            int directed, int ptr_on_device, void* stream, uint32_t flags,
                            bcm_graph_t* out);

/* bcm_graph_destroy -- free the handle and its device memory (NULL is a no-op). */
bcm_status bcm_graph_destroy(bcm_graph_t g);

/*
 * bcm_preprocess -- run PreProcessing now (Algorithm 1, first line):
 *   undirected: r(v) = size of v's connected component (Section 2.2);
 *   directed:   SCCs, the weighted SCC DAG and alpha(v) <= r(v) <= omega(v)
 *               (Section 2.3), omega held at n, with the section's
 *               biggest-SCC refinement (the largest SCC's reach measured,
 *               smallest member on ties) unless BCM_PLAIN_BOUNDS;
 * and the processing order (degree descending, id ascending; Section 2.1).
 * Idempotent.  Any output pointer may be NULL; when given, each receives n
 * uint32 values (host memory unless out_on_device):
 *   order : vertex ids in processing order;
 *   x_lo  : r(v) (undirected) or alpha(v);  x_hi : r(v) or omega(v).
 */
bcm_status bcm_preprocess(bcm_graph_t g, uint32_t* order, uint32_t* x_lo, uint32_t* x_hi,
                          int out_on_device);

/*
 * bcm_scc_bounds -- Section 1.3 / 2.3 for a directed graph: comp[v] (SCC
 * label in [0, n_scc), labels ordered by smallest member id), alpha[v],
 * omega[v] (n uint32 each) and the SCC count.  Any pointer may be NULL.
 * Undirected graphs: components play the role of SCCs and
 * alpha = omega = r.  Host memory unless out_on_device.
 */
bcm_status bcm_scc_bounds(bcm_graph_t g, uint32_t* comp, uint32_t* alpha, uint32_t* omega,
                          uint32_t* n_scc, int out_on_device);

/*
 * bcm_topk -- the k most central vertices (Algorithm 1).
 *   k      : 1 <= k <= 1024.  min(k, n) entries are written.
 *   opt    : NULL for defaults.
 *   ids, farness, reach : min(k, n) entries each, best first: vertex id,
 *            f(v) (uint64) and r(v) (uint32).
 *   stats  : NULL or receives counters and timings.
 * Errors: BCM_ERR_INVALID (k outside 1..1024, NULL outputs),
 * BCM_ERR_TIMEOUT, BCM_ERR_OOM, BCM_ERR_CUDA.
 */
bcm_status bcm_topk(bcm_graph_t g, uint32_t k, const bcm_options* opt, uint32_t* ids,
                    uint64_t* farness, uint32_t* reach, bcm_stats* stats);

/*
 * bcm_topk_start / bcm_topk_finish -- bcm_topk in two halves, for callers
 * that keep several graphs' runs in flight at once (each graph's work goes
 * to its own stream, so runs on different graphs overlap on the device).
 * bcm_topk_start takes bcm_topk's arguments, enqueues the run and the copies
 * of its results on the graph's stream and returns without waiting.  The
 * output arrays must stay valid until the run is finished; for the host
 * copies to be asynchronous they must be pinned host memory (pageable
 * memory works, but the copy then blocks the calling thread).  If the graph
 * has not been preprocessed yet, that happens first, synchronously.
 * bcm_topk_finish(wait = 1) waits for the run and returns its outcome, as
 * bcm_topk would, filling stats (may be NULL); with wait = 0 it returns
 * BCM_ERR_PENDING at once while the run is still going.  One run per graph:
 * starting another run, bcm_farness_all, bcm_trace or bcm_graph_trim before
 * the finish returns BCM_ERR_INVALID.  bcm_topk is start + finish(wait = 1).
 */
bcm_status bcm_topk_start(bcm_graph_t g, uint32_t k, const bcm_options* opt, uint32_t* ids,
                          uint64_t* farness, uint32_t* reach);
bcm_status bcm_topk_finish(bcm_graph_t g, int wait, bcm_stats* stats);

/*
 * bcm_key -- the rank key of one top-k entry, as the shards of one graph
 * exchange it (Section 2: the threads of the parallel version share the
 * current k-th value x_k):  N = (r-1)^2, F = f (N = 0, F = 1 when r = 1),
 * id = the vertex; valid = 0 means no key.  a ranks before b iff
 * N_a F_b > N_b F_a, or the products are equal and id_a < id_b.
 */
typedef struct {
    uint64_t N, F;
    uint32_t id, valid;
} bcm_key;

/*
 * bcm_topk_threshold -- a consistent snapshot of the k-th key the graph's
 * pending run has published so far (or of its last run's, once finished);
 * valid = 0 while it holds fewer than k entries.
 * bcm_topk_offer -- give the pending top-k run a key from outside: from then
 * on (at its next level) the run stops sources with the better of its own
 * k-th key and the best key offered.  Meant for the shards of one graph
 * (bcm_options.shard_*): the k-th key of any shard is a valid threshold for
 * all of them, because at least k vertices of the graph rank at or before
 * it.  A shard run that was offered a key returns the best of the sources it
 * did not stop, which still holds every member of the graph's top-k in its
 * shard, and may hold fewer than min(k, shard size) of them: the unused
 * entries are padding (id 0xFFFFFFFF, farness 0, reach 0), which
 * bcm_topk_merge skips.  An offer no better than an earlier one is ignored.
 * Both calls may be made from another thread while the run is pending (the
 * exception to the one-thread rule above); they use the graph's helper
 * stream, wait only for their own small copies, and do not wait for the run.
 * Errors: BCM_ERR_INVALID (NULL pointer; offer: no top-k run pending, or a
 * malformed key), BCM_ERR_CUDA.
 */
bcm_status bcm_topk_threshold(bcm_graph_t g, bcm_key* out);
bcm_status bcm_topk_offer(bcm_graph_t g, const bcm_key* key);

/*
 * bcm_trace -- the trace of the graph's last finished run made with
 * BCM_TRACE (none otherwise).  Up to cap records of 4 uint64 each are
 * copied to the host array records; *count receives how many records the
 * run wrote (the library keeps the first 65,536).  Record words:
 *   [0] time stamp (ns, the GPU's global timer)
 *   [1] kind << 60 | id << 32 | level, kind one of
 *       0  grid-wide level start  (id = wave; [2] frontier entries,
 *                                  [3] live lanes | 1 << 16 if pulled |
 *                                  out-arcs of the frontier's words << 20)
 *       1  grid-wide wave end     (id = wave; [2] words cleared,
 *                                  [3] frontier entries over the wave)
 *       2  per-CTA wave end       (id = CTA;  [2] words cleared,
 *                                  [3] the wave's start time stamp)
 *     and, with BCM_TRACE_LANES, per source v (id = v & 0xfffffff):
 *       3  lane at level d        (Table 1's quantities before the stopping
 *                                  rule is applied at level d: [2] f_d,
 *                                  [3] n_d | gamma~_{d+1} << 32)
 *       4  lane end               ([2] f_d, [3] n_d | 1 << 32 if the bound
 *                                  stopped the source at level d; 0 << 32
 *                                  if its BFS ended at level d, when
 *                                  f_d = f(v) and n_d = r(v))
 *     A source that runs twice (a per-CTA wave handing it to the grid-wide
 *     pass, or the level-0/1 prefilter before its wave) repeats its records.
 * Records of one kind are in time order only per wave or CTA.
 */
bcm_status bcm_trace(bcm_graph_t g, uint64_t* records, uint32_t cap, uint32_t* count);

/*
 * bcm_graph_trim -- give back the graph's run workspace (wave-kernel slots,
 * exhaustive outputs, plain-run buffers, trace): the slots go to a cache of
 * clean regions that other graphs' runs reuse, the rest is freed.  The CSR
 * and the preprocessing results stay.  The next run allocates again.
 */
bcm_status bcm_graph_trim(bcm_graph_t g);

/*
 * bcm_farness_all -- f(v) and r(v) of every vertex by a complete BFS from
 * each one (the textbook algorithm of Section 2.1, no cut), n entries each,
 * indexed by vertex id.  opt may be NULL.
 */
bcm_status bcm_farness_all(bcm_graph_t g, const bcm_options* opt, uint64_t* farness, uint32_t* reach,
                           bcm_stats* stats);

/*
 * bcm_farness_all_noalloc -- the same f(v) and r(v) as bcm_farness_all,
 * computed without allocating any memory.  The paper has no counterpart;
 * this serves callers that cannot allocate device memory when they need the
 * result: code under a host framework that owns all device memory, request
 * paths where an allocation's device synchronisation is not acceptable, and
 * programs with a fixed memory budget.
 *   row_ptr, col     : CSR in DEVICE memory (as for bcm_graph_create), not retained.
 *   n, m             : n <= 1,250,000 vertices (else BCM_ERR_UNSUPPORTED), m < 2^32.
 *   stream           : cudaStream_t for the work (NULL = legacy default); the call
 *                      returns once it has finished.
 *   farness, reach   : DEVICE outputs, n entries each, indexed by vertex id.
 * All working memory is one fixed 64 MiB device array inside the library;
 * its device address is looked up on the first call on each device (make
 * that first call before any stream capture) and kept for the life of the
 * process.  So only the device's primary context (the runtime API's) is
 * supported, and the device must not be reset (cudaDeviceReset) between
 * calls.  The call is synchronous: it returns after its work on the stream
 * has finished.  Every call on a device shares the array and clears what it
 * needs; calls whose GPU work overlaps (other streams or threads on the same
 * device) race on it and must be serialised by the caller.
 * Errors: BCM_ERR_INVALID (NULL pointer, malformed CSR), BCM_ERR_UNSUPPORTED,
 * BCM_ERR_CUDA, BCM_ERR_TIMEOUT; the message is in bcm_last_error().
 */
bcm_status bcm_farness_all_noalloc(const uint64_t* row_ptr, const uint32_t* col, uint32_t n, uint64_t m,
                                   void* stream, uint64_t* farness, uint32_t* reach);

/*
 * bcm_batch_create / bcm_batch_run / bcm_batch_destroy -- top-k runs on many
 * small graphs as one CUDA graph.  The runs of graphs[0..count) (k[i] each,
 * options opt, which must set BCM_OUT_DEVICE) are executed once to allocate
 * and check everything, then recorded back to back on `stream` (a
 * cudaStream_t; not the legacy default stream) and instantiated;
 * bcm_batch_run launches the recorded graph (one launch instead of several
 * per graph) and, with wait != 0, waits and checks every run, writing each
 * graph's min(k[i], n_i) entries to the device arrays ids[i], farness[i],
 * reach[i] given at creation (they must stay valid).  Only graphs below the
 * grid-wide threshold (n * grid_lanes/64 < heavy_words) can be batched: their
 * runs hold no cooperative launch.  A graph of a batch must not run anything
 * else while a batch run is in flight.  Errors: BCM_ERR_INVALID,
 * BCM_ERR_UNSUPPORTED (a graph too large, or plain / traced / grid-only /
 * sharded options), BCM_ERR_OOM, BCM_ERR_CUDA, BCM_ERR_TIMEOUT.
 */
typedef struct bcm_batch* bcm_batch_t;
bcm_status bcm_batch_create(bcm_graph_t* graphs, uint32_t count, const uint32_t* k, const bcm_options* opt,
                            void* stream, uint32_t* const* ids, uint64_t* const* farness, uint32_t* const* reach,
                            bcm_batch_t* out);
bcm_status bcm_batch_run(bcm_batch_t b, int wait);
bcm_status bcm_batch_destroy(bcm_batch_t b);

/*
 * bcm_topk_merge -- the best min(k, count) of `count` (id, farness, reach)
 * entries under the ranking above (exact 128-bit comparisons, equal scores
 * by id), written best first to out_ids / out_far / out_reach.  Host memory
 * only; runs on the CPU (it merges the k-entry lists of several shards,
 * whose union holds the graph's top-k).  Ids must be distinct, except that
 * entries with id 0xFFFFFFFF (the padding of a shard list, see
 * bcm_topk_offer) are skipped.  Returns the number of entries written in
 * *written.  Errors: BCM_ERR_INVALID (NULL pointer, k = 0), BCM_ERR_OOM.
 */
bcm_status bcm_topk_merge(const uint32_t* ids, const uint64_t* farness, const uint32_t* reach, uint32_t count,
                          uint32_t k, uint32_t* out_ids, uint64_t* out_far, uint32_t* out_reach,
                          uint32_t* written);

/* Thread-local message for the last failing call ("" if none). */
const char* bcm_last_error(void);

/* Kernels launched by this library in this process so far. */
uint64_t bcm_launch_count(void);

/* Device bytes a bcm_topk / bcm_farness_all run on this graph holds with
 * these options (graph copy excluded; bcm_graph_trim gives back all but the
 * preprocessing arrays); 0 on bad arguments. */
uint64_t bcm_workspace_bytes(bcm_graph_t g, const bcm_options* opt);

#ifdef __cplusplus
}
#endif

#endif /* BCM_H */
