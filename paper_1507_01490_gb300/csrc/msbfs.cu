// BFSCut on many sources at once (Algorithm 2 of the paper, run as a
// multi-source BFS with one bit lane per source) and the plain one-source
// version it is measured against.
//
// A wave is 64*W sources taken consecutively from the degree order
// (Algorithm 1 visits vertices in decreasing degree).  Each vertex holds W
// 64-bit words per array: `vis` (lanes that reached it), `F[cur]` (lanes
// whose frontier holds it) and `F[cur^1]` (lanes that reached it in the level
// being expanded).  At level d every surviving lane knows n_d, f_d and
// gamma~_{d+1} (Table 1), so the stopping rule of Lemma 1 / Lemma 2 is
// evaluated before Gamma_d is expanded.  The per-lane counts gamma_{d+1} and
// sum of deg over Gamma_{d+1} come out of the expansion itself: an arc that
// sets new bits in vis[x] discovers x for exactly those lanes.
//
// Kernels
//   k_wave_cta   persistent; every CTA runs its own waves back to back,
//                taking sources from a global atomic queue.  A level costs
//                three __syncthreads.  Completed lanes go to the shared top-k
//                under a bounded lock; its k-th key is published with a
//                sequence counter and read once per level.
//   k_wave_grid  cooperative; the whole grid runs waves one at a time, from
//                the highest-degree sources, while they are heavy (their
//                frontiers span much of the graph), so a heavy wave gets the
//                whole GPU's bandwidth; the first light wave hands the queue
//                to k_wave_cta.  Two bounded grid barriers per level.
//   k_plain      cooperative; one source per launch, level-synchronous with
//                a vertex queue and visit stamps: the baseline.
#include <cuda_runtime.h>

#include "internal.h"

namespace bcm {

// Two layouts of the bit words of a (vertex, 64-lane word) pair -- vis,
// F[0], F[1] -- chosen per kernel by the template parameter R, the stride
// between consecutive words of one array:
//   R = 4  records: the three words sit in one 32-byte record (vis, a key
//          word, F[0], F[1]), so a push's check and atomics and the wave-end
//          clear touch a single sector (per-CTA waves: push only).  The
//          records of a per-CTA slot are a vertex table (CtaTab below);
//   R = 1  planes: each array is its own plane, and the W words of a vertex
//          are consecutive in it, so a pulled level reads the vis words of 32
//          consecutive vertices in one coalesced sweep and an in-neighbour's
//          frontier words in one sector (grid-wide waves).
// vis, F[0] and F[1] below point at word 0 of each array; ri<R>(word) is the
// offset of a word.
constexpr int REC = 4;

template <int R>
__device__ __forceinline__ size_t ri(u32 word) { return (size_t)word * R; }

struct SlotPtrs {
    u64* vis;
    u64* F[2];
    u32* list[2];
    u32* clog;
};

// n vertices with W words each (the arrays' capacity; a run may use fewer).
template <int R>
__device__ __forceinline__ SlotPtrs slot_ptrs(char* base, u32 n, int W) {
    size_t nw = (size_t)n * W;
    SlotPtrs s;
    s.vis = (u64*)base;
    if (R == 1) {
        s.F[0] = s.vis + nw;
        s.F[1] = s.vis + 2 * nw;
        s.list[0] = (u32*)(s.vis + 3 * nw);
    } else {
        s.F[0] = s.vis + 2;   // vis + 1: the key word
        s.F[1] = s.vis + 3;
        s.list[0] = (u32*)(s.vis + REC * nw);
    }
    s.list[1] = s.list[0] + nw;
    s.clog = s.list[1] + nw;
    return s;
}

template <int R>
__device__ __forceinline__ void clear_word(const SlotPtrs& S, u32 word) {
    if (R == 1) {
        S.vis[word] = 0;
        S.F[0][word] = 0;
        S.F[1][word] = 0;
    } else {
        ulonglong2* r = (ulonglong2*)&S.vis[ri<R>(word)];
        r[0] = make_ulonglong2(0, 0);
        r[1] = make_ulonglong2(0, 0);
    }
}

// A per-CTA wave's vertex table: which records hold vertex x.
//   dense  (shift 0): x owns entry x (n entries; the key word is unused);
//   hashed (shift > 0): x's entry is found from h(x) = (x * kTabMul) >> shift
//          by linear probing over 2^(32 - shift) entries; the record of the
//          entry's word 0 keeps x + 1 in its key word, 0 marking a free entry.
// A wave touches few vertices once the grid-wide waves and the prefilter
// have run, so a table of 2^16 entries replaces n records per CTA.  Inserts
// are counted; once `limit` is passed no new entry is made, and the wave is
// given up at the end of the level: its live sources go to the grid-wide
// pass, which runs them again from the start (the counts of a level with a
// dropped arc are incomplete and never used).  The limit (half the table)
// keeps the table from filling: past it, only the inserts already in
// flight (two per thread) land.
struct CtaTab {
    u32 shift, mask, limit;
    u32* ins;              // shared: entries this wave inserted
    volatile u32* full;    // shared: set once an insert passed the limit
};
constexpr u32 kTabMul = 0x9E3779B1u;   // 2^32 / golden ratio: Fibonacci hashing
__device__ constexpr CtaTab kDenseTab{0, 0, 0, nullptr, nullptr};   // the grid kernel's planes

// Entry e of vertex x in a hashed table, inserted if x has none (fl |= 2:
// the clear log then takes the entry); seen = vis word 0 of the entry as
// read.  False when x has no entry and the table is past its limit.  Kept
// out of line: inlined at its call sites it pushed the dense path's
// registers into spills (out of line, the dense path has none at 64 lanes).
template <int W>
__device__ __noinline__ bool tab_find(const CtaTab& T, u64* rec, u32 x, u32& e, u64& seen, u32& fl) {
    const u32 key = x + 1;
    e = (x * kTabMul) >> T.shift;
    for (u32 probe = 0; probe <= T.mask; ++probe) {
        u64* r = rec + (size_t)e * W * REC;
        const ulonglong2 kv = __ldcg((const ulonglong2*)r);   // vis word 0, key
        u32 k = (u32)kv.y;
        if (k == key) { seen = kv.x; return true; }
        if (k == 0) {
            if (*T.full) return false;
            k = atomicCAS((u32*)(r + 1), 0u, key);
            if (k == 0) {
                fl |= 2u;
                if (atomicAdd(T.ins, 1u) >= T.limit) *T.full = 1;
                seen = 0;
                return true;
            }
            if (k == key) { seen = __ldcg(r); return true; }
        }
        e = (e + 1) & T.mask;
    }
    *T.full = 1;   // every entry taken: cannot happen below the limit, and the wave is given up
    return false;
}

// Counters of the expansion loops, per thread (kept small: they live in
// registers through the hot loops).  Rare events (completions, cuts, waves,
// levels, cleared words) go to a per-block shared array instead.
struct LocalStats {
    u64 mvis = 0;
    u64 fwarcs = 0;      // out-arcs of the words this thread put in the next frontier (this level)
    u32 disc = 0, entries = 0, arcwords = 0, discwords = 0;
};

// Adds the warp's next-frontier arc words to *dst and clears the counters.
__device__ __forceinline__ void flush_fwarcs(LocalStats& st, unsigned long long* dst) {
    u64 x = st.fwarcs;
    for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if ((threadIdx.x & 31) == 0 && x) atomicAdd(dst, (unsigned long long)x);
    st.fwarcs = 0;
}

// per-block counters of rare events, indexed by Stat
struct BlockStats { unsigned long long v[ST_COUNT]; };

__device__ __forceinline__ void bstat_init(BlockStats& b) {
    for (int i = threadIdx.x; i < ST_COUNT; i += blockDim.x) b.v[i] = 0;
}
__device__ __forceinline__ void bstat_add(BlockStats& b, int i, u64 x) { atomicAdd(&b.v[i], (unsigned long long)x); }
__device__ __forceinline__ void bstat_max(BlockStats& b, int i, u64 x) { atomicMax(&b.v[i], (unsigned long long)x); }

// Warp-reduces the per-thread counters, then one global atomic per counter
// per warp; thread 0 adds the block's rare-event counters.  Call with the
// whole block, after a __syncthreads that follows the last bstat update.
__device__ inline void flush_stats(const LocalStats& s, const BlockStats& b, unsigned long long* g) {
    u64 v[5] = {s.mvis, s.disc, s.entries, s.arcwords, s.discwords};
    const int idx[5] = {ST_MVIS, ST_DISC, ST_ENTRIES, ST_ARCWORDS, ST_DISCWORDS};
#pragma unroll
    for (int i = 0; i < 5; ++i) {
        u64 x = v[i];
        for (int o = 16; o; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
        if ((threadIdx.x & 31) == 0 && x) atomicAdd(&g[idx[i]], x);
    }
    if (threadIdx.x == 0) {
        const int rare[9] = {ST_COMPLETED, ST_CUT,    ST_WAVES,   ST_LEVELS,     ST_CLEARED,
                             ST_MAXLEVEL,  ST_DEFERRED, ST_ENTRIES, ST_PULLENTRIES};
        for (int i = 0; i < 9; ++i) {
            u64 x = b.v[rare[i]];
            if (!x) continue;
            if (rare[i] == ST_MAXLEVEL) atomicMax(&g[rare[i]], x);
            else atomicAdd(&g[rare[i]], x);
        }
    }
}

// One trace record (4 words), when tracing is on.  The second word holds
// the kind in bits 60..63, an identifier (wave or CTA) in bits 32..59 and a
// level in bits 0..31.
__device__ __forceinline__ void trace_record(const WaveParams& p, u32 kind, u32 id, u32 level, u64 a, u64 b,
                                             u64 t) {
    if (!p.trace) return;
    const u32 i = atomicAdd(p.trace_n, 1u);
    if (i >= p.trace_cap) return;
    unsigned long long* r = p.trace + 4 * (size_t)i;
    r[0] = t;
    r[1] = ((u64)kind << 60) | ((u64)(id & 0xfffffffu) << 32) | level;
    r[2] = a;
    r[3] = b;
}

// Lane records (BCM_TRACE_LANES): source v's Table 1 state before the
// stopping rule at level d, and how its BFS ended.
__device__ __noinline__ void lane_level(const WaveParams& p, u32 v, u32 d, u64 f, u32 nd, u32 gt) {
    trace_record(p, TR_LANE_LEVEL, v, d, f, (u64)nd | ((u64)gt << 32), global_ns());
}
__device__ __noinline__ void lane_end(const WaveParams& p, u32 v, u32 d, u64 f, u32 nd, bool cut) {
    trace_record(p, TR_LANE_END, v, d, f, (u64)nd | ((u64)(cut ? 1u : 0u) << 32), global_ns());
}

// ------------------------------------------------------- staged appends
// Frontier and clear-log appends go first to a per-warp staging area in
// shared memory and reach the list with one counter reservation per flush:
// a dense level appends millions of words, and one global counter taking an
// atomic per warp step serialises them.
struct WarpQueue {
    u32* sbuf;      // this warp's staging area (cap entries)
    u32* dst;       // the list
    u32* counter;   // its length
    u32 cap;
    u32 n;          // staged entries (the same in every lane)
    __device__ __forceinline__ void push(bool want, u32 item) {
        const u32 m = __ballot_sync(0xffffffffu, want);
        if (want) sbuf[n + __popc(m & lanemask_lt())] = item;
        n += __popc(m);
    }
    __device__ __forceinline__ void flush() {
        if (n == 0) return;
        __syncwarp();
        u32 base = 0;
        if ((threadIdx.x & 31) == 0) base = atomicAdd(counter, n);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (u32 i = threadIdx.x & 31; i < n; i += 32) dst[base + i] = sbuf[i];
        __syncwarp();
        n = 0;
    }
    // room for one more step of up to `need` entries
    __device__ __forceinline__ void reserve(u32 need) {
        if (n + need > cap) flush();
    }
};

// ------------------------------------------------------------ push step
// Lanes F of word g reach x: the bits of F not yet in vis[x] are x's
// discoveries at this level.  push_begin loads what the step needs;
// push_end issues the atomics.  Splitting them lets a thread keep two arcs'
// memory operations in flight at once.
struct Push {
    u32 x, g, word, r0, r1;
    u32 lw;          // hashed table: the entry's word 0, which the clear log takes (dense: the word)
    u64 F, nb;
    u32 fl;          // bit 0: word enters the next frontier; bit 1: log lw (a vis word was empty,
                     // or a table entry was made)
    u32 degp;
};

template <int W>
__device__ __forceinline__ void push_load(const u32* __restrict__ col, u32 e, u64 F, u32 g, Push& q) {
    q.x = __ldg(&col[e]);
    q.F = F;
    q.g = g;
}

template <int W, int R>
__device__ __forceinline__ void push_check(const u32* __restrict__ rp, u64* vis, Push& q, const CtaTab& T) {
    q.fl = 0;
    q.degp = 0;
    u64 seen;
    if (R == REC && T.shift) {
        u32 e;
        if (!tab_find<W>(T, vis, q.x, e, seen, q.fl)) {   // table past its limit: the wave is given up
            q.nb = 0;
            q.word = 0;
            q.lw = 0;
            return;
        }
        q.word = e * W + q.g;
        q.lw = e * W;
        if (W > 1 && q.g) seen = __ldcg(&vis[ri<R>(q.word)]);
    } else {
        q.word = q.x * W + q.g;
        seen = __ldcg(&vis[ri<R>(q.word)]);
    }
    q.nb = q.F & ~seen;
    if (q.nb) {
        q.r0 = __ldg(&rp[q.x]);
        q.r1 = __ldg(&rp[q.x + 1]);
    }
}

template <int R>
__device__ __forceinline__ void push_vis(u64* vis, Push& q, u64& old) {
    old = q.nb ? atomicOr(&vis[ri<R>(q.word)], q.nb) : ~0ull;
}

template <int R>
__device__ __forceinline__ void push_next(u64* Fnext, Push& q, u64 old, u32 foot, LocalStats& st,
                                          const CtaTab& T) {
    if (!q.nb) return;
    if (!(R == REC && T.shift)) q.fl = (old == 0) ? 2u : 0u;   // hashed: logged when the entry was made
    q.nb &= ~old;
    if (!q.nb) return;
    u64 oldF = atomicOr(&Fnext[ri<R>(q.word)], q.nb);
    if (oldF == 0) {
        q.fl |= 1u;
        st.discwords++;
        st.fwarcs += q.r1 - q.r0;
    }
    q.degp = q.r1 - q.r0 - foot;
    st.disc += __popcll(q.nb);
}

// Per-lane counts of this step's discoveries, summed across the warp:
// cg[lane] += how many vertices the lane discovered, cs[lane] += the sum of
// their degrees (minus the footnote).  Transposed: the warp walks the
// threads holding discoveries (at most 32) and thread t keeps the counts of
// bit lanes t and t+32 of the word group being walked, so the shared-memory
// updates are one per thread and bit lane, with no two threads on one
// counter.
#ifndef BCM_COUNT_LOOP
#define BCM_COUNT_LOOP 8
#endif
constexpr int kCountLoop = BCM_COUNT_LOOP;   // at most this many reaching lanes: count by the loop
__device__ __forceinline__ void warp_count(u64 nb, u32 degp, u32 g, u32* cg, u32* cs) {
    const u32 lane = threadIdx.x & 31;
    u32 active = __ballot_sync(0xffffffffu, nb != 0);
    while (active) {
        const u32 g0 = __shfl_sync(0xffffffffu, g, __ffs(active) - 1);
        u32 grp = __ballot_sync(0xffffffffu, nb != 0 && g == g0);
        active &= ~grp;
        u32 c_lo = 0, c_hi = 0, s_lo = 0, s_hi = 0;
        while (grp) {
            const int i = __ffs(grp) - 1;
            grp &= grp - 1;
            const u32 lo = __shfl_sync(0xffffffffu, (u32)nb, i);
            const u32 hi = __shfl_sync(0xffffffffu, (u32)(nb >> 32), i);
            const u32 dg = __shfl_sync(0xffffffffu, degp, i);
            if ((lo >> lane) & 1u) { ++c_lo; s_lo += dg; }
            if ((hi >> lane) & 1u) { ++c_hi; s_hi += dg; }
        }
        if (c_lo) { atomicAdd(&cg[g0 * 64 + lane], c_lo); atomicAdd(&cs[g0 * 64 + lane], s_lo); }
        if (c_hi) { atomicAdd(&cg[g0 * 64 + 32 + lane], c_hi); atomicAdd(&cs[g0 * 64 + 32 + lane], s_hi); }
    }
}

// 32x32 bit transpose across the warp: lane i passes row i (bit j = entry
// (i, j)) and gets column i back (bit j = entry (j, i)).  Five rounds of
// swapping off-diagonal blocks of halving size.
__device__ __forceinline__ u32 warp_transpose32(u32 x) {
    const u32 lane = threadIdx.x & 31;
    const u32 masks[5] = {0x0000FFFFu, 0x00FF00FFu, 0x0F0F0F0Fu, 0x33333333u, 0x55555555u};
#pragma unroll
    for (int r = 0; r < 5; ++r) {
        const int sh = 16 >> r;
        const u32 m = masks[r];
        const u32 y = __shfl_xor_sync(0xffffffffu, x, sh);
        x = (lane & sh) ? ((x & ~m) | ((y >> sh) & m)) : ((x & m) | ((y & m) << sh));
    }
    return x;
}

// warp_count for a warp whose lanes all hold word g: with many lanes
// reaching something, the counts come from the transposed bit matrix (lane
// b's column word marks the lanes whose nb has bit b) and the degree sums
// from its AND with each bit plane of degp; with few, warp_count's loop.
__device__ __forceinline__ void warp_count_word(u64 nb, u32 degp, u32 g, u32* cg, u32* cs) {
    const u32 lane = threadIdx.x & 31;
    const u32 active = __ballot_sync(0xffffffffu, nb != 0);
    if (__popc(active) <= kCountLoop) {
        warp_count(nb, degp, g, cg, cs);
        return;
    }
    const u32 lo = warp_transpose32((u32)nb), hi = warp_transpose32((u32)(nb >> 32));
    const u32 dmax = __reduce_max_sync(0xffffffffu, nb ? degp : 0u);
    u32 s_lo = 0, s_hi = 0;
    for (int k = 0; k < 32 && (dmax >> k); ++k) {
        const u32 plane = __ballot_sync(0xffffffffu, (degp >> k) & 1u);
        s_lo += (u32)__popc(lo & plane) << k;
        s_hi += (u32)__popc(hi & plane) << k;
    }
    const u32 c_lo = __popc(lo), c_hi = __popc(hi);
    if (c_lo) { atomicAdd(&cg[g * 64 + lane], c_lo); atomicAdd(&cs[g * 64 + lane], s_lo); }
    if (c_hi) { atomicAdd(&cg[g * 64 + 32 + lane], c_hi); atomicAdd(&cs[g * 64 + 32 + lane], s_hi); }
}

template <int R>
__device__ __forceinline__ void push_finish(const Push& q, u32* cg, u32* cs, WarpQueue& nq, WarpQueue& lq,
                                            const CtaTab& T) {
    warp_count(q.nb, q.degp, q.g, cg, cs);
    nq.push(q.fl & 1u, q.word);
    lq.push(q.fl & 2u, (R == REC && T.shift) ? q.lw : q.word);
}

// Prefix sums of the live sources' degrees (s_pre[0..L]) and their first
// arcs (s_beg), for expand_sources.  Called by the whole block.
template <int THREADS>
__device__ inline void source_prefix(const GraphDev& G, const u32* s_src, const u32* s_alive32, int L, u32* s_pre,
                                     u32* s_beg, u32* s_wsum) {
    const u32 tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    u32 incl = 0;
    if (tid < (u32)L) {
        // only live lanes hold a source (others may hold a stale or unset id)
        const bool a = (s_alive32[tid >> 5] >> lane) & 1u;
        u32 b = 0;
        if (a) {
            const u32 v = s_src[tid];
            b = __ldg(&G.rp[v]);
            incl = __ldg(&G.rp[v + 1]) - b;
        }
        s_beg[tid] = b;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (u32)o) incl += t;
        }
        if (lane == 31) s_wsum[wid] = incl;
    }
    __syncthreads();
    if (tid < (u32)L) {
        u32 off = 0;
        for (u32 w = 0; w < wid; ++w) off += s_wsum[w];
        s_pre[tid + 1] = off + incl;
        if (tid == 0) s_pre[0] = 0;
    }
    __syncthreads();
}

// Level 0: lane j's frontier is its source.  The live sources' arc ranges
// are laid end to end (s_pre holds the prefix sums of their degrees) and
// walked 32 arcs at a time by every warp of the caller (the block, or the
// whole grid), so a wave of hubs spreads over all
// warps instead of one warp per source.  Each source's own bit is set by one
// thread; an arc back to the lane's own source (a self-loop) is skipped, so
// no arc can find the source before its bit is set.
template <int W, int R>
__device__ inline void expand_sources(const GraphDev& G, const u32* s_src, const u32* s_alive32, const u32* s_pre,
                                      const u32* s_beg, int L, u64* vis, u64* Fnext, u32* cg, u32* cs, u32 foot,
                                      WarpQueue& nq, WarpQueue& lq, u32 wid, u32 nw, u32 tid, u32 nthreads,
                                      const CtaTab& T, LocalStats& st) {
    const u32 lane = threadIdx.x & 31;
    lq.reserve(32);
    for (u32 j0 = tid - lane; j0 < (u32)L; j0 += nthreads) {
        const u32 j = j0 + lane;
        bool first = false;
        u32 lw = 0;
        if (j < (u32)L && ((s_alive32[j >> 5] >> (j & 31)) & 1u)) {
            const u32 deg = s_pre[j + 1] - s_pre[j];
            u32 e = s_src[j];
            bool have = true;
            if (R == REC && T.shift) {
                u64 seen;
                u32 fl = 0;
                have = tab_find<W>(T, vis, s_src[j], e, seen, fl);
                first = fl != 0;
                lw = e * W;
            }
            if (have) {
                const u32 word = e * W + (j >> 6);
                const bool empty = atomicOr(&vis[ri<R>(word)], 1ull << (j & 63)) == 0;
                if (!(R == REC && T.shift)) {
                    first = empty;
                    lw = word;
                }
            }
            st.mvis += deg;
            st.arcwords += deg;
        }
        lq.reserve(32);
        lq.push(first, lw);
    }
    const u32 total = s_pre[L];
    for (u32 t0 = wid * 32; t0 < total; t0 += nw * 32) {
        const u32 idx = t0 + lane;
        bool v = idx < total;
        Push q;
        q.nb = 0; q.fl = 0; q.degp = 0; q.g = 0; q.word = 0; q.lw = 0;
        if (v) {
            // the lane owning arc idx: the last j with s_pre[j] <= idx
            u32 lo = 0, hi = (u32)L;
            while (hi - lo > 1) {
                const u32 mid = (lo + hi) >> 1;
                if (s_pre[mid] <= idx) lo = mid; else hi = mid;
            }
            push_load<W>(G.col, s_beg[lo] + idx - s_pre[lo], 1ull << (lo & 63), lo >> 6, q);
            if (q.x == s_src[lo]) v = false;   // self-loop
        }
        nq.reserve(32);
        lq.reserve(32);
        if (v) {
            push_check<W, R>(G.rp, vis, q, T);
            u64 old;
            push_vis<R>(vis, q, old);
            push_next<R>(Fnext, q, old, foot, st, T);
        } else {
            q.nb = 0;
        }
        push_finish<R>(q, cg, cs, nq, lq, T);
    }
}

// Frontier entries with more than kHeavyArcs out-arcs are not expanded by
// the warp that reads them: they go to a heavy list, and once every warp is
// past the main pass, all warps share their arcs (expand_heavy).  A list
// that is full leaves the entry with its warp.
constexpr u32 kHeavyArcs = 256;
constexpr u32 kHeavyCapCta = 64;
struct HeavyList {
    HeavyEntry* e;
    u32* n;       // entries claimed (may pass cap; only the first cap are stored)
    u32 cap;
};

// Level >= 1: frontier words from `list`.  Warps take chunks of 32 entries
// from a shared counter (so a chunk holding a high-degree vertex does not
// hold back the others), form the exclusive scan of the chunk's degrees and
// walk the combined arc range 64 arcs at a time, two per thread.
template <int W, int R>
__device__ inline void expand_entries(const GraphDev& G, const u32* list, u32 cnt, u64* Fcur,
                                      const u32* s_alive32, u64* vis, u64* Fnext, u32* cg, u32* cs,
                                      u32 foot, WarpQueue& nq, WarpQueue& lq, u32* chunk_ctr, u32 wid, u32 nw,
                                      const HeavyList& H, const CtaTab& T, LocalStats& st) {
    const u32 lane = threadIdx.x & 31;
    // entries taken per chunk: 32 when the frontier is small, up to 256 when
    // it is large enough to keep every warp busy anyway.  Warp wid's first
    // chunk is the wid-th; the rest come from the shared counter, which only
    // runs past the first nw chunks -- a narrow level then costs no atomic.
    u32 grab = cnt / (nw * 8u);
    grab = grab < 32u ? 32u : (grab > 256u ? 256u : (grab & ~31u));
    const u64 fixed = (u64)nw * grab;
    u32 base = 0, lim = 0;
    bool first = true;
    for (;;) {
        if (base >= lim) {
            // the warp's own first chunk, then chunks from the shared counter;
            // every path either takes a chunk below cnt or leaves the loop
            u64 b = first ? (u64)wid * grab : ~0ull;
            first = false;
            if (b >= cnt) {
                if (fixed >= cnt) break;   // all entries lie in the first chunks
                u32 c = 0;
                if (lane == 0) c = atomicAdd(chunk_ctr, grab);
                b = fixed + __shfl_sync(0xffffffffu, c, 0);
                if (b >= cnt) break;
            }
            base = (u32)b;
            lim = base + grab < cnt ? base + grab : cnt;
        }
        const u32 e = base + lane;
        base += 32;
        u32 g = 0, beg = 0, deg = 0;
        u64 F = 0;
        if (e < cnt) {
            u32 word = __ldcg(&list[e]);
            u32 u = word / W;
            g = word - u * W;
            if (R == REC && T.shift) u = (u32)__ldcg(&vis[ri<R>(u * W) + 1]) - 1;   // the entry's vertex
            F = __ldcg(&Fcur[ri<R>(word)]);
            Fcur[ri<R>(word)] = 0;
            F &= ((u64)s_alive32[2 * g + 1] << 32) | s_alive32[2 * g];
            st.entries++;
            if (F) {
                beg = __ldg(&G.rp[u]);
                deg = __ldg(&G.rp[u + 1]) - beg;
                st.mvis += (u64)__popcll(F) * deg;
                st.arcwords += deg;
                if (deg > kHeavyArcs) {
                    const u32 slot = atomicAdd(H.n, 1u);
                    if (slot < H.cap) {
                        H.e[slot].F = F;
                        H.e[slot].beg = beg;
                        H.e[slot].deg = deg;
                        H.e[slot].g = g;
                        deg = 0;          // expanded by expand_heavy
                    }
                }
            }
        }
        u32 incl = deg;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            u32 t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (u32)o) incl += t;
        }
        const u32 total = __shfl_sync(0xffffffffu, incl, 31);
        const u32 excl = incl - deg;
        for (u32 t0 = 0; t0 < total; t0 += 64) {
            Push q[2];
            bool v[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) {
                const u32 idx = t0 + 32 * h + lane;
                int owner = 0;
#pragma unroll
                for (int step = 16; step; step >>= 1) {
                    u32 ex = __shfl_sync(0xffffffffu, excl, owner + step);
                    if (ex <= idx) owner += step;
                }
                const u32 o_beg = __shfl_sync(0xffffffffu, beg, owner);
                const u32 o_excl = __shfl_sync(0xffffffffu, excl, owner);
                const u64 o_F = __shfl_sync(0xffffffffu, F, owner);
                const u32 o_g = __shfl_sync(0xffffffffu, g, owner);
                v[h] = idx < total;
                q[h].nb = 0; q[h].fl = 0; q[h].degp = 0; q[h].g = o_g; q[h].word = 0; q[h].lw = 0;
                if (v[h]) push_load<W>(G.col, o_beg + idx - o_excl, o_F, o_g, q[h]);
            }
            nq.reserve(64);
            lq.reserve(64);
#pragma unroll
            for (int h = 0; h < 2; ++h)
                if (v[h]) push_check<W, R>(G.rp, vis, q[h], T);
            u64 old[2];
#pragma unroll
            for (int h = 0; h < 2; ++h) push_vis<R>(vis, q[h], old[h]);
#pragma unroll
            for (int h = 0; h < 2; ++h) push_next<R>(Fnext, q[h], old[h], foot, st, T);
#pragma unroll
            for (int h = 0; h < 2; ++h) push_finish<R>(q[h], cg, cs, nq, lq, T);
        }
    }
}

// The heavy list's arcs, 64 at a time, piece c to warp c mod nw (warp wid
// of nw); run by every warp after all of them have left expand_entries.
template <int W, int R>
__device__ __noinline__ void expand_heavy(const GraphDev& G, const HeavyEntry* H, u32 hn, u64* vis, u64* Fnext,
                                    u32* cg, u32* cs, u32 foot, WarpQueue& nq, WarpQueue& lq, u32 wid, u32 nw,
                                    const CtaTab& T, LocalStats& st) {
    const u32 lane = threadIdx.x & 31;
    u32 base = 0;   // pieces in the batches before this one
    for (u32 h0 = 0; h0 < hn; h0 += 32) {
        const u32 h = h0 + lane;
        u32 pc = 0, beg = 0, deg = 0, g = 0;
        u64 F = 0;
        if (h < hn) {
            F = H[h].F;
            beg = H[h].beg;
            deg = H[h].deg;
            g = H[h].g;
            pc = (deg + 63) / 64;
        }
        u32 incl = pc;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= (u32)o) incl += t;
        }
        const u32 total = __shfl_sync(0xffffffffu, incl, 31);
        const u32 excl = incl - pc;
        // this warp's pieces: base + idx with (base + idx) % nw == wid
        for (u32 idx = (wid + nw - base % nw) % nw; idx < total; idx += nw) {
            int owner = 0;
#pragma unroll
            for (int step = 16; step; step >>= 1) {
                const u32 ex = __shfl_sync(0xffffffffu, excl, owner + step);
                if (ex <= idx) owner += step;
            }
            const u32 o_beg = __shfl_sync(0xffffffffu, beg, owner);
            const u32 o_deg = __shfl_sync(0xffffffffu, deg, owner);
            const u32 o_excl = __shfl_sync(0xffffffffu, excl, owner);
            const u32 o_g = __shfl_sync(0xffffffffu, g, owner);
            const u64 o_F = ((u64)__shfl_sync(0xffffffffu, (u32)(F >> 32), owner) << 32) |
                            __shfl_sync(0xffffffffu, (u32)F, owner);
            const u32 off = (idx - o_excl) * 64;
            Push q[2];
            bool v[2];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) {
                const u32 a = off + 32 * hh + lane;
                v[hh] = a < o_deg;
                q[hh].nb = 0; q[hh].fl = 0; q[hh].degp = 0; q[hh].g = o_g; q[hh].word = 0; q[hh].lw = 0;
                if (v[hh]) push_load<W>(G.col, o_beg + a, o_F, o_g, q[hh]);
            }
            nq.reserve(64);
            lq.reserve(64);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh)
                if (v[hh]) push_check<W, R>(G.rp, vis, q[hh], T);
            u64 old[2];
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) push_vis<R>(vis, q[hh], old[hh]);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) push_next<R>(Fnext, q[hh], old[hh], foot, st, T);
#pragma unroll
            for (int hh = 0; hh < 2; ++hh) push_finish<R>(q[hh], cg, cs, nq, lq, T);
        }
        base += total;
    }
}

// Level >= 1 by pull, for a frontier that covers much of the graph: each
// vertex x whose vis words miss live lanes ("pending") ORs in the frontier
// words of its in-neighbours, stopping once every pending lane is found.
// Warps take 32 consecutive vertices at a time from a shared counter.
// A vertex with at most kPullSerial in-arcs is scanned by its own thread;
// a larger one by the whole warp, 32*kPullCoop in-arcs per step with an
// OR-reduction and the same early stop, so a hub's in-list does not hold one
// thread for thousands of dependent loads.  vis/F-next of x are written by x's own
// thread, without atomics.  The frontier words themselves are cleared
// afterwards (pull_clear), once no thread can still be reading them.
#ifndef BCM_PULL_SERIAL
#define BCM_PULL_SERIAL 32
#endif
constexpr u32 kPullSerial = BCM_PULL_SERIAL;
#ifndef BCM_PULL_UNROLL
#define BCM_PULL_UNROLL 2
#endif
constexpr int kPullUnroll = BCM_PULL_UNROLL;   // in-neighbours per step of a thread's scan
#ifndef BCM_PULL_COOP
#define BCM_PULL_COOP 4
#endif
constexpr int kPullCoop = BCM_PULL_COOP;   // in-neighbours per thread and step of a warp's scan

// The W words of one vertex in a plane (R = 1 layout), as 16-byte loads and stores.
template <int W>
__device__ __forceinline__ void load_words_cg(const u64* p, u64 (&w)[W]) {
    if (W == 1) {
        w[0] = __ldcg(p);
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2) {
            const ulonglong2 t = __ldcg((const ulonglong2*)(p + i));
            w[i] = t.x;
            w[i + 1] = t.y;
        }
    }
}

template <int W>
__device__ __forceinline__ void store_words(u64* p, const u64 (&w)[W]) {
    if (W == 1) {
        p[0] = w[0];
    } else {
#pragma unroll
        for (int i = 0; i < W; i += 2) *(ulonglong2*)(p + i) = make_ulonglong2(w[i], w[i + 1]);
    }
}

// Grid-wide waves only (planar layout).  An in-neighbour outside the
// frontier has zero frontier words, so its words are loaded without first
// asking whether it is in the frontier: one sector either way, and a
// one-bit-per-vertex frontier map in front of it was a second dependent
// load that measured slower on every workload.
template <int W>
__device__ inline void pull_level(const GraphDev& G, const u64* Fcur, const u32* s_alive32, u64* vis, u64* Fnext,
                                  u32* cg, u32* cs, u32 foot, WarpQueue& nq, WarpQueue& lq, u32* chunk_ctr,
                                  u32 wid, u32 nw, LocalStats& st) {
    const u32 lane = threadIdx.x & 31;
    constexpr u32 NONE = 0xffffffffu;
    u64 alive[W];
#pragma unroll
    for (int g = 0; g < W; ++g) alive[g] = ((u64)s_alive32[2 * g + 1] << 32) | s_alive32[2 * g];
    // batches of 32 consecutive vertices: about three quarters of them dealt
    // out in turn (warp wid takes wid, wid + nw, ...), the rest from a shared
    // counter (a warp held up by a large in-list takes fewer of those), so
    // that most batches cost no atomic on the one counter
    const u32 nb = (G.n + 31) / 32;
    const u32 dealt = ((nb / 4) * 3 / nw) * nw;
    u32 next = wid;
    for (;;) {
        u32 bi;
        if (next < dealt) {
            bi = next;
            next += nw;
        } else {
            u32 c = 0;
            if (lane == 0) c = atomicAdd(chunk_ctr, 1u);
            bi = dealt + __shfl_sync(0xffffffffu, c, 0);
        }
        if (bi >= nb) break;
        const u32 x0 = bi * 32;
        const u32 x = x0 + lane;
        u64 pend[W], acc[W], v0[W];
        bool any = false;
        u32 b = 0, e = 0, dx = 0;
#pragma unroll
        for (int g = 0; g < W; ++g) { pend[g] = 0; acc[g] = 0; v0[g] = 0; }
        if (x < G.n) {
            // in-list bounds and the out-degree used if x is reached, loaded
            // with the vis words rather than after them (32 consecutive
            // vertices: a few lines per warp)
            b = __ldg(&G.rrp[x]);
            e = __ldg(&G.rrp[x + 1]);
            dx = __ldg(&G.rp[x + 1]) - __ldg(&G.rp[x]);
            load_words_cg<W>(&vis[(size_t)x * W], v0);
#pragma unroll
            for (int g = 0; g < W; ++g) {
                pend[g] = alive[g] & ~v0[g];
                any = any || pend[g] != 0;
            }
        }
        const bool coop = any && e - b > kPullSerial;
        if (any && !coop) {
            // kPullUnroll in-neighbours per step: their col entries, then
            // their frontier words, are loaded together (independent loads
            // in flight), and the early stop is checked once per step
            u32 i = b;
            while (i < e) {
                u32 u[kPullUnroll];
#pragma unroll
                for (int j = 0; j < kPullUnroll; ++j) u[j] = i + j < e ? __ldg(&G.rcol[i + j]) : NONE;
#pragma unroll
                for (int j = 0; j < kPullUnroll; ++j) {
                    if (u[j] == NONE) continue;
                    u64 w[W];
                    load_words_cg<W>(&Fcur[(size_t)u[j] * W], w);
#pragma unroll
                    for (int g = 0; g < W; ++g) acc[g] |= w[g];
                }
                bool done = true;
#pragma unroll
                for (int g = 0; g < W; ++g) done = done && !(pend[g] & ~acc[g]);
                i = i + kPullUnroll < e ? i + kPullUnroll : e;
                if (done) break;
            }
            st.arcwords += i - b;
        }
        // the large in-lists, one at a time by the whole warp
        u32 todo = __ballot_sync(0xffffffffu, coop);
        while (todo) {
            const int l0 = __ffs(todo) - 1;
            todo &= todo - 1;
            const u32 cb = __shfl_sync(0xffffffffu, b, l0), ce = __shfl_sync(0xffffffffu, e, l0);
            u64 cp[W], ca[W];
#pragma unroll
            for (int g = 0; g < W; ++g) {
                const u32 lo = __shfl_sync(0xffffffffu, (u32)pend[g], l0);
                const u32 hi = __shfl_sync(0xffffffffu, (u32)(pend[g] >> 32), l0);
                cp[g] = ((u64)hi << 32) | lo;
                ca[g] = 0;
            }
            // kPullCoop arcs per thread and step: a hub's in-list is the
            // level's longest chain of dependent loads, so each step puts
            // kPullCoop independent col / frontier-word loads in flight
            u32 i = cb;
            for (; i < ce; i += 32 * kPullCoop) {
                u32 u[kPullCoop];
#pragma unroll
                for (int j = 0; j < kPullCoop; ++j) {
                    const u32 a = i + 32 * j + lane;
                    u[j] = a < ce ? __ldg(&G.rcol[a]) : NONE;
                }
                u64 f[W];
#pragma unroll
                for (int g = 0; g < W; ++g) f[g] = 0;
#pragma unroll
                for (int j = 0; j < kPullCoop; ++j) {
                    if (u[j] == NONE) continue;
                    u64 w[W];
                    load_words_cg<W>(&Fcur[(size_t)u[j] * W], w);
#pragma unroll
                    for (int g = 0; g < W; ++g) f[g] |= w[g];
                }
                bool done = true;
#pragma unroll
                for (int g = 0; g < W; ++g) {
                    f[g] &= cp[g];
                    const u32 lo = __reduce_or_sync(0xffffffffu, (u32)f[g]);
                    const u32 hi = __reduce_or_sync(0xffffffffu, (u32)(f[g] >> 32));
                    ca[g] |= ((u64)hi << 32) | lo;
                    done = done && !(cp[g] & ~ca[g]);
                }
                if (done) { i = (i + 32 * kPullCoop < ce) ? i + 32 * kPullCoop : ce; break; }
            }
            if (i > ce) i = ce;
            if (lane == (u32)l0) {
                st.arcwords += i - cb;
#pragma unroll
                for (int g = 0; g < W; ++g) acc[g] = ca[g];
            }
        }
        u64 nb[W];
        u32 degp = 0;
        bool found = false;
#pragma unroll
        for (int g = 0; g < W; ++g) nb[g] = 0;
        if (any) {
            degp = dx - foot;
#pragma unroll
            for (int g = 0; g < W; ++g) {
                nb[g] = acc[g] & pend[g];
                if (nb[g]) {
                    st.disc += __popcll(nb[g]);
                    st.discwords++;
                    st.fwarcs += degp + foot;
                    found = true;
                }
            }
            if (found) {   // x's own words: no other thread touches them in a pulled level
                u64 nv[W];
#pragma unroll
                for (int g = 0; g < W; ++g) nv[g] = v0[g] | nb[g];
                store_words<W>(&vis[(size_t)x * W], nv);
                store_words<W>(&Fnext[(size_t)x * W], nb);   // zero where nothing was found: they were zero
            }
        }
#pragma unroll
        for (int g = 0; g < W; ++g) {
            nq.reserve(32);
            lq.reserve(32);
            warp_count_word(nb[g], degp, (u32)g, cg, cs);
            nq.push(nb[g] != 0, x * W + g);
            lq.push(nb[g] != 0 && v0[g] == 0, x * W + g);
        }
    }
}

// After a pulled level: clear the frontier words just consumed.  Four list
// entries per thread are loaded before any of their stores, so the loads
// are in flight together (the stores could alias the list as far as the
// compiler knows).
template <int R>
__device__ inline void pull_clear(const u32* list, u32 cnt, u64* Fcur, u32 gtid, u32 gthreads) {
    u64 i = gtid;
    for (; i + 3ull * gthreads < cnt; i += 4ull * gthreads) {
        u32 w[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) w[j] = __ldcg(&list[i + (u64)j * gthreads]);
#pragma unroll
        for (int j = 0; j < 4; ++j) Fcur[ri<R>(w[j])] = 0;
    }
    for (; i < cnt; i += gthreads) Fcur[ri<R>(__ldcg(&list[i]))] = 0;
}

// Completed lanes: exhaustive runs write (f, r) by vertex id; top-k runs
// merge the ones that beat the cached k-th key into the shared top-k, under
// the lock, with the whole block: the held entries (best first) are copied
// to shared memory, the new ones ranked among themselves, every entry's
// final place found by binary search in the other list, and the first k
// written back in rank order.  Call with every thread of the block; nc is
// the same in all of them.  scratch: 4608 u32 of shared memory not otherwise
// in use during the call.
__device__ __noinline__ void flush_completions(const WaveParams& p, const u32* cid, const u64* cf, const u32* cr,
                                         u32 nc, const ThrCache& thr, u32 nthreads, u32* scratch, int* s_go) {
    if (nc == 0) return;
    const u32 tid = threadIdx.x;
    if (p.exhaustive) {
        for (u32 i = tid; i < nc; i += nthreads) {
            p.out_far[cid[i]] = cf[i];
            p.out_reach[cid[i]] = cr[i];
        }
        return;
    }
    const TopK& T = p.topk;
    if (tid == 0) {
        bool any = !thr.valid;
        for (u32 i = 0; i < nc && !any; ++i) {
            u64 N, F;
            score_key(cf[i], cr[i], N, F);
            any = ranks_before(N, F, cid[i], thr.N, thr.F, thr.id);
        }
        *s_go = any && lock_acquire(T.lock, p.lock_limit_ns, p.err);
    }
    __syncthreads();
    if (!*s_go) return;
    u32* hid = scratch;                      // held entries [cnt]
    u64* hf = (u64*)(scratch + 1024);
    u32* hr = scratch + 3072;
    u32* nrank = scratch + 4096;             // rank of new entry j among the new ones
    u32* order = scratch + 4352;             // new entries by that rank
    const u32 cnt = vload(T.count);
    for (u32 i = tid; i < cnt; i += nthreads) {
        hid[i] = vload(&T.id[i]);
        hf[i] = vload(&T.f[i]);
        hr[i] = vload(&T.r[i]);
    }
    for (u32 j = tid; j < nc; j += nthreads) {
        u64 N, F;
        score_key(cf[j], cr[j], N, F);
        u32 rk = 0;
        for (u32 q = 0; q < nc; ++q) {
            u64 Nq, Fq;
            score_key(cf[q], cr[q], Nq, Fq);
            rk += ranks_before(Nq, Fq, cid[q], N, F, cid[j]) ? 1u : 0u;
        }
        nrank[j] = rk;
        order[rk] = j;
    }
    __syncthreads();
    // new entry j lands at nrank[j] + (held entries before it)
    for (u32 j = tid; j < nc; j += nthreads) {
        u64 N, F;
        score_key(cf[j], cr[j], N, F);
        u32 lo = 0, hi = cnt;               // first held entry that j ranks before
        while (lo < hi) {
            const u32 mid = (lo + hi) >> 1;
            u64 Nh, Fh;
            score_key(hf[mid], hr[mid], Nh, Fh);
            if (ranks_before(N, F, cid[j], Nh, Fh, hid[mid])) hi = mid; else lo = mid + 1;
        }
        const u32 pos = nrank[j] + lo;
        if (pos < T.k) {
            vstore(&T.id[pos], cid[j]);
            vstore(&T.f[pos], cf[j]);
            vstore(&T.r[pos], cr[j]);
        }
    }
    // held entry i lands at i + (new entries before it)
    for (u32 i = tid; i < cnt; i += nthreads) {
        u64 Nh, Fh;
        score_key(hf[i], hr[i], Nh, Fh);
        u32 lo = 0, hi = nc;                // first new entry (in rank order) that i ranks before
        while (lo < hi) {
            const u32 mid = (lo + hi) >> 1;
            const u32 q = order[mid];
            u64 Nq, Fq;
            score_key(cf[q], cr[q], Nq, Fq);
            if (ranks_before(Nh, Fh, hid[i], Nq, Fq, cid[q])) hi = mid; else lo = mid + 1;
        }
        const u32 pos = i + lo;
        if (pos < T.k) {
            vstore(&T.id[pos], hid[i]);
            vstore(&T.f[pos], hf[i]);
            vstore(&T.r[pos], hr[i]);
        }
    }
    __threadfence();
    __syncthreads();
    if (tid == 0) {
        vstore(T.count, cnt + nc < T.k ? cnt + nc : T.k);
        topk_publish_locked(T);
        lock_release(T.lock);
    }
    __syncthreads();
}

// ------------------------------------------------------------ prefilter
// On a simple graph (sorted rows, no repeated arc, no self-loop) level 1 of
// v's BFS is known without expanding it: Gamma_1 = N(v), so gamma_1 = deg(v),
// n_1 = 1 + deg(v), f_1 = deg(v), and gamma~_2 (Table 1, with the footnote's
// deg(u) - 1 on undirected graphs) = sum over u in N(v) of deg(u) - footnote.
// One warp per source applies the stopping rule at levels 0 and 1, exactly as
// a wave would, against the threshold the grid-wide waves left (no higher
// than the one a later wave would read); the sources it cannot stop go to
// `out` for the per-CTA waves.  Sources p.sources[*p.head .. p.n_end).
__global__ void __launch_bounds__(256) k_prefilter(WaveParams p, u32* out, u32* out_n) {
    __shared__ ThrCache s_thr;
    __shared__ BlockStats s_bst;
    __shared__ u32 s_begin;
    const GraphDev& G = p.g;
    if (threadIdx.x == 0) {
        s_thr.valid = 0; s_thr.N = 0; s_thr.F = 1; s_thr.id = 0;
        read_thresholds(p.topk, s_thr);
        s_begin = vload(p.head);
    }
    bstat_init(s_bst);
    __syncthreads();
    LocalStats st;
    const u32 lane = threadIdx.x & 31;
    const size_t gw = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
    const size_t gnw = ((size_t)gridDim.x * blockDim.x) >> 5;
    // 32 sources per warp step, one per thread; a source with more than 32
    // neighbours has its degree sum taken by the whole warp afterwards.  In
    // each pass over gnw*32 positions, lane l of warp w takes position
    // l*gnw + w: the sources come by degree, so consecutive positions would
    // give the first warps all the hubs (and the step's critical path)
    for (size_t base = s_begin; base < p.n_end; base += gnw * 32) {
        const size_t pos = base + lane * gnw + gw;
        const bool have = pos < p.n_end;
        u32 v = 0, b = 0, deg = 0, xlo = 0, xhi = 0;
        bool cut = false, done = !have || !s_thr.valid;
        if (have) {
            v = __ldg(&p.sources[pos]);
            b = __ldg(&G.rp[v]);
            deg = __ldg(&G.rp[v + 1]) - b;
        }
        if (!done && p.trace_lanes) lane_level(p, v, 0, 0, 1, deg);
        if (!done && deg == 0) {
            // R(v) = {v}: complete with key (0, 1); it only goes on (to be
            // merged by a wave) if it ranks before the k-th
            done = true;
            if (!ranks_before(0, 1, v, s_thr.N, s_thr.F, s_thr.id)) {
                cut = true;
                bstat_add(s_bst, ST_COMPLETED, 1);
                if (p.trace_lanes) lane_end(p, v, 0, 0, 1, false);
            }
        }
        if (!done) {
            xlo = __ldg(&G.xlo[v]);
            xhi = __ldg(&G.xhi[v]);
            if (bfscut_stops(0, deg, 0, 1, xlo, xhi, v, s_thr)) {
                cut = done = true;
                bstat_add(s_bst, ST_CUT, 1);
                if (p.trace_lanes) lane_end(p, v, 0, 0, 1, true);
            }
        }
        // level 1: gamma~_2 = sum over N(v) of deg(u) - footnote
        u64 g2 = 0;
        const bool serial = !done && deg <= 32;
        if (serial) {   // four neighbours per step: their col entries, then their degrees, in flight together
            for (u32 i = 0; i < deg; i += 4) {
                u32 u[4];
#pragma unroll
                for (int j = 0; j < 4; ++j) u[j] = i + j < deg ? __ldg(&G.col[b + i + j]) : 0xffffffffu;
#pragma unroll
                for (int j = 0; j < 4; ++j)
                    if (u[j] != 0xffffffffu) g2 += __ldg(&G.rp[u[j] + 1]) - __ldg(&G.rp[u[j]]) - p.footnote;
            }
        }
        u32 big = __ballot_sync(0xffffffffu, !done && !serial);
        while (big) {
            const int l0 = __ffs(big) - 1;
            big &= big - 1;
            const u32 cb = __shfl_sync(0xffffffffu, b, l0), cd = __shfl_sync(0xffffffffu, deg, l0);
            u64 part = 0;
            for (u32 i = lane; i < cd; i += 32) {
                const u32 u = __ldg(&G.col[cb + i]);
                part += __ldg(&G.rp[u + 1]) - __ldg(&G.rp[u]) - p.footnote;
            }
            for (int o = 16; o; o >>= 1) part += __shfl_xor_sync(0xffffffffu, part, o);
            if (lane == (u32)l0) g2 = part;
        }
        if (!done) {
            if (p.trace_lanes) lane_level(p, v, 1, deg, 1 + deg, (u32)g2);
            if (bfscut_stops(deg, g2, 1, 1 + deg, xlo, xhi, v, s_thr)) {
                cut = true;
                bstat_add(s_bst, ST_CUT, 1);
                st.mvis += deg;       // level 0 was expanded
                st.arcwords += deg;
                if (p.trace_lanes) lane_end(p, v, 1, deg, 1 + deg, true);
            }
        }
        const bool keep = have && !cut;
        const u32 m = __ballot_sync(0xffffffffu, keep);
        if (m) {
            u32 at = 0;
            if (lane == 0) at = atomicAdd(out_n, (u32)__popc(m));
            at = __shfl_sync(0xffffffffu, at, 0);
            if (keep) out[at + __popc(m & lanemask_lt())] = v;
        }
    }
    __syncthreads();
    flush_stats(st, s_bst, p.stats);
}

int launch_prefilter(const WaveParams& p, uint32_t* out, uint32_t* out_n, cudaStream_t s) {
    k_prefilter<<<152 * 8, 256, 0, s>>>(p, out, out_n);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

// --------------------------------------------------------- per-CTA waves
template <int W, int THREADS>
__global__ void __launch_bounds__(THREADS, (1024 / THREADS) > 0 ? (1024 / THREADS) : 1) k_wave_cta(WaveParams p) {
    constexpr int L = 64 * W;
    constexpr int NWARP = THREADS / 32;
    static_assert(THREADS >= L, "one thread per lane");
    __shared__ u32 s_src[L], s_nd[L], s_gt[L], s_xlo[L], s_xhi[L];
    __shared__ u64 s_f[L];
    __shared__ u32 s_cg[L], s_cs[L];
    __shared__ u32 s_alive32[2 * W];
    __shared__ u32 s_ln[2], s_logn, s_base, s_nc, s_stop, s_chunk;
    __shared__ u32 s_ins, s_full;   // the wave's table entries; set once past the table's limit
    __shared__ u64 s_twave;
    __shared__ unsigned long long s_arcs[2];   // out-arcs of each frontier list's words
    __shared__ HeavyEntry s_heavy[kHeavyCapCta];
    __shared__ u32 s_hn;
    __shared__ ThrCache s_thr;
    __shared__ BlockStats s_bst;
    constexpr u32 QCAP = 4096 / NWARP;
    __shared__ __align__(16) u32 s_stage[NWARP * 2 * QCAP];
    static_assert(NWARP * 2 * QCAP >= 4608, "flush_completions scratch");
    __shared__ u32 s_cid[L], s_cr[L];
    __shared__ u64 s_cf[L];
    __shared__ u32 s_pre[L + 1], s_beg[L], s_wsum[L / 32];
    __shared__ int s_go;

    const u32 tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const GraphDev& G = p.g;
    const u32 n_end = p.n_end_dev ? vload(p.n_end_dev) : p.n_end;
    // dense tables hold n entries whatever cta_entries says
    const u32 entries = p.tab_shift ? p.cta_entries : G.n;
    SlotPtrs S = slot_ptrs<REC>(p.slot_base + (size_t)blockIdx.x * p.slot_stride, entries, W);
    const CtaTab T{p.tab_shift, entries - 1, p.tab_limit, &s_ins, &s_full};
    LocalStats st;
    if (tid == 0) {
        s_thr.valid = 0; s_thr.N = 0; s_thr.F = 1; s_thr.id = 0;
        s_nc = 0; s_logn = 0; s_ln[0] = 0; s_ln[1] = 0; s_arcs[0] = 0; s_arcs[1] = 0; s_hn = 0;
    }
    const HeavyList Hc{s_heavy, &s_hn, kHeavyCapCta};
    bstat_init(s_bst);
    __syncthreads();

    for (u32 waves_done = 0;; ++waves_done) {
        if (tid == 0) {
            if (p.max_cta_waves && waves_done >= p.max_cta_waves) {
                s_stop = 1;
            } else {
                s_base = atomicAdd(p.head, (u32)L);
                s_stop = (s_base >= n_end) || (vload(p.err) != 0);
            }
            s_ins = 0;
            s_full = 0;
        }
        __syncthreads();
        if (s_stop) break;
        const u32 base = s_base;
        if (p.trace && tid == 0) s_twave = global_ns();   // kept in shared memory, not a register
        if (tid == 0) bstat_add(s_bst, ST_WAVES, 1);
        if (tid < L) {
            bool alive = false;
            s_cg[tid] = 0;
            s_cs[tid] = 0;
            if (base + tid < n_end) {
                u32 v = __ldg(&p.sources[base + tid]);
                u32 deg = __ldg(&G.rp[v + 1]) - __ldg(&G.rp[v]);
                s_src[tid] = v; s_nd[tid] = 1; s_f[tid] = 0; s_gt[tid] = deg;
                s_xlo[tid] = __ldg(&G.xlo[v]); s_xhi[tid] = __ldg(&G.xhi[v]);
                if (deg == 0) {          // R(v) = {v}: r = 1, f = 0
                    u32 c = atomicAdd(&s_nc, 1u);
                    s_cid[c] = v; s_cf[c] = 0; s_cr[c] = 1;
                    bstat_add(s_bst, ST_COMPLETED, 1);
                    if (p.trace_lanes) { lane_level(p, v, 0, 0, 1, 0); lane_end(p, v, 0, 0, 1, false); }
                } else {
                    alive = true;
                }
            }
            u32 m = __ballot_sync(0xffffffffu, alive);
            if (lane == 0) s_alive32[tid >> 5] = m;
        }
        // the current k-th key before the wave's first completions are
        // merged: sources of degree 0 rarely beat it, and a stale (empty)
        // key would send every CTA through the top-k lock
        if (tid == 0 && !p.exhaustive) read_thresholds(p.topk, s_thr);
        __syncthreads();
        flush_completions(p, s_cid, s_cf, s_cr, s_nc, s_thr, THREADS, s_stage, &s_go);
        __syncthreads();
        if (tid == 0) s_nc = 0;

        u32 d = 0, cur = 0;
        for (;;) {
            if (tid == 0) {
                if (!p.exhaustive) read_thresholds(p.topk, s_thr);
                s_chunk = 0;
            }
            __syncthreads();
            if (tid < L) {   // stopping rule at level d, before Gamma_d is expanded
                bool a = (s_alive32[tid >> 5] >> lane) & 1u;
                if (a && p.trace_lanes) lane_level(p, s_src[tid], d, s_f[tid], s_nd[tid], s_gt[tid]);
                if (a && !p.exhaustive && !p.nocut &&
                    bfscut_stops(s_f[tid], s_gt[tid], d, s_nd[tid], s_xlo[tid], s_xhi[tid], s_src[tid], s_thr)) {
                    a = false;
                    bstat_add(s_bst, ST_CUT, 1);
                    if (p.trace_lanes) lane_end(p, s_src[tid], d, s_f[tid], s_nd[tid], true);
                }
                u32 m = __ballot_sync(0xffffffffu, a);
                if (lane == 0) s_alive32[tid >> 5] = m;
            }
            __syncthreads();
            u32 any = 0;
#pragma unroll
            for (int i = 0; i < 2 * W; ++i) any |= s_alive32[i];
            if (!any) break;

            if (d > 0 && p.defer_words && (s_ln[cur] >= p.defer_words || s_arcs[cur] >= 8ull * p.defer_words)) {
                // a level too wide for one CTA is next (many frontier words,
                // or few with very many out-arcs): the live sources go to the
                // grid-wide pass, which runs them again from the start; the
                // wave ends here and its clear log resets every word it
                // touched
                if (tid < L) {
                    const bool a = (s_alive32[tid >> 5] >> lane) & 1u;
                    const u32 m = __ballot_sync(0xffffffffu, a);
                    u32 at = 0;
                    if (lane == 0 && m) {
                        at = atomicAdd(p.defer_n, (u32)__popc(m));
                        bstat_add(s_bst, ST_DEFERRED, __popc(m));
                    }
                    at = __shfl_sync(0xffffffffu, at, 0);
                    if (a) p.defer_src[at + __popc(m & lanemask_lt())] = s_src[tid];
                }
                break;
            }
            if (d == 0) source_prefix<THREADS>(G, s_src, s_alive32, L, s_pre, s_beg, s_wsum);
            u64* Fnext = S.F[cur ^ 1];
            {
                WarpQueue nq{&s_stage[(2 * wid) * QCAP], S.list[cur ^ 1], &s_ln[cur ^ 1], QCAP, 0};
                WarpQueue lq{&s_stage[(2 * wid + 1) * QCAP], S.clog, &s_logn, QCAP, 0};
                if (d == 0)
                    expand_sources<W, REC>(G, s_src, s_alive32, s_pre, s_beg, L, S.vis, Fnext, s_cg, s_cs,
                                           p.footnote, nq, lq, wid, NWARP, tid, THREADS, T, st);
                else
                    expand_entries<W, REC>(G, S.list[cur], s_ln[cur], S.F[cur], s_alive32, S.vis, Fnext, s_cg,
                                           s_cs, p.footnote, nq, lq, &s_chunk, wid, NWARP, Hc, T, st);
                if (d > 0) {
                    __syncthreads();   // the heavy list is complete
                    const u32 hn = s_hn < kHeavyCapCta ? s_hn : kHeavyCapCta;
                    if (hn)
                        expand_heavy<W, REC>(G, s_heavy, hn, S.vis, Fnext, s_cg, s_cs, p.footnote, nq, lq, wid,
                                             NWARP, T, st);
                }
                nq.flush();
                lq.flush();
                flush_fwarcs(st, &s_arcs[cur ^ 1]);
            }
            __syncthreads();
            if (s_full) {
                // the table passed its limit during this level, so some arcs
                // were dropped and the level's counts are incomplete: the
                // lanes live in it go to the grid-wide pass (where no such
                // pass follows, the run fails rather than use the counts)
                if (tid < L) {
                    const bool a = (s_alive32[tid >> 5] >> lane) & 1u;
                    const u32 m = __ballot_sync(0xffffffffu, a);
                    if (p.defer_src) {
                        u32 at = 0;
                        if (lane == 0 && m) {
                            at = atomicAdd(p.defer_n, (u32)__popc(m));
                            bstat_add(s_bst, ST_DEFERRED, __popc(m));
                        }
                        at = __shfl_sync(0xffffffffu, at, 0);
                        if (a) p.defer_src[at + __popc(m & lanemask_lt())] = s_src[tid];
                    }
                    s_cg[tid] = 0;
                    s_cs[tid] = 0;
                }
                if (tid == 0) {
                    s_hn = 0;
                    if (!p.defer_src) atomicOr(p.err, DEV_ERR_TABLE_FULL);
                }
                break;
            }
            if (tid < L) {   // level d+1 is known: gamma_{d+1} and its degree sum
                bool a = (s_alive32[tid >> 5] >> lane) & 1u;
                if (a) {
                    u32 gam = s_cg[tid];
                    if (gam == 0) {
                        u32 c = atomicAdd(&s_nc, 1u);
                        s_cid[c] = s_src[tid]; s_cf[c] = s_f[tid]; s_cr[c] = s_nd[tid];
                        a = false;
                        bstat_add(s_bst, ST_COMPLETED, 1);
                        if (p.trace_lanes) lane_end(p, s_src[tid], d, s_f[tid], s_nd[tid], false);
                    } else {
                        s_nd[tid] += gam;
                        s_f[tid] += (u64)(d + 1) * gam;
                        s_gt[tid] = s_cs[tid];
                    }
                }
                s_cg[tid] = 0;
                s_cs[tid] = 0;
                u32 m = __ballot_sync(0xffffffffu, a);
                if (lane == 0) s_alive32[tid >> 5] = m;
            }
            if (tid == 0) { s_ln[cur] = 0; s_arcs[cur] = 0; s_hn = 0; }
            __syncthreads();
            flush_completions(p, s_cid, s_cf, s_cr, s_nc, s_thr, THREADS, s_stage, &s_go);
            __syncthreads();
            if (tid == 0) s_nc = 0;
            cur ^= 1;
            ++d;
        }
        if (tid == 0) {
            bstat_add(s_bst, ST_LEVELS, d);
            bstat_max(s_bst, ST_MAXLEVEL, d);
        }
        // the wave's footprint: every word whose vis became non-zero (dense),
        // or every table entry it made, with its W words (hashed)
        const u32 nlog = s_logn;
        if (p.tab_shift) {
            for (u32 i = tid; i < nlog * W; i += THREADS) clear_word<REC>(S, __ldcg(&S.clog[i / W]) + i % W);
        } else {
            for (u32 i = tid; i < nlog; i += THREADS) clear_word<REC>(S, S.clog[i]);
        }
        if (tid == 0) {
            bstat_add(s_bst, ST_CLEARED, p.tab_shift ? nlog * W : nlog);
            trace_record(p, TR_CTA_WAVE, blockIdx.x, d, nlog, s_twave, global_ns());
        }
        __syncthreads();
        if (tid == 0) { s_logn = 0; s_ln[0] = 0; s_ln[1] = 0; s_arcs[0] = 0; s_arcs[1] = 0; }
    }
    __syncthreads();
    flush_stats(st, s_bst, p.stats);
}

// ------------------------------------------------------ one source per CTA
// BFSCut of one source at a time per CTA (Algorithm 2 as written: one BFS,
// the same stopping rule on the same per-level state as the wave kernels),
// on a visited bitmap of one bit per vertex and two queues.  For graphs
// whose sources' searches share almost no frontier: on a lattice the
// sources of a wave are consecutive vertices, and two BFS spheres cross only
// at points, so a bit lane per source fills one bit of each 64-bit word it
// touches and every arc costs a 32-byte record; here an arc costs a bit of a
// bitmap that stays in L2.
//
// The kernel is bound by the latency of each level's chain of dependent
// loads, so the chain is kept short.  A queue entry is the frontier
// vertex's arc range (first arc, degree), loaded with the vertex's degree by
// the thread that discovered it; each warp takes 32 entries at a time (its
// first chunk fixed, the rest from a counter), lays their arcs end to end
// and walks them 128 per step, four independent arcs per thread: the
// target's id, then its bitmap word and its own arc range (read for every
// arc, so that a discovery needs no further load), then atomicOr where the
// bit was clear; the thread whose atomicOr set the bit has discovered the
// vertex, appends its arc range to the next queue and counts it (gamma_{d+1})
// with its degree (for gamma~_{d+2}).  The threshold for the next level is
// read by one thread while the others expand; the stopping rule for level
// d+1 is evaluated with the level's update, so a level costs two block
// barriers.  Bitmap words that were zero are logged and cleared when the
// source ends.  A frontier longer than the queue gives the source up to the
// grid-wide pass (deferral), which runs it again from the start.
struct SQueue {   // WarpQueue of 8-byte entries with a capacity: entries past it are dropped and flagged
    uint2* sbuf;
    uint2* dst;
    u32* counter;
    u32 cap;
    u32 n;
    u32 lim;
    volatile u32* ovf;
    __device__ __forceinline__ void push(bool want, uint2 item) {
        const u32 m = __ballot_sync(0xffffffffu, want);
        if (want) sbuf[n + __popc(m & lanemask_lt())] = item;
        n += __popc(m);
    }
    __device__ __forceinline__ void flush() {
        if (n == 0) return;
        __syncwarp();
        u32 base = 0;
        if ((threadIdx.x & 31) == 0) base = atomicAdd(counter, n);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (u32 i = threadIdx.x & 31; i < n; i += 32)
            if (base + i < lim) dst[base + i] = sbuf[i];
        if ((threadIdx.x & 31) == 0 && base + n > lim) *ovf = 1;
        __syncwarp();
        n = 0;
    }
    __device__ __forceinline__ void reserve(u32 need) {
        if (n + need > cap) flush();
    }
};

constexpr int kSparseArcs = 4;   // independent arcs per thread and step

template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_sparse(WaveParams p) {
    constexpr int NWARP = THREADS / 32;
    constexpr u32 QCAP = 1024 / NWARP;   // staged entries per warp: next queue (8 B each) and log (4 B)
    static_assert(QCAP >= 32, "a warp stages up to 32 entries per push");
    constexpr u32 SCR = NWARP * QCAP * 3 > 4608 ? NWARP * QCAP * 3 : 4608;
    __shared__ __align__(16) u32 s_stage[SCR];   // staging, and flush_completions' scratch
    __shared__ u32 s_qn[2], s_logn, s_base, s_stop, s_cut, s_gam, s_dsum, s_ovf, s_chunk, s_nc;
    __shared__ u32 s_src, s_nd, s_gt, s_xlo, s_xhi;
    __shared__ u64 s_f;
    __shared__ u32 s_cid[1], s_cr[1];
    __shared__ u64 s_cf[1];
    __shared__ int s_go;
    __shared__ ThrCache s_thr, s_thr_next;
    __shared__ BlockStats s_bst;

    const u32 tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const GraphDev& G = p.g;
    const u32 n_end = p.n_end_dev ? vload(p.n_end_dev) : p.n_end;
    char* slot = p.slot_base + (size_t)blockIdx.x * p.slot_stride;
    u32* const vis = (u32*)slot;
    u32* const wlog = (u32*)(slot + sparse_bitmap_bytes(G.n));
    uint2* const q0 = (uint2*)(slot + 2 * sparse_bitmap_bytes(G.n));
    uint2* const q1 = q0 + al256((size_t)p.sparse_qcap * sizeof(uint2)) / sizeof(uint2);
    uint2* const stq = (uint2*)&s_stage[wid * QCAP * 3];   // QCAP entries of 8 bytes
    u32* const stl = &s_stage[wid * QCAP * 3 + 2 * QCAP];  // QCAP entries of 4 bytes
    LocalStats st;
    if (tid == 0) {
        s_thr.valid = 0; s_thr.N = 0; s_thr.F = 1; s_thr.id = 0;
        s_thr_next = s_thr;
        s_qn[0] = 0; s_qn[1] = 0; s_logn = 0; s_nc = 0;
    }
    bstat_init(s_bst);
    __syncthreads();

    for (;;) {
        if (tid == 0) {
            s_base = atomicAdd(p.head, 1u);
            s_stop = (s_base >= n_end) || (vload(p.err) != 0);
        }
        __syncthreads();
        if (s_stop) break;
        if (tid == 0) {
            const u32 v = __ldg(&p.sources[s_base]);
            const u32 beg = __ldg(&G.rp[v]);
            const u32 deg = __ldg(&G.rp[v + 1]) - beg;
            s_src = v; s_nd = 1; s_f = 0; s_gt = deg;
            s_xlo = __ldg(&G.xlo[v]); s_xhi = __ldg(&G.xhi[v]);
            s_ovf = 0; s_cut = 0; s_gam = 0; s_dsum = 0; s_chunk = 0;
            bstat_add(s_bst, ST_WAVES, 1);
            if (!p.exhaustive) read_thresholds(p.topk, s_thr);
            if (deg == 0) {   // R(v) = {v}: r = 1, f = 0
                s_cid[0] = v; s_cf[0] = 0; s_cr[0] = 1; s_nc = 1;
                bstat_add(s_bst, ST_COMPLETED, 1);
                if (p.trace_lanes) { lane_level(p, v, 0, 0, 1, 0); lane_end(p, v, 0, 0, 1, false); }
            } else {
                vis[v >> 5] = 1u << (v & 31);   // the bitmap is clean: no other bit of this word is set
                wlog[0] = v >> 5;
                s_logn = 1;
                q0[0] = make_uint2(beg, deg);
                s_qn[0] = 1;
                // stopping rule at level 0
                if (p.trace_lanes) lane_level(p, v, 0, 0, 1, deg);
                if (!p.exhaustive && !p.nocut && bfscut_stops(0, deg, 0, 1, s_xlo, s_xhi, v, s_thr)) {
                    s_cut = 1;
                    bstat_add(s_bst, ST_CUT, 1);
                    if (p.trace_lanes) lane_end(p, v, 0, 0, 1, true);
                }
            }
        }
        __syncthreads();
        u32 d = 0, cur = 0;
        while (!s_nc && !s_cut) {
            {
                if (wid == NWARP - 1 && lane == 0 && !p.exhaustive) read_thresholds(p.topk, s_thr_next);
                const u32 cnt = s_qn[cur];
                const uint2* qc = cur ? q1 : q0;
                SQueue nq{stq, cur ? q0 : q1, &s_qn[cur ^ 1], QCAP, 0, p.sparse_qcap, &s_ovf};
                WarpQueue lq{stl, wlog, &s_logn, QCAP, 0};
                u32 gam = 0, dsum = 0;
                bool first = true;
                for (;;) {
                    u32 b = wid * 32;
                    if (!first) {
                        u32 c = 0;
                        if (lane == 0) c = atomicAdd(&s_chunk, 32u);
                        b = NWARP * 32 + __shfl_sync(0xffffffffu, c, 0);
                    }
                    first = false;
                    if (b >= cnt) break;
                    const u32 e = b + lane;
                    uint2 ent = make_uint2(0, 0);
                    if (e < cnt) {
                        ent = __ldcg(&qc[e]);
                        st.mvis += ent.y;
                        st.arcwords += ent.y;
                        st.entries++;
                    }
                    const u32 beg = ent.x, deg = ent.y;
                    u32 incl = deg;
#pragma unroll
                    for (int o = 1; o < 32; o <<= 1) {
                        const u32 t = __shfl_up_sync(0xffffffffu, incl, o);
                        if (lane >= (u32)o) incl += t;
                    }
                    const u32 total = __shfl_sync(0xffffffffu, incl, 31);
                    const u32 excl = incl - deg;
                    for (u32 t0 = 0; t0 < total; t0 += 32 * kSparseArcs) {
                        u32 x[kSparseArcs], w[kSparseArcs], r0[kSparseArcs], r1[kSparseArcs];
                        bool v[kSparseArcs];
#pragma unroll
                        for (int j = 0; j < kSparseArcs; ++j) {
                            const u32 idx = t0 + 32 * j + lane;
                            int owner = 0;
#pragma unroll
                            for (int step = 16; step; step >>= 1) {
                                const u32 ex = __shfl_sync(0xffffffffu, excl, owner + step);
                                if (ex <= idx) owner += step;
                            }
                            const u32 o_beg = __shfl_sync(0xffffffffu, beg, owner);
                            const u32 o_excl = __shfl_sync(0xffffffffu, excl, owner);
                            v[j] = idx < total;
                            x[j] = v[j] ? __ldg(&G.col[o_beg + idx - o_excl]) : 0u;
                        }
#pragma unroll
                        for (int j = 0; j < kSparseArcs; ++j) {
                            w[j] = v[j] ? __ldcg(&vis[x[j] >> 5]) : ~0u;
                            r0[j] = v[j] ? __ldg(&G.rp[x[j]]) : 0u;
                            r1[j] = v[j] ? __ldg(&G.rp[x[j] + 1]) : 0u;
                        }
                        bool found[kSparseArcs], fresh[kSparseArcs];
#pragma unroll
                        for (int j = 0; j < kSparseArcs; ++j) {
                            const u32 bit = 1u << (x[j] & 31);
                            found[j] = false;
                            fresh[j] = false;
                            if (v[j] && !(w[j] & bit)) {
                                const u32 old = atomicOr(&vis[x[j] >> 5], bit);
                                found[j] = !(old & bit);
                                fresh[j] = old == 0;
                            }
                        }
#pragma unroll
                        for (int j = 0; j < kSparseArcs; ++j) {
                            if (found[j]) {
                                gam++;
                                dsum += r1[j] - r0[j] - p.footnote;
                            }
                            nq.reserve(32);
                            lq.reserve(32);
                            nq.push(found[j], make_uint2(r0[j], r1[j] - r0[j]));
                            lq.push(fresh[j], x[j] >> 5);
                        }
                    }
                }
                nq.flush();
                lq.flush();
                st.disc += gam;
                st.discwords += gam;
                for (int o = 16; o; o >>= 1) {
                    gam += __shfl_xor_sync(0xffffffffu, gam, o);
                    dsum += __shfl_xor_sync(0xffffffffu, dsum, o);
                }
                if (lane == 0 && gam) {
                    atomicAdd(&s_gam, gam);
                    atomicAdd(&s_dsum, dsum);
                }
            }
            __syncthreads();
            if (s_ovf) {
                // the next frontier did not fit its queue: the source goes to
                // the grid-wide pass (where none follows, the run fails
                // rather than use the level's counts)
                if (tid == 0) {
                    if (p.defer_src) {
                        p.defer_src[atomicAdd(p.defer_n, 1u)] = s_src;
                        bstat_add(s_bst, ST_DEFERRED, 1);
                    } else {
                        atomicOr(p.err, DEV_ERR_TABLE_FULL);
                    }
                }
                break;
            }
            if (tid == 0) {   // level d+1 is known: gamma_{d+1} and its degree sum; its stopping rule
                const u32 gam = s_gam;
                if (gam == 0) {
                    s_cid[0] = s_src; s_cf[0] = s_f; s_cr[0] = s_nd; s_nc = 1;
                    bstat_add(s_bst, ST_COMPLETED, 1);
                    if (p.trace_lanes) lane_end(p, s_src, d, s_f, s_nd, false);
                } else {
                    s_nd += gam;
                    s_f += (u64)(d + 1) * gam;
                    s_gt = s_dsum;
                    if (!p.exhaustive) s_thr = s_thr_next;
                    if (p.trace_lanes) lane_level(p, s_src, d + 1, s_f, s_nd, s_gt);
                    if (!p.exhaustive && !p.nocut &&
                        bfscut_stops(s_f, s_gt, d + 1, s_nd, s_xlo, s_xhi, s_src, s_thr)) {
                        s_cut = 1;
                        bstat_add(s_bst, ST_CUT, 1);
                        if (p.trace_lanes) lane_end(p, s_src, d + 1, s_f, s_nd, true);
                    }
                }
                s_qn[cur] = 0;
                s_gam = 0;
                s_dsum = 0;
                s_chunk = 0;
            }
            __syncthreads();
            cur ^= 1;
            ++d;
        }
        if (tid == 0) {
            bstat_add(s_bst, ST_LEVELS, d);
            bstat_max(s_bst, ST_MAXLEVEL, d);
        }
        // the source's footprint: every bitmap word it made non-zero
        const u32 nlog = s_logn;
        for (u32 i = tid; i < nlog; i += THREADS) vis[__ldcg(&wlog[i])] = 0;
        flush_completions(p, s_cid, s_cf, s_cr, s_nc, s_thr, THREADS, s_stage, &s_go);
        __syncthreads();
        if (tid == 0) {
            bstat_add(s_bst, ST_CLEARED, nlog);
            s_logn = 0; s_qn[0] = 0; s_qn[1] = 0; s_nc = 0;
        }
        __syncthreads();
    }
    __syncthreads();
    flush_stats(st, s_bst, p.stats);
}

// ------------------------------------------------------------ grid waves
// The whole grid runs waves one after another, taking 64*W sources at
// order[*head] each time.  Each block keeps an identical copy of the lane
// state; per-level counters are summed in global memory between two grid
// barriers; block 0 owns the top-k.  After each wave the grid decides, from
// values every block read after the same barriers, whether the wave was
// wide (its frontiers averaged at least p.heavy_words words per level):
// only wide levels use the whole GPU well, while a long thin wave (a
// high-diameter graph) is better left to one CTA.  On the first narrow wave
// the kernel returns and leaves *head where the per-CTA kernel continues;
// exhaustive runs stay until the queue is empty.
// Push or pull for a level whose frontier words have `farcs` out-arcs.
// Push pays per frontier arc.  Pull pays a scan of every vertex's vis words
// plus the in-lists of the vertices some live lane has not reached, and in a
// multi-source BFS those rarely end early (every pending lane must be found),
// so its cost is estimated as n/4 + (n - min n_d) * m/n, with min n_d the
// fewest vertices any live lane has reached: a lattice's thin frontiers stay
// push while most of the graph is unreached, a power-law graph's wide ones
// pull.  A level also needs at least n*W/pull_div frontier arcs to be pulled.
constexpr u64 kPullAlpha = 4;   // push arcs worth one unit of the pull estimate

__device__ __forceinline__ bool pull_wanted(const WaveParams& p, int W, u64 farcs, u32 min_nd) {
    const GraphDev& G = p.g;
    if (p.all_pull) return true;
    if (!p.pull_div || farcs < ((u64)G.n * W + p.pull_div - 1) / p.pull_div) return false;
    const u64 pending = (u64)(G.n - (min_nd < G.n ? min_nd : G.n));
    return kPullAlpha * farcs >= G.n / 4 + pending * G.m / (G.n ? G.n : 1);
}

// CTAs per SM the grid kernel is compiled for (its register budget is
// 65536 / (this * THREADS) per thread)
#ifndef BCM_GRID_MIN_BLOCKS
#define BCM_GRID_MIN_BLOCKS 2
#endif

template <int W, int THREADS>
__global__ void __launch_bounds__(THREADS, BCM_GRID_MIN_BLOCKS) k_wave_grid(WaveParams p) {
    constexpr int L = 64 * W;
    constexpr int NWARP = THREADS / 32;
    static_assert(THREADS >= L, "one thread per lane");
    __shared__ u32 s_src[L], s_nd[L], s_gt[L], s_xlo[L], s_xhi[L];
    __shared__ u64 s_f[L];
    __shared__ u32 s_cg[L], s_cs[L];
    __shared__ u32 s_alive32[2 * W];
    __shared__ u32 s_nc, s_base;
    __shared__ u32 s_minnd;   // fewest vertices a live lane has reached (push or pull)
    __shared__ u32 s_pgam[L]; // each lane's gamma of the frontier being expanded (m_vis of a pulled level)
    __shared__ ThrCache s_thr;
    __shared__ BlockStats s_bst;
    constexpr u32 QCAP = 4096 / NWARP;
    __shared__ __align__(16) u32 s_stage[NWARP * 2 * QCAP];
    static_assert(NWARP * 2 * QCAP >= 4608, "flush_completions scratch");
    __shared__ u32 s_cid[L], s_cr[L];
    __shared__ u64 s_cf[L];
    __shared__ u32 s_pre[L + 1], s_beg[L], s_wsum[L / 32];
    __shared__ int s_go;

    const u32 tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool leader = blockIdx.x == 0;
    const GraphDev& G = p.g;
    // planes of 4 words per vertex whatever W is, so runs of different
    // widths never put bit arrays where another left lists or logs
    SlotPtrs S = slot_ptrs<1>(p.seed_base, G.n, 4);

    LocalStats st;
    const u32 gnw = gridDim.x * NWARP;
    // the same warps numbered across blocks first: work dealt by warp number
    // (first chunks, pulled batches, heavy pieces) then spreads over every
    // block and SM before a second warp of any block gets some
    const u32 pw = wid * gridDim.x + blockIdx.x;
    const u32 n_end = p.n_end_dev ? vload(p.n_end_dev) : p.n_end;
    const HeavyList Hg{p.gheavy, p.gheavy_n, p.gheavy_cap};
    if (tid == 0) { s_nc = 0; s_thr.valid = 0; s_thr.N = 0; s_thr.F = 1; s_thr.id = 0; }
    // every block cuts with the leader's snapshot of the threshold, taken
    // before a barrier and read after it
    if (leader && tid == 0) {
        if (!p.exhaustive) read_thresholds(p.topk, s_thr);
        store_snapshot(p.snap, s_thr);
    }
    bstat_init(s_bst);
    bool ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err);

    for (u32 wave = 0; ok && wave < p.max_grid_waves; ++wave) {
        if (tid == 0) s_base = vload(p.head);
        __syncthreads();
        const u32 base = s_base;
        if (base >= n_end) break;
        if (tid < L) {
            bool alive = false;
            s_cg[tid] = 0;
            s_cs[tid] = 0;
            if (base + tid < n_end) {
                u32 v = __ldg(&p.sources[base + tid]);
                u32 deg = __ldg(&G.rp[v + 1]) - __ldg(&G.rp[v]);
                s_src[tid] = v; s_nd[tid] = 1; s_f[tid] = 0; s_gt[tid] = deg;
                s_xlo[tid] = __ldg(&G.xlo[v]); s_xhi[tid] = __ldg(&G.xhi[v]);
                if (deg == 0) {
                    if (leader) {
                        u32 c = atomicAdd(&s_nc, 1u);
                        s_cid[c] = v; s_cf[c] = 0; s_cr[c] = 1;
                        bstat_add(s_bst, ST_COMPLETED, 1);
                        if (p.trace_lanes) { lane_level(p, v, 0, 0, 1, 0); lane_end(p, v, 0, 0, 1, false); }
                    }
                } else {
                    alive = true;
                }
            }
            u32 m = __ballot_sync(0xffffffffu, alive);
            if (lane == 0) s_alive32[tid >> 5] = m;
        }
        __syncthreads();
        if (leader) flush_completions(p, s_cid, s_cf, s_cr, s_nc, s_thr, THREADS, s_stage, &s_go);
        __syncthreads();
        if (tid == 0) s_nc = 0;
        if (leader && tid == 0 && !p.exhaustive) {
            read_thresholds(p.topk, s_thr);
            store_snapshot(p.snap, s_thr);
        }
        if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;

        u32 d = 0, cur = 0;
        u64 wave_entries = 0;
        bool pulled = false;
        u32 level_cnt = 0;   // entries of the level's frontier list, read before it can be reset
        for (;;) {
            if (tid == 0) {
                if (!p.exhaustive) load_snapshot(p.snap, s_thr);
                s_minnd = 0xffffffffu;
            }
            __syncthreads();
            if (tid < L) {
                bool a = (s_alive32[tid >> 5] >> lane) & 1u;
                if (a && leader && p.trace_lanes) lane_level(p, s_src[tid], d, s_f[tid], s_nd[tid], s_gt[tid]);
                if (a && !p.exhaustive && !p.nocut &&
                    bfscut_stops(s_f[tid], s_gt[tid], d, s_nd[tid], s_xlo[tid], s_xhi[tid], s_src[tid], s_thr)) {
                    a = false;
                    if (leader) bstat_add(s_bst, ST_CUT, 1);
                    if (leader && p.trace_lanes) lane_end(p, s_src[tid], d, s_f[tid], s_nd[tid], true);
                }
                if (a) atomicMin(&s_minnd, s_nd[tid]);
                u32 m = __ballot_sync(0xffffffffu, a);
                if (lane == 0) s_alive32[tid >> 5] = m;
            }
            __syncthreads();
            u32 any = 0;
#pragma unroll
            for (int i = 0; i < 2 * W; ++i) any |= s_alive32[i];
            if (!any) break;

            if (p.trace && leader && tid == 0) {
                u32 alive = 0;
                for (int i = 0; i < 2 * W; ++i) alive += __popc(s_alive32[i]);
                const u32 cnt = d ? vload(&p.glist_n[cur]) : 0u;
                const u64 arcs = d ? vload(&p.garc[cur]) : 0ull;
                const bool pull = d && pull_wanted(p, W, arcs, s_minnd);
                trace_record(p, TR_GRID_LEVEL, wave, d, cnt, alive | ((u64)pull << 16) | (arcs << 20), global_ns());
            }
            if (d == 0) source_prefix<THREADS>(G, s_src, s_alive32, L, s_pre, s_beg, s_wsum);
            const u32 par = d & 1;
            u32* const gcpar = p.gcnt + par * kCntParity;                   // this level's counters
            u32* gcg = gcpar + (blockIdx.x % kCntCopies) * 512;             // this block's copy
            u32* gcs = gcg + 256;
            {
                WarpQueue nq{&s_stage[(2 * wid) * QCAP], S.list[cur ^ 1], &p.glist_n[cur ^ 1], QCAP, 0};
                WarpQueue lq{&s_stage[(2 * wid + 1) * QCAP], S.clog, p.glog_n, QCAP, 0};
                if (d == 0) {
                    expand_sources<W, 1>(G, s_src, s_alive32, s_pre, s_beg, L, S.vis, S.F[cur ^ 1], s_cg, s_cs,
                                         p.footnote, nq, lq, pw, gnw, blockIdx.x * THREADS + tid,
                                         gridDim.x * THREADS, kDenseTab, st);
                } else {
                    const u32 cnt = vload(&p.glist_n[cur]);
                    level_cnt = cnt;
                    wave_entries += cnt;
                    pulled = pull_wanted(p, W, vload(&p.garc[cur]), s_minnd);
                    if (pulled) {
                        pull_level<W>(G, S.F[cur], s_alive32, S.vis, S.F[cur ^ 1], s_cg, s_cs, p.footnote, nq, lq,
                                      &p.gchunk[cur], pw, gnw, st);
                    } else {
                        expand_entries<W, 1>(G, S.list[cur], cnt, S.F[cur], s_alive32, S.vis, S.F[cur ^ 1], s_cg,
                                             s_cs, p.footnote, nq, lq, &p.gchunk[cur], pw, gnw, Hg, kDenseTab, st);
                    }
                }
                nq.flush();
                lq.flush();
                flush_fwarcs(st, &p.garc[cur ^ 1]);
            }
            __syncthreads();
            if (tid < L) {
                if (s_cg[tid]) { atomicAdd(&gcg[tid], s_cg[tid]); atomicAdd(&gcs[tid], s_cs[tid]); }
                s_cg[tid] = 0;
                s_cs[tid] = 0;
            }
            if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
            {
                // the heavy entries of a push level, shared by every warp of
                // the grid (one more barrier, only when there are any)
                u32 hn = vload(p.gheavy_n);
                hn = hn < p.gheavy_cap ? hn : p.gheavy_cap;
                if (hn) {
                    {
                        WarpQueue nq{&s_stage[(2 * wid) * QCAP], S.list[cur ^ 1], &p.glist_n[cur ^ 1], QCAP, 0};
                        WarpQueue lq{&s_stage[(2 * wid + 1) * QCAP], S.clog, p.glog_n, QCAP, 0};
                        expand_heavy<W, 1>(G, p.gheavy, hn, S.vis, S.F[cur ^ 1], s_cg, s_cs, p.footnote, nq, lq,
                                           pw, gnw, kDenseTab, st);
                        nq.flush();
                        lq.flush();
                        flush_fwarcs(st, &p.garc[cur ^ 1]);
                    }
                    __syncthreads();
                    if (tid < L) {
                        if (s_cg[tid]) { atomicAdd(&gcg[tid], s_cg[tid]); atomicAdd(&gcs[tid], s_cs[tid]); }
                        s_cg[tid] = 0;
                        s_cs[tid] = 0;
                    }
                    if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
                }
            }
            if (pulled) {   // every block is past the pull: retire the frontier words
                // (the count read at the level's start: the leader resets
                // glist_n[cur] below while slower blocks may still be here)
                pull_clear<1>(S.list[cur], level_cnt, S.F[cur], blockIdx.x * THREADS + tid, gridDim.x * THREADS);
                // the arcs a push would have scanned (m_vis counts those
                // whichever direction ran): a live lane's frontier out-arcs
                // are its gamma-tilde sum plus the footnote's 1 per vertex,
                // and its frontier count is still in the previous level's
                // counters (cleared at this level's end)
                if (leader) {
                    if (tid < L && ((s_alive32[tid >> 5] >> lane) & 1u))
                        st.mvis += (u64)s_gt[tid] + (u64)p.footnote * s_pgam[tid];
                    if (tid == 0) {
                        bstat_add(s_bst, ST_ENTRIES, level_cnt);
                        bstat_add(s_bst, ST_PULLENTRIES, level_cnt);
                    }
                }
                pulled = false;
                __syncthreads();
            }
            if (tid < L) {
                bool a = (s_alive32[tid >> 5] >> lane) & 1u;
                if (a) {
                    u32 gam = 0, dsum = 0;
#pragma unroll
                    for (u32 c = 0; c < kCntCopies; ++c) {
                        gam += vload(&gcpar[c * 512 + tid]);
                        dsum += vload(&gcpar[c * 512 + 256 + tid]);
                    }
                    s_pgam[tid] = gam;
                    if (gam == 0) {
                        if (leader) {
                            u32 c = atomicAdd(&s_nc, 1u);
                            s_cid[c] = s_src[tid]; s_cf[c] = s_f[tid]; s_cr[c] = s_nd[tid];
                            bstat_add(s_bst, ST_COMPLETED, 1);
                            if (p.trace_lanes) lane_end(p, s_src[tid], d, s_f[tid], s_nd[tid], false);
                        }
                        a = false;
                    } else {
                        s_nd[tid] += gam;
                        s_f[tid] += (u64)(d + 1) * gam;
                        s_gt[tid] = dsum;
                    }
                }
                u32 m = __ballot_sync(0xffffffffu, a);
                if (lane == 0) s_alive32[tid >> 5] = m;
            }
            if (leader) {   // buffers of the next level: counters par^1, list count and chunk counter
                u32* nx = p.gcnt + (par ^ 1) * kCntParity;
                for (u32 i = tid; i < kCntParity; i += THREADS) nx[i] = 0;
                if (tid == 0) {
                    p.glist_n[cur] = 0;
                    p.garc[cur] = 0;
                    p.gchunk[cur ^ 1] = 0;
                    *p.gheavy_n = 0;
                }
            }
            __syncthreads();
            if (leader) flush_completions(p, s_cid, s_cf, s_cr, s_nc, s_thr, THREADS, s_stage, &s_go);
            __syncthreads();
            if (tid == 0) s_nc = 0;
            if (leader && tid == 0 && !p.exhaustive) {
                read_thresholds(p.topk, s_thr);
                store_snapshot(p.snap, s_thr);
            }
            if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
            cur ^= 1;
            ++d;
        }
        if (!ok) break;
        if (leader && tid == 0) {
            bstat_add(s_bst, ST_WAVES, 1);
            bstat_add(s_bst, ST_LEVELS, d);
            bstat_max(s_bst, ST_MAXLEVEL, d);
        }
        // clear the wave's footprint: every block has finished expanding
        // (the level loop ends at a barrier or on a decision all blocks share)
        if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
        const u32 nlog = vload(p.glog_n);
        for (u32 i = blockIdx.x * THREADS + tid; i < nlog; i += gridDim.x * THREADS) clear_word<1>(S, __ldcg(&S.clog[i]));
        if (leader && tid == 0) bstat_add(s_bst, ST_CLEARED, nlog);
        if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
        if (leader && tid == 0) trace_record(p, TR_GRID_WAVE, wave, d, nlog, wave_entries, global_ns());
        if (leader) {   // reset per-wave counters and advance the queue
            for (u32 i = tid; i < 2 * kCntParity; i += THREADS) p.gcnt[i] = 0;
            if (tid == 0) {
                p.glist_n[0] = 0;
                p.glist_n[1] = 0;
                p.garc[0] = 0;
                p.garc[1] = 0;
                p.gchunk[0] = 0;
                p.gchunk[1] = 0;
                *p.glog_n = 0;
                *p.head = base + L;
            }
        }
        if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
        // light (its levels averaged fewer than heavy_words frontier words):
        // hand the rest of the queue over to the CTAs
        if (!p.exhaustive && wave_entries < p.heavy_words * (u64)(d ? d : 1)) break;
    }
    __syncthreads();
    flush_stats(st, s_bst, p.stats);
}

// --------------------------------------------------- plain, one source
// BFSCut(v, x_k) for v = order[it] alone: visit stamps (stamp[w] == it+1 means
// visited), a vertex queue per level, the same stopping rule and schedule.
template <int THREADS>
__global__ void __launch_bounds__(THREADS) k_plain(WaveParams p, u32 it, u32* stamp, u32* lists) {
    constexpr int NWARP = THREADS / 32;
    __shared__ u32 s_cg, s_cs;
    __shared__ ThrCache s_thr;
    __shared__ int s_go;
    __shared__ BlockStats s_bst;
    const u32 tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool leader = blockIdx.x == 0;
    const GraphDev& G = p.g;
    const u32 n = G.n;
    const u32 v = __ldg(&G.order[it]);
    const u32 s = it + 1;
    LocalStats st;
    if (tid == 0) {
        s_cg = 0; s_cs = 0;
        s_thr.valid = 0; s_thr.N = 0; s_thr.F = 1; s_thr.id = 0;
        load_snapshot(p.snap, s_thr);   // fixed for this launch: the previous launch's end took it
    }
    bstat_init(s_bst);
    __syncthreads();
    const u32 xlo = __ldg(&G.xlo[v]), xhi = __ldg(&G.xhi[v]);
    u32 d = 0, cur = 0, nd = 1;
    u64 f = 0;
    u32 gt = __ldg(&G.rp[v + 1]) - __ldg(&G.rp[v]);
    bool done = false, cut = false, ok = true;
    const u32 gw = blockIdx.x * NWARP + wid, gnw = gridDim.x * NWARP;
    while (ok) {
        if (leader && tid == 0 && p.trace_lanes) lane_level(p, v, d, f, nd, gt);
        if (!p.nocut && bfscut_stops(f, gt, d, nd, xlo, xhi, v, s_thr)) { cut = true; break; }
        const u32 par = d & 1;
        u32* gcg = p.gcnt + par * kCntParity;
        u32* gcs = gcg + 256;
        u32* nlist = lists + (size_t)(cur ^ 1) * n;
        u32* nn = &p.glist_n[cur ^ 1];
        if (d == 0) {
            if (leader && tid == 0) stamp[v] = s;
            u32 beg = __ldg(&G.rp[v]), end = __ldg(&G.rp[v + 1]);
            if (gw == 0 && lane == 0) st.mvis += end - beg;
            for (u32 e0 = beg + gw * 32; e0 < end; e0 += gnw * 32) {
                u32 e = e0 + lane;
                bool app = false;
                u32 x = 0;
                if (e < end) {
                    x = __ldg(&G.col[e]);
                    if (x != v && __ldcg(&stamp[x]) != s && atomicExch(&stamp[x], s) != s) {
                        app = true;
                        atomicAdd(&s_cg, 1u);
                        atomicAdd(&s_cs, __ldg(&G.rp[x + 1]) - __ldg(&G.rp[x]) - p.footnote);
                    }
                }
                warp_append(app, x, nlist, nn);
            }
        } else {
            const u32* clist = lists + (size_t)cur * n;
            const u32 cnt = vload(&p.glist_n[cur]);
            for (u32 base = gw * 32; base < cnt; base += gnw * 32) {
                u32 e = base + lane;
                u32 beg = 0, deg = 0;
                if (e < cnt) {
                    u32 u = __ldcg(&clist[e]);
                    beg = __ldg(&G.rp[u]);
                    deg = __ldg(&G.rp[u + 1]) - beg;
                    st.mvis += deg;
                }
                u32 incl = deg;
#pragma unroll
                for (int o = 1; o < 32; o <<= 1) {
                    u32 t = __shfl_up_sync(0xffffffffu, incl, o);
                    if (lane >= (u32)o) incl += t;
                }
                u32 total = __shfl_sync(0xffffffffu, incl, 31);
                u32 excl = incl - deg;
                for (u32 t0 = 0; t0 < total; t0 += 32) {
                    u32 idx = t0 + lane;
                    int owner = 0;
#pragma unroll
                    for (int step = 16; step; step >>= 1) {
                        u32 ex = __shfl_sync(0xffffffffu, excl, owner + step);
                        if (ex <= idx) owner += step;
                    }
                    u32 o_beg = __shfl_sync(0xffffffffu, beg, owner);
                    u32 o_excl = __shfl_sync(0xffffffffu, excl, owner);
                    bool app = false;
                    u32 x = 0;
                    if (idx < total) {
                        x = __ldg(&G.col[o_beg + idx - o_excl]);
                        if (__ldcg(&stamp[x]) != s && atomicExch(&stamp[x], s) != s) {
                            app = true;
                            atomicAdd(&s_cg, 1u);
                            atomicAdd(&s_cs, __ldg(&G.rp[x + 1]) - __ldg(&G.rp[x]) - p.footnote);
                        }
                    }
                    warp_append(app, x, nlist, nn);
                }
            }
        }
        __syncthreads();
        if (tid == 0 && s_cg) { atomicAdd(&gcg[0], s_cg); atomicAdd(&gcs[0], s_cs); s_cg = 0; s_cs = 0; }
        if (!grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err)) { ok = false; break; }
        u32 gam = vload(&gcg[0]);
        if (leader && tid == 0) {
            u32* nx = p.gcnt + (par ^ 1) * kCntParity;
            nx[0] = 0; nx[256] = 0;
            p.glist_n[cur] = 0;
        }
        if (gam == 0) { done = true; }
        else { ++d; nd += gam; f += (u64)d * gam; gt = vload(&gcs[0]); }
        if (!grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err)) { ok = false; break; }
        if (done) break;
        cur ^= 1;
    }
    // leave the shared buffers zeroed for the next launch, then insert
    if (ok) ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err);
    if (leader && tid == 0) {
        p.gcnt[0] = 0; p.gcnt[256] = 0; p.gcnt[kCntParity] = 0; p.gcnt[kCntParity + 256] = 0;
        p.glist_n[0] = 0; p.glist_n[1] = 0;
        bstat_add(s_bst, ST_LEVELS, d);
        bstat_max(s_bst, ST_MAXLEVEL, d);
        bstat_add(s_bst, ST_WAVES, 1);
        if (cut) bstat_add(s_bst, ST_CUT, 1);
        if (p.trace_lanes && ((done && ok) || cut)) lane_end(p, v, d, f, nd, cut);
        if (done && ok) {
            bstat_add(s_bst, ST_COMPLETED, 1);
            if (lock_acquire(p.topk.lock, p.lock_limit_ns, p.err)) {
                topk_insert_locked(p.topk, v, f, nd);
                topk_publish_locked(p.topk);
                lock_release(p.topk.lock);
            }
        }
        // the next launch's threshold, the same for all its blocks
        ThrCache c = s_thr;
        read_thresholds(p.topk, c);
        store_snapshot(p.snap, c);
    }
    (void)s_go;
    __syncthreads();
    flush_stats(st, s_bst, p.stats);
}

// ------------------------------------------------------------- launchers
template <int W, int T>
static int launch_cta_t(const WaveParams& p, int blocks, cudaStream_t s) {
    k_wave_cta<W, T><<<blocks, T, 0, s>>>(p);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_cta_waves(const WaveParams& p, int W, int blocks, int threads, cudaStream_t s) {
#define CASE(w, t) if (W == w && threads == t) return launch_cta_t<w, t>(p, blocks, s);
    CASE(1, 256) CASE(1, 512) CASE(1, 1024)
    CASE(2, 256) CASE(2, 512) CASE(2, 1024)
    CASE(4, 256) CASE(4, 512) CASE(4, 1024)
#undef CASE
    return -2;
}

template <int W, int T>
static int launch_grid_t(const WaveParams& p, int blocks, cudaStream_t s) {
    void* args[] = {(void*)&p};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_wave_grid<W, T>, dim3(blocks), dim3(T), args, 0, s);
    note_launch();
    return e == cudaSuccess ? 0 : -1;
}

int launch_grid_waves(const WaveParams& p, int W, int blocks, int threads, cudaStream_t s) {
    if (threads != 512) return -2;
    if (W == 1) return launch_grid_t<1, 512>(p, blocks, s);
    if (W == 2) return launch_grid_t<2, 512>(p, blocks, s);
    if (W == 4) return launch_grid_t<4, 512>(p, blocks, s);
    return -2;
}

int launch_plain_source(const WaveParams& p, uint32_t it, uint32_t* stamp, uint32_t* lists, int blocks,
                        int threads, cudaStream_t s) {
    if (threads != 256) return -2;
    void* args[] = {(void*)&p, (void*)&it, (void*)&stamp, (void*)&lists};
    cudaError_t e = cudaLaunchCooperativeKernel((const void*)k_plain<256>, dim3(blocks), dim3(256), args, 0, s);
    note_launch();
    return e == cudaSuccess ? 0 : -1;
}

int max_coop_blocks(int kind, int W, int threads) {
    int dev = 0, sms = 0, per = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const void* f = nullptr;
    if (kind == 1) f = (const void*)k_plain<256>;
    else if (W == 1) f = (const void*)k_wave_grid<1, 512>;
    else if (W == 2) f = (const void*)k_wave_grid<2, 512>;
    else f = (const void*)k_wave_grid<4, 512>;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, threads, 0) != cudaSuccess) return 0;
    return per * sms;
}

template <int T>
static int launch_sparse_t(const WaveParams& p, int blocks, cudaStream_t s) {
    k_sparse<T><<<blocks, T, 0, s>>>(p);
    note_launch();
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_sparse(const WaveParams& p, int blocks, int threads, cudaStream_t s) {
    if (threads == 128) return launch_sparse_t<128>(p, blocks, s);
    if (threads == 256) return launch_sparse_t<256>(p, blocks, s);
    if (threads == 512) return launch_sparse_t<512>(p, blocks, s);
    if (threads == 1024) return launch_sparse_t<1024>(p, blocks, s);
    return -2;
}

int sparse_blocks_per_sm(int threads) {
    const void* f = threads == 128 ? (const void*)k_sparse<128>
                  : threads == 256 ? (const void*)k_sparse<256>
                  : threads == 512 ? (const void*)k_sparse<512>
                  : threads == 1024 ? (const void*)k_sparse<1024> : nullptr;
    if (!f) return 0;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, threads, 0) != cudaSuccess) return 0;
    return per;
}

int cta_blocks_per_sm(int W, int threads) {
    const void* f = nullptr;
#define CASE(w, t) if (W == w && threads == t) f = (const void*)k_wave_cta<w, t>;
    CASE(1, 256) CASE(1, 512) CASE(1, 1024)
    CASE(2, 256) CASE(2, 512) CASE(2, 1024)
    CASE(4, 256) CASE(4, 512) CASE(4, 1024)
#undef CASE
    if (!f) return 0;
    int per = 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, f, threads, 0) != cudaSuccess) return 0;
    return per;
}

}  // namespace bcm
