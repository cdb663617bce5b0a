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

struct SlotPtrs {
    u64* vis;
    u64* F[2];
    u32* list[2];
    u32* clog;
};

__device__ __forceinline__ SlotPtrs slot_ptrs(char* base, u32 n, int W) {
    size_t nw = (size_t)n * W;
    SlotPtrs s;
    s.vis = (u64*)base;
    s.F[0] = s.vis + nw;
    s.F[1] = s.F[0] + nw;
    s.list[0] = (u32*)(s.F[1] + nw);
    s.list[1] = s.list[0] + nw;
    s.clog = s.list[1] + nw;
    return s;
}

struct LocalStats {
    u64 mvis = 0, disc = 0, entries = 0, arcwords = 0, discwords = 0, cleared = 0;
    u64 completed = 0, cut = 0, waves = 0, levels = 0, maxlevel = 0;
};

__device__ inline void flush_stats(const LocalStats& s, unsigned long long* g) {
    // warp-reduce then one atomic per warp and counter
    u64 v[ST_COUNT] = {s.mvis, s.disc, s.completed, s.cut, s.waves, s.levels, s.maxlevel,
                       s.entries, s.arcwords, s.discwords, s.cleared};
#pragma unroll
    for (int i = 0; i < ST_COUNT; ++i) {
        u64 x = v[i];
        for (int o = 16; o; o >>= 1) {
            u64 t = __shfl_xor_sync(0xffffffffu, x, o);
            x = (i == ST_MAXLEVEL) ? (t > x ? t : x) : x + t;
        }
        if ((threadIdx.x & 31) == 0 && x) {
            if (i == ST_MAXLEVEL) atomicMax(&g[i], x);
            else atomicAdd(&g[i], x);
        }
    }
}

// ------------------------------------------------------------ push step
// Lanes F of word g reach x.  Returns bit 0: x's F-next word was empty
// (append it to the next frontier); bit 1: x's vis word was empty (append it
// to the clear log).  Discoveries are counted per lane in cg (gamma) and cs
// (sum of deg, minus one under the undirected footnote).
template <int W>
__device__ __forceinline__ u32 push_word(const u32* __restrict__ rp, u64* vis, u64* Fnext, u32* cg, u32* cs,
                                         u32 foot, u32 x, u64 F, u32 g, LocalStats& st) {
    u32 word = x * W + g;
    u64 nb = F & ~__ldcg(&vis[word]);
    if (!nb) return 0;
    u64 old = atomicOr(&vis[word], nb);
    u32 fl = (old == 0) ? 2u : 0u;
    nb &= ~old;
    if (!nb) return fl;
    u64 oldF = atomicOr(&Fnext[word], nb);
    if (oldF == 0) { fl |= 1u; st.discwords++; }
    u32 degp = __ldg(&rp[x + 1]) - __ldg(&rp[x]) - foot;
    st.disc += __popcll(nb);
    u32* cgg = cg + g * 64;
    u32* csg = cs + g * 64;
    while (nb) {
        int j = __ffsll((long long)nb) - 1;
        nb &= nb - 1;
        atomicAdd(&cgg[j], 1u);
        atomicAdd(&csg[j], degp);
    }
    return fl;
}

// Level 0: lane j's frontier is its source.  One warp per source, arcs in
// warp-wide strips.  The source's own bit is set first, by the same warp.
template <int W>
__device__ inline void expand_sources(const GraphDev& G, const u32* s_src, const u32* s_alive32, int L,
                                      u64* vis, u64* Fnext, u32* cg, u32* cs, u32 foot,
                                      u32* next_list, u32* next_n, u32* clog, u32* log_n,
                                      u32 wid, u32 nw, LocalStats& st) {
    const u32 lane = threadIdx.x & 31;
    for (u32 j = wid; j < (u32)L; j += nw) {
        if (!((s_alive32[j >> 5] >> (j & 31)) & 1u)) continue;
        u32 u = s_src[j], g = j >> 6;
        u64 F = 1ull << (j & 63);
        u32 beg = __ldg(&G.rp[u]), end = __ldg(&G.rp[u + 1]);
        if (lane == 0) {
            u64 old = atomicOr(&vis[u * W + g], F);
            if (old == 0) clog[atomicAdd(log_n, 1u)] = u * W + g;
            st.mvis += end - beg;
            st.arcwords += end - beg;
        }
        __syncwarp();
        for (u32 e0 = beg; e0 < end; e0 += 32) {
            u32 e = e0 + lane;
            u32 fl = 0, word = 0;
            if (e < end) {
                u32 x = __ldg(&G.col[e]);
                word = x * W + g;
                fl = push_word<W>(G.rp, vis, Fnext, cg, cs, foot, x, F, g, st);
            }
            warp_append(fl & 1u, word, next_list, next_n);
            warp_append(fl & 2u, word, clog, log_n);
        }
    }
}

// Level >= 1: frontier words from `list`; each warp takes 32 entries, forms
// the exclusive scan of their degrees, and walks the combined arc range 32
// arcs at a time (balanced across high- and low-degree entries).
template <int W>
__device__ inline void expand_entries(const GraphDev& G, const u32* list, u32 cnt, u64* Fcur,
                                      const u32* s_alive32, u64* vis, u64* Fnext, u32* cg, u32* cs,
                                      u32 foot, u32* next_list, u32* next_n, u32* clog, u32* log_n,
                                      u32 wid, u32 nw, LocalStats& st) {
    const u32 lane = threadIdx.x & 31;
    for (u32 base = wid * 32; base < cnt; base += nw * 32) {
        u32 e = base + lane;
        u32 g = 0, beg = 0, deg = 0;
        u64 F = 0;
        if (e < cnt) {
            u32 word = __ldcg(&list[e]);
            u32 u = word / W;
            g = word - u * W;
            F = __ldcg(&Fcur[word]);
            Fcur[word] = 0;
            F &= ((u64)s_alive32[2 * g + 1] << 32) | s_alive32[2 * g];
            st.entries++;
            if (F) {
                beg = __ldg(&G.rp[u]);
                deg = __ldg(&G.rp[u + 1]) - beg;
                st.mvis += (u64)__popcll(F) * deg;
                st.arcwords += deg;
            }
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
            u64 o_F = __shfl_sync(0xffffffffu, F, owner);
            u32 o_g = __shfl_sync(0xffffffffu, g, owner);
            u32 fl = 0, word = 0;
            if (idx < total) {
                u32 x = __ldg(&G.col[o_beg + idx - o_excl]);
                word = x * W + o_g;
                fl = push_word<W>(G.rp, vis, Fnext, cg, cs, foot, x, o_F, o_g, st);
            }
            warp_append(fl & 1u, word, next_list, next_n);
            warp_append(fl & 2u, word, clog, log_n);
        }
    }
}

// Completed lanes: exhaustive runs write (f, r) by vertex id; top-k runs
// insert, under the lock, the entries that beat the cached k-th key.
__device__ inline void flush_completions(const WaveParams& p, const u32* cid, const u64* cf, const u32* cr,
                                         u32 nc, const ThrCache& thr, u32 nthreads) {
    if (nc == 0) return;
    if (p.exhaustive) {
        for (u32 i = threadIdx.x; i < nc; i += nthreads) {
            p.out_far[cid[i]] = cf[i];
            p.out_reach[cid[i]] = cr[i];
        }
        return;
    }
    if (threadIdx.x != 0) return;
    bool any = false;
    for (u32 i = 0; i < nc && !any; ++i) {
        if (!thr.valid) { any = true; break; }
        u64 N, F;
        score_key(cf[i], cr[i], N, F);
        any = ranks_before(N, F, cid[i], thr.N, thr.F, thr.id);
    }
    if (!any) return;
    if (!lock_acquire(p.topk.lock, p.lock_limit_ns, p.err)) return;
    for (u32 i = 0; i < nc; ++i) topk_insert_locked(p.topk, cid[i], cf[i], cr[i]);
    topk_publish_locked(p.topk);
    lock_release(p.topk.lock);
}

// --------------------------------------------------------- per-CTA waves
template <int W, int THREADS>
__global__ void __launch_bounds__(THREADS) k_wave_cta(WaveParams p) {
    constexpr int L = 64 * W;
    constexpr int NWARP = THREADS / 32;
    static_assert(THREADS >= L, "one thread per lane");
    __shared__ u32 s_src[L], s_nd[L], s_gt[L], s_xlo[L], s_xhi[L];
    __shared__ u64 s_f[L];
    __shared__ u32 s_cg[L], s_cs[L];
    __shared__ u32 s_alive32[2 * W];
    __shared__ u32 s_ln[2], s_logn, s_base, s_nc, s_stop;
    __shared__ ThrCache s_thr;
    __shared__ u32 s_cid[L], s_cr[L];
    __shared__ u64 s_cf[L];

    const u32 tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const GraphDev& G = p.g;
    SlotPtrs S = slot_ptrs(p.slot_base + (size_t)blockIdx.x * p.slot_stride, G.n, W);
    LocalStats st;
    if (tid == 0) {
        s_thr.valid = 0; s_thr.N = 0; s_thr.F = 1; s_thr.id = 0;
        s_nc = 0; s_logn = 0; s_ln[0] = 0; s_ln[1] = 0;
    }
    __syncthreads();

    for (;;) {
        if (tid == 0) {
            s_base = atomicAdd(p.head, (u32)L);
            s_stop = (s_base >= p.n_end) || (vload(p.err) != 0);
        }
        __syncthreads();
        if (s_stop) break;
        const u32 base = s_base;
        if (tid == 0) st.waves++;
        if (tid < L) {
            bool alive = false;
            s_cg[tid] = 0;
            s_cs[tid] = 0;
            if (base + tid < p.n_end) {
                u32 v = __ldg(&G.order[base + tid]);
                u32 deg = __ldg(&G.rp[v + 1]) - __ldg(&G.rp[v]);
                s_src[tid] = v; s_nd[tid] = 1; s_f[tid] = 0; s_gt[tid] = deg;
                s_xlo[tid] = __ldg(&G.xlo[v]); s_xhi[tid] = __ldg(&G.xhi[v]);
                if (deg == 0) {          // R(v) = {v}: r = 1, f = 0
                    u32 c = atomicAdd(&s_nc, 1u);
                    s_cid[c] = v; s_cf[c] = 0; s_cr[c] = 1;
                    st.completed++;
                } else {
                    alive = true;
                }
            }
            u32 m = __ballot_sync(0xffffffffu, alive);
            if (lane == 0) s_alive32[tid >> 5] = m;
        }
        __syncthreads();
        flush_completions(p, s_cid, s_cf, s_cr, s_nc, s_thr, THREADS);
        __syncthreads();
        if (tid == 0) s_nc = 0;

        u32 d = 0, cur = 0;
        for (;;) {
            if (!p.exhaustive && tid == 0) read_threshold(p.topk.thr, s_thr);
            __syncthreads();
            if (tid < L) {   // stopping rule at level d, before Gamma_d is expanded
                bool a = (s_alive32[tid >> 5] >> lane) & 1u;
                if (a && !p.exhaustive &&
                    bfscut_stops(s_f[tid], s_gt[tid], d, s_nd[tid], s_xlo[tid], s_xhi[tid], s_src[tid], s_thr)) {
                    a = false;
                    st.cut++;
                }
                u32 m = __ballot_sync(0xffffffffu, a);
                if (lane == 0) s_alive32[tid >> 5] = m;
            }
            __syncthreads();
            u32 any = 0;
#pragma unroll
            for (int i = 0; i < 2 * W; ++i) any |= s_alive32[i];
            if (!any) break;

            u64* Fnext = S.F[cur ^ 1];
            if (d == 0)
                expand_sources<W>(G, s_src, s_alive32, L, S.vis, Fnext, s_cg, s_cs, p.footnote,
                                  S.list[cur ^ 1], &s_ln[cur ^ 1], S.clog, &s_logn, wid, NWARP, st);
            else
                expand_entries<W>(G, S.list[cur], s_ln[cur], S.F[cur], s_alive32, S.vis, Fnext, s_cg, s_cs,
                                  p.footnote, S.list[cur ^ 1], &s_ln[cur ^ 1], S.clog, &s_logn, wid, NWARP, st);
            __syncthreads();
            if (tid < L) {   // level d+1 is known: gamma_{d+1} and its degree sum
                bool a = (s_alive32[tid >> 5] >> lane) & 1u;
                if (a) {
                    u32 gam = s_cg[tid];
                    if (gam == 0) {
                        u32 c = atomicAdd(&s_nc, 1u);
                        s_cid[c] = s_src[tid]; s_cf[c] = s_f[tid]; s_cr[c] = s_nd[tid];
                        a = false;
                        st.completed++;
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
            if (tid == 0) s_ln[cur] = 0;
            __syncthreads();
            flush_completions(p, s_cid, s_cf, s_cr, s_nc, s_thr, THREADS);
            __syncthreads();
            if (tid == 0) s_nc = 0;
            cur ^= 1;
            ++d;
        }
        if (tid == 0) {
            st.levels += d;
            if (d > st.maxlevel) st.maxlevel = d;
        }
        // the wave's footprint: every word whose vis became non-zero
        const u32 nlog = s_logn;
        for (u32 i = tid; i < nlog; i += THREADS) {
            u32 w = S.clog[i];
            S.vis[w] = 0;
            S.F[0][w] = 0;
            S.F[1][w] = 0;
        }
        if (tid == 0) st.cleared += nlog;
        __syncthreads();
        if (tid == 0) { s_logn = 0; s_ln[0] = 0; s_ln[1] = 0; }
    }
    flush_stats(st, p.stats);
}

// ------------------------------------------------------------ grid waves
// The whole grid runs waves one after another, taking 64*W sources at
// order[*head] each time.  Each block keeps an identical copy of the lane
// state; per-level counters are summed in global memory between two grid
// barriers; block 0 owns the top-k.  After each wave the grid decides, from
// values every block read after the same barriers, whether the wave was
// heavy (its frontiers held more than p.heavy_words words in total).  On
// the first light wave the kernel returns and leaves *head where the
// per-CTA kernel continues; exhaustive runs (or max_grid_waves reached) end it
// too.
template <int W, int THREADS>
__global__ void __launch_bounds__(THREADS) k_wave_grid(WaveParams p) {
    constexpr int L = 64 * W;
    constexpr int NWARP = THREADS / 32;
    static_assert(THREADS >= L, "one thread per lane");
    __shared__ u32 s_src[L], s_nd[L], s_gt[L], s_xlo[L], s_xhi[L];
    __shared__ u64 s_f[L];
    __shared__ u32 s_cg[L], s_cs[L];
    __shared__ u32 s_alive32[2 * W];
    __shared__ u32 s_nc, s_base;
    __shared__ ThrCache s_thr;
    __shared__ u32 s_cid[L], s_cr[L];
    __shared__ u64 s_cf[L];

    const u32 tid = threadIdx.x, lane = tid & 31, wid = tid >> 5;
    const bool leader = blockIdx.x == 0;
    const GraphDev& G = p.g;
    // arrays placed at their 4-word offsets whatever W is, so runs of
    // different widths never put bit arrays where another left lists or logs
    SlotPtrs S = slot_ptrs(p.seed_base, G.n, 4);
    LocalStats st;
    const u32 gw = blockIdx.x * NWARP + wid, gnw = gridDim.x * NWARP;
    if (tid == 0) { s_nc = 0; s_thr.valid = 0; s_thr.N = 0; s_thr.F = 1; s_thr.id = 0; }
    bool ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err);

    for (u32 wave = 0; ok && wave < p.max_grid_waves; ++wave) {
        if (tid == 0) s_base = vload(p.head);
        __syncthreads();
        const u32 base = s_base;
        if (base >= p.n_end) break;
        if (tid < L) {
            bool alive = false;
            s_cg[tid] = 0;
            s_cs[tid] = 0;
            if (base + tid < p.n_end) {
                u32 v = __ldg(&G.order[base + tid]);
                u32 deg = __ldg(&G.rp[v + 1]) - __ldg(&G.rp[v]);
                s_src[tid] = v; s_nd[tid] = 1; s_f[tid] = 0; s_gt[tid] = deg;
                s_xlo[tid] = __ldg(&G.xlo[v]); s_xhi[tid] = __ldg(&G.xhi[v]);
                if (deg == 0) {
                    if (leader) {
                        u32 c = atomicAdd(&s_nc, 1u);
                        s_cid[c] = v; s_cf[c] = 0; s_cr[c] = 1;
                        st.completed++;
                    }
                } else {
                    alive = true;
                }
            }
            u32 m = __ballot_sync(0xffffffffu, alive);
            if (lane == 0) s_alive32[tid >> 5] = m;
        }
        __syncthreads();
        if (leader) flush_completions(p, s_cid, s_cf, s_cr, s_nc, s_thr, THREADS);
        __syncthreads();
        if (tid == 0) s_nc = 0;
        if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;

        u32 d = 0, cur = 0;
        u64 wave_entries = 0;
        for (;;) {
            if (!p.exhaustive && tid == 0) read_threshold(p.topk.thr, s_thr);
            __syncthreads();
            if (tid < L) {
                bool a = (s_alive32[tid >> 5] >> lane) & 1u;
                if (a && !p.exhaustive &&
                    bfscut_stops(s_f[tid], s_gt[tid], d, s_nd[tid], s_xlo[tid], s_xhi[tid], s_src[tid], s_thr)) {
                    a = false;
                    if (leader) st.cut++;
                }
                u32 m = __ballot_sync(0xffffffffu, a);
                if (lane == 0) s_alive32[tid >> 5] = m;
            }
            __syncthreads();
            u32 any = 0;
#pragma unroll
            for (int i = 0; i < 2 * W; ++i) any |= s_alive32[i];
            if (!any) break;

            const u32 par = d & 1;
            u32* gcg = p.gcnt + par * 512;
            u32* gcs = gcg + 256;
            if (d == 0) {
                expand_sources<W>(G, s_src, s_alive32, L, S.vis, S.F[cur ^ 1], s_cg, s_cs, p.footnote,
                                  S.list[cur ^ 1], &p.glist_n[cur ^ 1], S.clog, p.glog_n, gw, gnw, st);
            } else {
                const u32 cnt = vload(&p.glist_n[cur]);
                wave_entries += cnt;
                expand_entries<W>(G, S.list[cur], cnt, S.F[cur], s_alive32, S.vis, S.F[cur ^ 1], s_cg, s_cs,
                                  p.footnote, S.list[cur ^ 1], &p.glist_n[cur ^ 1], S.clog, p.glog_n, gw, gnw, st);
            }
            __syncthreads();
            if (tid < L) {
                if (s_cg[tid]) { atomicAdd(&gcg[tid], s_cg[tid]); atomicAdd(&gcs[tid], s_cs[tid]); }
                s_cg[tid] = 0;
                s_cs[tid] = 0;
            }
            if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
            if (tid < L) {
                bool a = (s_alive32[tid >> 5] >> lane) & 1u;
                if (a) {
                    u32 gam = vload(&gcg[tid]);
                    if (gam == 0) {
                        if (leader) {
                            u32 c = atomicAdd(&s_nc, 1u);
                            s_cid[c] = s_src[tid]; s_cf[c] = s_f[tid]; s_cr[c] = s_nd[tid];
                            st.completed++;
                        }
                        a = false;
                    } else {
                        s_nd[tid] += gam;
                        s_f[tid] += (u64)(d + 1) * gam;
                        s_gt[tid] = vload(&gcs[tid]);
                    }
                }
                u32 m = __ballot_sync(0xffffffffu, a);
                if (lane == 0) s_alive32[tid >> 5] = m;
            }
            if (leader) {   // buffers of the next level: counters par^1, list count cur
                u32* nx = p.gcnt + (par ^ 1) * 512;
                for (u32 i = tid; i < 512; i += THREADS) nx[i] = 0;
                if (tid == 0) p.glist_n[cur] = 0;
            }
            __syncthreads();
            if (leader) flush_completions(p, s_cid, s_cf, s_cr, s_nc, s_thr, THREADS);
            __syncthreads();
            if (tid == 0) s_nc = 0;
            if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
            cur ^= 1;
            ++d;
        }
        if (!ok) break;
        if (leader && tid == 0) {
            st.waves++;
            st.levels += d;
            if (d > st.maxlevel) st.maxlevel = d;
        }
        // clear the wave's footprint: every block has finished expanding
        // (the level loop ends at a barrier or on a decision all blocks share)
        if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
        const u32 nlog = vload(p.glog_n);
        for (u32 i = blockIdx.x * THREADS + tid; i < nlog; i += gridDim.x * THREADS) {
            u32 w = __ldcg(&S.clog[i]);
            S.vis[w] = 0;
            S.F[0][w] = 0;
            S.F[1][w] = 0;
        }
        if (leader && tid == 0) st.cleared += nlog;
        if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
        if (leader) {   // reset per-wave counters and advance the queue
            for (u32 i = tid; i < 1024; i += THREADS) p.gcnt[i] = 0;
            if (tid == 0) {
                p.glist_n[0] = 0;
                p.glist_n[1] = 0;
                *p.glog_n = 0;
                *p.head = base + L;
            }
        }
        if (!(ok = grid_sync(p.bar, gridDim.x, p.barrier_limit_ns, p.err))) break;
        if (!p.exhaustive && wave_entries < p.heavy_words) break;   // light: hand over to the CTAs
    }
    flush_stats(st, p.stats);
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
        read_threshold(p.topk.thr, s_thr);   // fixed for this launch: only its end inserts
    }
    __syncthreads();
    const u32 xlo = __ldg(&G.xlo[v]), xhi = __ldg(&G.xhi[v]);
    u32 d = 0, cur = 0, nd = 1;
    u64 f = 0;
    u32 gt = __ldg(&G.rp[v + 1]) - __ldg(&G.rp[v]);
    bool done = false, cut = false, ok = true;
    const u32 gw = blockIdx.x * NWARP + wid, gnw = gridDim.x * NWARP;
    while (ok) {
        if (bfscut_stops(f, gt, d, nd, xlo, xhi, v, s_thr)) { cut = true; break; }
        const u32 par = d & 1;
        u32* gcg = p.gcnt + par * 512;
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
            u32* nx = p.gcnt + (par ^ 1) * 512;
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
        p.gcnt[0] = 0; p.gcnt[256] = 0; p.gcnt[512] = 0; p.gcnt[768] = 0;
        p.glist_n[0] = 0; p.glist_n[1] = 0;
        st.levels = d;
        st.maxlevel = d;
        st.waves = 1;
        if (cut) st.cut = 1;
        if (done && ok) {
            st.completed = 1;
            if (lock_acquire(p.topk.lock, p.lock_limit_ns, p.err)) {
                topk_insert_locked(p.topk, v, f, nd);
                topk_publish_locked(p.topk);
                lock_release(p.topk.lock);
            }
        }
    }
    (void)s_go;
    flush_stats(st, p.stats);
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
