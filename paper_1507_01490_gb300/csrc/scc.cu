// Strongly connected components, the weighted SCC DAG (Section 1.3) and the
// alpha/omega bounds on r(v) (Section 2.3) for directed graphs.
//
// SCCs:  (1) trimming: a vertex with no remaining in- or out-neighbour is an
//        SCC by itself; (2) forward and backward reachability from a pivot of
//        large in*out degree: their intersection is the pivot's SCC (this
//        takes the giant SCC of a power-law digraph in one step); (3) for
//        what is left, max-label colouring: every vertex takes the largest id
//        that reaches it, then a backward search from each vertex that kept
//        its own id, restricted to its colour, collects that vertex's SCC.
// DAG:   arcs (C(u), C(w)) with C(u) != C(w), sorted and made unique.
// Bounds: sinks first (Kahn on the reversed DAG); a component is evaluated
//        once all its successors are, with
//           alpha(C) = w(C) + max over arcs (C,D) of alpha(D)
//           omega(C) = min(n, w(C) + sum over arcs (C,D) of omega(D)).
#include <cstdio>
#include <cuda_runtime.h>

#include "internal.h"

namespace bcm {

static constexpr uint32_t UNSET = 0xffffffffu;
// a reachability level is pulled once its frontier holds n / kReachPullDiv vertices
#ifndef BCM_REACH_PULL_DIV
#define BCM_REACH_PULL_DIV 64
#endif
static constexpr uint32_t kReachPullDiv = BCM_REACH_PULL_DIV;
static inline bool reach_pull(uint32_t fsize, uint32_t n) { return kReachPullDiv && fsize >= n / kReachPullDiv; }

static inline unsigned grid_for(size_t work, int threads = 256) {
    size_t b = (work + threads - 1) / threads;
    if (b < 1) b = 1;
    if (b > 152 * 32) b = 152 * 32;
    return (unsigned)b;
}

#define GRID_STRIDE(i, n) \
    for (size_t i = blockIdx.x * (size_t)blockDim.x + threadIdx.x; i < (n); i += (size_t)gridDim.x * blockDim.x)

#define WARP_PER_ITEM(u, n)                                                      \
    const uint32_t lane_ = threadIdx.x & 31;                                     \
    for (size_t u = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5; u < (n); \
         u += ((size_t)gridDim.x * blockDim.x) >> 5)

// Items of a frontier (vertices, or SCCs of the DAG) with more than
// kHeavyEdges arcs: each is taken by the whole grid in a second kernel
// instead of one warp.  A full list leaves the item with its warp.
constexpr uint32_t kHeavyEdges = 2048;
constexpr uint32_t kSccHeavyCap = 256;
struct SccHeavy {
    uint32_t n;
    uint32_t pad;
    uint32_t item[kSccHeavyCap];
    unsigned long long acc[kSccHeavyCap][3];   // k_dp_eval_heavy: max alpha, sum omega, sum Wm
};

__device__ __forceinline__ bool heavy_claim(SccHeavy* H, uint32_t c, uint32_t deg) {
    if (deg <= kHeavyEdges) return false;
    uint32_t slot = 0;
    if ((threadIdx.x & 31) == 0) slot = atomicAdd(&H->n, 1u);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= kSccHeavyCap) return false;
    if ((threadIdx.x & 31) == 0) H->item[slot] = c;
    return true;
}

// Rows (a vertex's out-arcs) longer than kHeavyEdges, for the per-arc
// passes below: one warp per row would hold an R-MAT hub's tens of
// thousands of arcs, so such rows go to a list whose arcs the whole grid
// shares in a second kernel.  A full list leaves the row with its warp.
constexpr uint32_t kRowHeavyCap = 4096;
struct RowHeavy {
    uint32_t n;
    uint32_t item[kRowHeavyCap];
};

__device__ __forceinline__ bool row_claim(RowHeavy* H, uint32_t u, uint32_t deg) {
    if (!H || deg <= kHeavyEdges) return false;
    uint32_t slot = 0;
    if ((threadIdx.x & 31) == 0) slot = atomicAdd(&H->n, 1u);
    slot = __shfl_sync(0xffffffffu, slot, 0);
    if (slot >= kRowHeavyCap) return false;
    if ((threadIdx.x & 31) == 0) H->item[slot] = u;
    return true;
}

// The heavy rows' arcs over the whole grid: f(u, e) for each arc e of row u.
#define ROW_HEAVY_LOOP(H, rp, u, e)                                                           \
    const uint32_t hn_ = (H)->n < kRowHeavyCap ? (H)->n : kRowHeavyCap;                      \
    for (uint32_t h_ = 0; h_ < hn_; ++h_)                                                    \
        for (uint32_t u = (H)->item[h_], e = (rp)[u] + blockIdx.x * blockDim.x + threadIdx.x; \
             e < (rp)[u + 1]; e += gridDim.x * blockDim.x)

__global__ void k_count_in(const uint32_t* rp, const uint32_t* col, uint32_t n, uint32_t* indeg, RowHeavy* H) {
    WARP_PER_ITEM(u, n) {
        if (row_claim(H, (uint32_t)u, rp[u + 1] - rp[u])) continue;
        for (uint32_t e = rp[u] + lane_; e < rp[u + 1]; e += 32) atomicAdd(&indeg[col[e]], 1u);
    }
}

__global__ void k_count_in_heavy(const uint32_t* rp, const uint32_t* col, uint32_t* indeg, const RowHeavy* H) {
    ROW_HEAVY_LOOP(H, rp, u, e) atomicAdd(&indeg[col[e]], 1u);
}

__global__ void k_fill_rev(const uint32_t* rp, const uint32_t* col, uint32_t n, uint32_t* cursor, uint32_t* rcol,
                           RowHeavy* H) {
    WARP_PER_ITEM(u, n) {
        if (row_claim(H, (uint32_t)u, rp[u + 1] - rp[u])) continue;
        for (uint32_t e = rp[u] + lane_; e < rp[u + 1]; e += 32) rcol[atomicAdd(&cursor[col[e]], 1u)] = (uint32_t)u;
    }
}

__global__ void k_fill_rev_heavy(const uint32_t* rp, const uint32_t* col, uint32_t* cursor, uint32_t* rcol,
                                 const RowHeavy* H) {
    ROW_HEAVY_LOOP(H, rp, u, e) rcol[atomicAdd(&cursor[col[e]], 1u)] = u;
}

__global__ void k_set_last(uint32_t* a, uint32_t idx, uint32_t v) { a[idx] = v; }

__global__ void k_fill(uint32_t* a, size_t n, uint32_t v) {
    GRID_STRIDE(i, n) a[i] = v;
}

// (1) trimming
__global__ void k_trim(const uint32_t* rp, const uint32_t* col, const uint32_t* rrp, const uint32_t* rcol,
                       uint32_t n, uint32_t* scc, uint32_t* changed) {
    GRID_STRIDE(v, n) {
        if (vload(&scc[v]) != UNSET) continue;
        bool out = false, in = false;
        for (uint32_t e = rp[v]; e < rp[v + 1] && !out; ++e) {
            uint32_t w = col[e];
            out = (w != v) && vload(&scc[w]) == UNSET;
        }
        if (out)
            for (uint32_t e = rrp[v]; e < rrp[v + 1] && !in; ++e) {
                uint32_t w = rcol[e];
                in = (w != v) && vload(&scc[w]) == UNSET;
            }
        if (!out || !in) {
            scc[v] = (uint32_t)v;
            *changed = 1;
        }
    }
}

__global__ void k_pivot(const uint32_t* rp, const uint32_t* rrp, uint32_t n, const uint32_t* scc,
                        unsigned long long* best) {
    // each thread's best, then the warp's: one atomic per warp on the one word
    unsigned long long b = 0;
    GRID_STRIDE(v, n) {
        if (scc[v] != UNSET) continue;
        unsigned long long p = (unsigned long long)(rp[v + 1] - rp[v]) * (rrp[v + 1] - rrp[v]);
        if (p > 0xffffffffull) p = 0xffffffffull;
        const unsigned long long key = (p << 32) | (0xffffffffull - v);
        b = key > b ? key : b;
    }
    for (int o = 16; o; o >>= 1) {
        const unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = t > b ? t : b;
    }
    if ((threadIdx.x & 31) == 0 && b) atomicMax(best, b);
}

__global__ void k_seed_mark(uint32_t v, uint32_t* mark, uint32_t* list, uint32_t* cnt) {
    mark[v] = 1;
    list[0] = v;
    *cnt = 1;
}

// one BFS level over unassigned vertices; same_color restricts to color[w] == color[u]
__device__ __forceinline__ void reach_arc(const uint32_t* col, uint32_t e, bool valid, uint32_t cu, uint32_t* next,
                                          uint32_t* ncnt, uint32_t* mark, const uint32_t* scc, const uint32_t* color,
                                          int same_color) {
    bool app = false;
    uint32_t w = 0;
    if (valid) {
        w = col[e];
        if (scc[w] == UNSET && (!same_color || color[w] == cu) && vload(&mark[w]) == 0 &&
            atomicExch(&mark[w], 1u) == 0)
            app = true;
    }
    warp_append(app, w, next, ncnt);
}

__global__ void k_reach(const uint32_t* rp, const uint32_t* col, const uint32_t* front, const uint32_t* fcnt,
                        uint32_t* next, uint32_t* ncnt, uint32_t* mark, const uint32_t* scc, const uint32_t* color,
                        int same_color, SccHeavy* H) {
    const uint32_t cnt = *fcnt;
    WARP_PER_ITEM(i, cnt) {
        uint32_t u = front[i];
        if (H && heavy_claim(H, u, rp[u + 1] - rp[u])) continue;
        uint32_t cu = same_color ? color[u] : 0;
        for (uint32_t e0 = rp[u]; e0 < rp[u + 1]; e0 += 32)
            reach_arc(col, e0 + lane_, e0 + lane_ < rp[u + 1], cu, next, ncnt, mark, scc, color, same_color);
    }
}

__global__ void k_reach_heavy(const uint32_t* rp, const uint32_t* col, uint32_t* next, uint32_t* ncnt,
                              uint32_t* mark, const uint32_t* scc, const uint32_t* color, int same_color,
                              const SccHeavy* H) {
    const uint32_t hn = H->n < kSccHeavyCap ? H->n : kSccHeavyCap;
    for (uint32_t h = 0; h < hn; ++h) {
        const uint32_t u = H->item[h], b = rp[u], e = rp[u + 1];
        const uint32_t cu = same_color ? color[u] : 0;
        WARP_PER_ITEM(j, ((size_t)(e - b) + 31) / 32) {
            const size_t a = b + j * 32 + lane_;
            reach_arc(col, (uint32_t)a, a < e, cu, next, ncnt, mark, scc, color, same_color);
        }
    }
}

// The same level by pull (direction-optimising BFS): every unassigned,
// unmarked vertex v looks through its arcs of the other direction for a
// marked unassigned vertex (of its colour) and stops at the first.  For
// the reachable set a marked vertex of any earlier level serves as well as
// one of the last, so marks need no level; each v is marked by its own
// thread only.  Used when the frontier is a large part of the graph.
__global__ void k_reach_pull(const uint32_t* rp, const uint32_t* col, uint32_t n, uint32_t* next, uint32_t* ncnt,
                             uint32_t* mark, const uint32_t* scc, const uint32_t* color, int same_color) {
    const uint32_t lane = threadIdx.x & 31;
    for (size_t v0 = blockIdx.x * (size_t)blockDim.x + (threadIdx.x & ~31u); v0 < n;
         v0 += (size_t)gridDim.x * blockDim.x) {
        const size_t v = v0 + lane;
        bool app = false;
        if (v < n && scc[v] == UNSET && vload(&mark[v]) == 0) {
            const uint32_t cv = same_color ? color[v] : 0u;
            const uint32_t end = rp[v + 1];
            for (uint32_t e = rp[v]; e < end; ++e) {
                const uint32_t u = col[e];
                if (vload(&mark[u]) != 0 && scc[u] == UNSET && (!same_color || color[u] == cv)) {
                    app = true;
                    break;
                }
            }
            if (app) vstore(&mark[v], 1u);
        }
        warp_append(app, (uint32_t)v, next, ncnt);
    }
}

__global__ void k_assign_both(uint32_t n, const uint32_t* fw, const uint32_t* bw, uint32_t* scc, uint32_t rep) {
    GRID_STRIDE(v, n) if (scc[v] == UNSET && fw[v] && bw[v]) scc[v] = rep;
}

// (3) colouring
__global__ void k_color_init(uint32_t n, const uint32_t* scc, uint32_t* color) {
    GRID_STRIDE(v, n) color[v] = (scc[v] == UNSET) ? (uint32_t)v : 0u;
}

__global__ void k_color_prop(const uint32_t* rp, const uint32_t* col, uint32_t n, const uint32_t* scc, uint32_t* color,
                             uint32_t* changed) {
    WARP_PER_ITEM(u, n) {
        if (scc[u] != UNSET) continue;
        uint32_t c = vload(&color[u]);
        for (uint32_t e = rp[u] + lane_; e < rp[u + 1]; e += 32) {
            uint32_t w = col[e];
            if (scc[w] == UNSET && vload(&color[w]) < c) {
                atomicMax(&color[w], c);
                *changed = 1;
            }
        }
    }
}

__global__ void k_color_roots(uint32_t n, const uint32_t* scc, const uint32_t* color, uint32_t* mark, uint32_t* list,
                              uint32_t* cnt) {
    const uint32_t lane = threadIdx.x & 31;
    for (size_t b = (blockIdx.x * (size_t)blockDim.x) + (threadIdx.x & ~31u); b < n;
         b += (size_t)gridDim.x * blockDim.x) {
        size_t v = b + lane;
        bool root = v < n && scc[v] == UNSET && color[v] == (uint32_t)v;
        if (root) mark[v] = 1;
        warp_append(root, (uint32_t)v, list, cnt);
    }
}

__global__ void k_assign_marked(uint32_t n, uint32_t* scc, const uint32_t* color, const uint32_t* mark,
                                uint32_t* remaining) {
    GRID_STRIDE(v, n) {
        if (scc[v] != UNSET) continue;
        if (mark[v]) scc[v] = color[v];
        else atomicAdd(remaining, 1u);
    }
}

__global__ void k_count_unset(uint32_t n, const uint32_t* scc, uint32_t* cnt) {
    uint32_t c = 0;
    GRID_STRIDE(v, n) c += scc[v] == UNSET;
    for (int o = 16; o; o >>= 1) c += __shfl_xor_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(cnt, c);
}

// labels ordered by smallest member
// The smallest member of every SCC; lanes of one SCC (most of them, in a
// graph with a giant SCC) take their minimum first, then one atomic.
__global__ void k_minrep(uint32_t n, const uint32_t* scc, uint32_t* minv) {
    const uint32_t lane = threadIdx.x & 31;
    for (size_t v0 = blockIdx.x * (size_t)blockDim.x + (threadIdx.x & ~31u); v0 < n;
         v0 += (size_t)gridDim.x * blockDim.x) {
        const size_t v = v0 + lane;
        const uint32_t c = v < n ? scc[v] : UNSET;
        const uint32_t peers = __match_any_sync(0xffffffffu, c);
        const uint32_t m = __reduce_min_sync(peers, v < n ? (uint32_t)v : UNSET);
        if (c != UNSET && lane == (uint32_t)(__ffs(peers) - 1)) atomicMin(&minv[c], m);
    }
}

__global__ void k_min_flags(uint32_t n, const uint32_t* scc, const uint32_t* minv, uint32_t* flags) {
    GRID_STRIDE(v, n) flags[v] = minv[scc[v]] == (uint32_t)v ? 1u : 0u;
}

__global__ void k_label(uint32_t n, const uint32_t* scc, const uint32_t* minv, const uint32_t* rank, uint32_t* comp) {
    GRID_STRIDE(v, n) comp[v] = rank[minv[scc[v]]];
}

// DAG
// The key (comp[u] << b | comp[w]) of an arc between two SCCs, appended to
// keys (in no particular order: they are sorted next); arcs inside an SCC,
// most of a graph with a giant SCC, are left out of the sort.  Each warp
// stages its keys in shared memory and reserves room in keys once per
// kKeyStage of them, not once per 32 arcs (the count is one word that
// every warp of the grid would otherwise hit).
constexpr uint32_t kKeyStage = 256;
struct KeyStage {
    unsigned long long* buf;   // this warp's kKeyStage shared entries
    unsigned long long* dst;
    uint32_t* cnt;
    uint32_t n;                // staged (the same in every lane)
    __device__ __forceinline__ void flush() {
        __syncwarp();
        uint32_t base = 0;
        if ((threadIdx.x & 31) == 0 && n) base = atomicAdd(cnt, n);
        base = __shfl_sync(0xffffffffu, base, 0);
        for (uint32_t i = threadIdx.x & 31; i < n; i += 32) dst[base + i] = buf[i];
        __syncwarp();
        n = 0;
    }
    __device__ __forceinline__ void push(bool want, unsigned long long key) {
        const uint32_t m = __ballot_sync(0xffffffffu, want);
        if (want) buf[n + __popc(m & ((1u << (threadIdx.x & 31)) - 1u))] = key;
        n += __popc(m);
        if (n + 32 > kKeyStage) flush();
    }
};

__device__ __forceinline__ void dag_key(const uint32_t* col, const uint32_t* comp, uint32_t cu, int b, uint32_t e,
                                        bool valid, KeyStage& ks) {
    unsigned long long key = 0;
    bool inter = false;
    if (valid) {
        const uint32_t cw = comp[col[e]];
        inter = cu != cw;
        key = ((unsigned long long)cu << b) | cw;
    }
    ks.push(inter, key);
}

// launched with 256 threads: 8 warps' stages
__global__ void k_dag_keys(const uint32_t* rp, const uint32_t* col, uint32_t n, const uint32_t* comp, int b,
                           unsigned long long* keys, uint32_t* kcnt, RowHeavy* H) {
    __shared__ unsigned long long s_stage[8 * kKeyStage];
    KeyStage ks{&s_stage[(threadIdx.x >> 5) * kKeyStage], keys, kcnt, 0};
    WARP_PER_ITEM(u, n) {
        if (row_claim(H, (uint32_t)u, rp[u + 1] - rp[u])) continue;
        const uint32_t cu = comp[u], end = rp[u + 1];
        for (uint32_t e0 = rp[u]; e0 < end; e0 += 32) dag_key(col, comp, cu, b, e0 + lane_, e0 + lane_ < end, ks);
    }
    ks.flush();
}

// the rows row_claim listed, 32 arcs per warp at a time over the whole grid
__global__ void k_dag_keys_heavy(const uint32_t* rp, const uint32_t* col, const uint32_t* comp, int b,
                                 unsigned long long* keys, uint32_t* kcnt, const RowHeavy* H) {
    __shared__ unsigned long long s_stage[8 * kKeyStage];
    KeyStage ks{&s_stage[(threadIdx.x >> 5) * kKeyStage], keys, kcnt, 0};
    const uint32_t hn = H->n < kRowHeavyCap ? H->n : kRowHeavyCap;
    const uint32_t lane = threadIdx.x & 31;
    const size_t warp = (blockIdx.x * (size_t)blockDim.x + threadIdx.x) >> 5;
    const size_t nwarps = ((size_t)gridDim.x * blockDim.x) >> 5;
    for (uint32_t h = 0; h < hn; ++h) {
        const uint32_t u = H->item[h], beg = rp[u], end = rp[u + 1], cu = comp[u];
        for (size_t e0 = beg + warp * 32; e0 < end; e0 += nwarps * 32)
            dag_key(col, comp, cu, b, (uint32_t)(e0 + lane), e0 + lane < end, ks);
    }
    ks.flush();
}

__global__ void k_unique_flags(const unsigned long long* keys, uint64_t m, uint32_t* flags) {
    GRID_STRIDE(i, m) {
        unsigned long long k = keys[i];
        flags[i] = (k != ~0ull && (i == 0 || keys[i - 1] != k)) ? 1u : 0u;
    }
}

__global__ void k_unique_scatter(const unsigned long long* keys, uint64_t m, const uint32_t* flags,
                                 const uint32_t* pos, int b, uint32_t* dsrc, uint32_t* ddst) {
    GRID_STRIDE(i, m) {
        if (!flags[i]) continue;
        unsigned long long k = keys[i];
        dsrc[pos[i]] = (uint32_t)(k >> b);
        ddst[pos[i]] = (uint32_t)(k & ((1ull << b) - 1));
    }
}

// Counts of each value; lanes holding the same value (a giant SCC's label,
// runs of a sorted array) add their count with one atomic.
__global__ void k_hist(const uint32_t* a, size_t cnt, uint32_t* h) {
    const uint32_t lane = threadIdx.x & 31;
    for (size_t i0 = blockIdx.x * (size_t)blockDim.x + (threadIdx.x & ~31u); i0 < cnt;
         i0 += (size_t)gridDim.x * blockDim.x) {
        const size_t i = i0 + lane;
        const uint32_t x = i < cnt ? a[i] : UNSET;
        const uint32_t peers = __match_any_sync(0xffffffffu, x);
        if (i < cnt && lane == (uint32_t)(__ffs(peers) - 1)) atomicAdd(&h[x], (uint32_t)__popc(peers));
    }
}

__global__ void k_scatter_pred(const uint32_t* dsrc, const uint32_t* ddst, uint32_t nd, uint32_t* cursor,
                               uint32_t* pred) {
    GRID_STRIDE(i, nd) pred[atomicAdd(&cursor[ddst[i]], 1u)] = dsrc[i];
}

__global__ void k_sinks(uint32_t nc, const uint32_t* drp, uint32_t* outcnt, uint32_t* list, uint32_t* cnt) {
    const uint32_t lane = threadIdx.x & 31;
    for (size_t b = (blockIdx.x * (size_t)blockDim.x) + (threadIdx.x & ~31u); b < nc;
         b += (size_t)gridDim.x * blockDim.x) {
        size_t c = b + lane;
        bool sink = false;
        if (c < nc) {
            uint32_t d = drp[c + 1] - drp[c];
            outcnt[c] = d;
            sink = d == 0;
        }
        warp_append(sink, (uint32_t)c, list, cnt);
    }
}

// Section 2.3 for the SCCs of one topological level (all successors done).
// With the biggest-SCC refinement (big != ~0): big itself gets alpha =
// omega = R; for an SCC outside big's descendants, Wm is the programme on
// the DAG without them, and SCCs reaching big keep min(omega, Wm + R).
struct Refine {
    uint32_t big;              // largest SCC, or 0xffffffff for the plain programme
    const uint32_t* R;         // its reach
    const uint32_t* desc;      // 1: reachable from big (big included)
    const uint32_t* anc;       // 1: reaches big
    uint32_t* Wm;
};

// The programme's value of SCC c from its successors' max alpha and sums.
__device__ void dp_finish(uint32_t c, uint32_t amax, unsigned long long osum, unsigned long long msum,
                          const uint32_t* wsz, uint32_t* A, uint32_t* Om, uint32_t n, const Refine& rf) {
    const bool refine = rf.big != 0xffffffffu;
    if (refine && c == rf.big) {
        A[c] = *rf.R;
        Om[c] = *rf.R;
        rf.Wm[c] = 0;
        return;
    }
    A[c] = wsz[c] + amax;
    unsigned long long o = wsz[c] + (osum > n ? n : osum);
    o = o > n ? n : o;
    if (refine) {
        unsigned long long wm = rf.desc[c] ? 0 : wsz[c] + (msum > n ? n : msum);
        wm = wm > n ? n : wm;
        rf.Wm[c] = (uint32_t)wm;
        if (rf.anc[c] && wm + *rf.R < o) o = wm + *rf.R;
    }
    Om[c] = (uint32_t)o;
}

// One warp per SCC of the level: lanes take its successors 32 at a time
// and the warp reduces max alpha and the sums (exact in 64 bits: at most
// 2^32 terms below 2^30; held at n at the end, as the programme's running
// minimum with n gives the same value for non-negative terms).  An SCC with
// more than kHeavyEdges successors goes to the heavy list (k_dp_eval_heavy).
__global__ void k_dp_eval(const uint32_t* front, const uint32_t* fcnt, const uint32_t* drp, const uint32_t* ddst,
                          const uint32_t* wsz, uint32_t* A, uint32_t* Om, uint32_t n, Refine rf, SccHeavy* H) {
    const uint32_t cnt = *fcnt;
    const bool refine = rf.big != 0xffffffffu;
    WARP_PER_ITEM(i, cnt) {
        const uint32_t c = front[i];
        const uint32_t b = drp[c], e = drp[c + 1];
        if (heavy_claim(H, c, e - b)) continue;
        uint32_t amax = 0;
        unsigned long long osum = 0, msum = 0;
        for (uint32_t k = b + lane_; k < e; k += 32) {
            const uint32_t d = ddst[k];
            const uint32_t a = A[d];
            amax = a > amax ? a : amax;
            osum += Om[d];
            if (refine && !rf.desc[d]) msum += rf.Wm[d];
        }
        for (int o = 16; o; o >>= 1) {
            const uint32_t t = __shfl_xor_sync(0xffffffffu, amax, o);
            amax = t > amax ? t : amax;
            osum += __shfl_xor_sync(0xffffffffu, osum, o);
            msum += __shfl_xor_sync(0xffffffffu, msum, o);
        }
        if (lane_ == 0) dp_finish(c, amax, osum, msum, wsz, A, Om, n, rf);
    }
}

// the heavy SCCs' successors over the whole grid, into per-SCC accumulators
__global__ void k_dp_eval_heavy(const uint32_t* drp, const uint32_t* ddst, const uint32_t* A, const uint32_t* Om,
                                Refine rf, SccHeavy* H) {
    const uint32_t hn = H->n < kSccHeavyCap ? H->n : kSccHeavyCap;
    const bool refine = rf.big != 0xffffffffu;
    const uint32_t lane = threadIdx.x & 31;
    for (uint32_t h = 0; h < hn; ++h) {
        const uint32_t c = H->item[h], b = drp[c], e = drp[c + 1];
        uint32_t amax = 0;
        unsigned long long osum = 0, msum = 0;
        GRID_STRIDE(k, (size_t)(e - b)) {
            const uint32_t d = ddst[b + k];
            const uint32_t a = A[d];
            amax = a > amax ? a : amax;
            osum += Om[d];
            if (refine && !rf.desc[d]) msum += rf.Wm[d];
        }
        for (int o = 16; o; o >>= 1) {
            const uint32_t t = __shfl_xor_sync(0xffffffffu, amax, o);
            amax = t > amax ? t : amax;
            osum += __shfl_xor_sync(0xffffffffu, osum, o);
            msum += __shfl_xor_sync(0xffffffffu, msum, o);
        }
        if (lane == 0) {
            atomicMax(&H->acc[h][0], (unsigned long long)amax);
            atomicAdd(&H->acc[h][1], osum);
            atomicAdd(&H->acc[h][2], msum);
        }
    }
}

__global__ void k_dp_heavy_finish(const uint32_t* wsz, uint32_t* A, uint32_t* Om, uint32_t n, Refine rf,
                                  const SccHeavy* H) {
    const uint32_t hn = H->n < kSccHeavyCap ? H->n : kSccHeavyCap;
    GRID_STRIDE(h, hn)
    dp_finish(H->item[h], (uint32_t)H->acc[h][0], H->acc[h][1], H->acc[h][2], wsz, A, Om, n, rf);
}

__device__ __forceinline__ void dp_release_arc(const uint32_t* pred, uint32_t e, bool valid, uint32_t* outcnt,
                                               uint32_t* next, uint32_t* ncnt) {
    bool ready = false;
    uint32_t p = 0;
    if (valid) {
        p = pred[e];
        ready = atomicSub(&outcnt[p], 1u) == 1u;
    }
    warp_append(ready, p, next, ncnt);
}

__global__ void k_dp_release(const uint32_t* front, const uint32_t* fcnt, const uint32_t* prp, const uint32_t* pred,
                             uint32_t* outcnt, uint32_t* next, uint32_t* ncnt, SccHeavy* H) {
    const uint32_t cnt = *fcnt;
    WARP_PER_ITEM(i, cnt) {
        uint32_t c = front[i];
        if (heavy_claim(H, c, prp[c + 1] - prp[c])) continue;
        for (uint32_t e0 = prp[c]; e0 < prp[c + 1]; e0 += 32)
            dp_release_arc(pred, e0 + lane_, e0 + lane_ < prp[c + 1], outcnt, next, ncnt);
    }
}

__global__ void k_dp_release_heavy(const uint32_t* prp, const uint32_t* pred, uint32_t* outcnt, uint32_t* next,
                                   uint32_t* ncnt, const SccHeavy* H) {
    const uint32_t hn = H->n < kSccHeavyCap ? H->n : kSccHeavyCap;
    for (uint32_t h = 0; h < hn; ++h) {
        const uint32_t c = H->item[h], b = prp[c], e = prp[c + 1];
        WARP_PER_ITEM(j, ((size_t)(e - b) + 31) / 32) {
            const size_t a = b + j * 32 + lane_;
            dp_release_arc(pred, (uint32_t)a, a < e, outcnt, next, ncnt);
        }
    }
}

// Largest SCC: labels follow smallest members, so the smallest label wins ties.
__global__ void k_argmax_comp(const uint32_t* wsz, uint32_t nc, unsigned long long* best) {
    unsigned long long b = 0;
    GRID_STRIDE(c, nc) {
        unsigned long long key = ((unsigned long long)wsz[c] << 32) | (0xffffffffull - c);
        b = key > b ? key : b;
    }
    for (int o = 16; o; o >>= 1) {
        unsigned long long t = __shfl_xor_sync(0xffffffffu, b, o);
        b = t > b ? t : b;
    }
    if ((threadIdx.x & 31) == 0) atomicMax(best, b);
}

__global__ void k_mark_seed(const unsigned long long* best, uint32_t* mark, uint32_t* list, uint32_t* cnt,
                            uint32_t* big) {
    uint32_t c = 0xffffffffu - (uint32_t)(*best & 0xffffffffull);
    mark[c] = 1;
    list[0] = c;
    *cnt = 1;
    *big = c;
}

// one BFS level over a DAG given as CSR (successors or predecessors); an
// SCC with more than kHeavyEdges arcs goes to the heavy list, whose arcs
// k_dag_reach_heavy spreads over the whole grid
__device__ __forceinline__ void dag_reach_arc(const uint32_t* adj, uint32_t e, bool valid, uint32_t* next,
                                              uint32_t* ncnt, uint32_t* mark) {
    bool app = false;
    uint32_t d = 0;
    if (valid) {
        d = adj[e];
        app = vload(&mark[d]) == 0 && atomicExch(&mark[d], 1u) == 0;
    }
    warp_append(app, d, next, ncnt);
}

__global__ void k_dag_reach(const uint32_t* ptr, const uint32_t* adj, const uint32_t* front, const uint32_t* fcnt,
                            uint32_t* next, uint32_t* ncnt, uint32_t* mark, SccHeavy* H) {
    const uint32_t cnt = *fcnt;
    WARP_PER_ITEM(i, cnt) {
        uint32_t c = front[i];
        if (heavy_claim(H, c, ptr[c + 1] - ptr[c])) continue;
        for (uint32_t e0 = ptr[c]; e0 < ptr[c + 1]; e0 += 32)
            dag_reach_arc(adj, e0 + lane_, e0 + lane_ < ptr[c + 1], next, ncnt, mark);
    }
}

__global__ void k_dag_reach_heavy(const uint32_t* ptr, const uint32_t* adj, uint32_t* next, uint32_t* ncnt,
                                  uint32_t* mark, const SccHeavy* H) {
    const uint32_t hn = H->n < kSccHeavyCap ? H->n : kSccHeavyCap;
    for (uint32_t h = 0; h < hn; ++h) {
        const uint32_t c = H->item[h], b = ptr[c], e = ptr[c + 1];
        WARP_PER_ITEM(j, ((size_t)(e - b) + 31) / 32) {
            const size_t a = b + j * 32 + lane_;
            dag_reach_arc(adj, (uint32_t)a, a < e, next, ncnt, mark);
        }
    }
}

__global__ void k_sum_marked(const uint32_t* wsz, const uint32_t* mark, uint32_t nc, unsigned long long* sum) {
    unsigned long long s = 0;
    GRID_STRIDE(c, nc) if (mark[c]) s += wsz[c];
    for (int o = 16; o; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
    if ((threadIdx.x & 31) == 0 && s) atomicAdd(sum, s);
}

__global__ void k_xbounds(uint32_t n, const uint32_t* comp, const uint32_t* A, const uint32_t* Om, uint32_t* xlo,
                          uint32_t* xhi) {
    GRID_STRIDE(v, n) {
        xlo[v] = A[comp[v]];
        xhi[v] = Om[comp[v]];
    }
}

// ---------------------------------------------------------------- host
static inline size_t al(size_t b) { return (b + 255) & ~(size_t)255; }

size_t scc_scratch_bytes(uint32_t n, uint64_t m) {
    size_t nb = al(((size_t)n + 1) * 4), mb = al((m ? m : 1) * 4), m8 = al((m ? m : 1) * 8);
    size_t s = 0;
    s += nb * 12;                 // cursor, drp, color, fw, bw, lists x2, minv, flags, ...
    s += mb * 4;                  // pred, dsrc, ddst, flags
    s += m8 * 2;                  // keys, keys_tmp
    s += al(scan_scratch_bytes((m > n ? m : n) + 1));
    s += al(radix_scratch_bytes(m ? m : 1));
    s += nb * 5 + 4096;           // refinement: desc, anc, Wm, two queues
    s += al(sizeof(SccHeavy) > sizeof(RowHeavy) ? sizeof(SccHeavy) : sizeof(RowHeavy));
    return s;
}

namespace {
struct Bump {
    char* p; size_t left;
    void* take(size_t b) {
        b = al(b);
        if (b > left) return nullptr;
        void* r = p;
        p += b;
        left -= b;
        return r;
    }
};

int read_u32(const uint32_t* d, uint32_t* h, cudaStream_t s) {
    if (cudaMemcpyAsync(h, d, 4, cudaMemcpyDeviceToHost, s) != cudaSuccess) return -1;
    return cudaStreamSynchronize(s) == cudaSuccess ? 0 : -1;
}
}  // namespace

#define LAUNCH(...)                                                  \
    do {                                                             \
        __VA_ARGS__;                                                 \
        note_launch();                                               \
        if (cudaGetLastError() != cudaSuccess) return -1;            \
    } while (0)

// In-arcs as a CSR: rrp[n+1], rcol[m] (rows unsorted).
int launch_reverse_csr(const uint32_t* rp, const uint32_t* col, uint32_t n, uint64_t m, uint32_t* rrp,
                       uint32_t* rcol, void* scratch, size_t scratch_bytes, cudaStream_t s) {
    if (n == 0) return 0;
    Bump B{(char*)scratch, scratch_bytes};
    uint32_t* cursor = (uint32_t*)B.take(((size_t)n + 1) * 4);
    uint32_t* total = (uint32_t*)B.take(64);
    void* scan_scr = B.take(scan_scratch_bytes((size_t)n + 1));
    RowHeavy* H = (RowHeavy*)B.take(sizeof(RowHeavy));
    if (!cursor || !total || !scan_scr || !H) return -1;
    const unsigned gw = grid_for((size_t)n * 32);
    cudaMemsetAsync(cursor, 0, ((size_t)n + 1) * 4, s);
    cudaMemsetAsync(&H->n, 0, 4, s);
    LAUNCH(k_count_in<<<gw, 256, 0, s>>>(rp, col, n, cursor, H));
    LAUNCH(k_count_in_heavy<<<152 * 8, 256, 0, s>>>(rp, col, cursor, H));
    if (exclusive_scan_u32(cursor, rrp, n, total, scan_scr, s)) return -1;
    LAUNCH(k_set_last<<<1, 1, 0, s>>>(rrp, n, (uint32_t)m));
    cudaMemcpyAsync(cursor, rrp, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    cudaMemsetAsync(&H->n, 0, 4, s);
    LAUNCH(k_fill_rev<<<gw, 256, 0, s>>>(rp, col, n, cursor, rcol, H));
    LAUNCH(k_fill_rev_heavy<<<152 * 8, 256, 0, s>>>(rp, col, cursor, rcol, H));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

int launch_scc_bounds(const uint32_t* rp, const uint32_t* col, const uint32_t* rrp, const uint32_t* rcol,
                      uint32_t n, uint64_t m, uint32_t* comp, uint32_t* xlo, uint32_t* xhi, uint32_t* n_scc_host,
                      int refine, void* scratch, size_t scratch_bytes, int* err, cudaStream_t s) {
    if (n == 0) { *n_scc_host = 0; return 0; }
    Bump B{(char*)scratch, scratch_bytes};
    uint32_t* cursor = (uint32_t*)B.take(((size_t)n + 1) * 4);
    uint32_t* drp_buf = (uint32_t*)B.take(((size_t)n + 1) * 4);
    uint32_t* pred_buf = (uint32_t*)B.take((m ? m : 1) * 4);
    uint32_t* sccv = comp;        // representative per vertex until the final labels
    uint32_t* color = (uint32_t*)B.take(((size_t)n + 1) * 4);
    uint32_t* fw = (uint32_t*)B.take(((size_t)n + 1) * 4);
    uint32_t* bw = (uint32_t*)B.take(((size_t)n + 1) * 4);
    uint32_t* L0 = (uint32_t*)B.take(((size_t)n + 1) * 4);
    uint32_t* L1 = (uint32_t*)B.take(((size_t)n + 1) * 4);
    uint32_t* minv = (uint32_t*)B.take(((size_t)n + 1) * 4);
    uint32_t* flags = (uint32_t*)B.take(((size_t)(m > n ? m : n) + 1) * 4);
    uint32_t* cnts = (uint32_t*)B.take(256);     // [0] changed, [1],[2] list counts, [3] total, [4] remaining,
                                                 // [5] arcs between SCCs
    SccHeavy* heavy = (SccHeavy*)B.take(sizeof(SccHeavy) > sizeof(RowHeavy) ? sizeof(SccHeavy) : sizeof(RowHeavy));
    if (!heavy) return -1;
    unsigned long long* best = (unsigned long long*)B.take(64);
    void* scan_scr = B.take(scan_scratch_bytes((m > n ? m : n) + 1));
    if (!cursor || !drp_buf || !pred_buf || !color || !fw || !bw || !L0 || !L1 || !minv || !flags || !cnts ||
        !best || !scan_scr)
        return -1;
    const unsigned gv = grid_for(n), gw = grid_for((size_t)n * 32);
    (void)err;
    LAUNCH(k_fill<<<gv, 256, 0, s>>>(sccv, n, UNSET));

    uint32_t h = 0;
    // (1) trimming, a few rounds
    for (int round = 0; round < 8; ++round) {
        cudaMemsetAsync(cnts, 0, 4, s);
        LAUNCH(k_trim<<<gv, 256, 0, s>>>(rp, col, rrp, rcol, n, sccv, cnts));
        if (read_u32(cnts, &h, s)) return -1;
        if (!h) break;
    }
    // (2) forward-backward from the pivot
    cudaMemsetAsync(best, 0, 8, s);
    LAUNCH(k_pivot<<<gv, 256, 0, s>>>(rp, rrp, n, sccv, best));
    unsigned long long hb = 0;
    cudaMemcpyAsync(&hb, best, 8, cudaMemcpyDeviceToHost, s);
    if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    if (hb) {
        uint32_t pivot = 0xffffffffu - (uint32_t)(hb & 0xffffffffull);
        for (int dir = 0; dir < 2; ++dir) {
            uint32_t* mark = dir ? bw : fw;
            cudaMemsetAsync(mark, 0, (size_t)n * 4, s);
            LAUNCH(k_seed_mark<<<1, 1, 0, s>>>(pivot, mark, L0, &cnts[1]));
            uint32_t *cur = L0, *nxt = L1, *cc = &cnts[1], *nc = &cnts[2];
            uint32_t fsize = 1;   // frontier size: the pivot
            for (;;) {
                cudaMemsetAsync(nc, 0, 4, s);
                if (reach_pull(fsize, n)) {
                    LAUNCH(k_reach_pull<<<gv, 256, 0, s>>>(dir ? rp : rrp, dir ? col : rcol, n, nxt, nc, mark, sccv,
                                                           color, 0));
                } else {
                    cudaMemsetAsync(&heavy->n, 0, 4, s);
                    LAUNCH(k_reach<<<gw, 256, 0, s>>>(dir ? rrp : rp, dir ? rcol : col, cur, cc, nxt, nc, mark, sccv,
                                                      color, 0, heavy));
                    LAUNCH(k_reach_heavy<<<152 * 8, 256, 0, s>>>(dir ? rrp : rp, dir ? rcol : col, nxt, nc, mark,
                                                                 sccv, color, 0, heavy));
                }
                if (read_u32(nc, &h, s)) return -1;
                if (!h) break;
                fsize = h;
                uint32_t* t = cur; cur = nxt; nxt = t;
                uint32_t* tc = cc; cc = nc; nc = tc;
            }
        }
        LAUNCH(k_assign_both<<<gv, 256, 0, s>>>(n, fw, bw, sccv, pivot));
        for (int round = 0; round < 8; ++round) {
            cudaMemsetAsync(cnts, 0, 4, s);
            LAUNCH(k_trim<<<gv, 256, 0, s>>>(rp, col, rrp, rcol, n, sccv, cnts));
            if (read_u32(cnts, &h, s)) return -1;
            if (!h) break;
        }
    }
    // (3) colouring until every vertex has an SCC
    cudaMemsetAsync(&cnts[4], 0, 4, s);
    LAUNCH(k_count_unset<<<gv, 256, 0, s>>>(n, sccv, &cnts[4]));
    uint32_t remaining = 0;
    if (read_u32(&cnts[4], &remaining, s)) return -1;
    while (remaining) {
        LAUNCH(k_color_init<<<gv, 256, 0, s>>>(n, sccv, color));
        for (;;) {
            cudaMemsetAsync(cnts, 0, 4, s);
            LAUNCH(k_color_prop<<<gw, 256, 0, s>>>(rp, col, n, sccv, color, cnts));
            if (read_u32(cnts, &h, s)) return -1;
            if (!h) break;
        }
        cudaMemsetAsync(bw, 0, (size_t)n * 4, s);
        cudaMemsetAsync(&cnts[1], 0, 8, s);
        LAUNCH(k_color_roots<<<gv, 256, 0, s>>>(n, sccv, color, bw, L0, &cnts[1]));
        uint32_t *cur = L0, *nxt = L1, *cc = &cnts[1], *nc = &cnts[2];
        uint32_t fsize = 0;
        if (read_u32(cc, &fsize, s)) return -1;   // the colour roots
        for (;;) {
            cudaMemsetAsync(nc, 0, 4, s);
            if (reach_pull(fsize, n)) {
                LAUNCH(k_reach_pull<<<gv, 256, 0, s>>>(rp, col, n, nxt, nc, bw, sccv, color, 1));
            } else {
                cudaMemsetAsync(&heavy->n, 0, 4, s);
                LAUNCH(k_reach<<<gw, 256, 0, s>>>(rrp, rcol, cur, cc, nxt, nc, bw, sccv, color, 1, heavy));
                LAUNCH(k_reach_heavy<<<152 * 8, 256, 0, s>>>(rrp, rcol, nxt, nc, bw, sccv, color, 1, heavy));
            }
            if (read_u32(nc, &h, s)) return -1;
            if (!h) break;
            fsize = h;
            uint32_t* t = cur; cur = nxt; nxt = t;
            uint32_t* tc = cc; cc = nc; nc = tc;
        }
        cudaMemsetAsync(&cnts[4], 0, 4, s);
        LAUNCH(k_assign_marked<<<gv, 256, 0, s>>>(n, sccv, color, bw, &cnts[4]));
        if (read_u32(&cnts[4], &remaining, s)) return -1;
    }
    // labels by smallest member
    LAUNCH(k_fill<<<gv, 256, 0, s>>>(minv, n, UNSET));
    LAUNCH(k_minrep<<<gv, 256, 0, s>>>(n, sccv, minv));
    LAUNCH(k_min_flags<<<gv, 256, 0, s>>>(n, sccv, minv, flags));
    if (exclusive_scan_u32(flags, flags, n, &cnts[3], scan_scr, s)) return -1;
    LAUNCH(k_label<<<gv, 256, 0, s>>>(n, sccv, minv, flags, color));   // labels into color
    uint32_t nscc = 0;
    if (read_u32(&cnts[3], &nscc, s)) return -1;
    cudaMemcpyAsync(comp, color, (size_t)n * 4, cudaMemcpyDeviceToDevice, s);
    *n_scc_host = nscc;

    // DAG arcs, unique, sorted by (source, target)
    int b = 1;
    while ((1ull << b) < (unsigned long long)nscc) ++b;
    uint32_t* wsz = minv;         // reuse
    uint32_t* A = fw;
    uint32_t* Om = bw;
    uint32_t* outcnt = cursor;
    uint32_t* drp = drp_buf;
    uint32_t* prp = L1;
    uint32_t ndag = 0;
    uint32_t* dsrc = nullptr;
    uint32_t* ddst = nullptr;
    uint32_t* pred = nullptr;
    if (m) {
        unsigned long long* keys = (unsigned long long*)B.take(m * 8);
        unsigned long long* ktmp = (unsigned long long*)B.take(m * 8);
        dsrc = (uint32_t*)B.take(m * 4);
        ddst = (uint32_t*)B.take(m * 4);
        pred = pred_buf;
        void* rscr = B.take(radix_scratch_bytes(m));
        if (!keys || !ktmp || !dsrc || !ddst || !rscr) return -1;
        RowHeavy* RH = (RowHeavy*)heavy;   // the SCC heavy area is free here and at least as large
        cudaMemsetAsync(&RH->n, 0, 4, s);
        cudaMemsetAsync(&cnts[5], 0, 4, s);
        LAUNCH(k_dag_keys<<<gw, 256, 0, s>>>(rp, col, n, comp, b, keys, &cnts[5], RH));
        LAUNCH(k_dag_keys_heavy<<<152 * 8, 256, 0, s>>>(rp, col, comp, b, keys, &cnts[5], RH));
        uint32_t mk = 0;   // arcs between SCCs
        if (read_u32(&cnts[5], &mk, s)) return -1;
        if (mk) {
            bool in_tmp = false;
            if (radix_sort_u64((uint64_t*)keys, (uint64_t*)ktmp, mk, 2 * b, rscr, s, &in_tmp)) return -1;
            unsigned long long* sk = in_tmp ? ktmp : keys;
            LAUNCH(k_unique_flags<<<grid_for(mk), 256, 0, s>>>(sk, mk, flags));
            uint32_t* pos = (uint32_t*)(in_tmp ? (void*)keys : (void*)ktmp);   // the other key buffer as scratch
            if (exclusive_scan_u32(flags, pos, mk, &cnts[3], scan_scr, s)) return -1;
            LAUNCH(k_unique_scatter<<<grid_for(mk), 256, 0, s>>>(sk, mk, flags, pos, b, dsrc, ddst));
            if (read_u32(&cnts[3], &ndag, s)) return -1;
        }
    }
    // component sizes; DAG CSR (successors) and predecessor lists
    cudaMemsetAsync(wsz, 0, ((size_t)nscc + 1) * 4, s);
    LAUNCH(k_hist<<<gv, 256, 0, s>>>(comp, n, wsz));
    cudaMemsetAsync(outcnt, 0, ((size_t)nscc + 1) * 4, s);
    if (ndag) LAUNCH(k_hist<<<grid_for(ndag), 256, 0, s>>>(dsrc, ndag, outcnt));
    if (exclusive_scan_u32(outcnt, drp, nscc, &cnts[3], scan_scr, s)) return -1;
    LAUNCH(k_set_last<<<1, 1, 0, s>>>(drp, nscc, ndag));
    cudaMemsetAsync(outcnt, 0, ((size_t)nscc + 1) * 4, s);
    if (ndag) LAUNCH(k_hist<<<grid_for(ndag), 256, 0, s>>>(ddst, ndag, outcnt));
    if (exclusive_scan_u32(outcnt, prp, nscc, &cnts[3], scan_scr, s)) return -1;
    LAUNCH(k_set_last<<<1, 1, 0, s>>>(prp, nscc, ndag));
    cudaMemcpyAsync(outcnt, prp, (size_t)nscc * 4, cudaMemcpyDeviceToDevice, s);
    if (ndag) LAUNCH(k_scatter_pred<<<grid_for(ndag), 256, 0, s>>>(dsrc, ddst, ndag, outcnt, pred));
    // biggest-SCC refinement: the largest SCC, its descendants and ancestors
    Refine rf{0xffffffffu, nullptr, nullptr, nullptr, nullptr};
    if (refine && nscc > 1) {
        uint32_t* desc = (uint32_t*)B.take(((size_t)nscc + 1) * 4);
        uint32_t* anc = (uint32_t*)B.take(((size_t)nscc + 1) * 4);
        uint32_t* Wm = (uint32_t*)B.take(((size_t)nscc + 1) * 4);
        uint32_t* Q0 = (uint32_t*)B.take(((size_t)nscc + 1) * 4);
        uint32_t* Q1 = (uint32_t*)B.take(((size_t)nscc + 1) * 4);
        unsigned long long* rsum = (unsigned long long*)B.take(64);
        uint32_t* dbig = (uint32_t*)B.take(64);
        uint32_t* R32 = (uint32_t*)B.take(64);
        if (!desc || !anc || !Wm || !Q0 || !Q1 || !rsum || !dbig || !R32) return -1;
        cudaMemsetAsync(best, 0, 8, s);
        LAUNCH(k_argmax_comp<<<grid_for(nscc), 256, 0, s>>>(wsz, nscc, best));
        for (int dir = 0; dir < 2; ++dir) {     // 0: descendants, 1: ancestors
            uint32_t* mark = dir ? anc : desc;
            cudaMemsetAsync(mark, 0, (size_t)nscc * 4, s);
            cudaMemsetAsync(&cnts[1], 0, 8, s);
            LAUNCH(k_mark_seed<<<1, 1, 0, s>>>(best, mark, Q0, &cnts[1], dbig));
            uint32_t *cur = Q0, *nxt = Q1, *cc = &cnts[1], *nc2 = &cnts[2];
            for (;;) {
                cudaMemsetAsync(nc2, 0, 4, s);
                cudaMemsetAsync(&heavy->n, 0, 4, s);
                LAUNCH(k_dag_reach<<<grid_for((size_t)nscc * 32), 256, 0, s>>>(dir ? prp : drp, dir ? pred : ddst,
                                                                               cur, cc, nxt, nc2, mark, heavy));
                LAUNCH(k_dag_reach_heavy<<<152 * 8, 256, 0, s>>>(dir ? prp : drp, dir ? pred : ddst, nxt, nc2, mark,
                                                                  heavy));
                if (read_u32(nc2, &h, s)) return -1;
                if (!h) break;
                uint32_t* t = cur; cur = nxt; nxt = t;
                uint32_t* tc = cc; cc = nc2; nc2 = tc;
            }
        }
        cudaMemsetAsync(rsum, 0, 8, s);
        LAUNCH(k_sum_marked<<<grid_for(nscc), 256, 0, s>>>(wsz, desc, nscc, rsum));
        uint32_t hbig = 0;
        unsigned long long hR = 0;
        cudaMemcpyAsync(&hbig, dbig, 4, cudaMemcpyDeviceToHost, s);
        cudaMemcpyAsync(&hR, rsum, 8, cudaMemcpyDeviceToHost, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
        uint32_t R = (uint32_t)hR;
        cudaMemcpyAsync(R32, &R, 4, cudaMemcpyHostToDevice, s);
        // anc marks big itself (the BFS seed); the programme treats big apart
        rf = Refine{hbig, R32, desc, anc, Wm};
        if (cudaStreamSynchronize(s) != cudaSuccess) return -1;
    }
    // alpha / omega, sinks first
    uint32_t* F0 = L0;
    uint32_t* F1 = color;         // labels were copied out to comp
    cudaMemsetAsync(&cnts[1], 0, 8, s);
    LAUNCH(k_sinks<<<grid_for(nscc), 256, 0, s>>>(nscc, drp, outcnt, F0, &cnts[1]));
    uint32_t *cur = F0, *nxt = F1, *cc = &cnts[1], *nc = &cnts[2];
    uint32_t fcount = 0;
    if (read_u32(cc, &fcount, s)) return -1;
    uint32_t done = 0;
    while (fcount) {
        done += fcount;
        cudaMemsetAsync(heavy, 0, sizeof(SccHeavy), s);
        LAUNCH(k_dp_eval<<<grid_for((size_t)fcount * 32), 256, 0, s>>>(cur, cc, drp, ddst, wsz, A, Om, n, rf, heavy));
        LAUNCH(k_dp_eval_heavy<<<152 * 8, 256, 0, s>>>(drp, ddst, A, Om, rf, heavy));
        LAUNCH(k_dp_heavy_finish<<<1, 256, 0, s>>>(wsz, A, Om, n, rf, heavy));
        cudaMemsetAsync(nc, 0, 4, s);
        cudaMemsetAsync(&heavy->n, 0, 4, s);
        LAUNCH(k_dp_release<<<grid_for((size_t)fcount * 32), 256, 0, s>>>(cur, cc, prp, pred, outcnt, nxt, nc, heavy));
        LAUNCH(k_dp_release_heavy<<<152 * 8, 256, 0, s>>>(prp, pred, outcnt, nxt, nc, heavy));
        if (read_u32(nc, &fcount, s)) return -1;
        uint32_t* t = cur; cur = nxt; nxt = t;
        uint32_t* tc = cc; cc = nc; nc = tc;
    }
    if (done != nscc) return -1;   // the DAG must be acyclic
    LAUNCH(k_xbounds<<<gv, 256, 0, s>>>(n, comp, A, Om, xlo, xhi));
    return cudaGetLastError() == cudaSuccess ? 0 : -1;
}

}  // namespace bcm
