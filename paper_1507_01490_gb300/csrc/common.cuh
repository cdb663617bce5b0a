// Device-side building blocks shared by the BCM kernels: the ranking key,
// the stopping rule of BFSCut, the shared top-k with its published
// threshold, bounded waits, and the MS-BFS push step.
//
// Paper: Borassi, Crescenzi, Marino, "Fast and Simple Computation of Top-k
// Closeness Centralities" (arXiv 1507.01490).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace bcm {

typedef unsigned long long u64;
typedef unsigned int u32;

// ---------------------------------------------------------------- errors
enum DevErr : int {
    DEV_OK = 0,
    DEV_ERR_BARRIER_TIMEOUT = 1,   // a grid barrier wait ran past its limit
    DEV_ERR_LOCK_TIMEOUT = 2,      // the top-k lock wait ran past its limit
    DEV_ERR_INVALID_CSR = 4,       // input validation failed
    DEV_ERR_RETRY_LIMIT = 8,       // a lock-free retry loop exceeded its cap
    DEV_ERR_TABLE_FULL = 16,       // a per-CTA wave's vertex table filled where no grid pass could take it
};

__device__ __forceinline__ u64 global_ns() {
    u64 t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ u32 lanemask_lt() {
    u32 m;
    asm("mov.u32 %0, %%lanemask_lt;" : "=r"(m));
    return m;
}

template <typename T>
__device__ __forceinline__ T vload(const T* p) { return *(const volatile T*)p; }
template <typename T>
__device__ __forceinline__ void vstore(T* p, T v) { *(volatile T*)p = v; }

// ---------------------------------------------------------- ranking key
// c(v) = (r-1)^2 / ((n-1) f) (Section 1).  n-1 is common to every vertex, so
// vertices are ranked by s = (r-1)^2 / f held as the exact pair (N, F);
// r = 1 gives s = 0 with the pair (0, 1).  Ties: the smaller id ranks first.
__device__ __forceinline__ void score_key(u64 f, u32 r, u64& N, u64& F) {
    if (r <= 1 || f == 0) { N = 0; F = 1; return; }
    u64 a = (u64)(r - 1);
    N = a * a;
    F = f;
}

__device__ __forceinline__ bool ranks_before(u64 Na, u64 Fa, u32 ida, u64 Nb, u64 Fb, u32 idb) {
    unsigned __int128 l = (unsigned __int128)Na * Fb, r = (unsigned __int128)Nb * Fa;
    if (l != r) return l > r;
    return ida < idb;
}

// Published threshold: the rank key of the current k-th entry (x_k of
// Algorithm 1).  Writers hold the top-k lock and bump seq to odd, write,
// then bump to even; readers retry until they see one even seq on both
// sides of their reads.
struct Threshold {
    u64 seq;
    u64 N, F;
    u32 id, valid;
};

struct ThrCache { u64 N, F; u32 id, valid; };

// A consistent snapshot, or the previous one if none could be taken.  The
// threshold only rises, so an older snapshot is a weaker (still valid) one.
__device__ __forceinline__ void read_threshold(const Threshold* t, ThrCache& c) {
    for (int tries = 0; tries < 64; ++tries) {
        u64 s1 = vload(&t->seq);
        if (s1 & 1) { __nanosleep(32); continue; }
        __threadfence();
        u64 N = vload(&t->N), F = vload(&t->F);
        u32 id = vload(&t->id), valid = vload(&t->valid);
        __threadfence();
        if (vload(&t->seq) == s1) { c.N = N; c.F = F; c.id = id; c.valid = valid; return; }
    }
}

// The threshold every block of a grid-wide launch cuts with at one level:
// taken by the leader block's thread 0 before a grid barrier and read by all
// blocks after it, so that they agree on which lanes live (a key offered by
// the host may arrive between two blocks' own reads of the published ones).
__device__ __forceinline__ void store_snapshot(Threshold* snap, const ThrCache& c) {
    vstore(&snap->N, c.N);
    vstore(&snap->F, c.F);
    vstore(&snap->id, c.id);
    vstore(&snap->valid, c.valid);
}
__device__ __forceinline__ void load_snapshot(const Threshold* snap, ThrCache& c) {
    c.N = vload(&snap->N);
    c.F = vload(&snap->F);
    c.id = vload(&snap->id);
    c.valid = vload(&snap->valid);
}

// ------------------------------------------------- stopping rule (BFSCut)
// Lemma 1: f(v) >= f~_d(v, x) = f_d - g + (d+2)(x - n_d), g >= gamma_{d+1}.
// Lemma 2: on digraphs the bound is taken at x = alpha(v) and x = omega(v).
// v cannot enter the top-k once, for every x,
//   f~ * N_k >  F_k (x-1)^2          (v ranks strictly below the k-th), or
//   f~ * N_k >= F_k (x-1)^2 and v > id_k   (a tie that v loses on its id).
// Every product is formed exactly in 128-bit integers (n < 2^31).
__device__ __forceinline__ bool bfscut_stops(u64 f_d, u64 g, u32 d, u32 n_d, u32 xlo, u32 xhi,
                                             u32 v, const ThrCache& t) {
    if (!t.valid) return false;
    bool all_strict = true, all_weak = true;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
        u32 x = i ? xhi : xlo;
        __int128 ft = (__int128)f_d - (__int128)g + (__int128)(d + 2) * ((__int128)x - (__int128)n_d);
        __int128 lhs = ft * (__int128)t.N;
        __int128 xm1 = (__int128)x - 1;
        __int128 rhs = (__int128)t.F * xm1 * xm1;
        all_strict = all_strict && (lhs > rhs);
        all_weak = all_weak && (lhs >= rhs);
    }
    return all_strict || (all_weak && v > t.id);
}

// ------------------------------------------------------- shared top-k
struct TopK {
    u32* id;          // [k] rank order, best first
    u64* f;
    u32* r;
    u32* count;       // entries held (<= k)
    u32* lock;        // 0 free, 1 held
    Threshold* thr;   // published k-th key
    Threshold* ext;   // a key offered from outside the run (another shard's k-th), or NULL
    u32 k;
};

// The threshold a run cuts with: its own published k-th key or the offered
// one, whichever ranks first.  Both are valid: the offered key is the k-th of
// another shard of the same graph, and at least k vertices of the graph rank
// at or before it, so a source ranking after it cannot be in the top-k.
__device__ __forceinline__ void read_thresholds(const TopK& T, ThrCache& c) {
    read_threshold(T.thr, c);
    if (!T.ext || vload(&T.ext->seq) == 0) return;   // nothing offered (yet)
    ThrCache e;
    e.valid = 0; e.N = 0; e.F = 1; e.id = 0;
    read_threshold(T.ext, e);
    if (e.valid && (!c.valid || ranks_before(e.N, e.F, e.id, c.N, c.F, c.id))) c = e;
}

__device__ __forceinline__ bool lock_acquire(u32* lock, u64 limit_ns, int* err) {
    u64 t0 = global_ns();
    u32 ns = 32;
    while (atomicCAS(lock, 0u, 1u) != 0u) {
        if (global_ns() - t0 > limit_ns) { atomicOr(err, DEV_ERR_LOCK_TIMEOUT); return false; }
        __nanosleep(ns);
        if (ns < 1024) ns <<= 1;
    }
    __threadfence();
    return true;
}

__device__ __forceinline__ void lock_release(u32* lock) {
    __threadfence();
    atomicExch(lock, 0u);
}

// Inserts (v, f, r) if it ranks before the current k-th (or fewer than k are
// held).  Caller holds the lock.  One thread.
__device__ inline void topk_insert_locked(const TopK& T, u32 v, u64 f, u32 r) {
    u64 Nv, Fv;
    score_key(f, r, Nv, Fv);
    u32 cnt = vload(T.count);
    if (cnt == T.k) {
        u64 Nk, Fk;
        score_key(vload(&T.f[cnt - 1]), vload(&T.r[cnt - 1]), Nk, Fk);
        if (!ranks_before(Nv, Fv, v, Nk, Fk, vload(&T.id[cnt - 1]))) return;
        --cnt;
    }
    u32 pos = cnt;
    while (pos > 0) {
        u64 Np, Fp;
        u32 idp = vload(&T.id[pos - 1]);
        u64 fp = vload(&T.f[pos - 1]);
        u32 rp = vload(&T.r[pos - 1]);
        score_key(fp, rp, Np, Fp);
        if (!ranks_before(Nv, Fv, v, Np, Fp, idp)) break;
        vstore(&T.id[pos], idp); vstore(&T.f[pos], fp); vstore(&T.r[pos], rp);
        --pos;
    }
    vstore(&T.id[pos], v); vstore(&T.f[pos], f); vstore(&T.r[pos], r);
    vstore(T.count, cnt + 1);
}

// Publishes the k-th key (caller holds the lock).
__device__ inline void topk_publish_locked(const TopK& T) {
    u32 cnt = vload(T.count);
    if (cnt < T.k) return;
    u64 N, F;
    score_key(vload(&T.f[T.k - 1]), vload(&T.r[T.k - 1]), N, F);
    u32 id = vload(&T.id[T.k - 1]);
    atomicAdd(&T.thr->seq, 1ull);          // odd: write in progress
    __threadfence();
    vstore(&T.thr->N, N); vstore(&T.thr->F, F); vstore(&T.thr->id, id); vstore(&T.thr->valid, 1u);
    __threadfence();
    atomicAdd(&T.thr->seq, 1ull);          // even: consistent
}

// --------------------------------------------------------- grid barrier
// Sense-free counting barrier for co-resident (cooperatively launched)
// grids.  Every wait is bounded: past limit_ns the barrier records
// DEV_ERR_BARRIER_TIMEOUT and returns false, and callers leave their loops.
struct GridBarrier { u32 count; u32 gen; };

__device__ inline bool grid_sync(GridBarrier* b, u32 nblocks, u64 limit_ns, int* err) {
    __shared__ int s_ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int ok = 1;
        u32 g = vload(&b->gen);
        __threadfence();
        u32 prev = atomicAdd(&b->count, 1u);
        if (prev == nblocks - 1) {
            atomicExch(&b->count, 0u);
            __threadfence();
            atomicAdd(&b->gen, 1u);
        } else {
            u64 t0 = global_ns();
            u32 ns = 32;
            while (vload(&b->gen) == g) {
                if (vload(err) != 0) { ok = 0; break; }   // another block gave up: leave at once
                if (global_ns() - t0 > limit_ns) { atomicOr(err, DEV_ERR_BARRIER_TIMEOUT); ok = 0; break; }
                __nanosleep(ns);
                if (ns < 256) ns <<= 1;
            }
        }
        __threadfence();
        s_ok = ok && (vload(err) == 0);
    }
    __syncthreads();
    return s_ok;
}

// ------------------------------------------------------ warp utilities
// Appends `item` for every lane with `want` set: one atomic per warp.
__device__ __forceinline__ void warp_append(bool want, u32 item, u32* list, u32* counter) {
    u32 m = __ballot_sync(0xffffffffu, want);
    if (m == 0) return;
    int leader = __ffs(m) - 1;
    u32 base = 0;
    if ((int)(threadIdx.x & 31) == leader) base = atomicAdd(counter, (u32)__popc(m));
    base = __shfl_sync(0xffffffffu, base, leader);
    if (want) list[base + __popc(m & lanemask_lt())] = item;
}

}  // namespace bcm
