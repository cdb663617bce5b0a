/*
 * CPU oracle for exact top-k closeness -- TEST INFRASTRUCTURE ONLY.
 *
 * Only tests/, __graft_entry__.smoke() and bench.py's CPU-baseline leg may
 * load this file's library.  The CUDA path never calls it, and the two share
 * no code: this file includes nothing from the package and the package
 * includes nothing from here.
 *
 * Paper: Borassi, Crescenzi, Marino, "Fast and Simple Computation of Top-k
 * Closeness Centralities" (arXiv 1507.01490).  Citations below name the
 * paper's section, table, lemma or algorithm.
 *
 * Contents
 *   oracle_farness_all  the plain definition (Table 1; Section 1 formula):
 *                       one FIFO BFS per source, r(v) = |R(v)|,
 *                       f(v) = sum of d(v,w) over R(v).
 *   oracle_topk         the k largest closeness values, exact rational order,
 *                       ties by smaller id.
 *   oracle_scc          strongly connected components (Tarjan's algorithm).
 *   oracle_alpha_omega  Section 2.3: weighted SCC DAG, topological sort, then
 *                       the reverse-order dynamic programme for alpha and omega.
 *   oracle_bound_trace  Lemma 1's bound f~_d(v,x) at every level of one BFS.
 *   oracle_bcm          Algorithm 1 driving BFSCut (Algorithm 2, generalised
 *                       as Sections 2.2-2.3 describe), sequential.
 *   oracle_bcm_sources  the same loop over one shard's sources, resumable,
 *                       with an outside k-th key (Section 2's shared x_k).
 *
 * Ranking key.  c(v) = (r-1)^2 / ((n-1) f) (Section 1).  n-1 is common to all
 * vertices, so the ranking uses s(v) = (r-1)^2 / f kept as the exact pair
 * (N, F) = ((r-1)^2, f); a vertex with r = 1 has s = 0 and key (0, 1).
 * a ranks before b iff N_a F_b > N_b F_a, or equal and id_a < id_b.
 * Products are formed in 128-bit integers; vertex counts are below 2^31.
 *
 * Parity pins live in tests/test_oracle_*.py: closed-form farness (path, star,
 * cycle, complete, grid, directed path and cycle), Floyd-Warshall on small
 * graphs, scipy's BFS and SCC routines, brute-force ranking with exact
 * fractions, alpha <= r <= omega, and BCM's top-k = exhaustive top-k.
 */
#define _GNU_SOURCE   /* qsort_r */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <pthread.h>

typedef __int128 i128;
typedef unsigned __int128 u128;

/* ------------------------------------------------------------ ranking */

static void score_key(uint64_t f, uint32_t r, uint64_t *N, uint64_t *F) {
    if (r <= 1 || f == 0) { *N = 0; *F = 1; return; }
    uint64_t a = (uint64_t)(r - 1);
    *N = a * a;
    *F = f;
}

/* 1 if vertex a ranks strictly before vertex b */
static int ranks_before(uint64_t Na, uint64_t Fa, uint32_t ida,
                        uint64_t Nb, uint64_t Fb, uint32_t idb) {
    u128 l = (u128)Na * Fb, r = (u128)Nb * Fa;
    if (l != r) return l > r;
    return ida < idb;
}

/* ------------------------------------------------------ one plain BFS */

typedef struct {
    uint32_t *queue;     /* FIFO */
    uint32_t *dist;
    uint32_t *seen;      /* seen[w] == epoch  <=>  w visited by the current BFS */
    uint32_t epoch;
} bfs_ws;

static int ws_init(bfs_ws *ws, uint32_t n) {
    ws->queue = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    ws->dist = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    ws->seen = (uint32_t *)calloc(n ? n : 1, sizeof(uint32_t));
    ws->epoch = 0;
    return ws->queue && ws->dist && ws->seen;
}

static void ws_free(bfs_ws *ws) { free(ws->queue); free(ws->dist); free(ws->seen); }

static void ws_next_epoch(bfs_ws *ws, uint32_t n) {
    if (++ws->epoch == 0) { memset(ws->seen, 0, sizeof(uint32_t) * n); ws->epoch = 1; }
}

/* BFS from v over out-arcs.  r = |R(v)|, f = sum of distances, arcs = number
 * of arcs scanned (sum of outdeg over R(v)). */
static void bfs_one(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, uint32_t v,
                    bfs_ws *ws, uint64_t *f_out, uint32_t *r_out, uint64_t *arcs_out) {
    ws_next_epoch(ws, n);
    uint32_t head = 0, tail = 0;
    ws->queue[tail++] = v;
    ws->seen[v] = ws->epoch;
    ws->dist[v] = 0;
    uint64_t f = 0, arcs = 0;
    while (head < tail) {
        uint32_t u = ws->queue[head++];
        f += ws->dist[u];
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            uint32_t w = col[e];
            if (ws->seen[w] != ws->epoch) {
                ws->seen[w] = ws->epoch;
                ws->dist[w] = ws->dist[u] + 1;
                ws->queue[tail++] = w;
            }
        }
        arcs += row_ptr[u + 1] - row_ptr[u];
    }
    *f_out = f;
    *r_out = tail;
    *arcs_out = arcs;
}

/* ---------------------------------------------- exhaustive (textbook) */

typedef struct {
    uint32_t n; const uint64_t *row_ptr; const uint32_t *col;
    const uint32_t *sources; uint64_t nsrc;
    uint64_t *farness; uint32_t *reach; uint64_t *arcs;
    uint64_t next;      /* shared work counter */
    uint64_t grain;     /* sources per grab */
    int failed;
    int workers;        /* threads that took at least one source */
} fa_job;

typedef struct { fa_job *J; uint64_t first; } fa_arg;

/* Grab `first` (a block fixed per thread, so that every thread has work
 * whenever there are enough sources), then blocks from the shared counter. */
static void *fa_worker(void *arg) {
    fa_job *J = ((fa_arg *)arg)->J;
    uint64_t first = ((fa_arg *)arg)->first;
    bfs_ws ws;
    if (!ws_init(&ws, J->n)) { __atomic_store_n(&J->failed, 1, __ATOMIC_RELAXED); ws_free(&ws); return NULL; }
    int took = 0;
    for (;;) {
        uint64_t i0 = first;
        first = UINT64_MAX;
        if (i0 == UINT64_MAX) i0 = __atomic_fetch_add(&J->next, J->grain, __ATOMIC_RELAXED);
        if (i0 >= J->nsrc) break;
        if (!took) { took = 1; __atomic_fetch_add(&J->workers, 1, __ATOMIC_RELAXED); }
        uint64_t i1 = i0 + J->grain < J->nsrc ? i0 + J->grain : J->nsrc;
        for (uint64_t i = i0; i < i1; ++i) {
            uint32_t v = J->sources ? J->sources[i] : (uint32_t)i;
            uint64_t f, a; uint32_t r;
            bfs_one(J->n, J->row_ptr, J->col, v, &ws, &f, &r, &a);
            J->farness[i] = f;
            J->reach[i] = r;
            if (J->arcs) J->arcs[i] = a;
        }
    }
    ws_free(&ws);
    return NULL;
}

/* f and r of each listed source (all vertices when sources == NULL, nsrc = n).
 * Output i belongs to sources[i].  arcs (nullable) receives the arcs each BFS
 * scanned, whose sum over all v is the textbook algorithm's m_tot (Section 3.1).
 * Threads take sources in grabs of nsrc / (4 threads), at least 1 and at most
 * 64, so that every thread gets work even on a short list.  Returns the
 * number of threads that took work (0 when nsrc = 0), or -1 on allocation
 * failure. */
int oracle_farness_all(uint32_t n, const uint64_t *row_ptr, const uint32_t *col,
                       const uint32_t *sources, uint64_t nsrc,
                       uint64_t *farness, uint32_t *reach, uint64_t *arcs, int threads) {
    if (threads < 1) threads = 1;
    if (threads > 256) threads = 256;
    uint64_t total = sources ? nsrc : n;
    uint64_t grain = total / (4 * (uint64_t)threads);
    if (grain < 1) grain = 1;
    if (grain > 64) grain = 64;
    fa_job J = { n, row_ptr, col, sources, total, farness, reach, arcs, grain * (uint64_t)threads, grain, 0, 0 };
    pthread_t th[256];
    fa_arg args[256];
    int started = 0;
    for (int t = 0; t < threads; ++t) {
        args[t].J = &J;
        args[t].first = grain * (uint64_t)t;
        if (pthread_create(&th[started], NULL, fa_worker, &args[t]) == 0) ++started;
        else fa_worker(&args[t]);   /* no thread: its block (and whatever is left) runs here */
    }
    for (int t = 0; t < started; ++t) pthread_join(th[t], NULL);
    return J.failed ? -1 : J.workers;
}

/* ------------------------------------------------------------- top-k */

typedef struct { const uint64_t *f; const uint32_t *r; } rank_ctx;

static int rank_cmp(const void *pa, const void *pb, void *pc) {
    const rank_ctx *c = (const rank_ctx *)pc;
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    uint64_t Na, Fa, Nb, Fb;
    score_key(c->f[a], c->r[a], &Na, &Fa);
    score_key(c->f[b], c->r[b], &Nb, &Fb);
    if (ranks_before(Na, Fa, a, Nb, Fb, b)) return -1;
    if (ranks_before(Nb, Fb, b, Na, Fa, a)) return 1;
    return 0;
}

/* ids of the min(k, n) vertices of largest closeness, in rank order. */
int oracle_topk(uint32_t n, const uint64_t *farness, const uint32_t *reach, uint32_t k,
                uint32_t *ids_out) {
    uint32_t *ids = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    if (!ids) return -1;
    for (uint32_t i = 0; i < n; ++i) ids[i] = i;
    rank_ctx c = { farness, reach };
    qsort_r(ids, n, sizeof(uint32_t), rank_cmp, &c);
    uint32_t kk = k < n ? k : n;
    memcpy(ids_out, ids, sizeof(uint32_t) * kk);
    free(ids);
    return (int)kk;
}

/* ---------------------------------------------------- SCC (Tarjan) */

/* comp[v] in [0, n_scc).  Tarjan's algorithm, iterative.  Returns n_scc, or
 * -1 on allocation failure. */
int64_t oracle_scc(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, uint32_t *comp) {
    const uint32_t UNSEEN = 0xffffffffu;
    uint32_t *index = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *low = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint8_t *on = (uint8_t *)calloc(n ? n : 1, 1);
    uint32_t *stk = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint32_t *cs_v = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    uint64_t *cs_e = (uint64_t *)malloc(sizeof(uint64_t) * (n ? n : 1));
    if (!index || !low || !on || !stk || !cs_v || !cs_e) {
        free(index); free(low); free(on); free(stk); free(cs_v); free(cs_e); return -1;
    }
    for (uint32_t v = 0; v < n; ++v) index[v] = UNSEEN;
    uint32_t counter = 0, sp = 0, ncomp = 0;
    for (uint32_t root = 0; root < n; ++root) {
        if (index[root] != UNSEEN) continue;
        uint32_t csp = 0;
        cs_v[csp] = root; cs_e[csp] = row_ptr[root]; ++csp;
        index[root] = low[root] = counter++;
        stk[sp++] = root; on[root] = 1;
        while (csp > 0) {
            uint32_t v = cs_v[csp - 1];
            if (cs_e[csp - 1] < row_ptr[v + 1]) {
                uint32_t w = col[cs_e[csp - 1]++];
                if (index[w] == UNSEEN) {
                    index[w] = low[w] = counter++;
                    stk[sp++] = w; on[w] = 1;
                    cs_v[csp] = w; cs_e[csp] = row_ptr[w]; ++csp;
                } else if (on[w] && index[w] < low[v]) {
                    low[v] = index[w];
                }
            } else {
                --csp;
                if (csp > 0) {
                    uint32_t p = cs_v[csp - 1];
                    if (low[v] < low[p]) low[p] = low[v];
                }
                if (low[v] == index[v]) {
                    uint32_t w;
                    do { w = stk[--sp]; on[w] = 0; comp[w] = ncomp; } while (w != v);
                    ++ncomp;
                }
            }
        }
    }
    free(index); free(low); free(on); free(stk); free(cs_v); free(cs_e);
    return (int64_t)ncomp;
}

/* --------------------------------------------- alpha / omega (Sec. 2.3) */

static int cmp_u64(const void *a, const void *b) {
    uint64_t x = *(const uint64_t *)a, y = *(const uint64_t *)b;
    return x < y ? -1 : x > y;
}

/* Section 2.3.  Build the weighted SCC DAG (w(C) = |C|; arc C->D iff some arc
 * of G goes from C to D), sort it topologically (Kahn), then visit the SCCs in
 * reverse topological order setting
 *     alpha(C) = w(C) + max over arcs (C,D) of alpha(D)
 *     omega(C) = w(C) + sum over arcs (C,D) of omega(D)
 * Omega is held at n: the sum counts an SCC once per DAG path to it and can
 * exceed the vertex count, which never bounds r(v) from below.  Per-vertex
 * outputs alpha[v] = alpha(C(v)), omega[v] = omega(C(v)); comp[v] as
 * oracle_scc.  Returns n_scc or -1. */
int64_t oracle_alpha_omega(uint32_t n, const uint64_t *row_ptr, const uint32_t *col,
                           uint32_t *comp, uint32_t *alpha, uint32_t *omega) {
    int64_t nc = oracle_scc(n, row_ptr, col, comp);
    if (nc < 0) return -1;
    uint64_t m = n ? row_ptr[n] : 0;
    uint64_t *arc = (uint64_t *)malloc(sizeof(uint64_t) * (m ? m : 1));
    uint64_t *w = (uint64_t *)calloc(nc ? nc : 1, sizeof(uint64_t));
    uint64_t *dptr = (uint64_t *)calloc((size_t)nc + 1, sizeof(uint64_t));
    uint32_t *indeg = (uint32_t *)calloc(nc ? nc : 1, sizeof(uint32_t));
    uint32_t *topo = (uint32_t *)malloc(sizeof(uint32_t) * (nc ? nc : 1));
    uint64_t *A = (uint64_t *)malloc(sizeof(uint64_t) * (nc ? nc : 1));
    uint64_t *W = (uint64_t *)malloc(sizeof(uint64_t) * (nc ? nc : 1));
    if (!arc || !w || !dptr || !indeg || !topo || !A || !W) {
        free(arc); free(w); free(dptr); free(indeg); free(topo); free(A); free(W); return -1;
    }
    for (uint32_t v = 0; v < n; ++v) w[comp[v]]++;
    uint64_t na = 0;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (comp[u] != comp[col[e]]) arc[na++] = ((uint64_t)comp[u] << 32) | comp[col[e]];
    qsort(arc, na, sizeof(uint64_t), cmp_u64);
    uint64_t nu = 0;                                    /* distinct DAG arcs */
    for (uint64_t i = 0; i < na; ++i) if (i == 0 || arc[i] != arc[i - 1]) arc[nu++] = arc[i];
    for (uint64_t i = 0; i < nu; ++i) { dptr[(arc[i] >> 32) + 1]++; indeg[arc[i] & 0xffffffffu]++; }
    for (int64_t c = 0; c < nc; ++c) dptr[c + 1] += dptr[c];
    /* Kahn: C_1..C_l with every DAG arc going forward */
    uint64_t qh = 0, qt = 0;
    for (int64_t c = 0; c < nc; ++c) if (indeg[c] == 0) topo[qt++] = (uint32_t)c;
    while (qh < qt) {
        uint32_t c = topo[qh++];
        for (uint64_t i = dptr[c]; i < dptr[c + 1]; ++i) {
            uint32_t d = (uint32_t)(arc[i] & 0xffffffffu);
            if (--indeg[d] == 0) topo[qt++] = d;
        }
    }
    /* reverse topological order: successors are final when C is visited */
    for (int64_t t = (int64_t)qt - 1; t >= 0; --t) {
        uint32_t c = topo[t];
        uint64_t amax = 0, osum = 0;
        for (uint64_t i = dptr[c]; i < dptr[c + 1]; ++i) {
            uint32_t d = (uint32_t)(arc[i] & 0xffffffffu);
            if (A[d] > amax) amax = A[d];
            osum += W[d];
            if (osum > n) osum = n;
        }
        A[c] = w[c] + amax;
        W[c] = w[c] + osum;
        if (W[c] > n) W[c] = n;
    }
    for (uint32_t v = 0; v < n; ++v) { alpha[v] = (uint32_t)A[comp[v]]; omega[v] = (uint32_t)W[comp[v]]; }
    free(arc); free(w); free(dptr); free(indeg); free(topo); free(A); free(W);
    return nc;
}

/* Section 2.3, second paragraph: the largest SCC C~ is not bounded by the
 * programme but measured, R~ = sum of w(D) over the SCCs D reachable from C~
 * (what one BFS from a vertex of C~ counts), so alpha(C~) = omega(C~) = R~,
 * and alpha improves for every SCC that reaches C~ through the max.  For
 * those SCCs omega is also taken from the programme run on the DAG without
 * the SCCs reachable from C~, plus R~; the smaller of that and the plain
 * omega is kept (both bound r from above).  C~ is the largest SCC, on ties
 * the one with the smallest vertex id.  Returns n_scc or -1. */
int64_t oracle_alpha_omega_refined(uint32_t n, const uint64_t *row_ptr, const uint32_t *col,
                                   uint32_t *comp, uint32_t *alpha, uint32_t *omega) {
    int64_t nc = oracle_scc(n, row_ptr, col, comp);
    if (nc < 0) return -1;
    if (nc == 0) return 0;
    uint64_t m = n ? row_ptr[n] : 0;
    uint64_t *arc = (uint64_t *)malloc(sizeof(uint64_t) * (m ? m : 1));
    uint64_t *w = (uint64_t *)calloc(nc, sizeof(uint64_t));
    uint32_t *minv = (uint32_t *)malloc(sizeof(uint32_t) * nc);
    uint64_t *dptr = (uint64_t *)calloc((size_t)nc + 1, sizeof(uint64_t));
    uint32_t *indeg = (uint32_t *)calloc(nc, sizeof(uint32_t));
    uint32_t *topo = (uint32_t *)malloc(sizeof(uint32_t) * nc);
    uint8_t *desc = (uint8_t *)calloc(nc, 1), *anc = (uint8_t *)calloc(nc, 1);
    uint64_t *A = (uint64_t *)malloc(sizeof(uint64_t) * nc), *Wf = (uint64_t *)malloc(sizeof(uint64_t) * nc);
    uint64_t *Wm = (uint64_t *)malloc(sizeof(uint64_t) * nc);
    if (!arc || !w || !minv || !dptr || !indeg || !topo || !desc || !anc || !A || !Wf || !Wm) {
        free(arc); free(w); free(minv); free(dptr); free(indeg); free(topo); free(desc); free(anc);
        free(A); free(Wf); free(Wm);
        return -1;
    }
    for (int64_t c = 0; c < nc; ++c) minv[c] = 0xffffffffu;
    for (uint32_t v = 0; v < n; ++v) { w[comp[v]]++; if (v < minv[comp[v]]) minv[comp[v]] = v; }
    uint64_t na = 0;
    for (uint32_t u = 0; u < n; ++u)
        for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (comp[u] != comp[col[e]]) arc[na++] = ((uint64_t)comp[u] << 32) | comp[col[e]];
    qsort(arc, na, sizeof(uint64_t), cmp_u64);
    uint64_t nu = 0;
    for (uint64_t i = 0; i < na; ++i) if (i == 0 || arc[i] != arc[i - 1]) arc[nu++] = arc[i];
    for (uint64_t i = 0; i < nu; ++i) { dptr[(arc[i] >> 32) + 1]++; indeg[arc[i] & 0xffffffffu]++; }
    for (int64_t c = 0; c < nc; ++c) dptr[c + 1] += dptr[c];
    uint64_t qh = 0, qt = 0;
    for (int64_t c = 0; c < nc; ++c) if (indeg[c] == 0) topo[qt++] = (uint32_t)c;
    while (qh < qt) {
        uint32_t c = topo[qh++];
        for (uint64_t i = dptr[c]; i < dptr[c + 1]; ++i) {
            uint32_t d = (uint32_t)(arc[i] & 0xffffffffu);
            if (--indeg[d] == 0) topo[qt++] = d;
        }
    }
    uint32_t big = 0;                       /* C~ */
    for (int64_t c = 1; c < nc; ++c)
        if (w[c] > w[big] || (w[c] == w[big] && minv[c] < minv[big])) big = (uint32_t)c;
    /* SCCs reachable from C~: in topological order, a successor of a marked SCC is marked */
    desc[big] = 1;
    for (uint64_t t = 0; t < qt; ++t) {
        uint32_t c = topo[t];
        if (!desc[c]) continue;
        for (uint64_t i = dptr[c]; i < dptr[c + 1]; ++i) desc[arc[i] & 0xffffffffu] = 1;
    }
    uint64_t R = 0;
    for (int64_t c = 0; c < nc; ++c) if (desc[c]) R += w[c];
    /* SCCs that reach C~: in reverse topological order, an SCC with a marked successor is marked */
    for (int64_t t = (int64_t)qt - 1; t >= 0; --t) {
        uint32_t c = topo[t];
        for (uint64_t i = dptr[c]; i < dptr[c + 1]; ++i) {
            uint32_t d = (uint32_t)(arc[i] & 0xffffffffu);
            if (d == big || anc[d]) anc[c] = 1;
        }
    }
    for (int64_t t = (int64_t)qt - 1; t >= 0; --t) {
        uint32_t c = topo[t];
        uint64_t amax = 0, fs = 0, ms = 0;
        for (uint64_t i = dptr[c]; i < dptr[c + 1]; ++i) {
            uint32_t d = (uint32_t)(arc[i] & 0xffffffffu);
            if (A[d] > amax) amax = A[d];
            fs += Wf[d]; if (fs > n) fs = n;
            if (!desc[d]) { ms += Wm[d]; if (ms > n) ms = n; }
        }
        if (c == big) { A[c] = R; Wf[c] = R; Wm[c] = 0; continue; }
        A[c] = w[c] + amax;
        Wf[c] = w[c] + fs; if (Wf[c] > n) Wf[c] = n;
        Wm[c] = desc[c] ? 0 : w[c] + ms; if (Wm[c] > n) Wm[c] = n;
        if (anc[c] && Wm[c] + R < Wf[c]) Wf[c] = Wm[c] + R;
    }
    for (uint32_t v = 0; v < n; ++v) { alpha[v] = (uint32_t)A[comp[v]]; omega[v] = (uint32_t)Wf[comp[v]]; }
    free(arc); free(w); free(minv); free(dptr); free(indeg); free(topo); free(desc); free(anc);
    free(A); free(Wf); free(Wm);
    return nc;
}

/* ------------------------------------------------- Lemma 1's bound */

/* f~_d(v, x) = f_d - g + (d+2)(x - n_d)   (Table 1; Lemma 1), where g is the
 * upper bound on gamma_{d+1} in use. */
static i128 lower_farness(uint64_t f_d, uint64_t g, uint32_t d, uint64_t x, uint64_t n_d) {
    return (i128)f_d - (i128)g + (i128)(d + 2) * ((i128)x - (i128)n_d);
}

/* Bound on gamma_{d+1} (Table 1): the sum over Gamma_d of deg(u) (outdeg on
 * digraphs).  mode 1 adds the footnote of Section 2.2 for undirected graphs:
 * for d >= 1 each u in Gamma_d spends one edge on Gamma_{d-1}, so deg(u)-1.
 * mode 2 is Algorithm 2's running sum over all of N_d. */
enum { GT_TABLE1 = 0, GT_FOOTNOTE = 1, GT_ALG2 = 2 };

/* Per-level BFS state shared by the bound trace and BFSCut. */
typedef struct {
    uint32_t *cur, *nxt;     /* Gamma_d and Gamma_{d+1} */
    uint32_t *seen; uint32_t epoch;
} lvl_ws;

static int lvl_init(lvl_ws *L, uint32_t n) {
    L->cur = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    L->nxt = (uint32_t *)malloc(sizeof(uint32_t) * (n ? n : 1));
    L->seen = (uint32_t *)calloc(n ? n : 1, sizeof(uint32_t));
    L->epoch = 0;
    return L->cur && L->nxt && L->seen;
}

static void lvl_free(lvl_ws *L) { free(L->cur); free(L->nxt); free(L->seen); }

static uint64_t gamma_tilde(const uint64_t *row_ptr, const uint32_t *lvl, uint32_t cnt,
                            uint32_t d, int mode) {
    uint64_t s = 0;
    for (uint32_t i = 0; i < cnt; ++i) {
        uint64_t deg = row_ptr[lvl[i] + 1] - row_ptr[lvl[i]];
        s += (mode == GT_FOOTNOTE && d >= 1 && deg > 0) ? deg - 1 : deg;
    }
    return s;
}

/* f~_d(v, x) for d = 0 .. ecc(v) into out[] (capacity cap).  Returns the
 * number of levels written, -1 on allocation failure, -2 if cap is short. */
int64_t oracle_bound_trace(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, uint32_t v,
                           int mode, uint64_t x, int64_t *out, uint64_t cap) {
    lvl_ws L;
    if (!lvl_init(&L, n)) { lvl_free(&L); return -1; }
    L.epoch = 1;
    uint32_t ncur = 1, d = 0;
    L.cur[0] = v; L.seen[v] = 1;
    uint64_t f = 0, nd = 1, g = 0;
    int64_t k = 0;
    for (;;) {
        uint64_t gl = gamma_tilde(row_ptr, L.cur, ncur, d, mode);
        g = (mode == GT_ALG2) ? g + gl : gl;
        if ((uint64_t)k >= cap) { lvl_free(&L); return -2; }
        out[k++] = (int64_t)lower_farness(f, g, d, x, nd);
        uint32_t nn = 0;
        for (uint32_t i = 0; i < ncur; ++i) {
            uint32_t u = L.cur[i];
            for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                uint32_t w = col[e];
                if (L.seen[w] != 1) { L.seen[w] = 1; L.nxt[nn++] = w; }
            }
        }
        if (nn == 0) break;
        ++d;
        nd += nn;
        f += (uint64_t)d * nn;
        uint32_t *t = L.cur; L.cur = L.nxt; L.nxt = t; ncur = nn;
    }
    lvl_free(&L);
    return k;
}

/* ------------------------------------------- BCM: Algorithms 1 and 2 */

typedef struct {
    uint64_t m_vis;       /* arcs scanned over all BFSCut calls (Section 3.1) */
    uint64_t completed;   /* BFSCut calls that returned the exact closeness */
    uint64_t cut;         /* BFSCut calls stopped by the bound */
    uint64_t max_level;
} bcm_oracle_stats;

typedef struct {
    uint32_t k, cnt;
    uint32_t *id; uint64_t *f; uint32_t *r;   /* rank order, best first */
} topk_buf;

/* x_k of Algorithm 1 as the rank key of the k-th entry; valid iff cnt == k */
static void topk_insert(topk_buf *T, uint32_t v, uint64_t f, uint32_t r) {
    uint64_t Nv, Fv; score_key(f, r, &Nv, &Fv);
    if (T->cnt == T->k) {
        uint64_t Nk, Fk; score_key(T->f[T->k - 1], T->r[T->k - 1], &Nk, &Fk);
        if (!ranks_before(Nv, Fv, v, Nk, Fk, T->id[T->k - 1])) return;
        T->cnt--;
    }
    uint32_t pos = T->cnt;
    while (pos > 0) {
        uint64_t Np, Fp; score_key(T->f[pos - 1], T->r[pos - 1], &Np, &Fp);
        if (!ranks_before(Nv, Fv, v, Np, Fp, T->id[pos - 1])) break;
        T->id[pos] = T->id[pos - 1]; T->f[pos] = T->f[pos - 1]; T->r[pos] = T->r[pos - 1];
        --pos;
    }
    T->id[pos] = v; T->f[pos] = f; T->r[pos] = r;
    T->cnt++;
}

/* The stopping rule of BFSCut at level d.  X holds r(v) (undirected) or
 * alpha(v), omega(v) (Lemma 2); the bound must hold at every x in X.  In the
 * ranking key, v cannot beat the k-th entry (Nk, Fk, idk) once
 *     f~_d(v,x) * Nk >  Fk * (x-1)^2   for all x   (v ranks strictly lower), or
 *     f~_d(v,x) * Nk >= Fk * (x-1)^2   for all x and v > idk (ties go to smaller ids). */
static int bfscut_stops(uint64_t f_d, uint64_t g, uint32_t d, uint64_t n_d,
                        const uint64_t *X, int nx, uint32_t v,
                        uint64_t Nk, uint64_t Fk, uint32_t idk) {
    int all_strict = 1, all_weak = 1;
    for (int i = 0; i < nx; ++i) {
        i128 ft = lower_farness(f_d, g, d, X[i], n_d);
        i128 lhs = ft * (i128)Nk;
        i128 xm1 = (i128)X[i] - 1;
        i128 rhs = (i128)Fk * xm1 * xm1;
        if (!(lhs > rhs)) all_strict = 0;
        if (!(lhs >= rhs)) all_weak = 0;
    }
    return all_strict || (all_weak && v > idk);
}

/* Algorithm 1's loop over sources[from..to): BFSCut(v, x_k) for each v in
 * turn, the exact ones kept in T (the best k, rank order).  x_k is T's own
 * k-th entry once T holds k, or -- when ext != 0 -- the outside key (eN, eF,
 * eid) if that ranks first: the k-th entry of another shard of the same
 * graph (Section 2's shared x_k), valid because at least k vertices of the
 * graph rank at or before it.  X of v: xa[v], xb[v] (r(v) twice, or
 * alpha(v), omega(v)).  S accumulates the counters. */
static void bcm_loop(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, int gamma_mode, int early_test,
                     const uint32_t *xa, const uint32_t *xb, const uint32_t *sources, uint64_t from, uint64_t to,
                     int ext, uint64_t eN, uint64_t eF, uint32_t eid, topk_buf *T, lvl_ws *L,
                     bcm_oracle_stats *S) {
    for (uint64_t it = from; it < to; ++it) {
        uint32_t v = sources[it];
        uint64_t X[2] = { xa[v], xb[v] };
        int nx = (X[0] == X[1]) ? 1 : 2;
        int have_xk = (T->cnt == T->k);
        uint64_t Nk = 0, Fk = 1; uint32_t idk = 0;
        if (have_xk) { score_key(T->f[T->k - 1], T->r[T->k - 1], &Nk, &Fk); idk = T->id[T->k - 1]; }
        if (ext && (!have_xk || ranks_before(eN, eF, eid, Nk, Fk, idk))) { Nk = eN; Fk = eF; idk = eid; have_xk = 1; }

        /* BFSCut(v, x_k), level by level: Gamma_d in L->cur */
        if (++L->epoch == 0) { memset(L->seen, 0, sizeof(uint32_t) * n); L->epoch = 1; }
        uint32_t ncur = 1, d = 0;
        L->cur[0] = v; L->seen[v] = L->epoch;
        uint64_t f = 0, nd = 1, g = 0;
        int stopped = 0;
        for (;;) {
            uint64_t gl = gamma_tilde(row_ptr, L->cur, ncur, d, gamma_mode);
            g = (gamma_mode == GT_ALG2) ? g + gl : gl;
            if (early_test && have_xk && bfscut_stops(f, g, d, nd, X, nx, v, Nk, Fk, idk)) {
                stopped = 1; break;
            }
            uint32_t nn = 0;
            for (uint32_t i = 0; i < ncur; ++i) {
                uint32_t u = L->cur[i];
                for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
                    uint32_t w = col[e];
                    if (L->seen[w] != L->epoch) { L->seen[w] = L->epoch; L->nxt[nn++] = w; }
                }
                S->m_vis += row_ptr[u + 1] - row_ptr[u];
            }
            if (nn == 0) break;
            if (!early_test && have_xk && bfscut_stops(f, g, d, nd, X, nx, v, Nk, Fk, idk)) {
                stopped = 1; break;
            }
            ++d;
            nd += nn;
            f += (uint64_t)d * nn;
            uint32_t *t = L->cur; L->cur = L->nxt; L->nxt = t; ncur = nn;
        }
        if (d > S->max_level) S->max_level = d;
        if (stopped) { S->cut++; continue; }
        S->completed++;
        topk_insert(T, v, f, (uint32_t)nd);
    }
}

static int cmp_order(const void *pa, const void *pb, void *pc) {
    const uint64_t *rp = (const uint64_t *)pc;
    uint32_t a = *(const uint32_t *)pa, b = *(const uint32_t *)pb;
    uint64_t da = rp[a + 1] - rp[a], db = rp[b + 1] - rp[b];
    if (da != db) return da > db ? -1 : 1;
    return a < b ? -1 : (a > b);
}

/* Algorithm 1's processing order: decreasing degree (outdeg on digraphs),
 * equal degrees by increasing id. */
void oracle_order(uint32_t n, const uint64_t *row_ptr, uint32_t *order) {
    for (uint32_t v = 0; v < n; ++v) order[v] = v;
    qsort_r(order, n, sizeof(uint32_t), cmp_order, (void *)row_ptr);
}

/* Algorithm 1: preprocessing, vertices in decreasing order of degree
 * (outdeg on digraphs; equal degrees by increasing id), BFSCut(v, x_k) each,
 * the k-th best kept in a size-k rank-ordered buffer.
 *   gamma_mode: GT_TABLE1, GT_FOOTNOTE (undirected only) or GT_ALG2.
 *   early_test: 0 = Algorithm 2's schedule (level d is tested after the arcs
 *               of Gamma_d are scanned, when Gamma_{d+1} is non-empty);
 *               1 = the same bound tested before those arcs are scanned.
 * Writes min(k, n) entries to ids/f/r in rank order; returns their count or
 * a negative value on failure. */
int64_t oracle_bcm2(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, int directed,
                    uint32_t k, int gamma_mode, int early_test, int refined,
                    uint32_t *ids, uint64_t *f_out, uint32_t *r_out, bcm_oracle_stats *st);

int64_t oracle_bcm(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, int directed,
                   uint32_t k, int gamma_mode, int early_test,
                   uint32_t *ids, uint64_t *f_out, uint32_t *r_out, bcm_oracle_stats *st) {
    return oracle_bcm2(n, row_ptr, col, directed, k, gamma_mode, early_test, 0, ids, f_out, r_out, st);
}

/* As oracle_bcm; refined != 0 takes alpha/omega from the biggest-SCC
 * refinement on digraphs. */
int64_t oracle_bcm2(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, int directed,
                    uint32_t k, int gamma_mode, int early_test, int refined,
                    uint32_t *ids, uint64_t *f_out, uint32_t *r_out, bcm_oracle_stats *st) {
    if (k == 0 || n == 0) { if (st) memset(st, 0, sizeof(*st)); return 0; }
    if (gamma_mode == GT_FOOTNOTE && directed) gamma_mode = GT_TABLE1;
    uint32_t *xa = (uint32_t *)malloc(sizeof(uint32_t) * n);
    uint32_t *xb = (uint32_t *)malloc(sizeof(uint32_t) * n);
    uint32_t *order = (uint32_t *)malloc(sizeof(uint32_t) * n);
    uint32_t kk = k < n ? k : n;
    topk_buf T = { kk, 0, (uint32_t *)malloc(sizeof(uint32_t) * kk),
                   (uint64_t *)malloc(sizeof(uint64_t) * kk), (uint32_t *)malloc(sizeof(uint32_t) * kk) };
    lvl_ws L;
    int ok = xa && xb && order && T.id && T.f && T.r && lvl_init(&L, n);
    if (!ok) { free(xa); free(xb); free(order); free(T.id); free(T.f); free(T.r); return -1; }

    /* PreProcessing: r(v) from connected components (Section 2.2) or the
     * alpha/omega bounds (Section 2.3). */
    if (!directed) {
        uint32_t *lab = xb;
        uint32_t *size = (uint32_t *)calloc(n, sizeof(uint32_t));
        if (!size) { ok = 0; goto done; }
        for (uint32_t v = 0; v < n; ++v) lab[v] = 0xffffffffu;
        for (uint32_t s = 0; s < n; ++s) {
            if (lab[s] != 0xffffffffu) continue;
            uint32_t h = 0, t = 0;
            L.cur[t++] = s; lab[s] = s;
            while (h < t) {
                uint32_t u = L.cur[h++];
                for (uint64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
                    if (lab[col[e]] == 0xffffffffu) { lab[col[e]] = s; L.cur[t++] = col[e]; }
            }
            size[s] = t;
        }
        for (uint32_t v = 0; v < n; ++v) xa[v] = size[lab[v]];
        memcpy(xb, xa, sizeof(uint32_t) * n);
        free(size);
    } else {
        uint32_t *comp = (uint32_t *)malloc(sizeof(uint32_t) * n);
        if (!comp || (refined ? oracle_alpha_omega_refined(n, row_ptr, col, comp, xa, xb)
                              : oracle_alpha_omega(n, row_ptr, col, comp, xa, xb)) < 0) {
            free(comp); ok = 0; goto done;
        }
        free(comp);
    }

    for (uint32_t v = 0; v < n; ++v) order[v] = v;
    qsort_r(order, n, sizeof(uint32_t), cmp_order, (void *)row_ptr);

    bcm_oracle_stats S = { 0, 0, 0, 0 };
    bcm_loop(n, row_ptr, col, gamma_mode, early_test, xa, xb, order, 0, n, 0, 0, 1, 0, &T, &L, &S);
    for (uint32_t i = 0; i < T.cnt; ++i) { ids[i] = T.id[i]; f_out[i] = T.f[i]; r_out[i] = T.r[i]; }
    if (st) *st = S;
done:
    lvl_free(&L);
    free(xa); free(xb); free(order);
    int64_t ret = ok ? (int64_t)T.cnt : -1;
    free(T.id); free(T.f); free(T.r);
    return ret;
}

/* Algorithm 1 over the sources of one shard, resumable (the threshold
 * exchange of Section 2's parallel version, run between calls).  The caller
 * gives the preprocessing results xa, xb (r(v), or alpha(v) and omega(v)),
 * the shard's sources in processing order, and the range [from, to) to run
 * now; ids/f/r/count (capacity k) carry the shard's top-k from call to call
 * (count = 0 before the first).  ext_valid != 0 offers the outside key
 * (ext_N, ext_F, ext_id).  st accumulates.  Returns the entries held, or -1
 * on allocation failure. */
int64_t oracle_bcm_sources(uint32_t n, const uint64_t *row_ptr, const uint32_t *col, int directed, uint32_t k,
                           int gamma_mode, const uint32_t *xa, const uint32_t *xb, const uint32_t *sources,
                           uint64_t from, uint64_t to, int ext_valid, uint64_t ext_N, uint64_t ext_F,
                           uint32_t ext_id, uint32_t *ids, uint64_t *f, uint32_t *r, uint32_t *count,
                           bcm_oracle_stats *st) {
    if (k == 0) return 0;
    if (gamma_mode == GT_FOOTNOTE && directed) gamma_mode = GT_TABLE1;
    lvl_ws L;
    if (!lvl_init(&L, n)) { lvl_free(&L); return -1; }
    topk_buf T = { k, *count, ids, f, r };
    bcm_loop(n, row_ptr, col, gamma_mode, 1, xa, xb, sources, from, to, ext_valid, ext_N, ext_F, ext_id, &T, &L,
             st);
    lvl_free(&L);
    *count = T.cnt;
    return (int64_t)T.cnt;
}
