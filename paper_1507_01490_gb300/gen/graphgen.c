/*
 * Seeded synthetic graph generators.
 *
 * This file builds inputs only: it holds no closeness, BFS or bound
 * arithmetic.  Both the CUDA library's tests and the CPU oracle's tests
 * receive the arrays produced here.
 *
 * Random numbers: splitmix64 (to expand a 64-bit seed) feeding xoshiro256**
 * (Blackman and Vigna, "Scrambled linear pseudorandom number generators",
 * 2018), written from the published definitions.  Everything is integer
 * arithmetic or IEEE-754 +,-,*,/ with contraction disabled, so the same seed
 * gives the same graph on x86-64 and AArch64.
 *
 * Outputs are edge lists (src, dst) in caller-provided buffers; gen_csr at
 * the end turns an edge list into CSR (mirroring, self-loop and duplicate
 * removal, sorted rows).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>

/* ---------------------------------------------------------------- PRNG */
typedef struct { uint64_t s[4]; } rng_t;

static uint64_t splitmix64_next(uint64_t *x) {
    uint64_t z = (*x += 0x9e3779b97f4a7c15ULL);
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

static inline uint64_t rotl64(uint64_t x, int k) { return (x << k) | (x >> (64 - k)); }

static void rng_seed(rng_t *r, uint64_t seed) {
    uint64_t x = seed;
    for (int i = 0; i < 4; ++i) r->s[i] = splitmix64_next(&x);
}

static inline uint64_t rng_next(rng_t *r) {
    uint64_t *s = r->s;
    const uint64_t out = rotl64(s[1] * 5, 7) * 9;
    const uint64_t t = s[1] << 17;
    s[2] ^= s[0];
    s[3] ^= s[1];
    s[1] ^= s[2];
    s[0] ^= s[3];
    s[2] ^= t;
    s[3] = rotl64(s[3], 45);
    return out;
}

/* uniform integer in [0, bound) by the multiply-high map */
static inline uint64_t rng_below(rng_t *r, uint64_t bound) {
    return (uint64_t)(((unsigned __int128)rng_next(r) * bound) >> 64);
}

/* uniform double in (0, 1) */
static inline double rng_open01(rng_t *r) {
    return ((double)(rng_next(r) >> 11) + 0.5) * (1.0 / 9007199254740992.0);
}

/* ------------------------------------------- portable log / exp (host) */
/* Series evaluations with exact range reduction (frexp/ldexp/floor), so the
 * result depends only on IEEE basic operations.  Accuracy is ~1e-15 relative,
 * far beyond what a degree-weight recipe needs; the point is reproducibility. */
static const double LN2 = 0.69314718055994530942;

static double gen_log(double x) {
    int e;
    double m = frexp(x, &e);                 /* x = m * 2^e, m in [0.5, 1) */
    if (m < 0.70710678118654752440) { m *= 2.0; e -= 1; }
    double z = (m - 1.0) / (m + 1.0), z2 = z * z, term = z, sum = 0.0;
    for (int k = 0; k < 40; ++k) { sum += term / (double)(2 * k + 1); term *= z2; }
    return 2.0 * sum + (double)e * LN2;
}

static double gen_exp(double x) {
    double kf = floor(x / LN2 + 0.5);
    double r = x - kf * LN2;
    double sum = 1.0, term = 1.0;
    for (int i = 1; i < 30; ++i) { term *= r / (double)i; sum += term; }
    return ldexp(sum, (int)kf);
}

/* ------------------------------------------------- Barabasi-Albert */
/* Start from the complete graph on m+1 nodes; node t = m+1..n-1 attaches to m
 * distinct existing nodes, each drawn with probability proportional to its
 * degree (uniform position in the endpoint list), duplicates redrawn.
 * Edge count: m(m+1)/2 + m(n-m-1).  Returns the number of edges written. */
int64_t gen_ba(uint32_t n, uint32_t m, uint64_t seed, uint32_t *src, uint32_t *dst) {
    if (m < 1 || n < m + 1) return -1;
    rng_t r; rng_seed(&r, seed);
    uint64_t m0 = m + 1;
    uint64_t ne_max = m0 * (m0 - 1) / 2 + (uint64_t)m * (n - m0);
    uint32_t *ends = (uint32_t *)malloc(sizeof(uint32_t) * 2 * ne_max);
    uint32_t *pick = (uint32_t *)malloc(sizeof(uint32_t) * m);
    if (!ends || !pick) { free(ends); free(pick); return -2; }
    uint64_t ne = 0, nends = 0;
    for (uint32_t a = 0; a < m0; ++a)
        for (uint32_t b = a + 1; b < m0; ++b) {
            src[ne] = a; dst[ne] = b; ++ne;
            ends[nends++] = a; ends[nends++] = b;
        }
    for (uint32_t t = (uint32_t)m0; t < n; ++t) {
        uint32_t got = 0;
        while (got < m) {
            uint32_t c = ends[rng_below(&r, nends)];
            int dup = 0;
            for (uint32_t i = 0; i < got; ++i) if (pick[i] == c) { dup = 1; break; }
            if (!dup) pick[got++] = c;
        }
        for (uint32_t i = 0; i < m; ++i) {
            src[ne] = t; dst[ne] = pick[i]; ++ne;
            ends[nends++] = t; ends[nends++] = pick[i];
        }
    }
    free(ends); free(pick);
    return (int64_t)ne;
}

/* ------------------------------------------------------ Chung-Lu */
/* Expected-degree model with power-law weights: w_i = U^(-1/(gamma-1))
 * (Pareto, x_min = 1, so the degree distribution has exponent gamma), scaled
 * to the requested mean, capped at sqrt(n * mean), quantised to integers.
 * n_draw edges are drawn with both endpoints proportional to w; self-loops
 * and repeats are left for the CSR builder to drop.  Returns n_draw. */
int64_t gen_chung_lu(uint32_t n, double mean_deg, double gamma, uint64_t n_draw,
                     uint64_t seed, uint32_t *src, uint32_t *dst) {
    if (n < 2 || gamma <= 1.0 || mean_deg <= 0.0) return -1;
    rng_t r; rng_seed(&r, seed);
    double *w = (double *)malloc(sizeof(double) * n);
    uint64_t *cum = (uint64_t *)malloc(sizeof(uint64_t) * n);
    if (!w || !cum) { free(w); free(cum); return -2; }
    double inv_shape = 1.0 / (gamma - 1.0), total = 0.0;
    for (uint32_t i = 0; i < n; ++i) {
        w[i] = gen_exp(-gen_log(rng_open01(&r)) * inv_shape);
        total += w[i];
    }
    double scale = mean_deg * (double)n / total;
    double cap = sqrt(mean_deg * (double)n);
    uint64_t acc = 0;
    for (uint32_t i = 0; i < n; ++i) {
        double x = w[i] * scale;
        if (x > cap) x = cap;
        uint64_t q = (uint64_t)(x * 1048576.0) + 1;   /* weight in 2^-20 units, never zero */
        acc += q;
        cum[i] = acc;
    }
    for (uint64_t e = 0; e < n_draw; ++e) {
        for (int side = 0; side < 2; ++side) {
            uint64_t t = rng_below(&r, acc);
            uint32_t lo = 0, hi = n - 1;              /* first i with cum[i] > t */
            while (lo < hi) {
                uint32_t mid = lo + (hi - lo) / 2;
                if (cum[mid] > t) hi = mid; else lo = mid + 1;
            }
            if (side == 0) src[e] = lo; else dst[e] = lo;
        }
    }
    free(w); free(cum);
    return (int64_t)n_draw;
}

/* ---------------------------------------------------------- R-MAT */
/* Recursive-matrix arcs (Chakrabarti, Zhan, Faloutsos 2004): for each of
 * `scale` bit positions pick a quadrant with probabilities (a, b, c, d), given
 * as 32-bit thresholds ta < tab < tabc.  Vertices are then relabelled by a
 * seeded Fisher-Yates permutation.  Returns the number of arcs (n_arcs). */
int64_t gen_rmat(uint32_t scale, uint64_t n_arcs, uint32_t ta, uint32_t tab, uint32_t tabc,
                 uint64_t seed, uint32_t *src, uint32_t *dst) {
    if (scale < 1 || scale > 31) return -1;
    rng_t r; rng_seed(&r, seed);
    uint32_t n = 1u << scale;
    for (uint64_t e = 0; e < n_arcs; ++e) {
        uint32_t u = 0, v = 0;
        for (uint32_t bit = 0; bit < scale; bit += 2) {
            uint64_t x = rng_next(&r);
            for (int h = 0; h < 2 && bit + (uint32_t)h < scale; ++h) {
                uint32_t q = (uint32_t)(x >> (32 * h));
                uint32_t pos = scale - 1 - (bit + (uint32_t)h);
                if (q < ta) { }
                else if (q < tab) v |= 1u << pos;
                else if (q < tabc) u |= 1u << pos;
                else { u |= 1u << pos; v |= 1u << pos; }
            }
        }
        src[e] = u; dst[e] = v;
    }
    uint32_t *perm = (uint32_t *)malloc(sizeof(uint32_t) * n);
    if (!perm) return -2;
    for (uint32_t i = 0; i < n; ++i) perm[i] = i;
    for (uint32_t i = n - 1; i > 0; --i) {
        uint32_t j = (uint32_t)rng_below(&r, (uint64_t)i + 1);
        uint32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
    }
    for (uint64_t e = 0; e < n_arcs; ++e) { src[e] = perm[src[e]]; dst[e] = perm[dst[e]]; }
    free(perm);
    return (int64_t)n_arcs;
}

/* -------------------------------------------------- damaged grid */
static uint32_t uf_find(uint32_t *p, uint32_t x) {
    while (p[x] != x) { p[x] = p[p[x]]; x = p[x]; }
    return x;
}

/* rows x cols 4-neighbour grid (vertex id = row*cols + col); exactly n_del of
 * its edges are deleted, chosen by a seeded partial Fisher-Yates shuffle of the
 * edge indices (horizontal edges first, then vertical).  The largest connected
 * component is kept (ties: the one holding the smallest vertex id) and
 * relabelled in ascending original id.  Writes the kept edges and returns their
 * count; *n_out receives the component's size. */
int64_t gen_grid_lcc(uint32_t rows, uint32_t cols, uint64_t n_del, uint64_t seed,
                     uint32_t *src, uint32_t *dst, uint32_t *n_out) {
    if (rows < 1 || cols < 1) return -1;
    uint64_t nh = (uint64_t)rows * (cols - 1), nv = (uint64_t)(rows - 1) * cols;
    uint64_t ne = nh + nv;
    if (n_del > ne) return -1;
    uint64_t nvtx = (uint64_t)rows * cols;
    rng_t r; rng_seed(&r, seed);
    uint32_t *idx = (uint32_t *)malloc(sizeof(uint32_t) * ne);
    uint8_t *dead = (uint8_t *)calloc(ne, 1);
    uint32_t *par = (uint32_t *)malloc(sizeof(uint32_t) * nvtx);
    uint32_t *cnt = (uint32_t *)calloc(nvtx, sizeof(uint32_t));
    uint32_t *lab = (uint32_t *)malloc(sizeof(uint32_t) * nvtx);
    if (!idx || !dead || !par || !cnt || !lab) {
        free(idx); free(dead); free(par); free(cnt); free(lab); return -2;
    }
    for (uint64_t i = 0; i < ne; ++i) idx[i] = (uint32_t)i;
    for (uint64_t t = 0; t < n_del; ++t) {
        uint64_t s = t + rng_below(&r, ne - t);
        uint32_t tmp = idx[t]; idx[t] = idx[s]; idx[s] = tmp;
        dead[idx[t]] = 1;
    }
    for (uint64_t v = 0; v < nvtx; ++v) par[v] = (uint32_t)v;
    #define GRID_EDGE(e, a, b) do { \
        if ((e) < nh) { uint64_t rr = (e) / (cols - 1), cc = (e) % (cols - 1); \
                        a = (uint32_t)(rr * cols + cc); b = a + 1; } \
        else { uint64_t f = (e) - nh; a = (uint32_t)f; b = (uint32_t)(f + cols); } } while (0)
    for (uint64_t e = 0; e < ne; ++e) {
        if (dead[e]) continue;
        uint32_t a, b; GRID_EDGE(e, a, b);
        uint32_t ra = uf_find(par, a), rb = uf_find(par, b);
        if (ra != rb) { if (ra < rb) par[rb] = ra; else par[ra] = rb; }
    }
    uint32_t best = 0; uint32_t best_cnt = 0;
    for (uint64_t v = 0; v < nvtx; ++v) cnt[uf_find(par, (uint32_t)v)]++;
    for (uint64_t v = 0; v < nvtx; ++v)
        if (cnt[v] > best_cnt) { best_cnt = cnt[v]; best = (uint32_t)v; }
    uint32_t next = 0;
    for (uint64_t v = 0; v < nvtx; ++v)
        lab[v] = (uf_find(par, (uint32_t)v) == best) ? next++ : 0xffffffffu;
    uint64_t k = 0;
    for (uint64_t e = 0; e < ne; ++e) {
        if (dead[e]) continue;
        uint32_t a, b; GRID_EDGE(e, a, b);
        if (lab[a] == 0xffffffffu) continue;
        src[k] = lab[a]; dst[k] = lab[b]; ++k;
    }
    #undef GRID_EDGE
    *n_out = next;
    free(idx); free(dead); free(par); free(cnt); free(lab);
    return (int64_t)k;
}

/* --------------------------------------------------- random G(n,p) */
/* Each ordered (directed) or unordered (undirected) pair independently with
 * probability p_num / 2^32; self-pairs excluded.  Returns the count written,
 * or -3 if more than cap pairs were drawn. */
int64_t gen_gnp(uint32_t n, uint32_t p_num, int directed, uint64_t seed, uint64_t cap,
                uint32_t *src, uint32_t *dst) {
    rng_t r; rng_seed(&r, seed);
    uint64_t k = 0;
    for (uint32_t a = 0; a < n; ++a)
        for (uint32_t b = directed ? 0 : a + 1; b < n; ++b) {
            if (a == b) continue;
            if ((uint32_t)(rng_next(&r) >> 32) < p_num) {
                if (k >= cap) return -3;
                src[k] = a; dst[k] = b; ++k;
            }
        }
    return (int64_t)k;
}

/* uniform integers in [0, bound), used for seeded sampling in tests/bench */
void gen_uniform_u32(uint64_t seed, uint64_t count, uint32_t bound, uint32_t *out) {
    rng_t r; rng_seed(&r, seed);
    for (uint64_t i = 0; i < count; ++i) out[i] = (uint32_t)rng_below(&r, bound);
}

/* exponential inter-arrival gaps with the given mean (for request streams) */
void gen_exponential(uint64_t seed, uint64_t count, double mean, double *out) {
    rng_t r; rng_seed(&r, seed);
    for (uint64_t i = 0; i < count; ++i) out[i] = -gen_log(rng_open01(&r)) * mean;
}

/* ------------------------------------------------------------ CSR build */
static int cmp_u32(const void *a, const void *b) {
    uint32_t x = *(const uint32_t *)a, y = *(const uint32_t *)b;
    return (x > y) - (x < y);
}

/* CSR from k arcs (src[i], dst[i]): undirected lists are mirrored first,
 * self-loops dropped if drop_loops, rows sorted ascending, repeats removed if
 * dedup.  row_ptr has n+1 entries; col must hold k arcs (2k if undirected).
 * Returns the arc count written, or -1 if a working array cannot be
 * allocated or an endpoint is >= n. */
int64_t gen_csr(uint32_t n, const uint32_t *src, const uint32_t *dst, uint64_t k, int undirected,
                int drop_loops, int dedup, uint64_t *row_ptr, uint32_t *col) {
    memset(row_ptr, 0, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < k; ++i) {
        uint32_t s = src[i], d = dst[i];
        if (s >= n || d >= n) return -1;
        if (drop_loops && s == d) continue;
        row_ptr[s + 1]++;
        if (undirected) row_ptr[d + 1]++;
    }
    for (uint32_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
    uint64_t *pos = (uint64_t *)malloc(((size_t)n + 1) * sizeof(uint64_t));
    if (!pos) return -1;
    memcpy(pos, row_ptr, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t i = 0; i < k; ++i) {
        uint32_t s = src[i], d = dst[i];
        if (drop_loops && s == d) continue;
        col[pos[s]++] = d;
        if (undirected) col[pos[d]++] = s;
    }
    free(pos);
    /* sort each row, drop repeats, compact in place (the write cursor never
     * passes the row being read) */
    uint64_t w = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint64_t b = row_ptr[v], e = row_ptr[v + 1];
        uint64_t len = e - b;
        uint32_t *r = col + b;
        if (len > 32) {
            qsort(r, len, sizeof(uint32_t), cmp_u32);
        } else {
            for (uint64_t i = 1; i < len; ++i) {
                uint32_t x = r[i];
                uint64_t j = i;
                while (j > 0 && r[j - 1] > x) { r[j] = r[j - 1]; --j; }
                r[j] = x;
            }
        }
        row_ptr[v] = w;
        for (uint64_t i = 0; i < len; ++i) {
            if (dedup && i > 0 && r[i] == r[i - 1]) continue;
            col[w++] = r[i];
        }
    }
    row_ptr[n] = w;
    return (int64_t)w;
}
