/*
 * tcgen.c -- seeded synthetic graph generators (input data only).
 *
 * This module produces the undirected simple graphs that both the CUDA path
 * and the CPU oracle consume.  It holds none of the triangle-counting method:
 * no degree ordering, orientation, intersection or counting.  Its only graph
 * processing is turning a raw pair list into a simple undirected CSR (drop
 * self-loops, symmetrise, sort, de-duplicate), which is how the paper's
 * datasets were prepared (Table 1 caption: edges counted in both directions
 * after de-duplication).
 *
 * Randomness: one counter-based stream per (tag, seed), SplitMix64 (Steele,
 * Lea, Flood, "Fast splittable pseudorandom number generators", OOPSLA 2014):
 * value i of a stream with key K is mix64(K + (i+1) * 0x9E3779B97F4A7C15).
 * Every draw is addressed by its counter, so parallel and serial generation
 * give the same graph.
 *
 * Generators (workload recipes):
 *   ER    G(n, m): m distinct non-loop unordered pairs, uniform.
 *   RMAT  scale s, edge factor ef, quadrant probabilities (a, b, c, d):
 *         ef * 2^s pairs, one quadrant draw per level, no noise, then a
 *         seeded uniform relabelling of the 2^s ids.
 *   GRID  R x C lattice, one diagonal (i,j)-(i+1,j+1) per cell with
 *         probability p, plus round(frac * (lattice + diagonal edges))
 *         uniform random pairs.
 *   BA    Barabasi-Albert: seed clique K_{k+1}; each new vertex picks k
 *         distinct targets with probability proportional to degree (uniform
 *         pick from the list of edge endpoints, repeats rejected).
 *   BA batch: graph i draws n_i ~ U{n_lo..n_hi}, k_i ~ U{k_lo..k_hi} from
 *         its own stream and is then BA(n_i, k_i, seed i); the graphs are
 *         concatenated (int64 vertex and entry offsets, local vertex ids).
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define GOLDEN 0x9E3779B97F4A7C15ULL

static inline uint64_t mix64(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ULL;
    z = (z ^ (z >> 27)) * 0x94D049BB133111EBULL;
    return z ^ (z >> 31);
}
static inline uint64_t rng_at(uint64_t key, uint64_t i) { return mix64(key + (i + 1) * GOLDEN); }
static inline double u01(uint64_t x) { return (double)(x >> 11) * (1.0 / 9007199254740992.0); }
/* uniform integer in [0, r) by multiply-high (Lemire 2019) */
static inline uint64_t below(uint64_t x, uint64_t r) { return (uint64_t)(((unsigned __int128)x * r) >> 64); }
static uint64_t stream_key(uint64_t tag, uint64_t seed) {
    return mix64(mix64(tag * GOLDEN + 0x632BE59BD9B4E019ULL) ^ mix64(seed + 0x2545F4914F6CDD1DULL));
}

enum { TAG_ER = 0x4552, TAG_RMAT = 0x524D, TAG_PERM = 0x5045, TAG_GRID = 0x4744,
       TAG_LONG = 0x4C52, TAG_BA = 0x4241, TAG_BATCH = 0x4242 };

typedef struct tcg_graph {
    int64_t n, nnz;          /* vertices; CSR entries (2m) */
    int64_t* row_ptr;        /* n+1 */
    int32_t* col;            /* nnz, ascending within a row */
    int64_t npairs;          /* raw pairs before canonicalisation */
    int32_t* src; int32_t* dst;
    int64_t G;               /* >0 for a batch */
    int64_t* vtx_off;        /* G+1 */
    int64_t* edge_off;       /* G+1 */
} tcg_graph;

static tcg_graph* alloc_graph(void) { return (tcg_graph*)calloc(1, sizeof(tcg_graph)); }

/* ---- raw pairs -> simple undirected CSR (input preparation) ---------------- */
/* Two stable counting sorts of the directed pair keys (by v, then by u) give
 * (u, v) order; equal neighbours are then adjacent and dropped. */
static int pairs_to_csr(int64_t n, int64_t np, const int32_t* s, const int32_t* d,
                        int64_t** row_ptr_out, int32_t** col_out, int64_t* nnz_out) {
    int64_t cnt = 0;
    for (int64_t i = 0; i < np; ++i) if (s[i] != d[i]) cnt += 2;
    uint64_t* a = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(cnt ? cnt : 1));
    uint64_t* b = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(cnt ? cnt : 1));
    int64_t* bucket = (int64_t*)malloc(sizeof(int64_t) * (size_t)(n + 1));
    if (!a || !b || !bucket) { free(a); free(b); free(bucket); return -1; }
    int64_t k = 0;
    for (int64_t i = 0; i < np; ++i) {
        uint32_t u = (uint32_t)s[i], v = (uint32_t)d[i];
        if (u == v) continue;
        a[k++] = ((uint64_t)u << 32) | v;
        a[k++] = ((uint64_t)v << 32) | u;
    }
    for (int pass = 0; pass < 2; ++pass) {
        int sh = pass == 0 ? 0 : 32;
        memset(bucket, 0, sizeof(int64_t) * (size_t)(n + 1));
        for (int64_t i = 0; i < cnt; ++i) bucket[((a[i] >> sh) & 0xffffffffULL)]++;
        int64_t run = 0;
        for (int64_t v = 0; v < n; ++v) { int64_t c = bucket[v]; bucket[v] = run; run += c; }
        for (int64_t i = 0; i < cnt; ++i) b[bucket[(a[i] >> sh) & 0xffffffffULL]++] = a[i];
        uint64_t* t = a; a = b; b = t;
    }
    free(b);
    int64_t* rp = (int64_t*)calloc((size_t)(n + 1), sizeof(int64_t));
    int64_t u_nnz = 0;
    for (int64_t i = 0; i < cnt; ++i) if (i == 0 || a[i] != a[i - 1]) ++u_nnz;
    int32_t* col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(u_nnz ? u_nnz : 1));
    if (!rp || !col) { free(a); free(bucket); free(rp); free(col); return -1; }
    int64_t j = 0;
    for (int64_t i = 0; i < cnt; ++i) {
        if (i > 0 && a[i] == a[i - 1]) continue;
        rp[(a[i] >> 32) + 1]++;
        col[j++] = (int32_t)(a[i] & 0xffffffffULL);
    }
    for (int64_t v = 0; v < n; ++v) rp[v + 1] += rp[v];
    free(a); free(bucket);
    *row_ptr_out = rp; *col_out = col; *nnz_out = u_nnz;
    return 0;
}

static tcg_graph* finish(tcg_graph* g, int64_t n, int64_t np, int32_t* s, int32_t* d, int keep_pairs) {
    g->n = n; g->npairs = np;
    if (pairs_to_csr(n, np, s, d, &g->row_ptr, &g->col, &g->nnz) != 0) {
        free(s); free(d); free(g); return NULL;
    }
    if (keep_pairs) { g->src = s; g->dst = d; } else { free(s); free(d); }
    return g;
}

/* ---- Erdos-Renyi G(n, m) ------------------------------------------------- */
tcg_graph* tcg_er(int64_t n, int64_t m, uint64_t seed, int keep_pairs) {
    if (n < 2 || m < 0 || m > n * (n - 1) / 2) return NULL;
    uint64_t key = stream_key(TAG_ER, seed);
    int64_t cap = 1; while (cap < 4 * m + 16) cap <<= 1;
    uint64_t* set = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)cap);
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    int32_t* d = (int32_t*)malloc(sizeof(int32_t) * (size_t)(m ? m : 1));
    if (!set || !s || !d) { free(set); free(s); free(d); return NULL; }
    memset(set, 0xff, sizeof(uint64_t) * (size_t)cap);
    int64_t got = 0; uint64_t ctr = 0;
    while (got < m) {
        uint64_t u = below(rng_at(key, ctr++), (uint64_t)n);
        uint64_t v = below(rng_at(key, ctr++), (uint64_t)n);
        if (u == v) continue;
        uint64_t lo = u < v ? u : v, hi = u < v ? v : u;
        uint64_t kk = (lo << 32) | hi;
        uint64_t h = mix64(kk) & (uint64_t)(cap - 1);
        int fresh = 1;
        while (set[h] != ~0ULL) { if (set[h] == kk) { fresh = 0; break; } h = (h + 1) & (uint64_t)(cap - 1); }
        if (!fresh) continue;
        set[h] = kk;
        s[got] = (int32_t)lo; d[got] = (int32_t)hi; ++got;
    }
    free(set);
    return finish(alloc_graph(), n, m, s, d, keep_pairs);
}

/* ---- R-MAT ---------------------------------------------------------------- */
tcg_graph* tcg_rmat(int scale, int64_t edge_factor, double a, double b, double c,
                    uint64_t seed, int relabel, int keep_pairs) {
    if (scale < 1 || scale > 30 || edge_factor < 1) return NULL;
    int64_t n = (int64_t)1 << scale;
    int64_t np = edge_factor * n;
    uint64_t key = stream_key(TAG_RMAT, seed);
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)np);
    int32_t* d = (int32_t*)malloc(sizeof(int32_t) * (size_t)np);
    int32_t* perm = (int32_t*)malloc(sizeof(int32_t) * (size_t)n);
    if (!s || !d || !perm) { free(s); free(d); free(perm); return NULL; }
    double ab = a + b, abc = a + b + c;
    #pragma omp parallel for schedule(static)
    for (int64_t i = 0; i < np; ++i) {
        uint32_t u = 0, v = 0;
        for (int l = 0; l < scale; ++l) {
            double r = u01(rng_at(key, (uint64_t)i * (uint64_t)scale + (uint64_t)l));
            uint32_t bu = 0, bv = 0;
            if (r < a) { } else if (r < ab) { bv = 1; } else if (r < abc) { bu = 1; } else { bu = 1; bv = 1; }
            u = (u << 1) | bu; v = (v << 1) | bv;
        }
        s[i] = (int32_t)u; d[i] = (int32_t)v;
    }
    for (int64_t i = 0; i < n; ++i) perm[i] = (int32_t)i;
    if (relabel) {
        uint64_t pk = stream_key(TAG_PERM, seed);
        for (int64_t i = n - 1; i > 0; --i) {
            int64_t j = (int64_t)below(rng_at(pk, (uint64_t)i), (uint64_t)(i + 1));
            int32_t t = perm[i]; perm[i] = perm[j]; perm[j] = t;
        }
        #pragma omp parallel for schedule(static)
        for (int64_t i = 0; i < np; ++i) { s[i] = perm[s[i]]; d[i] = perm[d[i]]; }
    }
    free(perm);
    return finish(alloc_graph(), n, np, s, d, keep_pairs);
}

/* ---- road-like grid ------------------------------------------------------- */
tcg_graph* tcg_grid(int64_t R, int64_t C, double p_diag, double frac_long, uint64_t seed, int keep_pairs) {
    if (R < 1 || C < 1 || R * C > 0x7fffffffLL) return NULL;
    int64_t n = R * C;
    uint64_t gk = stream_key(TAG_GRID, seed), lk = stream_key(TAG_LONG, seed);
    int64_t lattice = R * (C - 1) + (R - 1) * C;
    int64_t ndiag = 0;
    for (int64_t cell = 0; cell < (R - 1) * (C - 1); ++cell)
        if (u01(rng_at(gk, (uint64_t)cell)) < p_diag) ++ndiag;
    int64_t nlong = llround(frac_long * (double)(lattice + ndiag));
    int64_t np = lattice + ndiag + nlong;
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)(np ? np : 1));
    int32_t* d = (int32_t*)malloc(sizeof(int32_t) * (size_t)(np ? np : 1));
    if (!s || !d) { free(s); free(d); return NULL; }
    int64_t k = 0;
    for (int64_t i = 0; i < R; ++i)
        for (int64_t j = 0; j < C; ++j) {
            int64_t v = i * C + j;
            if (j + 1 < C) { s[k] = (int32_t)v; d[k] = (int32_t)(v + 1); ++k; }
            if (i + 1 < R) { s[k] = (int32_t)v; d[k] = (int32_t)(v + C); ++k; }
        }
    for (int64_t i = 0; i + 1 < R; ++i)
        for (int64_t j = 0; j + 1 < C; ++j) {
            int64_t cell = i * (C - 1) + j;
            if (u01(rng_at(gk, (uint64_t)cell)) < p_diag) {
                s[k] = (int32_t)(i * C + j); d[k] = (int32_t)((i + 1) * C + j + 1); ++k;
            }
        }
    for (int64_t l = 0; l < nlong; ++l) {
        s[k] = (int32_t)below(rng_at(lk, 2 * (uint64_t)l), (uint64_t)n);
        d[k] = (int32_t)below(rng_at(lk, 2 * (uint64_t)l + 1), (uint64_t)n);
        ++k;
    }
    return finish(alloc_graph(), n, np, s, d, keep_pairs);
}

/* ---- Barabasi-Albert ------------------------------------------------------ */
/* Fills s/d (capacity C(k+1,2) + (n-k-1)*k) and returns the pair count. */
static int64_t ba_pairs(int64_t n, int64_t k, uint64_t key, int32_t* s, int32_t* d, int32_t* ends) {
    int64_t np = 0, ne = 0;
    uint64_t ctr = 0;
    for (int64_t i = 0; i <= k; ++i)
        for (int64_t j = i + 1; j <= k; ++j) {
            s[np] = (int32_t)i; d[np] = (int32_t)j; ++np;
            ends[ne++] = (int32_t)i; ends[ne++] = (int32_t)j;
        }
    int32_t pick[64];
    for (int64_t v = k + 1; v < n; ++v) {
        int64_t got = 0;
        while (got < k) {
            int32_t t = ends[below(rng_at(key, ctr++), (uint64_t)ne)];
            int dup = 0;
            for (int64_t q = 0; q < got; ++q) if (pick[q] == t) { dup = 1; break; }
            if (!dup) pick[got++] = t;
        }
        for (int64_t q = 0; q < k; ++q) {
            s[np] = (int32_t)v; d[np] = pick[q]; ++np;
            ends[ne++] = (int32_t)v; ends[ne++] = pick[q];
        }
    }
    return np;
}

static int64_t ba_pair_cap(int64_t n, int64_t k) { return (k + 1) * k / 2 + (n - k - 1) * k; }

tcg_graph* tcg_ba(int64_t n, int64_t k, uint64_t seed, int keep_pairs) {
    if (k < 1 || k > 64 || n < k + 2) return NULL;
    int64_t cap = ba_pair_cap(n, k);
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t* d = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
    int32_t* e = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * cap));
    if (!s || !d || !e) { free(s); free(d); free(e); return NULL; }
    int64_t np = ba_pairs(n, k, stream_key(TAG_BA, seed), s, d, e);
    free(e);
    return finish(alloc_graph(), n, np, s, d, keep_pairs);
}

/* Batch of G BA graphs; graph i uses seed (seed0 + i).  Returns the
 * concatenation: row_ptr has sum(n_i)+1 entries holding offsets into the
 * concatenated col array; col holds LOCAL ids (0..n_i-1). */
tcg_graph* tcg_ba_batch(int64_t G, int64_t n_lo, int64_t n_hi, int64_t k_lo, int64_t k_hi, uint64_t seed0) {
    if (G < 1 || n_lo > n_hi || k_lo > k_hi || k_lo < 1 || k_hi > 64 || n_lo < k_hi + 2) return NULL;
    int64_t* ns = (int64_t*)malloc(sizeof(int64_t) * (size_t)G);
    int64_t* nnzs = (int64_t*)malloc(sizeof(int64_t) * (size_t)G);
    int64_t** rps = (int64_t**)calloc((size_t)G, sizeof(int64_t*));
    int32_t** cols = (int32_t**)calloc((size_t)G, sizeof(int32_t*));
    if (!ns || !nnzs || !rps || !cols) { free(ns); free(nnzs); free(rps); free(cols); return NULL; }
    int failed = 0;
    #pragma omp parallel for schedule(dynamic, 1) reduction(|:failed)
    for (int64_t i = 0; i < G; ++i) {
        uint64_t pk = stream_key(TAG_BATCH, seed0 + (uint64_t)i);
        int64_t n = n_lo + (int64_t)below(rng_at(pk, 0), (uint64_t)(n_hi - n_lo + 1));
        int64_t k = k_lo + (int64_t)below(rng_at(pk, 1), (uint64_t)(k_hi - k_lo + 1));
        int64_t cap = ba_pair_cap(n, k);
        int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
        int32_t* d = (int32_t*)malloc(sizeof(int32_t) * (size_t)cap);
        int32_t* e = (int32_t*)malloc(sizeof(int32_t) * (size_t)(2 * cap));
        if (!s || !d || !e) { free(s); free(d); free(e); failed |= 1; continue; }
        int64_t np = ba_pairs(n, k, stream_key(TAG_BA, seed0 + (uint64_t)i), s, d, e);
        free(e);
        ns[i] = n;
        if (pairs_to_csr(n, np, s, d, &rps[i], &cols[i], &nnzs[i]) != 0) failed |= 1;
        free(s); free(d);
    }
    tcg_graph* g = failed ? NULL : alloc_graph();
    if (g) {
        g->G = G;
        g->vtx_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(G + 1));
        g->edge_off = (int64_t*)malloc(sizeof(int64_t) * (size_t)(G + 1));
        g->vtx_off[0] = 0; g->edge_off[0] = 0;
        for (int64_t i = 0; i < G; ++i) {
            g->vtx_off[i + 1] = g->vtx_off[i] + ns[i];
            g->edge_off[i + 1] = g->edge_off[i] + nnzs[i];
        }
        g->n = g->vtx_off[G]; g->nnz = g->edge_off[G];
        g->row_ptr = (int64_t*)malloc(sizeof(int64_t) * (size_t)(g->n + 1));
        g->col = (int32_t*)malloc(sizeof(int32_t) * (size_t)(g->nnz ? g->nnz : 1));
        #pragma omp parallel for schedule(dynamic, 4)
        for (int64_t i = 0; i < G; ++i) {
            int64_t vo = g->vtx_off[i], eo = g->edge_off[i];
            for (int64_t v = 0; v < ns[i]; ++v) g->row_ptr[vo + v] = eo + rps[i][v];
            memcpy(g->col + eo, cols[i], sizeof(int32_t) * (size_t)nnzs[i]);
        }
        g->row_ptr[g->n] = g->nnz;
    }
    for (int64_t i = 0; i < G; ++i) { free(rps[i]); free(cols[i]); }
    free(rps); free(cols); free(ns); free(nnzs);
    return g;
}

/* Canonicalise caller-given pairs into a simple undirected CSR. */
tcg_graph* tcg_from_pairs(int64_t n, int64_t np, const int32_t* src, const int32_t* dst, int keep_pairs) {
    if (n < 0 || np < 0) return NULL;
    for (int64_t i = 0; i < np; ++i)
        if (src[i] < 0 || src[i] >= n || dst[i] < 0 || dst[i] >= n) return NULL;
    int32_t* s = (int32_t*)malloc(sizeof(int32_t) * (size_t)(np ? np : 1));
    int32_t* d = (int32_t*)malloc(sizeof(int32_t) * (size_t)(np ? np : 1));
    if (!s || !d) { free(s); free(d); return NULL; }
    memcpy(s, src, sizeof(int32_t) * (size_t)np);
    memcpy(d, dst, sizeof(int32_t) * (size_t)np);
    return finish(alloc_graph(), n, np, s, d, keep_pairs);
}

int64_t tcg_n(const tcg_graph* g) { return g->n; }
int64_t tcg_nnz(const tcg_graph* g) { return g->nnz; }
int64_t tcg_npairs(const tcg_graph* g) { return g->src ? g->npairs : 0; }
int64_t tcg_batch_count(const tcg_graph* g) { return g->G; }
void tcg_copy_csr(const tcg_graph* g, int64_t* row_ptr, int32_t* col) {
    memcpy(row_ptr, g->row_ptr, sizeof(int64_t) * (size_t)(g->n + 1));
    memcpy(col, g->col, sizeof(int32_t) * (size_t)g->nnz);
}
void tcg_copy_pairs(const tcg_graph* g, int32_t* src, int32_t* dst) {
    if (!g->src) return;
    memcpy(src, g->src, sizeof(int32_t) * (size_t)g->npairs);
    memcpy(dst, g->dst, sizeof(int32_t) * (size_t)g->npairs);
}
void tcg_copy_batch(const tcg_graph* g, int64_t* vtx_off, int64_t* edge_off) {
    if (g->G < 1) return;
    memcpy(vtx_off, g->vtx_off, sizeof(int64_t) * (size_t)(g->G + 1));
    memcpy(edge_off, g->edge_off, sizeof(int64_t) * (size_t)(g->G + 1));
}
void tcg_free(tcg_graph* g) {
    if (!g) return;
    free(g->row_ptr); free(g->col); free(g->src); free(g->dst);
    free(g->vtx_off); free(g->edge_off); free(g);
}
