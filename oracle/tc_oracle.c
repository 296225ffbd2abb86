/*
 * tc_oracle.c -- TEST INFRASTRUCTURE ONLY.  The plain, slow, obviously correct
 * CPU statement of exact triangle counting.  Only tests/, the smoke check and
 * the benchmark's CPU-baseline leg may load it; the library never does.  It
 * shares no code with the CUDA path.
 *
 * What it computes (paper, Sec. 3 "Parallel Triangle Counting Algorithms" and
 * Sec. 3.2 "TC using Set Intersection"):
 *   T    = number of unordered vertex triples that are pairwise adjacent in a
 *          simple undirected graph;
 *   t(v) = number of those triples that contain v.
 * It follows the sequential *forward* algorithm of Schank and Wagner that the
 * paper uses as its CPU baseline (Sec. 5) and that Alg. 2 parallelises:
 *   1. canonicalise the input (drop self-loops, both directions, de-duplicate;
 *      Table 1 caption);
 *   2. order vertices by rank(v) = (d(v), v) and keep every undirected edge
 *      once, from the lower to the higher rank (Sec. 4.2.1, filtering by
 *      degree with ties broken by id);
 *   3. for every kept edge (u, v) intersect the two kept-neighbour lists by a
 *      sorted two-pointer merge; every common w closes the triangle {u, v, w}
 *      (Sec. 3.2: the intersection of the neighbour lists of u and v lists the
 *      triangles on edge (u, v));
 *   4. sum the intersection sizes (Alg. 2, Reduce).
 * All counters are int64.  Nothing here is blocked, fused or reordered.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

static int cmp_u64(const void* a, const void* b) {
    uint64_t x = *(const uint64_t*)a, y = *(const uint64_t*)b;
    return x < y ? -1 : (x > y ? 1 : 0);
}

/* Step 1.  Pairs (src[i], dst[i]) with ids in [0, n) -> simple undirected
 * CSR: row_ptr[n+1], col[cap]; both directions present, neighbours ascending.
 * Returns the number of CSR entries, or -1 (bad id or cap too small). */
int64_t oracle_canonicalize(int64_t n, int64_t npairs, const int32_t* src, const int32_t* dst,
                            int64_t* row_ptr, int32_t* col, int64_t cap) {
    uint64_t* key = (uint64_t*)malloc(sizeof(uint64_t) * (size_t)(2 * npairs + 1));
    if (!key) return -1;
    int64_t k = 0;
    for (int64_t i = 0; i < npairs; ++i) {
        int64_t u = src[i], v = dst[i];
        if (u < 0 || u >= n || v < 0 || v >= n) { free(key); return -1; }
        if (u == v) continue;                                  /* self-loop: no edge */
        key[k++] = ((uint64_t)u << 32) | (uint64_t)v;          /* both directions */
        key[k++] = ((uint64_t)v << 32) | (uint64_t)u;
    }
    qsort(key, (size_t)k, sizeof(uint64_t), cmp_u64);
    for (int64_t v = 0; v <= n; ++v) row_ptr[v] = 0;
    int64_t nnz = 0;
    for (int64_t i = 0; i < k; ++i) {
        if (i > 0 && key[i] == key[i - 1]) continue;           /* duplicate edge */
        if (nnz >= cap) { free(key); return -1; }
        col[nnz++] = (int32_t)(key[i] & 0xffffffffu);
        row_ptr[(key[i] >> 32) + 1] += 1;
    }
    for (int64_t v = 0; v < n; ++v) row_ptr[v + 1] += row_ptr[v];
    free(key);
    return nnz;
}

/* rank(a) < rank(b) with rank(v) = (d(v), v) compared lexicographically. */
static int rank_less(int64_t da, int64_t a, int64_t db, int64_t b) {
    return da < db || (da == db && a < b);
}

/* Step 2.  Simple undirected CSR -> oriented CSR: N+(u) = neighbours v of u
 * with rank(u) < rank(v), kept in ascending id order.  rpp[n+1], colp[cap].
 * Returns |E+| or -1 when cap is too small. */
int64_t oracle_orient(int64_t n, const int64_t* row_ptr, const int32_t* col,
                      int64_t* rpp, int32_t* colp, int64_t cap) {
    int64_t kept = 0;
    rpp[0] = 0;
    for (int64_t u = 0; u < n; ++u) {
        int64_t du = row_ptr[u + 1] - row_ptr[u];
        for (int64_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e) {
            int64_t v = col[e];
            int64_t dv = row_ptr[v + 1] - row_ptr[v];
            if (rank_less(du, u, dv, v)) {
                if (kept >= cap) return -1;
                colp[kept++] = (int32_t)v;
            }
        }
        rpp[u + 1] = kept;
    }
    return kept;
}

/* Steps 3-4 for source rows u = u_begin, u_begin+stride, ... < u_end.
 * Returns the number of triangles whose lowest-ranked vertex is one of those
 * rows; when t != NULL adds each such triangle to t[u], t[v] and t[w]. */
int64_t oracle_count_rows(int64_t n, const int64_t* rpp, const int32_t* colp,
                          int64_t u_begin, int64_t u_end, int64_t stride, int64_t* t) {
    int64_t T = 0;
    if (stride < 1) stride = 1;
    if (u_end > n) u_end = n;
    for (int64_t u = u_begin; u < u_end; u += stride) {
        for (int64_t e = rpp[u]; e < rpp[u + 1]; ++e) {
            int64_t v = colp[e];
            /* sorted merge of N+(u) and N+(v) */
            int64_t i = rpp[u], iend = rpp[u + 1];
            int64_t j = rpp[v], jend = rpp[v + 1];
            while (i < iend && j < jend) {
                if (colp[i] < colp[j]) ++i;
                else if (colp[i] > colp[j]) ++j;
                else {
                    int64_t w = colp[i];
                    T += 1;
                    if (t) { t[u] += 1; t[v] += 1; t[w] += 1; }
                    ++i; ++j;
                }
            }
        }
    }
    return T;
}

/* Steps 3-4 over all rows.  t may be NULL; when given it is zeroed first. */
int64_t oracle_count(int64_t n, const int64_t* rpp, const int32_t* colp, int64_t* t) {
    if (t) memset(t, 0, sizeof(int64_t) * (size_t)n);
    return oracle_count_rows(n, rpp, colp, 0, n, 1, t);
}

/* t(v) straight from the definition on the undirected CSR: the number of
 * adjacent pairs among N(v) = (1/2) * sum over x in N(v) of |N(v) & N(x)|.
 * Used to check single vertices of graphs too large for a full count. */
int64_t oracle_vertex_triangles(int64_t n, const int64_t* row_ptr, const int32_t* col, int64_t v) {
    if (v < 0 || v >= n) return 0;
    int64_t twice = 0;
    for (int64_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
        int64_t x = col[e];
        int64_t i = row_ptr[v], iend = row_ptr[v + 1];
        int64_t j = row_ptr[x], jend = row_ptr[x + 1];
        while (i < iend && j < jend) {
            if (col[i] < col[j]) ++i;
            else if (col[i] > col[j]) ++j;
            else { twice += 1; ++i; ++j; }
        }
    }
    return twice / 2;
}

/* Per-edge support by definition: sup[e] = |N(a) & N(b)| for every entry
 * e = (a, b) of the undirected CSR, the number of triangles containing the
 * edge {a, b} (sorted merge of the two full neighbour lists). */
void oracle_edge_support(int64_t n, const int64_t* row_ptr, const int32_t* col, int64_t* sup) {
    for (int64_t a = 0; a < n; ++a) {
        for (int64_t e = row_ptr[a]; e < row_ptr[a + 1]; ++e) {
            int64_t b = col[e], c = 0;
            int64_t i = row_ptr[a], iend = row_ptr[a + 1];
            int64_t j = row_ptr[b], jend = row_ptr[b + 1];
            while (i < iend && j < jend) {
                if (col[i] < col[j]) ++i;
                else if (col[i] > col[j]) ++j;
                else { ++c; ++i; ++j; }
            }
            sup[e] = c;
        }
    }
}

/* Triangle listing with the forward algorithm: every triangle once as
 * (u, v, w), u the lowest and w the highest rank.  Writes at most cap
 * triples into tri[3*cap]; returns the number of triangles. */
int64_t oracle_list_triangles(int64_t n, const int64_t* rpp, const int32_t* colp, int32_t* tri, int64_t cap) {
    int64_t T = 0;
    for (int64_t u = 0; u < n; ++u) {
        for (int64_t e = rpp[u]; e < rpp[u + 1]; ++e) {
            int64_t v = colp[e];
            int64_t i = rpp[u], iend = rpp[u + 1];
            int64_t j = rpp[v], jend = rpp[v + 1];
            while (i < iend && j < jend) {
                if (colp[i] < colp[j]) ++i;
                else if (colp[i] > colp[j]) ++j;
                else {
                    if (T < cap) {
                        tri[3 * T] = (int32_t)u;
                        tri[3 * T + 1] = (int32_t)v;
                        tri[3 * T + 2] = colp[i];
                    }
                    ++T; ++i; ++j;
                }
            }
        }
    }
    return T;
}
