/*
 * CPU oracle for exact k-clique counting.
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product path may link, load or
 * call this file; only the tests, the graft entry's smoke check and the CPU
 * baseline leg of the benchmark use it.  It shares no code with the CUDA
 * library: no headers, no tables, no helpers.
 *
 * What it computes (the plain definition, "Parallel K-clique Counting on
 * GPUs", Section 1 and Section 2.1):
 *     c_k(G)  = #{ S subset of V : |S| = k, every pair of S adjacent }
 *     c_k(v)  = #{ such S : v in S }            (per-vertex counts)
 * by the paper's own two routes, written plainly:
 *   - or_count_orient: the graph-orientation traversal of Fig. 2 (Section 2.2)
 *     over a DAG, with sorted-merge list intersections;
 *   - or_count_pivot:  the pivoting traversal of Fig. 3 (Section 2.3): level 1
 *     oriented, deeper levels on the undirected sub-graph induced by the root's
 *     out-neighbours (Section 2.4), pivot = candidate with most neighbours in
 *     the candidate set, leaf adds C(q, j - h) to count[j];
 *   - or_count_vertex: c_k(v) for one vertex as the (k-1)-cliques of G[N(v)],
 *     enumerated by increasing vertex id (a third, independent route).
 * Orientation orders (Section 3.1): degree order (deg, id) and degeneracy
 * order from sequential min-degree peeling (Batagelj-Zaversnik bucket form).
 *
 * Counts are accumulated in unsigned 128-bit integers that saturate at
 * 2^128 - 1 and raise a flag; callers learn whether the exact value exceeds
 * 2^64 - 1 from the high word or the flag.
 *
 * Pins (tests/test_oracle_pins.py): complete graphs (C(n, k)), complete
 * multipartite graphs (elementary symmetric polynomials), disjoint unions and
 * joins, triangle-free graphs, trace(A^3)/6, brute force over all k-subsets,
 * networkx core numbers and clique enumeration, orientation invariance and
 * agreement of the three routes.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef unsigned __int128 u128;
static const u128 U128_MAX = ~(u128)0;

static u128 sat_add(u128 a, u128 b) {
    u128 s = a + b;
    return (s < a) ? U128_MAX : s;
}

static int cmp_u32(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------------ */
/* Canonicalisation: symmetrise, drop self-loops and duplicates, sort rows.  */
/* Returns 0, or -1 when an endpoint is out of range, -2 when cap is short.  */
/* ------------------------------------------------------------------------ */
int or_canonicalize(uint32_t n, uint64_t ne, const uint32_t* src, const uint32_t* dst,
                    uint32_t* row_ptr, uint32_t* col, uint64_t cap, uint64_t* nnz_out) {
    uint64_t* cnt = (uint64_t*)calloc((size_t)n + 1, sizeof(uint64_t));
    for (uint64_t e = 0; e < ne; ++e) {
        if (src[e] >= n || dst[e] >= n) { free(cnt); return -1; }
        if (src[e] == dst[e]) continue;
        cnt[src[e]]++;
        cnt[dst[e]]++;
    }
    uint64_t total = 0;
    uint64_t* start = (uint64_t*)malloc(((size_t)n + 1) * sizeof(uint64_t));
    for (uint32_t v = 0; v < n; ++v) { start[v] = total; total += cnt[v]; }
    start[n] = total;
    uint32_t* tmp = (uint32_t*)malloc((size_t)(total ? total : 1) * sizeof(uint32_t));
    memset(cnt, 0, ((size_t)n + 1) * sizeof(uint64_t));
    for (uint64_t e = 0; e < ne; ++e) {
        uint32_t a = src[e], b = dst[e];
        if (a == b) continue;
        tmp[start[a] + cnt[a]++] = b;
        tmp[start[b] + cnt[b]++] = a;
    }
    uint64_t out = 0;
    row_ptr[0] = 0;
    for (uint32_t v = 0; v < n; ++v) {
        uint32_t* row = tmp + start[v];
        uint64_t len = start[v + 1] - start[v];
        qsort(row, (size_t)len, sizeof(uint32_t), cmp_u32);
        for (uint64_t i = 0; i < len; ++i) {
            if (i > 0 && row[i] == row[i - 1]) continue;
            if (out >= cap) { free(cnt); free(start); free(tmp); return -2; }
            col[out++] = row[i];
        }
        row_ptr[v + 1] = (uint32_t)out;
    }
    *nnz_out = out;
    free(cnt); free(start); free(tmp);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Orders.                                                                   */
/* ------------------------------------------------------------------------ */

static const uint32_t* g_sort_deg;
static int cmp_deg_id(const void* a, const void* b) {
    uint32_t x = *(const uint32_t*)a, y = *(const uint32_t*)b;
    if (g_sort_deg[x] != g_sort_deg[y]) return g_sort_deg[x] < g_sort_deg[y] ? -1 : 1;
    return (x > y) - (x < y);
}

/* rank[v] = position of v when vertices are sorted by (degree, id). */
void or_degree_rank(uint32_t n, const uint32_t* row_ptr, uint32_t* rank) {
    uint32_t* deg = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    uint32_t* ord = (uint32_t*)malloc((size_t)(n ? n : 1) * sizeof(uint32_t));
    for (uint32_t v = 0; v < n; ++v) { deg[v] = row_ptr[v + 1] - row_ptr[v]; ord[v] = v; }
    g_sort_deg = deg;
    qsort(ord, n, sizeof(uint32_t), cmp_deg_id);
    for (uint32_t i = 0; i < n; ++i) rank[ord[i]] = i;
    free(deg); free(ord);
}

/* Sequential peeling: repeatedly remove a vertex of minimum remaining degree
 * (bucket queue of Batagelj and Zaversnik).  order[i] = i-th removed vertex,
 * rank[v] = its removal position, core[v] = core number.  Returns the
 * degeneracy (max core number). */
uint32_t or_degeneracy_order(uint32_t n, const uint32_t* row_ptr, const uint32_t* col,
                             uint32_t* rank, uint32_t* core, uint32_t* order) {
    if (n == 0) return 0;
    uint32_t* deg = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    uint32_t* pos = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    uint32_t* vert = (uint32_t*)malloc((size_t)n * sizeof(uint32_t));
    uint32_t md = 0;
    for (uint32_t v = 0; v < n; ++v) {
        deg[v] = row_ptr[v + 1] - row_ptr[v];
        if (deg[v] > md) md = deg[v];
    }
    uint32_t* bin = (uint32_t*)calloc((size_t)md + 2, sizeof(uint32_t));
    for (uint32_t v = 0; v < n; ++v) bin[deg[v]]++;
    uint32_t s = 0;
    for (uint32_t d = 0; d <= md; ++d) { uint32_t c = bin[d]; bin[d] = s; s += c; }
    for (uint32_t v = 0; v < n; ++v) { pos[v] = bin[deg[v]]++; vert[pos[v]] = v; }
    for (uint32_t d = md; d >= 1; --d) bin[d] = bin[d - 1];
    bin[0] = 0;
    uint32_t degeneracy = 0;
    for (uint32_t i = 0; i < n; ++i) {
        uint32_t v = vert[i];
        if (deg[v] > degeneracy) degeneracy = deg[v];
        for (uint32_t e = row_ptr[v]; e < row_ptr[v + 1]; ++e) {
            uint32_t u = col[e];
            if (deg[u] > deg[v]) {
                uint32_t du = deg[u], pu = pos[u], pw = bin[du], w = vert[pw];
                if (u != w) { pos[u] = pw; vert[pu] = w; pos[w] = pu; vert[pw] = u; }
                bin[du]++;
                deg[u]--;
            }
        }
    }
    for (uint32_t i = 0; i < n; ++i) {
        rank[vert[i]] = i;
        if (order) order[i] = vert[i];
    }
    if (core) for (uint32_t v = 0; v < n; ++v) core[v] = deg[v];
    free(deg); free(pos); free(vert); free(bin);
    return degeneracy;
}

/* DAG: keep u -> w iff rank[u] < rank[w]; rows stay in id order.
 * dag_row_ptr has n+1 entries, dag_col at least nnz/2.  Returns max out-degree. */
uint32_t or_orient(uint32_t n, const uint32_t* row_ptr, const uint32_t* col, const uint32_t* rank,
                   uint32_t* dag_row_ptr, uint32_t* dag_col) {
    uint32_t out = 0, dmax = 0;
    dag_row_ptr[0] = 0;
    for (uint32_t u = 0; u < n; ++u) {
        uint32_t start = out;
        for (uint32_t e = row_ptr[u]; e < row_ptr[u + 1]; ++e)
            if (rank[u] < rank[col[e]]) dag_col[out++] = col[e];
        dag_row_ptr[u + 1] = out;
        if (out - start > dmax) dmax = out - start;
    }
    return dmax;
}

/* ------------------------------------------------------------------------ */
/* Orientation traversal (Fig. 2).                                           */
/* ------------------------------------------------------------------------ */

typedef struct {
    const uint32_t* rp;
    const uint32_t* ci;
    uint32_t k;
    uint32_t* lists;   /* level l list at lists + l * stride */
    uint64_t stride;
    uint32_t* path;    /* vertices on the current path */
    u128 total;
    u128* pv;          /* per-vertex accumulators (or NULL) */
} orient_ctx;

/* |A ∩ B| written to out (both sorted ascending). */
static uint32_t merge_intersect(const uint32_t* a, uint32_t na, const uint32_t* b, uint32_t nb, uint32_t* out) {
    uint32_t i = 0, j = 0, o = 0;
    while (i < na && j < nb) {
        if (a[i] < b[j]) ++i;
        else if (a[i] > b[j]) ++j;
        else { out[o++] = a[i]; ++i; ++j; }
    }
    return o;
}

/* I holds the level-l vertices (the common out-neighbours of the l-1 vertices
 * on the path).  For each v in I, I' = I ∩ Adj(v); at level k-1 the |I'|
 * k-cliques are counted, otherwise the traversal continues at level l+1. */
static void orient_traverse(orient_ctx* c, uint32_t l, const uint32_t* I, uint32_t nI) {
    uint32_t* Inext = c->lists + (uint64_t)(l + 1) * c->stride;
    for (uint32_t t = 0; t < nI; ++t) {
        uint32_t v = I[t];
        const uint32_t* adj = c->ci + c->rp[v];
        uint32_t nadj = c->rp[v + 1] - c->rp[v];
        uint32_t nn = merge_intersect(I, nI, adj, nadj, Inext);
        c->path[l - 1] = v;
        if (l + 1 == c->k) {
            c->total = sat_add(c->total, nn);
            if (c->pv) {
                for (uint32_t p = 0; p < l; ++p) c->pv[c->path[p]] = sat_add(c->pv[c->path[p]], nn);
                for (uint32_t p = 0; p < nn; ++p) c->pv[Inext[p]] = sat_add(c->pv[Inext[p]], 1);
            }
        } else if (nn > 0) {
            orient_traverse(c, l + 1, Inext, nn);
        }
    }
}

static void split128(u128 x, uint64_t* lo, uint64_t* hi) {
    *lo = (uint64_t)x;
    *hi = (uint64_t)(x >> 64);
}

/* c_k by Fig. 2 over the DAG (rows sorted by id).  roots: list of level-1
 * vertices to expand (NULL = all).  per_root (NULL or n entries) gets the
 * low 64 bits of the count found under each root; per_vertex_lo/hi (NULL or n
 * entries each) get c_k(v) split in two words (only when roots == NULL, and
 * then only with one thread).  Returns 1 if the total saturated at 2^128-1. */
int or_count_orient(uint32_t n, const uint32_t* dag_rp, const uint32_t* dag_ci, uint32_t k,
                     const uint32_t* roots, uint32_t nroots, int nthreads,
                     uint64_t* total_lo, uint64_t* total_hi, uint64_t* per_root,
                     uint64_t* per_vertex_lo, uint64_t* per_vertex_hi) {
    if (k == 0) { *total_lo = 1; *total_hi = 0; return 0; }
    uint32_t dmax = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (dag_rp[v + 1] - dag_rp[v] > dmax) dmax = dag_rp[v + 1] - dag_rp[v];
    uint32_t nr = roots ? nroots : n;
    int want_pv = (per_vertex_lo != NULL);
    if (want_pv) nthreads = 1;
    if (nthreads < 1) nthreads = 1;
    u128* totals = (u128*)calloc((size_t)nthreads, sizeof(u128));
    u128* pv = want_pv ? (u128*)calloc((size_t)(n ? n : 1), sizeof(u128)) : NULL;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        orient_ctx c;
        c.rp = dag_rp; c.ci = dag_ci; c.k = k;
        c.stride = (uint64_t)dmax + 1;
        c.lists = (uint32_t*)malloc((size_t)(c.stride * (k + 2)) * sizeof(uint32_t));
        c.path = (uint32_t*)malloc((size_t)(k + 2) * sizeof(uint32_t));
        c.total = 0;
        c.pv = pv;
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (uint32_t r = 0; r < nr; ++r) {
            uint32_t v = roots ? roots[r] : r;
            u128 before = c.total;
            if (k == 1) {
                c.total = sat_add(c.total, 1);
                if (c.pv) c.pv[v] = sat_add(c.pv[v], 1);
            } else {
                /* level 1: I = V, choosing v gives I' = N+(v) at level 2 */
                const uint32_t* adj = dag_ci + dag_rp[v];
                uint32_t nadj = dag_rp[v + 1] - dag_rp[v];
                c.path[0] = v;
                if (k == 2) {
                    c.total = sat_add(c.total, nadj);
                    if (c.pv) {
                        c.pv[v] = sat_add(c.pv[v], nadj);
                        for (uint32_t p = 0; p < nadj; ++p) c.pv[adj[p]] = sat_add(c.pv[adj[p]], 1);
                    }
                } else if (nadj > 0) {
                    memcpy(c.lists + 2 * c.stride, adj, (size_t)nadj * sizeof(uint32_t));
                    orient_traverse(&c, 2, c.lists + 2 * c.stride, nadj);
                }
            }
            if (per_root) per_root[r] = (uint64_t)(c.total - before);
        }
        totals[tid] = c.total;
        free(c.lists);
        free(c.path);
    }
    u128 t = 0;
    for (int i = 0; i < nthreads; ++i) t = sat_add(t, totals[i]);
    split128(t, total_lo, total_hi);
    if (want_pv)
        for (uint32_t v = 0; v < n; ++v) split128(pv[v], per_vertex_lo + v, per_vertex_hi + v);
    free(totals);
    free(pv);
    return t == U128_MAX;
}

/* ------------------------------------------------------------------------ */
/* Pivoting traversal (Fig. 3) with level-1 orientation (Section 2.3-2.4).  */
/* ------------------------------------------------------------------------ */

typedef struct {
    uint32_t cap;          /* counts[0..cap-1] */
    uint32_t kfix;         /* 0 = all k; otherwise only k = kfix is needed */
    uint32_t pvk;          /* per-vertex k (0 = none) */
    const u128* binom;     /* binom[a * bstride + b] */
    uint32_t bstride;
    const uint8_t* adj;    /* d x d local adjacency of the root's sub-graph */
    uint32_t d;
    const uint32_t* S0;    /* global ids of the local vertices */
    uint32_t* lists;       /* level buffers */
    uint32_t* held;        /* local ids of held vertices (root excluded) */
    uint32_t* piv;         /* local ids of pivots */
    uint32_t root;
    u128* counts;
    u128* pv;
    uint32_t max_clique;   /* largest h + q seen at a leaf */
} piv_ctx;

static u128 binom_at(const piv_ctx* c, uint32_t a, uint32_t b) {
    if (b > a) return 0;
    return c->binom[(uint64_t)a * c->bstride + b];
}

static void pivot_leaf(piv_ctx* c, uint32_t h, uint32_t q) {
    if (h + q > c->max_clique) c->max_clique = h + q;
    for (uint32_t j = h; j <= h + q && j < c->cap; ++j)
        c->counts[j] = sat_add(c->counts[j], binom_at(c, q, j - h));
    if (c->pv && c->pvk >= h && c->pvk <= h + q) {
        u128 held_gain = binom_at(c, q, c->pvk - h);
        c->pv[c->root] = sat_add(c->pv[c->root], held_gain);
        for (uint32_t i = 0; i + 1 < h; ++i) c->pv[c->S0[c->held[i]]] = sat_add(c->pv[c->S0[c->held[i]]], held_gain);
        if (q >= 1 && c->pvk >= h + 1) {
            u128 piv_gain = binom_at(c, q - 1, c->pvk - h - 1);
            for (uint32_t i = 0; i < q; ++i) c->pv[c->S0[c->piv[i]]] = sat_add(c->pv[c->S0[c->piv[i]]], piv_gain);
        }
    }
}

/* S: local ids (ascending) of the candidates, all adjacent to every vertex on
 * the path.  h = held vertices on the path (root included), q = pivots. */
static void pivot_traverse(piv_ctx* c, uint32_t depth, const uint32_t* S, uint32_t nS, uint32_t h, uint32_t q) {
    if (nS == 0) { pivot_leaf(c, h, q); return; }
    /* pivot: the candidate with the most neighbours inside S, lowest position on ties */
    uint32_t p = S[0], best = 0;
    for (uint32_t a = 0; a < nS; ++a) {
        uint32_t cnt = 0;
        for (uint32_t b = 0; b < nS; ++b) cnt += c->adj[(uint64_t)S[a] * c->d + S[b]];
        if (a == 0 || cnt > best) { best = cnt; p = S[a]; }
    }
    /* branch set: S minus the pivot's neighbours (the pivot itself included) */
    uint32_t* B = c->lists + (uint64_t)(2 * depth) * (c->d + 1);
    uint32_t nB = 0;
    for (uint32_t a = 0; a < nS; ++a)
        if (S[a] == p || !c->adj[(uint64_t)p * c->d + S[a]]) B[nB++] = S[a];
    uint32_t* Snext = c->lists + (uint64_t)(2 * depth + 1) * (c->d + 1);
    for (uint32_t i = 0; i < nB; ++i) {
        uint32_t x = B[i];
        uint32_t h2 = h + (x != p), q2 = q + (x == p);
        /* stopping criterion: more held vertices than the wanted clique size */
        if (c->kfix && h2 > c->kfix) continue;
        /* S' = S ∩ N(x) minus the branch vertices already visited */
        uint32_t ns = 0;
        for (uint32_t a = 0; a < nS; ++a) {
            uint32_t y = S[a];
            if (!c->adj[(uint64_t)x * c->d + y]) continue;
            int earlier = 0;
            for (uint32_t e = 0; e < i; ++e) if (B[e] == y) { earlier = 1; break; }
            if (!earlier) Snext[ns++] = y;
        }
        if (x == p) c->piv[q] = x; else c->held[h - 1] = x;
        /* the child writes only the buffers of depth + 1, so Snext stays intact */
        pivot_traverse(c, depth + 1, Snext, ns, h2, q2);
    }
}

/* All-k (kfix = 0) or fixed-k counts by pivoting.  undirected CSR (rp, ci)
 * supplies adjacency inside each root's candidate set; the DAG supplies the
 * level-1 candidate sets N+(v).  counts_lo/hi/sat get cap entries
 * (counts[0] = 1 by convention).  per_vertex (NULL or n entries each) gets
 * c_pvk(v).  max_clique_out gets the clique number.  roots as in
 * or_count_orient.  Returns 1 if any count saturated. */
int or_count_pivot(uint32_t n, const uint32_t* rp, const uint32_t* ci,
                   const uint32_t* dag_rp, const uint32_t* dag_ci,
                   uint32_t cap, uint32_t kfix, const uint32_t* roots, uint32_t nroots, int nthreads,
                   uint64_t* counts_lo, uint64_t* counts_hi, uint8_t* counts_sat,
                   uint32_t pvk, uint64_t* per_vertex_lo, uint64_t* per_vertex_hi,
                   uint32_t* max_clique_out) {
    uint32_t dmax = 0;
    for (uint32_t v = 0; v < n; ++v)
        if (dag_rp[v + 1] - dag_rp[v] > dmax) dmax = dag_rp[v + 1] - dag_rp[v];
    uint32_t B = dmax + 2;
    if (B < cap + 1) B = cap + 1;
    /* Pascal's triangle, saturating */
    u128* binom = (u128*)calloc((size_t)B * B, sizeof(u128));
    for (uint32_t a = 0; a < B; ++a) {
        binom[(uint64_t)a * B] = 1;
        for (uint32_t b = 1; b <= a; ++b)
            binom[(uint64_t)a * B + b] = sat_add(binom[(uint64_t)(a - 1) * B + b - 1],
                                                 binom[(uint64_t)(a - 1) * B + b]);
    }
    uint32_t nr = roots ? nroots : n;
    int want_pv = (per_vertex_lo != NULL && pvk > 0);
    if (want_pv) nthreads = 1;
    if (nthreads < 1) nthreads = 1;
    u128* all_counts = (u128*)calloc((size_t)nthreads * cap, sizeof(u128));
    uint32_t* all_omega = (uint32_t*)calloc((size_t)nthreads, sizeof(uint32_t));
    u128* pv = want_pv ? (u128*)calloc((size_t)(n ? n : 1), sizeof(u128)) : NULL;
#ifdef _OPENMP
#pragma omp parallel num_threads(nthreads)
#endif
    {
        int tid = 0;
#ifdef _OPENMP
        tid = omp_get_thread_num();
#endif
        piv_ctx c;
        memset(&c, 0, sizeof(c));
        c.cap = cap; c.kfix = kfix; c.pvk = want_pv ? pvk : 0;
        c.binom = binom; c.bstride = B;
        c.counts = all_counts + (uint64_t)tid * cap;
        c.pv = pv;
        uint8_t* adj = (uint8_t*)malloc((size_t)(dmax ? dmax : 1) * (dmax ? dmax : 1));
        c.lists = (uint32_t*)malloc((size_t)(2 * (dmax + 3)) * (dmax + 1) * sizeof(uint32_t));
        c.held = (uint32_t*)malloc((size_t)(dmax + 2) * sizeof(uint32_t));
        c.piv = (uint32_t*)malloc((size_t)(dmax + 2) * sizeof(uint32_t));
        uint32_t* S = (uint32_t*)malloc((size_t)(dmax + 1) * sizeof(uint32_t));
#ifdef _OPENMP
#pragma omp for schedule(dynamic, 16)
#endif
        for (uint32_t r = 0; r < nr; ++r) {
            uint32_t v = roots ? roots[r] : r;
            const uint32_t* cand = dag_ci + dag_rp[v];
            uint32_t d = dag_rp[v + 1] - dag_rp[v];
            /* undirected adjacency among the candidates (binary search in N(x)) */
            for (uint32_t a = 0; a < d; ++a) {
                const uint32_t* row = ci + rp[cand[a]];
                size_t len = rp[cand[a] + 1] - rp[cand[a]];
                for (uint32_t b = 0; b < d; ++b)
                    adj[(uint64_t)a * d + b] = bsearch(&cand[b], row, len, sizeof(uint32_t), cmp_u32) != NULL;
            }
            c.adj = adj; c.d = d; c.S0 = cand; c.root = v;
            for (uint32_t a = 0; a < d; ++a) S[a] = a;
            pivot_traverse(&c, 0, S, d, 1, 0);
        }
        all_omega[tid] = c.max_clique;
        free(adj); free(c.lists); free(c.held); free(c.piv); free(S);
    }
    int any_sat = 0;
    uint32_t omega = 0;
    for (uint32_t j = 0; j < cap; ++j) {
        u128 t = 0;
        for (int i = 0; i < nthreads; ++i) t = sat_add(t, all_counts[(uint64_t)i * cap + j]);
        if (j == 0) t = 1;
        split128(t, counts_lo + j, counts_hi + j);
        counts_sat[j] = (t == U128_MAX);
        any_sat |= counts_sat[j];
    }
    for (int i = 0; i < nthreads; ++i) if (all_omega[i] > omega) omega = all_omega[i];
    if (max_clique_out) *max_clique_out = (n == 0) ? 0 : omega;
    if (want_pv)
        for (uint32_t v = 0; v < n; ++v) split128(pv[v], per_vertex_lo + v, per_vertex_hi + v);
    free(binom); free(all_counts); free(all_omega); free(pv);
    return any_sat;
}

/* ------------------------------------------------------------------------ */
/* c_k(v) of one vertex: the (k-1)-cliques of G[N(v)], by increasing id.     */
/* ------------------------------------------------------------------------ */

static u128 cliques_in(const uint32_t* rp, const uint32_t* ci, const uint32_t* L, uint32_t nL,
                       uint32_t r, uint32_t* buf, uint64_t stride) {
    if (r == 0) return 1;
    if (r == 1) return nL;
    u128 s = 0;
    uint32_t* next = buf;
    for (uint32_t i = 0; i < nL; ++i) {
        uint32_t x = L[i];
        /* candidates after x in L that are neighbours of x */
        uint32_t nn = merge_intersect(L + i + 1, nL - i - 1, ci + rp[x], rp[x + 1] - rp[x], next);
        if (nn + 1 < r) continue;
        s = sat_add(s, cliques_in(rp, ci, next, nn, r - 1, buf + stride, stride));
    }
    return s;
}

int or_count_vertex(uint32_t n, const uint32_t* rp, const uint32_t* ci, uint32_t v, uint32_t k,
                    uint64_t* lo, uint64_t* hi) {
    (void)n;
    if (k == 0) { *lo = 0; *hi = 0; return 0; }
    uint32_t d = rp[v + 1] - rp[v];
    uint64_t stride = (uint64_t)d + 1;
    uint32_t* buf = (uint32_t*)malloc((size_t)(stride * (k + 1)) * sizeof(uint32_t));
    u128 s = cliques_in(rp, ci, ci + rp[v], d, k - 1, buf, stride);
    free(buf);
    split128(s, lo, hi);
    return s == U128_MAX;
}
