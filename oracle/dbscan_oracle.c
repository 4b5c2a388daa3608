/*
 * CPU oracle for exact Euclidean DBSCAN.
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the checker for the CUDA library:
 * only the test suite, the smoke check and the benchmark's CPU-baseline leg
 * may build, load or call it.  It shares no code, header, table or helper
 * with the CUDA path.
 *
 * It writes out the DBSCAN definition of Sec. 2 ("DBSCAN Definition") as
 * plainly as possible, in IEEE FP64:
 *
 *   within(p, q)  :=  sum_{i=0}^{d-1} (p_i - q_i)^2  <=  eps^2
 *       evaluated left to right over i, every subtraction, product and sum
 *       rounded to nearest, no fused multiply-add (the file is compiled with
 *       -ffp-contract=off), eps^2 = fl(eps * eps).  The paper writes
 *       d(p, q) <= eps and leaves the arithmetic open; the squared form is the
 *       reading taken here.
 *   core(p)       :=  |{ q in P : within(p, q) }| >= minPts   (q = p counts)
 *   clusters      :=  connected components of the graph on core points with
 *                     an edge between core p and q iff within(p, q); a
 *                     cluster is named by the smallest input index of its
 *                     core points.
 *   border sets   :=  for non-core p, the sorted set of the names of the
 *                     clusters of all core q with within(p, q); empty = noise.
 *
 * The only device beyond the definition is a sort of the points by their first
 * coordinate, used to skip pairs that cannot be within eps: with the points in
 * that order, fl((p_0 - q_0)^2) grows monotonically as q moves away from p, and
 * the rounded sum of non-negative terms is never below its first term, so once
 * the first term exceeds eps^2 no later pair can pass within().  Every pair that
 * is not skipped this way goes through within() itself.
 *
 * Connected components use a textbook sequential union-find (union by
 * smaller root index), so the root of a component is its smallest index.
 * The predicate is evaluated by OpenMP threads; the unions are applied by one
 * thread, in a fixed order.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

/* Sec. 2: d(p, q) <= eps, squared, FP64, left to right, no contraction. */
static int within(const double *p, const double *q, int d, double eps2) {
    double s = 0.0;
    for (int i = 0; i < d; ++i) {
        double t = p[i] - q[i];
        double sq = t * t;
        s = s + sq;
    }
    return s <= eps2;
}

static double first_term(const double *p, const double *q) {
    double t = p[0] - q[0];
    return t * t;
}

/* ---- sort of point indices by first coordinate (ties by index) ---------- */
static const double *g_sort_x;
static int g_sort_d;
static int cmp_first(const void *a, const void *b) {
    int64_t i = *(const int64_t *)a, j = *(const int64_t *)b;
    double xi = g_sort_x[i * g_sort_d], xj = g_sort_x[j * g_sort_d];
    if (xi < xj) return -1;
    if (xi > xj) return 1;
    return (i < j) ? -1 : (i > j);
}

static int64_t *order_by_first(const double *X, int64_t n, int d) {
    int64_t *ord = (int64_t *)malloc(sizeof(int64_t) * (size_t)(n > 0 ? n : 1));
    if (!ord) return NULL;
    for (int64_t i = 0; i < n; ++i) ord[i] = i;
    g_sort_x = X;
    g_sort_d = d;
    qsort(ord, (size_t)n, sizeof(int64_t), cmp_first);
    return ord;
}

/* ---- union-find (sequential) -------------------------------------------- */
static int64_t uf_find(int64_t *parent, int64_t x) {
    while (parent[x] != x) {
        parent[x] = parent[parent[x]];
        x = parent[x];
    }
    return x;
}

static void uf_union(int64_t *parent, int64_t a, int64_t b) {
    int64_t ra = uf_find(parent, a), rb = uf_find(parent, b);
    if (ra == rb) return;
    if (ra < rb) parent[rb] = ra; else parent[ra] = rb;
}

static int cmp_i32(const void *a, const void *b) {
    int32_t x = *(const int32_t *)a, y = *(const int32_t *)b;
    return (x > y) - (x < y);
}

typedef struct { int64_t *v; int64_t len, cap; } pairbuf;

static int pb_push(pairbuf *b, int64_t x, int64_t y) {
    if (b->len + 2 > b->cap) {
        int64_t nc = b->cap ? 2 * b->cap : 4096;
        int64_t *nv = (int64_t *)realloc(b->v, sizeof(int64_t) * (size_t)nc);
        if (!nv) return -1;
        b->v = nv;
        b->cap = nc;
    }
    b->v[b->len++] = x;
    b->v[b->len++] = y;
    return 0;
}

static void set_threads(int nthreads) {
#ifdef _OPENMP
    if (nthreads > 0) omp_set_num_threads(nthreads);
#else
    (void)nthreads;
#endif
}

int oracle_num_threads(void) {
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

void oracle_free(void *p) { free(p); }

/*
 * Full DBSCAN by the definition.
 *   X          [n, d] row-major FP64
 *   core       [n]   out: 1 iff core
 *   labels     [n]   out: core -> cluster name; border -> smallest name of
 *                    its set; noise -> -1
 *   border_off [n+1] out: CSR offsets of the border sets (core and noise
 *                    points have empty sets here)
 *   border_ids out: malloc'd array of the set members (free with oracle_free)
 * Returns 0 on success, -1 on allocation failure, -2 on bad arguments.
 */
int oracle_dbscan(const double *X, int64_t n, int d, double eps, int64_t min_pts,
                  int nthreads, uint8_t *core, int32_t *labels,
                  int64_t *border_off, int32_t **border_ids) {
    if (n < 0 || d < 1 || !(eps > 0.0) || min_pts < 1) return -2;
    set_threads(nthreads);
    const double eps2 = eps * eps;
    *border_ids = NULL;
    border_off[0] = 0;
    if (n == 0) {
        *border_ids = (int32_t *)malloc(sizeof(int32_t));
        return *border_ids ? 0 : -1;
    }
    int64_t *ord = order_by_first(X, n, d);
    int64_t *parent = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    int64_t *bcount = (int64_t *)calloc((size_t)n, sizeof(int64_t));
    if (!ord || !parent || !bcount) { free(ord); free(parent); free(bcount); return -1; }

    /* core(p): count every q (p included) that passes within(). */
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t a = 0; a < n; ++a) {
        const double *p = X + ord[a] * d;
        int64_t count = 0;
        for (int64_t b = a; b >= 0; --b) {
            const double *q = X + ord[b] * d;
            if (first_term(p, q) > eps2) break;
            count += within(p, q, d, eps2);
        }
        for (int64_t b = a + 1; b < n; ++b) {
            const double *q = X + ord[b] * d;
            if (first_term(p, q) > eps2) break;
            count += within(p, q, d, eps2);
        }
        core[ord[a]] = (uint8_t)(count >= min_pts);
    }

    /* Clusters: components of the core graph.  Edges are found in chunks by
     * all threads, then applied by one thread. */
    for (int64_t i = 0; i < n; ++i) parent[i] = i;
    int nt = oracle_num_threads();
    pairbuf *bufs = (pairbuf *)calloc((size_t)nt, sizeof(pairbuf));
    if (!bufs) { free(ord); free(parent); free(bcount); return -1; }
    const int64_t chunk = 8192;
    int failed = 0;
    for (int64_t a0 = 0; a0 < n && !failed; a0 += chunk) {
        int64_t a1 = a0 + chunk < n ? a0 + chunk : n;
        for (int t = 0; t < nt; ++t) bufs[t].len = 0;
#pragma omp parallel
        {
#ifdef _OPENMP
            int t = omp_get_thread_num();
#else
            int t = 0;
#endif
#pragma omp for schedule(dynamic, 64)
            for (int64_t a = a0; a < a1; ++a) {
                int64_t pi = ord[a];
                if (!core[pi]) continue;
                const double *p = X + pi * d;
                for (int64_t b = a + 1; b < n; ++b) {
                    int64_t qi = ord[b];
                    const double *q = X + qi * d;
                    if (first_term(p, q) > eps2) break;
                    if (core[qi] && within(p, q, d, eps2))
                        if (pb_push(&bufs[t], pi, qi)) failed = 1;
                }
            }
        }
        for (int t = 0; t < nt; ++t)
            for (int64_t k = 0; k < bufs[t].len; k += 2)
                uf_union(parent, bufs[t].v[k], bufs[t].v[k + 1]);
    }
    for (int t = 0; t < nt; ++t) free(bufs[t].v);
    free(bufs);
    if (failed) { free(ord); free(parent); free(bcount); return -1; }
    for (int64_t i = 0; i < n; ++i)
        labels[i] = core[i] ? (int32_t)uf_find(parent, i) : -1;

    /* Border sets: names of the clusters of core points within eps. */
    int64_t total = 0;
    for (int pass = 0; pass < 2; ++pass) {
        if (pass == 1) {
            for (int64_t i = 0; i < n; ++i) border_off[i + 1] = border_off[i] + bcount[i];
            total = border_off[n];
            *border_ids = (int32_t *)malloc(sizeof(int32_t) * (size_t)(total > 0 ? total : 1));
            if (!*border_ids) { failed = 1; break; }
        }
#pragma omp parallel
        {
            int64_t cap = 64, len;
            int32_t *tmp = (int32_t *)malloc(sizeof(int32_t) * (size_t)cap);
#pragma omp for schedule(dynamic, 256)
            for (int64_t a = 0; a < n; ++a) {
                int64_t pi = ord[a];
                if (core[pi] || !tmp) continue;
                const double *p = X + pi * d;
                len = 0;
                for (int dir = 0; dir < 2; ++dir) {
                    int64_t b = dir == 0 ? a - 1 : a + 1, step = dir == 0 ? -1 : 1;
                    for (; b >= 0 && b < n; b += step) {
                        int64_t qi = ord[b];
                        const double *q = X + qi * d;
                        if (first_term(p, q) > eps2) break;
                        if (!core[qi] || !within(p, q, d, eps2)) continue;
                        if (len == cap) {
                            int32_t *nt2 = (int32_t *)realloc(tmp, sizeof(int32_t) * (size_t)(2 * cap));
                            if (!nt2) { failed = 1; break; }
                            tmp = nt2;
                            cap *= 2;
                        }
                        tmp[len++] = labels[qi];
                    }
                }
                qsort(tmp, (size_t)len, sizeof(int32_t), cmp_i32);
                int64_t u = 0;
                for (int64_t k = 0; k < len; ++k)
                    if (u == 0 || tmp[k] != tmp[u - 1]) tmp[u++] = tmp[k];
                if (pass == 0) {
                    bcount[pi] = u;
                    labels[pi] = u > 0 ? tmp[0] : -1;
                } else {
                    memcpy(*border_ids + border_off[pi], tmp, sizeof(int32_t) * (size_t)u);
                }
            }
            free(tmp);
        }
    }
    free(ord);
    free(parent);
    free(bcount);
    return failed ? -1 : 0;
}

/*
 * Per-point query, straight from the definition: for each sampled index s,
 * count every q in P (self included) with within(X[s], q), scanning all n
 * points.  Used to check single outputs of large runs one by one.
 */
int oracle_sample_counts(const double *X, int64_t n, int d, double eps,
                         const int64_t *samples, int64_t S, int nthreads,
                         int64_t *counts) {
    if (n < 0 || d < 1 || !(eps > 0.0)) return -2;
    set_threads(nthreads);
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(dynamic, 1)
    for (int64_t s = 0; s < S; ++s) {
        const double *p = X + samples[s] * d;
        int64_t c = 0;
        for (int64_t q = 0; q < n; ++q) c += within(p, X + q * d, d, eps2);
        counts[s] = c;
    }
    return 0;
}

/*
 * All q with within(X[p], q), by a scan over all n points, in index order.
 * Writes up to cap indices to out and returns the full count (or -2).
 */
int64_t oracle_neighbors(const double *X, int64_t n, int d, double eps, int64_t p,
                         int64_t *out, int64_t cap) {
    if (n < 0 || d < 1 || !(eps > 0.0) || p < 0 || p >= n) return -2;
    const double eps2 = eps * eps;
    int64_t c = 0;
    for (int64_t q = 0; q < n; ++q)
        if (within(X + p * d, X + q * d, d, eps2)) {
            if (c < cap) out[c] = q;
            ++c;
        }
    return c;
}

/*
 * The predicate of Sec. 2 on given pairs: out[k] = within(X[i_k], X[j_k]) for
 * pairs[2k] = i_k, pairs[2k+1] = j_k.  Used to verify, one by one, pairs that a
 * run claims are within eps (for instance the witnesses of its cluster
 * links).  Returns 0, or -2 for bad arguments (an index outside [0, n)).
 */
int oracle_within_pairs(const double *X, int64_t n, int d, double eps, const int64_t *pairs, int64_t k,
                        int nthreads, uint8_t *out) {
    if (n < 0 || d < 1 || !(eps > 0.0) || k < 0) return -2;
    for (int64_t t = 0; t < 2 * k; ++t)
        if (pairs[t] < 0 || pairs[t] >= n) return -2;
    set_threads(nthreads);
    const double eps2 = eps * eps;
#pragma omp parallel for schedule(static)
    for (int64_t t = 0; t < k; ++t)
        out[t] = (uint8_t)within(X + pairs[2 * t] * d, X + pairs[2 * t + 1] * d, d, eps2);
    return 0;
}
