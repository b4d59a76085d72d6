/*
 * grng_oracle.c -- plain, slow, FP64 CPU oracle for exact RNG / GRNG construction
 * (Foster, Sevilmis, Kimia, "Generalized Relative Neighborhood Graph (GRNG) for
 * Similarity Search", arXiv 2208.10022).
 *
 * TEST INFRASTRUCTURE ONLY.  Nothing in the product library links, includes or
 * calls this file; only the test-suite, the smoke check and the CPU-baseline leg of
 * the benchmark load it.  It shares no code, header, table or constant with the
 * CUDA path.
 *
 * Every function is the plain definition written out, in the paper's notation:
 *   - Eq. 1 (Sec. 1): x1 ~ x2 in RNG(S) iff max(d(x3,x1), d(x3,x2)) >= d(x1,x2)
 *     for every x3 in S; the lune is open, so only a strictly closer x3 blocks.
 *   - Eq. 2 (Sec. 1): pivot domain D(p,r) = { x : d(x,p) <= r }.
 *   - Definition of the GRNG (Sec. 2): p_i ~ p_j iff no p_k satisfies both
 *       d(p_k,p_i) < d(p_i,p_j) - (2 r_i + r_j)
 *       d(p_k,p_j) < d(p_i,p_j) - (r_i + 2 r_j).
 *   - Relative pivot domain (Sec. 3): a fine pivot (pb, rb) lies in D(p, r) iff
 *     d(p, pb) <= r - rb, so a coarse radius is max over its fine members of
 *     d(p, pb) + rb; delta_max(p) is the largest member distance (Sec. 2 Stage VI,
 *     Sec. 3 Stage VI).
 *
 * Canonical arithmetic (this is what "bit-exact" means for the whole project):
 *   - inputs are FP32 and are converted exactly to FP64;
 *   - L2 key  = sum_{k=0..D-1} (x_k - y_k)^2, accumulated in k order, every
 *     operation rounded to nearest, no fused multiply-add (build with
 *     -ffp-contract=off);  L2 distance = sqrt(key) (IEEE, correctly rounded);
 *   - L1 key  = distance = sum_k |x_k - y_k| in the same order;
 *   - RNG and nearest-pivot decisions compare keys;  GRNG decisions compare
 *     distances against t1 = d_ij - (2.0*r_i + r_j) and t2 = d_ij - (r_i + 2.0*r_j),
 *     except when r_i == r_j == 0, where they compare keys (so that the GRNG with
 *     zero radii is exactly the RNG, as the paper remarks after the definition).
 *
 * Readings of points the paper leaves open:
 *   - interceptors x3 in Eq. 1 range over S minus {x1, x2} (x1, x2 themselves can
 *     never be strictly inside their own lune);
 *   - nearest-pivot ties go to the lowest position in the layer's pivot list, and a
 *     pivot is always assigned to itself;
 *   - duplicate points follow Eq. 1 literally: a duplicate pair is linked, and a
 *     duplicate never blocks.
 */
#include <math.h>
#include <omp.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define ORC_L2 0
#define ORC_L1 1

/* OpenMP threads of the parallel loops below: set, and the number in use */
int32_t orc_set_threads(int32_t t) {
    int32_t prev = (int32_t)omp_get_max_threads();
    if (t > 0) omp_set_num_threads(t);
    return prev;
}
int32_t orc_max_threads(void) { return (int32_t)omp_get_max_threads(); }

/* ---- canonical FP64 distances (Eq. 1 metric; L2 or L1) ---------------------- */

double orc_key(const float *a, const float *b, int32_t D, int32_t metric) {
    double acc = 0.0;
    for (int32_t k = 0; k < D; ++k) {
        double t = (double)a[k] - (double)b[k];
        if (metric == ORC_L2) {
            double sq = t * t;
            acc = acc + sq;
        } else {
            acc = acc + fabs(t);
        }
    }
    return acc;
}

double orc_dist(const float *a, const float *b, int32_t D, int32_t metric) {
    double k = orc_key(a, b, D, metric);
    return metric == ORC_L2 ? sqrt(k) : k;
}

/* key matrix of n points (row-major n*n); returns NULL on allocation failure */
static double *key_matrix(const float *X, int64_t n, int32_t D, int32_t metric) {
    double *K = (double *)malloc((size_t)n * (size_t)n * sizeof(double));
    if (!K) return NULL;
#pragma omp parallel for schedule(dynamic, 16)
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = 0; j < n; ++j)
            K[i * n + j] = (i == j) ? 0.0 : orc_key(X + i * D, X + j * D, D, metric);
    return K;
}

/* ---- RNG by Eq. 1, brute force over all triples -------------------------------- */
/* Writes edges (i<j) in lexicographic order into edges[cap][2]; returns the edge
 * count (which may exceed cap: only the first cap are written), or -1 on
 * allocation failure. */
int64_t orc_rng_brute(const float *X, int64_t n, int32_t D, int32_t metric,
                      int32_t *edges, int64_t cap) {
    if (n < 2) return 0;
    double *K = key_matrix(X, n, D, metric);
    if (!K) return -1;
    unsigned char *lnk = (unsigned char *)calloc((size_t)n * (size_t)n, 1);
    if (!lnk) { free(K); return -1; }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double dij = K[i * n + j];
            int blocked = 0;
            for (int64_t k = 0; k < n && !blocked; ++k) {
                if (k == i || k == j) continue;
                double a = K[k * n + i], b = K[k * n + j];
                double m = a > b ? a : b;
                if (m < dij) blocked = 1;           /* strictly inside the open lune */
            }
            lnk[i * n + j] = (unsigned char)!blocked;
        }
    }
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (lnk[i * n + j]) {
                if (cnt < cap) { edges[2 * cnt] = (int32_t)i; edges[2 * cnt + 1] = (int32_t)j; }
                ++cnt;
            }
    free(lnk);
    free(K);
    return cnt;
}

/* ---- exact RNG neighbourhood of one point (Eq. 1), no matrix --------------------
 * Only z with key(x,z) < key(x,y) can lie in lune(x,y), so for each y the
 * candidates z are scanned in increasing key(x,z) and the scan stops at the first
 * blocker or at the first z that is not strictly closer to x than y.
 * Writes neighbour indices (ascending) into nbrs[cap]; returns the count or -1. */
typedef struct { double k; int64_t i; } kv_t;
static int kv_cmp(const void *a, const void *b) {
    const kv_t *p = (const kv_t *)a, *q = (const kv_t *)b;
    if (p->k < q->k) return -1;
    if (p->k > q->k) return 1;
    return (p->i > q->i) - (p->i < q->i);
}
/* Neighbours of x (ascending) into nbrs[cap]; o[n] and is[n] are caller scratch.
 * parallel = 1 spreads the candidates y over the OpenMP threads.  Returns the count. */
static int64_t rng_row_into(const float *X, int64_t n, int32_t D, int32_t metric, int64_t x,
                            int32_t *nbrs, int64_t cap, kv_t *o, unsigned char *is, int parallel) {
    for (int64_t z = 0; z < n; ++z) { o[z].k = orc_key(X + x * D, X + z * D, D, metric); o[z].i = z; }
    qsort(o, (size_t)n, sizeof(kv_t), kv_cmp);
    for (int64_t y = 0; y < n; ++y) is[y] = 0;
#pragma omp parallel for schedule(dynamic, 64) if (parallel)
    for (int64_t p = 0; p < n; ++p) {
        int64_t y = o[p].i;
        if (y == x) continue;
        double dxy = o[p].k;
        int blocked = 0;
        for (int64_t q = 0; q < n && !blocked; ++q) {
            if (!(o[q].k < dxy)) break;             /* z not strictly closer to x */
            int64_t z = o[q].i;
            if (z == x || z == y) continue;
            double dyz = orc_key(X + y * D, X + z * D, D, metric);
            if (dyz < dxy) blocked = 1;            /* max(d(x,z), d(y,z)) < d(x,y) */
        }
        is[y] = (unsigned char)!blocked;
    }
    int64_t cnt = 0;
    for (int64_t y = 0; y < n; ++y)
        if (is[y]) { if (cnt < cap) nbrs[cnt] = (int32_t)y; ++cnt; }
    return cnt;
}

int64_t orc_rng_row(const float *X, int64_t n, int32_t D, int32_t metric, int64_t x,
                    int32_t *nbrs, int64_t cap) {
    kv_t *o = (kv_t *)malloc(sizeof(kv_t) * (size_t)n);
    unsigned char *is = (unsigned char *)malloc((size_t)n);
    if (!o || !is) { free(o); free(is); return -1; }
    int64_t cnt = rng_row_into(X, n, D, metric, x, nbrs, cap, o, is, 1);
    free(o);
    free(is);
    return cnt;
}

/* The exact neighbourhoods of count points xs[] at once (rows spread over the OpenMP
 * threads, each row computed as orc_rng_row computes it).  Row t's neighbours go to
 * nbrs[t * row_cap ...], its count to cnt[t] (a count above row_cap means the row was
 * cut).  Returns 0, or -1 on allocation failure. */
int32_t orc_rng_rows(const float *X, int64_t n, int32_t D, int32_t metric, const int64_t *xs,
                     int64_t count, int32_t *nbrs, int64_t row_cap, int64_t *cnt) {
    int failed = 0;
#pragma omp parallel
    {
        kv_t *o = (kv_t *)malloc(sizeof(kv_t) * (size_t)n);
        unsigned char *is = (unsigned char *)malloc((size_t)n);
        if (!o || !is) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < count; ++t) {
            if (o && is)
                cnt[t] = rng_row_into(X, n, D, metric, xs[t], nbrs + t * row_cap, row_cap, o, is, 0);
        }
        free(o);
        free(is);
    }
    return failed ? -1 : 0;
}

/* ---- RNG search (Sec. 2, Algorithm 1 without Stage VII) ------------------------
 * The RNG neighbours among the n index points X of a query q that does not join the
 * index: x is a neighbour iff no index point z other than x lies strictly inside the
 * open lune of (q, x) (Eq. 1 over X plus q alone).  Other queries are not points of
 * the index, so they never block.  As in rng_row_into, the candidates z are scanned in
 * increasing key(q, z), and only while strictly closer to q than x is.
 * Neighbours (ascending index) into nbrs[cap]; o[n], is[n] are caller scratch. */
static int64_t search_row_into(const float *X, int64_t n, const float *q, int32_t D, int32_t metric,
                               int32_t *nbrs, int64_t cap, kv_t *o, unsigned char *is) {
    for (int64_t z = 0; z < n; ++z) { o[z].k = orc_key(q, X + z * D, D, metric); o[z].i = z; }
    qsort(o, (size_t)n, sizeof(kv_t), kv_cmp);
    for (int64_t p = 0; p < n; ++p) {
        int64_t x = o[p].i;
        double dqx = o[p].k;
        int blocked = 0;
        for (int64_t t = 0; t < n && !blocked; ++t) {
            if (!(o[t].k < dqx)) break;              /* z not strictly closer to q */
            int64_t z = o[t].i;
            if (z == x) continue;
            double dxz = orc_key(X + x * D, X + z * D, D, metric);
            if (dxz < dqx) blocked = 1;             /* max(d(q,z), d(x,z)) < d(q,x) */
        }
        is[x] = (unsigned char)!blocked;
    }
    int64_t cnt = 0;
    for (int64_t x = 0; x < n; ++x)
        if (is[x]) { if (cnt < cap) nbrs[cnt] = (int32_t)x; ++cnt; }
    return cnt;
}

/* The search neighbourhoods of m queries Q[m][D] over the index X[n][D] (queries spread
 * over the OpenMP threads).  Query t's neighbours go to nbrs[t * row_cap ...], its count
 * to cnt[t] (a count above row_cap means the row was cut).  Returns 0, or -1 on
 * allocation failure. */
int32_t orc_rng_search(const float *X, int64_t n, const float *Q, int64_t m, int32_t D, int32_t metric,
                       int32_t *nbrs, int64_t row_cap, int64_t *cnt) {
    int failed = 0;
#pragma omp parallel
    {
        kv_t *o = (kv_t *)malloc(sizeof(kv_t) * (size_t)(n > 0 ? n : 1));
        unsigned char *is = (unsigned char *)malloc((size_t)(n > 0 ? n : 1));
        if (!o || !is) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < m; ++t) {
            if (o && is)
                cnt[t] = search_row_into(X, n, Q + t * D, D, metric, nbrs + t * row_cap, row_cap, o, is);
        }
        free(o);
        free(is);
    }
    return failed ? -1 : 0;
}

/* ---- lune-based beta-skeletons, 1 <= beta <= 2, L2 (Sec. 1: the empty-region graphs
 * that contain the RNG; beta = 1 is the Gabriel graph, beta = 2 the RNG) -------------
 * (x, y) is an edge iff no third point z lies strictly inside both balls of radius
 * beta d(x,y) / 2 centred at (1 - beta/2) x + (beta/2) y and (beta/2) x + (1 - beta/2) y.
 * With lam = beta / 2 and the keys a = d(z,x)^2, b = d(z,y)^2, v = d(x,y)^2, the squared
 * distance of z to the first centre is (1-lam) a + lam b - lam (1-lam) v (Stewart's
 * theorem), so z is inside the first ball iff (1-lam) a + lam b < lam v and inside the
 * second iff lam a + (1-lam) b < lam v.  Canonical FP64: each side as written, the two
 * products first, then their sum.  Edges (i<j) in lexicographic order into edges[cap][2];
 * returns the count (which may exceed cap), -1 on allocation failure, -2 for beta outside
 * [1, 2]. */
int64_t orc_beta_brute(const float *X, int64_t n, int32_t D, double beta, int32_t *edges, int64_t cap) {
    if (!(beta >= 1.0 && beta <= 2.0)) return -2;
    if (n < 2) return 0;
    const double lam = beta / 2.0, mu = 1.0 - lam;
    double *K = key_matrix(X, n, D, ORC_L2);
    if (!K) return -1;
    unsigned char *lnk = (unsigned char *)calloc((size_t)n * (size_t)n, 1);
    if (!lnk) { free(K); return -1; }
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            double v = K[i * n + j];
            double t = lam * v;
            int blocked = 0;
            for (int64_t k = 0; k < n && !blocked; ++k) {
                if (k == i || k == j) continue;
                double a = K[k * n + i], b = K[k * n + j];
                double in1 = mu * a + lam * b;             /* against the first centre */
                double in2 = lam * a + mu * b;             /* against the second centre */
                if (in1 < t && in2 < t) blocked = 1;      /* strictly inside both balls */
            }
            lnk[i * n + j] = (unsigned char)!blocked;
        }
    }
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i)
        for (int64_t j = i + 1; j < n; ++j)
            if (lnk[i * n + j]) {
                if (cnt < cap) { edges[2 * cnt] = (int32_t)i; edges[2 * cnt + 1] = (int32_t)j; }
                ++cnt;
            }
    free(lnk);
    free(K);
    return cnt;
}

/* Witness check (Eq. 1): 1 if z is a point other than x and y lying strictly inside
 * the open lune of (x, y), i.e. max(d(x,z), d(y,z)) < d(x,y), so that z proves the pair
 * is not an RNG edge; else 0. */
int32_t orc_verify_witness(const float *X, int32_t D, int32_t metric, int64_t x, int64_t y, int64_t z) {
    if (z == x || z == y) return 0;
    double dxy = orc_key(X + x * D, X + y * D, D, metric);
    double a = orc_key(X + x * D, X + z * D, D, metric);
    double b = orc_key(X + y * D, X + z * D, D, metric);
    double m = a > b ? a : b;
    return m < dxy ? 1 : 0;
}

/* A minimum spanning tree of the complete graph on the n points under canonical keys
 * (Prim's algorithm, O(n^2 D)).  Every minimum spanning tree lies in the RNG: an edge
 * with a point strictly inside its lune could be swapped for a strictly lighter one
 * (Sec. 1, the RNG contains the MST).  Writes the n-1 tree edges (parent, child) into
 * edges[n-1][2]; returns n-1, or -1 on allocation failure. */
int64_t orc_emst(const float *X, int64_t n, int32_t D, int32_t metric, int32_t *edges) {
    if (n < 2) return 0;
    int nt = omp_get_max_threads();
    double *best = (double *)malloc(sizeof(double) * (size_t)n);
    int64_t *from = (int64_t *)malloc(sizeof(int64_t) * (size_t)n);
    unsigned char *in = (unsigned char *)calloc((size_t)n, 1);
    double *tmin = (double *)malloc(sizeof(double) * (size_t)nt);
    int64_t *targ = (int64_t *)malloc(sizeof(int64_t) * (size_t)nt);
    if (!best || !from || !in || !tmin || !targ) {
        free(best); free(from); free(in); free(tmin); free(targ);
        return -1;
    }
    for (int64_t v = 0; v < n; ++v) { best[v] = INFINITY; from[v] = 0; }
    int64_t u = 0;                                   /* the tree grows from point 0 */
    for (int64_t e = 0; e < n; ++e) {
        in[u] = 1;
        if (e > 0) {
            edges[2 * (e - 1)] = (int32_t)from[u];
            edges[2 * (e - 1) + 1] = (int32_t)u;
        }
        if (e == n - 1) break;
        /* relax every point outside the tree through u, and find the closest one */
#pragma omp parallel num_threads(nt)
        {
            int t = omp_get_thread_num();
            double lb = INFINITY;
            int64_t la = -1;
#pragma omp for schedule(static)
            for (int64_t v = 0; v < n; ++v) {
                if (in[v]) continue;
                double k = orc_key(X + u * D, X + v * D, D, metric);
                if (k < best[v]) { best[v] = k; from[v] = u; }
                if (la < 0 || best[v] < lb) { lb = best[v]; la = v; }
            }
            tmin[t] = lb;
            targ[t] = la;
        }
        int64_t nu = -1;
        double bu = INFINITY;
        for (int t = 0; t < nt; ++t)      /* threads own increasing ranges: ties keep the lowest */
            if (targ[t] >= 0 && (nu < 0 || tmin[t] < bu)) { nu = targ[t]; bu = tmin[t]; }
        u = nu;
    }
    free(best); free(from); free(in); free(tmin); free(targ);
    return n - 1;
}

/* ---- GRNG by its definition (Sec. 2) ------------------------------------------ */
/* One pivot triple: 1 if p_k lies in the generalized lune of (p_i, p_j).
 * dd[] are distances, kk[] keys (used only when r_i == r_j == 0). */
static int g_blocks(double dij, double dki, double dkj, double kij, double kki,
                    double kkj, double ri, double rj) {
    if (ri == 0.0 && rj == 0.0) return (kki < kij) && (kkj < kij);
    double t1 = dij - (2.0 * ri + rj);
    double t2 = dij - (ri + 2.0 * rj);
    return (dki < t1) && (dkj < t2);
}

/* ---- GRNG Stage VII: a new pivot joins a layer (Sec. 3, the GRNG's Stage VII) --------
 * P[m+1][D] holds the layer's pivots with the new one last, r[m+1] their radii, links[m*m]
 * the GRNG of the first m ([i*m + j], i < j).  Writes out[(m+1)*(m+1)] ([i*(m+1) + j], i < j),
 * the GRNG of all m+1: an old link survives unless the new pivot lies in its generalized lune
 * (a non-link stays one: the new pivot only adds interceptors), and the new pivot's own links
 * are decided over all m+1 pivots.  The new pivot k can block a link (i, j) only when
 * d(k, i) < d(i, j) - (2 r_i + r_j) <= mu_i - 2 r_i, mu_i the longest link at p_i (and likewise
 * at j), so a link is tested only when both ends lie that close to k.  stats (may be NULL):
 * [0] old links tested, [1] old links removed, [2] links of the new pivot.  Returns 0 or -1. */
int32_t orc_grng_insert_pivot(const float *P, const double *r, int64_t m, int32_t D, int32_t metric,
                              const unsigned char *links, unsigned char *out, int64_t *stats) {
    const int64_t m1 = m + 1;
    const float *pk = P + m * D;
    double *mu = (double *)calloc((size_t)(m > 0 ? m : 1), sizeof(double));
    double *dk = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    double *kk = (double *)malloc(sizeof(double) * (size_t)(m > 0 ? m : 1));
    if (!mu || !dk || !kk) { free(mu); free(dk); free(kk); return -1; }
    for (int64_t i = 0; i < m; ++i) {
        kk[i] = orc_key(pk, P + i * D, D, metric);
        dk[i] = metric == ORC_L2 ? sqrt(kk[i]) : kk[i];
    }
    for (int64_t i = 0; i < m; ++i)  /* longest link at each old pivot */
        for (int64_t j = i + 1; j < m; ++j)
            if (links[i * m + j]) {
                double d = orc_dist(P + i * D, P + j * D, D, metric);
                if (d > mu[i]) mu[i] = d;
                if (d > mu[j]) mu[j] = d;
            }
    int64_t tested = 0, removed = 0, added = 0;
    memset(out, 0, (size_t)m1 * (size_t)m1);
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = i + 1; j < m; ++j) {
            if (!links[i * m + j]) continue;
            int keep = 1;
            /* reachable from k at both ends (with a margin far above the FP64 rounding) */
            double ri = r[i], rj = r[j];
            double bi = mu[i] - 2.0 * ri, bj = mu[j] - 2.0 * rj;
            int near_i = dk[i] < bi + 1e-9 * (dk[i] + mu[i] + 2.0 * ri);
            int near_j = dk[j] < bj + 1e-9 * (dk[j] + mu[j] + 2.0 * rj);
            if (near_i && near_j) {
                ++tested;
                double kij = orc_key(P + i * D, P + j * D, D, metric);
                double dij = metric == ORC_L2 ? sqrt(kij) : kij;
                if (g_blocks(dij, dk[i], dk[j], kij, kk[i], kk[j], ri, rj)) { keep = 0; ++removed; }
            }
            out[i * m1 + j] = (unsigned char)keep;
        }
    for (int64_t i = 0; i < m; ++i) {  /* the new pivot's links, by the definition */
        double kij = kk[i], dij = dk[i];
        int blocked = 0;
        for (int64_t q = 0; q < m && !blocked; ++q) {
            if (q == i) continue;
            double kqi = orc_key(P + q * D, P + i * D, D, metric);
            double kqk = orc_key(P + q * D, pk, D, metric);
            double dqi = metric == ORC_L2 ? sqrt(kqi) : kqi, dqk = metric == ORC_L2 ? sqrt(kqk) : kqk;
            blocked = g_blocks(dij, dqi, dqk, kij, kqi, kqk, r[i], r[m]);
        }
        out[i * m1 + m] = (unsigned char)!blocked;
        added += !blocked;
    }
    if (stats) { stats[0] = tested; stats[1] = removed; stats[2] = added; }
    free(mu); free(dk); free(kk);
    return 0;
}

/* Brute GRNG over m pivots given by their coordinates P[m][D] and radii r[m].
 * Edges i<j in lexicographic order; returns count (may exceed cap) or -1. */
int64_t orc_grng_brute(const float *P, const double *r, int64_t m, int32_t D,
                       int32_t metric, int32_t *edges, int64_t cap) {
    if (m < 2) return 0;
    double *K = key_matrix(P, m, D, metric);
    if (!K) return -1;
    double *Dm = (double *)malloc((size_t)m * (size_t)m * sizeof(double));
    unsigned char *lnk = (unsigned char *)calloc((size_t)m * (size_t)m, 1);
    if (!Dm || !lnk) { free(K); free(Dm); free(lnk); return -1; }
    for (int64_t t = 0; t < m * m; ++t) Dm[t] = metric == ORC_L2 ? sqrt(K[t]) : K[t];
#pragma omp parallel for schedule(dynamic, 4)
    for (int64_t i = 0; i < m; ++i) {
        for (int64_t j = i + 1; j < m; ++j) {
            int blocked = 0;
            for (int64_t k = 0; k < m && !blocked; ++k) {
                if (k == i || k == j) continue;
                blocked = g_blocks(Dm[i * m + j], Dm[k * m + i], Dm[k * m + j], K[i * m + j],
                                   K[k * m + i], K[k * m + j], r[i], r[j]);
            }
            lnk[i * m + j] = (unsigned char)!blocked;
        }
    }
    int64_t cnt = 0;
    for (int64_t i = 0; i < m; ++i)
        for (int64_t j = i + 1; j < m; ++j)
            if (lnk[i * m + j]) {
                if (cnt < cap) { edges[2 * cnt] = (int32_t)i; edges[2 * cnt + 1] = (int32_t)j; }
                ++cnt;
            }
    free(lnk);
    free(Dm);
    free(K);
    return cnt;
}

/* GRNG neighbourhood of pivot i (positions j != i, ascending), by the definition.
 * For each j only the p_k with d(p_k,p_i) < t1 (resp. key < key_ij) can satisfy the
 * first condition, so candidates k are scanned in increasing d(p_k,p_i) and the
 * scan stops once that first condition fails.  Returns count or -1. */
int64_t orc_grng_row(const float *P, const double *r, int64_t m, int32_t D, int32_t metric,
                     int64_t i, int32_t *nbrs, int64_t cap) {
    kv_t *o = (kv_t *)malloc(sizeof(kv_t) * (size_t)m);
    unsigned char *is = (unsigned char *)calloc((size_t)m, 1);
    if (!o || !is) { free(o); free(is); return -1; }
    for (int64_t k = 0; k < m; ++k) { o[k].k = orc_key(P + i * D, P + k * D, D, metric); o[k].i = k; }
    qsort(o, (size_t)m, sizeof(kv_t), kv_cmp);
    double *kik = (double *)malloc(sizeof(double) * (size_t)m);
    if (!kik) { free(o); free(is); return -1; }
    for (int64_t q = 0; q < m; ++q) kik[o[q].i] = o[q].k;
#pragma omp parallel for schedule(dynamic, 64)
    for (int64_t j = 0; j < m; ++j) {
        if (j == i) continue;
        double kij = kik[j];
        double dij = metric == ORC_L2 ? sqrt(kij) : kij;
        int zero = (r[i] == 0.0 && r[j] == 0.0);
        double t1 = dij - (2.0 * r[i] + r[j]);
        int blocked = 0;
        for (int64_t q = 0; q < m && !blocked; ++q) {
            int64_t k = o[q].i;
            double kki = o[q].k;
            double dki = metric == ORC_L2 ? sqrt(kki) : kki;
            if (zero ? !(kki < kij) : !(dki < t1)) break;   /* first condition fails */
            if (k == i || k == j) continue;
            double kkj = orc_key(P + k * D, P + j * D, D, metric);
            double dkj = metric == ORC_L2 ? sqrt(kkj) : kkj;
            blocked = g_blocks(dij, dki, dkj, kij, kki, kkj, r[i], r[j]);
        }
        is[j] = (unsigned char)!blocked;
    }
    int64_t cnt = 0;
    for (int64_t j = 0; j < m; ++j)
        if (is[j]) { if (cnt < cap) nbrs[cnt] = (int32_t)j; ++cnt; }
    free(kik);
    free(o);
    free(is);
    return cnt;
}

/* ---- pivot layer: assignment, radii, delta_max (Eq. 2; Sec. 3) ------------------
 * members[nmem]   point indices of the layer's members (all points for the finest
 *                 layer; the next finer layer's pivots otherwise)
 * member_r[nmem]  their radii (NULL: all zero, i.e. exemplars)
 * piv[m]          point indices of the layer's pivots
 * Outputs (any may be NULL):
 *   assign[nmem]  position (0..m-1) of the nearest pivot by canonical key, ties to the
 *                 lowest position; a member that is itself a pivot gets that pivot
 *   dist[nmem]    d(member, its pivot) (FP64 distance)
 *   radius[m]     max over assigned members of dist + member_r   (0 if none)
 *   delta_max[m]  max over assigned members of dist               (0 if none)
 * Returns 0, or -1 on allocation failure. */
int32_t orc_assign(const float *X, int32_t D, int32_t metric, const int32_t *members,
                   int64_t nmem, const double *member_r, const int32_t *piv, int32_t m,
                   int32_t *assign, double *dist, double *radius, double *delta_max) {
    int32_t *as = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nmem > 0 ? nmem : 1));
    double *ds = (double *)malloc(sizeof(double) * (size_t)(nmem > 0 ? nmem : 1));
    if (!as || !ds) { free(as); free(ds); return -1; }
#pragma omp parallel for schedule(dynamic, 256)
    for (int64_t t = 0; t < nmem; ++t) {
        const float *x = X + (int64_t)members[t] * D;
        int32_t best = -1;
        double bk = 0.0;
        for (int32_t p = 0; p < m; ++p) {
            if (piv[p] == members[t]) { best = p; break; }  /* a pivot owns itself */
        }
        if (best < 0) {
            for (int32_t p = 0; p < m; ++p) {
                double k = orc_key(x, X + (int64_t)piv[p] * D, D, metric);
                if (best < 0 || k < bk) { best = p; bk = k; }
            }
        }
        as[t] = best;
        ds[t] = orc_dist(x, X + (int64_t)piv[best] * D, D, metric);
    }
    /* delta_max(p) is the largest d(p, member) over the members assigned to p, without
     * the member radii (Sec. 2 Stage VI bounds d(p, z) for the exemplars below p by it);
     * the radius adds each member's own radius (relative pivot domain, Sec. 3), so on a
     * coarse layer the two differ. */
    if (radius || delta_max) {
        for (int32_t p = 0; p < m; ++p) {
            if (radius) radius[p] = 0.0;
            if (delta_max) delta_max[p] = 0.0;
        }
        for (int64_t t = 0; t < nmem; ++t) {
            double rr = ds[t] + (member_r ? member_r[t] : 0.0);
            if (radius && rr > radius[as[t]]) radius[as[t]] = rr;
            if (delta_max && ds[t] > delta_max[as[t]]) delta_max[as[t]] = ds[t];
        }
    }
    if (assign) memcpy(assign, as, sizeof(int32_t) * (size_t)nmem);
    if (dist) memcpy(dist, ds, sizeof(double) * (size_t)nmem);
    free(as);
    free(ds);
    return 0;
}
