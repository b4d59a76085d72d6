/*
 * guided_oracle.c -- the paper's pivot-guided exact RNG construction, plain FP64 on the CPU
 * (Foster, Sevilmis, Kimia, arXiv 2208.10022, Secs. 2 and 3).
 *
 * TEST INFRASTRUCTURE ONLY, like grng_oracle.c: nothing in the product library links or
 * calls it, and it shares no code with the CUDA path.  It is an independent second route to
 * the RNG of Eq. 1, following the method's stages instead of the definition, so that the two
 * CPU routes can be checked against each other (tests) and the method's own cost -- distance
 * computations, the measure the paper reports -- can be timed on the host.
 *
 * Steps, in the paper's order:
 *   1. Pivot layers, finest first (Eq. 2; relative pivot domains, Sec. 3): every member joins
 *      its nearest pivot; radius = max(d + member radius), delta_max = max d.
 *   2. GRNG of every layer, coarsest first.  The top layer by the definition over all pairs
 *      (Sec. 2).  A lower layer only over the pairs whose parents are equal or linked
 *      (Theorem 2), the interceptors restricted by Prop. GRNG_S6: the children of a coarse
 *      pivot c cannot satisfy the first condition when d(c, p_i) - delta_max(c) >= t1, nor the
 *      second when d(c, p_j) - delta_max(c) >= t2.
 *   3. RNG: the exemplar pairs whose finest pivots are equal or linked (Stage I, Theorem 1).
 *      For each x the finest pivots are visited in increasing d(x, p); the pivot itself is an
 *      interceptor (Stage IV), and its members are tested unless Prop. 4 excludes the domain
 *      (d(x, p) - delta_max(p) >= d(x, y) or d(y, p) - delta_max(p) >= d(x, y), Stage VI).
 *      The visit ends once d(x, p) - (the largest delta_max) >= d(x, y): no member of that
 *      pivot or of any farther one can be closer to x than y.
 *
 * Rounding.  Every graph decision is the canonical FP64 comparison of the definitions (the
 * same as grng_oracle.c).  The prunings above are exact in the reals; in FP64 they are taken
 * only with a relative margin of 2^-30 of the quantities involved, far above the rounding of
 * sums of a few hundred terms, and the guidance graph that restricts candidates (Theorems 1
 * and 2) calls a pair non-linked only when some blocker clears both thresholds by that margin.
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define G_L2 0
#define G_MARGIN 9.313225746154785e-10 /* 2^-30 */

static double g_key(const float *a, const float *b, int32_t D, int32_t metric) {
    double acc = 0.0;
    for (int32_t k = 0; k < D; ++k) {
        double t = (double)a[k] - (double)b[k];
        if (metric == G_L2) {
            double sq = t * t;
            acc = acc + sq;
        } else {
            acc = acc + fabs(t);
        }
    }
    return acc;
}
static double g_dist_of(double key, int32_t metric) { return metric == G_L2 ? sqrt(key) : key; }

typedef struct {
    int32_t m;
    const int32_t *piv;   /* point indices */
    int32_t *assign;      /* members -> position */
    double *mdist;        /* member distances */
    double *radius, *dmax;
    int32_t *coff, *cidx; /* CSR of members per pivot (member positions) */
    unsigned char *gx;    /* GRNG by the definition, m x m */
    unsigned char *gg;    /* guidance: not non-linked with the margin */
} g_layer;

/* 1: p_k blocks (p_i, p_j) by the definition; 2: also with the margin */
static int g_block(double kij, double kki, double kkj, double ri, double rj, int32_t metric) {
    if (ri == 0.0 && rj == 0.0) {
        double mx = kki > kkj ? kki : kkj;
        int b = mx < kij;
        int g = (kij - mx) > G_MARGIN * kij;
        return b | ((b && g) << 1);
    }
    double dij = g_dist_of(kij, metric), dki = g_dist_of(kki, metric), dkj = g_dist_of(kkj, metric);
    double t1 = dij - (2.0 * ri + rj);
    double t2 = dij - (ri + 2.0 * rj);
    int b = (dki < t1) && (dkj < t2);
    double m1 = t1 - dki, m2 = t2 - dkj, mm = m1 < m2 ? m1 : m2;
    int g = b && mm > G_MARGIN * (dij + 2.0 * ri + 2.0 * rj);
    return b | (g << 1);
}

static void g_members(g_layer *L, int64_t nmem) {
    L->coff = (int32_t *)calloc((size_t)L->m + 1, sizeof(int32_t));
    L->cidx = (int32_t *)malloc(sizeof(int32_t) * (size_t)(nmem > 0 ? nmem : 1));
    for (int64_t t = 0; t < nmem; ++t) L->coff[L->assign[t] + 1]++;
    for (int32_t p = 0; p < L->m; ++p) L->coff[p + 1] += L->coff[p];
    int32_t *cur = (int32_t *)malloc(sizeof(int32_t) * (size_t)L->m);
    memcpy(cur, L->coff, sizeof(int32_t) * (size_t)L->m);
    for (int64_t t = 0; t < nmem; ++t) L->cidx[cur[L->assign[t]]++] = (int32_t)t;
    free(cur);
}

/* nearest pivot (ties to the lowest position, a pivot owns itself), distances, radii */
static void g_assign(const float *X, int32_t D, int32_t metric, const int32_t *members, int64_t nmem,
                     const double *mem_r, g_layer *L, int64_t *ndist) {
    int64_t cnt = 0;
#pragma omp parallel for schedule(dynamic, 64) reduction(+ : cnt)
    for (int64_t t = 0; t < nmem; ++t) {
        int32_t best = -1;
        double bk = 0.0;
        for (int32_t p = 0; p < L->m; ++p)
            if (L->piv[p] == members[t]) { best = p; break; }
        if (best < 0) {
            for (int32_t p = 0; p < L->m; ++p) {
                double k = g_key(X + (int64_t)members[t] * D, X + (int64_t)L->piv[p] * D, D, metric);
                ++cnt;
                if (best < 0 || k < bk) { best = p; bk = k; }
            }
        }
        L->assign[t] = best;
        L->mdist[t] = g_dist_of(g_key(X + (int64_t)members[t] * D, X + (int64_t)L->piv[best] * D, D, metric), metric);
    }
    *ndist += cnt;
    for (int32_t p = 0; p < L->m; ++p) L->radius[p] = L->dmax[p] = 0.0;
    for (int64_t t = 0; t < nmem; ++t) {
        double rr = L->mdist[t] + (mem_r ? mem_r[t] : 0.0);
        if (rr > L->radius[L->assign[t]]) L->radius[L->assign[t]] = rr;
        if (L->mdist[t] > L->dmax[L->assign[t]]) L->dmax[L->assign[t]] = L->mdist[t];
    }
    g_members(L, nmem);
}

/* GRNG of layer L (pivots' keys to each other computed on demand); parents: the coarser
 * layer (or NULL for the top layer) with this layer's assignment to it */
static void g_link(const float *X, int32_t D, int32_t metric, g_layer *L, const g_layer *C,
                   const int32_t *par, int64_t *ndist) {
    const int32_t m = L->m;
    L->gx = (unsigned char *)calloc((size_t)m * (size_t)m, 1);
    L->gg = (unsigned char *)calloc((size_t)m * (size_t)m, 1);
    int64_t cnt = 0;
#pragma omp parallel for schedule(dynamic, 4) reduction(+ : cnt)
    for (int32_t i = 0; i < m; ++i) {
        const float *pi = X + (int64_t)L->piv[i] * D;
        for (int32_t j = i + 1; j < m; ++j) {
            if (C) {  /* Theorem 2: parents equal or linked in the guidance graph */
                int32_t a = par[i], b = par[j];
                if (a != b && !C->gg[(int64_t)(a < b ? a : b) * C->m + (a < b ? b : a)]) continue;
            }
            const float *pj = X + (int64_t)L->piv[j] * D;
            double kij = g_key(pi, pj, D, metric);
            ++cnt;
            double ri = L->radius[i], rj = L->radius[j];
            double dij = g_dist_of(kij, metric);
            double t1 = dij - (2.0 * ri + rj), t2 = dij - (ri + 2.0 * rj);
            int res = 0;
            if (!C) {
                for (int32_t k = 0; k < m && !(res & 2); ++k) {
                    if (k == i || k == j) continue;
                    const float *pk = X + (int64_t)L->piv[k] * D;
                    res |= g_block(kij, g_key(pk, pi, D, metric), g_key(pk, pj, D, metric), ri, rj, metric);
                    cnt += 2;
                }
            } else {
                for (int32_t c = 0; c < C->m && !(res & 2); ++c) {
                    /* Prop. GRNG_S6: no child of c can satisfy a condition whose bound fails */
                    const float *pc = X + (int64_t)C->piv[c] * D;
                    double dci = g_dist_of(g_key(pc, pi, D, metric), metric);
                    double dcj = g_dist_of(g_key(pc, pj, D, metric), metric);
                    cnt += 2;
                    double dm = C->dmax[c];
                    if (dci - dm >= t1 + G_MARGIN * (dci + dm + fabs(t1))) continue;
                    if (dcj - dm >= t2 + G_MARGIN * (dcj + dm + fabs(t2))) continue;
                    for (int32_t q = C->coff[c]; q < C->coff[c + 1] && !(res & 2); ++q) {
                        int32_t k = C->cidx[q];  /* members of c are this layer's positions */
                        if (k == i || k == j) continue;
                        const float *pk = X + (int64_t)L->piv[k] * D;
                        res |= g_block(kij, g_key(pk, pi, D, metric), g_key(pk, pj, D, metric), ri, rj, metric);
                        cnt += 2;
                    }
                }
            }
            if (!(res & 1)) L->gx[(int64_t)i * m + j] = 1;
            if (!(res & 2)) L->gg[(int64_t)i * m + j] = 1;
        }
    }
    *ndist += cnt;
}

typedef struct { double d; int32_t p; } g_dp;
static int g_dp_cmp(const void *a, const void *b) {
    const g_dp *x = (const g_dp *)a, *y = (const g_dp *)b;
    if (x->d < y->d) return -1;
    if (x->d > y->d) return 1;
    return (x->p > y->p) - (x->p < y->p);
}

/* Exact RNG by the pivot-guided method.  layer_piv holds the L layers' pivot indices
 * concatenated, coarsest first (nested, as in grng_oracle.c's orc_assign callers);
 * layer_m their sizes.  Edges (i < j, lexicographic) go to edges[cap][2]; the count is
 * returned (may exceed cap), or -1 on allocation failure.  stats (may be NULL):
 * [0] distance computations, [1] candidate exemplar pairs, [2] member tests (Stage VI). */
int64_t orc_rng_guided(const float *X, int64_t n, int32_t D, int32_t metric, const int32_t *layer_piv,
                       const int32_t *layer_m, int32_t L, int32_t *edges, int64_t cap, int64_t *stats) {
    if (n < 2 || L < 1) return 0;
    g_layer *Ls = (g_layer *)calloc((size_t)L, sizeof(g_layer));
    int64_t ndist = 0, ncand = 0, nmemt = 0;
    int64_t off = 0;
    for (int32_t l = 0; l < L; ++l) { Ls[l].m = layer_m[l]; Ls[l].piv = layer_piv + off; off += layer_m[l]; }
    /* 1. layers, finest first */
    int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    for (int64_t t = 0; t < n; ++t) members[t] = (int32_t)t;
    const int32_t *mem = members;
    int64_t nmem = n;
    const double *mem_r = NULL;
    for (int32_t l = L - 1; l >= 0; --l) {
        g_layer *Y = &Ls[l];
        Y->assign = (int32_t *)malloc(sizeof(int32_t) * (size_t)nmem);
        Y->mdist = (double *)malloc(sizeof(double) * (size_t)nmem);
        Y->radius = (double *)malloc(sizeof(double) * (size_t)Y->m);
        Y->dmax = (double *)malloc(sizeof(double) * (size_t)Y->m);
        g_assign(X, D, metric, mem, nmem, mem_r, Y, &ndist);
        mem = Y->piv;
        nmem = Y->m;
        mem_r = Y->radius;
    }
    /* 2. GRNGs, coarsest first */
    for (int32_t l = 0; l < L; ++l)
        g_link(X, D, metric, &Ls[l], l ? &Ls[l - 1] : NULL, l ? Ls[l - 1].assign : NULL, &ndist);
    /* 3. exemplar pairs of equal or linked finest domains, tested stage by stage */
    const g_layer *F = &Ls[L - 1];
    const int32_t M = F->m;
    double dmax_all = 0.0;
    for (int32_t p = 0; p < M; ++p) if (F->dmax[p] > dmax_all) dmax_all = F->dmax[p];
    int32_t **nbr = (int32_t **)calloc((size_t)n, sizeof(int32_t *));  /* neighbours y > x of each x */
    int32_t *nbc = (int32_t *)calloc((size_t)n, sizeof(int32_t));
    if (!nbr || !nbc) return -1;
#pragma omp parallel for schedule(dynamic, 8) reduction(+ : ndist, ncand, nmemt)
    for (int64_t x = 0; x < n; ++x) {
        int32_t cap_x = 0;
        const float *px = X + x * D;
        g_dp *order = (g_dp *)malloc(sizeof(g_dp) * (size_t)M);
        for (int32_t p = 0; p < M; ++p) {
            order[p].d = g_dist_of(g_key(px, X + (int64_t)F->piv[p] * D, D, metric), metric);
            order[p].p = p;
        }
        ndist += M;
        qsort(order, (size_t)M, sizeof(g_dp), g_dp_cmp);
        const int32_t ax = F->assign[x];
        for (int64_t y = x + 1; y < n; ++y) {
            const int32_t ay = F->assign[y];
            if (ax != ay && !F->gg[(int64_t)(ax < ay ? ax : ay) * M + (ax < ay ? ay : ax)]) continue;  /* Thm 1 */
            ++ncand;
            const float *py = X + y * D;
            const double kxy = g_key(px, py, D, metric), dxy = g_dist_of(kxy, metric);
            ++ndist;
            int blocked = 0;
            for (int32_t q = 0; q < M && !blocked; ++q) {
                const int32_t p = order[q].p;
                const double dxp = order[q].d, dm = F->dmax[p];
                /* every later pivot is at least as far: no member of theirs is closer to x than y */
                if (dxp - dmax_all >= dxy + G_MARGIN * (dxp + dmax_all + dxy)) break;
                const float *pp = X + (int64_t)F->piv[p] * D;
                /* Stage IV: the pivot itself */
                const int64_t pid = F->piv[p];
                double kyp = -1.0;
                if (pid != x && pid != y) {
                    const double kxp = g_key(px, pp, D, metric);
                    kyp = g_key(py, pp, D, metric);
                    ndist += 2;
                    if ((kxp > kyp ? kxp : kyp) < kxy) { blocked = 1; break; }
                }
                /* Prop. 4: no member of p lies in the lune when either bound fails */
                if (dxp - dm >= dxy + G_MARGIN * (dxp + dm + dxy)) continue;
                if (kyp < 0.0) { kyp = g_key(py, pp, D, metric); ++ndist; }
                const double dyp = g_dist_of(kyp, metric);
                if (dyp - dm >= dxy + G_MARGIN * (dyp + dm + dxy)) continue;
                /* Stage VI: the members of p */
                for (int32_t t = F->coff[p]; t < F->coff[p + 1] && !blocked; ++t) {
                    const int64_t z = F->cidx[t];
                    if (z == x || z == y || z == pid) continue;
                    const double kxz = g_key(px, X + z * D, D, metric);
                    const double kyz = g_key(py, X + z * D, D, metric);
                    ndist += 2;
                    ++nmemt;
                    if ((kxz > kyz ? kxz : kyz) < kxy) blocked = 1;  /* strictly inside the open lune */
                }
            }
            if (!blocked) {
                if (nbc[x] == cap_x) {
                    cap_x = cap_x ? 2 * cap_x : 16;
                    nbr[x] = (int32_t *)realloc(nbr[x], sizeof(int32_t) * (size_t)cap_x);
                }
                nbr[x][nbc[x]++] = (int32_t)y;  /* ascending y */
            }
        }
        free(order);
    }
    int64_t cnt = 0;
    for (int64_t i = 0; i < n; ++i) {
        for (int32_t t = 0; t < nbc[i]; ++t) {
            if (cnt < cap) { edges[2 * cnt] = (int32_t)i; edges[2 * cnt + 1] = nbr[i][t]; }
            ++cnt;
        }
        free(nbr[i]);
    }
    if (stats) { stats[0] = ndist; stats[1] = ncand; stats[2] = nmemt; }
    free(nbr);
    free(nbc);
    free(members);
    for (int32_t l = 0; l < L; ++l) {
        free(Ls[l].assign); free(Ls[l].mdist); free(Ls[l].radius); free(Ls[l].dmax);
        free(Ls[l].coff); free(Ls[l].cidx); free(Ls[l].gx); free(Ls[l].gg);
    }
    free(Ls);
    return cnt;
}

/* ---- Stage I candidates under two membership rules (Sec. 2) --------------------------
 * One pivot layer piv[m] over the points X[n].  Rule A (this project's, readings 4-5): every
 * point joins its nearest pivot, whose radius is the largest member distance (Eq. 2).
 * Rule B (the paper's uniform radius): every pivot within distance r of a point is a parent of
 * it, all radii are r.  Each rule's GRNG is the definition over all pivot pairs, with the
 * guidance margin.  Theorem 1 holds for every parent pair, so under rule B a pair (x, y) stays
 * a candidate only when each parent of x and each parent of y are equal or linked; a point
 * without a parent restricts nothing.  With promote = 1, rule B first makes every point that
 * has no pivot within r a pivot itself, in index order (a new point with no parent becomes a
 * pivot, Sec. 2), so that every point has a parent.
 * cand_a / cand_b (n*n bytes each, may be NULL) receive the candidate flags of the pairs i < j
 * at [i*n + j].  stats (may be NULL): [0] candidates under A, [1] under B, [2] points without a
 * parent under B, [3] parent memberships under B (sum over the points), [4] pivots under B,
 * [5] candidates under rule A on B's pivots (the two rules at equal pivot sets).
 * Returns 0, -1 on allocation failure. */
int32_t orc_candidates_rules(const float *X, int64_t n, int32_t D, int32_t metric, const int32_t *piv0,
                             int32_t m0, double r, int32_t promote, unsigned char *cand_a, unsigned char *cand_b,
                             int64_t *stats) {
    if (m0 < 1) return -1;
    /* rule B's pivots: the given ones, then (promote) every point not covered by them yet */
    int32_t *pivb = (int32_t *)malloc(sizeof(int32_t) * (size_t)(m0 + (n > 0 ? n : 1)));
    if (!pivb) return -1;
    memcpy(pivb, piv0, sizeof(int32_t) * (size_t)m0);
    int32_t mb = m0;
    if (promote)
        for (int64_t x = 0; x < n; ++x) {
            int covered = 0;
            for (int32_t p = 0; p < mb && !covered; ++p)
                covered = g_dist_of(g_key(X + x * D, X + (int64_t)pivb[p] * D, D, metric), metric) <= r;
            if (!covered) pivb[mb++] = (int32_t)x;
        }
    const int32_t *piv = piv0;
    const int32_t m = m0;
    g_layer A, B;
    memset(&A, 0, sizeof(A));
    memset(&B, 0, sizeof(B));
    A.m = m;
    A.piv = piv;
    B.m = mb;
    B.piv = pivb;
    int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    A.assign = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
    A.mdist = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
    A.radius = (double *)malloc(sizeof(double) * (size_t)m);
    A.dmax = (double *)malloc(sizeof(double) * (size_t)m);
    B.radius = (double *)malloc(sizeof(double) * (size_t)mb);
    B.dmax = (double *)malloc(sizeof(double) * (size_t)mb);
    int32_t *pcnt = (int32_t *)calloc((size_t)(n > 0 ? n : 1), sizeof(int32_t));
    int32_t *plist = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1) * (size_t)mb);
    if (!members || !A.assign || !A.mdist || !A.radius || !A.dmax || !B.radius || !B.dmax || !pcnt || !plist) {
        free(members); free(A.assign); free(A.mdist); free(A.radius); free(A.dmax); free(B.radius);
        free(B.dmax); free(pcnt); free(plist); free(pivb);
        return -1;
    }
    for (int64_t t = 0; t < n; ++t) members[t] = (int32_t)t;
    int64_t nd = 0;
    g_assign(X, D, metric, members, n, NULL, &A, &nd);  /* rule A: nearest pivot, own radius */
    g_link(X, D, metric, &A, NULL, NULL, &nd);
    for (int32_t p = 0; p < mb; ++p) B.radius[p] = B.dmax[p] = r;
    g_link(X, D, metric, &B, NULL, NULL, &nd);          /* rule B: every radius r */
    int64_t memberships = 0, orphans = 0;
    for (int64_t x = 0; x < n; ++x) {                    /* rule B parents: every pivot within r */
        for (int32_t p = 0; p < mb; ++p)
            if (g_dist_of(g_key(X + x * D, X + (int64_t)pivb[p] * D, D, metric), metric) <= r)
                plist[x * mb + pcnt[x]++] = p;
        memberships += pcnt[x];
        orphans += pcnt[x] == 0;
    }
    int64_t ca = 0, cb = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : ca, cb)
    for (int64_t i = 0; i < n; ++i) {
        for (int64_t j = i + 1; j < n; ++j) {
            int32_t a = A.assign[i], b = A.assign[j];
            int in_a = a == b || A.gg[(int64_t)(a < b ? a : b) * m + (a < b ? b : a)];
            int in_b = 1;
            for (int32_t s = 0; s < pcnt[i] && in_b; ++s)
                for (int32_t t = 0; t < pcnt[j] && in_b; ++t) {
                    int32_t p = plist[i * mb + s], q = plist[j * mb + t];
                    if (p != q && !B.gg[(int64_t)(p < q ? p : q) * mb + (p < q ? q : p)]) in_b = 0;
                }
            ca += in_a;
            cb += in_b;
            if (cand_a) cand_a[i * n + j] = (unsigned char)in_a;
            if (cand_b) cand_b[i * n + j] = (unsigned char)in_b;
        }
    }
    /* rule A again, on B's pivots */
    int64_t ca2 = ca;
    if (mb != m) {
        g_layer A2;
        memset(&A2, 0, sizeof(A2));
        A2.m = mb;
        A2.piv = pivb;
        A2.assign = (int32_t *)malloc(sizeof(int32_t) * (size_t)(n > 0 ? n : 1));
        A2.mdist = (double *)malloc(sizeof(double) * (size_t)(n > 0 ? n : 1));
        A2.radius = (double *)malloc(sizeof(double) * (size_t)mb);
        A2.dmax = (double *)malloc(sizeof(double) * (size_t)mb);
        if (!A2.assign || !A2.mdist || !A2.radius || !A2.dmax) {
            ca2 = -1;
        } else {
            g_assign(X, D, metric, members, n, NULL, &A2, &nd);
            g_link(X, D, metric, &A2, NULL, NULL, &nd);
            ca2 = 0;
#pragma omp parallel for schedule(dynamic, 16) reduction(+ : ca2)
            for (int64_t i = 0; i < n; ++i)
                for (int64_t j = i + 1; j < n; ++j) {
                    int32_t a = A2.assign[i], b = A2.assign[j];
                    ca2 += a == b || A2.gg[(int64_t)(a < b ? a : b) * mb + (a < b ? b : a)];
                }
        }
        free(A2.assign); free(A2.mdist); free(A2.radius); free(A2.dmax); free(A2.coff); free(A2.cidx);
        free(A2.gx); free(A2.gg);
    }
    if (stats) {
        stats[0] = ca; stats[1] = cb; stats[2] = orphans; stats[3] = memberships; stats[4] = mb; stats[5] = ca2;
    }
    free(members); free(A.assign); free(A.mdist); free(A.radius); free(A.dmax); free(A.coff); free(A.cidx);
    free(A.gx); free(A.gg); free(B.radius); free(B.dmax); free(B.gx); free(B.gg); free(pcnt); free(plist);
    free(pivb);
    return 0;
}

/* ---- RNG search by the paper's stages (Algorithm 1 without Stage VII, Sec. 2) -----------
 * One pivot layer piv[m] over the index X[n] (each point joins its nearest pivot, whose radius
 * is its largest member distance), its GRNG with the guidance margin, then for each query q of
 * Q[mq] (q joins nothing; only index points block):
 *   Stage I:   q's parents are the pivots whose ball holds q; a pivot stays only if it equals or
 *              is linked to every parent (Theorem 1); with no parent every pivot stays.
 *   Stage II:  q as a virtual zero-radius pivot: the domain of p_j is dropped when some pivot
 *              p_k has d(q,p_k) < d(q,p_j) - r_j and d(p_j,p_k) < d(q,p_j) - 2 r_j.
 *   Stage III: an exemplar x of a surviving domain p_j as a virtual zero-radius pivot against a
 *              parent p_i of q: x is dropped when some pivot p_k has d(p_k,p_i) < d(p_i,x) - 2 r_i
 *              and d(p_k,x) < d(p_i,x) - r_i, the latter through d(p_k,x) <= d(p_k,p_j) + d(x,p_j).
 *   Stages IV-VI: for each remaining x, the pivots in increasing d(q,p) as interceptors, then
 *              their members unless Prop. 4 excludes the domain, until no domain can hold a
 *              point closer to q than x.
 * Every pruning is taken with the relative margin of the construction above; every decision on
 * a triple is the canonical key comparison.  Query t's neighbours (ascending) go to
 * nbrs[t * row_cap ...], their count to cnt[t].  stats (may be NULL): [0] distance computations
 * (query-pivot, query-point, point-point; the layer's own are not counted), [1] exemplars left
 * after Stage I, [2] after Stage II, [3] after Stage III.  Returns 0, -1 on allocation failure. */
int32_t orc_rng_search_guided(const float *X, int64_t n, int32_t D, int32_t metric, const int32_t *piv, int32_t m,
                              const float *Q, int64_t mq, int32_t *nbrs, int64_t row_cap, int64_t *cnt,
                              int64_t *stats) {
    if (m < 1 || n < 1) return -1;
    g_layer F;
    memset(&F, 0, sizeof(F));
    F.m = m;
    F.piv = piv;
    int32_t *members = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    F.assign = (int32_t *)malloc(sizeof(int32_t) * (size_t)n);
    F.mdist = (double *)malloc(sizeof(double) * (size_t)n);
    F.radius = (double *)malloc(sizeof(double) * (size_t)m);
    F.dmax = (double *)malloc(sizeof(double) * (size_t)m);
    double *Dpp = (double *)malloc(sizeof(double) * (size_t)m * (size_t)m);
    if (!members || !F.assign || !F.mdist || !F.radius || !F.dmax || !Dpp) {
        free(members); free(F.assign); free(F.mdist); free(F.radius); free(F.dmax); free(Dpp);
        return -1;
    }
    for (int64_t t = 0; t < n; ++t) members[t] = (int32_t)t;
    int64_t nd0 = 0;
    g_assign(X, D, metric, members, n, NULL, &F, &nd0);
    g_link(X, D, metric, &F, NULL, NULL, &nd0);
#pragma omp parallel for schedule(dynamic, 8)
    for (int32_t i = 0; i < m; ++i)
        for (int32_t k = 0; k < m; ++k)
            Dpp[(int64_t)i * m + k] = g_dist_of(g_key(X + (int64_t)piv[i] * D, X + (int64_t)piv[k] * D, D, metric), metric);
    double dmax_all = 0.0;
    for (int32_t p = 0; p < m; ++p) if (F.dmax[p] > dmax_all) dmax_all = F.dmax[p];
    int64_t sd = 0, s1 = 0, s2 = 0, s3 = 0;
    int failed = 0;
#pragma omp parallel reduction(+ : sd, s1, s2, s3)
    {
        g_dp *order = (g_dp *)malloc(sizeof(g_dp) * (size_t)m);
        double *dq = (double *)malloc(sizeof(double) * (size_t)m);
        double *kqz = (double *)malloc(sizeof(double) * (size_t)n);  /* cached keys of q to points */
        unsigned char *keep = (unsigned char *)malloc((size_t)m);
        unsigned char *isn = (unsigned char *)malloc((size_t)n);
        int32_t *par = (int32_t *)malloc(sizeof(int32_t) * (size_t)m);
        if (!order || !dq || !kqz || !keep || !isn || !par) {
#pragma omp atomic write
            failed = 1;
        }
#pragma omp for schedule(dynamic, 1)
        for (int64_t t = 0; t < mq; ++t) {
            if (!order || !dq || !kqz || !keep || !isn || !par) continue;
            const float *q = Q + t * D;
            for (int64_t z = 0; z < n; ++z) { kqz[z] = -1.0; isn[z] = 0; }
            for (int32_t p = 0; p < m; ++p) {
                dq[p] = g_dist_of(g_key(q, X + (int64_t)piv[p] * D, D, metric), metric);
                order[p].d = dq[p];
                order[p].p = p;
            }
            sd += m;
            qsort(order, (size_t)m, sizeof(g_dp), g_dp_cmp);
            int32_t np = 0;
            for (int32_t p = 0; p < m; ++p) if (dq[p] <= F.radius[p]) par[np++] = p;
            /* Stage I */
            for (int32_t j = 0; j < m; ++j) {
                int ok = 1;
                for (int32_t s = 0; s < np && ok; ++s) {
                    const int32_t i = par[s];
                    if (i != j && !F.gg[(int64_t)(i < j ? i : j) * m + (i < j ? j : i)]) ok = 0;
                }
                keep[j] = (unsigned char)ok;
                if (ok) s1 += F.coff[j + 1] - F.coff[j];
            }
            /* Stage II */
            for (int32_t j = 0; j < m; ++j) {
                if (!keep[j]) continue;
                const double a1 = dq[j] - F.radius[j], a2 = dq[j] - 2.0 * F.radius[j];
                for (int32_t k = 0; k < m; ++k) {
                    if (k == j) continue;
                    const double b = Dpp[(int64_t)j * m + k];
                    if (dq[k] < a1 - G_MARGIN * (dq[k] + fabs(a1) + dq[j]) &&
                        b < a2 - G_MARGIN * (b + fabs(a2) + dq[j])) { keep[j] = 0; break; }
                }
                if (keep[j]) s2 += F.coff[j + 1] - F.coff[j];
            }
            /* Stage III, then Stages IV-VI for what is left */
            for (int32_t j = 0; j < m; ++j) {
                if (!keep[j]) continue;
                for (int32_t u = F.coff[j]; u < F.coff[j + 1]; ++u) {
                    const int64_t x = F.cidx[u];
                    const float *px = X + x * D;
                    int dropped = 0;
                    for (int32_t s = 0; s < np && !dropped; ++s) {
                        const int32_t i = par[s];
                        const double dpx = g_dist_of(g_key(X + (int64_t)piv[i] * D, px, D, metric), metric);
                        ++sd;
                        const double c1 = dpx - 2.0 * F.radius[i], c2 = dpx - F.radius[i];
                        for (int32_t k = 0; k < m && !dropped; ++k) {
                            const double e1 = Dpp[(int64_t)k * m + i];
                            const double e2 = Dpp[(int64_t)k * m + j] + F.mdist[x];  /* >= d(p_k, x) */
                            if (e1 < c1 - G_MARGIN * (e1 + fabs(c1) + dpx) && e2 < c2 - G_MARGIN * (e2 + fabs(c2) + dpx))
                                dropped = 1;
                        }
                    }
                    if (dropped) continue;
                    ++s3;
                    if (kqz[x] < 0.0) { kqz[x] = g_key(q, px, D, metric); ++sd; }
                    const double kqx = kqz[x], dqx = g_dist_of(kqx, metric);
                    int blocked = 0;
                    for (int32_t w = 0; w < m && !blocked; ++w) {
                        const int32_t p = order[w].p;
                        const double dqp = order[w].d, dm = F.dmax[p];
                        if (dqp - dmax_all >= dqx + G_MARGIN * (dqp + dmax_all + dqx)) break;
                        const int64_t pid = piv[p];
                        double kxp = -1.0;
                        if (pid != x) {  /* Stage IV: the pivot itself */
                            if (kqz[pid] < 0.0) { kqz[pid] = g_key(q, X + pid * D, D, metric); ++sd; }
                            kxp = g_key(px, X + pid * D, D, metric);
                            ++sd;
                            if (kqz[pid] < kqx && kxp < kqx) { blocked = 1; break; }
                        }
                        if (dqp - dm >= dqx + G_MARGIN * (dqp + dm + dqx)) continue;  /* Prop. 4 */
                        if (kxp < 0.0) { kxp = g_key(px, X + pid * D, D, metric); ++sd; }
                        const double dxp = g_dist_of(kxp, metric);
                        if (dxp - dm >= dqx + G_MARGIN * (dxp + dm + dqx)) continue;
                        for (int32_t v = F.coff[p]; v < F.coff[p + 1] && !blocked; ++v) {  /* Stage VI */
                            const int64_t z = F.cidx[v];
                            if (z == x || z == pid) continue;
                            if (kqz[z] < 0.0) { kqz[z] = g_key(q, X + z * D, D, metric); ++sd; }
                            if (!(kqz[z] < kqx)) continue;
                            const double kxz = g_key(px, X + z * D, D, metric);
                            ++sd;
                            if (kxz < kqx) blocked = 1;  /* strictly inside the open lune */
                        }
                    }
                    if (!blocked) isn[x] = 1;
                }
            }
            int64_t c = 0;
            for (int64_t x = 0; x < n; ++x)
                if (isn[x]) { if (c < row_cap) nbrs[t * row_cap + c] = (int32_t)x; ++c; }
            cnt[t] = c;
        }
        free(order); free(dq); free(kqz); free(keep); free(isn); free(par);
    }
    if (stats) { stats[0] = sd; stats[1] = s1; stats[2] = s2; stats[3] = s3; }
    free(members); free(F.assign); free(F.mdist); free(F.radius); free(F.dmax); free(F.coff); free(F.cidx);
    free(F.gx); free(F.gg); free(Dpp);
    return failed ? -1 : 0;
}
