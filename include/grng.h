/*
 * grng.h -- C ABI of the GB300 library for exact Relative Neighborhood Graph (RNG)
 * construction guided by Generalized Relative Neighborhood Graphs (GRNG), after
 * Foster, Sevilmis & Kimia, arXiv 2208.10022.
 *
 * Problem statement (Sec. 1): a set S of N points in a metric space (S, d), here
 * R^D under L2 or L1.  Pivot layers P_0 (coarsest) ... P_{L-1} (finest) are nested
 * subsets of S (every coarse pivot is also a fine pivot, as Theorem 2 requires).
 * Each pivot p has a domain D(p, r) = { x : d(x,p) <= r } (Eq. 2); the finest layer's
 * domains hold the points, a coarser layer's "relative" domains hold the next finer
 * layer's pivots together with their radii (Sec. 3).  Each layer's pivots are linked
 * by the GRNG (definition, Sec. 2) and the points by the RNG (Eq. 1, Sec. 1), which
 * is returned as an undirected edge list.
 *
 * Exactness.  Every decision is the canonical FP64 comparison of the definitions:
 * key(a,b) = sum_k (a_k - b_k)^2 (L2) or sum_k |a_k - b_k| (L1), summed left to right
 * in FP64 without fused multiply-add, d = sqrt(key) for L2; GRNG thresholds are
 * d_ij - (2 r_i + r_j) and d_ij - (r_i + 2 r_j), except that pairs with r_i = r_j = 0
 * compare keys.  The GPU computes FP32 (or lower) keys, brackets them by a proven
 * error bound and re-decides in FP64 only the comparisons the bracket cannot
 * settle, so the results are the definitions' results, bit for bit.
 *
 * Conventions.
 *  - Pointers: every input pointer may be host or device memory (detected with
 *    cudaPointerGetAttributes); the library copies inputs and never keeps a caller
 *    pointer after a call returns.  Output pointers may be host or device memory and
 *    receive copies.  Points are FP32 row-major [n][dim].
 *  - Buffers too small: the call returns GRNG_ETRUNC and reports the size needed.
 *  - Streams: work runs on opts.cuda_stream (a cudaStream_t, NULL = legacy default
 *    stream) of the device current at grng_create; every call returns after that
 *    stream has finished the call's work.
 *  - Errors: no exception crosses the ABI; a status is returned and the message of
 *    the last failure on the calling thread is available from grng_last_error().
 *    An index on which a call failed with GRNG_ECUDA must be destroyed.
 *  - Threads: an index is not safe for concurrent calls from several threads.
 */
#ifndef GRNG_H
#define GRNG_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef int32_t grng_status;
#define GRNG_OK 0
#define GRNG_EINVAL 1    /* invalid argument (sizes, indices, nesting, NULL) */
#define GRNG_ENOMEM 2    /* device or host allocation failed */
#define GRNG_ECUDA 3     /* a CUDA call failed */
#define GRNG_ETIMEOUT 4  /* a bounded device wait ran out (status set by a kernel) */
#define GRNG_ETRUNC 5    /* output buffer too small; the needed size is reported */
#define GRNG_EINTERNAL 6 /* internal consistency check failed */
#define GRNG_ESTATE 7    /* call order violated (e.g. a layer not built or not linked) */
#define GRNG_ENOTIMPL 8  /* option the library does not support */

typedef enum { GRNG_L2 = 0, GRNG_L1 = 1 } grng_metric;
typedef enum { GRNG_FP32 = 0, GRNG_BF16 = 1, GRNG_FP8 = 2 } grng_precision;

typedef struct grng_opts {
  int32_t metric;          /* grng_metric */
  int32_t precision;       /* grng_precision of the distance tiles (FP32: CUDA cores) */
  int32_t n_layers;        /* number of pivot layers L >= 1 */
  int32_t knn_k;           /* neighbour-list length of the exact tier, 1..32 (0: 32) */
  int32_t k_shortlist;     /* learned interceptor shortlist length, 0 (off) or 1..16 */
  int32_t reserved;        /* must be 0 */
  const void* mlp_weights; /* ranking network parameters, grng_mlp_nparams() FP32 values (host or
                              device; copied at grng_create), required when k_shortlist > 0 */
  size_t mlp_bytes;        /* 4 * grng_mlp_nparams() when mlp_weights is given */
  int64_t spin_limit;      /* iteration cap of bounded device waits (0: default) */
  void* cuda_stream;       /* cudaStream_t, or NULL */
  uint64_t flags;          /* 0, or GRNG_FLAG_SHORT_LISTS | GRNG_FLAG_SMALL_BUFFERS (testing) |
                              GRNG_FLAG_RECORD_MLP */
} grng_opts;

/* Testing aid: cap the pivot layers' range lists at 16 nodes so that more pairs take
 * the hierarchical exhaustive tier.  Results are identical; only the work changes. */
#define GRNG_FLAG_SHORT_LISTS 1ull
/* Record, during rng_build_exact, one training sample per candidate of the learned
 * shortlist's pool for every pair that reaches the exhaustive tier (see
 * grng_mlp_dataset).  Results are unchanged. */
#define GRNG_FLAG_RECORD_MLP 2ull
/* Testing aid: start every internal work buffer (tier-1 survivors, ambiguous triples,
 * the exhaustive tier's frontier) at a tiny capacity, so that the overflow paths run:
 * a repeated sweep with a larger buffer, or the exhaustive scan of every node.  Results
 * are identical; only the work changes. */
#define GRNG_FLAG_SMALL_BUFFERS 4ull

typedef struct grng_index grng_index; /* opaque; owns all device state */

/* Fill *o with defaults: L2, FP32, one layer, knn_k 32, default stream. */
void grng_default_opts(grng_opts* o);

/* Create an index over n points pts[n][dim] (host or device, FP32).  n >= 1,
 * 1 <= dim <= 4096, n < 2^31.  The points are copied; the device current on the
 * calling thread is the one used.  Paper: the point set S and metric d (Sec. 1). */
grng_status grng_create(grng_index** out, const float* pts, int64_t n, int32_t dim,
                        const grng_opts* opts);

/* Build pivot layer `layer` (0 = coarsest ... n_layers-1 = finest) from m pivot
 * point indices pivot_idx[m] (host or device int32, distinct, in [0, n)).
 * Layers are built finest first: the finest layer's members are all points, layer
 * l's members are the pivots of layer l+1, which must already be built and must
 * contain every pivot of layer l (nesting).
 * Each member is assigned to its nearest pivot by canonical key, ties to the lowest
 * position in pivot_idx, and a member that is itself a pivot to that pivot (Eq. 2).
 * radius[p] = max over p's members of d(p, member) + member radius (0 for points),
 * the relative pivot domain of Sec. 3; delta_max[p] = max over p's members of
 * d(p, member) (Stage VI of Secs. 2 and 3).  An empty domain has radius 0.
 * Outputs (each may be NULL, host or device): assign[n_members] (pivot positions),
 * radius[m], delta_max[m].  Rebuilding a layer invalidates its and every coarser
 * layer's GRNG and the RNG. */
grng_status grng_build_layer(grng_index* idx, int32_t layer, const int32_t* pivot_idx, int32_t m,
                             int32_t* assign, double* radius, double* delta_max);

/* GRNG of layer `layer` (definition, Sec. 2).  Every layer must be built; layer
 * l > 0 must have layer l-1 linked, whose GRNG restricts the candidate pairs
 * (Theorem 2).  With radius_override (m doubles, host or device) the GRNG of the
 * layer's pivots with those radii is computed over all pairs instead and is not
 * stored in the index.
 * Output: CSR over pivot positions in pivot_idx order, rows sorted ascending, both
 * directions listed: off[m+1] (int64) and adj[off[m]] (int32), host or device.
 * off/adj may be NULL (no output).  If adj_cap < off[m] the call stores off,
 * returns GRNG_ETRUNC and sets *adj_needed (if not NULL) to off[m]. */
grng_status grng_link_pivots(grng_index* idx, int32_t layer, const double* radius_override,
                             int64_t* off, int32_t* adj, int64_t adj_cap, int64_t* adj_needed);

/* Rows [row_begin, row_end) of a linked layer's GRNG in the same format: off has
 * row_end-row_begin+1 entries starting at 0.  For sampling very large layers. */
grng_status grng_adjacency_rows(grng_index* idx, int32_t layer, int64_t row_begin, int64_t row_end,
                                int64_t* off, int32_t* adj, int64_t adj_cap, int64_t* adj_needed);

/* Exact RNG of all points (Eq. 1): candidate pairs are the pairs whose finest
 * pivots are equal or GRNG-linked (Stage I, Theorem 1); each candidate pair is
 * tested for an empty lune.  Every layer must be built and linked. */
grng_status rng_build_exact(grng_index* idx);

/* Lune-based beta-skeleton of all points for 1 <= beta <= 2 (Sec. 1: the empty-region
 * graphs that contain the RNG; beta = 1 is the Gabriel graph, beta = 2 the RNG): (x, y) is
 * an edge iff no third point lies strictly inside both balls of radius beta d(x,y) / 2
 * centred at (1 - beta/2) x + (beta/2) y and (beta/2) x + (1 - beta/2) y.  The edges
 * replace the stored graph (read with rng_edges, same format); beta = 2 is exactly
 * rng_build_exact.  Below 2 Theorem 1 does not restrict the candidates (a GRNG non-link
 * proves a point inside the lune of Eq. 1, not inside the smaller beta-lune), so every pair
 * is a candidate; the interceptor tiers, the exhaustive search over the pivot layers and the
 * FP64 recheck are those of the RNG with the lune test replaced; FP32 tiles, no learned
 * shortlist.  Every layer must be built and linked.  Errors: GRNG_EINVAL for beta outside
 * [1, 2] or, below 2, an L1 index; GRNG_ESTATE when a layer is not linked.  rng_insert_batch
 * refuses an index whose stored graph is a skeleton with beta < 2 (GRNG_ESTATE). */
grng_status rng_build_skeleton(grng_index* idx, double beta);

/* Insert m new points pts[m][dim] (host or device) so that the stored RNG becomes
 * the RNG of the enlarged set (Algorithm 1 and Stage VII, Sec. 2).  Requires a
 * built RNG.  The new points get ids n .. n+m-1 and join the finest layer's domains;
 * every layer keeps its pivots.  Radii, delta_max, every GRNG and the RNG are then
 * those of a build from scratch on the enlarged set with the same pivots; only what
 * the batch can change is recomputed (grown radii, the GRNG pairs they reopen, the
 * batch points' pairs, and Stage VII for the old edges a batch point may enter).
 * On failure the index must be destroyed. */
grng_status rng_insert_batch(grng_index* idx, const float* pts, int64_t m);

/* RNG search (Algorithm 1 without Stage VII, Sec. 2): for each of m query points
 * queries[m][dim] (FP32, row-major, host or device), its RNG neighbours among the
 * index points: x is a neighbour of q iff no index point other than x lies strictly
 * inside the open lune of (q, x) (Eq. 1 over the index plus q alone).  The queries do
 * not join the index and never block one another; the index is not changed.  Every
 * layer must be built and linked (the finest GRNG restricts each query's candidates by
 * Theorem 1 when the query lies in its nearest finest pivot's ball).  *total (if not
 * NULL) receives the number of (query, neighbour) pairs; the result stays in the index
 * until the next search and is read with rng_search_result.  Between searches the index keeps
 * its points in sorted order with room for the largest batch so far (n + m rows), their
 * in-block keys and neighbour lists, and the rows' K-nearest lists (8 K bytes per row); they are
 * rebuilt after an insertion.  Errors: GRNG_EINVAL for NULL queries, m < 1 or n + m >= 2^31;
 * GRNG_ESTATE when a layer is not linked; GRNG_ENOMEM when the device memory runs out. */
grng_status rng_search_batch(grng_index* idx, const float* queries, int64_t m, int64_t* total);

/* The last search's result as CSR over the queries in input order: off[m+1] (int64) and
 * nbrs[off[m]] (int32 original point ids, ascending within a query), host or device;
 * either may be NULL.  GRNG_ESTATE before any search; GRNG_ETRUNC (off still written)
 * when cap < off[m]. */
grng_status rng_search_result(const grng_index* idx, int64_t* off, int32_t* nbrs, int64_t cap);

/* Copy the RNG edges: ij[cap][2] int32 point indices with i < j, lexicographically
 * sorted (host or device).  *n_edges receives the edge count; if cap < count the
 * call returns GRNG_ETRUNC after writing nothing. ij may be NULL to query. */
grng_status rng_edges(const grng_index* idx, int32_t* ij, int64_t cap, int64_t* n_edges);

/* ---- Learned shortlist (an extension of Stage V, Sec. 2: the "select group" of likely
 * interceptors tried before the exhaustive Stage VI search) ---------------------------
 * A ranking network scores candidate interceptors of the exemplar pairs that the exact
 * tiers leave to the exhaustive search; each such pair first tests its k best-scored
 * candidates exactly (Eq. 1) and, if none blocks it, goes on to the exhaustive search
 * as without the network.  The network never decides an edge: it only changes which
 * interceptors are tried first, so the edge set is identical with or without it.
 *
 * Network: 32 features -> 128 ReLU -> 128 ReLU -> 1 logit.  Parameter vector (FP32,
 * grng_mlp_nparams() values, in this order): W1[128][32] (row = hidden unit), b1[128],
 * W2[128][128], b2[128], w3[128], b3.  Inference inside the build (opts.mlp_weights with
 * opts.mlp_bytes = 4 * grng_mlp_nparams() and opts.k_shortlist in 1..16) and in
 * grng_mlp_score rounds the weights to BF16 and accumulates in FP32.
 *
 * Candidate pool of a pair (g, o): the K listed neighbours of each of the first 8
 * listed neighbours of g and of o.  Features (all distances divided by d(g,o) and
 * clamped to [0, 8]): side, neighbour rank, rank within its list, the two list
 * distances and the triangle bounds they give, distances of z, g, o to their pivots,
 * pivot equalities, pivot radii, the K-th list distance of g, o and the neighbour,
 * log2 d(g,o) / 8, and 8 hashed bits of the pivot ids (+-1).
 *
 * All pointers may be host or device memory; these calls use the legacy default
 * stream and return when their work is done. */
int64_t grng_mlp_nparams(void);

/* Logits scores[n] of the samples feats[n][32] under params (BF16 weights, FP32 sums). */
grng_status grng_mlp_score(const float* params, const float* feats, int64_t n, float* scores);

/* FP32 loss L = (1/n) sum_b w_b [log(1 + e^{s_b}) - y_b s_b] (w = 1 when weights is NULL)
 * and its gradient grad[nparams] with respect to params (FP32 weights, no rounding);
 * 1 <= n <= 2^20.  loss and grad may be NULL. */
grng_status grng_mlp_loss_grad(const float* params, const float* feats, const float* labels,
                               const float* weights, int64_t n, float* loss, float* grad);

/* Train params (in/out) with Adam (lr, betas 0.9 / 0.999) on mini-batches of `batch`
 * consecutive samples for `epochs` passes, on the GPU.  *loss_out (may be NULL) gets the
 * mean loss of the last pass.  The caller shuffles the samples and draws the initial
 * parameters. */
grng_status grng_mlp_train(const float* feats, const float* labels, const float* weights, int64_t n,
                           int32_t epochs, int32_t batch, float lr, float* params, float* loss_out);

/* Samples recorded by the last rng_build_exact of an index created with
 * GRNG_FLAG_RECORD_MLP: feats[count][32] and labels[count] (1 when the candidate blocks
 * the pair by FP32 keys, else 0).  *count receives the number of samples (at most
 * 4,194,304); with feats and labels NULL only the count is returned.  cap < count
 * returns GRNG_ETRUNC. */
grng_status grng_mlp_dataset(const grng_index* idx, float* feats, float* labels, int64_t cap, int64_t* count);

/* Counters and timings of the last calls as one JSON object (NUL-terminated).
 * If cap is too small, returns GRNG_ETRUNC and writes nothing. */
grng_status grng_stats(const grng_index* idx, char* json, size_t cap);

/* Release the index and all its device memory.  NULL is accepted. */
void grng_destroy(grng_index* idx);

/* Message of the last failed call on this thread ("" if none). */
const char* grng_last_error(void);

/* Diagnostic of the tensor-core distance tiles used when opts.precision = GRNG_BF16
 * (L2): keys[i*n + j] = |x_i|^2 + |x_j|^2 - 2 x_i.x_j for all pairs of n <= 256 points
 * pts[n][dim] (host or device, dim <= 128), with the dot products computed by tcgen05
 * MMAs on split BF16 operands (x = hi + lo; hi.hi + hi.lo + lo.hi) accumulated in FP32.
 * Their absolute error is at most (2^-12 + (3*Dp + 16) 2^-24) (|x_i|^2 + |x_j|^2),
 * Dp = dim rounded up to 16.  keys may be host or device memory. */
grng_status grng_tc_keys(const float* pts, int64_t n, int32_t dim, float* keys);

/* Nearest-pivot assignment that allocates nothing.  The paper has no counterpart: this
 * entry point exists for callers that cannot allocate device memory -- code that runs
 * inside a memory pool that forbids new allocations, plugins whose host application
 * owns every device allocation, or programs whose memory footprint must not change once
 * they are running.  It computes what grng_build_layer computes for the finest layer
 * (nearest pivot by canonical key, ties to the lowest position, a pivot owns itself),
 * without an index and without cudaMalloc/cudaFree or any allocating library call.
 *
 * pts[n][dim]       DEVICE pointer, FP32 row-major, 16-byte aligned; dim a positive
 *                   multiple of 8
 * pivot_idx[m]      DEVICE pointer, 4-byte aligned, distinct point indices in [0, n)
 * assign[n]         DEVICE output, 4-byte aligned: pivot position of every point
 * dist[n]           DEVICE output, 8-byte aligned: FP64 canonical distance to that pivot
 *                   (the layer's radius of pivot p is the maximum of dist over the points
 *                   assigned to p)
 * Every pointer must be device (or managed) memory of the current device, checked with
 * cudaPointerGetAttributes before any work is queued: a host pointer, a pointer of another
 * device or a misaligned one returns GRNG_EINVAL.
 * cuda_stream       cudaStream_t the work is queued on (NULL = legacy default stream);
 *                   the call returns after that stream has finished it.
 * Limits: 1 <= n <= 262,144; 1 <= m <= min(n, 65,536); m * dim <= 2,097,152; larger
 * sizes return GRNG_EINVAL.  Scratch memory is one fixed array of about 13 MB inside the
 * library image; every GPU that loads the library holds it until the process exits.
 * Every call shares that array and it keeps the previous call's contents, so calls that
 * overlap on the GPU (from several threads or streams) race: serialise them.  The first
 * call on a device looks up the array's device address with that device current; make
 * that first call before capturing any stream into a CUDA graph. */
grng_status grng_assign_static(const float* pts, int64_t n, int32_t dim, const int32_t* pivot_idx, int32_t m,
                               int32_t metric, int32_t* assign, double* dist, void* cuda_stream);

#ifdef __cplusplus
}
#endif
#endif /* GRNG_H */
