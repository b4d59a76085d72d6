// internal.h -- host-side interfaces between the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <stdint.h>

#include <string>

namespace grng {

// ---- device buffer ---------------------------------------------------------------
struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
  DevBuf() = default;
  DevBuf(const DevBuf&) = delete;
  DevBuf& operator=(const DevBuf&) = delete;
  DevBuf(DevBuf&& o) noexcept : p(o.p), bytes(o.bytes) { o.p = nullptr; o.bytes = 0; }
  DevBuf& operator=(DevBuf&& o) noexcept {
    if (this != &o) { release(); p = o.p; bytes = o.bytes; o.p = nullptr; o.bytes = 0; }
    return *this;
  }
  ~DevBuf() { release(); }
  cudaError_t alloc(size_t b) {
    if (b <= bytes && p) return cudaSuccess;
    release();
    if (b == 0) b = 16;
    cudaError_t e = cudaMalloc(&p, b);
    if (e != cudaSuccess) { p = nullptr; bytes = 0; cudaGetLastError(); return e; }
    bytes = b;
    return cudaSuccess;
  }
  void release() {
    if (p) cudaFree(p);
    p = nullptr;
    bytes = 0;
  }
  template <class T> T* as() const { return static_cast<T*>(p); }
};

// error raised inside the host orchestration; converted to a status at the C-ABI
struct Failure {
  int status;
  std::string msg;
};
[[noreturn]] void fail(int status, const std::string& msg);
void set_last_error(const std::string& msg);  // message returned by grng_last_error()
void cuda_check(cudaError_t e, const char* what);
#define GRNG_STR2(x) #x
#define GRNG_STR(x) GRNG_STR2(x)
#define GRNG_CUDA(call) ::grng::cuda_check((call), __FILE__ ":" GRNG_STR(__LINE__) ": " #call)
// every kernel launch of the library is counted (reported by grng_stats)
void note_launch();
unsigned long long launches();

// ---- utilities (kernels_util.cu) ------------------------------------------------------
void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s);  // out[n] = total
// counting sort of (key, value) int2 pairs by pair.x (which=0) or pair.y (which=1):
// off[nkeys+1], val[m] = the other component, grouped by key.
void group_pairs(const int2* pairs, int64_t m, int which, int64_t nkeys, int64_t* off,
                 int32_t* val, DevBuf& tmp, cudaStream_t s);
void sort_u64(uint64_t* keys, int64_t m, DevBuf& tmp, cudaStream_t s);  // ascending, in place
// stable counting sort of items 0..m-1 by key[] in [0,nkeys): order[m] (item ids), and
// rank[item] = position in that order
void stable_order(const int32_t* key, int64_t m, int64_t nkeys, int32_t* order, int32_t* rank,
                  DevBuf& tmp, cudaStream_t s);
void gather_rows(const float* X, int Dp, const int32_t* idx, int64_t m, float* out, cudaStream_t s);
void fill_u32(uint32_t* p, uint32_t v, size_t count, cudaStream_t s);
// CSR of a triangular bitmask (bit (a,b), a<b, sorted positions) in original order:
// rank[orig] = sorted position.  off may be null to count only.
void bitmask_csr(const uint32_t* bits, int64_t words, const int32_t* rank, int64_t m,
                 int64_t* off, int32_t* adj, DevBuf& tmp, cudaStream_t s);
void bitmask_rows(const uint32_t* bits, int64_t words, const int32_t* rank, int64_t m,
                  int64_t row_begin, int64_t row_end, int64_t* off, int32_t* adj, cudaStream_t s);

// ---- assignment (kernels_assign.cu) -----------------------------------------------------
struct AssignOut {
  int32_t* assign;    // [nmem] pivot position
  double* dist;       // [nmem]
  double* radius;     // [m]
  double* delta_max;  // [m]
};
// members: contiguous coordinates [nmem][Dp] (mem_id = their point indices, for the
// self-assignment rule); pivots: contiguous coordinates [m][Dp] (piv_id point indices)
// tc: the member x pivot keys from the tensor cores (L2, at least 256 pivots; split-BF16
// Gram keys with their error bound, the undecided members re-decided exactly), else FP32 tiles
void assign_layer(const float* Xmem, const int32_t* mem_id, const double* mem_r, int64_t nmem,
                  const float* Xpiv, const int32_t* piv_id, int64_t m, int64_t npoints, int D,
                  int Dp, int metric, const AssignOut& out, unsigned long long* stats,
                  cudaStream_t s, bool tc = false, long long spin = 1ll << 24);

// ---- pair pipeline (kernels_pair.cu) ----------------------------------------------------
#define GRNG_MAXL 16
// The coarser layers above a level, coarsest first, for the hierarchical exhaustive
// tier: sorted coordinates, an FP32 upper bound of the distance from each node to
// anything below it, and the range of its children in the next finer level.
struct Ancestors {
  int n = 0;
  const float* X[GRNG_MAXL];
  const float* Rhi[GRNG_MAXL];
  const int32_t* cstart[GRNG_MAXL];  // [m+1]
  int64_t m[GRNG_MAXL];
  int64_t toff[GRNG_MAXL];           // column of layer a in the node x ancestor key table
};
struct LevelIn {
  const float* X;           // node coordinates in sorted order [n][Dp]
  int64_t n;
  int D, Dp, metric;
  int grng;                 // 1: GRNG test with radii; 0: RNG of exemplars
  int K;                    // neighbour-list length (<= GRNG_KMAX)
  const int32_t* parent;    // [n] parent sorted position, or null (all pairs candidates)
  const uint32_t* gpar;     // guidance bitmask over parents (triangular), or null
  int64_t gpar_words;
  const double* r64;        // [n] radii (null: zeros)
  const float* rlo;         // [n] FP32 lower bounds of r64 (null: zeros)
  const float* rhi;
  const int32_t* orig;      // [n] original ids (edge output of the RNG level)
  Ancestors anc;            // layers above this level (none for the top GRNG layer)
  int64_t lmax = 0;         // cap of the range lists (0: the default)
  const float* pdist_hi = nullptr;  // [n] FP32 upper bound of d(node, parent), or null
  int precision = 0;                // 1: tensor-core (split BF16) distance tiles for the RNG level
  long long spin = 1ll << 24;       // poll limit of every bounded device wait
  const float* mlp_params = nullptr;  // RNG level: ranking network (GRNG_MLP_NPARAM floats, device)
  int kshort = 0;                     // shortlist length tried before tier 3 (0: off)
  int mlp_record = 0;                 // RNG level: record features and labels of the tier-3 pairs' pools
  int small_buffers = 0;              // testing: tiny first capacities, so every retry and fallback runs
  int lists = 1;                      // GRNG levels: range lists for the pairs tier 2 leaves open
  int64_t npts = 0;                   // rows [0, npts) may block a pair (0: all n); the rows
                                      // beyond are search queries, endpoints only
  double beta_lam = 1.0;              // RNG level, L2: beta / 2 of a lune-based beta-skeleton
                                      // (1: the RNG; below 1 needs parent = gpar = null, FP32)
};

// ---- tensor-core tiles (kernels_tc.cu) ------------------------------------------------------
struct TcLaunch {
  const uint8_t* img;
  const float* nrm;
  const unsigned int* bmax;
  int64_t n;
  int Dp, K;
  float nmax_all;
  const int32_t* parent;
  const uint32_t* gpar;
  int64_t gpar_words;
  const __half* A;
  const uint8_t* nbr_idx;
  const float* nbr_key;
  int32_t* knn_idx;
  float* knn_key;
  float* knn_rb;
  int2* surv;
  unsigned long long* surv_cnt;
  unsigned long long surv_cap;
  int* strip_ctr;
  unsigned long long* stats;
  int* status;
  long long spin;
};
bool tc_supported(int Dp);
float tc_gamma(int Dp);
void tc_prepare(const float* X, int64_t n, int Dp, DevBuf& img, DevBuf& nrm, DevBuf& bmax, float* nmax_all,
                cudaStream_t s);
void tc_sweep(const TcLaunch& L, cudaStream_t s);
// nearest pivot by split-BF16 Gram keys, per member: best1 (upper bound of the smallest
// exact key), arg1, best2 (lower bound of every other pivot's exact key), cand[4] (the
// pivots of the 4 smallest Gram keys) and rest (lower bound of every other pivot's exact key)
void tc_assign(const float* Xm, int64_t nmem, const float* Xp, int64_t m, int Dp, float* best1, int32_t* arg1,
               float* best2, int32_t* cand, float* rest, long long spin, cudaStream_t s,
               cudaEvent_t start = nullptr, cudaEvent_t done = nullptr);  // events around the kernel, if given
void tc_knn_fix(const float* X, int64_t n, int Dp, int K, int metric, const int32_t* knn_idx, float* knn_key,
                cudaStream_t s);
// children ranges: parent[] (non-decreasing, values in [0, m)) -> cstart[m+1]
void child_ranges(const int32_t* parent, int64_t n, int64_t m, int32_t* cstart, cudaStream_t s);
struct LevelOut {
  // GRNG level: triangular bitmasks over sorted positions, zero-filled by the caller
  uint32_t* gx = nullptr;
  uint32_t* gg = nullptr;
  int64_t words = 0;
  // RNG level: edges as (i << 32 | j), i < j original ids, unsorted
  DevBuf* edges = nullptr;
  int64_t n_edges = 0;
  // RNG level with mlp_record: samples [rec_n][GRNG_MLP_IN] features and [rec_n] labels
  DevBuf* rec_f = nullptr;
  DevBuf* rec_y = nullptr;
  int64_t rec_n = 0;
  // GRNG level, optional: the pairs whose guidance bit was newly set ([n_new_gg] int2, a < b)
  DevBuf* new_gg = nullptr;
  int64_t n_new_gg = 0;
};
struct LevelStats {
  unsigned long long c[42];
  double ms[8];  // prep, tile sweeps, tier-2 grouping + 2a, tier 2b, range lists, tier 3, recheck + emit
  double kms[4];  // CUDA-event time of the tile sweep kernel(s), the tier-3 kernel, the list tier kernel
                  // and the whole range-list phase (thresholds, both sweeps, cut, sides, list tier)
};
// ---- learned shortlist (kernels_mlp.cu) -------------------------------------------------------
#define GRNG_MLP_IN 32
#define GRNG_MLP_H 128
#define GRNG_MLP_NPARAM (GRNG_MLP_H * GRNG_MLP_IN + GRNG_MLP_H + GRNG_MLP_H * GRNG_MLP_H + 2 * GRNG_MLP_H + 1)
#define GRNG_MLP_KMAX 16
#define GRNG_MLP_PW 8  // neighbours of each endpoint whose lists form the candidate pool
struct MlpStage {
  const float* X;
  int64_t n;
  int Dp, metric, K;
  const int32_t* knn_idx;
  const float* knn_key;
  const int32_t* parent;
  const float* pdist_hi;
  const float* prad;     // radius upper bound of each parent, or null
  const int2* pairs;     // pairs entering tier 3
  int64_t m;
  int64_t slot0;         // pending slot of pairs[0]
  int* pflag;            // set to 3 for pairs the shortlist blocks
  int2* amb; unsigned long long* amb_cnt; unsigned long long amb_cap;
  const float* params;   // or null (record only)
  int kshort;
  float* rec_f; float* rec_y; unsigned long long* rec_cnt; unsigned long long rec_cap;  // or null
  unsigned long long* stats;  // [0] candidates scored, [1] shortlist tests, [2] pairs blocked,
                              // [3] samples recorded, [4] pairs with a blocker in the pool (recording)
};
void mlp_stage(const MlpStage& P, cudaStream_t s);

void run_level(const LevelIn& in, LevelOut& out, LevelStats& st, cudaStream_t s,
               float* tile_ms = nullptr);
// tiers 2-3, recheck and emission for explicit candidate pairs of a level (sorted positions);
// knn_idx null: straight to the exhaustive tiers.  GRNG levels OR their bits into out.gx /
// out.gg (never clearing one), the RNG level emits its edges.
void run_pairs(const LevelIn& in, LevelOut& out, LevelStats& st, cudaStream_t s, const int2* pairs, int64_t m,
               const int32_t* knn_idx, const float* knn_key, bool tier2b);
// in-block FP16 keys (rounded up) and the GRNG_KIN in-block nearest neighbours of every
// 128-node block of X [n][Dp]
void block_prep(const float* X, int64_t n, int Dp, int metric, __half* A, uint8_t* nbr_idx, float* nbr_key,
                cudaStream_t s);

// ---- batched insertion (kernels_insert.cu) ---------------------------------------------------
void merge_radii(double* r, double* dmax, const double* rb, const double* db, int64_t m, uint8_t* changed,
                 cudaStream_t s);
// radius[c] (holding the old radii) = max over members of mdist + member radius; changed[c] = grew
void coarse_radii(const double* mdist, const double* mem_r, const int32_t* assign, int64_t nmem, double* radius,
                  const double* old_radius, int64_t m, uint8_t* changed, cudaStream_t s);
// changed flags in sorted order and the list of changed sorted positions; returns its length
int64_t changed_sorted(const uint8_t* changed, const int32_t* order, int64_t m, uint8_t* chg_s, int32_t* list,
                       cudaStream_t s);
// the GRNG pairs an insertion may link: pairs of changed nodes not yet linked (parents equal or
// guidance-linked) and the children pairs of the coarse pairs newp[nnew] whose guidance link is new
int64_t grng_retest_pairs(const int32_t* chg_list, int64_t nchg, const uint8_t* chg_s, int64_t m, const uint32_t* gx,
                          const uint32_t* gg, int64_t words, const int32_t* parent, const uint32_t* gpar,
                          int64_t gpar_words, const int2* newp, int64_t nnew, const int32_t* cstart_par,
                          DevBuf& out, cudaStream_t s);
struct InsertSweep {
  const float* XB;        // batch rows in sorted order, padded to whole 128-row strips (zeros)
  const int32_t* rowpos;  // [mb] their sorted positions (ascending)
  int64_t mb;
  const __half* AB;       // block_prep of XB
  const uint8_t* nbrB_i;
  const float* nbrB_k;
  const float* X;         // every point in sorted order [n][Dp]
  int64_t n;
  int Dp, K, metric;
  const __half* A;        // block_prep of X
  const uint8_t* nbr_i;
  const float* nbr_k;
  const uint8_t* is_new;  // [n] 1 for batch points (sorted positions)
  const int32_t* parent;  // [n] finest pivot, sorted position
  const uint32_t* gpar;   // finest layer's guidance bitmask
  int64_t gpar_words;
  const float* maxe;      // [n] FP32 upper bound of each old point's longest edge key (0: none)
};
// candidate pairs (row, point) of the batch rows left open by tier 1, Stage VII candidates
// (row, old point, key) and the rows' exact K nearest neighbours (written at their sorted
// positions of knn_k / knn_i [n][K]); stats[0] += candidate pairs, stats[1] += Stage VII ones
void insert_sweep(const InsertSweep& S, DevBuf& surv, int64_t* nsurv, DevBuf& s7, int64_t* ns7, float* knn_k,
                  int32_t* knn_i, unsigned long long* stats, cudaStream_t s);
// RNG search: query rows against every index point (tier 1 and the queries' K nearest)
struct SearchSweep {
  const float* XQ;         // [mq][Dp] query rows (zero padded to Dp)
  int64_t mq;
  int64_t row0;            // level position of query row 0; the rows are row0 .. row0+mq-1
  const int32_t* rowpos;   // [mq] row0 + j
  const int32_t* qparent;  // [mq] finest pivot (sorted position) whose ball holds the query, or -1
  const float* X;          // index points in sorted order [n][Dp]
  int64_t n;
  int Dp, K, metric;
  const __half* A;         // block_prep of X
  const uint8_t* nbr_i;
  const float* nbr_k;
  const int32_t* parent;   // [n] finest pivot, sorted position
  const uint32_t* gpar;    // finest layer's guidance bitmask
  int64_t gpar_words;
  int small_buffers = 0;   // testing: a tiny first survivor buffer, so the retry runs
};
// pairs (row0 + j, point) tier 1 leaves open, and the rows' exact K nearest (written at their
// positions of knn_k / knn_i); stats[0] += candidate pairs, [1] += queued tests, [2] += retries
void search_sweep(const SearchSweep& S, DevBuf& surv, int64_t* nsurv, float* knn_k, int32_t* knn_i,
                  unsigned long long* stats, cudaStream_t s);
// maxe[sorted position] = FP32 upper bound of the point's longest edge key (edges in original ids)
void edge_max_keys(const uint64_t* edges, int64_t ne, const int32_t* rank, const float* X, int Dp, int metric,
                   float* maxe, int64_t n, cudaStream_t s);
// the old edges no batch point lies strictly inside of (Stage VII), written to kept; returns
// their count; stats[0] += lune tests, stats[1] += FP64 decisions
int64_t stage7_remove(const uint64_t* edges, int64_t ne, int64_t n_old, const int4* s7, int64_t ns7, const float* X,
                      int D, int Dp, int metric, const int32_t* order, const int32_t* rank, uint64_t* kept,
                      unsigned long long* stats, cudaStream_t s);

}  // namespace grng
