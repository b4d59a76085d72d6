// api.cu -- C ABI entry points and host orchestration (see include/grng.h).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdio>
#include <cstring>
#include <new>
#include <string>
#include <vector>

#include "../../include/grng.h"
#include "common.cuh"
#include "internal.h"

namespace grng {

static thread_local std::string g_last_error;

[[noreturn]] void fail(int status, const std::string& msg) { throw Failure{status, msg}; }
void set_last_error(const std::string& msg) { g_last_error = msg; }

static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
unsigned long long launches() { return g_launches.load(std::memory_order_relaxed); }

void cuda_check(cudaError_t e, const char* what) {
  if (e == cudaSuccess) return;
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) fail(GRNG_ENOMEM, m);
  fail(GRNG_ECUDA, m);
}

__global__ void compose_parent_kernel(const int32_t* __restrict__ rank_prev, const int32_t* __restrict__ assign,
                                      int64_t m, int32_t* __restrict__ key) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) key[t] = rank_prev[assign[t]];
}
__global__ void permute_parent_kernel(const int32_t* __restrict__ key, const int32_t* __restrict__ order,
                                      int64_t m, int32_t* __restrict__ out) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < m) out[s] = key[order[s]];
}
__global__ void permute_radius_kernel(const double* __restrict__ r, const int32_t* __restrict__ order, int64_t m,
                                      double* __restrict__ r64, float* __restrict__ rlo, float* __restrict__ rhi) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < m) {
    double v = r[order[s]];
    r64[s] = v;
    rlo[s] = __double2float_rd(v);
    rhi[s] = __double2float_ru(v);
  }
}
__global__ void permute_hi_kernel(const double* __restrict__ r, const int32_t* __restrict__ order, int64_t m,
                                  float* __restrict__ hi) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < m) hi[s] = __double2float_ru(r[order[s]]);
}
__global__ void iota_kernel(int32_t* a, int64_t m) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) a[i] = (int32_t)i;
}
__global__ void compose_ids_kernel(const int32_t* __restrict__ piv, const int32_t* __restrict__ order, int64_t m,
                                   int32_t* __restrict__ out) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < m) out[s] = piv[order[s]];
}
__global__ void edges_to_pairs_kernel(const uint64_t* __restrict__ k, int64_t m, int32_t* __restrict__ ij) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    ij[2 * i] = (int32_t)(k[i] >> 32);
    ij[2 * i + 1] = (int32_t)(k[i] & 0xffffffffu);
  }
}

// batch points in sorted positions: is_new[s] = 1 when the point at s has id >= n0
__global__ void mark_new_kernel(const int32_t* __restrict__ order, int64_t n, int64_t n0, uint8_t* __restrict__ is_new) {
  int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s < n) is_new[s] = order[s] >= n0 ? 1 : 0;
}
__global__ void batch_pos_kernel(const int32_t* __restrict__ rank, int64_t n0, int64_t m, uint64_t* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) out[t] = (uint64_t)(uint32_t)rank[n0 + t];
}
__global__ void narrow_kernel(const uint64_t* __restrict__ in, int64_t m, int32_t* __restrict__ out) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) out[t] = (int32_t)in[t];
}

// ---- search (queries that do not join the index) ----------------------------------------
__global__ void iota_from_kernel(int32_t* a, int64_t m, int64_t base) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) a[i] = (int32_t)(base + i);
}
// a query's parent for Theorem 1: its nearest finest pivot (sorted position) when the query
// lies in that pivot's ball D(p, r) (Eq. 2), else -1 (no pivot's GRNG links cover it)
__global__ void search_parent_kernel(const int32_t* __restrict__ assign, const double* __restrict__ dist,
                                     const double* __restrict__ radius, const int32_t* __restrict__ rank, int64_t m,
                                     int32_t* __restrict__ parent, unsigned long long* __restrict__ outside) {
  int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const int a = assign[t];
  const bool in = dist[t] <= radius[a];
  parent[t] = in ? rank[a] : -1;
  if (!in) atomicAdd(outside, 1ull);
}
// an edge (index id, n + j) of the level's output becomes (j, index id)
__global__ void search_key_kernel(uint64_t* __restrict__ k, int64_t ne, int64_t n) {
  int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= ne) return;
  const uint64_t v = k[i];
  const uint64_t lo = v >> 32, hi = v & 0xffffffffu;  // lo < n <= hi
  k[i] = ((hi - (uint64_t)n) << 32) | lo;
}
// CSR of the sorted (query, id) keys: nbr[i] = id, off[j] = first i of query j, off[m] = ne
__global__ void search_csr_kernel(const uint64_t* __restrict__ k, int64_t ne, int64_t m, int64_t* __restrict__ off,
                                  int32_t* __restrict__ nbr) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i > ne) return;
  if (i < ne) nbr[i] = (int32_t)(k[i] & 0xffffffffu);
  const int64_t prev = i == 0 ? -1 : (int64_t)(k[i - 1] >> 32);
  const int64_t cur = i == ne ? m : (int64_t)(k[i] >> 32);
  for (int64_t j = prev + 1; j <= cur; ++j) off[j] = i;
}

static inline unsigned nblk(int64_t m, int b = 256) { return (unsigned)((m + b - 1) / b); }

struct Layer {
  bool built = false, linked = false;
  int64_t m = 0;
  std::vector<int32_t> piv_h;
  DevBuf piv, Xp, assign, mdist, radius, delta;
  DevBuf order, rank, Xs, parent_s, r64s, rlos, rhis, ids_s;
  DevBuf dhis;    // FP32 upper bound of delta_max, sorted order
  DevBuf pdh;     // FP32 upper bound of d(pivot, its parent pivot), sorted order (layers > 0)
  DevBuf cstart;  // [m+1] children range in the next finer level (points for the finest)
  DevBuf gx, gg;
  int64_t words = 0;
  LevelStats st{};
  double assign_ms = 0, link_ms = 0, link_tile_ms = 0, assign_kernel_ms = 0;
  unsigned long long assign_amb = 0, assign_fp64 = 0, assign_tc = 0, assign_full = 0;
};

struct Timer {
  cudaEvent_t a, b;
  cudaStream_t s;
  explicit Timer(cudaStream_t st) : s(st) {
    GRNG_CUDA(cudaEventCreate(&a));
    GRNG_CUDA(cudaEventCreate(&b));
    GRNG_CUDA(cudaEventRecord(a, s));
  }
  double stop() {
    GRNG_CUDA(cudaEventRecord(b, s));
    GRNG_CUDA(cudaEventSynchronize(b));
    float ms = 0;
    GRNG_CUDA(cudaEventElapsedTime(&ms, a, b));
    return ms;
  }
  ~Timer() {
    cudaEventDestroy(a);
    cudaEventDestroy(b);
  }
};

}  // namespace grng

using namespace grng;

struct grng_index {
  int device = 0;
  cudaStream_t stream = nullptr;
  grng_opts opts{};
  int64_t n = 0;
  int D = 0, Dp = 0, metric = 0, K = 32;
  DevBuf X, ids;
  std::vector<Layer> layers;
  bool sorted = false;
  DevBuf xorder, xrank, Xs, xparent, xpdh;
  DevBuf edges;
  int64_t n_edges = 0;
  bool rng_built = false;
  LevelStats rng_st{};
  double rng_ms = 0, rng_tile_ms = 0, sort_ms = 0;
  double insert_ms = 0;  // batched insertion totals
  int64_t insert_batches = 0, inserted = 0;
  struct {
    long long changed_pivots = 0, grng_pairs = 0, grng_linked = 0, candidates = 0, survivors = 0,
              s7_candidates = 0, s7_tests = 0, s7_fp64 = 0, new_edges = 0, removed_edges = 0;
  } ins;
  DevBuf mlp;            // ranking network parameters (learned shortlist), or empty
  DevBuf rec_f, rec_y;   // recorded training samples of the last RNG build
  int64_t rec_n = 0;
  double skel_beta = 2.0;  // the stored graph: the RNG (2) or a beta-skeleton (1 <= beta < 2)
  int64_t version = 0;   // bumped whenever the points, their order or their parents change
  struct {               // search: rows kept for one index version, and the last result
    int64_t version = -1, cap = 0;
    DevBuf X, orig, parent, knn_k, knn_i;  // [n + cap] index rows (sorted order), then queries
    DevBuf A, nb_i, nb_k;                  // in-block keys and neighbours of the index blocks
    DevBuf off, nbrs;
    int64_t m = 0, total = 0;
    long long batches = 0, queries = 0, outside = 0, candidates = 0, survivors = 0, neighbours = 0;
    long long queued = 0, retries = 0;
    double ms = 0, last_ms = 0, assign_ms = 0, sweep_ms = 0, tiers_ms = 0;  // last batch's phases
    LevelStats st{};                                                     // last batch's tiers
  } srch;
};

namespace {

grng_status guard_status(const Failure& f) {
  g_last_error = f.msg;
  return f.status;
}

template <class F>
grng_status guarded(grng_index* idx, F&& fn) {
  try {
    if (idx) GRNG_CUDA(cudaSetDevice(idx->device));
    fn();
    g_last_error.clear();
    return GRNG_OK;
  } catch (const Failure& f) {
    return guard_status(f);
  } catch (const std::bad_alloc&) {
    g_last_error = "host allocation failed";
    return GRNG_ENOMEM;
  } catch (...) {
    g_last_error = "unexpected internal exception";
    return GRNG_EINTERNAL;
  }
}

void copy_out(void* dst, const void* src_dev, size_t bytes, cudaStream_t s) {
  if (!dst || !bytes) return;
  GRNG_CUDA(cudaMemcpyAsync(dst, src_dev, bytes, cudaMemcpyDefault, s));
}

int padded_dim(int d) { return d <= 8 ? 8 : d <= 16 ? 16 : ((d + 31) / 32) * 32; }

void sort_exemplars(grng_index* ix);

// DFS order of every layer (pivots grouped under their parents, coarsest first) and
// of the points; coordinates and radii gathered into that order.
void ensure_sorted(grng_index* ix) {
  if (ix->sorted) return;
  cudaStream_t s = ix->stream;
  Timer tm(s);
  const int L = (int)ix->layers.size();
  DevBuf key, tmp;
  for (int l = 0; l < L; ++l) {
    Layer& ly = ix->layers[l];
    const int64_t m = ly.m;
    GRNG_CUDA(ly.order.alloc(m * 4));
    GRNG_CUDA(ly.rank.alloc(m * 4));
    GRNG_CUDA(ly.parent_s.alloc(m * 4));
    GRNG_CUDA(key.alloc(m * 4));
    if (l == 0) {
      iota_kernel<<<nblk(m), 256, 0, s>>>(ly.order.as<int32_t>(), m); note_launch();
      iota_kernel<<<nblk(m), 256, 0, s>>>(ly.rank.as<int32_t>(), m); note_launch();
      GRNG_CUDA(cudaMemsetAsync(ly.parent_s.p, 0xff, m * 4, s));
    } else {
      Layer& up = ix->layers[l - 1];  // up.assign maps this layer's pivots to up's positions
      compose_parent_kernel<<<nblk(m), 256, 0, s>>>(up.rank.as<int32_t>(), up.assign.as<int32_t>(), m,
                                                     key.as<int32_t>()); note_launch();
      stable_order(key.as<int32_t>(), m, up.m, ly.order.as<int32_t>(), ly.rank.as<int32_t>(), tmp, s);
      permute_parent_kernel<<<nblk(m), 256, 0, s>>>(key.as<int32_t>(), ly.order.as<int32_t>(), m,
                                                     ly.parent_s.as<int32_t>()); note_launch();
    }
    GRNG_CUDA(ly.ids_s.alloc(m * 4));
    compose_ids_kernel<<<nblk(m), 256, 0, s>>>(ly.piv.as<int32_t>(), ly.order.as<int32_t>(), m,
                                                ly.ids_s.as<int32_t>()); note_launch();
    GRNG_CUDA(ly.Xs.alloc((size_t)m * ix->Dp * 4));
    gather_rows(ix->X.as<float>(), ix->Dp, ly.ids_s.as<int32_t>(), m, ly.Xs.as<float>(), s);
    GRNG_CUDA(ly.r64s.alloc(m * 8));
    GRNG_CUDA(ly.rlos.alloc(m * 4));
    GRNG_CUDA(ly.rhis.alloc(m * 4));
    permute_radius_kernel<<<nblk(m), 256, 0, s>>>(ly.radius.as<double>(), ly.order.as<int32_t>(), m,
                                                   ly.r64s.as<double>(), ly.rlos.as<float>(), ly.rhis.as<float>()); note_launch();
    GRNG_CUDA(ly.dhis.alloc(m * 4));
    permute_hi_kernel<<<nblk(m), 256, 0, s>>>(ly.delta.as<double>(), ly.order.as<int32_t>(), m,
                                               ly.dhis.as<float>()); note_launch();
    GRNG_CUDA(cudaGetLastError());
  }
  for (int l = 0; l + 1 < L; ++l) {
    Layer& ly = ix->layers[l];
    Layer& nx = ix->layers[l + 1];
    GRNG_CUDA(nx.pdh.alloc(nx.m * 4));  // ly.mdist is indexed by the finer layer's pivot positions
    permute_hi_kernel<<<nblk(nx.m), 256, 0, s>>>(ly.mdist.as<double>(), nx.order.as<int32_t>(), nx.m,
                                                  nx.pdh.as<float>()); note_launch();
    GRNG_CUDA(ly.cstart.alloc((ly.m + 1) * 4));
    child_ranges(ix->layers[l + 1].parent_s.as<int32_t>(), ix->layers[l + 1].m, ly.m, ly.cstart.as<int32_t>(), s);
  }
  sort_exemplars(ix);
  GRNG_CUDA(cudaStreamSynchronize(s));
  ix->sort_ms = tm.stop();
  ix->sorted = true;
}

// The points in DFS order of the finest layer (grouped under their pivots, pivots in their
// own DFS order), with their parents, parent distances and coordinates in that order.
void sort_exemplars(grng_index* ix) {
  cudaStream_t s = ix->stream;
  const int L = (int)ix->layers.size();
  DevBuf key, tmp;
  const int64_t n = ix->n;
  Layer& fin = ix->layers[L - 1];
  GRNG_CUDA(ix->xorder.alloc(n * 4));
  GRNG_CUDA(ix->xrank.alloc(n * 4));
  GRNG_CUDA(ix->xparent.alloc(n * 4));
  GRNG_CUDA(key.alloc(n * 4));
  compose_parent_kernel<<<nblk(n), 256, 0, s>>>(fin.rank.as<int32_t>(), fin.assign.as<int32_t>(), n,
                                                 key.as<int32_t>()); note_launch();
  stable_order(key.as<int32_t>(), n, fin.m, ix->xorder.as<int32_t>(), ix->xrank.as<int32_t>(), tmp, s);
  permute_parent_kernel<<<nblk(n), 256, 0, s>>>(key.as<int32_t>(), ix->xorder.as<int32_t>(), n,
                                                 ix->xparent.as<int32_t>()); note_launch();
  GRNG_CUDA(fin.cstart.alloc((fin.m + 1) * 4));
  child_ranges(ix->xparent.as<int32_t>(), n, fin.m, fin.cstart.as<int32_t>(), s);
  GRNG_CUDA(ix->xpdh.alloc(n * 4));
  permute_hi_kernel<<<nblk(n), 256, 0, s>>>(fin.mdist.as<double>(), ix->xorder.as<int32_t>(), n,
                                             ix->xpdh.as<float>()); note_launch();
  GRNG_CUDA(ix->Xs.alloc((size_t)n * ix->Dp * 4));
  gather_rows(ix->X.as<float>(), ix->Dp, ix->xorder.as<int32_t>(), n, ix->Xs.as<float>(), s);
  GRNG_CUDA(cudaGetLastError());
  GRNG_CUDA(cudaStreamSynchronize(s));
  ix->version += 1;
}

// layers 0..count-1 as the ancestors of a level (the last one is the direct parent,
// whose delta_max bounds the distance to its members; higher ones use their radius)
Ancestors ancestors_of(grng_index* ix, int count) {
  Ancestors a;
  a.n = count;
  for (int l = 0; l < count; ++l) {
    Layer& ly = ix->layers[l];
    a.X[l] = ly.Xs.as<float>();
    a.Rhi[l] = (l == count - 1) ? ly.dhis.as<float>() : ly.rhis.as<float>();
    a.cstart[l] = ly.cstart.as<int32_t>();
    a.m[l] = ly.m;
  }
  return a;
}

void check_layer(const grng_index* ix, int32_t layer) {
  if (layer < 0 || layer >= (int32_t)ix->layers.size()) fail(GRNG_EINVAL, "layer out of range");
}

// CSR output of a bitmask (rows [r0, r1) in pivot_idx order)
void output_rows(grng_index* ix, const uint32_t* bits, int64_t words, const int32_t* rank, int64_t m, int64_t r0,
                 int64_t r1, int64_t* off, int32_t* adj, int64_t cap, int64_t* needed) {
  cudaStream_t s = ix->stream;
  const int64_t rows = r1 - r0;
  DevBuf doff, dadj;
  GRNG_CUDA(doff.alloc((size_t)(rows + 1) * 8));
  bitmask_rows(bits, words, rank, m, r0, r1, doff.as<int64_t>(), nullptr, s);
  int64_t total = 0;
  GRNG_CUDA(cudaMemcpyAsync(&total, doff.as<int64_t>() + rows, 8, cudaMemcpyDeviceToHost, s));
  GRNG_CUDA(cudaStreamSynchronize(s));
  if (needed) *needed = total;
  copy_out(off, doff.p, (size_t)(rows + 1) * 8, s);
  GRNG_CUDA(cudaStreamSynchronize(s));
  if (!adj) return;
  if (cap < total) fail(GRNG_ETRUNC, "adjacency buffer too small");
  GRNG_CUDA(dadj.alloc((size_t)std::max<int64_t>(total, 1) * 4));
  bitmask_rows(bits, words, rank, m, r0, r1, doff.as<int64_t>(), dadj.as<int32_t>(), s);
  copy_out(adj, dadj.p, (size_t)total * 4, s);
  GRNG_CUDA(cudaStreamSynchronize(s));
}

void level_json(std::string& js, const char* name, const LevelStats& st) {
  static const char* nm[] = {"candidate_pairs", "quick_links", "tier1_survivors", "tier2a_links", "tier2a_pending",
                             "tier2a_unresolved", "tier2a_blocked", "tier2b_links", "tier2b_pending",
                             "tier2b_unresolved", "tier2b_blocked", "tier3_pairs", "fp64_triples",
                             "fp64_blocking", "edges", "tier3_overflows", "tier3_nodes_tested",
                             "list_certified", "range_pairs", "range_lists_cut", "range_listed_nodes",
                             "range_links", "range_nodes_tested", "tier3_blocked",
                             "tier3_descent_blocked", "learned_pairs", "learned_candidates", "learned_tests",
                             "learned_blocked", "learned_pool_hits", "tier1_attempts", "tier23_attempts",
                             "range_both_covered", "range_unused", "range_entries_read", "tier3_cycles_top",
                             "tier3_cycles_mid", "tier3_cycles_leaf", "tier3_pairs_mid", "tier3_probe_blocked",
                             "tier1_full_tests", "probe_blocked_before_lists"};
  char buf[1024];
  js += "\"";
  js += name;
  js += "\":{";
  for (int i = 0; i < 42; ++i) {
    snprintf(buf, sizeof(buf), "%s\"%s\":%llu", i ? "," : "", nm[i], (unsigned long long)st.c[i]);
    js += buf;
  }
  snprintf(buf, sizeof(buf),
           ",\"phase_ms\":{\"prep\":%.3f,\"tiles\":%.3f,\"tier2a\":%.3f,\"tier2b\":%.3f,\"range\":%.3f,"
           "\"tier3\":%.3f,\"recheck_emit\":%.3f},\"kernel_ms\":{\"tiles\":%.4f,\"tier3\":%.4f,\"lists\":%.4f,"
           "\"range_phase\":%.4f}",
           st.ms[0], st.ms[1], st.ms[2], st.ms[3], st.ms[4], st.ms[5], st.ms[6], st.kms[0], st.kms[1], st.kms[2],
           st.kms[3]);
  js += buf;
  js += "}";
}

}  // namespace

extern "C" {

void grng_default_opts(grng_opts* o) {
  if (!o) return;
  memset(o, 0, sizeof(*o));
  o->metric = GRNG_L2;
  o->precision = GRNG_FP32;
  o->n_layers = 1;
  o->knn_k = 32;
}

const char* grng_last_error(void) { return g_last_error.c_str(); }

grng_status grng_create(grng_index** out, const float* pts, int64_t n, int32_t dim, const grng_opts* opts) {
  if (!out) {
    g_last_error = "out is NULL";
    return GRNG_EINVAL;
  }
  *out = nullptr;
  grng_index* ix = nullptr;
  grng_status st = guarded(nullptr, [&] {
    if (!pts || !opts) fail(GRNG_EINVAL, "pts and opts must not be NULL");
    if (n < 1 || n >= (int64_t)1 << 31) fail(GRNG_EINVAL, "n must be in [1, 2^31)");
    if (dim < 1 || dim > 4096) fail(GRNG_EINVAL, "dim must be in [1, 4096]");
    if (opts->metric != GRNG_L2 && opts->metric != GRNG_L1) fail(GRNG_EINVAL, "unknown metric");
    if (opts->n_layers < 1 || opts->n_layers > 16) fail(GRNG_EINVAL, "n_layers must be in [1, 16]");
    if (opts->knn_k < 0 || opts->knn_k > GRNG_KMAX) fail(GRNG_EINVAL, "knn_k must be in [0, 32]");
    if (opts->precision != GRNG_FP32 && opts->precision != GRNG_BF16)
      fail(GRNG_ENOTIMPL, "FP32 and BF16 tile precisions are built");
    if (opts->k_shortlist < 0 || opts->k_shortlist > GRNG_MLP_KMAX)
      fail(GRNG_EINVAL, "k_shortlist must be in [0, 16]");
    if (opts->k_shortlist > 0 && (!opts->mlp_weights || opts->mlp_bytes != (size_t)GRNG_MLP_NPARAM * 4))
      fail(GRNG_EINVAL, "a shortlist needs mlp_weights of grng_mlp_nparams() floats (mlp_bytes)");
    if (opts->reserved != 0 ||
        (opts->flags & ~(uint64_t)(GRNG_FLAG_SHORT_LISTS | GRNG_FLAG_RECORD_MLP | GRNG_FLAG_SMALL_BUFFERS)) != 0)
      fail(GRNG_EINVAL, "reserved fields must be 0");
    ix = new grng_index();
    GRNG_CUDA(cudaGetDevice(&ix->device));
    ix->opts = *opts;
    ix->stream = static_cast<cudaStream_t>(opts->cuda_stream);
    ix->n = n;
    ix->D = dim;
    ix->Dp = padded_dim(dim);
    ix->metric = opts->metric;
    ix->K = opts->knn_k ? opts->knn_k : 32;
    ix->layers.resize(opts->n_layers);
    cudaStream_t s = ix->stream;
    if (opts->k_shortlist > 0) {
      GRNG_CUDA(ix->mlp.alloc((size_t)GRNG_MLP_NPARAM * 4));
      GRNG_CUDA(cudaMemcpyAsync(ix->mlp.p, opts->mlp_weights, (size_t)GRNG_MLP_NPARAM * 4, cudaMemcpyDefault, s));
    }
    ix->opts.mlp_weights = nullptr;  // the caller's pointer is not kept
    GRNG_CUDA(ix->X.alloc((size_t)n * ix->Dp * 4));
    GRNG_CUDA(cudaMemsetAsync(ix->X.p, 0, (size_t)n * ix->Dp * 4, s));
    GRNG_CUDA(cudaMemcpy2DAsync(ix->X.p, (size_t)ix->Dp * 4, pts, (size_t)dim * 4, (size_t)dim * 4, (size_t)n,
                                cudaMemcpyDefault, s));
    GRNG_CUDA(ix->ids.alloc((size_t)n * 4));
    iota_kernel<<<nblk(n), 256, 0, s>>>(ix->ids.as<int32_t>(), n); note_launch();
    GRNG_CUDA(cudaGetLastError());
    GRNG_CUDA(cudaStreamSynchronize(s));
  });
  if (st != GRNG_OK) {
    delete ix;
    return st;
  }
  *out = ix;
  return GRNG_OK;
}

void grng_destroy(grng_index* idx) {
  if (!idx) return;
  cudaSetDevice(idx->device);
  cudaStreamSynchronize(idx->stream);
  delete idx;
}

grng_status grng_build_layer(grng_index* ix, int32_t layer, const int32_t* pivot_idx, int32_t m, int32_t* assign,
                             double* radius, double* delta_max) {
  if (!ix) {
    g_last_error = "index is NULL";
    return GRNG_EINVAL;
  }
  return guarded(ix, [&] {
    check_layer(ix, layer);
    const int L = (int)ix->layers.size();
    if (!pivot_idx || m < 1 || m > ix->n) fail(GRNG_EINVAL, "need 1 <= m <= n pivot indices");
    if (layer < L - 1 && !ix->layers[layer + 1].built)
      fail(GRNG_ESTATE, "layers are built finest first: build the next finer layer first");
    cudaStream_t s = ix->stream;
    Layer& ly = ix->layers[layer];
    std::vector<int32_t> h(m);
    GRNG_CUDA(cudaMemcpyAsync(h.data(), pivot_idx, (size_t)m * 4, cudaMemcpyDefault, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    std::vector<char> seen(ix->n, 0);
    for (int32_t v : h) {
      if (v < 0 || v >= ix->n) fail(GRNG_EINVAL, "pivot index out of range");
      if (seen[v]) fail(GRNG_EINVAL, "duplicate pivot index");
      seen[v] = 1;
    }
    if (layer < L - 1) {
      std::vector<char> fine(ix->n, 0);
      for (int32_t v : ix->layers[layer + 1].piv_h) fine[v] = 1;
      for (int32_t v : h)
        if (!fine[v]) fail(GRNG_EINVAL, "layers must nest: a coarse pivot is missing from the next finer layer");
    }
    // invalidate everything that depends on this layer
    for (int l = 0; l < L; ++l) ix->layers[l].linked = false;
    for (int l = 0; l < layer; ++l) ix->layers[l].built = false;
    ix->sorted = false;
    ix->rng_built = false;
    Timer tm(s);
    ly.m = m;
    ly.piv_h = h;
    GRNG_CUDA(ly.piv.alloc((size_t)m * 4));
    GRNG_CUDA(cudaMemcpyAsync(ly.piv.p, h.data(), (size_t)m * 4, cudaMemcpyHostToDevice, s));
    GRNG_CUDA(ly.Xp.alloc((size_t)m * ix->Dp * 4));
    gather_rows(ix->X.as<float>(), ix->Dp, ly.piv.as<int32_t>(), m, ly.Xp.as<float>(), s);
    const bool finest = layer == L - 1;
    const int64_t nmem = finest ? ix->n : ix->layers[layer + 1].m;
    const float* Xmem = finest ? ix->X.as<float>() : ix->layers[layer + 1].Xp.as<float>();
    const int32_t* mem_id = finest ? ix->ids.as<int32_t>() : ix->layers[layer + 1].piv.as<int32_t>();
    const double* mem_r = finest ? nullptr : ix->layers[layer + 1].radius.as<double>();
    GRNG_CUDA(ly.assign.alloc((size_t)nmem * 4));
    GRNG_CUDA(ly.mdist.alloc((size_t)nmem * 8));
    GRNG_CUDA(ly.radius.alloc((size_t)m * 8));
    GRNG_CUDA(ly.delta.alloc((size_t)m * 8));
    AssignOut ao{ly.assign.as<int32_t>(), ly.mdist.as<double>(), ly.radius.as<double>(), ly.delta.as<double>()};
    unsigned long long ast[5] = {0, 0, 0, 0, 0};
    assign_layer(Xmem, mem_id, mem_r, nmem, ly.Xp.as<float>(), ly.piv.as<int32_t>(), m, ix->n, ix->D, ix->Dp,
                 ix->metric, ao, ast, s, ix->opts.precision == GRNG_BF16,
                 ix->opts.spin_limit > 0 ? ix->opts.spin_limit : 1ll << 24);
    ly.assign_amb = ast[0];
    ly.assign_fp64 = ast[1];
    ly.assign_kernel_ms = (double)ast[2] / 1000.0;
    ly.assign_tc = ast[3];
    ly.assign_full = ast[4];
    ly.built = true;
    ly.assign_ms = tm.stop();
    copy_out(assign, ly.assign.p, (size_t)nmem * 4, s);
    copy_out(radius, ly.radius.p, (size_t)m * 8, s);
    copy_out(delta_max, ly.delta.p, (size_t)m * 8, s);
    GRNG_CUDA(cudaStreamSynchronize(s));
  });
}

grng_status grng_link_pivots(grng_index* ix, int32_t layer, const double* radius_override, int64_t* off,
                             int32_t* adj, int64_t adj_cap, int64_t* adj_needed) {
  if (!ix) {
    g_last_error = "index is NULL";
    return GRNG_EINVAL;
  }
  return guarded(ix, [&] {
    check_layer(ix, layer);
    for (auto& l : ix->layers)
      if (!l.built) fail(GRNG_ESTATE, "every layer must be built before linking");
    if (!radius_override && layer > 0 && !ix->layers[layer - 1].linked)
      fail(GRNG_ESTATE, "link the coarser layer first (its GRNG guides this one, Theorem 2)");
    ensure_sorted(ix);
    cudaStream_t s = ix->stream;
    Layer& ly = ix->layers[layer];
    const int64_t m = ly.m;
    const int64_t words = (m + 31) / 32;
    LevelIn in{};
    in.X = ly.Xs.as<float>();
    in.n = m;
    in.D = ix->D;
    in.Dp = ix->Dp;
    in.metric = ix->metric;
    in.grng = 1;
    in.K = ix->K;
    in.orig = ly.order.as<int32_t>();
    in.anc = ancestors_of(ix, layer);
    in.lmax = (ix->opts.flags & GRNG_FLAG_SHORT_LISTS) ? 16 : 0;
    in.small_buffers = (ix->opts.flags & GRNG_FLAG_SMALL_BUFFERS) ? 1 : 0;
    in.pdist_hi = layer > 0 ? ly.pdh.as<float>() : nullptr;
    DevBuf ovr, o64, olo, ohi, tgx, tgg;
    Timer tm(s);
    if (radius_override) {
      GRNG_CUDA(ovr.alloc((size_t)m * 8));
      GRNG_CUDA(cudaMemcpyAsync(ovr.p, radius_override, (size_t)m * 8, cudaMemcpyDefault, s));
      std::vector<double> hr(m);
      GRNG_CUDA(cudaMemcpyAsync(hr.data(), ovr.p, (size_t)m * 8, cudaMemcpyDeviceToHost, s));
      GRNG_CUDA(cudaStreamSynchronize(s));
      for (double v : hr)
        if (!(v >= 0.0) || v == INFINITY) fail(GRNG_EINVAL, "radii must be finite and non-negative");
      GRNG_CUDA(o64.alloc((size_t)m * 8));
      GRNG_CUDA(olo.alloc((size_t)m * 4));
      GRNG_CUDA(ohi.alloc((size_t)m * 4));
      permute_radius_kernel<<<nblk(m), 256, 0, s>>>(ovr.as<double>(), ly.order.as<int32_t>(), m, o64.as<double>(),
                                                     olo.as<float>(), ohi.as<float>()); note_launch();
      GRNG_CUDA(cudaGetLastError());
      in.r64 = o64.as<double>();
      in.rlo = olo.as<float>();
      in.rhi = ohi.as<float>();
      in.parent = nullptr;
      in.gpar = nullptr;
      GRNG_CUDA(tgx.alloc((size_t)m * words * 4));
      GRNG_CUDA(tgg.alloc((size_t)m * words * 4));
      LevelOut lo;
      lo.gx = tgx.as<uint32_t>();
      lo.gg = tgg.as<uint32_t>();
      lo.words = words;
      LevelStats st;
      run_level(in, lo, st, s);
      output_rows(ix, tgx.as<uint32_t>(), words, ly.rank.as<int32_t>(), m, 0, m, off, adj, adj_cap, adj_needed);
      return;
    }
    in.r64 = ly.r64s.as<double>();
    in.rlo = ly.rlos.as<float>();
    in.rhi = ly.rhis.as<float>();
    if (layer > 0) {
      in.parent = ly.parent_s.as<int32_t>();
      in.gpar = ix->layers[layer - 1].gg.as<uint32_t>();
      in.gpar_words = ix->layers[layer - 1].words;
    }
    GRNG_CUDA(ly.gx.alloc((size_t)m * words * 4));
    GRNG_CUDA(ly.gg.alloc((size_t)m * words * 4));
    ly.words = words;
    LevelOut lo;
    lo.gx = ly.gx.as<uint32_t>();
    lo.gg = ly.gg.as<uint32_t>();
    lo.words = words;
    float tile_ms = 0;
    run_level(in, lo, ly.st, s, &tile_ms);
    ly.link_tile_ms = tile_ms;
    ly.link_ms = tm.stop();
    ly.linked = true;
    for (int l = layer + 1; l < (int)ix->layers.size(); ++l) ix->layers[l].linked = false;
    ix->rng_built = false;
    if (off || adj_needed)
      output_rows(ix, ly.gx.as<uint32_t>(), words, ly.rank.as<int32_t>(), m, 0, m, off, adj, adj_cap, adj_needed);
  });
}

grng_status grng_adjacency_rows(grng_index* ix, int32_t layer, int64_t row_begin, int64_t row_end, int64_t* off,
                                int32_t* adj, int64_t adj_cap, int64_t* adj_needed) {
  if (!ix) {
    g_last_error = "index is NULL";
    return GRNG_EINVAL;
  }
  return guarded(ix, [&] {
    check_layer(ix, layer);
    Layer& ly = ix->layers[layer];
    if (!ly.linked) fail(GRNG_ESTATE, "layer is not linked");
    if (row_begin < 0 || row_end > ly.m || row_begin > row_end) fail(GRNG_EINVAL, "row range out of bounds");
    output_rows(ix, ly.gx.as<uint32_t>(), ly.words, ly.rank.as<int32_t>(), ly.m, row_begin, row_end, off, adj,
                adj_cap, adj_needed);
  });
}

// The exemplar level: the RNG (beta = 2) or a lune-based beta-skeleton with 1 <= beta < 2.
// A skeleton below 2 takes no guidance (Theorem 1 proves a point inside the lune of Eq. 1,
// not inside the smaller beta-lune), FP32 tiles and no learned shortlist; every bound the
// tiers derive from the lune of Eq. 1 still holds, since it contains the beta-lune.
static void build_exemplar_graph(grng_index* ix, double beta) {
  for (auto& l : ix->layers)
    if (!l.linked) fail(GRNG_ESTATE, "every layer must be built and linked");
  ensure_sorted(ix);
  cudaStream_t s = ix->stream;
  Layer& fin = ix->layers.back();
  const bool skel = beta < 2.0;
  Timer tm(s);
  LevelIn in{};
  in.X = ix->Xs.as<float>();
  in.n = ix->n;
  in.D = ix->D;
  in.Dp = ix->Dp;
  in.metric = ix->metric;
  in.grng = 0;
  in.K = ix->K;
  in.parent = skel ? nullptr : ix->xparent.as<int32_t>();
  in.gpar = skel ? nullptr : fin.gg.as<uint32_t>();
  in.gpar_words = skel ? 0 : fin.words;
  in.orig = ix->xorder.as<int32_t>();
  in.anc = ancestors_of(ix, (int)ix->layers.size());
  in.pdist_hi = ix->xpdh.as<float>();
  in.precision = (!skel && ix->opts.precision == GRNG_BF16) ? 1 : 0;
  if (ix->opts.spin_limit > 0) in.spin = ix->opts.spin_limit;
  in.mlp_params = (!skel && ix->mlp.p) ? ix->mlp.as<float>() : nullptr;
  in.kshort = (!skel && ix->mlp.p) ? ix->opts.k_shortlist : 0;
  in.mlp_record = (!skel && (ix->opts.flags & GRNG_FLAG_RECORD_MLP)) ? 1 : 0;
  in.small_buffers = (ix->opts.flags & GRNG_FLAG_SMALL_BUFFERS) ? 1 : 0;
  in.beta_lam = beta / 2.0;
  LevelOut lo;
  lo.edges = &ix->edges;
  lo.rec_f = &ix->rec_f;
  lo.rec_y = &ix->rec_y;
  float tile_ms = 0;
  run_level(in, lo, ix->rng_st, s, &tile_ms);
  ix->n_edges = lo.n_edges;
  ix->rec_n = lo.rec_n;
  DevBuf tmp;
  if (ix->n_edges > 1) sort_u64(ix->edges.as<uint64_t>(), ix->n_edges, tmp, s);
  ix->rng_tile_ms = tile_ms;
  ix->rng_ms = tm.stop();
  ix->rng_built = true;
  ix->skel_beta = beta;
}

grng_status rng_build_exact(grng_index* ix) {
  if (!ix) {
    g_last_error = "index is NULL";
    return GRNG_EINVAL;
  }
  return guarded(ix, [&] { build_exemplar_graph(ix, 2.0); });
}

grng_status rng_build_skeleton(grng_index* ix, double beta) {
  if (!ix) {
    g_last_error = "index is NULL";
    return GRNG_EINVAL;
  }
  return guarded(ix, [&] {
    if (!(beta >= 1.0 && beta <= 2.0)) fail(GRNG_EINVAL, "beta must lie in [1, 2]");
    if (ix->metric != GRNG_L2 && beta < 2.0) fail(GRNG_EINVAL, "beta-skeletons below 2 need the L2 metric");
    build_exemplar_graph(ix, beta);
  });
}

grng_status grng_mlp_dataset(const grng_index* cix, float* feats, float* labels, int64_t cap, int64_t* count) {
  grng_index* ix = const_cast<grng_index*>(cix);
  if (!ix) {
    g_last_error = "index is NULL";
    return GRNG_EINVAL;
  }
  return guarded(ix, [&] {
    if (!ix->rng_built) fail(GRNG_ESTATE, "the RNG is not built");
    if (!(ix->opts.flags & GRNG_FLAG_RECORD_MLP)) fail(GRNG_ESTATE, "the index was created without GRNG_FLAG_RECORD_MLP");
    if (count) *count = ix->rec_n;
    if (!feats && !labels) return;
    if (cap < ix->rec_n) fail(GRNG_ETRUNC, "buffer smaller than the recorded sample count");
    cudaStream_t s = ix->stream;
    if (ix->rec_n > 0) {
      if (feats)
        GRNG_CUDA(cudaMemcpyAsync(feats, ix->rec_f.p, (size_t)ix->rec_n * GRNG_MLP_IN * 4, cudaMemcpyDefault, s));
      if (labels) GRNG_CUDA(cudaMemcpyAsync(labels, ix->rec_y.p, (size_t)ix->rec_n * 4, cudaMemcpyDefault, s));
    }
    GRNG_CUDA(cudaStreamSynchronize(s));
  });
}

grng_status rng_insert_batch(grng_index* ix, const float* pts, int64_t m) {
  if (!ix) {
    g_last_error = "index is NULL";
    return GRNG_EINVAL;
  }
  return guarded(ix, [&] {
    if (!pts || m < 1) fail(GRNG_EINVAL, "need pts and m >= 1");
    if (!ix->rng_built) fail(GRNG_ESTATE, "the RNG is not built");
    if (ix->skel_beta < 2.0) fail(GRNG_ESTATE, "the stored graph is a beta-skeleton, not the RNG");
    if (ix->n + m >= (int64_t)1 << 31) fail(GRNG_EINVAL, "n + m must stay below 2^31");
    cudaStream_t s = ix->stream;
    Timer tm(s);
    const int L = (int)ix->layers.size();
    const int Dp = ix->Dp, D = ix->D, K = ix->K, metric = ix->metric;
    // ---- the enlarged point set: old rows, then the batch (ids n .. n+m-1) ----------------
    const int64_t n0 = ix->n, n1 = n0 + m;
    {
      DevBuf X2, ids2;
      GRNG_CUDA(X2.alloc((size_t)n1 * Dp * 4));
      GRNG_CUDA(cudaMemcpyAsync(X2.p, ix->X.p, (size_t)n0 * Dp * 4, cudaMemcpyDeviceToDevice, s));
      float* Xnew = X2.as<float>() + n0 * Dp;
      GRNG_CUDA(cudaMemsetAsync(Xnew, 0, (size_t)m * Dp * 4, s));
      GRNG_CUDA(cudaMemcpy2DAsync(Xnew, (size_t)Dp * 4, pts, (size_t)D * 4, (size_t)D * 4, (size_t)m,
                                  cudaMemcpyDefault, s));
      GRNG_CUDA(ids2.alloc((size_t)n1 * 4));
      iota_kernel<<<nblk(n1), 256, 0, s>>>(ids2.as<int32_t>(), n1); note_launch();
      GRNG_CUDA(cudaGetLastError());
      GRNG_CUDA(cudaStreamSynchronize(s));
      ix->X = std::move(X2);
      ix->ids = std::move(ids2);
    }
    // ---- radii (Eq. 2; relative pivot domains, Sec. 3) ------------------------------------
    std::vector<DevBuf> changed(L);
    Layer& fin = ix->layers[L - 1];
    {
      const int64_t M = fin.m;
      DevBuf ab, db, rb, ddb, a2, d2;
      GRNG_CUDA(ab.alloc((size_t)m * 4));
      GRNG_CUDA(db.alloc((size_t)m * 8));
      GRNG_CUDA(rb.alloc((size_t)M * 8));
      GRNG_CUDA(ddb.alloc((size_t)M * 8));
      AssignOut ao{ab.as<int32_t>(), db.as<double>(), rb.as<double>(), ddb.as<double>()};
      assign_layer(ix->X.as<float>() + n0 * Dp, ix->ids.as<int32_t>() + n0, nullptr, m, fin.Xp.as<float>(),
                   fin.piv.as<int32_t>(), M, n1, D, Dp, metric, ao, nullptr, s, ix->opts.precision == GRNG_BF16,
                   ix->opts.spin_limit > 0 ? ix->opts.spin_limit : 1ll << 24);
      GRNG_CUDA(a2.alloc((size_t)n1 * 4));
      GRNG_CUDA(d2.alloc((size_t)n1 * 8));
      GRNG_CUDA(cudaMemcpyAsync(a2.p, fin.assign.p, (size_t)n0 * 4, cudaMemcpyDeviceToDevice, s));
      GRNG_CUDA(cudaMemcpyAsync(a2.as<int32_t>() + n0, ab.p, (size_t)m * 4, cudaMemcpyDeviceToDevice, s));
      GRNG_CUDA(cudaMemcpyAsync(d2.p, fin.mdist.p, (size_t)n0 * 8, cudaMemcpyDeviceToDevice, s));
      GRNG_CUDA(cudaMemcpyAsync(d2.as<double>() + n0, db.p, (size_t)m * 8, cudaMemcpyDeviceToDevice, s));
      GRNG_CUDA(changed[L - 1].alloc((size_t)M));
      merge_radii(fin.radius.as<double>(), fin.delta.as<double>(), rb.as<double>(), ddb.as<double>(), M,
                  changed[L - 1].as<uint8_t>(), s);
      GRNG_CUDA(cudaStreamSynchronize(s));
      fin.assign = std::move(a2);
      fin.mdist = std::move(d2);
    }
    for (int l = L - 2; l >= 0; --l) {  // coarse radii grow with their members' radii
      Layer& ly = ix->layers[l];
      Layer& fi = ix->layers[l + 1];
      DevBuf oldr;
      GRNG_CUDA(oldr.alloc((size_t)ly.m * 8));
      GRNG_CUDA(cudaMemcpyAsync(oldr.p, ly.radius.p, (size_t)ly.m * 8, cudaMemcpyDeviceToDevice, s));
      GRNG_CUDA(changed[l].alloc((size_t)ly.m));
      coarse_radii(ly.mdist.as<double>(), fi.radius.as<double>(), ly.assign.as<int32_t>(), fi.m,
                   ly.radius.as<double>(), oldr.as<double>(), ly.m, changed[l].as<uint8_t>(), s);
      GRNG_CUDA(cudaStreamSynchronize(s));
    }
    for (int l = 0; l < L; ++l) {  // the sorted copies of radii and delta_max
      Layer& ly = ix->layers[l];
      permute_radius_kernel<<<nblk(ly.m), 256, 0, s>>>(ly.radius.as<double>(), ly.order.as<int32_t>(), ly.m,
                                                       ly.r64s.as<double>(), ly.rlos.as<float>(),
                                                       ly.rhis.as<float>()); note_launch();
      permute_hi_kernel<<<nblk(ly.m), 256, 0, s>>>(ly.delta.as<double>(), ly.order.as<int32_t>(), ly.m,
                                                   ly.dhis.as<float>()); note_launch();
    }
    GRNG_CUDA(cudaGetLastError());
    // ---- GRNGs, coarsest first: a grown radius can only add links (definition, Sec. 2) ------
    DevBuf newg_prev;
    int64_t nnew_prev = 0;
    for (int l = 0; l < L; ++l) {
      Layer& ly = ix->layers[l];
      DevBuf chg_s, chg_list, pairs, newg_cur;
      GRNG_CUDA(chg_s.alloc((size_t)ly.m));
      GRNG_CUDA(chg_list.alloc((size_t)ly.m * 4));
      const int64_t nchg = changed_sorted(changed[l].as<uint8_t>(), ly.order.as<int32_t>(), ly.m,
                                         chg_s.as<uint8_t>(), chg_list.as<int32_t>(), s);
      const int64_t nnew = l > 0 ? nnew_prev : 0;
      ix->ins.changed_pivots += nchg;
      if (nchg == 0 && nnew == 0) {
        nnew_prev = 0;
        continue;
      }
      const int64_t np = grng_retest_pairs(
          chg_list.as<int32_t>(), nchg, chg_s.as<uint8_t>(), ly.m, ly.gx.as<uint32_t>(), ly.gg.as<uint32_t>(),
          ly.words, l > 0 ? ly.parent_s.as<int32_t>() : nullptr,
          l > 0 ? ix->layers[l - 1].gg.as<uint32_t>() : nullptr, l > 0 ? ix->layers[l - 1].words : 0,
          nnew ? newg_prev.as<int2>() : nullptr, nnew, l > 0 ? ix->layers[l - 1].cstart.as<int32_t>() : nullptr,
          pairs, s);
      ix->ins.grng_pairs += np;
      LevelIn in{};
      in.X = ly.Xs.as<float>();
      in.n = ly.m;
      in.D = D;
      in.Dp = Dp;
      in.metric = metric;
      in.grng = 1;
      in.K = K;
      in.orig = ly.order.as<int32_t>();
      in.anc = ancestors_of(ix, l);
      in.pdist_hi = l > 0 ? ly.pdh.as<float>() : nullptr;
      in.r64 = ly.r64s.as<double>();
      in.rlo = ly.rlos.as<float>();
      in.rhi = ly.rhis.as<float>();
      if (l > 0) {
        in.parent = ly.parent_s.as<int32_t>();
        in.gpar = ix->layers[l - 1].gg.as<uint32_t>();
        in.gpar_words = ix->layers[l - 1].words;
      }
      in.lists = 0;
      if (ix->opts.spin_limit > 0) in.spin = ix->opts.spin_limit;
      in.small_buffers = (ix->opts.flags & GRNG_FLAG_SMALL_BUFFERS) ? 1 : 0;
      LevelOut lo;
      lo.gx = ly.gx.as<uint32_t>();
      lo.gg = ly.gg.as<uint32_t>();
      lo.words = ly.words;
      lo.new_gg = &newg_cur;
      LevelStats st;
      run_pairs(in, lo, st, s, pairs.as<int2>(), np, nullptr, nullptr, false);
      ix->ins.grng_linked += lo.n_new_gg;
      newg_prev = std::move(newg_cur);
      nnew_prev = lo.n_new_gg;
    }
    // ---- the exemplars in DFS order of the finest layer, the batch among them ---------------
    ix->n = n1;
    sort_exemplars(ix);
    DevBuf is_new, bpos64, rowpos, XB, AB, nbB_i, nbB_k, A, nb_i, nb_k, maxe, knn_k, knn_i, surv, s7, newE;
    const int64_t strips = (m + 127) / 128;
    const int64_t nb1 = (n1 + 127) / 128;
    GRNG_CUDA(is_new.alloc((size_t)n1));
    GRNG_CUDA(bpos64.alloc((size_t)m * 8));
    GRNG_CUDA(rowpos.alloc((size_t)m * 4));
    mark_new_kernel<<<nblk(n1), 256, 0, s>>>(ix->xorder.as<int32_t>(), n1, n0, is_new.as<uint8_t>()); note_launch();
    batch_pos_kernel<<<nblk(m), 256, 0, s>>>(ix->xrank.as<int32_t>(), n0, m, bpos64.as<uint64_t>()); note_launch();
    GRNG_CUDA(cudaGetLastError());
    {
      DevBuf tmp;
      sort_u64(bpos64.as<uint64_t>(), m, tmp, s);  // batch rows in sorted order: coherent strips
    }
    narrow_kernel<<<nblk(m), 256, 0, s>>>(bpos64.as<uint64_t>(), m, rowpos.as<int32_t>()); note_launch();
    GRNG_CUDA(XB.alloc((size_t)strips * 128 * Dp * 4));
    GRNG_CUDA(cudaMemsetAsync(XB.p, 0, (size_t)strips * 128 * Dp * 4, s));
    gather_rows(ix->Xs.as<float>(), Dp, rowpos.as<int32_t>(), m, XB.as<float>(), s);
    GRNG_CUDA(AB.alloc((size_t)strips * 128 * 128 * 2));
    GRNG_CUDA(nbB_i.alloc((size_t)strips * 128 * GRNG_KIN));
    GRNG_CUDA(nbB_k.alloc((size_t)strips * 128 * GRNG_KIN * 4));
    block_prep(XB.as<float>(), m, Dp, metric, AB.as<__half>(), nbB_i.as<uint8_t>(), nbB_k.as<float>(), s);
    GRNG_CUDA(A.alloc((size_t)nb1 * 128 * 128 * 2));
    GRNG_CUDA(nb_i.alloc((size_t)nb1 * 128 * GRNG_KIN));
    GRNG_CUDA(nb_k.alloc((size_t)nb1 * 128 * GRNG_KIN * 4));
    block_prep(ix->Xs.as<float>(), n1, Dp, metric, A.as<__half>(), nb_i.as<uint8_t>(), nb_k.as<float>(), s);
    GRNG_CUDA(maxe.alloc((size_t)n1 * 4));
    edge_max_keys(ix->edges.as<uint64_t>(), ix->n_edges, ix->xrank.as<int32_t>(), ix->Xs.as<float>(), Dp, metric,
                  maxe.as<float>(), n1, s);
    GRNG_CUDA(knn_k.alloc((size_t)n1 * K * 4));
    GRNG_CUDA(knn_i.alloc((size_t)n1 * K * 4));
    InsertSweep S;
    S.XB = XB.as<float>(); S.rowpos = rowpos.as<int32_t>(); S.mb = m;
    S.AB = AB.as<__half>(); S.nbrB_i = nbB_i.as<uint8_t>(); S.nbrB_k = nbB_k.as<float>();
    S.X = ix->Xs.as<float>(); S.n = n1; S.Dp = Dp; S.K = K; S.metric = metric;
    S.A = A.as<__half>(); S.nbr_i = nb_i.as<uint8_t>(); S.nbr_k = nb_k.as<float>();
    S.is_new = is_new.as<uint8_t>(); S.parent = ix->xparent.as<int32_t>();
    S.gpar = fin.gg.as<uint32_t>(); S.gpar_words = fin.words; S.maxe = maxe.as<float>();
    int64_t nsurv = 0, ns7 = 0;
    unsigned long long sst[2] = {0, 0};
    insert_sweep(S, surv, &nsurv, s7, &ns7, knn_k.as<float>(), knn_i.as<int32_t>(), sst, s);
    ix->ins.candidates += sst[0];
    ix->ins.survivors += nsurv;
    ix->ins.s7_candidates += ns7;
    // ---- new edges: tiers 2 (the batch rows' exact lists) and 3, FP64 recheck --------------
    {
      LevelIn in{};
      in.X = ix->Xs.as<float>();
      in.n = n1;
      in.D = D;
      in.Dp = Dp;
      in.metric = metric;
      in.grng = 0;
      in.K = K;
      in.parent = ix->xparent.as<int32_t>();
      in.gpar = fin.gg.as<uint32_t>();
      in.gpar_words = fin.words;
      in.orig = ix->xorder.as<int32_t>();
      in.anc = ancestors_of(ix, L);
      in.pdist_hi = ix->xpdh.as<float>();
      if (ix->opts.spin_limit > 0) in.spin = ix->opts.spin_limit;
      in.small_buffers = (ix->opts.flags & GRNG_FLAG_SMALL_BUFFERS) ? 1 : 0;
      LevelOut lo;
      lo.edges = &newE;
      LevelStats st;
      run_pairs(in, lo, st, s, surv.as<int2>(), nsurv, knn_i.as<int32_t>(), knn_k.as<float>(), false);
      ix->ins.new_edges += lo.n_edges;
      // ---- Stage VII: old edges with a batch point strictly inside their lune ----------------
      DevBuf all;
      GRNG_CUDA(all.alloc((size_t)std::max<int64_t>(ix->n_edges + lo.n_edges, 1) * 8));
      unsigned long long s7st[2] = {0, 0};
      DevBuf s7c;
      GRNG_CUDA(s7c.alloc(16));
      GRNG_CUDA(cudaMemsetAsync(s7c.p, 0, 16, s));
      const int64_t kept = stage7_remove(ix->edges.as<uint64_t>(), ix->n_edges, n0, s7.as<int4>(), ns7,
                                         ix->Xs.as<float>(), D, Dp, metric, ix->xorder.as<int32_t>(),
                                         ix->xrank.as<int32_t>(), all.as<uint64_t>(),
                                         s7c.as<unsigned long long>(), s);
      GRNG_CUDA(cudaMemcpyAsync(s7st, s7c.p, 16, cudaMemcpyDeviceToHost, s));
      ix->ins.removed_edges += ix->n_edges - kept;
      if (lo.n_edges)
        GRNG_CUDA(cudaMemcpyAsync(all.as<uint64_t>() + kept, newE.p, (size_t)lo.n_edges * 8, cudaMemcpyDeviceToDevice,
                                  s));
      const int64_t ne = kept + lo.n_edges;
      DevBuf tmp;
      if (ne > 1) sort_u64(all.as<uint64_t>(), ne, tmp, s);
      GRNG_CUDA(cudaStreamSynchronize(s));
      ix->ins.s7_tests += s7st[0];
      ix->ins.s7_fp64 += s7st[1];
      ix->edges = std::move(all);
      ix->n_edges = ne;
    }
    ix->insert_ms += tm.stop();
    ix->insert_batches += 1;
    ix->inserted += m;
  });
}

// RNG search (Algorithm 1 without Stage VII, Sec. 2).  The queries are appended as rows
// n .. n+m-1 after the index's points in sorted order, with ids n + j; they are members of no
// pivot domain, so the exhaustive tier never takes one as an interceptor, and the sweep runs
// in its query mode, where only index points block.  Stage I: Theorem 1 restricts a query's
// candidates when the query lies in its nearest finest pivot's ball (the GRNG's guarantee
// covers exactly the points of the balls), else every index point is a candidate.
grng_status rng_search_batch(grng_index* ix, const float* queries, int64_t m, int64_t* total) {
  if (!ix) {
    g_last_error = "index is NULL";
    return GRNG_EINVAL;
  }
  return guarded(ix, [&] {
    if (!queries || m < 1) fail(GRNG_EINVAL, "need queries and m >= 1");
    if (ix->layers.empty()) fail(GRNG_ESTATE, "the index has no pivot layer");
    for (auto& l : ix->layers)
      if (!l.linked) fail(GRNG_ESTATE, "every layer must be built and linked");
    if (ix->n + m >= (int64_t)1 << 31) fail(GRNG_EINVAL, "n + m must stay below 2^31");
    ensure_sorted(ix);
    cudaStream_t s = ix->stream;
    Timer tm(s);
    auto& W = ix->srch;
    W.m = 0;
    W.total = 0;
    const int L = (int)ix->layers.size();
    const int Dp = ix->Dp, D = ix->D, K = ix->K, metric = ix->metric;
    const int64_t n = ix->n;
    Layer& fin = ix->layers[L - 1];
    if (W.version != ix->version) {  // in-block keys and neighbours of the index's 128-point blocks
      const int64_t nb = (n + 127) / 128;
      GRNG_CUDA(W.A.alloc((size_t)nb * 128 * 128 * 2));
      GRNG_CUDA(W.nb_i.alloc((size_t)nb * 128 * GRNG_KIN));
      GRNG_CUDA(W.nb_k.alloc((size_t)nb * 128 * GRNG_KIN * 4));
      block_prep(ix->Xs.as<float>(), n, Dp, metric, W.A.as<__half>(), W.nb_i.as<uint8_t>(), W.nb_k.as<float>(), s);
      W.cap = 0;
    }
    if (W.version != ix->version || W.cap < m) {  // index rows, then room for the queries
      const int64_t cap = (std::max(m, W.cap) + 127) / 128 * 128;
      const int64_t rows = n + cap;
      GRNG_CUDA(W.X.alloc((size_t)rows * Dp * 4));
      GRNG_CUDA(cudaMemcpyAsync(W.X.p, ix->Xs.p, (size_t)n * Dp * 4, cudaMemcpyDeviceToDevice, s));
      GRNG_CUDA(cudaMemsetAsync(W.X.as<float>() + n * Dp, 0, (size_t)cap * Dp * 4, s));
      GRNG_CUDA(W.orig.alloc((size_t)rows * 4));
      GRNG_CUDA(cudaMemcpyAsync(W.orig.p, ix->xorder.p, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
      iota_from_kernel<<<nblk(cap), 256, 0, s>>>(W.orig.as<int32_t>() + n, cap, n); note_launch();
      GRNG_CUDA(W.parent.alloc((size_t)rows * 4));
      GRNG_CUDA(cudaMemcpyAsync(W.parent.p, ix->xparent.p, (size_t)n * 4, cudaMemcpyDeviceToDevice, s));
      GRNG_CUDA(W.knn_k.alloc((size_t)rows * K * 4));
      GRNG_CUDA(W.knn_i.alloc((size_t)rows * K * 4));
      GRNG_CUDA(cudaGetLastError());
      W.cap = cap;
      W.version = ix->version;
    }
    // ---- the queries as rows n .. n+m-1 (zero padded to Dp) -------------------------------
    float* Xq = W.X.as<float>() + n * Dp;
    GRNG_CUDA(cudaMemsetAsync(Xq, 0, (size_t)m * Dp * 4, s));
    GRNG_CUDA(cudaMemcpy2DAsync(Xq, (size_t)Dp * 4, queries, (size_t)D * 4, (size_t)D * 4, (size_t)m,
                                cudaMemcpyDefault, s));
    // ---- nearest finest pivot (Eq. 2), and whether its ball holds the query ----------------
    DevBuf ab, db, rb, ddb, ctr, surv, E;
    Timer ta(s);
    {
      const int64_t M = fin.m;
      GRNG_CUDA(ab.alloc((size_t)m * 4));
      GRNG_CUDA(db.alloc((size_t)m * 8));
      GRNG_CUDA(rb.alloc((size_t)M * 8));
      GRNG_CUDA(ddb.alloc((size_t)M * 8));
      AssignOut ao{ab.as<int32_t>(), db.as<double>(), rb.as<double>(), ddb.as<double>()};
      assign_layer(Xq, W.orig.as<int32_t>() + n, nullptr, m, fin.Xp.as<float>(), fin.piv.as<int32_t>(), M, n + m, D,
                   Dp, metric, ao, nullptr, s, ix->opts.precision == GRNG_BF16,
                   ix->opts.spin_limit > 0 ? ix->opts.spin_limit : 1ll << 24);
      GRNG_CUDA(ctr.alloc(8));
      GRNG_CUDA(cudaMemsetAsync(ctr.p, 0, 8, s));
      search_parent_kernel<<<nblk(m), 256, 0, s>>>(ab.as<int32_t>(), db.as<double>(), fin.radius.as<double>(),
                                                   fin.rank.as<int32_t>(), m, W.parent.as<int32_t>() + n,
                                                   ctr.as<unsigned long long>()); note_launch();
      GRNG_CUDA(cudaGetLastError());
      unsigned long long outside = 0;
      GRNG_CUDA(cudaMemcpyAsync(&outside, ctr.p, 8, cudaMemcpyDeviceToHost, s));
      GRNG_CUDA(cudaStreamSynchronize(s));
      W.outside += (long long)outside;
    }
    W.assign_ms = ta.stop();
    Timer tsw(s);
    // ---- Stages I-V: the query rows against every index point (tier 1, K nearest) -------
    SearchSweep S;
    S.XQ = Xq; S.mq = m; S.row0 = n; S.rowpos = W.orig.as<int32_t>() + n;  // row j sits at n + j
    S.qparent = W.parent.as<int32_t>() + n;
    S.X = W.X.as<float>(); S.n = n; S.Dp = Dp; S.K = K; S.metric = metric;
    S.A = W.A.as<__half>(); S.nbr_i = W.nb_i.as<uint8_t>(); S.nbr_k = W.nb_k.as<float>();
    S.parent = W.parent.as<int32_t>(); S.gpar = fin.gg.as<uint32_t>(); S.gpar_words = fin.words;
    S.small_buffers = (ix->opts.flags & GRNG_FLAG_SMALL_BUFFERS) ? 1 : 0;
    int64_t nsurv = 0;
    unsigned long long sst[3] = {0, 0, 0};
    search_sweep(S, surv, &nsurv, W.knn_k.as<float>(), W.knn_i.as<int32_t>(), sst, s);
    W.candidates += (long long)sst[0];
    W.queued += (long long)sst[1];
    W.retries += (long long)sst[2];
    W.survivors += nsurv;
    W.sweep_ms = tsw.stop();
    Timer tt(s);
    // ---- Stage VI: tiers 2 (the queries' K nearest) and 3, FP64 recheck -------------------
    LevelIn in{};
    in.X = W.X.as<float>();
    in.n = n + m;
    in.D = D;
    in.Dp = Dp;
    in.metric = metric;
    in.grng = 0;
    in.K = K;
    in.parent = W.parent.as<int32_t>();
    in.gpar = fin.gg.as<uint32_t>();
    in.gpar_words = fin.words;
    in.orig = W.orig.as<int32_t>();
    in.anc = ancestors_of(ix, L);
    in.pdist_hi = ix->xpdh.as<float>();  // read for index points only (the interceptors)
    in.npts = n;
    if (ix->opts.spin_limit > 0) in.spin = ix->opts.spin_limit;
    in.small_buffers = (ix->opts.flags & GRNG_FLAG_SMALL_BUFFERS) ? 1 : 0;
    LevelOut lo;
    lo.edges = &E;
    LevelStats st;
    run_pairs(in, lo, st, s, surv.as<int2>(), nsurv, W.knn_i.as<int32_t>(), W.knn_k.as<float>(), false);
    W.tiers_ms = tt.stop();
    W.st = st;
    // ---- CSR over the queries ----------------------------------------------------------------
    const int64_t ne = lo.n_edges;
    GRNG_CUDA(W.off.alloc((size_t)(m + 1) * 8));
    GRNG_CUDA(W.nbrs.alloc((size_t)std::max<int64_t>(ne, 1) * 4));
    if (ne) {
      search_key_kernel<<<nblk(ne), 256, 0, s>>>(E.as<uint64_t>(), ne, n); note_launch();
      DevBuf tmp;
      if (ne > 1) sort_u64(E.as<uint64_t>(), ne, tmp, s);
    }
    search_csr_kernel<<<nblk(ne + 1), 256, 0, s>>>(E.p ? E.as<uint64_t>() : nullptr, ne, m, W.off.as<int64_t>(),
                                                   W.nbrs.as<int32_t>()); note_launch();
    GRNG_CUDA(cudaGetLastError());
    GRNG_CUDA(cudaStreamSynchronize(s));
    W.m = m;
    W.total = ne;
    W.neighbours += ne;
    W.batches += 1;
    W.queries += m;
    W.last_ms = tm.stop();
    W.ms += W.last_ms;
    if (total) *total = ne;
  });
}

grng_status rng_search_result(const grng_index* cix, int64_t* off, int32_t* nbrs, int64_t cap) {
  grng_index* ix = const_cast<grng_index*>(cix);
  if (!ix) {
    g_last_error = "index is NULL";
    return GRNG_EINVAL;
  }
  return guarded(ix, [&] {
    auto& W = ix->srch;
    if (W.m == 0) fail(GRNG_ESTATE, "no search result");
    cudaStream_t s = ix->stream;
    copy_out(off, W.off.p, (size_t)(W.m + 1) * 8, s);
    GRNG_CUDA(cudaStreamSynchronize(s));
    if (!nbrs) return;
    if (cap < W.total) fail(GRNG_ETRUNC, "neighbour buffer too small");
    copy_out(nbrs, W.nbrs.p, (size_t)W.total * 4, s);
    GRNG_CUDA(cudaStreamSynchronize(s));
  });
}

grng_status rng_edges(const grng_index* cix, int32_t* ij, int64_t cap, int64_t* n_edges) {
  grng_index* ix = const_cast<grng_index*>(cix);
  if (!ix) {
    g_last_error = "index is NULL";
    return GRNG_EINVAL;
  }
  return guarded(ix, [&] {
    if (!ix->rng_built) fail(GRNG_ESTATE, "the RNG is not built");
    if (n_edges) *n_edges = ix->n_edges;
    if (!ij) return;
    if (cap < ix->n_edges) fail(GRNG_ETRUNC, "edge buffer too small");
    cudaStream_t s = ix->stream;
    DevBuf pairs;
    GRNG_CUDA(pairs.alloc((size_t)std::max<int64_t>(ix->n_edges, 1) * 8));
    if (ix->n_edges) {
      edges_to_pairs_kernel<<<nblk(ix->n_edges), 256, 0, s>>>(ix->edges.as<uint64_t>(), ix->n_edges,
                                                               pairs.as<int32_t>()); note_launch();
      GRNG_CUDA(cudaGetLastError());
    }
    copy_out(ij, pairs.p, (size_t)ix->n_edges * 8, s);
    GRNG_CUDA(cudaStreamSynchronize(s));
  });
}

grng_status grng_stats(const grng_index* cix, char* json, size_t cap) {
  const grng_index* ix = cix;
  if (!ix || !json) {
    g_last_error = "index and json must not be NULL";
    return GRNG_EINVAL;
  }
  std::string js = "{";
  char buf[2048];
  snprintf(buf, sizeof(buf),
           "\"n\":%lld,\"dim\":%d,\"metric\":%d,\"knn_k\":%d,\"sort_ms\":%.4f,\"kernel_launches\":%llu,\"layers\":[",
           (long long)ix->n, ix->D, ix->metric, ix->K, ix->sort_ms, launches());
  js += buf;
  for (size_t l = 0; l < ix->layers.size(); ++l) {
    const Layer& ly = ix->layers[l];
    snprintf(buf, sizeof(buf),
             "%s{\"m\":%lld,\"built\":%d,\"linked\":%d,\"assign_ms\":%.4f,\"link_ms\":%.4f,\"link_tile_ms\":%.4f,"
             "\"assign_ambiguous\":%llu,\"assign_fp64_keys\":%llu,\"assign_kernel_ms\":%.4f,\"assign_tensor_cores\":%llu,\"assign_full_rechecks\":%llu,",
             l ? "," : "", (long long)ly.m, (int)ly.built, (int)ly.linked, ly.assign_ms, ly.link_ms,
             ly.link_tile_ms, ly.assign_amb, ly.assign_fp64, ly.assign_kernel_ms, ly.assign_tc, ly.assign_full);
    js += buf;
    level_json(js, "grng", ly.st);
    js += "}";
  }
  snprintf(buf, sizeof(buf),
           "],\"rng_built\":%d,\"skeleton_beta\":%.17g,\"n_edges\":%lld,\"rng_ms\":%.4f,\"rng_tile_ms\":%.4f,"
           "\"insert\":{\"batches\":%lld,\"points\":%lld,\"ms\":%.4f,\"changed_pivots\":%lld,"
           "\"grng_pairs\":%lld,\"grng_links_added\":%lld,\"candidate_pairs\":%lld,\"tier1_survivors\":%lld,"
           "\"stage7_candidates\":%lld,\"stage7_tests\":%lld,\"stage7_fp64\":%lld,\"new_edges\":%lld,"
           "\"removed_edges\":%lld},"
           "\"search\":{\"batches\":%lld,\"queries\":%lld,\"ms\":%.4f,\"last_ms\":%.4f,\"outside_ball\":%lld,"
           "\"candidate_pairs\":%lld,\"tier1_survivors\":%lld,\"neighbours\":%lld,"
           "\"tier1_queued\":%lld,\"sweep_retries\":%lld,"
           "\"last_assign_ms\":%.4f,\"last_sweep_ms\":%.4f,\"last_tiers_ms\":%.4f,",
           (int)ix->rng_built, ix->skel_beta, (long long)ix->n_edges, ix->rng_ms, ix->rng_tile_ms, (long long)ix->insert_batches,
           (long long)ix->inserted, ix->insert_ms, ix->ins.changed_pivots, ix->ins.grng_pairs, ix->ins.grng_linked,
           ix->ins.candidates, ix->ins.survivors, ix->ins.s7_candidates, ix->ins.s7_tests, ix->ins.s7_fp64,
           ix->ins.new_edges, ix->ins.removed_edges, ix->srch.batches, ix->srch.queries, ix->srch.ms,
           ix->srch.last_ms, ix->srch.outside, ix->srch.candidates, ix->srch.survivors, ix->srch.neighbours,
           ix->srch.queued, ix->srch.retries, ix->srch.assign_ms, ix->srch.sweep_ms, ix->srch.tiers_ms);
  js += buf;
  level_json(js, "last_tiers", ix->srch.st);
  js += "},";
  level_json(js, "rng", ix->rng_st);
  js += "}";
  if (js.size() + 1 > cap) {
    g_last_error = "stats buffer too small";
    return GRNG_ETRUNC;
  }
  memcpy(json, js.c_str(), js.size() + 1);
  return GRNG_OK;
}

}  // extern "C"
