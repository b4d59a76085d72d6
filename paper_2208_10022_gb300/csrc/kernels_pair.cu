// kernels_pair.cu -- the pair pipeline shared by the pivot-layer GRNG test and the
// exemplar lune-emptiness test.
//
// A "level" is a node set: the pivots of one layer (GRNG definition, Sec. 2, with
// their radii) or the exemplars (Eq. 1, radii zero).  Candidate pairs are the pairs
// whose parents are equal or linked in the parent layer's guidance graph (Stage I,
// Theorem 1 for exemplars; Theorem 2 for pivot layers).  Each candidate pair goes
// through tiers that differ only in which interceptors they try (the result never
// depends on the order, only the work does):
//   tier 1  all-pairs distance tiles; inside a tile the interceptors are the row
//           minimum of x over the column block, the column minimum of y over the row
//           block and the in-block nearest neighbours of x and y (the "select group"
//           of Stage V); the same sweep keeps each node's K nearest neighbours.
//   tier 2  the K nearest neighbours of one endpoint.  When the neighbour list
//           reaches past the first G-lune threshold of that endpoint, every node
//           that could satisfy that condition is in the list, so the test is exact
//           (the exhaustive check of Stage VI restricted by a ball bound).
//   lists   (pivot layers) per-node range lists of up to 16,384 nodes, cut by a key
//           histogram and kept in key bands; a pair whose threshold one endpoint's list
//           reaches is decided from that list alone, after warp-per-pair descents towards
//           the ball around its G-lune have dropped the pairs a node certainly blocks.
//   tier 3  the exhaustive Stage VI search down the pivot tree, pruned by domain
//           bounds (Prop. 4 / GRNG_S6, Prop. 5) and by the ball around the G-lune,
//           after greedy descents towards that ball's centre; at the exemplar level
//           the learned shortlist (kernels_mlp.cu) may decide a pair first.
// Comparisons whose FP32 brackets overlap are re-decided in canonical FP64.
// The exemplar level also builds lune-based beta-skeletons (1 <= beta <= 2): only the test of
// one interceptor changes (block_state, block64 with lam = beta / 2); every bound above is a
// bound on the lune of Eq. 1, which holds each beta-lune, so it stays valid as it is, and no
// guidance filters the pairs.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <functional>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tile.cuh"

namespace grng {

#define FULLMASK 0xffffffffu
static __device__ __forceinline__ float finf() { return __int_as_float(0x7f800000); }

// Lower bound E of d(x,y) - t_other, the other condition's threshold t_other given as
// an upper bound in key units: a node k with d(k,x) <= E has, by the triangle
// inequality, d(k,y) >= d(x,y) - d(k,x) >= t_other, so it cannot satisfy the other
// condition (GRNG definition, Sec. 2).
static __device__ __forceinline__ float excl_dist(float v, float t_other_key_hi, int metric, Err e) {
  const float u2 = 1.1920928955078125e-07f;
  const float vlo = fmaxf(lo_b(v, e), 0.0f);
  const float dlo = metric == L2 ? sqrtf(vlo) * (1.0f - u2) : vlo;
  const float t = metric == L2 ? sqrtf(fmaxf(t_other_key_hi, 0.0f)) * (1.0f + u2) : t_other_key_hi;
  return dlo - t - u2 * (dlo + t);
}

// 1 when no node can block through this side: the side's sorted neighbour keys kl[K]
// reach past the condition's threshold (so every node that could satisfy it is in the
// list) and every listed node that could satisfy it lies within E, where the other
// condition is impossible.  thr_hi: the condition's threshold, upper bound, key units.
// keys with hi_b(key) <= excl_key(E) belong to distances within E
static __device__ __forceinline__ float excl_key(float E, int metric) {
  const float u2 = 1.1920928955078125e-07f;
  if (!(E > 0.0f)) return -1.0f;
  if (metric == L2) {
    const float q = E * (1.0f - u2);
    return q * q * (1.0f - u2);
  }
  return E * (1.0f - u2);
}

static __device__ __forceinline__ bool side_certified(const float* kl, int K, float thr_hi, float E, int metric,
                                                      Err e) {
  if (lo_b(kl[K - 1], e) < thr_hi) return false;
  const float ekey = excl_key(E, metric);
  for (int j = 0; j < K; ++j) {
    const float kj = kl[j];
    if (lo_b(kj, e) >= thr_hi) break;  // ascending: no later entry satisfies the condition
    if (hi_b(kj, e) > ekey) return false;
  }
  return true;
}

// ---------------------------------------------------------------------------------
// Block preparation: intra-block keys (FP16 rounded up: a safe upper bound for the
// "certainly blocks" test) and the GRNG_KIN nearest in-block neighbours of each node.
// ---------------------------------------------------------------------------------
template <int KC, int METRIC>
__global__ void __launch_bounds__(GRNG_THREADS) block_prep_kernel(const float* __restrict__ X,
                                                                  int64_t n, int Dp,
                                                                  __half* __restrict__ A,
                                                                  uint8_t* __restrict__ nbr_idx,
                                                                  float* __restrict__ nbr_key) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* sA = reinterpret_cast<float*>(sm_raw);
  float* sB = sA + KC * GRNG_SSTRIDE;
  float* T = sB + KC * GRNG_SSTRIDE;  // [128][129]
  const int64_t b = blockIdx.x;
  const int64_t base = b * GRNG_TILE;
  const int nr = (int)(n - base < GRNG_TILE ? n - base : GRNG_TILE);
  float acc[8][8];
  tile_keys<KC, METRIC>(X + base * Dp, nr, X + base * Dp, nr, Dp, sA, sB, acc);
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      int r = tile_row(i), c = tile_col(j);
      float v = acc[i][j];
      if (r >= nr || c >= nr) v = finf();
      if (r == c) v = 0.0f;
      T[r * 129 + c] = v;
    }
  __syncthreads();
  for (int i = threadIdx.x; i < GRNG_TILE * GRNG_TILE; i += GRNG_THREADS) {
    int r = i >> 7, c = i & 127;
    A[b * GRNG_TILE * GRNG_TILE + i] = __float2half_ru(T[r * 129 + c]);
  }
  if (threadIdx.x < nr) {
    int r = threadIdx.x;
    float bk[GRNG_KIN];
    int bi[GRNG_KIN];
#pragma unroll
    for (int t = 0; t < GRNG_KIN; ++t) { bk[t] = finf(); bi[t] = 255; }
    for (int c = 0; c < nr; ++c) {
      if (c == r) continue;
      float v = T[r * 129 + c];
      if (v < bk[GRNG_KIN - 1]) {
        int pos = GRNG_KIN - 1;
        while (pos > 0 && bk[pos - 1] > v) { bk[pos] = bk[pos - 1]; bi[pos] = bi[pos - 1]; --pos; }
        bk[pos] = v;
        bi[pos] = c;
      }
    }
#pragma unroll
    for (int t = 0; t < GRNG_KIN; ++t) {
      nbr_idx[(base + r) * GRNG_KIN + t] = (uint8_t)bi[t];
      nbr_key[(base + r) * GRNG_KIN + t] = bk[t];
    }
  }
}

// ---------------------------------------------------------------------------------
// Tier 1: persistent all-pairs tile sweep.
// ---------------------------------------------------------------------------------
struct TileParams {
  const float* X;
  int64_t n;
  int Dp, grng, guide, K;
  const int32_t* parent;
  const uint32_t* gpar;
  int64_t gpar_words;
  const float* rlo;
  const float* rhi;
  const __half* A;
  const uint8_t* nbr_idx;
  const float* nbr_key;
  int32_t* knn_idx;
  float* knn_key;
  int2* surv;
  unsigned long long* surv_cnt;
  unsigned long long surv_cap;
  uint32_t* gx;
  uint32_t* gg;
  int64_t words;
  int* strip_ctr;
  unsigned long long* stats;  // [0] candidate pairs [1] linked in the tile [2] of which certified by a list
  int mode;  // 0: lists + filter in one sweep; 1: lists only; 2: filter with the lists of sweep 1
  float lam;  // beta / 2 of the lune test (1: Eq. 1)
};

// shared-memory layout of the tile sweep (bytes)
#define TP_U 66048                    // max(2*32*132*4, 128*129*4)
#define TP_AX (TP_U)
#define TP_AY (TP_AX + 32768)
#define TP_KNN (TP_AY + 32768)
static __host__ __device__ constexpr int tp_knn_bytes(int K) { return 128 * (K + 1) * 8; }
static __host__ __device__ constexpr int tp_bytes(int K) {
  return TP_KNN + tp_knn_bytes(K) + 128 * GRNG_KIN * 10 + 8 * 512 + 6 * 512 + 64;
}

template <int KC, int METRIC>
__global__ void __launch_bounds__(GRNG_THREADS, 1) tile_pass_kernel(TileParams p) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* sA = reinterpret_cast<float*>(sm_raw);
  float* sB = sA + KC * GRNG_SSTRIDE;
  float* T = reinterpret_cast<float*>(sm_raw);  // aliases sA/sB after the product
  __half* AX = reinterpret_cast<__half*>(sm_raw + TP_AX);
  __half* AY = reinterpret_cast<__half*>(sm_raw + TP_AY);
  const int K = p.K;
  float* knnK = reinterpret_cast<float*>(sm_raw + TP_KNN);
  int* knnI = reinterpret_cast<int*>(knnK + 128 * (K + 1));
  unsigned char* q = sm_raw + TP_KNN + tp_knn_bytes(K);
  float* nbrXk = reinterpret_cast<float*>(q); q += 128 * GRNG_KIN * 4;
  float* nbrYk = reinterpret_cast<float*>(q); q += 128 * GRNG_KIN * 4;
  uint8_t* nbrXi = q; q += 128 * GRNG_KIN;
  uint8_t* nbrYi = q; q += 128 * GRNG_KIN;
  float* rmin1 = reinterpret_cast<float*>(q); q += 512;
  float* rmin2 = reinterpret_cast<float*>(q); q += 512;
  int* rarg1 = reinterpret_cast<int*>(q); q += 512;
  int* rarg2 = reinterpret_cast<int*>(q); q += 512;
  float* cmin1 = reinterpret_cast<float*>(q); q += 512;
  float* cmin2 = reinterpret_cast<float*>(q); q += 512;
  int* carg1 = reinterpret_cast<int*>(q); q += 512;
  int* carg2 = reinterpret_cast<int*>(q); q += 512;
  int* parX = reinterpret_cast<int*>(q); q += 512;
  int* parY = reinterpret_cast<int*>(q); q += 512;
  float* rxlo = reinterpret_cast<float*>(q); q += 512;
  float* rxhi = reinterpret_cast<float*>(q); q += 512;
  float* rylo = reinterpret_cast<float*>(q); q += 512;
  float* ryhi = reinterpret_cast<float*>(q); q += 512;
  int* s_strip = reinterpret_cast<int*>(q);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int64_t n = p.n;
  const int Dp = p.Dp;
  const int64_t nb = (n + GRNG_TILE - 1) / GRNG_TILE;
  const Err e = err_fp32(Dp);
  unsigned long long st_cand = 0, st_quick = 0, st_cert = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) *s_strip = atomicAdd(p.strip_ctr, 1);
    __syncthreads();
    const int64_t bx = *s_strip;
    if (bx >= nb) break;
    const int64_t xb = bx * GRNG_TILE;
    const int nr = (int)(n - xb < GRNG_TILE ? n - xb : GRNG_TILE);
    {
      const uint4* src = reinterpret_cast<const uint4*>(p.A + bx * GRNG_TILE * GRNG_TILE);
      uint4* dst = reinterpret_cast<uint4*>(AX);
      for (int i = tid; i < GRNG_TILE * GRNG_TILE / 8; i += GRNG_THREADS) dst[i] = src[i];
      for (int i = tid; i < GRNG_TILE * GRNG_KIN; i += GRNG_THREADS) {
        int r = i / GRNG_KIN;
        bool ok = r < nr;
        nbrXi[i] = ok ? p.nbr_idx[xb * GRNG_KIN + i] : (uint8_t)255;
        nbrXk[i] = ok ? p.nbr_key[xb * GRNG_KIN + i] : finf();
      }
      if (tid < GRNG_TILE) {
        bool ok = tid < nr;
        parX[tid] = (p.parent && ok) ? p.parent[xb + tid] : 0;
        rxlo[tid] = (p.rlo && ok) ? p.rlo[xb + tid] : 0.0f;
        rxhi[tid] = (p.rhi && ok) ? p.rhi[xb + tid] : 0.0f;
      }
      for (int i = tid; i < GRNG_TILE * (K + 1); i += GRNG_THREADS) {
        if (p.mode == 2) {  // the final lists of the row nodes, from the first sweep
          int r = i / (K + 1), j = i % (K + 1);
          knnK[i] = (r < nr && j < K) ? p.knn_key[(xb + r) * K + j] : finf();
        } else {
          knnK[i] = finf();
          knnI[i] = -1;
        }
      }
    }
    int done = 0;
    for (int s = 0; done < nb; ++s) {
      const int64_t off = (s & 1) ? (int64_t)((s + 1) >> 1) : -(int64_t)(s >> 1);
      const int64_t by = bx + off;
      if (by < 0 || by >= nb) continue;
      ++done;
      const int64_t yb = by * GRNG_TILE;
      const int nc = (int)(n - yb < GRNG_TILE ? n - yb : GRNG_TILE);
      const bool filt = p.mode != 1 && by >= bx;
      float acc[8][8];
      tile_keys<KC, METRIC>(p.X + xb * Dp, nr, p.X + yb * Dp, nc, Dp, sA, sB, acc);
      __syncthreads();  // every thread is done with sA/sB: T may overwrite them
#pragma unroll
      for (int i = 0; i < 8; ++i)
#pragma unroll
        for (int j = 0; j < 8; ++j) {
          int r = tile_row(i), c = tile_col(j);
          float v = acc[i][j];
          if (r >= nr || c >= nc || (by == bx && r == c)) v = finf();
          T[r * 129 + c] = v;
        }
      if (filt) {
        const uint4* src = reinterpret_cast<const uint4*>(p.A + by * GRNG_TILE * GRNG_TILE);
        uint4* dst = reinterpret_cast<uint4*>(AY);
        for (int i = tid; i < GRNG_TILE * GRNG_TILE / 8; i += GRNG_THREADS) dst[i] = src[i];
        for (int i = tid; i < GRNG_TILE * GRNG_KIN; i += GRNG_THREADS) {
          int r = i / GRNG_KIN;
          bool ok = r < nc;
          nbrYi[i] = ok ? p.nbr_idx[yb * GRNG_KIN + i] : (uint8_t)255;
          nbrYk[i] = ok ? p.nbr_key[yb * GRNG_KIN + i] : finf();
        }
        if (tid < GRNG_TILE) {
          bool ok = tid < nc;
          parY[tid] = (p.parent && ok) ? p.parent[yb + tid] : 0;
          rylo[tid] = (p.rlo && ok) ? p.rlo[yb + tid] : 0.0f;
          ryhi[tid] = (p.rhi && ok) ? p.rhi[yb + tid] : 0.0f;
        }
        if (p.mode == 2) {  // the column nodes' lists (in the space of the row lists' indices)
          float* knnKY = reinterpret_cast<float*>(knnI);
          for (int i = tid; i < GRNG_TILE * (K + 1); i += GRNG_THREADS) {
            int c = i / (K + 1), j = i % (K + 1);
            knnKY[i] = (c < nc && j < K) ? p.knn_key[(yb + c) * K + j] : finf();
          }
        }
      }
      __syncthreads();
      // ---- neighbour lists (rows) and row / column minima --------------------------
      if (tid < GRNG_TILE) {
        const int r = tid;
        if (r < nr) {
          float* kk = knnK + r * (K + 1);
          int* ki = knnI + r * (K + 1);
          float thr = kk[K - 1];
          float m1 = finf(), m2 = finf();
          int a1 = -1, a2 = -1;
          const float* Tr = T + r * 129;
          for (int c = 0; c < GRNG_TILE; ++c) {
            float v = Tr[c];
            if (v < m2) {
              if (v < m1) { m2 = m1; a2 = a1; m1 = v; a1 = c; }
              else { m2 = v; a2 = c; }
            }
            if (p.mode != 2 && v < thr) {
              int pos = K - 1;
              while (pos > 0 && kk[pos - 1] > v) { kk[pos] = kk[pos - 1]; ki[pos] = ki[pos - 1]; --pos; }
              kk[pos] = v;
              ki[pos] = (int)(yb + c);
              thr = kk[K - 1];
            }
          }
          rmin1[r] = m1; rmin2[r] = m2; rarg1[r] = a1; rarg2[r] = a2;
        }
      } else if (filt) {
        const int c = tid - GRNG_TILE;
        float m1 = finf(), m2 = finf();
        int a1 = -1, a2 = -1;
        for (int r = 0; r < GRNG_TILE; ++r) {
          float v = T[r * 129 + c];
          if (v < m2) {
            if (v < m1) { m2 = m1; a2 = a1; m1 = v; a1 = r; }
            else { m2 = v; a2 = r; }
          }
        }
        cmin1[c] = m1; cmin2[c] = m2; carg1[c] = a1; carg2[c] = a2;
      }
      __syncthreads();
      // ---- tier-1 lune filter on the candidate pairs x < y ----------------------------
      if (filt) {
        const bool diag = by == bx;
        for (int rr = 0; rr < 16; ++rr) {
          const int r = warp * 16 + rr;
          if (r >= nr) break;
          const int64_t x = xb + r;
          const int px = parX[r];
          const float rxl = rxlo[r], rxh = rxhi[r];
          for (int cb = 0; cb < 4; ++cb) {
            if (cb * 32 >= nc) break;
            const int c = cb * 32 + lane;
            const int64_t y = yb + c;
            bool cand = c < nc && (!diag || c > r);
            if (cand && p.gpar) {
              int qy = parY[c];
              if (qy != px) {
                int a = min(px, qy), b = max(px, qy);
                cand = (__ldg(p.gpar + (int64_t)a * p.gpar_words + (b >> 5)) >> (b & 31)) & 1u;
              }
            }
            bool quick = false, surv = false;
            if (cand) {
              const float v = T[r * 129 + c];
              PairThr P = pair_thresholds(v, rxl, rxh, rylo[c], ryhi[c], METRIC, e, p.guide, p.lam);
              if (P.quick) {
                quick = true;
              } else if (p.mode == 2 &&
                         (side_certified(knnK + r * (K + 1), K, P.t1hi, excl_dist(v, P.t2hi, METRIC, e), METRIC, e) ||
                          side_certified(reinterpret_cast<const float*>(knnI) + c * (K + 1), K, P.t2hi,
                                         excl_dist(v, P.t1hi, METRIC, e), METRIC, e))) {
                quick = true;
                ++st_cert;
              } else {
                bool blocked = false;
                {  // row minimum of x over the column block
                  int z = (rarg1[r] != c) ? rarg1[r] : rarg2[r];
                  if (z >= 0) {
                    float a = T[r * 129 + z];
                    float bb = __half2float(AY[z * 128 + c]);
                    blocked = block_state(a, bb, P, e) == 2;
                  }
                }
                if (!blocked) {  // column minimum of y over the row block
                  int z = (carg1[c] != r) ? carg1[c] : carg2[c];
                  if (z >= 0) {
                    float a = __half2float(AX[r * 128 + z]);
                    float bb = T[z * 129 + c];
                    blocked = block_state(a, bb, P, e) == 2;
                  }
                }
                for (int t = 0; t < GRNG_KIN && !blocked; ++t) {  // neighbours of x
                  int z = nbrXi[r * GRNG_KIN + t];
                  if (z == 255) break;
                  if (diag && z == c) continue;
                  blocked = block_state(nbrXk[r * GRNG_KIN + t], T[z * 129 + c], P, e) == 2;
                }
                for (int t = 0; t < GRNG_KIN && !blocked; ++t) {  // neighbours of y
                  int z = nbrYi[c * GRNG_KIN + t];
                  if (z == 255) break;
                  if (diag && z == r) continue;
                  blocked = block_state(T[r * 129 + z], nbrYk[c * GRNG_KIN + t], P, e) == 2;
                }
                surv = !blocked;
              }
            }
            st_cand += cand ? 1 : 0;
            unsigned qm = __ballot_sync(FULLMASK, quick);
            if (qm && lane == 0) {
              int64_t w = x * p.words + ((yb + cb * 32) >> 5);
              atomicOr(p.gx + w, qm);
              atomicOr(p.gg + w, qm);
            }
            st_quick += quick ? 1 : 0;
            unsigned sm = __ballot_sync(FULLMASK, surv);
            if (sm) {
              unsigned long long base = 0;
              if (lane == 0) base = atomicAdd(p.surv_cnt, (unsigned long long)__popc(sm));
              base = __shfl_sync(FULLMASK, base, 0);
              if (surv) {
                unsigned long long pos = base + __popc(sm & ((1u << lane) - 1u));
                if (pos < p.surv_cap) p.surv[pos] = make_int2((int)x, (int)y);
              }
            }
          }
        }
      }
      __syncthreads();
    }
    if (p.mode != 2 && tid < nr) {
      const float* kk = knnK + tid * (K + 1);
      const int* ki = knnI + tid * (K + 1);
      for (int j = 0; j < K; ++j) {
        p.knn_idx[(xb + tid) * K + j] = ki[j];
        p.knn_key[(xb + tid) * K + j] = kk[j];
      }
    }
  }
  // per-thread counts folded per warp
  for (int o = 16; o > 0; o >>= 1) {
    st_cand += __shfl_down_sync(FULLMASK, st_cand, o);
    st_quick += __shfl_down_sync(FULLMASK, st_quick, o);
    st_cert += __shfl_down_sync(FULLMASK, st_cert, o);
  }
  if (lane == 0) {
    atomicAdd(p.stats + 0, st_cand);
    atomicAdd(p.stats + 1, st_quick);
    atomicAdd(p.stats + 2, st_cert);
  }
}

// ---------------------------------------------------------------------------------
// Tier 2: the K nearest neighbours of the group node g as interceptors of (g, o).
// ---------------------------------------------------------------------------------
struct Tier2Params {
  const float* X;
  int64_t n;
  int Dp, metric, guide, K;
  const float* rlo;
  const float* rhi;
  const int32_t* knn_idx;
  const float* knn_key;
  const float* knn_rb;   // [n] lower bound of unlisted keys, or null (the K-th listed key)
  const int64_t* off;    // [n+1] grouped by g
  const int32_t* other;  // partner o of each entry
  int2* links; unsigned long long* link_cnt; unsigned long long link_cap;
  int2* unres; unsigned long long* unres_cnt; unsigned long long unres_cap;
  int2* pend; unsigned long long* pend_cnt; unsigned long long pend_cap;
  int2* amb; unsigned long long* amb_cnt; unsigned long long amb_cap;
  unsigned long long* stats;  // [0] links [1] pendings [2] unresolved [3] blocked
  float lam;                  // beta / 2 of the lune test (1: Eq. 1)
};

__device__ __forceinline__ void push_pair(int2* buf, unsigned long long* cnt,
                                          unsigned long long cap, int2 v) {
  unsigned long long pos = atomicAdd(cnt, 1ull);
  if (pos < cap) buf[pos] = v;
}

__global__ void __launch_bounds__(128) tier2_kernel(Tier2Params p) {
  extern __shared__ __align__(16) float sm2[];
  const int Dp = p.Dp, K = p.K;
  float* KT = sm2;               // [Dp][32]: coordinates of the neighbours, transposed
  float* gs = KT + Dp * 32;      // [Dp] coordinates of g
  float* os = gs + Dp;           // [4][Dp] coordinates of o, one buffer per warp
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const Err e = err_fp32(Dp);
  unsigned long long c_link = 0, c_pend = 0, c_unres = 0, c_blk = 0;
  for (int64_t g = blockIdx.x; g < p.n; g += gridDim.x) {
    const int64_t s = p.off[g], t_end = p.off[g + 1];
    if (s == t_end) continue;
    __syncthreads();
    for (int i = tid; i < Dp * 32; i += 128) {
      int d = i >> 5, j = i & 31;
      int kid = j < K ? p.knn_idx[g * K + j] : -1;
      KT[i] = kid >= 0 ? p.X[(int64_t)kid * Dp + d] : 0.0f;
    }
    for (int d = tid; d < Dp; d += 128) gs[d] = p.X[g * Dp + d];
    __syncthreads();
    const int kidl = lane < K ? p.knn_idx[g * K + lane] : -1;
    const float akey = lane < K ? p.knn_key[g * K + lane] : finf();
    const int lastid = p.knn_idx[g * K + K - 1];
    // every unlisted node has a key of at least lo_b(Rk): the K-th listed key, or the bound
    // the tensor-core sweep leaves when the list was chosen from approximate keys
    const float Rk = p.knn_rb ? p.knn_rb[g] : (lastid >= 0 ? p.knn_key[g * K + K - 1] : finf());
    const float rgl = p.rlo ? p.rlo[g] : 0.0f, rgh = p.rhi ? p.rhi[g] : 0.0f;
    float* ow = os + warp * Dp;
    for (int64_t t = s + warp; t < t_end; t += 4) {
      const int o = p.other[t];
      __syncwarp();
      for (int d = lane; d < Dp; d += 32) ow[d] = p.X[(int64_t)o * Dp + d];
      __syncwarp();
      float part = 0.0f;
      for (int d = lane; d < Dp; d += 32) {
        float tt = gs[d] - ow[d];
        part = p.metric == L2 ? fmaf(tt, tt, part) : part + fabsf(tt);
      }
      for (int sh = 16; sh > 0; sh >>= 1) part += __shfl_xor_sync(FULLMASK, part, sh);
      const float v = part;
      const float rol = p.rlo ? p.rlo[o] : 0.0f, roh = p.rhi ? p.rhi[o] : 0.0f;
      PairThr P = pair_thresholds(v, rgl, rgh, rol, roh, p.metric, e, p.guide, p.lam);
      if (P.quick) {
        if (lane == 0) push_pair(p.links, p.link_cnt, p.link_cap, make_int2((int)g, o));
        c_link += lane == 0;
        continue;
      }
      int stt = 0;
      // a listed node is tested only if it may satisfy the first condition and is not
      // excluded from the second by the triangle inequality
      const float ekey = excl_key(excl_dist(v, P.t2hi, p.metric, e), p.metric);
      if (kidl >= 0 && kidl != o && lo_b(akey, e) < P.t1hi && hi_b(akey, e) > ekey) {
        float b = 0.0f;
        if (p.metric == L2) {
          for (int d = 0; d < Dp; ++d) { float tt = KT[d * 32 + lane] - ow[d]; b = fmaf(tt, tt, b); }
        } else {
          for (int d = 0; d < Dp; ++d) b += fabsf(KT[d * 32 + lane] - ow[d]);
        }
        stt = block_state(akey, b, P, e);
      }
      const unsigned blk = __ballot_sync(FULLMASK, stt == 2);
      const unsigned amb = __ballot_sync(FULLMASK, stt == 1);
      const bool near_ = lo_b(Rk, e) >= P.t1hi;
      if (blk) {
        c_blk += lane == 0;
      } else if (near_) {
        if (!amb) {
          if (lane == 0) push_pair(p.links, p.link_cnt, p.link_cap, make_int2((int)g, o));
          c_link += lane == 0;
        } else {
          unsigned long long slot = 0;
          if (lane == 0) slot = atomicAdd(p.pend_cnt, 1ull);
          slot = __shfl_sync(FULLMASK, slot, 0);
          if (lane == 0 && slot < p.pend_cap) p.pend[slot] = make_int2((int)g, o);
          if ((amb >> lane) & 1u)
            push_pair(p.amb, p.amb_cnt, p.amb_cap, make_int2((int)slot, kidl));
          c_pend += lane == 0;
        }
      } else {
        if (lane == 0) push_pair(p.unres, p.unres_cnt, p.unres_cap, make_int2((int)g, o));
        c_unres += lane == 0;
      }
    }
  }
  if (lane == 0) {
    atomicAdd(p.stats + 0, c_link);
    atomicAdd(p.stats + 1, c_pend);
    atomicAdd(p.stats + 2, c_unres);
    atomicAdd(p.stats + 3, c_blk);
  }
}

// ---------------------------------------------------------------------------------
// Tier 3: exhaustive scan over all nodes (Stage VI) for the pairs tier 2 left open.
// Each pair owns the pending slot slot0 + its index.
// ---------------------------------------------------------------------------------
// a range of nodes below one domain c, with lower bounds of d(c, g), d(c, o) and, for
// L2, of |c - c*| (0 when unknown)
struct Front {
  int s, e;
  float dg, dq, dcs, pad;
};

struct Tier3Params {
  const float* X;
  int64_t n;
  int64_t npts;    // rows [0, npts) are points that may block; rows beyond are queries
  int Dp, metric, guide;
  const float* rlo;
  const float* rhi;
  const int2* pairs;
  int64_t m;
  int2* pend;
  int* pflag;
  int64_t slot0;
  int2* amb; unsigned long long* amb_cnt; unsigned long long amb_cap;
  Ancestors anc;
  Front* fbuf;     // per CTA: two frontier buffers of fcap ranges
  const float* pdist_hi;  // [n] upper bound of d(node, its parent), or null
  const int32_t* idx;     // pairs to search: pairs[idx[t]] with slot slot0 + idx[t] (null: all, in order)
  const float* atab;      // [n][tabw] FP32 keys node x ancestor (columns anc.toff[a] + c), or null
  int64_t tabw;
  int fcap;
  int dense;              // ancestor levels scanned densely (needs atab, levels <= 65,536 nodes)
  int mkw;                // words of one candidate bitmask (dynamic shared memory, dense scans)
  unsigned long long* stats;  // [0] frontier overflows, [1] nodes tested, [2] pairs blocked, [3] by the descent
  unsigned long long* prof;   // SM cycles of thread 0: [0] top level and descents [1] lower ancestor levels
                              // [2] node level; [3] pairs reaching the lower ancestor levels
  float lam;                  // beta / 2 of the lune test (1: Eq. 1)
};

// asynchronous 16-byte copy global -> shared (src_bytes < 16: the rest is zero-filled, 0: no read)
__device__ __forceinline__ void cp_async16(void* dst, const void* src, int src_bytes) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src), "r"(src_bytes)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
// wait until at most one committed group of this thread is still in flight
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;" ::: "memory"); }

// lower / upper bound of the distance whose FP32 key is k
__device__ __forceinline__ float dist_lo(float k, int metric, Err e) {
  float lo = fmaxf(lo_b(k, e), 0.0f);
  return metric == L2 ? sqrtf(lo) * (1.0f - 1.1920928955078125e-07f) : lo;
}
__device__ __forceinline__ float dist_hi(float k, int metric, Err e) {
  float hi = hi_b(k, e);
  return metric == L2 ? sqrtf(hi) * (1.0f + 1.1920928955078125e-07f) : hi;
}

// FP32 keys of node pk against g and o, summed by the 8 lanes of a group (lane l8 takes
// the float4 columns l8, l8 + 8, ...): every lane of the group returns both sums.  The
// summation order differs from key32's; the bracket err_fp32 bounds any order.
__device__ __forceinline__ void group_keys(const float* __restrict__ pk, const float* gs, const float* os, int Dp,
                                           int metric, int l8, unsigned gmask, float& a, float& b) {
  const float4* x4 = reinterpret_cast<const float4*>(pk);
  const float4* g4 = reinterpret_cast<const float4*>(gs);
  const float4* o4 = reinterpret_cast<const float4*>(os);
  float sa = 0.0f, sb = 0.0f;
  for (int q = l8; q < (Dp >> 2); q += 8) {
    const float4 x = __ldg(x4 + q), G = g4[q], O = o4[q];
    if (metric == L2) {
      float d;
      d = x.x - G.x; sa = fmaf(d, d, sa); d = x.y - G.y; sa = fmaf(d, d, sa);
      d = x.z - G.z; sa = fmaf(d, d, sa); d = x.w - G.w; sa = fmaf(d, d, sa);
      d = x.x - O.x; sb = fmaf(d, d, sb); d = x.y - O.y; sb = fmaf(d, d, sb);
      d = x.z - O.z; sb = fmaf(d, d, sb); d = x.w - O.w; sb = fmaf(d, d, sb);
    } else {
      sa += fabsf(x.x - G.x); sa += fabsf(x.y - G.y); sa += fabsf(x.z - G.z); sa += fabsf(x.w - G.w);
      sb += fabsf(x.x - O.x); sb += fabsf(x.y - O.y); sb += fabsf(x.z - O.z); sb += fabsf(x.w - O.w);
    }
  }
#pragma unroll
  for (int sh = 4; sh > 0; sh >>= 1) {
    sa += __shfl_xor_sync(gmask, sa, sh);
    sb += __shfl_xor_sync(gmask, sb, sh);
  }
  a = sa;
  b = sb;
}

#define T3_T 256        // threads per CTA (one pair per CTA)
#define T3_MINB 4      // CTAs per SM (64 registers a thread)
#define T3_LIST 1024   // nodes gathered for one round of distance tests
#define T3_MKW 2048    // words of a level's candidate bitmask (levels of at most 65,536 nodes)

// Stage VI (Prop. 4 at the exemplar level, Prop. GRNG_S6 for pivot layers): a whole
// domain of ancestor c is skipped when d(c,x) - rho_c >= t1 or d(c,y) - rho_c >= t2,
// with rho_c bounding the distance from c to any node below it (its radius; delta_max
// for the direct parent).  Descendants of a node are contiguous in the layer order.
// One CTA per pair.  Ancestor levels are scanned either densely (every node of the
// level in order, the survivors of the level above marked in a shared-memory bitmask;
// used when a node x ancestor key table exists and each level has at most 65,536
// nodes), or as a list of index ranges flattened by a prefix sum.  The last ancestor
// level hands the node level a list of ranges with its bounds; the surviving nodes are
// gathered in shared memory and tested by groups of 8 lanes that read each node's
// coordinates as whole 128-byte lines.  For L2, after the top level one greedy descent
// towards the centre c* of the ball around the G-lune tests the nodes of a single
// domain first: a blocker found there ends the pair early.
__global__ void __launch_bounds__(T3_T, T3_MINB) tier3_kernel(Tier3Params p) {
  extern __shared__ __align__(16) float sm3[];
  float* gs = sm3;
  float* os = gs + p.Dp;
  unsigned* mk0 = reinterpret_cast<unsigned*>(os + p.Dp);  // two bitmasks of p.mkw words
  unsigned* mk1 = mk0 + p.mkw;
  __shared__ Front s_rg[T3_T];
  __shared__ int s_pre[T3_T + 1];
  __shared__ int s_wsum[T3_T / 32];
  __shared__ int s_list[T3_LIST];
  __shared__ float4 s_pf[2][2][T3_T];  // keys of the next 4 nodes per thread, copied ahead (cp.async)
  __shared__ unsigned long long s_best;
  __shared__ int s_block, s_nxt_n, s_nl;
  __shared__ float s_v;
  const Err e = err_fp32(p.Dp);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, tid = threadIdx.x;
  const int gid = tid >> 3, l8 = tid & 7;
  const unsigned gmask = 0xffu << (lane & 24);
  const float u2 = 1.1920928955078125e-07f;
  Front* bufA = p.fbuf + (int64_t)blockIdx.x * 2 * p.fcap;
  Front* bufB = bufA + p.fcap;
  unsigned long long n_over = 0, n_tested = 0, n_blk = 0, n_probe = 0;
  __shared__ unsigned long long s_prof[4];  // thread 0's phase cycles (kept out of registers)
  __shared__ long long s_ck[2];
  if (tid == 0) s_prof[0] = s_prof[1] = s_prof[2] = s_prof[3] = 0ull;
  for (int64_t t0 = blockIdx.x; t0 < p.m; t0 += gridDim.x) {
    const int64_t t = p.idx ? p.idx[t0] : t0;
    const int2 pr = p.pairs[t];
    const int64_t g = pr.x, o = pr.y;
    __syncthreads();
    for (int d = tid; d < p.Dp; d += blockDim.x) {
      gs[d] = p.X[g * p.Dp + d];
      os[d] = p.X[o * p.Dp + d];
    }
    if (tid == 0) {
      s_block = 0;
      s_best = ~0ull;
      bufA[0] = Front{0, (int)(p.anc.n ? p.anc.m[0] : p.npts), 0.0f, 0.0f, 0.0f, 0.0f};
    }
    __syncthreads();
    if (tid == 0) s_v = key32(gs, os, p.Dp, p.metric);
    __syncthreads();
    const float v = s_v;
    PairThr P = pair_thresholds(v, p.rlo ? p.rlo[g] : 0.0f, p.rhi ? p.rhi[g] : 0.0f,
                                p.rlo ? p.rlo[o] : 0.0f, p.rhi ? p.rhi[o] : 0.0f, p.metric, e,
                                p.guide, p.lam);
    const int64_t slot = p.slot0 + t;
    // a pair the learned shortlist has already blocked needs no exhaustive scan
    const bool pre = p.pflag[slot] == 3;
    if (!P.quick && !pre) {
      // thresholds as upper bounds in distance units
      const float t1d = p.metric == L2 ? sqrtf(fmaxf(P.t1hi, 0.0f)) * (1.0f + u2) : P.t1hi;
      const float t2d = p.metric == L2 ? sqrtf(fmaxf(P.t2hi, 0.0f)) * (1.0f + u2) : P.t2hi;
      // nodes within Eg of g (Eo of o) cannot satisfy the other condition (triangle)
      const float Eg = excl_dist(v, P.t2hi, p.metric, e), Eo = excl_dist(v, P.t1hi, p.metric, e);
      // L2: the G-lune lies in the ball B(c*, rho), c* = (1-lam) g + lam o, because
      // |k-c*|^2 = (1-lam)|k-g|^2 + lam |k-o|^2 - lam (1-lam) |g-o|^2 (Stewart) for any
      // point k; the same identity gives |c-c*| from the distances of c to g and o.
      const float vlo = fmaxf(lo_b(v, e), 0.0f), vhi = hi_b(v, e);
      float lam = 0.5f, rho2 = -1.0f;
      if (p.metric == L2) {
        lam = fminf(fmaxf((vhi + P.t1hi - P.t2hi) / (2.0f * fmaxf(vhi, 1e-30f)), 0.0f), 1.0f);
        // a beta-lune (zero radii, so lam = 1/2 here): its two ball conditions averaged give
        // (a + b) / 2 < (beta / 2) v, so the bound m1 of the lune of Eq. 1 scales by beta / 2
        const float m1 = ((1.0f - lam) * P.t1hi + lam * P.t2hi) * (P.lam < 1.0f ? P.lam : 1.0f);
        rho2 = m1 - lam * (1.0f - lam) * vlo + 8.0f * u2 * (m1 + lam * (1.0f - lam) * vhi);
      }
      const float rho = rho2 >= 0.0f ? sqrtf(rho2) * (1.0f + u2) : 0.0f;

      // test of one ancestor node c of level a from its keys; on survival, par = the
      // range of its children with its bounds
      auto test_node = [&](int a, int c, float kg, float kq, float R, Front& par) -> bool {
        if (p.metric == L2) {
          // the same pruning in key units, without square roots: d(c,g) >= T1 >= t1d + R
          // (T1 carries 8 rounding units of margin, its square 4 more), so no node of
          // the domain satisfies the first condition; likewise for o
          const float T1 = (t1d + R) * (1.0f + 8.0f * u2), T2 = (t2d + R) * (1.0f + 8.0f * u2);
          if (lo_b(kg, e) >= T1 * T1 * (1.0f + 4.0f * u2) || lo_b(kq, e) >= T2 * T2 * (1.0f + 4.0f * u2))
            return false;
        }
        const float dg = dist_lo(kg, p.metric, e);
        const float dq = dist_lo(kq, p.metric, e);
        bool skip = (dg - R - u2 * (dg + R) >= t1d) || (dq - R - u2 * (dq + R) >= t2d);
        if (!skip) {  // the whole domain lies within the exclusion ball of g or of o
          const float dgh = dist_hi(kg, p.metric, e), dqh = dist_hi(kq, p.metric, e);
          skip = (dgh + R + u2 * (dgh + R) <= Eg) || (dqh + R + u2 * (dqh + R) <= Eo);
        }
        float dcs = 0.0f;
        if (!skip && rho2 >= 0.0f) {  // L2: the domain misses the ball around the G-lune
          const float Alo = fmaxf(lo_b(kg, e), 0.0f), Blo = fmaxf(lo_b(kq, e), 0.0f);
          const float Ahi = hi_b(kg, e), Bhi = hi_b(kq, e);
          const float mm = (1.0f - lam) * Ahi + lam * Bhi + lam * (1.0f - lam) * vhi;
          const float q = (1.0f - lam) * Alo + lam * Blo - lam * (1.0f - lam) * vhi - 8.0f * u2 * mm;
          const float rr = sqrtf(rho2) + R;
          skip = q > 0.0f && q >= rr * rr * (1.0f + 4.0f * u2);
          dcs = q > 0.0f ? sqrtf(q) * (1.0f - u2) : 0.0f;
        }
        if (skip) return false;
        const int32_t* cs = p.anc.cstart[a];
        const int c0 = cs[c], c1 = cs[c + 1];
        par = Front{c0, c1, dg, dq, dcs, 0.0f};
        return c1 > c0;
      };
      // distance tests of nodes list[0..nl) (all threads; uniform call)
      auto test_nodes = [&](const int* list, int nl) {
        for (int i = gid; i < nl; i += T3_T / 8) {
          // one decision per group: its lanes must all reach the shuffles
          if (__shfl_sync(gmask, *(volatile int*)&s_block, 0, 8)) break;
          const int k = list[i];
          float ka, kb;
          group_keys(p.X + (int64_t)k * p.Dp, gs, os, p.Dp, p.metric, l8, gmask, ka, kb);
          if (l8 == 0) {
            ++n_tested;
            const int stt = block_state(ka, kb, P, e);
            if (stt == 2) s_block = 1;
            else if (stt == 1) push_pair(p.amb, p.amb_cnt, p.amb_cap, make_int2((int)slot, k));
          }
        }
      };

      Front* cur = bufA;
      Front* nxt = bufB;
      int ncur = 1;
      bool all = false;
      int a_leaf = 0;  // first level handled by the range loop below
      if (tid == 0) {
        s_ck[0] = clock64();
        s_ck[1] = -1;
      }
      if (p.dense) {
        // ---- dense ancestor levels ------------------------------------------------------
        const bool probe = rho2 >= 0.0f;
        for (int a = 0; a < p.anc.n; ++a) {
          if (a == 1 && tid == 0) {
            s_ck[1] = clock64();
            s_prof[3] += 1;
          }
          const bool last = a == p.anc.n - 1;
          const int ma = (int)p.anc.m[a];
          const unsigned* mk_in = (a & 1) ? mk1 : mk0;
          unsigned* mk_out = (a & 1) ? mk0 : mk1;
          __syncthreads();
          if (!last)
            for (int w = tid; w < (int)((p.anc.m[a + 1] + 31) >> 5); w += blockDim.x) mk_out[w] = 0u;
          if (tid == 0) s_nxt_n = 0;
          __syncthreads();
          const float* rg_ = p.atab + g * p.tabw + p.anc.toff[a];
          const float* ro_ = p.atab + o * p.tabw + p.anc.toff[a];
          unsigned long long best = ~0ull;
          // the keys of a thread's 4 nodes arrive by asynchronous copies one round ahead
          const int nch = (ma + 4 * T3_T - 1) / (4 * T3_T);
          const float* Ra = p.anc.Rhi[a];
          auto issue = [&](int it) {
            const int c = it * 4 * T3_T + 4 * tid;
            const bool in = c < ma;  // the table's rows are padded to 4 columns per level
            cp_async16(&s_pf[it & 1][0][tid], rg_ + (in ? c : 0), in ? 16 : 0);
            cp_async16(&s_pf[it & 1][1][tid], ro_ + (in ? c : 0), in ? 16 : 0);
            cp_async_commit();
          };
          issue(0);
          for (int it = 0; it < nch; ++it) {
            if (it + 1 < nch) issue(it + 1);
            else cp_async_commit();  // an empty group keeps the count uniform
            cp_async_wait1();
            const int c = it * 4 * T3_T + 4 * tid;
            unsigned vm = 0;  // candidate nodes among c .. c+3
#pragma unroll
            for (int u = 0; u < 4; ++u)
              if (c + u < ma && (a == 0 || ((mk_in[(c + u) >> 5] >> ((c + u) & 31)) & 1u))) vm |= 1u << u;
            const float4 G4 = s_pf[it & 1][0][tid], O4 = s_pf[it & 1][1][tid];
            const float kgv[4] = {G4.x, G4.y, G4.z, G4.w}, kqv[4] = {O4.x, O4.y, O4.z, O4.w};
            float Rv[4] = {0.0f, 0.0f, 0.0f, 0.0f};
            if (vm) {
              if (c + 3 < ma) {
                const float4 R4 = __ldg(reinterpret_cast<const float4*>(Ra + c));
                Rv[0] = R4.x; Rv[1] = R4.y; Rv[2] = R4.z; Rv[3] = R4.w;
              } else {
#pragma unroll
                for (int u = 0; u < 4; ++u)
                  if (c + u < ma) Rv[u] = Ra[c + u];
              }
            }
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              Front par;
              const bool keep = ((vm >> u) & 1u) && test_node(a, c + u, kgv[u], kqv[u], Rv[u], par);
              if (keep && a == 0 && probe) {  // Stewart estimate of |c - c*|^2
                const float s2 = fmaxf((1.0f - lam) * kgv[u] + lam * kqv[u] - lam * (1.0f - lam) * v, 0.0f);
                const unsigned long long key = ((unsigned long long)__float_as_uint(s2) << 32) | (unsigned)(c + u);
                best = key < best ? key : best;
              }
              if (!last) {
                if (keep)
                  for (int w = par.s >> 5; w <= (par.e - 1) >> 5; ++w) {
                    const int lo = max(par.s, w << 5), hi = min(par.e, (w << 5) + 32);
                    const unsigned msk = (hi - lo == 32) ? ~0u : (((1u << (hi - lo)) - 1u) << (lo & 31));
                    atomicOr(mk_out + w, msk);
                  }
              } else {
                const unsigned bm = __ballot_sync(FULLMASK, keep);
                int base = 0;
                if (lane == 0 && bm) base = atomicAdd(&s_nxt_n, __popc(bm));
                base = __shfl_sync(FULLMASK, base, 0);
                const int pos = base + __popc(bm & ((1u << lane) - 1u));
                if (keep && pos < p.fcap) nxt[pos] = par;
              }
            }
          }
          if (a == 0 && probe) {
            for (int sh = 16; sh > 0; sh >>= 1) {
              const unsigned long long y = __shfl_xor_sync(FULLMASK, best, sh);
              best = y < best ? y : best;
            }
            if (lane == 0 && best != ~0ull) atomicMin(&s_best, best);
          }
          __syncthreads();
          if (a == 0 && probe && s_best != ~0ull) {
            // ---- greedy descents towards c*, whose final domains' nodes are tested now:
            // warp w starts from the top-level node nearest c* among those its lanes
            // scanned (the nearest overall is one of them) ----
            if (best != ~0ull) {
              int cn = (int)(best & 0xffffffffu);
              int lvl = 0;
              bool ok = true;
              while (lvl < p.anc.n - 1) {
                const int c0 = p.anc.cstart[lvl][cn], c1 = p.anc.cstart[lvl][cn + 1];
                if (c1 <= c0) { ok = false; break; }
                ++lvl;
                unsigned long long bb = ~0ull;
                for (int c = c0 + lane; c < c1; c += 32) {
                  const float kg = p.atab[g * p.tabw + p.anc.toff[lvl] + c];
                  const float kq = p.atab[o * p.tabw + p.anc.toff[lvl] + c];
                  const float s2 = fmaxf((1.0f - lam) * kg + lam * kq - lam * (1.0f - lam) * v, 0.0f);
                  const unsigned long long key = ((unsigned long long)__float_as_uint(s2) << 32) | (unsigned)c;
                  bb = key < bb ? key : bb;
                }
                for (int sh = 16; sh > 0; sh >>= 1) {
                  const unsigned long long y = __shfl_xor_sync(FULLMASK, bb, sh);
                  bb = y < bb ? y : bb;
                }
                cn = (int)(bb & 0xffffffffu);
              }
              if (ok) {
                const int k0 = p.anc.cstart[lvl][cn], k1 = p.anc.cstart[lvl][cn + 1];
                for (int k = k0 + (lane >> 3); k < k1; k += 4) {
                  if (k == g || k == o) continue;  // uniform within the group
                  float ka, kb;
                  group_keys(p.X + (int64_t)k * p.Dp, gs, os, p.Dp, p.metric, l8, gmask, ka, kb);
                  if (l8 == 0) {
                    ++n_tested;
                    const int stt = block_state(ka, kb, P, e);
                    if (stt == 2) s_block = 1;
                    else if (stt == 1) push_pair(p.amb, p.amb_cnt, p.amb_cap, make_int2((int)slot, k));
                  }
                }
              }
            }
            __syncthreads();
            if (s_block) {  // uniform: read after a barrier
              n_probe += tid == 0;
              break;
            }
          }
        }
        a_leaf = p.anc.n;
        if (!s_block) {
          if (s_nxt_n > p.fcap) {
            all = true;
            n_over += tid == 0;
          } else {
            ncur = s_nxt_n;
            Front* tmp = cur; cur = nxt; nxt = tmp;
          }
        }
      }
      if (tid == 0) {  // the top level and descents, then the lower ancestor levels
        const long long ck2 = clock64();
        s_prof[0] += (unsigned long long)((s_ck[1] >= 0 ? s_ck[1] : ck2) - s_ck[0]);
        if (s_ck[1] >= 0) s_prof[1] += (unsigned long long)(ck2 - s_ck[1]);
        s_ck[0] = ck2;
      }
      // ---- range levels (a >= a_leaf); level a = anc.n is the layer's own nodes ----------
      for (int a = a_leaf; a <= p.anc.n && !all && !s_block; ++a) {
        const bool leaf = a == p.anc.n;
        __syncthreads();  // every thread has read the previous level's count
        if (tid == 0) { s_nxt_n = 0; s_nl = 0; }
        for (int cb = 0; cb < ncur; cb += T3_T) {
          // ---- flatten T3_T ranges: s_pre = exclusive prefix of their lengths ----
          __syncthreads();
          int len = 0;
          if (cb + tid < ncur) {
            const Front f = cur[cb + tid];
            s_rg[tid] = f;
            len = f.e - f.s;
          }
          int inc = len;
#pragma unroll
          for (int sh = 1; sh < 32; sh <<= 1) {
            const int y = __shfl_up_sync(FULLMASK, inc, sh);
            if (lane >= sh) inc += y;
          }
          if (lane == 31) s_wsum[warp] = inc;
          __syncthreads();
          int woff = 0;
          for (int w = 0; w < warp; ++w) woff += s_wsum[w];
          s_pre[tid + 1] = woff + inc;
          if (tid == 0) s_pre[0] = 0;
          __syncthreads();
          const int total = s_pre[T3_T];
          const int nrg = ncur - cb < T3_T ? ncur - cb : T3_T;
          for (int j0 = 0; j0 < total; j0 += T3_T) {
            const int j = j0 + tid;
            bool keep = false;
            int c = -1;
            Front par;
            if (j < total) {
              int lo = 0, hi = nrg - 1;  // the last range q with s_pre[q] <= j
              while (lo < hi) {
                const int mid = (lo + hi + 1) >> 1;
                if (s_pre[mid] <= j) lo = mid; else hi = mid - 1;
              }
              par = s_rg[lo];
              c = par.s + (j - s_pre[lo]);
              if (leaf) {
                keep = c != g && c != o;
                if (keep && p.pdist_hi && (par.dg > 0.0f || par.dq > 0.0f || par.dcs > 0.0f)) {
                  // Prop. 5 / GRNG_S6 (assisted): |c - g| >= d(parent,g) - d(c,parent), ...
                  const float mk = p.pdist_hi[c];
                  const float sl = u2 * (par.dg + par.dq + par.dcs + mk);
                  keep = !(par.dg - mk - sl >= t1d || par.dq - mk - sl >= t2d ||
                           (rho2 >= 0.0f && par.dcs - mk - sl >= rho));
                }
              } else {
                float kg, kq;
                if (p.atab) {
                  kg = p.atab[g * p.tabw + p.anc.toff[a] + c];
                  kq = p.atab[o * p.tabw + p.anc.toff[a] + c];
                } else {
                  const float* pc = p.anc.X[a] + (int64_t)c * p.Dp;
                  kg = key32(pc, gs, p.Dp, p.metric);
                  kq = key32(pc, os, p.Dp, p.metric);
                }
                keep = test_node(a, c, kg, kq, p.anc.Rhi[a][c], par);
              }
            }
            const unsigned bm = __ballot_sync(FULLMASK, keep);
            if (leaf) {
              int base = 0;
              if (lane == 0 && bm) base = atomicAdd(&s_nl, __popc(bm));
              base = __shfl_sync(FULLMASK, base, 0);
              if (keep) s_list[base + __popc(bm & ((1u << lane) - 1u))] = c;
              __syncthreads();
              const int nl = s_nl;
              // ---- distance tests once the list is nearly full, or at the end ----
              if (nl > T3_LIST - T3_T || (nl > 0 && j0 + T3_T >= total && cb + T3_T >= ncur)) {
                test_nodes(s_list, nl);
                __syncthreads();
                if (tid == 0) s_nl = 0;
              }
              __syncthreads();
              if (s_block) break;
            } else {
              int base = 0;
              if (lane == 0 && bm) base = atomicAdd(&s_nxt_n, __popc(bm));
              base = __shfl_sync(FULLMASK, base, 0);
              const int pos = base + __popc(bm & ((1u << lane) - 1u));
              if (keep && pos < p.fcap) nxt[pos] = par;
            }
          }
          if (leaf && s_block) break;  // s_block was read after a barrier: uniform
        }
        if (leaf) break;
        __syncthreads();
        if (s_nxt_n > p.fcap) {
          all = true;
          n_over += tid == 0;
        } else {
          ncur = s_nxt_n;
          Front* tmp = cur; cur = nxt; nxt = tmp;
        }
      }
      if (all) {  // frontier too large: test every node (still exact)
        for (int i = gid; i < (int)p.npts; i += T3_T / 8) {
          if (__shfl_sync(gmask, *(volatile int*)&s_block, 0, 8)) break;
          if (i == g || i == o) continue;
          float ka, kb;
          group_keys(p.X + (int64_t)i * p.Dp, gs, os, p.Dp, p.metric, l8, gmask, ka, kb);
          if (l8 == 0) {
            ++n_tested;
            const int stt = block_state(ka, kb, P, e);
            if (stt == 2) s_block = 1;
            else if (stt == 1) push_pair(p.amb, p.amb_cnt, p.amb_cap, make_int2((int)slot, i));
          }
        }
      }
      if (tid == 0) s_prof[2] += (unsigned long long)(clock64() - s_ck[0]);  // the node level
    }
    __syncthreads();
    if (tid == 0) {
      p.pend[slot] = make_int2((int)g, (int)o);
      if (s_block) p.pflag[slot] = 3;
      n_blk += s_block != 0;
    }
  }
  for (int sh = 16; sh > 0; sh >>= 1) n_tested += __shfl_down_sync(FULLMASK, n_tested, sh);
  if (lane == 0 && n_tested) atomicAdd(p.stats + 1, n_tested);
  if (tid == 0 && n_over) atomicAdd(p.stats + 0, n_over);
  if (tid == 0 && n_blk) atomicAdd(p.stats + 2, n_blk);
  if (tid == 0 && n_probe) atomicAdd(p.stats + 3, n_probe);
  if (tid == 0 && p.prof)
    for (int i = 0; i < 4; ++i) atomicAdd(p.prof + i, s_prof[i]);
}

// Before the exhaustive tier, one warp per pair: the centre c* of the ball around the G-lune
// is located through the ancestor key table (Stewart's identity, as in tier 3), and from each
// of the T3P_DESC top-level nodes nearest c* the warp descends greedily to one finest domain
// and tests its nodes.  A pair some node certainly blocks is decided here (its pending slot
// is flagged); the others are listed for the exhaustive tier.  Which pairs are decided here
// changes the work only, never a decision.
#define T3P_DESC 3
#define T3P_WARPS 8
__global__ void __launch_bounds__(T3P_WARPS * 32) tier3_probe_kernel(Tier3Params p, int32_t* __restrict__ rest,
                                                                     unsigned long long* __restrict__ nrest,
                                                                     unsigned long long* __restrict__ nblocked,
                                                                     unsigned long long* __restrict__ next) {
  extern __shared__ __align__(16) float t3p_sm[];
  const int lane = threadIdx.x & 31, wib = threadIdx.x >> 5;
  const int l8 = lane & 7;
  const unsigned gmask = 0xffu << (lane & 24);
  float* gs = t3p_sm + wib * 2 * p.Dp;
  float* os = gs + p.Dp;
  const Err e = err_fp32(p.Dp);
  const float u2 = 1.1920928955078125e-07f;
  const int na = p.anc.n;
  unsigned long long c_blk = 0;
  for (;;) {  // pairs in order, from an atomic counter (neighbouring pairs share table rows)
    unsigned long long tt = 0;
    if (lane == 0) tt = atomicAdd(next, 1ull);
    const int64_t t = (int64_t)__shfl_sync(FULLMASK, tt, 0);
    if (t >= p.m) break;
    const int2 pr = p.pairs[t];
    const int64_t g = pr.x, o = pr.y;
    __syncwarp();
    for (int d = lane; d < p.Dp; d += 32) {
      gs[d] = p.X[g * p.Dp + d];
      os[d] = p.X[o * p.Dp + d];
    }
    __syncwarp();
    float v = 0.0f;
    if (lane == 0) v = key32(gs, os, p.Dp, p.metric);
    v = __shfl_sync(FULLMASK, v, 0);
    const PairThr P = pair_thresholds(v, p.rlo ? p.rlo[g] : 0.0f, p.rhi ? p.rhi[g] : 0.0f,
                                      p.rlo ? p.rlo[o] : 0.0f, p.rhi ? p.rhi[o] : 0.0f, p.metric, e, p.guide,
                                      p.lam);
    bool blocked = false;
    if (!P.quick) {
      const float vlo = fmaxf(lo_b(v, e), 0.0f), vhi = hi_b(v, e);
      const float lam = fminf(fmaxf((vhi + P.t1hi - P.t2hi) / (2.0f * fmaxf(vhi, 1e-30f)), 0.0f), 1.0f);
      (void)vlo;
      (void)u2;
      // the lane's three top-level nodes nearest c* (Stewart estimate of |c - c*|^2)
      unsigned long long b0 = ~0ull, b1 = ~0ull, b2 = ~0ull;
      const float* rg = p.atab + g * p.tabw + p.anc.toff[0];
      const float* ro = p.atab + o * p.tabw + p.anc.toff[0];
      for (int c = lane; c < (int)p.anc.m[0]; c += 32) {
        const float s2 = fmaxf((1.0f - lam) * rg[c] + lam * ro[c] - lam * (1.0f - lam) * v, 0.0f);
        const unsigned long long key = ((unsigned long long)__float_as_uint(s2) << 32) | (unsigned)c;
        if (key < b2) {
          if (key < b1) {
            b2 = b1;
            if (key < b0) { b1 = b0; b0 = key; }
            else b1 = key;
          } else {
            b2 = key;
          }
        }
      }
      for (int round = 0; round < T3P_DESC && !blocked; ++round) {
        unsigned long long best = b0;
        for (int sh = 16; sh > 0; sh >>= 1) {
          const unsigned long long y2 = __shfl_xor_sync(FULLMASK, best, sh);
          best = y2 < best ? y2 : best;
        }
        if (best == ~0ull) break;
        if (b0 == best) { b0 = b1; b1 = b2; b2 = ~0ull; }  // the winning lane moves on
        int cn = (int)(best & 0xffffffffu);
        int lvl = 0;
        bool ok = true;
        while (lvl < na - 1) {
          const int c0 = p.anc.cstart[lvl][cn], c1 = p.anc.cstart[lvl][cn + 1];
          if (c1 <= c0) { ok = false; break; }
          ++lvl;
          unsigned long long bb = ~0ull;
          for (int c = c0 + lane; c < c1; c += 32) {
            const float kg = p.atab[g * p.tabw + p.anc.toff[lvl] + c];
            const float kq = p.atab[o * p.tabw + p.anc.toff[lvl] + c];
            const float s2 = fmaxf((1.0f - lam) * kg + lam * kq - lam * (1.0f - lam) * v, 0.0f);
            const unsigned long long key = ((unsigned long long)__float_as_uint(s2) << 32) | (unsigned)c;
            bb = key < bb ? key : bb;
          }
          for (int sh = 16; sh > 0; sh >>= 1) {
            const unsigned long long y2 = __shfl_xor_sync(FULLMASK, bb, sh);
            bb = y2 < bb ? y2 : bb;
          }
          cn = (int)(bb & 0xffffffffu);
        }
        if (!ok) continue;
        const int k0 = p.anc.cstart[lvl][cn], k1 = p.anc.cstart[lvl][cn + 1];
        for (int kb = k0; kb < k1; kb += 4) {
          const int k = kb + (lane >> 3);
          const bool in = k < k1 && k != (int)g && k != (int)o;  // uniform within the group
          float ka = 0.0f, kb2 = 0.0f;
          group_keys(p.X + (int64_t)(in ? k : (int)g) * p.Dp, gs, os, p.Dp, p.metric, l8, gmask, ka, kb2);
          const bool hit = in && l8 == 0 && block_state(ka, kb2, P, e) == 2;
          if (__any_sync(FULLMASK, hit)) { blocked = true; break; }
        }
      }
    }
    if (lane == 0) {
      if (blocked) {
        if (p.pend) {  // null: a blocked pair is dropped (its bits are zero in both graphs)
          p.pend[p.slot0 + t] = pr;
          p.pflag[p.slot0 + t] = 3;
        }
        ++c_blk;
      } else {
        rest[atomicAdd(nrest, 1ull)] = (int32_t)t;
      }
    }
  }
  if (lane == 0 && c_blk) atomicAdd(nblocked, c_blk);
}

__global__ void gather_pairs_kernel(const int2* __restrict__ pairs, const int32_t* __restrict__ idx, int64_t m,
                                    int2* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = pairs[idx[i]];
}

// node x ancestor keys: out[r * ld + c] = key(Xr[r], Xc[c]) for a 128 x 128 tile per CTA
template <int KC, int METRIC>
__global__ void __launch_bounds__(GRNG_THREADS) cross_keys_kernel(const float* __restrict__ Xr, int64_t nr_all,
                                                                  const float* __restrict__ Xc, int64_t nc_all,
                                                                  int Dp, float* __restrict__ out, int64_t ld) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* sA = reinterpret_cast<float*>(sm_raw);
  float* sB = sA + KC * GRNG_SSTRIDE;
  float* T = sB + KC * GRNG_SSTRIDE;
  const int64_t rb = (int64_t)blockIdx.x * GRNG_TILE, cb = (int64_t)blockIdx.y * GRNG_TILE;
  const int nr = (int)(nr_all - rb < GRNG_TILE ? nr_all - rb : GRNG_TILE);
  const int nc = (int)(nc_all - cb < GRNG_TILE ? nc_all - cb : GRNG_TILE);
  float acc[8][8];
  tile_keys<KC, METRIC>(Xr + rb * Dp, nr, Xc + cb * Dp, nc, Dp, sA, sB, acc);
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) T[tile_row(i) * 129 + tile_col(j)] = acc[i][j];
  __syncthreads();
  for (int i = threadIdx.x; i < GRNG_TILE * GRNG_TILE; i += GRNG_THREADS) {
    const int r = i >> 7, c = i & 127;
    if (r < nr && c < nc) out[(rb + r) * ld + cb + c] = T[r * 129 + c];
  }
}

template <int KC>
static void launch_cross_kc(const float* Xr, int64_t nr, const float* Xc, int64_t nc, int Dp, int metric, float* out,
                            int64_t ld, cudaStream_t s) {
  const size_t smem = (size_t)(2 * KC * GRNG_SSTRIDE + 128 * 129) * 4;
  dim3 grid((unsigned)((nr + GRNG_TILE - 1) / GRNG_TILE), (unsigned)((nc + GRNG_TILE - 1) / GRNG_TILE));
  if (metric == L2) {
    GRNG_CUDA(cudaFuncSetAttribute(cross_keys_kernel<KC, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cross_keys_kernel<KC, L2><<<grid, GRNG_THREADS, smem, s>>>(Xr, nr, Xc, nc, Dp, out, ld); note_launch();
  } else {
    GRNG_CUDA(cudaFuncSetAttribute(cross_keys_kernel<KC, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    cross_keys_kernel<KC, L1><<<grid, GRNG_THREADS, smem, s>>>(Xr, nr, Xc, nc, Dp, out, ld); note_launch();
  }
  GRNG_CUDA(cudaGetLastError());
}
static void launch_cross(const float* Xr, int64_t nr, const float* Xc, int64_t nc, int Dp, int metric, float* out,
                         int64_t ld, cudaStream_t s) {
  const int KC = Dp % 32 == 0 ? 32 : (Dp % 16 == 0 ? 16 : 8);
  if (KC == 32) launch_cross_kc<32>(Xr, nr, Xc, nc, Dp, metric, out, ld, s);
  else if (KC == 16) launch_cross_kc<16>(Xr, nr, Xc, nc, Dp, metric, out, ld, s);
  else launch_cross_kc<8>(Xr, nr, Xc, nc, Dp, metric, out, ld, s);
}

// ---------------------------------------------------------------------------------
// Range lists (pivot layers): pairs that neither endpoint's neighbour list covers.
// Every endpoint s of such a pair gets T_s, the largest threshold among its pairs.
// One sweep histograms, per node, the keys below T_s in buckets of 1/16 octave of
// key (bucket = hist_bin(key, T_s)); the list keeps the lowest buckets whose total
// stays within the list length, and a second sweep writes every such node into its
// bucket's slots, so a list is ordered by bucket (unordered inside one).  T'_s, a
// lower bound of every key the list leaves out, decides coverage: a pair is covered
// from a side whose T'_s reaches past its threshold on that side, because every node
// that could satisfy that condition is then listed (GRNG definition, Sec. 2).
//   - covered from one side (or both: the shorter annulus): that list's annulus is
//     bounded node by node through the node's parent (ancestor key table) and only the
//     nodes no bound settles are tested by distance to the other endpoint;
//   - uncovered pairs go to the exhaustive tier.
// ---------------------------------------------------------------------------------
#define GRNG_LMAX 16384  // list length (a list never exceeds it: its buckets are counted first)
#define GRNG_LCAP 16384  // list slots per node
#define GRNG_HBINS 128

struct SideParams {
  const float* X;
  int Dp, metric, guide, K;
  const float* rlo;
  const float* rhi;
  const int2* pairs;
  int64_t m;
  int8_t* side;               // 3: linked; 0 / 1: covered from x / y only; 4 / 5: both, x's / y's annulus
                              // the shorter; 2: neither
  unsigned int* tkey;         // [n] float bits of T_s (key units)
  const unsigned int* tcut;   // [n] float bits of T'_s
  const int* lcnt;            // [n] listed nodes
  const int* lastb;           // [n] last listed bucket (side choice, once the lists exist)
  const int* boff;            // [n][GRNG_HBINS + 1] bucket starts
};

__device__ __forceinline__ PairThr thr_of(const SideParams& p, int a, int b, float v, Err e) {
  return pair_thresholds(v, p.rlo ? p.rlo[a] : 0.0f, p.rhi ? p.rhi[a] : 0.0f, p.rlo ? p.rlo[b] : 0.0f,
                         p.rhi ? p.rhi[b] : 0.0f, p.metric, e, p.guide);
}

// thresholds of both sides raise T_s of both endpoints
__global__ void range_thresholds_kernel(SideParams p) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.m) return;
  const Err e = err_fp32(p.Dp);
  const int a = p.pairs[t].x, b = p.pairs[t].y;
  const float v = key32(p.X + (int64_t)a * p.Dp, p.X + (int64_t)b * p.Dp, p.Dp, p.metric);
  const PairThr P = thr_of(p, a, b, v, e);
  if (P.quick) { p.side[t] = 3; return; }
  p.side[t] = 2;
  atomicMax(p.tkey + a, __float_as_uint(P.t1hi));  // positive floats order like their bits
  atomicMax(p.tkey + b, __float_as_uint(P.t2hi));
}

// Bucket of a key below T: 16 buckets per octave of key, 0 for everything under
// T / 2^(127/16).  The same function (same inputs, same code) places keys in the
// histogram and in the lists, so the bucket counts are the list's.
__device__ __forceinline__ int hist_bin(float v, float T) {
  const float l = log2f(fmaxf(v, 1e-37f) / T);  // < 0 for v < T
  return max(0, min(GRNG_HBINS - 1, (int)floorf(16.0f * l) + GRNG_HBINS));
}

// Entries [first, last) of s's list whose keys may lie in (klo, khi): the buckets from
// one below klo's to one above khi's (hist_bin carries far less than a bucket of error,
// the FP32 brackets of the filters less again; for bounds below 1e-30 the absolute term
// of the bracket could span buckets, so the span then runs to the end of the list).
__device__ __forceinline__ int2 list_span(const int* lastb, const int* boff, const unsigned int* tkey, int s,
                                          float klo, float khi) {
  const int last = lastb[s];
  if (last < 0 || !(khi > 0.0f)) return make_int2(0, 0);
  const float T = __uint_as_float(tkey[s]);
  const int b0 = klo > 1e-30f ? max(hist_bin(klo, T) - 1, 0) : 0;
  const int b1 = khi > 1e-30f ? min(hist_bin(khi, T) + 1, last) : last;
  if (b1 < b0) return make_int2(0, 0);
  const int* bo = boff + (int64_t)s * (GRNG_HBINS + 1);
  return make_int2(bo[b0], bo[b1 + 1]);
}

// which sides cover the pair; covered from both, the side whose annulus is shorter
__global__ void pick_side_kernel(SideParams p) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= p.m || p.side[t] == 3) return;
  const Err e = err_fp32(p.Dp);
  const int a = p.pairs[t].x, b = p.pairs[t].y;
  const float v = key32(p.X + (int64_t)a * p.Dp, p.X + (int64_t)b * p.Dp, p.Dp, p.metric);
  const PairThr P = thr_of(p, a, b, v, e);
  const bool ca = p.lcnt[a] <= GRNG_LCAP && lo_b(__uint_as_float(p.tcut[a]), e) >= P.t1hi;
  const bool cb = p.lcnt[b] <= GRNG_LCAP && lo_b(__uint_as_float(p.tcut[b]), e) >= P.t2hi;
  int sd = ca && cb ? 4 : ca ? 0 : cb ? 1 : 2;
  if (sd == 4 && !P.quick) {
    const float ekx = excl_key(excl_dist(v, P.t2hi, p.metric, e), p.metric);
    const float eky = excl_key(excl_dist(v, P.t1hi, p.metric, e), p.metric);
    const int2 ax = list_span(p.lastb, p.boff, p.tkey, a, ekx, P.t1hi);
    const int2 ay = list_span(p.lastb, p.boff, p.tkey, b, eky, P.t2hi);
    sd = (ay.y - ay.x) < (ax.y - ax.x) ? 5 : 4;
  }
  p.side[t] = (int8_t)sd;
}

// The list tier's pairs regrouped (counting sort) by the block of 256 (or more) nodes of the
// endpoint whose list they scan and the block of the other endpoint, and handed to the warps
// in that order by an atomic counter: the warps at work at one time then read a few lists
// and a few rows of the ancestor key table, which stay in L2.
static __device__ __forceinline__ int scan_node(int2 pr, int sd) { return (sd == 1 || sd == 5) ? pr.y : pr.x; }
// group key: (block of the scanned node, block of the other node), blocks of `bs` nodes
static __device__ __forceinline__ int64_t side_key(int2 pr, int sd, int bs, int64_t nbk) {
  const int sn = scan_node(pr, sd), on = (sn == pr.x) ? pr.y : pr.x;
  return (int64_t)(sn / bs) * nbk + on / bs;
}
__global__ void side_count_kernel(const int2* __restrict__ pairs, const int8_t* __restrict__ side, int64_t m,
                                  int64_t* __restrict__ cnt, int bs, int64_t nbk) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) atomicAdd(reinterpret_cast<unsigned long long*>(cnt + side_key(pairs[t], side[t], bs, nbk)), 1ull);
}
__global__ void side_scatter_kernel(const int2* __restrict__ pairs, const int8_t* __restrict__ side, int64_t m,
                                    int64_t* __restrict__ cur, int2* __restrict__ opairs, int8_t* __restrict__ oside,
                                    int bs, int64_t nbk) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const int2 pr = pairs[t];
  const int sd = side[t];
  const int64_t q = (int64_t)atomicAdd(reinterpret_cast<unsigned long long*>(cur + side_key(pr, sd, bs, nbk)), 1ull);
  opairs[q] = pr;
  oside[q] = (int8_t)sd;
}

// Per list entry, when the level has parents and a node x ancestor key table: the listed
// node's parent, the upper bound of its distance to that parent, and the parent's key to
// the list's own node -- what the list tier's bounds read, kept beside the entry so that
// one pass over a list streams them.
struct ListAux {
  const int32_t* parent = nullptr;  // [n] parent positions
  const float* pdist = nullptr;     // [n] upper bounds of d(node, parent)
  const float* atab = nullptr;      // node x ancestor keys, the parent level at column toff
  int64_t tabw = 0, toff = 0;
  int32_t* par = nullptr;           // [n][GRNG_LCAP] outputs beside lidx / lkey
  float* pdh = nullptr;
  float* pkey = nullptr;
};

// mode 0: per-row histogram of keys below T_s; mode 1: every node with key < T_s whose
// bucket is at most the row's last listed bucket, written at its bucket's cursor.  Each
// thread scans the 8 x 8 keys it holds in registers and counts (or claims list slots) with
// shared-memory atomics, so all 256 threads scan and no key tile is staged; the order of
// the nodes within one bucket of a list is then the order of the atomics (the list tier
// reads a bucket whole or stops at a blocker, so the decisions do not depend on it).
template <int KC, int METRIC>
__global__ void __launch_bounds__(GRNG_THREADS, 2) range_sweep_kernel(const float* __restrict__ X, int64_t n, int Dp,
                                                                      const unsigned int* __restrict__ tkey,
                                                                      int* __restrict__ hist,
                                                                      const int* __restrict__ lastb,
                                                                      const int* __restrict__ boff,
                                                                      int32_t* __restrict__ lidx,
                                                                      float* __restrict__ lkey, int fill,
                                                                      ListAux aux) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* sA = reinterpret_cast<float*>(sm_raw);
  float* sB = sA + KC * GRNG_SSTRIDE;
  int* H = reinterpret_cast<int*>(sB + KC * GRNG_SSTRIDE);  // [GRNG_HBINS][128]: counts or cursors
  float* Ts = reinterpret_cast<float*>(H + GRNG_HBINS * 128);  // [128] T_s of the rows (0: inactive)
  int* Ls = reinterpret_cast<int*>(Ts + 128);                 // [128] last listed bucket
  const int64_t xb = (int64_t)blockIdx.x * GRNG_TILE;
  const int nr = (int)(n - xb < GRNG_TILE ? n - xb : GRNG_TILE);
  const int tid = threadIdx.x;
  bool act = false;
  if (tid < 128) {
    const float Tr = tid < nr ? __uint_as_float(tkey[xb + tid]) : 0.0f;
    const int lastr = (fill && tid < nr) ? lastb[xb + tid] : GRNG_HBINS - 1;
    act = tid < nr && Tr > 0.0f && lastr >= 0;
    Ts[tid] = act ? Tr : 0.0f;
    Ls[tid] = lastr;
  }
  if (!__syncthreads_or(act)) return;
  for (int i = tid; i < GRNG_HBINS * 128; i += GRNG_THREADS) {
    const int b = i >> 7, r = i & 127;
    H[i] = (fill && r < nr) ? boff[(xb + r) * (GRNG_HBINS + 1) + b] : 0;
  }
  __syncthreads();
  const int64_t nb = (n + GRNG_TILE - 1) / GRNG_TILE;
  for (int64_t by = 0; by < nb; ++by) {
    const int64_t yb = by * GRNG_TILE;
    const int nc = (int)(n - yb < GRNG_TILE ? n - yb : GRNG_TILE);
    float acc[8][8];
    tile_keys<KC, METRIC>(X + xb * Dp, nr, X + yb * Dp, nc, Dp, sA, sB, acc);
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      const int row = tile_row(i);
      const float Tr = Ts[row];
      if (!(Tr > 0.0f)) continue;
      const int lastr = Ls[row];
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int col = tile_col(j);
        const float v = acc[i][j];
        if (!(v < Tr) || col >= nc || yb + col == xb + row) continue;
        const int b = hist_bin(v, Tr);
        if (!fill) {
          atomicAdd(&H[b * 128 + row], 1);
        } else if (b <= lastr) {
          const int pos = atomicAdd(&H[b * 128 + row], 1);
          if (pos < GRNG_LCAP) {  // always: the counts of both sweeps agree
            const int64_t k = yb + col;
            const int64_t q = (xb + row) * GRNG_LCAP + pos;
            lidx[q] = (int32_t)k;
            lkey[q] = v;
            if (aux.par) {  // the listed node's parent, its distance bound and the parent's key to the row
              const int c = aux.parent[k];
              aux.par[q] = c;
              aux.pdh[q] = aux.pdist[k];
              aux.pkey[q] = aux.atab[(xb + row) * aux.tabw + aux.toff + c];
            }
          }
        }
      }
    }
  }
  __syncthreads();
  if (!fill && tid < nr)
    for (int b = 0; b < GRNG_HBINS; ++b) hist[(xb + tid) * GRNG_HBINS + b] = H[b * 128 + tid];
}

// The last bucket that keeps the cumulative count <= lmax, the bucket offsets of the
// list, its length, and T'_s: T_s when every bucket is listed, otherwise the lower edge
// of the first bucket left out, shrunk by 2^-16 relative -- far more than the error of
// hist_bin (a float log2 of a quotient, a few 2^-24 in 16 log2 units against 16 * 2^-16
// / ln 2), so every key below T'_s lies in a listed bucket.
__global__ void range_cut_kernel(const unsigned int* __restrict__ tkey, const int* __restrict__ hist, int64_t n,
                                 unsigned int* __restrict__ tcut, int* __restrict__ lastb, int* __restrict__ boff,
                                 int* __restrict__ lcnt, int lmax) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const float T = __uint_as_float(tkey[s]);
  int last = -1, cum = 0;
  int* bo = boff + s * (GRNG_HBINS + 1);
  bo[0] = 0;
  if (T > 0.0f) {
    for (int b = 0; b < GRNG_HBINS; ++b) {
      const int h = hist[s * GRNG_HBINS + b];
      if (cum + h > lmax) break;
      cum += h;
      last = b;
      bo[b + 1] = cum;
    }
  }
  for (int b = last + 1; b < GRNG_HBINS; ++b) bo[b + 1] = cum;
  float cut = 0.0f;
  if (last == GRNG_HBINS - 1) cut = T;
  else if (last >= 0) cut = T * exp2f((float)(last + 1 - GRNG_HBINS) / 16.0f) * (1.0f - 1.52587890625e-05f);
  tcut[s] = __float_as_uint(cut);
  lastb[s] = last;
  lcnt[s] = cum;
}

struct ListParams {
  const float* X;
  int Dp, metric, guide;
  const float* rlo;
  const float* rhi;
  const int2* pairs;
  int64_t m;
  const int8_t* side;
  const unsigned int* tkey;  // [n] T_s
  const int* lastb;          // [n] last listed bucket (-1: empty list)
  const int* boff;           // [n][GRNG_HBINS + 1] start of each bucket in the list
  const int32_t* lidx;
  const float* lkey;
  // node x ancestor key table (or null): column toff + c holds key(node, parent-level node c);
  // parent[k] is k's parent, pdh[k] an upper bound of d(k, parent[k])
  const float* atab;
  int64_t tabw, toff;
  const int32_t* lpar;   // per entry: the listed node's parent, d(node, parent) bound, parent's key to s
  const float* lpdh;
  const float* lpk;
  int2* links; unsigned long long* link_cnt; unsigned long long link_cap;
  int2* unres; unsigned long long* unres_cnt; unsigned long long unres_cap;
  int2* pend; unsigned long long* pend_cnt; unsigned long long pend_cap;
  int2* amb; unsigned long long* amb_cnt; unsigned long long amb_cap;
  unsigned long long* stats;  // [0] links [1] pending [2] to tier 3 [3] blocked [4] listed nodes tested by
                              // distance [5] pairs covered from both sides [6] the pair counter [7] list
                              // entries read
};

__device__ __forceinline__ int2 bucket_span(const ListParams& p, int s, float klo, float khi) {
  return list_span(p.lastb, p.boff, p.tkey, s, klo, khi);
}

#define LT_WARPS 8

// Decision of one list-tier pair, counted per warp.
struct LtCount {
  unsigned long long link = 0, pend = 0, un = 0, blk = 0, test = 0, both = 0, read = 0;
};

// Ambiguous triples of a pair that nothing blocked are recorded in a second pass; the
// pair takes a pending slot first.
__device__ __forceinline__ unsigned long long lt_pend_slot(const ListParams& p, int2 pr, int lane) {
  unsigned long long slot = 0;
  if (lane == 0) slot = atomicAdd(p.pend_cnt, 1ull);
  slot = __shfl_sync(FULLMASK, slot, 0);
  if (lane == 0 && slot < p.pend_cap) p.pend[slot] = pr;
  return slot;
}

// Pairs covered from one side s: the annulus of s's list, tested against the other
// endpoint o.  Each listed node k is first bounded through its parent c, whose keys to x and
// y the ancestor table holds: d(k,o) >= d(c,o) - d(k,c) settles "k fails the condition at o"
// (triangle inequality); for L2, a lower bound of |k - c*| (Stewart's identity, from k's own
// key to s and that bound, or from c) of at least rho puts k outside the ball around the
// G-lune, as in tier 3; and d(k,o) <= d(c,o) + d(k,c) can settle "k blocks".  Only the nodes
// no bound settles get their distance to o, computed by groups of G lanes.
template <int G, int NQ>
__device__ __forceinline__ void lt_scan(const ListParams& p, int2 pr, int sd, float v, const PairThr& P, float ekx,
                                        float eky, Err e, int lane, LtCount& c, bool& blocked, bool& anyamb) {
  const int x = pr.x, y = pr.y;
  const int gl = lane % G, gi = lane / G;
  const int s = sd ? y : x, o = sd ? x : y;
  const float slo = sd ? eky : ekx, shi = sd ? P.t2hi : P.t1hi;
  const float olo_k = sd ? P.t1lo : P.t2lo, ohi_k = sd ? P.t1hi : P.t2hi;  // thresholds at o (keys)
  const float slo_k = sd ? P.t2lo : P.t1lo;                                // certain side at s
  const int2 sp = bucket_span(p, s, slo, shi);
  const int64_t sb = (int64_t)s * GRNG_LCAP;
  const float* xo = p.X + (int64_t)o * p.Dp;
  const float u2 = 1.1920928955078125e-07f;
  // thresholds at o in distance units: above ohd no node satisfies it, below old every one does
  const float ohd = p.metric == L2 ? sqrtf(fmaxf(ohi_k, 0.0f)) * (1.0f + u2) : ohi_k;
  const float old_ = p.metric == L2 ? (olo_k > 0.0f ? sqrtf(olo_k) * (1.0f - u2) : -1.0f) : olo_k;
  // ball around the G-lune (L2): centre c* = (1-lam) x + lam y, radius rho
  const float vlo = fmaxf(lo_b(v, e), 0.0f), vhi = hi_b(v, e);
  float lam = 0.5f, rho2 = -1.0f;
  if (p.metric == L2) {
    lam = fminf(fmaxf((vhi + P.t1hi - P.t2hi) / (2.0f * fmaxf(vhi, 1e-30f)), 0.0f), 1.0f);
    const float m1 = (1.0f - lam) * P.t1hi + lam * P.t2hi;
    rho2 = m1 - lam * (1.0f - lam) * vlo + 8.0f * u2 * (m1 + lam * (1.0f - lam) * vhi);
  }
  const float rho = rho2 >= 0.0f ? sqrtf(rho2) * (1.0f + u2) : -1.0f;
  const float* tab_x = p.atab ? p.atab + (int64_t)x * p.tabw + p.toff : nullptr;
  const float* tab_y = p.atab ? p.atab + (int64_t)y * p.tabw + p.toff : nullptr;
  float4 orow[NQ > 0 ? NQ : 1];
#pragma unroll
  for (int q = 0; q < NQ; ++q) orow[q] = __ldg(reinterpret_cast<const float4*>(xo) + gl + G * q);
  unsigned long long slot = 0;
  for (int pass = 0; pass < 2; ++pass) {
    if (pass == 1) {
      if (blocked || !anyamb) break;
      slot = lt_pend_slot(p, pr, lane);
    }
    // the next 64 entries' fields are loaded while the current ones are filtered and
    // tested, so that one chunk's loads overlap the previous chunk's work
    float nkk[2];
    int nkj[2], npar[2] = {0, 0};
    float ndk[2] = {0.0f, 0.0f}, nkcs[2] = {0.0f, 0.0f};
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      const int j = sp.x + lane + 32 * u;
      nkk[u] = j < sp.y ? p.lkey[sb + j] : 0.0f;
      nkj[u] = j < sp.y ? p.lidx[sb + j] : -1;
      if (p.atab && j < sp.y) {
        npar[u] = p.lpar[sb + j];
        ndk[u] = p.lpdh[sb + j];
        nkcs[u] = p.lpk[sb + j];
      }
    }
    for (int jb = sp.x; jb < sp.y; jb += 64) {
      // ---- two entries per lane: filters and bounds ----
      float kk[2];
      int kj[2];
      bool need[2];
      int stt = 0;
      int cpar[2];
      float dk[2], kcs[2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        kk[u] = nkk[u]; kj[u] = nkj[u]; cpar[u] = npar[u]; dk[u] = ndk[u]; kcs[u] = nkcs[u];
        const int j = jb + 64 + lane + 32 * u;
        nkk[u] = j < sp.y ? p.lkey[sb + j] : 0.0f;
        nkj[u] = j < sp.y ? p.lidx[sb + j] : -1;
        if (p.atab && j < sp.y) {
          npar[u] = p.lpar[sb + j];
          ndk[u] = p.lpdh[sb + j];
          nkcs[u] = p.lpk[sb + j];
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        if (kj[u] >= 0) c.read += pass == 0;
        need[u] = kj[u] >= 0 && kj[u] != o && lo_b(kk[u], e) < shi && hi_b(kk[u], e) > slo;
      }
      if (p.atab) {
        float kcx[2], kcy[2];
        const float* tab_o = sd ? tab_x : tab_y;
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          const float kco = need[u] ? tab_o[cpar[u]] : 0.0f;  // the parent's key to o
          kcx[u] = sd ? kco : kcs[u];
          kcy[u] = sd ? kcs[u] : kco;
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (!need[u]) continue;
          const float kco = sd ? kcx[u] : kcy[u];
          const float dlo_ = dist_lo(kco, p.metric, e), dhi_ = dist_hi(kco, p.metric, e);
          const float dko = dlo_ - dk[u] - u2 * (dlo_ + dk[u]);  // lower bound of d(k,o)
          if (dko >= ohd) {
            need[u] = false;  // k fails the condition at o
          } else if (rho >= 0.0f) {
            // |k - c*|^2 from k's own key to s and the lower bound of its distance to o
            const float ko2 = dko > 0.0f ? dko * dko * (1.0f - u2) : 0.0f;
            const float ks2 = fmaxf(lo_b(kk[u], e), 0.0f);
            const float Ak = sd ? ko2 : ks2, Bk = sd ? ks2 : ko2;  // lower bounds of the keys to x and y
            const float mk = (1.0f - lam) * Ak + lam * Bk + lam * (1.0f - lam) * vhi;
            const float qk = (1.0f - lam) * Ak + lam * Bk - lam * (1.0f - lam) * vhi - 8.0f * u2 * mk;
            if (qk > 0.0f && qk >= rho * rho * (1.0f + 4.0f * u2)) {
              need[u] = false;
            } else {  // the same through the parent's keys to both endpoints
              const float Alo = fmaxf(lo_b(kcx[u], e), 0.0f), Blo = fmaxf(lo_b(kcy[u], e), 0.0f);
              const float Ahi = hi_b(kcx[u], e), Bhi = hi_b(kcy[u], e);
              const float mm = (1.0f - lam) * Ahi + lam * Bhi + lam * (1.0f - lam) * vhi;
              const float qq = (1.0f - lam) * Alo + lam * Blo - lam * (1.0f - lam) * vhi - 8.0f * u2 * mm;
              const float dcs = qq > 0.0f ? sqrtf(qq) * (1.0f - u2) : 0.0f;
              if (dcs - dk[u] - u2 * (dcs + dk[u]) >= rho) need[u] = false;  // outside the lune's ball
            }
          }
          if (need[u] && old_ > 0.0f && dhi_ + dk[u] + u2 * (dhi_ + dk[u]) < old_ && hi_b(kk[u], e) < slo_k) {
            need[u] = false;  // d(k,o) < the certain threshold at o, and k certainly meets s's
            stt = 2;
          }
        }
      }
      if (pass == 0) {
        blocked = __any_sync(FULLMASK, stt == 2);
        if (blocked) break;
      }
      // ---- the unsettled entries, G lanes per distance ----
#pragma unroll 1
      for (int u = 0; u < 2; ++u) {
        unsigned nm = __ballot_sync(FULLMASK, need[u]);
        while (nm) {
          // group gi takes the gi-th remaining entry
          unsigned mm_ = nm;
          for (int t = 0; t < gi && mm_; ++t) mm_ &= mm_ - 1u;
          const int src = mm_ ? __ffs(mm_) - 1 : -1;
          for (int t = 0; t < 32 / G && nm; ++t) nm &= nm - 1u;
          const int kq = __shfl_sync(FULLMASK, kj[u], src < 0 ? 0 : src);
          const float kkq = __shfl_sync(FULLMASK, kk[u], src < 0 ? 0 : src);
          const int krow = src < 0 ? o : kq;  // a safe row to read when the group has no entry
          const float4* xk = reinterpret_cast<const float4*>(p.X + (int64_t)krow * p.Dp);
          float acc = 0.0f;
          if (NQ > 0) {
#pragma unroll
            for (int q = 0; q < (NQ > 0 ? NQ : 1); ++q) {
              const float4 a4 = __ldg(xk + gl + G * q), b4 = orow[q];
              if (p.metric == L2) {
                float d;
                d = a4.x - b4.x; acc = fmaf(d, d, acc); d = a4.y - b4.y; acc = fmaf(d, d, acc);
                d = a4.z - b4.z; acc = fmaf(d, d, acc); d = a4.w - b4.w; acc = fmaf(d, d, acc);
              } else {
                acc += fabsf(a4.x - b4.x); acc += fabsf(a4.y - b4.y); acc += fabsf(a4.z - b4.z);
                acc += fabsf(a4.w - b4.w);
              }
            }
          } else {
            const float4* x4 = reinterpret_cast<const float4*>(xo);
            for (int q = gl; q < (p.Dp >> 2); q += G) {
              const float4 a4 = __ldg(xk + q), b4 = __ldg(x4 + q);
              if (p.metric == L2) {
                float d;
                d = a4.x - b4.x; acc = fmaf(d, d, acc); d = a4.y - b4.y; acc = fmaf(d, d, acc);
                d = a4.z - b4.z; acc = fmaf(d, d, acc); d = a4.w - b4.w; acc = fmaf(d, d, acc);
              } else {
                acc += fabsf(a4.x - b4.x); acc += fabsf(a4.y - b4.y); acc += fabsf(a4.z - b4.z);
                acc += fabsf(a4.w - b4.w);
              }
            }
          }
#pragma unroll
          for (int sh = G / 2; sh > 0; sh >>= 1) acc += __shfl_xor_sync(FULLMASK, acc, sh);
          int st2 = 0;
          if (src >= 0) {
            // keys of kq to x and to y: the listed key is to s
            const float a = sd ? acc : kkq, b = sd ? kkq : acc;
            st2 = block_state(a, b, P, e);
            c.test += (gl == 0 && pass == 0);
          }
          if (pass == 0) {
            if (__any_sync(FULLMASK, st2 == 2)) { blocked = true; break; }
            anyamb |= __any_sync(FULLMASK, st2 == 1);
          } else if (st2 == 1 && gl == 0) {
            push_pair(p.amb, p.amb_cnt, p.amb_cap, make_int2((int)slot, kq));
          }
        }
        if (blocked) break;
      }
      if (pass == 0 && blocked) break;
    }
  }
}

// One warp per pair.  A pair covered from one side is scanned in that side's annulus; a
// pair covered from both sides in the shorter annulus of the two (intersecting the two
// annuli in shared-memory hash tables was measured slower: 3.02 s against 2.74 s for the
// 131,072-pivot layer at 1,000,000 points).  G lanes share one listed node in the distance
// tests (G = 8 for dimensions that are multiples of 32, fewer for 8 and 16), NQ float4
// columns per lane (0: any dimension, the other endpoint's row read from memory).
template <int G, int NQ>
__global__ void __launch_bounds__(LT_WARPS * 32, 3) list_tier_kernel(ListParams p) {
  const int lane = threadIdx.x & 31;
  const Err e = err_fp32(p.Dp);
  LtCount c;
  for (;;) {  // the next pair in the grouped order (stats[6]: the counter)
    unsigned long long tt = 0;
    if (lane == 0) tt = atomicAdd(p.stats + 6, 1ull);
    const int64_t t = (int64_t)__shfl_sync(FULLMASK, tt, 0);
    if (t >= p.m) break;
    int sd = p.side[t];
    const int2 pr = p.pairs[t];
    if (sd == 3) {
      if (lane == 0) push_pair(p.links, p.link_cnt, p.link_cap, pr);
      c.link += lane == 0;
      continue;
    }
    if (sd == 2) {
      if (lane == 0) push_pair(p.unres, p.unres_cnt, p.unres_cap, pr);
      c.un += lane == 0;
      continue;
    }
    const int x = pr.x, y = pr.y;
    const float v = key32(p.X + (int64_t)x * p.Dp, p.X + (int64_t)y * p.Dp, p.Dp, p.metric);
    const PairThr P = pair_thresholds(v, p.rlo ? p.rlo[x] : 0.0f, p.rhi ? p.rhi[x] : 0.0f,
                                      p.rlo ? p.rlo[y] : 0.0f, p.rhi ? p.rhi[y] : 0.0f, p.metric, e, p.guide);
    if (P.quick) {
      if (lane == 0) push_pair(p.links, p.link_cnt, p.link_cap, pr);
      c.link += lane == 0;
      continue;
    }
    // nodes within E of one endpoint cannot satisfy the other endpoint's condition
    const float ekx = excl_key(excl_dist(v, P.t2hi, p.metric, e), p.metric);
    const float eky = excl_key(excl_dist(v, P.t1hi, p.metric, e), p.metric);
    if (sd >= 4) {  // both lists cover: the shorter annulus, chosen with the sides
      sd -= 4;
      c.both += lane == 0;
    }
    bool blocked = false, anyamb = false;
    lt_scan<G, NQ>(p, pr, sd, v, P, ekx, eky, e, lane, c, blocked, anyamb);
    if (blocked) {
      c.blk += lane == 0;
    } else if (!anyamb) {
      if (lane == 0) push_pair(p.links, p.link_cnt, p.link_cap, pr);
      c.link += lane == 0;
    } else {
      c.pend += lane == 0;
    }
  }
  for (int sh = 16; sh > 0; sh >>= 1) {
    c.test += __shfl_down_sync(FULLMASK, c.test, sh);
    c.read += __shfl_down_sync(FULLMASK, c.read, sh);
  }
  if (lane == 0) {
    atomicAdd(p.stats + 0, c.link);
    atomicAdd(p.stats + 1, c.pend);
    atomicAdd(p.stats + 2, c.un);
    atomicAdd(p.stats + 3, c.blk);
    atomicAdd(p.stats + 4, c.test);
    atomicAdd(p.stats + 5, c.both);
    atomicAdd(p.stats + 7, c.read);
  }
}

// ---------------------------------------------------------------------------------
// FP64 recheck of ambiguous (pair, interceptor) triples, then emission.
// ---------------------------------------------------------------------------------
__global__ void recheck_kernel(const float* __restrict__ X, int D, int Dp, int metric,
                               const double* __restrict__ r64, const int2* __restrict__ amb,
                               int64_t m, const int2* __restrict__ pend, int* __restrict__ pflag,
                               unsigned long long* stats, double lam) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int2 a = amb[i];
  int2 pr = pend[a.x];
  double rx = r64 ? r64[pr.x] : 0.0, ry = r64 ? r64[pr.y] : 0.0;
  int bits = block64(X, D, Dp, metric, pr.x, pr.y, a.y, rx, ry, lam);
  if (bits) {
    atomicOr(pflag + a.x, bits);
    atomicAdd(stats, 1ull);
  }
}

// pendings -> links (definition: not blocked; guidance: not blocked with margin)
__global__ void resolve_emit_kernel(const int2* __restrict__ pend, const int* __restrict__ pflag,
                                    int64_t m, int grng, uint32_t* gx, uint32_t* gg,
                                    int64_t words, const int32_t* __restrict__ orig,
                                    unsigned long long* ecnt, unsigned long long ecap,
                                    uint64_t* edges, int2* newg, unsigned long long* newg_cnt,
                                    unsigned long long newg_cap) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int f = pflag ? pflag[i] : 0;
  int2 pr = pend[i];
  int a = min(pr.x, pr.y), b = max(pr.x, pr.y);
  if (grng) {
    if (!(f & 1)) atomicOr(gx + (int64_t)a * words + (b >> 5), 1u << (b & 31));
    if (!(f & 2)) {
      const unsigned bit = 1u << (b & 31);
      const unsigned old = atomicOr(gg + (int64_t)a * words + (b >> 5), bit);
      if (newg && !(old & bit)) {
        const unsigned long long pos = atomicAdd(newg_cnt, 1ull);
        if (pos < newg_cap) newg[pos] = make_int2(a, b);
      }
    }
  } else if (!(f & 1)) {
    int oa = orig[pr.x], ob = orig[pr.y];
    uint64_t key = ((uint64_t)(uint32_t)min(oa, ob) << 32) | (uint32_t)max(oa, ob);
    unsigned long long pos = atomicAdd(ecnt, 1ull);
    if (pos < ecap) edges[pos] = key;
  }
}

// ---------------------------------------------------------------------------------
// host orchestration of one level
// ---------------------------------------------------------------------------------
template <int KC>
static void launch_prep(const LevelIn& in, __half* A, uint8_t* ni, float* nk, cudaStream_t s) {
  int64_t nb = (in.n + GRNG_TILE - 1) / GRNG_TILE;
  size_t smem = (size_t)(2 * KC * GRNG_SSTRIDE + 128 * 129) * 4;
  if (in.metric == L2) {
    GRNG_CUDA(cudaFuncSetAttribute(block_prep_kernel<KC, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    block_prep_kernel<KC, L2><<<(unsigned)nb, GRNG_THREADS, smem, s>>>(in.X, in.n, in.Dp, A, ni, nk); note_launch();
  } else {
    GRNG_CUDA(cudaFuncSetAttribute(block_prep_kernel<KC, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    block_prep_kernel<KC, L1><<<(unsigned)nb, GRNG_THREADS, smem, s>>>(in.X, in.n, in.Dp, A, ni, nk); note_launch();
  }
  GRNG_CUDA(cudaGetLastError());
}

void block_prep(const float* X, int64_t n, int Dp, int metric, __half* A, uint8_t* nbr_idx, float* nbr_key,
                cudaStream_t s) {
  if (n < 1) return;
  LevelIn in{};
  in.X = X;
  in.n = n;
  in.Dp = Dp;
  in.metric = metric;
  const int KC = Dp % 32 == 0 ? 32 : (Dp % 16 == 0 ? 16 : 8);
  if (KC == 32) launch_prep<32>(in, A, nbr_idx, nbr_key, s);
  else if (KC == 16) launch_prep<16>(in, A, nbr_idx, nbr_key, s);
  else launch_prep<8>(in, A, nbr_idx, nbr_key, s);
}

template <int KC>
static void launch_tile(const LevelIn& in, TileParams tp, int grid, cudaStream_t s) {
  size_t smem = tp_bytes(in.K);
  if (in.metric == L2) {
    GRNG_CUDA(cudaFuncSetAttribute(tile_pass_kernel<KC, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tile_pass_kernel<KC, L2><<<grid, GRNG_THREADS, smem, s>>>(tp); note_launch();
  } else {
    GRNG_CUDA(cudaFuncSetAttribute(tile_pass_kernel<KC, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tile_pass_kernel<KC, L1><<<grid, GRNG_THREADS, smem, s>>>(tp); note_launch();
  }
  GRNG_CUDA(cudaGetLastError());
}

template <int KC>
static void launch_range_kc(const LevelIn& in, const unsigned int* tk, int* hist, const int* lastb, const int* boff,
                            int32_t* li, float* lk, int fill, cudaStream_t s, const ListAux& aux) {
  const int64_t nb = (in.n + GRNG_TILE - 1) / GRNG_TILE;
  const size_t smem = (size_t)(2 * KC * GRNG_SSTRIDE) * 4 + (size_t)GRNG_HBINS * 128 * 4 + 2 * 128 * 4;
  if (in.metric == L2) {
    GRNG_CUDA(cudaFuncSetAttribute(range_sweep_kernel<KC, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    range_sweep_kernel<KC, L2><<<(unsigned)nb, GRNG_THREADS, smem, s>>>(in.X, in.n, in.Dp, tk, hist, lastb, boff, li,
                                                                         lk, fill, aux); note_launch();
  } else {
    GRNG_CUDA(cudaFuncSetAttribute(range_sweep_kernel<KC, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    range_sweep_kernel<KC, L1><<<(unsigned)nb, GRNG_THREADS, smem, s>>>(in.X, in.n, in.Dp, tk, hist, lastb, boff, li,
                                                                         lk, fill, aux); note_launch();
  }
  GRNG_CUDA(cudaGetLastError());
}
static void launch_range(const LevelIn& in, const unsigned int* tk, int* hist, const int* lastb, const int* boff,
                         int32_t* li, float* lk, int fill, cudaStream_t s, const ListAux& aux) {
  const int KC = in.Dp % 32 == 0 ? 32 : (in.Dp % 16 == 0 ? 16 : 8);
  if (KC == 32) launch_range_kc<32>(in, tk, hist, lastb, boff, li, lk, fill, s, aux);
  else if (KC == 16) launch_range_kc<16>(in, tk, hist, lastb, boff, li, lk, fill, s, aux);
  else launch_range_kc<8>(in, tk, hist, lastb, boff, li, lk, fill, s, aux);
}

template <int G, int NQ>
static void launch_list_gq(const ListParams& lp, unsigned grid, cudaStream_t s) {
  list_tier_kernel<G, NQ><<<grid, LT_WARPS * 32, 0, s>>>(lp); note_launch();
  GRNG_CUDA(cudaGetLastError());
}
// group width and float4 columns per lane for the padded dimension (8, 16 or a multiple of 32)
static void launch_list(const ListParams& lp, unsigned grid, cudaStream_t s) {
  switch (lp.Dp) {
    case 8: launch_list_gq<2, 1>(lp, grid, s); break;
    case 16: launch_list_gq<4, 1>(lp, grid, s); break;
    case 32: launch_list_gq<8, 1>(lp, grid, s); break;
    case 64: launch_list_gq<8, 2>(lp, grid, s); break;
    case 96: launch_list_gq<8, 3>(lp, grid, s); break;
    case 128: launch_list_gq<8, 4>(lp, grid, s); break;
    default: launch_list_gq<8, 0>(lp, grid, s); break;
  }
}

static unsigned long long read_u64(const unsigned long long* d, cudaStream_t s) {
  unsigned long long h = 0;
  GRNG_CUDA(cudaMemcpyAsync(&h, d, sizeof(h), cudaMemcpyDeviceToHost, s));
  GRNG_CUDA(cudaStreamSynchronize(s));
  return h;
}

static int num_sms() {
  static int sms = 0;
  if (!sms) {
    int dev = 0;
    GRNG_CUDA(cudaGetDevice(&dev));
    GRNG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  }
  return sms;
}

// pairs[m] (and their sides) regrouped by (block of the scanned endpoint, block of the other),
// blocks of 256 or more nodes (at most 2,048 blocks), into opairs / oside
static void group_by_blocks(const int2* pairs, const int8_t* side, int64_t m, int64_t n, DevBuf& opairs,
                            DevBuf& oside, cudaStream_t s) {
  int bs = 256;
  while ((n + bs - 1) / bs > 2048) bs *= 2;
  const int64_t nbk = (n + bs - 1) / bs, nkeys = nbk * nbk;
  DevBuf cnt, off;
  GRNG_CUDA(cnt.alloc((size_t)(nkeys + 1) * 8));
  GRNG_CUDA(off.alloc((size_t)(nkeys + 1) * 8));
  GRNG_CUDA(opairs.alloc((size_t)std::max<int64_t>(m, 1) * 8));
  GRNG_CUDA(oside.alloc((size_t)std::max<int64_t>(m, 1)));
  GRNG_CUDA(cudaMemsetAsync(cnt.p, 0, (size_t)(nkeys + 1) * 8, s));
  if (m == 0) return;
  side_count_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(pairs, side, m, cnt.as<int64_t>(), bs, nbk); note_launch();
  GRNG_CUDA(cudaGetLastError());
  exclusive_scan_i64(cnt.as<int64_t>(), off.as<int64_t>(), nkeys, s);
  side_scatter_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(pairs, side, m, off.as<int64_t>(),
                                                                   opairs.as<int2>(), oside.as<int8_t>(), bs, nbk); note_launch();
  GRNG_CUDA(cudaGetLastError());
}

// Tiers 2 and 3, the FP64 recheck and the emission, for the candidate pairs surv[nsurv]
// that tier 1 (or an incremental update) leaves open.  knn_idx / knn_key / knn_rb are the
// level's neighbour lists (knn_idx null: no tier 2, every pair goes on); tier2b = false
// skips the lists of the pairs' second endpoints (when only the first ones are exact).
static void finish_level(const LevelIn& in, LevelOut& out, LevelStats& st, cudaStream_t s, const int2* surv,
                         unsigned long long nsurv, const int32_t* knn_idx, const float* knn_key,
                         const float* knn_rb, bool tier2b, unsigned long long* dc,
                         const std::function<void(int)>& tick) {
  const int64_t n = in.n;
  // ---- tiers 2 and 3 ---------------------------------------------------------------------
  DevBuf off, oth, tmp, links, unres, pend, amb, pflag, unres2, off2, oth2, fbuf;
  DevBuf side, tkey, tcut, hist, lcnt, lastb, boff, lidx, lkey, lpar, lpdh, lpk, unres3, atab;
  int64_t toff[GRNG_MAXL] = {0}, tabw = 0;  // columns of the node x ancestor key table
  if (knn_idx) {
    GRNG_CUDA(off.alloc((size_t)(n + 1) * 8));
    GRNG_CUDA(oth.alloc(std::max<size_t>(nsurv, 1) * 4));
    group_pairs(surv, (int64_t)nsurv, 0, n, off.as<int64_t>(), oth.as<int32_t>(), tmp, s);
  }
  unsigned long long cap = std::max<unsigned long long>(nsurv, 1024);
  unsigned long long amb_cap = in.small_buffers ? 8ull : std::max<unsigned long long>(4 * nsurv, 1 << 20);
  for (int attempt = 0;; ++attempt) {
    st.c[31] = attempt + 1;  // passes of tiers 2-3 (an ambiguity buffer overflow repeats them)
    GRNG_CUDA(links.alloc(cap * 8));
    GRNG_CUDA(unres.alloc(cap * 8));
    GRNG_CUDA(pend.alloc(cap * 8 * 2));
    GRNG_CUDA(amb.alloc(amb_cap * 8));
    GRNG_CUDA(cudaMemsetAsync(dc + 8, 0, 16 * sizeof(unsigned long long), s));
    Tier2Params t2;
    t2.X = in.X; t2.n = n; t2.Dp = in.Dp; t2.metric = in.metric; t2.guide = in.grng; t2.K = in.K;
    t2.lam = (float)in.beta_lam;
    t2.rlo = in.rlo; t2.rhi = in.rhi; t2.knn_idx = knn_idx; t2.knn_key = knn_key;
    t2.knn_rb = knn_rb;
    t2.off = off.as<int64_t>(); t2.other = oth.as<int32_t>();
    t2.links = links.as<int2>(); t2.link_cnt = dc + 16; t2.link_cap = cap;
    t2.unres = unres.as<int2>(); t2.unres_cnt = dc + 18; t2.unres_cap = cap;
    t2.pend = pend.as<int2>(); t2.pend_cnt = dc + 17; t2.pend_cap = 2 * cap;
    t2.amb = amb.as<int2>(); t2.amb_cnt = dc + 19; t2.amb_cap = amb_cap;
    t2.stats = dc + 8;
    size_t smem2 = (size_t)(in.Dp * 32 + in.Dp + 4 * in.Dp) * 4;
    int grid2 = (int)std::min<int64_t>(n, 32 * num_sms());
    unsigned long long nun = nsurv;
    if (knn_idx) {
      if (nsurv) {
        tier2_kernel<<<grid2, 128, smem2, s>>>(t2); note_launch();
        GRNG_CUDA(cudaGetLastError());
      }
      nun = read_u64(dc + 18, s);
    } else if (nsurv) {  // no neighbour lists: every pair goes on
      GRNG_CUDA(cudaMemcpyAsync(unres.p, surv, (size_t)nsurv * sizeof(int2), cudaMemcpyDeviceToDevice, s));
    }
    tick(2);
    // tier 2b: the other endpoint's neighbours
    GRNG_CUDA(unres2.alloc(std::max<unsigned long long>(nun, 1) * 8));
    unsigned long long nun2 = nun;
    if (knn_idx && tier2b) {
      GRNG_CUDA(off2.alloc((size_t)(n + 1) * 8));
      GRNG_CUDA(oth2.alloc(std::max<unsigned long long>(nun, 1) * 4));
      group_pairs(unres.as<int2>(), (int64_t)std::min(nun, cap), 1, n, off2.as<int64_t>(),
                  oth2.as<int32_t>(), tmp, s);
      t2.off = off2.as<int64_t>(); t2.other = oth2.as<int32_t>();
      t2.unres = unres2.as<int2>(); t2.unres_cnt = dc + 20; t2.unres_cap = std::max<unsigned long long>(nun, 1);
      t2.stats = dc + 12;
      if (nun) {
        tier2_kernel<<<grid2, 128, smem2, s>>>(t2); note_launch();
        GRNG_CUDA(cudaGetLastError());
      }
      nun2 = read_u64(dc + 20, s);
    } else if (nun) {
      GRNG_CUDA(cudaMemcpyAsync(unres2.p, unres.p, (size_t)nun * sizeof(int2), cudaMemcpyDeviceToDevice, s));
    }
    tick(3);
    const int2* t3pairs = unres2.as<int2>();
    GRNG_CUDA(cudaMemsetAsync(dc + 26, 0, 8 * sizeof(unsigned long long), s));
    GRNG_CUDA(cudaMemsetAsync(dc + 50, 0, 8 * sizeof(unsigned long long), s));
    if (in.grng && in.anc.n > 0 && nun2 && !atab.p) {
      // pivot layers: node x ancestor keys once (the list tier's bounds and tier 3)
      tabw = 0;  // each level's columns start on a 16-byte boundary
      for (int a = 0; a < in.anc.n; ++a) { toff[a] = tabw; tabw += (in.anc.m[a] + 3) & ~(int64_t)3; }
      GRNG_CUDA(atab.alloc((size_t)n * tabw * 4));
      for (int a = 0; a < in.anc.n; ++a)
        launch_cross(in.X, n, in.anc.X[a], in.anc.m[a], in.Dp, in.metric, atab.as<float>() + toff[a], tabw, s);
    }
    DevBuf prest, pkept;
    bool probed = false;  // the descents ran: tier 3 does not repeat them
    if (in.grng && in.lists && nun2 && atab.p && in.metric == L2) {
      // warp-per-pair descents towards the ball around each G-lune first: a pair a node
      // certainly blocks is dropped before the range lists are sized and scanned
      bool dense = true;
      for (int a = 1; a < in.anc.n; ++a) dense &= in.anc.m[a] <= 32 * T3_MKW;
      if (dense) {
        {  // in (block of x, block of y) order, so that the warps at work share ancestor-table rows
          DevBuf zside, gpairs, gside;
          GRNG_CUDA(zside.alloc(nun2));
          GRNG_CUDA(cudaMemsetAsync(zside.p, 0, nun2, s));
          group_by_blocks(unres2.as<int2>(), zside.as<int8_t>(), (int64_t)nun2, n, gpairs, gside, s);
          std::swap(unres2, gpairs);
        }
        Tier3Params pp{};
        pp.X = in.X; pp.n = n; pp.npts = in.npts ? in.npts : n; pp.Dp = in.Dp; pp.metric = in.metric;
        pp.guide = in.grng;
        pp.lam = (float)in.beta_lam;
        pp.rlo = in.rlo; pp.rhi = in.rhi; pp.pairs = unres2.as<int2>(); pp.m = (int64_t)nun2;
        pp.anc = in.anc;
        for (int a = 0; a < in.anc.n; ++a) pp.anc.toff[a] = toff[a];
        pp.atab = atab.as<float>(); pp.tabw = tabw; pp.dense = 1;
        GRNG_CUDA(prest.alloc((size_t)nun2 * 4));
        GRNG_CUDA(cudaMemsetAsync(dc + 62, 0, 2 * sizeof(unsigned long long), s));
        GRNG_CUDA(cudaMemsetAsync(dc + 24, 0, sizeof(unsigned long long), s));
        const unsigned gp = (unsigned)std::min<unsigned long long>((nun2 + T3P_WARPS - 1) / T3P_WARPS,
                                                                   (unsigned long long)8 * num_sms());
        tier3_probe_kernel<<<gp, T3P_WARPS * 32, (size_t)T3P_WARPS * 2 * in.Dp * 4, s>>>(
            pp, prest.as<int32_t>(), dc + 62, dc + 63, dc + 24); note_launch();
        GRNG_CUDA(cudaGetLastError());
        unsigned long long hr[2];
        GRNG_CUDA(cudaMemcpyAsync(hr, dc + 62, sizeof(hr), cudaMemcpyDeviceToHost, s));
        GRNG_CUDA(cudaStreamSynchronize(s));
        st.c[41] = hr[1];  // pairs the descents block before the range lists
        GRNG_CUDA(pkept.alloc(std::max<unsigned long long>(hr[0], 1) * 8));
        if (hr[0])
          gather_pairs_kernel<<<(unsigned)((hr[0] + 255) / 256), 256, 0, s>>>(
              unres2.as<int2>(), prest.as<int32_t>(), (int64_t)hr[0], pkept.as<int2>()); note_launch();
        GRNG_CUDA(cudaGetLastError());
        std::swap(unres2, pkept);
        nun2 = hr[0];
        probed = true;
        t3pairs = unres2.as<int2>();
      }
    }
    if (in.grng && in.lists && nun2) {
      // range lists for the pairs no neighbour list covers
      GRNG_CUDA(side.alloc(nun2));
      GRNG_CUDA(tkey.alloc((size_t)n * 4));
      GRNG_CUDA(tcut.alloc((size_t)n * 4));
      GRNG_CUDA(hist.alloc((size_t)n * GRNG_HBINS * 4));
      GRNG_CUDA(lcnt.alloc((size_t)n * 4));
      GRNG_CUDA(lastb.alloc((size_t)n * 4));
      GRNG_CUDA(boff.alloc((size_t)n * (GRNG_HBINS + 1) * 4));
      GRNG_CUDA(cudaMemsetAsync(tkey.p, 0, (size_t)n * 4, s));
      SideParams sp{};
      sp.X = in.X; sp.Dp = in.Dp; sp.metric = in.metric; sp.guide = in.grng; sp.K = in.K;
      sp.rlo = in.rlo; sp.rhi = in.rhi; sp.pairs = unres2.as<int2>(); sp.m = (int64_t)nun2;
      sp.side = side.as<int8_t>(); sp.tkey = tkey.as<unsigned int>(); sp.tcut = tcut.as<unsigned int>();
      sp.lcnt = lcnt.as<int>();
      cudaEvent_t l0, l1;
      GRNG_CUDA(cudaEventCreate(&l0));
      GRNG_CUDA(cudaEventCreate(&l1));
      GRNG_CUDA(cudaEventRecord(l0, s));
      range_thresholds_kernel<<<(unsigned)((nun2 + 255) / 256), 256, 0, s>>>(sp); note_launch();
      GRNG_CUDA(cudaGetLastError());
      launch_range(in, tkey.as<unsigned int>(), hist.as<int>(), nullptr, nullptr, nullptr, nullptr, 0, s, ListAux());
      const int lmax = in.lmax > 0 ? (int)std::min<int64_t>(in.lmax, GRNG_LCAP) : GRNG_LMAX;
      range_cut_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(tkey.as<unsigned int>(), hist.as<int>(), n,
                                                                  tcut.as<unsigned int>(), lastb.as<int>(),
                                                                  boff.as<int>(), lcnt.as<int>(), lmax); note_launch();
      GRNG_CUDA(cudaGetLastError());
      GRNG_CUDA(lidx.alloc((size_t)n * GRNG_LCAP * 4));
      GRNG_CUDA(lkey.alloc((size_t)n * GRNG_LCAP * 4));
      ListAux aux;
      if (atab.p && in.parent && in.pdist_hi) {
        GRNG_CUDA(lpar.alloc((size_t)n * GRNG_LCAP * 4));
        GRNG_CUDA(lpdh.alloc((size_t)n * GRNG_LCAP * 4));
        GRNG_CUDA(lpk.alloc((size_t)n * GRNG_LCAP * 4));
        aux.parent = in.parent;
        aux.pdist = in.pdist_hi;
        aux.atab = atab.as<float>();
        aux.tabw = tabw;
        aux.toff = toff[in.anc.n - 1];
        aux.par = lpar.as<int32_t>();
        aux.pdh = lpdh.as<float>();
        aux.pkey = lpk.as<float>();
      }
      launch_range(in, tkey.as<unsigned int>(), nullptr, lastb.as<int>(), boff.as<int>(), lidx.as<int32_t>(),
                   lkey.as<float>(), 1, s, aux);
      sp.lastb = lastb.as<int>();
      sp.boff = boff.as<int>();
      pick_side_kernel<<<(unsigned)((nun2 + 255) / 256), 256, 0, s>>>(sp); note_launch();
      GRNG_CUDA(cudaGetLastError());
      // the pairs grouped by the endpoint whose list they scan
      DevBuf spairs, sside;
      group_by_blocks(unres2.as<int2>(), side.as<int8_t>(), (int64_t)nun2, n, spairs, sside, s);
      GRNG_CUDA(unres3.alloc(nun2 * 8));
      ListParams lp;
      lp.X = in.X; lp.Dp = in.Dp; lp.metric = in.metric; lp.guide = in.grng; lp.rlo = in.rlo; lp.rhi = in.rhi;
      lp.pairs = spairs.as<int2>(); lp.m = (int64_t)nun2; lp.side = sside.as<int8_t>();
      lp.tkey = tkey.as<unsigned int>(); lp.lastb = lastb.as<int>(); lp.boff = boff.as<int>();
      lp.lidx = lidx.as<int32_t>(); lp.lkey = lkey.as<float>();
      lp.atab = aux.par ? atab.as<float>() : nullptr;  // the bounds need the per-entry fields
      lp.tabw = tabw;
      lp.toff = in.anc.n > 0 ? toff[in.anc.n - 1] : 0;
      lp.lpar = lpar.as<int32_t>();
      lp.lpdh = lpdh.as<float>();
      lp.lpk = lpk.as<float>();
      lp.links = links.as<int2>(); lp.link_cnt = dc + 16; lp.link_cap = cap;
      lp.unres = unres3.as<int2>(); lp.unres_cnt = dc + 27; lp.unres_cap = nun2;
      lp.pend = pend.as<int2>(); lp.pend_cnt = dc + 17; lp.pend_cap = 2 * cap;
      lp.amb = amb.as<int2>(); lp.amb_cnt = dc + 19; lp.amb_cap = amb_cap;
      lp.stats = dc + 50;
      cudaEvent_t k0;
      GRNG_CUDA(cudaEventCreate(&k0));
      GRNG_CUDA(cudaEventRecord(k0, s));
      launch_list(lp, (unsigned)std::min<unsigned long long>((nun2 + LT_WARPS - 1) / LT_WARPS,
                                                             (unsigned long long)3 * num_sms()), s);
      GRNG_CUDA(cudaEventRecord(l1, s));
      GRNG_CUDA(cudaEventSynchronize(l1));
      float lms = 0.0f, kms = 0.0f;
      GRNG_CUDA(cudaEventElapsedTime(&lms, l0, l1));
      GRNG_CUDA(cudaEventElapsedTime(&kms, k0, l1));
      cudaEventDestroy(l0);
      cudaEventDestroy(l1);
      cudaEventDestroy(k0);
      st.kms[2] += kms;   // the list tier kernel
      st.kms[3] += lms;   // thresholds, both sweeps, cut, sides and the list tier
      unsigned long long h8[8];  // links, pending, to tier 3, blocked, tested by distance, intersections, probes
      GRNG_CUDA(cudaMemcpyAsync(h8, dc + 50, sizeof(h8), cudaMemcpyDeviceToHost, s));
      unsigned long long n3 = 0;
      GRNG_CUDA(cudaMemcpyAsync(&n3, dc + 27, sizeof(n3), cudaMemcpyDeviceToHost, s));
      std::vector<int> hl((size_t)n), hlb((size_t)n);
      std::vector<unsigned int> htk((size_t)n);
      GRNG_CUDA(cudaMemcpyAsync(hl.data(), lcnt.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
      GRNG_CUDA(cudaMemcpyAsync(hlb.data(), lastb.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
      GRNG_CUDA(cudaMemcpyAsync(htk.data(), tkey.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
      GRNG_CUDA(cudaStreamSynchronize(s));
      unsigned long long ltot = 0, lcut = 0;
      for (size_t i = 0; i < hl.size(); ++i) {
        ltot += (unsigned long long)hl[i];
        lcut += htk[i] != 0 && hlb[i] < GRNG_HBINS - 1;
      }
      st.c[18] = nun2;    // pairs given range lists
      st.c[19] = lcut;    // lists cut below their T_s
      st.c[20] = ltot;    // listed nodes
      st.c[21] = h8[0];   // links from the lists
      st.c[22] = h8[4];   // listed nodes tested by distance
      st.c[32] = h8[5];   // pairs covered from both sides
      st.c[33] = 0;
      st.c[34] = h8[7];   // list entries read
      nun2 = n3;          // left for tier 3
      t3pairs = unres3.as<int2>();
    }
    tick(4);
    unsigned long long npend = read_u64(dc + 17, s);
    unsigned long long nlink = read_u64(dc + 16, s);
    if (npend + nun2 > 2 * cap || nlink > cap || nun > cap) fail(6, "tier-2 buffer overflow");
    // tier 3 appends its pairs after the tier-2 pendings
    GRNG_CUDA(pflag.alloc((size_t)std::max<unsigned long long>(npend + nun2, 1) * 4));
    GRNG_CUDA(cudaMemsetAsync(pflag.p, 0, (size_t)std::max<unsigned long long>(npend + nun2, 1) * 4, s));
    if (nun2) {
      Tier3Params t3;
      t3.X = in.X; t3.n = n; t3.npts = in.npts ? in.npts : n; t3.Dp = in.Dp; t3.metric = in.metric;
      t3.guide = in.grng;
      t3.lam = (float)in.beta_lam;
      t3.rlo = in.rlo; t3.rhi = in.rhi; t3.pairs = t3pairs; t3.m = (int64_t)nun2;
      t3.pend = pend.as<int2>(); t3.pflag = pflag.as<int>(); t3.slot0 = (int64_t)npend;
      t3.amb = amb.as<int2>(); t3.amb_cnt = dc + 19; t3.amb_cap = amb_cap;
      t3.anc = in.anc;
      int grid3 = (int)std::min<unsigned long long>(nun2, (unsigned long long)T3_MINB * num_sms());
      t3.fcap = in.small_buffers ? 4 : 1 << 15;
      GRNG_CUDA(fbuf.alloc((size_t)grid3 * 2 * t3.fcap * sizeof(Front)));
      t3.fbuf = fbuf.as<Front>();
      t3.pdist_hi = in.pdist_hi;
      t3.atab = nullptr;
      t3.tabw = 0;
      t3.dense = 0;
      t3.mkw = 0;
      if (in.grng && in.anc.n > 0 && atab.p) {
        // pivot layers: the node x ancestor keys computed before the list tier
        for (int a = 0; a < in.anc.n; ++a) t3.anc.toff[a] = toff[a];
        t3.atab = atab.as<float>();
        t3.tabw = tabw;
        t3.dense = 1;
        for (int a = 1; a < in.anc.n; ++a) {
          t3.dense &= in.anc.m[a] <= 32 * T3_MKW;
          t3.mkw = std::max<int>(t3.mkw, (int)((in.anc.m[a] + 31) / 32));
        }
        if (!t3.dense) t3.mkw = 0;
      }
      t3.stats = dc + 34;
      t3.prof = dc + 58;
      GRNG_CUDA(cudaMemsetAsync(dc + 34, 0, 4 * sizeof(unsigned long long), s));
      GRNG_CUDA(cudaMemsetAsync(dc + 58, 0, 4 * sizeof(unsigned long long), s));
      if (!in.grng && knn_idx && tier2b && ((in.mlp_params && in.kshort > 0) || (in.mlp_record && out.rec_f))) {
        // learned shortlist (extension of Stage V): k scored candidates per pair first
        MlpStage ms;
        ms.X = in.X; ms.n = n; ms.Dp = in.Dp; ms.metric = in.metric; ms.K = in.K;
        ms.knn_idx = knn_idx; ms.knn_key = knn_key;
        ms.parent = in.parent; ms.pdist_hi = in.pdist_hi;
        ms.prad = in.anc.n ? in.anc.Rhi[in.anc.n - 1] : nullptr;
        ms.pairs = t3pairs; ms.m = (int64_t)nun2; ms.slot0 = (int64_t)npend; ms.pflag = pflag.as<int>();
        ms.amb = amb.as<int2>(); ms.amb_cnt = dc + 19; ms.amb_cap = amb_cap;
        ms.params = in.kshort > 0 ? in.mlp_params : nullptr;
        ms.kshort = in.kshort;
        ms.rec_f = nullptr; ms.rec_y = nullptr; ms.rec_cnt = dc + 47; ms.rec_cap = 0;
        if (in.mlp_record && out.rec_f) {
          const unsigned long long rc = std::min<unsigned long long>(
              nun2 * 2ull * GRNG_MLP_PW * in.K, 4ull << 20);
          GRNG_CUDA(out.rec_f->alloc((size_t)rc * GRNG_MLP_IN * 4));
          GRNG_CUDA(out.rec_y->alloc((size_t)rc * 4));
          ms.rec_f = out.rec_f->as<float>(); ms.rec_y = out.rec_y->as<float>(); ms.rec_cap = rc;
        }
        ms.stats = dc + 44;
        GRNG_CUDA(cudaMemsetAsync(dc + 44, 0, 5 * sizeof(unsigned long long), s));
        mlp_stage(ms, s);
        unsigned long long hm[5];
        GRNG_CUDA(cudaMemcpyAsync(hm, dc + 44, sizeof(hm), cudaMemcpyDeviceToHost, s));
        GRNG_CUDA(cudaStreamSynchronize(s));
        st.c[25] = ms.params ? nun2 : 0;  // pairs given a shortlist
        st.c[26] = hm[0];                 // candidates scored
        st.c[27] = hm[1];                 // shortlist tests
        st.c[28] = hm[2];                 // pairs blocked by the shortlist
        st.c[29] = hm[4];                 // recording: pairs with a blocker among the candidates
        if (ms.rec_f) out.rec_n = (int64_t)std::min<unsigned long long>(hm[3], ms.rec_cap);
      }
      cudaEvent_t f0, f1;
      GRNG_CUDA(cudaEventCreate(&f0));
      GRNG_CUDA(cudaEventCreate(&f1));
      GRNG_CUDA(cudaEventRecord(f0, s));
      DevBuf rest;
      t3.idx = nullptr;
      if (t3.dense && in.metric == L2 && in.anc.n > 0 && !probed) {
        // warp-per-pair descents first; the exhaustive tier takes the pairs they leave
        GRNG_CUDA(rest.alloc((size_t)nun2 * 4));
        GRNG_CUDA(cudaMemsetAsync(dc + 62, 0, 2 * sizeof(unsigned long long), s));
        GRNG_CUDA(cudaMemsetAsync(dc + 24, 0, sizeof(unsigned long long), s));
        const unsigned gp = (unsigned)std::min<unsigned long long>((nun2 + T3P_WARPS - 1) / T3P_WARPS,
                                                                   (unsigned long long)8 * num_sms());
        tier3_probe_kernel<<<gp, T3P_WARPS * 32, (size_t)T3P_WARPS * 2 * in.Dp * 4, s>>>(
            t3, rest.as<int32_t>(), dc + 62, dc + 63, dc + 24); note_launch();
        GRNG_CUDA(cudaGetLastError());
        unsigned long long hr[2];
        GRNG_CUDA(cudaMemcpyAsync(hr, dc + 62, sizeof(hr), cudaMemcpyDeviceToHost, s));
        GRNG_CUDA(cudaStreamSynchronize(s));
        st.c[39] = hr[1];  // pairs the probe descents block
        t3.idx = rest.as<int32_t>();
        t3.m = (int64_t)hr[0];
      }
      if (t3.m) {
        tier3_kernel<<<grid3, T3_T, 2 * in.Dp * 4 + 2 * (size_t)t3.mkw * 4, s>>>(t3); note_launch();
      }
      GRNG_CUDA(cudaGetLastError());
      GRNG_CUDA(cudaEventRecord(f1, s));
      GRNG_CUDA(cudaEventSynchronize(f1));
      float fms = 0.0f;
      GRNG_CUDA(cudaEventElapsedTime(&fms, f0, f1));
      cudaEventDestroy(f0);
      cudaEventDestroy(f1);
      st.kms[1] += fms;
    }
    unsigned long long namb = read_u64(dc + 19, s);
    tick(5);
    if (namb > amb_cap) {
      if (attempt >= 3) fail(2, "ambiguity buffer overflow");
      amb_cap = namb + namb / 4;
      continue;
    }
    if (namb) {
      recheck_kernel<<<(unsigned)((namb + 255) / 256), 256, 0, s>>>(
          in.X, in.D, in.Dp, in.metric, in.r64, amb.as<int2>(), (int64_t)namb, pend.as<int2>(),
          pflag.as<int>(), dc + 22, in.beta_lam); note_launch();
      GRNG_CUDA(cudaGetLastError());
    }
    // ---- emission ----------------------------------------------------------------------
    const unsigned long long npp = npend + nun2;
    unsigned long long ecap = nlink + npp + 1;
    if (!in.grng) {
      GRNG_CUDA(out.edges->alloc(ecap * 8));
    }
    int2* newg = nullptr;
    unsigned long long newg_cap = 0;
    if (in.grng && out.new_gg) {  // pairs whose guidance bit this pass sets (incremental updates)
      newg_cap = nlink + npp + 1;
      GRNG_CUDA(out.new_gg->alloc(newg_cap * sizeof(int2)));
      newg = out.new_gg->as<int2>();
    }
    if (nlink)
      resolve_emit_kernel<<<(unsigned)((nlink + 255) / 256), 256, 0, s>>>(
          links.as<int2>(), nullptr, (int64_t)nlink, in.grng, out.gx, out.gg, out.words, in.orig,
          dc + 21, ecap, in.grng ? nullptr : out.edges->as<uint64_t>(), newg, dc + 23, newg_cap); note_launch();
    if (npp)
      resolve_emit_kernel<<<(unsigned)((npp + 255) / 256), 256, 0, s>>>(
          pend.as<int2>(), pflag.as<int>(), (int64_t)npp, in.grng, out.gx, out.gg, out.words,
          in.orig, dc + 21, ecap, in.grng ? nullptr : out.edges->as<uint64_t>(), newg, dc + 23, newg_cap); note_launch();
    GRNG_CUDA(cudaGetLastError());
    unsigned long long h[40];
    GRNG_CUDA(cudaMemcpyAsync(h, dc, sizeof(h), cudaMemcpyDeviceToHost, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    {
      unsigned long long hp[4] = {0, 0, 0, 0};
      if (nun2) GRNG_CUDA(cudaMemcpyAsync(hp, dc + 58, sizeof(hp), cudaMemcpyDeviceToHost, s));
      GRNG_CUDA(cudaStreamSynchronize(s));
      st.c[35] = hp[0];  // tier-3 cycles: top level and descents
      st.c[36] = hp[1];  //   lower ancestor levels
      st.c[37] = hp[2];  //   node level
      st.c[38] = hp[3];  // tier-3 pairs reaching the lower ancestor levels
    }
    st.c[15] = nun2 ? h[34] : 0;  // tier-3 frontier overflows
    st.c[16] = nun2 ? h[35] : 0;  // tier-3 nodes tested
    st.c[23] = nun2 ? h[36] : 0;  // tier-3 pairs blocked
    st.c[24] = nun2 ? h[37] : 0;  // of which by the greedy descent
    out.n_edges = (int64_t)h[21];
    out.n_new_gg = newg ? (int64_t)std::min<unsigned long long>(h[23], newg_cap) : 0;
    st.c[3] = h[8];  st.c[4] = h[9];  st.c[5] = h[10]; st.c[6] = h[11];   // tier 2a
    st.c[7] = h[12]; st.c[8] = h[13]; st.c[9] = h[14]; st.c[10] = h[15];  // tier 2b
    st.c[11] = nun2;   // tier-3 pairs
    st.c[12] = namb;   // ambiguous triples rechecked in FP64
    st.c[13] = h[22];  // of which blocking
    st.c[14] = h[21];  // edges emitted (RNG level)
    tick(6);
    break;
  }
}

void run_level(const LevelIn& in, LevelOut& out, LevelStats& st, cudaStream_t s, float* tile_ms) {
  memset(&st, 0, sizeof(st));
  auto t_last = std::chrono::steady_clock::now();
  std::function<void(int)> tick = [&](int slot) {  // host time of one phase (each ends in a synchronisation)
    GRNG_CUDA(cudaStreamSynchronize(s));
    auto now = std::chrono::steady_clock::now();
    st.ms[slot] += std::chrono::duration<double, std::milli>(now - t_last).count();
    t_last = now;
  };
  const int64_t n = in.n;
  if (n < 2) {
    out.n_edges = 0;
    return;
  }
  if (in.K < 1 || in.K > GRNG_KMAX) fail(1, "neighbour-list length must be in [1, 32]");
  const int64_t nb = (n + GRNG_TILE - 1) / GRNG_TILE;
  const int KC = in.Dp % 32 == 0 ? 32 : (in.Dp % 16 == 0 ? 16 : 8);
  if (in.Dp % 8 != 0) fail(6, "padded dimension must be a multiple of 8");

  DevBuf A, nbi, nbk, knni, knnk, ctr;
  GRNG_CUDA(A.alloc((size_t)nb * GRNG_TILE * GRNG_TILE * sizeof(__half)));
  GRNG_CUDA(nbi.alloc((size_t)nb * GRNG_TILE * GRNG_KIN));
  GRNG_CUDA(nbk.alloc((size_t)nb * GRNG_TILE * GRNG_KIN * 4));
  GRNG_CUDA(knni.alloc((size_t)n * in.K * 4));
  GRNG_CUDA(knnk.alloc((size_t)n * in.K * 4));
  GRNG_CUDA(ctr.alloc(64 * sizeof(unsigned long long)));
  unsigned long long* dc = ctr.as<unsigned long long>();
  // counters: 0 strip, 1 surv, 2..5 tile stats, 8.. tier2a, 12.. tier2b, 16 links, 17 pend,
  // 18 unres, 19 amb, 20 unres2, 21 edges, 22 recheck blocked, 23 new guidance links, 24 the
  // descents' pair counter, 26..33 range lists, 34..37 tier 3, 40 tensor-core status, 44..48
  // learned shortlist, 50..57 list tier, 58..61 tier-3 cycles, 62..63 descents
  if (KC == 32) launch_prep<32>(in, A.as<__half>(), nbi.as<uint8_t>(), nbk.as<float>(), s);
  else if (KC == 16) launch_prep<16>(in, A.as<__half>(), nbi.as<uint8_t>(), nbk.as<float>(), s);
  else launch_prep<8>(in, A.as<__half>(), nbi.as<uint8_t>(), nbk.as<float>(), s);

  tick(0);
  // ---- tier 1 -------------------------------------------------------------------------
  // survivors per node: about 160 at the exemplar level of the 1M-point workloads, about
  // 1,500 at its finest pivot layer (the overflow path repeats only the filter sweep)
  unsigned long long surv_cap =
      in.small_buffers ? 64ull
                       : (unsigned long long)std::max<int64_t>(1 << 20, std::min<int64_t>((in.grng ? 2048 : 256) * n,
                                                                                          n * (n - 1) / 2 + 1));
  const bool use_tc = !in.grng && in.precision == 1 && in.metric == L2 && tc_supported(in.Dp);
  DevBuf tcimg, tcnrm, tcbmax, knnrb;
  float nmax_all = 0.0f;
  if (use_tc) {
    tc_prepare(in.X, n, in.Dp, tcimg, tcnrm, tcbmax, &nmax_all, s);
    GRNG_CUDA(knnrb.alloc((size_t)n * 4));
  }
  DevBuf surv;
  unsigned long long nsurv = 0;
  for (int attempt = 0;; ++attempt) {
    GRNG_CUDA(surv.alloc(surv_cap * sizeof(int2)));
    GRNG_CUDA(cudaMemsetAsync(dc, 0, 64 * sizeof(unsigned long long), s));
    if (in.grng && out.gx) {
      fill_u32(out.gx, 0u, (size_t)n * out.words, s);
      fill_u32(out.gg, 0u, (size_t)n * out.words, s);
    }
    TileParams tp;
    tp.X = in.X; tp.n = n; tp.Dp = in.Dp; tp.grng = in.grng; tp.guide = in.grng; tp.K = in.K;
    tp.lam = (float)in.beta_lam;
    tp.parent = in.parent; tp.gpar = in.gpar; tp.gpar_words = in.gpar_words;
    tp.rlo = in.rlo; tp.rhi = in.rhi; tp.A = A.as<__half>(); tp.nbr_idx = nbi.as<uint8_t>();
    tp.nbr_key = nbk.as<float>(); tp.knn_idx = knni.as<int32_t>(); tp.knn_key = knnk.as<float>();
    tp.surv = surv.as<int2>(); tp.surv_cnt = dc + 1; tp.surv_cap = surv_cap;
    tp.gx = out.gx; tp.gg = out.gg; tp.words = out.words;
    tp.strip_ctr = reinterpret_cast<int*>(dc + 0); tp.stats = dc + 2;
    int grid = (int)std::min<int64_t>(nb, num_sms());
    cudaEvent_t e0, e1;
    GRNG_CUDA(cudaEventCreate(&e0));
    GRNG_CUDA(cudaEventCreate(&e1));
    GRNG_CUDA(cudaEventRecord(e0, s));
    // pivot layers: a first sweep for the neighbour lists, then the filter, which can
    // certify links from the final lists; exemplars: one sweep doing both
    tp.mode = in.grng ? 1 : 0;
    if (use_tc) {
      // precision form: tensor-core Gram tiles, then the listed keys again in FP32
      TcLaunch L;
      L.img = tcimg.as<uint8_t>(); L.nrm = tcnrm.as<float>(); L.bmax = tcbmax.as<unsigned int>();
      L.n = n; L.Dp = in.Dp; L.K = in.K; L.nmax_all = nmax_all;
      L.parent = in.parent; L.gpar = in.gpar; L.gpar_words = in.gpar_words;
      L.A = A.as<__half>(); L.nbr_idx = nbi.as<uint8_t>(); L.nbr_key = nbk.as<float>();
      L.knn_idx = knni.as<int32_t>(); L.knn_key = knnk.as<float>(); L.knn_rb = knnrb.as<float>();
      L.surv = surv.as<int2>(); L.surv_cnt = dc + 1; L.surv_cap = surv_cap;
      L.strip_ctr = reinterpret_cast<int*>(dc + 0); L.stats = dc + 2;
      L.status = reinterpret_cast<int*>(dc + 40); L.spin = in.spin;
      tc_sweep(L, s);
    } else {
      // pivot layers: the lists of the first sweep are final, so a repeat after a survivor
      // buffer overflow runs the filter sweep alone
      for (int sweep = (in.grng && attempt > 0) ? 1 : 0; sweep < (in.grng ? 2 : 1); ++sweep) {
        if (sweep == 1) {
          GRNG_CUDA(cudaMemsetAsync(dc, 0, sizeof(unsigned long long), s));  // strip counter
          tp.mode = 2;
        }
        if (KC == 32) launch_tile<32>(in, tp, grid, s);
        else if (KC == 16) launch_tile<16>(in, tp, grid, s);
        else launch_tile<8>(in, tp, grid, s);
      }
    }
    {
      GRNG_CUDA(cudaEventRecord(e1, s));
      GRNG_CUDA(cudaEventSynchronize(e1));
      float ems = 0.0f;
      GRNG_CUDA(cudaEventElapsedTime(&ems, e0, e1));
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
      if (tile_ms) *tile_ms = ems;
      st.kms[0] = ems;
    }
    nsurv = read_u64(dc + 1, s);
    st.c[30] = attempt + 1;  // tier-1 sweeps run (a survivor buffer overflow repeats the sweep)
    if (use_tc) {
      if (read_u64(dc + 40, s) != 0) fail(4 /* GRNG_ETIMEOUT */, "a bounded tensor-core wait ran out");
      if (nsurv <= surv_cap) tc_knn_fix(in.X, n, in.Dp, in.K, in.metric, knni.as<int32_t>(), knnk.as<float>(), s);
    }
    if (nsurv <= surv_cap) break;
    if (attempt >= 3) fail(2, "tier-1 survivor buffer overflow");
    surv_cap = nsurv + nsurv / 4;
  }
  unsigned long long hst[4];
  GRNG_CUDA(cudaMemcpyAsync(hst, dc + 2, sizeof(hst), cudaMemcpyDeviceToHost, s));
  GRNG_CUDA(cudaStreamSynchronize(s));
  st.c[0] = hst[0];  // candidate pairs
  st.c[1] = hst[1];  // quick links
  st.c[2] = nsurv;
  st.c[17] = hst[2];  // links certified from the neighbour lists in the tile
  st.c[40] = use_tc ? hst[3] : 0;  // pairs the tensor-core sweep's quick test left to the full filter

  tick(1);
  finish_level(in, out, st, s, surv.as<int2>(), nsurv, knni.as<int32_t>(), knnk.as<float>(),
               use_tc ? knnrb.as<float>() : nullptr, true, dc, tick);
}

// The pair pipeline from tier 2 on, for explicit candidate pairs (sorted positions of the
// level): an incremental update hands over the pairs whose decision may have changed.
void run_pairs(const LevelIn& in, LevelOut& out, LevelStats& st, cudaStream_t s, const int2* pairs, int64_t m,
               const int32_t* knn_idx, const float* knn_key, bool tier2b) {
  memset(&st, 0, sizeof(st));
  auto t_last = std::chrono::steady_clock::now();
  std::function<void(int)> tick = [&](int slot) {
    GRNG_CUDA(cudaStreamSynchronize(s));
    auto now = std::chrono::steady_clock::now();
    st.ms[slot] += std::chrono::duration<double, std::milli>(now - t_last).count();
    t_last = now;
  };
  out.n_edges = 0;
  out.n_new_gg = 0;
  if (in.n < 2 || m == 0) return;
  DevBuf ctr;
  GRNG_CUDA(ctr.alloc(64 * sizeof(unsigned long long)));
  GRNG_CUDA(cudaMemsetAsync(ctr.p, 0, 64 * sizeof(unsigned long long), s));
  st.c[2] = (unsigned long long)m;
  finish_level(in, out, st, s, pairs, (unsigned long long)m, knn_idx, knn_key, nullptr, tier2b,
               ctr.as<unsigned long long>(), tick);
}

}  // namespace grng
