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
//   tier 3  exhaustive scan of all nodes (Stage VI) for the few pairs left.
// Comparisons whose FP32 brackets overlap are re-decided in canonical FP64.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tile.cuh"

namespace grng {

#define FULLMASK 0xffffffffu
static __device__ __forceinline__ float finf() { return __int_as_float(0x7f800000); }

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
  unsigned long long* stats;
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
  unsigned long long st_cand = 0, st_quick = 0;

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
        knnK[i] = finf();
        knnI[i] = -1;
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
      const bool filt = by >= bx;
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
            if (v < thr) {
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
              PairThr P = pair_thresholds(v, rxl, rxh, rylo[c], ryhi[c], METRIC, e, p.guide);
              if (P.quick) {
                quick = true;
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
    if (tid < nr) {
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
  }
  if (lane == 0) {
    atomicAdd(p.stats + 0, st_cand);
    atomicAdd(p.stats + 1, st_quick);
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
  const int64_t* off;    // [n+1] grouped by g
  const int32_t* other;  // partner o of each entry
  int2* links; unsigned long long* link_cnt; unsigned long long link_cap;
  int2* unres; unsigned long long* unres_cnt; unsigned long long unres_cap;
  int2* pend; unsigned long long* pend_cnt; unsigned long long pend_cap;
  int2* amb; unsigned long long* amb_cnt; unsigned long long amb_cap;
  unsigned long long* stats;  // [0] links [1] pendings [2] unresolved [3] blocked
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
    const float Rk = lastid >= 0 ? p.knn_key[g * K + K - 1] : finf();
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
      PairThr P = pair_thresholds(v, rgl, rgh, rol, roh, p.metric, e, p.guide);
      if (P.quick) {
        if (lane == 0) push_pair(p.links, p.link_cnt, p.link_cap, make_int2((int)g, o));
        c_link += lane == 0;
        continue;
      }
      int stt = 0;
      if (kidl >= 0 && kidl != o) {
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
struct Tier3Params {
  const float* X;
  int64_t n;
  int Dp, metric, guide;
  const float* rlo;
  const float* rhi;
  const int2* pairs;
  int64_t m;
  int2* pend;
  int* pflag;
  int64_t slot0;
  int2* amb; unsigned long long* amb_cnt; unsigned long long amb_cap;
};

__global__ void __launch_bounds__(256) tier3_kernel(Tier3Params p) {
  extern __shared__ __align__(16) float sm3[];
  float* gs = sm3;
  float* os = gs + p.Dp;
  __shared__ int s_block;
  __shared__ float s_v;
  const Err e = err_fp32(p.Dp);
  for (int64_t t = blockIdx.x; t < p.m; t += gridDim.x) {
    const int2 pr = p.pairs[t];
    const int64_t g = pr.x, o = pr.y;
    __syncthreads();
    for (int d = threadIdx.x; d < p.Dp; d += blockDim.x) {
      gs[d] = p.X[g * p.Dp + d];
      os[d] = p.X[o * p.Dp + d];
    }
    if (threadIdx.x == 0) s_block = 0;
    __syncthreads();
    if (threadIdx.x == 0) s_v = key32(gs, os, p.Dp, p.metric);
    __syncthreads();
    const float v = s_v;
    PairThr P = pair_thresholds(v, p.rlo ? p.rlo[g] : 0.0f, p.rhi ? p.rhi[g] : 0.0f,
                                p.rlo ? p.rlo[o] : 0.0f, p.rhi ? p.rhi[o] : 0.0f, p.metric, e,
                                p.guide);
    const int64_t slot = p.slot0 + t;
    if (!P.quick) {
      for (int64_t k0 = 0; k0 < p.n; k0 += blockDim.x) {
        if (*(volatile int*)&s_block) break;
        const int64_t k = k0 + threadIdx.x;
        if (k < p.n && k != g && k != o) {
          const float* pk = p.X + k * p.Dp;
          float a = key32(pk, gs, p.Dp, p.metric);
          float b = key32(pk, os, p.Dp, p.metric);
          int stt = block_state(a, b, P, e);
          if (stt == 2) s_block = 1;
          else if (stt == 1) push_pair(p.amb, p.amb_cnt, p.amb_cap, make_int2((int)slot, (int)k));
        }
      }
    }
    __syncthreads();
    if (threadIdx.x == 0) {
      p.pend[slot] = make_int2((int)g, (int)o);
      p.pflag[slot] = s_block ? 3 : 0;
    }
  }
}

// ---------------------------------------------------------------------------------
// FP64 recheck of ambiguous (pair, interceptor) triples, then emission.
// ---------------------------------------------------------------------------------
__global__ void recheck_kernel(const float* __restrict__ X, int D, int Dp, int metric,
                               const double* __restrict__ r64, const int2* __restrict__ amb,
                               int64_t m, const int2* __restrict__ pend, int* __restrict__ pflag,
                               unsigned long long* stats) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int2 a = amb[i];
  int2 pr = pend[a.x];
  double rx = r64 ? r64[pr.x] : 0.0, ry = r64 ? r64[pr.y] : 0.0;
  int bits = block64(X, D, Dp, metric, pr.x, pr.y, a.y, rx, ry);
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
                                    uint64_t* edges) {
  int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
  if (i >= m) return;
  int f = pflag ? pflag[i] : 0;
  int2 pr = pend[i];
  int a = min(pr.x, pr.y), b = max(pr.x, pr.y);
  if (grng) {
    if (!(f & 1)) atomicOr(gx + (int64_t)a * words + (b >> 5), 1u << (b & 31));
    if (!(f & 2)) atomicOr(gg + (int64_t)a * words + (b >> 5), 1u << (b & 31));
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
    block_prep_kernel<KC, L2><<<(unsigned)nb, GRNG_THREADS, smem, s>>>(in.X, in.n, in.Dp, A, ni, nk);
  } else {
    GRNG_CUDA(cudaFuncSetAttribute(block_prep_kernel<KC, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    block_prep_kernel<KC, L1><<<(unsigned)nb, GRNG_THREADS, smem, s>>>(in.X, in.n, in.Dp, A, ni, nk);
  }
  GRNG_CUDA(cudaGetLastError());
}

template <int KC>
static void launch_tile(const LevelIn& in, TileParams tp, int grid, cudaStream_t s) {
  size_t smem = tp_bytes(in.K);
  if (in.metric == L2) {
    GRNG_CUDA(cudaFuncSetAttribute(tile_pass_kernel<KC, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tile_pass_kernel<KC, L2><<<grid, GRNG_THREADS, smem, s>>>(tp);
  } else {
    GRNG_CUDA(cudaFuncSetAttribute(tile_pass_kernel<KC, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tile_pass_kernel<KC, L1><<<grid, GRNG_THREADS, smem, s>>>(tp);
  }
  GRNG_CUDA(cudaGetLastError());
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

void run_level(const LevelIn& in, LevelOut& out, LevelStats& st, cudaStream_t s, float* tile_ms) {
  memset(&st, 0, sizeof(st));
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
  // 18 unres, 19 amb, 20 unres2, 21 edges, 22 recheck blocked
  if (KC == 32) launch_prep<32>(in, A.as<__half>(), nbi.as<uint8_t>(), nbk.as<float>(), s);
  else if (KC == 16) launch_prep<16>(in, A.as<__half>(), nbi.as<uint8_t>(), nbk.as<float>(), s);
  else launch_prep<8>(in, A.as<__half>(), nbi.as<uint8_t>(), nbk.as<float>(), s);

  // ---- tier 1 -------------------------------------------------------------------------
  unsigned long long surv_cap = (unsigned long long)std::max<int64_t>(1 << 20, 16 * n);
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
    tp.parent = in.parent; tp.gpar = in.gpar; tp.gpar_words = in.gpar_words;
    tp.rlo = in.rlo; tp.rhi = in.rhi; tp.A = A.as<__half>(); tp.nbr_idx = nbi.as<uint8_t>();
    tp.nbr_key = nbk.as<float>(); tp.knn_idx = knni.as<int32_t>(); tp.knn_key = knnk.as<float>();
    tp.surv = surv.as<int2>(); tp.surv_cnt = dc + 1; tp.surv_cap = surv_cap;
    tp.gx = out.gx; tp.gg = out.gg; tp.words = out.words;
    tp.strip_ctr = reinterpret_cast<int*>(dc + 0); tp.stats = dc + 2;
    int grid = (int)std::min<int64_t>(nb, num_sms());
    cudaEvent_t e0, e1;
    if (tile_ms) {
      GRNG_CUDA(cudaEventCreate(&e0));
      GRNG_CUDA(cudaEventCreate(&e1));
      GRNG_CUDA(cudaEventRecord(e0, s));
    }
    if (KC == 32) launch_tile<32>(in, tp, grid, s);
    else if (KC == 16) launch_tile<16>(in, tp, grid, s);
    else launch_tile<8>(in, tp, grid, s);
    if (tile_ms) {
      GRNG_CUDA(cudaEventRecord(e1, s));
      GRNG_CUDA(cudaEventSynchronize(e1));
      GRNG_CUDA(cudaEventElapsedTime(tile_ms, e0, e1));
      cudaEventDestroy(e0);
      cudaEventDestroy(e1);
    }
    nsurv = read_u64(dc + 1, s);
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

  // ---- tiers 2 and 3 ---------------------------------------------------------------------
  DevBuf off, oth, tmp, links, unres, pend, amb, pflag, unres2, off2, oth2;
  GRNG_CUDA(off.alloc((size_t)(n + 1) * 8));
  GRNG_CUDA(oth.alloc(std::max<size_t>(nsurv, 1) * 4));
  group_pairs(surv.as<int2>(), (int64_t)nsurv, 0, n, off.as<int64_t>(), oth.as<int32_t>(), tmp, s);
  unsigned long long cap = std::max<unsigned long long>(nsurv, 1024);
  unsigned long long amb_cap = std::max<unsigned long long>(4 * nsurv, 1 << 20);
  for (int attempt = 0;; ++attempt) {
    GRNG_CUDA(links.alloc(cap * 8));
    GRNG_CUDA(unres.alloc(cap * 8));
    GRNG_CUDA(pend.alloc(cap * 8 * 2));
    GRNG_CUDA(amb.alloc(amb_cap * 8));
    GRNG_CUDA(cudaMemsetAsync(dc + 8, 0, 16 * sizeof(unsigned long long), s));
    Tier2Params t2;
    t2.X = in.X; t2.n = n; t2.Dp = in.Dp; t2.metric = in.metric; t2.guide = in.grng; t2.K = in.K;
    t2.rlo = in.rlo; t2.rhi = in.rhi; t2.knn_idx = knni.as<int32_t>(); t2.knn_key = knnk.as<float>();
    t2.off = off.as<int64_t>(); t2.other = oth.as<int32_t>();
    t2.links = links.as<int2>(); t2.link_cnt = dc + 16; t2.link_cap = cap;
    t2.unres = unres.as<int2>(); t2.unres_cnt = dc + 18; t2.unres_cap = cap;
    t2.pend = pend.as<int2>(); t2.pend_cnt = dc + 17; t2.pend_cap = 2 * cap;
    t2.amb = amb.as<int2>(); t2.amb_cnt = dc + 19; t2.amb_cap = amb_cap;
    t2.stats = dc + 8;
    size_t smem2 = (size_t)(in.Dp * 32 + in.Dp + 4 * in.Dp) * 4;
    int grid2 = (int)std::min<int64_t>(n, 32 * num_sms());
    if (nsurv) {
      tier2_kernel<<<grid2, 128, smem2, s>>>(t2);
      GRNG_CUDA(cudaGetLastError());
    }
    unsigned long long nun = read_u64(dc + 18, s);
    // tier 2b: the other endpoint's neighbours
    GRNG_CUDA(off2.alloc((size_t)(n + 1) * 8));
    GRNG_CUDA(oth2.alloc(std::max<unsigned long long>(nun, 1) * 4));
    group_pairs(unres.as<int2>(), (int64_t)std::min(nun, cap), 1, n, off2.as<int64_t>(),
                oth2.as<int32_t>(), tmp, s);
    t2.off = off2.as<int64_t>(); t2.other = oth2.as<int32_t>();
    GRNG_CUDA(unres2.alloc(std::max<unsigned long long>(nun, 1) * 8));
    t2.unres = unres2.as<int2>(); t2.unres_cnt = dc + 20; t2.unres_cap = std::max<unsigned long long>(nun, 1);
    t2.stats = dc + 12;
    if (nun) {
      tier2_kernel<<<grid2, 128, smem2, s>>>(t2);
      GRNG_CUDA(cudaGetLastError());
    }
    unsigned long long nun2 = read_u64(dc + 20, s);
    unsigned long long npend = read_u64(dc + 17, s);
    unsigned long long nlink = read_u64(dc + 16, s);
    if (npend + nun2 > 2 * cap || nlink > cap || nun > cap) fail(6, "tier-2 buffer overflow");
    // tier 3 appends its pairs after the tier-2 pendings
    GRNG_CUDA(pflag.alloc((size_t)std::max<unsigned long long>(npend + nun2, 1) * 4));
    GRNG_CUDA(cudaMemsetAsync(pflag.p, 0, (size_t)std::max<unsigned long long>(npend + nun2, 1) * 4, s));
    if (nun2) {
      Tier3Params t3;
      t3.X = in.X; t3.n = n; t3.Dp = in.Dp; t3.metric = in.metric; t3.guide = in.grng;
      t3.rlo = in.rlo; t3.rhi = in.rhi; t3.pairs = unres2.as<int2>(); t3.m = (int64_t)nun2;
      t3.pend = pend.as<int2>(); t3.pflag = pflag.as<int>(); t3.slot0 = (int64_t)npend;
      t3.amb = amb.as<int2>(); t3.amb_cnt = dc + 19; t3.amb_cap = amb_cap;
      int grid3 = (int)std::min<unsigned long long>(nun2, 8ull * num_sms());
      tier3_kernel<<<grid3, 256, 2 * in.Dp * 4, s>>>(t3);
      GRNG_CUDA(cudaGetLastError());
    }
    unsigned long long namb = read_u64(dc + 19, s);
    if (namb > amb_cap) {
      if (attempt >= 3) fail(2, "ambiguity buffer overflow");
      amb_cap = namb + namb / 4;
      continue;
    }
    if (namb) {
      recheck_kernel<<<(unsigned)((namb + 255) / 256), 256, 0, s>>>(
          in.X, in.D, in.Dp, in.metric, in.r64, amb.as<int2>(), (int64_t)namb, pend.as<int2>(),
          pflag.as<int>(), dc + 22);
      GRNG_CUDA(cudaGetLastError());
    }
    // ---- emission ----------------------------------------------------------------------
    const unsigned long long npp = npend + nun2;
    unsigned long long ecap = nlink + npp + 1;
    if (!in.grng) {
      GRNG_CUDA(out.edges->alloc(ecap * 8));
    }
    if (nlink)
      resolve_emit_kernel<<<(unsigned)((nlink + 255) / 256), 256, 0, s>>>(
          links.as<int2>(), nullptr, (int64_t)nlink, in.grng, out.gx, out.gg, out.words, in.orig,
          dc + 21, ecap, in.grng ? nullptr : out.edges->as<uint64_t>());
    if (npp)
      resolve_emit_kernel<<<(unsigned)((npp + 255) / 256), 256, 0, s>>>(
          pend.as<int2>(), pflag.as<int>(), (int64_t)npp, in.grng, out.gx, out.gg, out.words,
          in.orig, dc + 21, ecap, in.grng ? nullptr : out.edges->as<uint64_t>());
    GRNG_CUDA(cudaGetLastError());
    unsigned long long h[24];
    GRNG_CUDA(cudaMemcpyAsync(h, dc, sizeof(h), cudaMemcpyDeviceToHost, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    out.n_edges = (int64_t)h[21];
    st.c[3] = h[8];  st.c[4] = h[9];  st.c[5] = h[10]; st.c[6] = h[11];   // tier 2a
    st.c[7] = h[12]; st.c[8] = h[13]; st.c[9] = h[14]; st.c[10] = h[15];  // tier 2b
    st.c[11] = nun2;   // tier-3 pairs
    st.c[12] = namb;   // ambiguous triples rechecked in FP64
    st.c[13] = h[22];  // of which blocking
    st.c[14] = h[21];  // edges emitted (RNG level)
    break;
  }
}

}  // namespace grng
