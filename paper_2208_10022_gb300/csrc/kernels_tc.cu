// kernels_tc.cu -- precision form of the exemplar distance tiles: Gram keys
//     key(x, y) ~ |x|^2 + |y|^2 - 2 x.y
// with x.y on the tcgen05 tensor cores (BF16 inputs, FP32 accumulation in tensor
// memory), then the same tier-1 lune filter and neighbour lists as the FP32 sweep.
//
// Split BF16.  x = hi + lo with hi = bf16(x), lo = bf16(x - hi), and
//     x.y ~ hi.hi' + hi.lo' + lo.hi'
// (three MMAs per 16-wide chunk of K).  With u = 2^-8 the dropped terms are at most
// (2u^2 + u^3) |x||y| per coordinate pair, i.e. about 2^-15 |x||y| in total, and the
// FP32 accumulation of 3*Dp products adds at most 3*Dp*2^-24 sum|x_k y_k|.  The norms are
// FP32 sums (D+2)*2^-24 relative.  Using |x||y| <= (|x|^2 + |y|^2)/2, every key of a tile
// of blocks X, Y is within
//     E = gam * (max_X |x|^2 + max_Y |y|^2),  gam = 2^-12 + (3*Dp + 16) * 2^-24
// of the exact key (and of the canonical FP64 key).  Comparisons take this absolute
// bound on top of the FP32 relative bracket; whatever they cannot settle goes to the
// FP32-exact tiers and, when those cannot settle it either, to the FP64 recheck.
#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/grng.h"
#include "common.cuh"
#include "internal.h"
#include "tc.cuh"

namespace grng {

#define FULLMASK 0xffffffffu
static __device__ __forceinline__ float finf_tc() { return __int_as_float(0x7f800000); }

// ---- images, squared norms and per-block maxima ------------------------------------------
__global__ void tc_prep_kernel(const float* __restrict__ X, int64_t n, int Dp, uint8_t* __restrict__ img,
                               float* __restrict__ nrm, unsigned int* __restrict__ bmax) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= n) return;
  const int64_t b = s >> 7;
  const int r = (int)(s & 127);
  const size_t imgb = (size_t)128 * Dp * 2;
  uint8_t* hi = img + (size_t)b * 2 * imgb;
  uint8_t* lo = hi + imgb;
  float acc = 0.0f;
  for (int k = 0; k < Dp; ++k) {
    const float x = X[s * Dp + k];
    const __nv_bfloat16 h = __float2bfloat16_rn(x);
    const __nv_bfloat16 l = __float2bfloat16_rn(x - __bfloat162float(h));
    *reinterpret_cast<__nv_bfloat16*>(hi + img_off(r, k, Dp)) = h;
    *reinterpret_cast<__nv_bfloat16*>(lo + img_off(r, k, Dp)) = l;
    acc = fmaf(x, x, acc);
  }
  nrm[s] = acc;
  atomicMax(bmax + b, __float_as_uint(acc));  // non-negative floats order like their bits
}

struct TcParams {
  const uint8_t* img;
  const float* nrm;
  const unsigned int* bmax;  // float bits
  int64_t n;
  int Dp, K;
  float gam, nmax_all;
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
  unsigned long long* stats;  // [0] candidate pairs, [3] pairs taking the full filter
  int* status;                // bit 0: a bounded wait ran out
  long long spin;
};

static __host__ __device__ constexpr size_t tc_img_bytes(int Dp) { return (size_t)128 * Dp * 4; }  // hi + lo
static __host__ __device__ constexpr size_t tc_t16_bytes() { return (size_t)128 * 130 * 2; }
#define TC_SMEM_MAX (227 * 1024)
#define TC_QMAX 4096  // full-filter queue entries (8 bytes each), as many as shared memory leaves room for
#define TC_QMIN 512   // the fewest entries the pipelined form keeps
// AX, AY, the neighbour lists (the column block's twice), nx, ny x2, cmin/carg x4, parX,
// parY x2, rowx, barriers
static __host__ __device__ constexpr size_t tc_rest_bytes() {
  return 33280 + 34816 + 128 * GRNG_KIN * 15 + 10 * 512 + 4096 + 128;
}
// Pipelined form: T16 has a buffer of its own, so the next column block's image can be
// copied into sB and multiplied into the second TMEM accumulator while this tile's
// epilogue runs.  Without room for it, T16 reuses sB once the tile's MMAs have completed.
static __host__ __device__ constexpr bool tc_pipe(int Dp) {
  return 2 * tc_img_bytes(Dp) + tc_t16_bytes() + tc_rest_bytes() + (size_t)TC_QMIN * 8 <= TC_SMEM_MAX;
}
static __host__ __device__ constexpr size_t tc_base_bytes(int Dp) {
  return 2 * tc_img_bytes(Dp) + ((tc_pipe(Dp) || tc_img_bytes(Dp) < tc_t16_bytes()) ? tc_t16_bytes() : 0) +
         tc_rest_bytes();
}
static __host__ __device__ constexpr int tc_qcap(int Dp) {
  return tc_base_bytes(Dp) >= TC_SMEM_MAX ? 0
         : (int)((TC_SMEM_MAX - tc_base_bytes(Dp)) / 8 < TC_QMAX ? (TC_SMEM_MAX - tc_base_bytes(Dp)) / 8 : TC_QMAX);
}
// the s-th column block of strip bx in visiting order (bx, bx+1, bx-1, bx+2, ...), skipping
// those out of range; s advances past the block returned
__device__ __forceinline__ int64_t tc_next_by(int64_t bx, int64_t nb, int64_t& s) {
  for (;; ++s) {
    const int64_t off = (s & 1) ? ((s + 1) >> 1) : -(s >> 1);
    const int64_t by = bx + off;
    if (by >= 0 && by < nb) {
      ++s;
      return by;
    }
  }
}
static __host__ __device__ constexpr size_t tc_smem_bytes(int Dp, int K) {
  return (void)K, tc_base_bytes(Dp) + (size_t)tc_qcap(Dp) * 8;
}

// Insert (v, id) into the ascending register list kk/ki (32 slots, the first K in use)
// and return the new K-th key.  Fully unrolled so that the list stays in registers.
__device__ __forceinline__ float knn_insert_reg(float (&kk)[GRNG_KMAX], int (&ki)[GRNG_KMAX], float v, int id,
                                                int K) {
#pragma unroll
  for (int i = GRNG_KMAX - 1; i > 0; --i) {
    if (kk[i - 1] > v) {
      kk[i] = kk[i - 1];
      ki[i] = ki[i - 1];
    } else if (kk[i] > v) {
      kk[i] = v;
      ki[i] = id;
    }
  }
  if (kk[0] > v) {
    kk[0] = v;
    ki[0] = id;
  }
  float t = kk[0];
#pragma unroll
  for (int i = 1; i < GRNG_KMAX; ++i)
    if (i == K - 1) t = kk[i];
  return t;
}

// a[j] for a runtime j in [0, 16), by a tree of selects on j's bits (the array stays in
// registers; an indexed read would move it to local memory)
__device__ __forceinline__ float sel16(const float (&a)[16], int j) {
  float b[8], c[4], d[2];
#pragma unroll
  for (int i = 0; i < 8; ++i) b[i] = (j & 1) ? a[2 * i + 1] : a[2 * i];
#pragma unroll
  for (int i = 0; i < 4; ++i) c[i] = (j & 2) ? b[2 * i + 1] : b[2 * i];
#pragma unroll
  for (int i = 0; i < 2; ++i) d[i] = (j & 4) ? c[2 * i + 1] : c[2 * i];
  return (j & 8) ? d[1] : d[0];
}

__device__ __forceinline__ float sel32(const float (&a)[32], int j) {
  float b[16];
#pragma unroll
  for (int i = 0; i < 16; ++i) b[i] = (j & 1) ? a[2 * i + 1] : a[2 * i];
  return sel16(b, j >> 1);
}

// top-2 of (m1, a1), (m2, a2) merged with (b1, i1), (b2, i2)
__device__ __forceinline__ void top2_merge(float& m1, int& a1, float& m2, int& a2, float b1, int i1, float b2,
                                           int i2) {
  if (b1 < m1) {
    if (b2 < m1) { m2 = b2; a2 = i2; }
    else { m2 = m1; a2 = a1; }
    m1 = b1; a1 = i1;
  } else if (b1 < m2) {
    m2 = b1; a2 = i1;
  }
}

// Shared-memory views of one tile that the full tier-1 test reads.
struct TcTile {
  const __half* T16;    // [128][130] keys of the tile, rounded up
  const __half* AX;     // [128][130] in-block keys of the row block
  const __half* AY;     // [128][136] in-block keys of the column block
  const float* nbrXk;   // [t][row]
  const uint8_t* nbrXi;
  const float* nbrYk;   // [row][t]
  const uint8_t* nbrYi;
  const float* cmin1; const float* cmin2; const int* carg1; const int* carg2;
  float E;
  bool diag;
};

// Whether a tile-local interceptor certainly blocks (x = row r, y = column c) with key v:
// the row minimum of x over the column block (the second one when the first is y), the
// column minimum of y over the row block, the in-block neighbours of x and of y.
// (m1, a1), (m2, a2): the two smallest keys of row r over the column block.
__device__ __forceinline__ bool tc_full_test(const TcTile& T, int r, int c, float v, Err e, float m1, float m2,
                                             int a1, int a2) {
  const float vlo = lo_b(v - T.E, e);
  {  // row minimum of x over the column block
    const int z = (a1 != c) ? a1 : a2;
    if (z >= 0) {
      const float a = (a1 != c) ? m1 : m2;
      if (hi_b(a + T.E, e) < vlo && hi_b(__half2float(T.AY[z * 136 + c]), e) < vlo) return true;
    }
  }
  {  // column minimum of y over the row block (cmin: bounds of the exact keys, E included)
    const int z = (T.carg1[c] != r) ? T.carg1[c] : T.carg2[c];
    if (z >= 0) {
      const float b = (T.carg1[c] != r) ? T.cmin1[c] : T.cmin2[c];
      if (hi_b(__half2float(T.AX[r * 130 + z]), e) < vlo && b < vlo) return true;
    }
  }
  for (int t = 0; t < GRNG_KIN; ++t) {  // neighbours of x
    const int z = T.nbrXi[t * 128 + r];
    if (z == 255) break;
    if (T.diag && z == c) continue;
    if (hi_b(T.nbrXk[t * 128 + r], e) < vlo && hi_b(__half2float(T.T16[z * 130 + c]) + T.E, e) < vlo) return true;
  }
  for (int t = 0; t < GRNG_KIN; ++t) {  // neighbours of y
    const int z = T.nbrYi[c * GRNG_KIN + t];
    if (z == 255) break;
    if (T.diag && z == r) continue;
    if (hi_b(__half2float(T.T16[r * 130 + z]) + T.E, e) < vlo && hi_b(T.nbrYk[c * GRNG_KIN + t], e) < vlo) return true;
  }
  return false;
}

// One CTA of 256 threads per SM, persistent over row strips.  Per 128 x 128 tile: one
// thread issues the 3*Dp/16 MMAs into TMEM; then warp w reads the TMEM lanes of rows
// 32*(w%4).. and the 64 columns of half w/4.  Pass 1: keys to a rounded-up FP16 copy,
// row minima and the K-nearest lists (registers, one per half, merged at the end of
// the strip).  Upper tiles (y block >= x block) also run the tier-1 filter: column
// minima over the FP16 copy, then pass 2 over TMEM again.  The y block's in-block key
// matrix arrives by a bulk copy while pass 1 runs.
__global__ void __launch_bounds__(256, 1) tc_sweep_kernel(TcParams p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int Dp = p.Dp, K = p.K;
  const uint32_t IMG = (uint32_t)tc_img_bytes(Dp);
  uint8_t* sA = sm;
  uint8_t* sB = sm + IMG;
  size_t o = 2 * (size_t)IMG;
  const bool pipe = tc_pipe(Dp);
  const uint32_t TCOLS = pipe ? 256u : 128u;  // two accumulators when pipelined
  __half* T16;
  if (!pipe && IMG >= tc_t16_bytes()) {
    T16 = reinterpret_cast<__half*>(sB);  // the operand is dead once the MMA has completed
  } else {
    T16 = reinterpret_cast<__half*>(sm + o);
    o += tc_t16_bytes();
  }
  __half* AX = reinterpret_cast<__half*>(sm + o); o += 33280;   // [128][130]
  __half* AY = reinterpret_cast<__half*>(sm + o); o += 34816;   // [128][136]: rows 16-byte aligned
  // the column block's arrays come twice: the pipelined form loads the next tile's during
  // this one
  float* nbrXk = reinterpret_cast<float*>(sm + o); o += 128 * GRNG_KIN * 4;     // [t][row]
  float* nbrYk2 = reinterpret_cast<float*>(sm + o); o += 2 * 128 * GRNG_KIN * 4;  // [2][row][t]
  uint8_t* nbrXi = sm + o; o += 128 * GRNG_KIN;
  uint8_t* nbrYi2 = sm + o; o += 2 * 128 * GRNG_KIN;
  float* nx = reinterpret_cast<float*>(sm + o); o += 512;
  float* ny2 = reinterpret_cast<float*>(sm + o); o += 1024;
  float* cmin1 = reinterpret_cast<float*>(sm + o); o += 512;
  float* cmin2 = reinterpret_cast<float*>(sm + o); o += 512;
  int* carg1 = reinterpret_cast<int*>(sm + o); o += 512;
  int* carg2 = reinterpret_cast<int*>(sm + o); o += 512;
  int* parX = reinterpret_cast<int*>(sm + o); o += 512;
  int* parY2 = reinterpret_cast<int*>(sm + o); o += 1024;
  float4* rowx = reinterpret_cast<float4*>(sm + o); o += 4096;  // [2][128] partial row top-2
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + o);           // A image, B image, MMA done, AY
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + o + 32);
  int* s_strip = reinterpret_cast<int*>(sm + o + 36);
  int* s_abort = reinterpret_cast<int*>(sm + o + 40);
  int* s_qn = reinterpret_cast<int*>(sm + o + 44);               // full-filter queue length
  // per barrier: an issued copy or MMA batch not yet seen complete, and its phase parity
  int* s_pend = reinterpret_cast<int*>(sm + o + 48);
  int* s_par = s_pend + 4;
  uint2* Q = reinterpret_cast<uint2*>(sm + o + 128);              // (row | column << 8, key bits)
  const int qcap = tc_qcap(Dp);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lq = warp & 3, h = warp >> 2;
  const int r = lq * 32 + lane;  // this thread's row (its TMEM lane)
  const int cb = h * 64;         // first column of this thread's half
  const int64_t n = p.n;
  const int64_t nb = (n + 127) / 128;
  const Err e = err_fp32(Dp);
  const float INF = finf_tc();
  unsigned long long st_cand = 0, st_full = 0;

  if (warp == 0) {
    tmem_alloc(tslot, TCOLS);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) {
      mbar_init(&bars[i], 1);
      s_pend[i] = 0;
      s_par[i] = 0;
    }
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t trow = tbase + ((uint32_t)(lq * 32) << 16) + (uint32_t)cb;
  uint32_t phA = 0, phB = 0, phM = 0, phY = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) *s_strip = atomicAdd(p.strip_ctr, 1);
    __syncthreads();
    const int64_t bx = *s_strip;
    if (bx >= nb || __syncthreads_or(*s_abort)) break;
    const int64_t xb = bx * 128;
    const int nr = (int)(n - xb < 128 ? n - xb : 128);
    if (tid == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bars[0], IMG);
      bulk_g2s(sA, p.img + (size_t)bx * IMG, IMG, &bars[0]);
      s_pend[0] = 1;
      s_par[0] = (int)phA;
    }
    {
      const uint32_t* srcA = reinterpret_cast<const uint32_t*>(p.A + bx * 16384);
      for (int w = tid; w < 8192; w += 256)
        *reinterpret_cast<uint32_t*>(AX + (w >> 6) * 130 + (w & 63) * 2) = srcA[w];
    }
    for (int i = tid; i < 128 * GRNG_KIN; i += 256) {
      const int rr = i / GRNG_KIN, tt = i % GRNG_KIN;  // stored [t][row]: lanes = rows
      const bool ok = rr < nr;
      nbrXi[tt * 128 + rr] = ok ? p.nbr_idx[xb * GRNG_KIN + i] : (uint8_t)255;
      nbrXk[tt * 128 + rr] = ok ? p.nbr_key[xb * GRNG_KIN + i] : INF;
    }
    if (tid < 128) {
      nx[tid] = tid < nr ? p.nrm[xb + tid] : 0.0f;
      parX[tid] = (p.parent && tid < nr) ? p.parent[xb + tid] : 0;
    }
    float kk[GRNG_KMAX];
    int ki[GRNG_KMAX];
#pragma unroll
    for (int j = 0; j < GRNG_KMAX; ++j) { kk[j] = INF; ki[j] = -1; }
    float thr = INF;
    if (tid == 0) {
      if (mbar_wait(&bars[0], phA, p.spin)) s_pend[0] = 0;
      else *s_abort = 1;
    }
    if (tid == 0 && s_pend[0]) {
      atomicOr(p.status, 1);
    }
    phA ^= 1;
    const float bmx = __uint_as_float(p.bmax[bx]);
    const bool vr = r < nr;
    // norms, parents and neighbour lists of column block yy into buffer b
    auto load_cols = [&](int64_t yy, int b) {
      const int64_t y0 = yy * 128;
      const int ncc = (int)(n - y0 < 128 ? n - y0 : 128);
      if (tid < 128) {
        ny2[b * 128 + tid] = tid < ncc ? p.nrm[y0 + tid] : 0.0f;
        parY2[b * 128 + tid] = (p.parent && tid < ncc) ? p.parent[y0 + tid] : 0;
      }
      if (yy >= bx)
        for (int i = tid; i < 128 * GRNG_KIN; i += 256) {
          const bool ok = i / GRNG_KIN < ncc;
          nbrYi2[b * 128 * GRNG_KIN + i] = ok ? p.nbr_idx[y0 * GRNG_KIN + i] : (uint8_t)255;
          nbrYk2[b * 128 * GRNG_KIN + i] = ok ? p.nbr_key[y0 * GRNG_KIN + i] : INF;
        }
    };
    int64_t sidx = 0;
    int64_t by = tc_next_by(bx, nb, sidx);
    if (pipe) load_cols(by, 0);  // published by the first tile's barrier
    uint32_t acc = 0;  // TMEM column of this tile's accumulator
    int64_t by_nx = -1;
    if (pipe) {        // the strip's first tile: copy and MMAs now, the later ones a tile ahead
      if (tid == 0 && !*s_abort) {
        mbar_expect_tx(&bars[1], IMG);
        bulk_g2s(sB, p.img + (size_t)by * IMG, IMG, &bars[1]);
        s_pend[1] = 1;
        s_par[1] = (int)phB;
        if (mbar_wait(&bars[1], phB, p.spin)) {
          s_pend[1] = 0;
          tc_fence_after();
          issue_gram_tile(tbase, sA, sB, Dp);
          umma_commit(&bars[2]);
          s_pend[2] = 1;
          s_par[2] = (int)phM;
        } else {
          *s_abort = 1;
          atomicOr(p.status, 1);
        }
      }
      phB ^= 1;
    }
    for (int64_t t = 0; t < nb; ++t, acc ^= (pipe ? 128u : 0u)) {
      if (t > 0) by = by_nx;
      const int64_t by_next = t + 1 < nb ? tc_next_by(bx, nb, sidx) : -1;
      by_nx = by_next;
      const int64_t yb = by * 128;
      const int nc = (int)(n - yb < 128 ? n - yb : 128);
      const bool filt = by >= bx;
      const bool diag = by == bx;
      // the previous tile's generic accesses to T16 (which may alias sB) and AY are
      // ordered before the bulk copies that overwrite them: each thread fences, then all meet
      fence_proxy_async();
      if (__syncthreads_or(*s_abort)) break;  // one answer for all threads
      if (tid == 0) {
        *s_qn = 0;
        if (!pipe) {
          mbar_expect_tx(&bars[1], IMG);
          bulk_g2s(sB, p.img + (size_t)by * IMG, IMG, &bars[1]);
          s_pend[1] = 1;
          s_par[1] = (int)phB;
        }
        if (filt) {
          mbar_expect_tx(&bars[3], 32768);
          s_pend[3] = 1;
          s_par[3] = (int)phY;
        }
      }
      if (filt && warp == 0) {
        // one 256-byte copy per row into rows of 272 bytes: lanes reading one column of
        // different rows then meet at most 4 to a bank, not 32
        __syncwarp();
        for (int rr = lane; rr < 128; rr += 32)
          bulk_g2s(AY + rr * 136, p.A + by * 16384 + rr * 128, 256, &bars[3]);
      }
      const int cbuf = pipe ? (int)(t & 1) : 0;
      float* ny = ny2 + cbuf * 128;
      int* parY = parY2 + cbuf * 128;
      float* nbrYk = nbrYk2 + cbuf * 128 * GRNG_KIN;
      uint8_t* nbrYi = nbrYi2 + cbuf * 128 * GRNG_KIN;
      if (!pipe) load_cols(by, 0);       // published by the barrier after the MMAs
      else if (by_next >= 0) load_cols(by_next, cbuf ^ 1);  // published by the next tile's first barrier
      if (!pipe) {
        if (tid == 0) {
          if (mbar_wait(&bars[1], phB, p.spin)) {
            s_pend[1] = 0;
            tc_fence_after();
            issue_gram_tile(tbase, sA, sB, Dp);
            umma_commit(&bars[2]);
            s_pend[2] = 1;
            s_par[2] = (int)phM;
          } else {
            *s_abort = 1;
            atomicOr(p.status, 1);
          }
        }
        phB ^= 1;
        if (__syncthreads_or(*s_abort)) break;
      }
      if (mbar_wait(&bars[2], phM, p.spin)) {
        if (tid == 0) s_pend[2] = 0;
      } else {
        *s_abort = 1;
        atomicOr(p.status, 1);
      }
      phM ^= 1;
      tc_fence_after();
      if (!pipe) {  // also: this tile's column arrays are in place
        if (__syncthreads_or(*s_abort)) break;
      }
      if (pipe && tid == 0 && by_next >= 0 && !*s_abort) {
        // this tile's MMAs have completed: sB takes the next column block's image now
        mbar_expect_tx(&bars[1], IMG);
        bulk_g2s(sB, p.img + (size_t)by_next * IMG, IMG, &bars[1]);
        s_pend[1] = 1;
        s_par[1] = (int)phB;
      }
      const uint32_t tacc = trow + acc;  // this thread's lane and half in this tile's accumulator
      // ---- pass 1: keys -> T16, row minima, neighbour lists (thread = row, half) ----------
      // 16 columns per TMEM load; list insertions, rare once the lists fill, are taken out
      // of the unrolled part so that the loop stays small
      const float nxr = nx[r];
      float m1 = INF, m2 = INF;
      int a1 = -1, a2 = -1;
      // lower tiles feed only the neighbour lists; full tiles need no per-key mask
      const bool full = vr && nc == 128 && !diag;
#pragma unroll 1
      for (int q = 0; q < 4; ++q) {
        float g[16], vv[16];
        tmem_ld16(tacc + (uint32_t)(q * 16), g);
        unsigned pm = 0;
        const int c0 = cb + q * 16;
        if (!filt) {
          // only the chunk's smallest key is compared with the list's bound (insertions are rare)
          float mn = INF;
#pragma unroll
          for (int j = 0; j < 16; ++j) {
            const int c = c0 + j;
            float v = nxr + ny[c] - 2.0f * g[j];
            if (!full && (!vr || c >= nc)) v = INF;
            vv[j] = v;
            mn = fminf(mn, v);
          }
          if (mn < thr)
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (vv[j] < thr) pm |= 1u << j;
        } else {
          const float m1in = m1;  // the chunk's smallest key is below the row's minimum before it, or none is
#pragma unroll
          for (int j = 0; j < 16; j += 2) {
            float w[2];
#pragma unroll
            for (int u = 0; u < 2; ++u) {
              const int c = c0 + j + u;
              float v = nxr + ny[c] - 2.0f * g[j + u];
              if (!full && (!vr || c >= nc || (diag && c == r))) v = INF;
              vv[j + u] = v;
              w[u] = v;
              if (v < m2) {
                if (v < m1) { m2 = m1; a2 = a1; m1 = v; a1 = c; }
                else { m2 = v; a2 = c; }
              }
            }
            // two keys per 4-byte store (rows of T16 start on 4-byte boundaries)
            *reinterpret_cast<__half2*>(T16 + r * 130 + c0 + j) = __halves2half2(__float2half_ru(w[0]), __float2half_ru(w[1]));
          }
          // a key below the list's bound is at most the running minimum m1 (m2 >= m1); the list
          // is checked key by key only when the chunk lowered m1 below the bound or m2 lies below it
          if (fminf(m1 < m1in ? m1 : INF, m2) < thr)
#pragma unroll
            for (int j = 0; j < 16; ++j)
              if (vv[j] < thr) pm |= 1u << j;
        }
        while (pm) {
          const int j = __ffs(pm) - 1;
          pm &= pm - 1u;
          const float v = sel16(vv, j);
          if (v < thr) thr = knn_insert_reg(kk, ki, v, (int)(yb + c0 + j), K);
        }
      }
      tc_fence_before();
      if (filt) {  // (a lower tile's epilogue ends here: the next tile's first barrier follows)
        rowx[h * 128 + r] = make_float4(m1, m2, __int_as_float(a1), __int_as_float(a2));
        if (__syncthreads_or(*s_abort)) break;
      }
      if (pipe && by_next >= 0) {
        // the next tile's MMAs into the other accumulator, under this tile's epilogue (that
        // accumulator's last reads, in the previous tile, are ordered by the barriers since)
        if (tid == 0 && !*s_abort) {
          if (mbar_wait(&bars[1], phB, p.spin)) {
            s_pend[1] = 0;
            tc_fence_after();
            issue_gram_tile(tbase + (acc ^ 128u), sA, sB, Dp);
            umma_commit(&bars[2]);
            s_pend[2] = 1;
            s_par[2] = (int)phM;
          } else {
            *s_abort = 1;
            atomicOr(p.status, 1);
          }
        }
        phB ^= 1;
      }
      if (filt) {
        // ---- column minima over the row block: two lanes of a warp per column, 64 rows
        // each (the second half-warp runs 16 rows ahead in its half: rows 65 words apart in
        // T16 shift the bank by one, so the two half-warps read disjoint banks), merged by a
        // shuffle ---------------------------------------------------------------------------
        const float E = p.gam * (bmx + __uint_as_float(p.bmax[by]));
        {
          const int c = warp * 16 + (lane & 15), hr = lane >> 4;
          float c1 = INF, c2 = INF;
          int b1 = -1, b2 = -1;
          for (int i = 0; i < 64; ++i) {
            const int rr = hr * 64 + ((i + hr * 16) & 63);
            const float v = __half2float(T16[rr * 130 + c]);
            if (v < c2) {
              if (v < c1) { c2 = c1; b2 = b1; c1 = v; b1 = rr; }
              else { c2 = v; b2 = rr; }
            }
          }
          const float o1 = __shfl_xor_sync(FULLMASK, c1, 16), o2 = __shfl_xor_sync(FULLMASK, c2, 16);
          const int ob1 = __shfl_xor_sync(FULLMASK, b1, 16), ob2 = __shfl_xor_sync(FULLMASK, b2, 16);
          top2_merge(c1, b1, c2, b2, o1, ob1, o2, ob2);
          if (hr == 0) {  // as certain upper bounds of the exact keys
            cmin1[c] = hi_b(c1 + E, e); cmin2[c] = hi_b(c2 + E, e); carg1[c] = b1; carg2[c] = b2;
          }
        }
        {  // the other half's row minima
          const float4 w4 = rowx[(1 - h) * 128 + r];
          top2_merge(m1, a1, m2, a2, w4.x, __float_as_int(w4.z), w4.y, __float_as_int(w4.w));
        }
        if (mbar_wait(&bars[3], phY, p.spin)) {
          if (tid == 0) s_pend[3] = 0;
        } else {
          *s_abort = 1;
          atomicOr(p.status, 1);
        }
        phY ^= 1;
        __syncthreads();
        tc_fence_after();
        // ---- tier-1 filter: thread = row x, one column y of its half at a time ----------
        const int px = parX[r];
        // link bits of px's row of the parents' GRNG: y parents lie in [parY[0], parY[nc-1]]
        // and are >= px in every upper tile (nodes are sorted by parent)
        uint32_t gw[5] = {0u, 0u, 0u, 0u, 0u};
        int wlo = 0, nw = 0;
        bool all_linked = !p.gpar;  // every y parent equal to or linked with px: no per-pair test
        if (p.gpar && vr) {
          wlo = parY[0] >> 5;
          nw = (parY[nc - 1] >> 5) - wlo + 1;
#pragma unroll
          for (int k = 0; k < 5; ++k)
            if (k < nw) gw[k] = __ldg(p.gpar + (int64_t)px * p.gpar_words + wlo + k);
          if (nw <= 5 && parY[0] > px) {
            // bits parY[0] .. parY[nc-1] of px's row, relative to word wlo
            const int b0 = parY[0] - (wlo << 5), b1 = parY[nc - 1] - (wlo << 5);
            all_linked = true;
#pragma unroll
            for (int k = 0; k < 5; ++k) {
              if (k >= nw) break;
              const int lo = max(b0 - 32 * k, 0), hi = min(b1 - 32 * k, 31);
              if (lo > hi) continue;
              const uint32_t msk = (hi - lo == 31) ? ~0u : (((1u << (hi - lo + 1)) - 1u) << lo);
              all_linked = all_linked && ((gw[k] & msk) == msk);
            }
          }
        }
        // the whole tile's row minima, for the full tests of any thread (the other half read
        // its slot of rowx before the last barrier)
        if (h == 0) rowx[r] = make_float4(m1, m2, __int_as_float(a1), __int_as_float(a2));
        // quick tests, uniform over the row's 64 columns so that the warp stays converged:
        //  - the row minimum z = a1 of x over the column block blocks (x, y) once key(x, z)
        //    and key(z, y) (the in-block key, AY row z) are both certainly below key(x, y);
        //  - the column minimum z' of y over the row block blocks it once key(x, z') (the
        //    in-block key, AX row x) and key(z', y) are.
        // (For y = z or x = z' a test fails by itself: a key cannot be certainly below
        // itself.)  The columns both leave go to a queue that all 256 threads share once the
        // tile's TMEM has been read, so that no warp waits for another's divergent tests.
        const float A1 = hi_b(m1 + E, e);
        const bool rq = vr && a1 >= 0;
        const bool fast = vr && nc == 128 && !diag && all_linked;  // every column a candidate
        if (fast) st_cand += 64;
        const __half* AYz = AY + (rq ? a1 : 0) * 136 + cb;
        const __half* AXr = AX + r * 130;  // x's in-block keys
#pragma unroll 1
        for (int q = 0; q < 2; ++q) {  // two chunks of 32 columns, one tensor-memory wait each
          float g[32];
          tmem_ld32(tacc + (uint32_t)(q * 32), g);
          unsigned nd = 0;
#pragma unroll
          for (int q8 = 0; q8 < 4; ++q8) {
            const int c8 = cb + q * 32 + q8 * 8;
            const uint4 ayw = *reinterpret_cast<const uint4*>(AYz + q * 32 + q8 * 8);
            const __half2* ay2 = reinterpret_cast<const __half2*>(&ayw);
            const float4 nya = *reinterpret_cast<const float4*>(ny + c8);
            const float4 nyb = *reinterpret_cast<const float4*>(ny + c8 + 4);
            const float nyv[8] = {nya.x, nya.y, nya.z, nya.w, nyb.x, nyb.y, nyb.z, nyb.w};
            const int4 za = *reinterpret_cast<const int4*>(carg1 + c8);
            const int4 zb = *reinterpret_cast<const int4*>(carg1 + c8 + 4);
            const int zcv[8] = {za.x, za.y, za.z, za.w, zb.x, zb.y, zb.z, zb.w};
            const float4 cma = *reinterpret_cast<const float4*>(cmin1 + c8);
            const float4 cmb = *reinterpret_cast<const float4*>(cmin1 + c8 + 4);
            const float cmv[8] = {cma.x, cma.y, cma.z, cma.w, cmb.x, cmb.y, cmb.z, cmb.w};
#pragma unroll
            for (int j = 0; j < 8; ++j) {
              const int c = c8 + j;
              bool cand = true;
              if (!fast) {
                cand = vr && c < nc && (!diag || c > r);
                if (cand && !all_linked) {
                  const int qy = parY[c];
                  if (qy != px) {
                    const int b = qy - (wlo << 5);
                    if (qy > px && b >= 0 && (b >> 5) < nw && nw <= 5) {
                      const int wi = b >> 5;
                      uint32_t w = gw[0];
#pragma unroll
                      for (int k = 1; k < 5; ++k)
                        if (wi == k) w = gw[k];
                      cand = (w >> (b & 31)) & 1u;
                    } else {
                      const int lo = min(px, qy), hi = max(px, qy);
                      cand = (__ldg(p.gpar + (int64_t)lo * p.gpar_words + (hi >> 5)) >> (hi & 31)) & 1u;
                    }
                  }
                }
                st_cand += cand ? 1 : 0;
              }
              const float v = nxr + nyv[j] - 2.0f * g[q8 * 8 + j];
              const float vlo = lo_b(v - E, e);  // below every key this pair can have
              const float2 a2f = __half22float2(ay2[j >> 1]);
              const float ayz = (j & 1) ? a2f.y : a2f.x;
              const int zc = zcv[j];
              const float axz = __half2float(AXr[zc < 0 ? 0 : zc]);
              const bool quick = (rq && fmaxf(A1, hi_b(ayz, e)) < vlo) ||
                                 (zc >= 0 && fmaxf(hi_b(axz, e), cmv[j]) < vlo);
              if (cand && !quick) nd |= 1u << (q8 * 8 + j);
            }
          }
          // ---- the columns the quick test left: queued (key from the registers) -----------
          const int cnt = __popc(nd);
          st_full += cnt;
          int incl = cnt;
#pragma unroll
          for (int o2 = 1; o2 < 32; o2 <<= 1) {
            const int y2 = __shfl_up_sync(FULLMASK, incl, o2);
            if (lane >= o2) incl += y2;
          }
          int base = 0;
          const int wtot = __shfl_sync(FULLMASK, incl, 31);
          if (lane == 31 && wtot) base = atomicAdd(s_qn, wtot);
          base = __shfl_sync(FULLMASK, base, 31);
          int pos = base + incl - cnt;
          // few columns per warp fail both tests: each lane walks its own bits; with the queue
          // full (near the diagonal) the pair goes on to the exact tiers untested
          while (nd) {
            const int jj = __ffs(nd) - 1;
            nd &= nd - 1u;
            const int c = cb + q * 32 + jj;
            const float v = nxr + ny[c] - 2.0f * sel32(g, jj);
            if (pos < qcap) {
              Q[pos] = make_uint2((unsigned)r | ((unsigned)c << 8), __float_as_uint(v));
            } else {
              const unsigned long long sp = atomicAdd(p.surv_cnt, 1ull);
              if (sp < p.surv_cap) p.surv[sp] = make_int2((int)(xb + r), (int)(yb + c));
            }
            ++pos;
          }
        }
        tc_fence_before();
        __syncthreads();
        // ---- the queued full tests, shared by all threads; survivors by warp ------------
        {
          const int qn = min(*s_qn, qcap);
          const TcTile Tt{T16, AX, AY, nbrXk, nbrXi, nbrYk, nbrYi, cmin1, cmin2, carg1, carg2, E, diag};
          for (int i0 = 0; i0 < qn; i0 += 256) {
            const int i = i0 + tid;
            bool sv = false;
            int sr = 0, sc = 0;
            if (i < qn) {
              const uint2 it = Q[i];
              sr = (int)(it.x & 255u);
              sc = (int)(it.x >> 8);
              const float4 rm = rowx[sr];
              sv = !tc_full_test(Tt, sr, sc, __uint_as_float(it.y), e, rm.x, rm.y, __float_as_int(rm.z),
                                 __float_as_int(rm.w));
            }
            const unsigned bm = __ballot_sync(FULLMASK, sv);
            if (bm) {
              unsigned long long b0 = 0;
              if (lane == 0) b0 = atomicAdd(p.surv_cnt, (unsigned long long)__popc(bm));
              b0 = __shfl_sync(FULLMASK, b0, 0);
              if (sv) {
                const unsigned long long sp = b0 + (unsigned long long)__popc(bm & ((1u << lane) - 1u));
                if (sp < p.surv_cap) p.surv[sp] = make_int2((int)(xb + sr), (int)(yb + sc));
              }
            }
          }
        }
        tc_fence_before();
      }
    }
    // ---- the two halves' neighbour lists, merged (T16 and AY are free now) -------------
    __syncthreads();
    {
      float* LK = reinterpret_cast<float*>(h ? static_cast<void*>(AY) : static_cast<void*>(T16));  // [t][row]
      int* LI = reinterpret_cast<int*>(LK + GRNG_KMAX * 128);
#pragma unroll
      for (int t = 0; t < GRNG_KMAX; ++t) {
        LK[t * 128 + r] = kk[t];
        LI[t * 128 + r] = ki[t];
      }
    }
    __syncthreads();
    if (h == 0 && vr) {
      const float* K0 = reinterpret_cast<const float*>(T16);
      const int* I0 = reinterpret_cast<const int*>(K0 + GRNG_KMAX * 128);
      const float* K1 = reinterpret_cast<const float*>(AY);
      const int* I1 = reinterpret_cast<const int*>(K1 + GRNG_KMAX * 128);
      int i0 = 0, i1 = 0;
      float lastk = INF;
      int lasti = -1;
      for (int j = 0; j < K; ++j) {
        const float k0 = i0 < K ? K0[i0 * 128 + r] : INF;
        const float k1 = i1 < K ? K1[i1 * 128 + r] : INF;
        float kv;
        int iv;
        if (k0 <= k1) { kv = k0; iv = i0 < K ? I0[i0 * 128 + r] : -1; ++i0; }
        else { kv = k1; iv = I1[i1 * 128 + r]; ++i1; }
        p.knn_idx[(xb + r) * K + j] = iv;
        p.knn_key[(xb + r) * K + j] = kv;
        lastk = kv;
        lasti = iv;
      }
      // every unlisted node z has tile key >= the K-th listed, hence exact key >= that - E(x, z)
      p.knn_rb[xb + r] = lasti >= 0 ? lastk - p.gam * (nx[r] + p.nmax_all) : INF;
    }
  }
  for (int o2 = 16; o2 > 0; o2 >>= 1) {
    st_cand += __shfl_down_sync(FULLMASK, st_cand, o2);
    st_full += __shfl_down_sync(FULLMASK, st_full, o2);
  }
  if (lane == 0) {
    atomicAdd(p.stats, st_cand);
    atomicAdd(p.stats + 3, st_full);
  }
  // teardown.  After a bounded wait ran out, copies into this CTA's shared memory or MMAs
  // into its tensor memory may still be in flight: wait (again bounded, far longer) for every
  // barrier with an outstanding phase before the memory is released.
  __syncthreads();
  if (*s_abort && tid == 0) {
    const long long lim = p.spin > (1ll << 26) ? p.spin : (1ll << 26);
    for (int b = 0; b < 4; ++b)
      if (s_pend[b] && !mbar_wait(&bars[b], (uint32_t)s_par[b], lim)) atomicOr(p.status, 2);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, TCOLS);
}

// the listed neighbours' keys again, exactly in FP32 (the tiers compare FP32 keys)
__global__ void tc_knn_fix_kernel(const float* __restrict__ X, int64_t n, int Dp, int K, int metric,
                                  const int32_t* __restrict__ knn_idx, float* __restrict__ knn_key) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n * K) return;
  const int64_t x = i / K;
  const int k = knn_idx[i];
  if (k >= 0) knn_key[i] = key32(X + x * Dp, X + (int64_t)k * Dp, Dp, metric);
}

// ---- nearest pivot on the tensor cores (Eq. 2 assignment, split-BF16 Gram keys) ----------
// One persistent CTA per SM walks 128-member strips; per strip the pivot blocks go by in
// order through two image buffers and two TMEM accumulators: while the keys of block pb
// are read, block pb+1's MMAs run and block pb+2's image is copied.  Thread (row r, half h)
// keeps the two smallest Gram keys of its member over its 64 columns and the pivot of the
// smallest; the halves merge at the end of the strip.  With E = gam (max |x|^2 of the strip +
// max |p|^2 of all pivots) bounding every key's error, best1 = an upper bound of the
// smallest exact key (its pivot in arg1) and best2 = a lower bound of every other pivot's
// exact key; the caller accepts arg1 when best1 < best2 and re-decides the member exactly
// otherwise.
struct TcAssignParams {
  const uint8_t* imgX; const float* nX; const unsigned int* bmaxX;
  const uint8_t* imgP; const float* nP;
  int64_t nmem, m;
  int Dp;
  float gam, pmax;
  float* best1; int32_t* arg1; float* best2;
  int32_t* cand;  // [nmem][TCA_K] the pivots of the TCA_K smallest Gram keys, smallest first
  float* rest;    // [nmem] lower bound of every other pivot's exact key
  int* strip_ctr; int* status; long long spin;
};

#define TCA_K 4
static __host__ __device__ constexpr size_t tc_assign_smem(int Dp) {
  return 3 * tc_img_bytes(Dp) + 512 + 128 * TCA_K * 8 + 128;
}

__global__ void __launch_bounds__(256, 1) tc_assign_kernel(TcAssignParams p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int Dp = p.Dp;
  const uint32_t IMG = (uint32_t)tc_img_bytes(Dp);
  uint8_t* sA = sm;
  uint8_t* sBb[2] = {sm + IMG, sm + 2 * IMG};
  size_t o = 3 * (size_t)IMG;
  float* np_ = reinterpret_cast<float*>(sm + o); o += 512;        // pivot norms of the block
  float2* half2 = reinterpret_cast<float2*>(sm + o); o += 128 * TCA_K * 8;  // [TCA_K][128] the second half's list
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + o);            // A image, B images, MMA done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + o + 32);
  int* s_strip = reinterpret_cast<int*>(sm + o + 36);
  int* s_abort = reinterpret_cast<int*>(sm + o + 40);
  int* s_pend = reinterpret_cast<int*>(sm + o + 48);              // outstanding phases per barrier
  int* s_par = s_pend + 4;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int lq = warp & 3, h = warp >> 2;
  const int r = lq * 32 + lane;
  const int cb = h * 64;
  const int64_t nbx = (p.nmem + 127) / 128, npb = (p.m + 127) / 128;
  const Err e = err_fp32(Dp);
  const float INF = finf_tc();
  if (warp == 0) {
    tmem_alloc(tslot, 256);
    tmem_relinquish();
  }
  if (tid == 0) {
    for (int i = 0; i < 4; ++i) {
      mbar_init(&bars[i], 1);
      s_pend[i] = 0;
      s_par[i] = 0;
    }
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t trow = tbase + ((uint32_t)(lq * 32) << 16) + (uint32_t)cb;
  uint32_t phA = 0, phB = 0, phM = 0;
  // tid 0: copy of pivot block q into its buffer (par: the parity its wait will use); wait
  // for it and issue its MMAs
  auto copy_b = [&](int64_t q, uint32_t par) {
    mbar_expect_tx(&bars[1], IMG);
    bulk_g2s(sBb[q & 1], p.imgP + (size_t)q * IMG, IMG, &bars[1]);
    s_pend[1] = 1;
    s_par[1] = (int)par;
  };
  auto mma_b = [&](int64_t q) -> bool {
    if (!mbar_wait(&bars[1], phB, p.spin)) return false;
    s_pend[1] = 0;
    tc_fence_after();
    issue_gram_tile(tbase + (uint32_t)(q & 1) * 128u, sA, sBb[q & 1], Dp);
    umma_commit(&bars[2]);
    s_pend[2] = 1;
    s_par[2] = (int)phM;
    return true;
  };
  for (;;) {
    __syncthreads();
    if (tid == 0) *s_strip = atomicAdd(p.strip_ctr, 1);
    __syncthreads();
    const int64_t bx = *s_strip;
    if (bx >= nbx || __syncthreads_or(*s_abort)) break;
    const int64_t xb = bx * 128;
    const int nr = (int)(p.nmem - xb < 128 ? p.nmem - xb : 128);
    if (tid == 0) {  // the strip's image, block 0's MMAs, block 1's copy
      fence_proxy_async();
      mbar_expect_tx(&bars[0], IMG);
      bulk_g2s(sA, p.imgX + (size_t)bx * IMG, IMG, &bars[0]);
      s_pend[0] = 1;
      s_par[0] = (int)phA;
      copy_b(0, phB);
      bool ok = mbar_wait(&bars[0], phA, p.spin);
      if (ok) s_pend[0] = 0;
      ok = ok && mma_b(0);
      if (ok && npb > 1) copy_b(1, phB ^ 1u);
      if (!ok) {
        *s_abort = 1;
        atomicOr(p.status, 1);
      }
    }
    phA ^= 1;
    phB ^= 1;
    const float nxr = r < nr ? p.nX[xb + r] : 0.0f;
    const float E = p.gam * (__uint_as_float(p.bmaxX[bx]) + p.pmax);
    float tv[TCA_K];  // the TCA_K smallest keys of this half, ascending, and their pivots
    int ti[TCA_K];
#pragma unroll
    for (int k = 0; k < TCA_K; ++k) { tv[k] = INF; ti[k] = -1; }
    for (int64_t pb = 0; pb < npb; ++pb) {
      const int64_t pc = pb * 128;
      const int nc = (int)(p.m - pc < 128 ? p.m - pc : 128);
      if (tid < 128) np_[tid] = tid < nc ? p.nP[pc + tid] : 0.0f;
      // also: every read of the accumulator block pb+1 will take is done
      if (__syncthreads_or(*s_abort)) break;
      if (mbar_wait(&bars[2], phM, p.spin)) {  // block pb's MMAs
        if (tid == 0) s_pend[2] = 0;
      } else {
        *s_abort = 1;
        atomicOr(p.status, 1);
      }
      phM ^= 1;
      tc_fence_after();
      if (tid == 0 && pb + 1 < npb && !*s_abort) {  // block pb+1's MMAs, block pb+2's copy
        bool ok = mma_b(pb + 1);
        if (ok && pb + 2 < npb) copy_b(pb + 2, phB ^ 1u);
        if (!ok) {
          *s_abort = 1;
          atomicOr(p.status, 1);
        }
      }
      if (pb + 1 < npb) phB ^= 1;
      const uint32_t tacc = trow + (uint32_t)(pb & 1) * 128u;
#pragma unroll 1
      for (int q = 0; q < 2; ++q) {
        float g[32];
        tmem_ld32(tacc + (uint32_t)(q * 32), g);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = cb + q * 32 + j;
          float v = nxr + np_[c] - 2.0f * g[j];
          if (c >= nc) v = INF;
          if (v < tv[TCA_K - 1]) {  // rare once the list holds near pivots
            int id = (int)(pc + c);
#pragma unroll
            for (int k = 0; k < TCA_K; ++k)
              if (v < tv[k]) {
                const float tvk = tv[k];
                const int tik = ti[k];
                tv[k] = v; ti[k] = id;
                v = tvk; id = tik;
              }
          }
        }
      }
      tc_fence_before();
      __syncthreads();  // np_ is rewritten next
    }
    // the two halves merged: h = 1 hands its list to h = 0.  Keys outside the merged list
    // are at least the fifth of the eight listed or either half's last listed one.
    __syncthreads();
    if (h == 1)
#pragma unroll
      for (int k = 0; k < TCA_K; ++k) half2[k * 128 + r] = make_float2(tv[k], __int_as_float(ti[k]));
    __syncthreads();
    if (h == 0 && r < nr && !*s_abort) {
      float lb = tv[TCA_K - 1];
#pragma unroll
      for (int k = 0; k < TCA_K; ++k) {
        const float2 w = half2[k * 128 + r];
        float v = w.x;
        int id = __float_as_int(w.y);
        if (k == TCA_K - 1) lb = fminf(lb, v);
#pragma unroll
        for (int q = 0; q < TCA_K; ++q)
          if (v < tv[q]) {
            const float tq = tv[q];
            const int iq = ti[q];
            tv[q] = v; ti[q] = id;
            v = tq; id = iq;
          }
        lb = fminf(lb, v);  // pushed out of the list
      }
      p.best1[xb + r] = hi_b(tv[0] + E, e);
      p.arg1[xb + r] = ti[0];
      p.best2[xb + r] = lo_b(tv[1] - E, e);  // a tie keeps tv[1] = tv[0]: re-decided exactly
#pragma unroll
      for (int k = 0; k < TCA_K; ++k) p.cand[(xb + r) * TCA_K + k] = ti[k];
      p.rest[xb + r] = lo_b(lb - E, e);
    }
  }
  __syncthreads();
  if (*s_abort && tid == 0) {
    const long long lim = p.spin > (1ll << 26) ? p.spin : (1ll << 26);
    for (int b = 0; b < 3; ++b)
      if (s_pend[b] && !mbar_wait(&bars[b], (uint32_t)s_par[b], lim)) atomicOr(p.status, 2);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, 256);
}

// ---- diagnostic: tensor-core keys of all pairs among at most 256 points -------------------
__global__ void __launch_bounds__(128, 1) tc_keys_kernel(const uint8_t* __restrict__ img,
                                                         const float* __restrict__ nrm, int64_t n, int Dp,
                                                         float* __restrict__ out, int* status, long long spin) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const uint32_t IMG = (uint32_t)tc_img_bytes(Dp);
  uint8_t* sA = sm;
  uint8_t* sB = sm + IMG;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + 2 * IMG);
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + 2 * IMG + 24);
  const int tid = threadIdx.x, warp = tid >> 5;
  const int64_t nb = (n + 127) / 128;
  if (warp == 0) {
    tmem_alloc(tslot, 128);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  uint32_t ph0 = 0, ph1 = 0;
  bool ok = true;
  for (int64_t bx = 0; bx < nb && ok; ++bx)
    for (int64_t by = 0; by < nb && ok; ++by) {
      __syncthreads();
      if (tid == 0) {
        fence_proxy_async();
        mbar_expect_tx(&bars[0], 2 * IMG);
        bulk_g2s(sA, img + (size_t)bx * IMG, IMG, &bars[0]);
        bulk_g2s(sB, img + (size_t)by * IMG, IMG, &bars[0]);
        if (mbar_wait(&bars[0], ph0, spin)) {
          tc_fence_after();
          issue_gram_tile(tbase, sA, sB, Dp);
          umma_commit(&bars[1]);
        } else {
          atomicOr(status, 1);
        }
      }
      ph0 ^= 1;
      __syncthreads();
      if (*reinterpret_cast<volatile int*>(status)) { ok = false; break; }
      if (!mbar_wait(&bars[1], ph1, spin)) atomicOr(status, 1);
      ph1 ^= 1;
      tc_fence_after();
      __syncthreads();
      if (*reinterpret_cast<volatile int*>(status)) { ok = false; break; }
      const int64_t x = bx * 128 + tid;
      for (int q = 0; q < 4; ++q) {
        float g[32];
        tmem_ld32(tbase + ((uint32_t)(warp * 32) << 16) + (uint32_t)(q * 32), g);
        for (int j = 0; j < 32; ++j) {
          const int64_t y = by * 128 + q * 32 + j;
          if (x < n && y < n) out[x * n + y] = nrm[x] + nrm[y] - 2.0f * g[j];
        }
      }
      tc_fence_before();
    }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, 128);
}

// ---- host side ---------------------------------------------------------------------------
static int sm_count() {
  int dev = 0, sms = 0;
  GRNG_CUDA(cudaGetDevice(&dev));
  GRNG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  return sms;
}

bool tc_supported(int Dp) { return Dp % 16 == 0 && Dp >= 16 && tc_smem_bytes(Dp, GRNG_KMAX) <= 227 * 1024; }

float tc_gamma(int Dp) { return ldexpf(1.0f, -12) + (float)(3 * Dp + 16) * ldexpf(1.0f, -24); }

void tc_prepare(const float* X, int64_t n, int Dp, DevBuf& img, DevBuf& nrm, DevBuf& bmax, float* nmax_all,
                cudaStream_t s) {
  const int64_t nb = (n + 127) / 128;
  GRNG_CUDA(img.alloc((size_t)nb * tc_img_bytes(Dp)));
  GRNG_CUDA(nrm.alloc((size_t)n * 4));
  GRNG_CUDA(bmax.alloc((size_t)nb * 4));
  GRNG_CUDA(cudaMemsetAsync(img.p, 0, (size_t)nb * tc_img_bytes(Dp), s));
  GRNG_CUDA(cudaMemsetAsync(bmax.p, 0, (size_t)nb * 4, s));
  tc_prep_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, n, Dp, img.as<uint8_t>(), nrm.as<float>(),
                                                             bmax.as<unsigned int>()); note_launch();
  GRNG_CUDA(cudaGetLastError());
  if (nmax_all) {
    std::vector<unsigned int> h((size_t)nb);
    GRNG_CUDA(cudaMemcpyAsync(h.data(), bmax.p, (size_t)nb * 4, cudaMemcpyDeviceToHost, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    float m = 0.0f;
    for (unsigned int v : h) {
      float f;
      memcpy(&f, &v, 4);
      m = std::max(m, f);
    }
    *nmax_all = m;
  }
}

void tc_sweep(const TcLaunch& L, cudaStream_t s) {
  TcParams p;
  p.img = L.img; p.nrm = L.nrm; p.bmax = L.bmax; p.n = L.n; p.Dp = L.Dp; p.K = L.K;
  p.gam = tc_gamma(L.Dp); p.nmax_all = L.nmax_all;
  p.parent = L.parent; p.gpar = L.gpar; p.gpar_words = L.gpar_words;
  p.A = L.A; p.nbr_idx = L.nbr_idx; p.nbr_key = L.nbr_key;
  p.knn_idx = L.knn_idx; p.knn_key = L.knn_key; p.knn_rb = L.knn_rb;
  p.surv = L.surv; p.surv_cnt = L.surv_cnt; p.surv_cap = L.surv_cap;
  p.strip_ctr = L.strip_ctr; p.stats = L.stats; p.status = L.status; p.spin = L.spin;
  const size_t smem = tc_smem_bytes(L.Dp, L.K);
  GRNG_CUDA(cudaFuncSetAttribute(tc_sweep_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t nb = (L.n + 127) / 128;
  const int grid = (int)std::min<int64_t>(nb, sm_count());
  tc_sweep_kernel<<<grid, 256, smem, s>>>(p); note_launch();
  GRNG_CUDA(cudaGetLastError());
}

void tc_assign(const float* Xm, int64_t nmem, const float* Xp, int64_t m, int Dp, float* best1, int32_t* arg1,
               float* best2, int32_t* cand, float* rest, long long spin, cudaStream_t s, cudaEvent_t start,
               cudaEvent_t done) {
  DevBuf imgX, nX, bX, imgP, nP, bP, ctr;
  float pmax = 0.0f;
  tc_prepare(Xm, nmem, Dp, imgX, nX, bX, nullptr, s);
  tc_prepare(Xp, m, Dp, imgP, nP, bP, &pmax, s);
  GRNG_CUDA(ctr.alloc(16));
  GRNG_CUDA(cudaMemsetAsync(ctr.p, 0, 16, s));
  TcAssignParams p;
  p.imgX = imgX.as<uint8_t>(); p.nX = nX.as<float>(); p.bmaxX = bX.as<unsigned int>();
  p.imgP = imgP.as<uint8_t>(); p.nP = nP.as<float>();
  p.nmem = nmem; p.m = m; p.Dp = Dp; p.gam = tc_gamma(Dp); p.pmax = pmax;
  p.best1 = best1; p.arg1 = arg1; p.best2 = best2; p.cand = cand; p.rest = rest;
  p.strip_ctr = ctr.as<int>(); p.status = ctr.as<int>() + 1; p.spin = spin;
  const size_t smem = tc_assign_smem(Dp);
  GRNG_CUDA(cudaFuncSetAttribute(tc_assign_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  const int64_t nbx = (nmem + 127) / 128;
  if (start) GRNG_CUDA(cudaEventRecord(start, s));
  tc_assign_kernel<<<(unsigned)std::min<int64_t>(nbx, sm_count()), 256, smem, s>>>(p); note_launch();
  GRNG_CUDA(cudaGetLastError());
  if (done) GRNG_CUDA(cudaEventRecord(done, s));
  int st = 0;
  GRNG_CUDA(cudaMemcpyAsync(&st, ctr.as<int>() + 1, 4, cudaMemcpyDeviceToHost, s));
  GRNG_CUDA(cudaStreamSynchronize(s));
  if (st) fail(4 /* GRNG_ETIMEOUT */, "a bounded tensor-core wait ran out");
}

void tc_knn_fix(const float* X, int64_t n, int Dp, int K, int metric, const int32_t* knn_idx, float* knn_key,
                cudaStream_t s) {
  const int64_t tot = n * K;
  tc_knn_fix_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, n, Dp, K, metric, knn_idx, knn_key); note_launch();
  GRNG_CUDA(cudaGetLastError());
}

}  // namespace grng

// Diagnostic entry point (see include/grng.h): tensor-core keys of all pairs of at most
// 256 points, for checking the MMA path against plain arithmetic.
extern "C" grng_status grng_tc_keys(const float* pts, int64_t n, int32_t dim, float* keys) {
  using namespace grng;
  try {
    if (!pts || !keys || n < 1 || n > 256 || dim < 1 || dim > 128) fail(GRNG_EINVAL, "need 1 <= n <= 256, 1 <= dim <= 128");
    const int Dp = ((dim + 15) / 16) * 16;
    cudaStream_t s = nullptr;
    DevBuf X, img, nrm, bmax, out, st;
    GRNG_CUDA(X.alloc((size_t)n * Dp * 4));
    GRNG_CUDA(cudaMemsetAsync(X.p, 0, (size_t)n * Dp * 4, s));
    GRNG_CUDA(cudaMemcpy2DAsync(X.p, (size_t)Dp * 4, pts, (size_t)dim * 4, (size_t)dim * 4, (size_t)n,
                                cudaMemcpyDefault, s));
    tc_prepare(X.as<float>(), n, Dp, img, nrm, bmax, nullptr, s);
    GRNG_CUDA(out.alloc((size_t)n * n * 4));
    GRNG_CUDA(st.alloc(16));
    GRNG_CUDA(cudaMemsetAsync(st.p, 0, 16, s));
    const size_t smem = 2 * tc_img_bytes(Dp) + 64;
    GRNG_CUDA(cudaFuncSetAttribute(tc_keys_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    tc_keys_kernel<<<1, 128, smem, s>>>(img.as<uint8_t>(), nrm.as<float>(), n, Dp, out.as<float>(), st.as<int>(),
                                        1ll << 26); note_launch();
    GRNG_CUDA(cudaGetLastError());
    int hs = 0;
    GRNG_CUDA(cudaMemcpyAsync(&hs, st.p, 4, cudaMemcpyDeviceToHost, s));
    GRNG_CUDA(cudaMemcpyAsync(keys, out.p, (size_t)n * n * 4, cudaMemcpyDefault, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    if (hs) fail(GRNG_ETIMEOUT, "a bounded tensor-core wait ran out");
    set_last_error("");
    return GRNG_OK;
  } catch (const Failure& f) {
    set_last_error(f.msg);
    return f.status;
  } catch (...) {
    set_last_error("unexpected internal exception");
    return GRNG_EINTERNAL;
  }
}
