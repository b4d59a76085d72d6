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
  unsigned long long* stats;  // [0] candidate pairs
  int* status;                // bit 0: a bounded wait ran out
  long long spin;
};

static __host__ __device__ constexpr size_t tc_img_bytes(int Dp) { return (size_t)128 * Dp * 4; }  // hi + lo
static __host__ __device__ constexpr size_t tc_t16_bytes() { return (size_t)128 * 130 * 2; }
static __host__ __device__ constexpr size_t tc_smem_bytes(int Dp, int K) {
  return 2 * tc_img_bytes(Dp) + (tc_img_bytes(Dp) >= tc_t16_bytes() ? 0 : tc_t16_bytes()) + 33280 + 32768 +
         (size_t)128 * (K + 1) * 8 + 128 * GRNG_KIN * 10 + 8 * 512 + 128;
}

__global__ void __launch_bounds__(128, 1) tc_sweep_kernel(TcParams p) {
  extern __shared__ __align__(1024) unsigned char sm[];
  const int Dp = p.Dp, K = p.K;
  const uint32_t IMG = (uint32_t)tc_img_bytes(Dp);
  uint8_t* sA = sm;
  uint8_t* sB = sm + IMG;
  size_t o = 2 * (size_t)IMG;
  __half* T16;
  if (IMG >= tc_t16_bytes()) {
    T16 = reinterpret_cast<__half*>(sB);  // the operand is dead once the MMA has completed
  } else {
    T16 = reinterpret_cast<__half*>(sm + o);
    o += tc_t16_bytes();
  }
  __half* AX = reinterpret_cast<__half*>(sm + o); o += 33280;   // [128][130]
  __half* AY = reinterpret_cast<__half*>(sm + o); o += 32768;   // [128][128]
  float* knnK = reinterpret_cast<float*>(sm + o); o += (size_t)128 * (K + 1) * 4;
  int* knnI = reinterpret_cast<int*>(sm + o); o += (size_t)128 * (K + 1) * 4;
  float* nbrXk = reinterpret_cast<float*>(sm + o); o += 128 * GRNG_KIN * 4;
  float* nbrYk = reinterpret_cast<float*>(sm + o); o += 128 * GRNG_KIN * 4;
  uint8_t* nbrXi = sm + o; o += 128 * GRNG_KIN;
  uint8_t* nbrYi = sm + o; o += 128 * GRNG_KIN;
  float* nx = reinterpret_cast<float*>(sm + o); o += 512;
  float* ny = reinterpret_cast<float*>(sm + o); o += 512;
  float* cmin1 = reinterpret_cast<float*>(sm + o); o += 512;
  float* cmin2 = reinterpret_cast<float*>(sm + o); o += 512;
  int* carg1 = reinterpret_cast<int*>(sm + o); o += 512;
  int* carg2 = reinterpret_cast<int*>(sm + o); o += 512;
  int* parX = reinterpret_cast<int*>(sm + o); o += 512;
  int* parY = reinterpret_cast<int*>(sm + o); o += 512;
  uint64_t* bars = reinterpret_cast<uint64_t*>(sm + o);           // A image, B image, MMA done
  uint32_t* tslot = reinterpret_cast<uint32_t*>(sm + o + 24);
  int* s_strip = reinterpret_cast<int*>(sm + o + 28);
  int* s_abort = reinterpret_cast<int*>(sm + o + 32);

  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int64_t n = p.n;
  const int64_t nb = (n + 127) / 128;
  const Err e = err_fp32(Dp);
  const float INF = finf_tc();
  unsigned long long st_cand = 0;

  if (warp == 0) {
    tmem_alloc(tslot, 128);
    tmem_relinquish();
  }
  if (tid == 0) {
    mbar_init(&bars[0], 1);
    mbar_init(&bars[1], 1);
    mbar_init(&bars[2], 1);
    *s_abort = 0;
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tbase = *tslot;
  const uint32_t trow = tbase + ((uint32_t)(warp * 32) << 16);  // this warp's 32 lanes
  uint32_t phA = 0, phB = 0, phM = 0;

  for (;;) {
    __syncthreads();
    if (tid == 0) *s_strip = atomicAdd(p.strip_ctr, 1);
    __syncthreads();
    const int64_t bx = *s_strip;
    if (bx >= nb || *s_abort) break;
    const int64_t xb = bx * 128;
    const int nr = (int)(n - xb < 128 ? n - xb : 128);
    if (tid == 0) {
      fence_proxy_async();
      mbar_expect_tx(&bars[0], IMG);
      bulk_g2s(sA, p.img + (size_t)bx * IMG, IMG, &bars[0]);
    }
    for (int i = tid; i < 128 * 128; i += 128) AX[(i >> 7) * 130 + (i & 127)] = p.A[bx * 16384 + i];
    for (int i = tid; i < 128 * GRNG_KIN; i += 128) {
      const bool ok = i / GRNG_KIN < nr;
      const int rr = i / GRNG_KIN, tt = i % GRNG_KIN;  // stored [t][row]: lanes = rows
      nbrXi[tt * 128 + rr] = ok ? p.nbr_idx[xb * GRNG_KIN + i] : (uint8_t)255;
      nbrXk[tt * 128 + rr] = ok ? p.nbr_key[xb * GRNG_KIN + i] : INF;
    }
    nx[tid] = tid < nr ? p.nrm[xb + tid] : 0.0f;
    parX[tid] = (p.parent && tid < nr) ? p.parent[xb + tid] : 0;
    for (int j = 0; j <= K; ++j) {
      knnK[tid * (K + 1) + j] = INF;
      knnI[tid * (K + 1) + j] = -1;
    }
    if (tid == 0 && !mbar_wait(&bars[0], phA, p.spin)) {
      *s_abort = 1;
      atomicOr(p.status, 1);
    }
    phA ^= 1;
    const float bmx = __uint_as_float(p.bmax[bx]);
    int done = 0;
    for (int s = 0; done < nb; ++s) {
      const int64_t off = (s & 1) ? (int64_t)((s + 1) >> 1) : -(int64_t)(s >> 1);
      const int64_t by = bx + off;
      if (by < 0 || by >= nb) continue;
      ++done;
      const int64_t yb = by * 128;
      const int nc = (int)(n - yb < 128 ? n - yb : 128);
      const bool filt = by >= bx;
      const bool diag = by == bx;
      // the previous tile's generic accesses to T16 (which may alias sB) are ordered
      // before the bulk copy that overwrites it: each thread fences, then all meet
      fence_proxy_async();
      __syncthreads();
      if (*s_abort) break;
      if (tid == 0) {
        mbar_expect_tx(&bars[1], IMG);
        bulk_g2s(sB, p.img + (size_t)by * IMG, IMG, &bars[1]);
      }
      ny[tid] = tid < nc ? p.nrm[yb + tid] : 0.0f;
      if (filt) {
        const uint4* src = reinterpret_cast<const uint4*>(p.A + by * 16384);
        uint4* dst = reinterpret_cast<uint4*>(AY);
        for (int i = tid; i < 16384 / 8; i += 128) dst[i] = src[i];
        for (int i = tid; i < 128 * GRNG_KIN; i += 128) {
          const bool ok = i / GRNG_KIN < nc;
          nbrYi[i] = ok ? p.nbr_idx[yb * GRNG_KIN + i] : (uint8_t)255;
          nbrYk[i] = ok ? p.nbr_key[yb * GRNG_KIN + i] : INF;
        }
        parY[tid] = (p.parent && tid < nc) ? p.parent[yb + tid] : 0;
      }
      if (tid == 0) {
        if (mbar_wait(&bars[1], phB, p.spin)) {
          tc_fence_after();
          issue_gram_tile(tbase, sA, sB, Dp);
          umma_commit(&bars[2]);
        } else {
          *s_abort = 1;
          atomicOr(p.status, 1);
        }
      }
      phB ^= 1;
      __syncthreads();
      if (*s_abort) break;
      if (!mbar_wait(&bars[2], phM, p.spin)) {
        *s_abort = 1;
        atomicOr(p.status, 1);
      }
      phM ^= 1;
      tc_fence_after();
      __syncthreads();
      if (*s_abort) break;
      // ---- keys -> T16, neighbour lists and row minima (thread = row) --------------------
      const int r = tid;
      const bool vr = r < nr;
      float m1 = INF, m2 = INF;
      int a1 = -1, a2 = -1;
      float* kk = knnK + r * (K + 1);
      int* ki = knnI + r * (K + 1);
      float thr = kk[K - 1];
      const float nxr = nx[r];
      for (int q = 0; q < 4; ++q) {
        float g[32];
        tmem_ld32(trow + (uint32_t)(q * 32), g);
#pragma unroll
        for (int j = 0; j < 32; ++j) {
          const int c = q * 32 + j;
          float v = nxr + ny[c] - 2.0f * g[j];
          if (!vr || c >= nc || (diag && c == r)) v = INF;
          T16[r * 130 + c] = __float2half_ru(v);
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
      }
      tc_fence_before();
      __syncthreads();
      if (filt) {
        // ---- column minima over the row block (thread = column) -----------------------
        {
          const int c = tid;
          float c1 = INF, c2 = INF;
          int b1 = -1, b2 = -1;
          for (int rr = 0; rr < 128; ++rr) {
            const float v = __half2float(T16[rr * 130 + c]);
            if (v < c2) {
              if (v < c1) { c2 = c1; b2 = b1; c1 = v; b1 = rr; }
              else { c2 = v; b2 = rr; }
            }
          }
          cmin1[c] = c1; cmin2[c] = c2; carg1[c] = b1; carg2[c] = b2;
        }
        __syncthreads();
        tc_fence_after();
        // ---- tier-1 filter: thread = row x, one column y at a time ------------------------
        const float E = p.gam * (bmx + __uint_as_float(p.bmax[by]));
        const int px = parX[r];
        for (int q = 0; q < 4; ++q) {
          float g[32];
          tmem_ld32(trow + (uint32_t)(q * 32), g);
#pragma unroll
          for (int j = 0; j < 32; ++j) {
            const int c = q * 32 + j;
            bool cand = vr && c < nc && (!diag || c > r);
            if (cand && p.gpar) {
              const int qy = parY[c];
              if (qy != px) {
                const int lo = min(px, qy), hi = max(px, qy);
                cand = (__ldg(p.gpar + (int64_t)lo * p.gpar_words + (hi >> 5)) >> (hi & 31)) & 1u;
              }
            }
            bool surv = false;
            if (cand) {
              ++st_cand;
              const float v = nxr + ny[c] - 2.0f * g[j];
              const float vlo = lo_b(v - E, e);  // below every key this pair can have
              bool blocked = false;
              {  // row minimum of x over the column block
                const int z = (a1 != c) ? a1 : a2;
                if (z >= 0) {
                  const float a = (a1 != c) ? m1 : m2;
                  blocked = hi_b(a + E, e) < vlo && hi_b(__half2float(AY[z * 128 + c]), e) < vlo;
                }
              }
              if (!blocked) {  // column minimum of y over the row block
                const int z = (carg1[c] != r) ? carg1[c] : carg2[c];
                if (z >= 0) {
                  const float b = (carg1[c] != r) ? cmin1[c] : cmin2[c];
                  blocked = hi_b(__half2float(AX[r * 130 + z]), e) < vlo && hi_b(b + E, e) < vlo;
                }
              }
              for (int t = 0; t < GRNG_KIN && !blocked; ++t) {  // neighbours of x
                const int z = nbrXi[t * 128 + r];
                if (z == 255) break;
                if (diag && z == c) continue;
                blocked = hi_b(nbrXk[t * 128 + r], e) < vlo &&
                          hi_b(__half2float(T16[z * 130 + c]) + E, e) < vlo;
              }
              for (int t = 0; t < GRNG_KIN && !blocked; ++t) {  // neighbours of y
                const int z = nbrYi[c * GRNG_KIN + t];
                if (z == 255) break;
                if (diag && z == r) continue;
                blocked = hi_b(__half2float(T16[r * 130 + z]) + E, e) < vlo &&
                          hi_b(nbrYk[c * GRNG_KIN + t], e) < vlo;
              }
              surv = !blocked;
            }
            const unsigned sm_ = __ballot_sync(FULLMASK, surv);
            if (sm_) {
              unsigned long long base = 0;
              if (lane == 0) base = atomicAdd(p.surv_cnt, (unsigned long long)__popc(sm_));
              base = __shfl_sync(FULLMASK, base, 0);
              if (surv) {
                const unsigned long long pos = base + __popc(sm_ & ((1u << lane) - 1u));
                if (pos < p.surv_cap) p.surv[pos] = make_int2((int)(xb + r), (int)(yb + c));
              }
            }
          }
        }
        tc_fence_before();
      }
    }
    __syncthreads();
    if (tid < nr) {
      const float* kkr = knnK + tid * (K + 1);
      const int* kir = knnI + tid * (K + 1);
      for (int j = 0; j < K; ++j) {
        p.knn_idx[(xb + tid) * K + j] = kir[j];
        p.knn_key[(xb + tid) * K + j] = kkr[j];
      }
      // every unlisted node z has tile key >= kkr[K-1], hence exact key >= that - E(x, z)
      p.knn_rb[xb + tid] = kir[K - 1] >= 0 ? kkr[K - 1] - p.gam * (nx[tid] + p.nmax_all) : INF;
    }
  }
  for (int o2 = 16; o2 > 0; o2 >>= 1) st_cand += __shfl_down_sync(FULLMASK, st_cand, o2);
  if (lane == 0) atomicAdd(p.stats, st_cand);
  // teardown: every tensor-core operation of this CTA has completed (or was never issued)
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0) tmem_dealloc(tbase, 128);
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
  tc_sweep_kernel<<<grid, 128, smem, s>>>(p); note_launch();
  GRNG_CUDA(cudaGetLastError());
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
    if (!pts || !keys || n < 1 || n > 256 || dim < 1 || dim > 96) fail(GRNG_EINVAL, "need 1 <= n <= 256, 1 <= dim <= 96");
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
