// kernels_mlp.cu -- the learned form: a ranking network that proposes likely
// interceptors for the exemplar pairs the exact tiers leave to the exhaustive
// Stage VI search.  It extends the paper's Stage V ("select group" of likely
// interceptors tried before Stage VI): each such pair scores a pool of candidates,
// tests the k best exactly, and only if none of them blocks goes on to the
// exhaustive tier as before -- the exact test of Eq. 1 decides every edge.
//
// Network: 32 features -> 128 ReLU -> 128 ReLU -> 1 logit.  Parameters (FP32, in this
// order): W1[128][32], b1[128], W2[128][128], b2[128], w3[128], b3.  Inference keeps
// the weights in shared memory as BF16 and accumulates in FP32; training runs the
// same network in FP32 with hand-written forward, backward and Adam kernels on the
// weighted logistic loss L = (1/N) sum_b w_b [log(1 + e^{s_b}) - y_b s_b].
//
// Candidate pool of a pair (g, o): for each endpoint e and each of its first
// GRNG_MLP_PW listed neighbours w, the K nodes of w's neighbour list (the pairs that
// reach this stage were already tested against g's and o's own lists).  Features use
// only stored quantities (list keys, parent distances and radii), never a new
// distance: the network has to guess which candidates fall inside the lune.
#include <cuda_bf16.h>

#include <algorithm>
#include <cstring>
#include <vector>

#include "../../include/grng.h"
#include "common.cuh"
#include "internal.h"

namespace grng {

#define FULLMASK 0xffffffffu
#define M_OFF_W1 0
#define M_OFF_B1 (M_OFF_W1 + GRNG_MLP_H * GRNG_MLP_IN)
#define M_OFF_W2 (M_OFF_B1 + GRNG_MLP_H)
#define M_OFF_B2 (M_OFF_W2 + GRNG_MLP_H * GRNG_MLP_H)
#define M_OFF_W3 (M_OFF_B2 + GRNG_MLP_H)
#define M_OFF_B3 (M_OFF_W3 + GRNG_MLP_H)
static_assert(M_OFF_B3 + 1 == GRNG_MLP_NPARAM, "parameter layout");

static __device__ __forceinline__ float minf_() { return __int_as_float(0xff800000); }
static __device__ __forceinline__ void push_pair_(int2* buf, unsigned long long* cnt, unsigned long long cap,
                                                  int2 v) {
  const unsigned long long pos = atomicAdd(cnt, 1ull);
  if (pos < cap) buf[pos] = v;
}
// shared-memory bytes of the weights, rounded so that what follows stays 16-byte aligned
#define MLPW_BYTES ((sizeof(MlpW) + 15) & ~(size_t)15)

// ---- inference: BF16 weights in shared memory, FP32 accumulation ---------------------------
struct MlpW {
  __nv_bfloat16 w1[GRNG_MLP_H * GRNG_MLP_IN];   // row = hidden unit
  __nv_bfloat16 w2t[GRNG_MLP_H * GRNG_MLP_H];   // transposed: row i = weights of input unit i
  float b1[GRNG_MLP_H], b2[GRNG_MLP_H], w3[GRNG_MLP_H];
  float b3;
};

__device__ void mlp_load_w(MlpW* m, const float* __restrict__ P) {
  for (int i = threadIdx.x; i < GRNG_MLP_H * GRNG_MLP_IN; i += blockDim.x)
    m->w1[i] = __float2bfloat16_rn(P[M_OFF_W1 + i]);
  for (int idx = threadIdx.x; idx < GRNG_MLP_H * GRNG_MLP_H; idx += blockDim.x) {
    const int j = idx / GRNG_MLP_H, i = idx % GRNG_MLP_H;
    m->w2t[i * GRNG_MLP_H + j] = __float2bfloat16_rn(P[M_OFF_W2 + idx]);
  }
  for (int j = threadIdx.x; j < GRNG_MLP_H; j += blockDim.x) {
    m->b1[j] = P[M_OFF_B1 + j];
    m->b2[j] = P[M_OFF_B2 + j];
    m->w3[j] = P[M_OFF_W3 + j];
  }
  if (threadIdx.x == 0) m->b3 = P[M_OFF_B3];
}

__device__ __forceinline__ float bf_lo(uint32_t u) { return __uint_as_float(u << 16); }
__device__ __forceinline__ float bf_hi(uint32_t u) { return __uint_as_float(u & 0xffff0000u); }

// logit of one sample; the second layer is accumulated unit by unit of the first so
// that only its 128 sums live in registers
__device__ float mlp_score(const MlpW* m, const float (&f)[GRNG_MLP_IN]) {
  float z2[GRNG_MLP_H];
#pragma unroll
  for (int j = 0; j < GRNG_MLP_H; ++j) z2[j] = m->b2[j];
#pragma unroll 1
  for (int i = 0; i < GRNG_MLP_H; ++i) {
    float a = m->b1[i];
    const uint4* r1 = reinterpret_cast<const uint4*>(m->w1 + i * GRNG_MLP_IN);
#pragma unroll
    for (int q = 0; q < GRNG_MLP_IN / 8; ++q) {
      const uint4 u = r1[q];
      a = fmaf(bf_lo(u.x), f[q * 8 + 0], a); a = fmaf(bf_hi(u.x), f[q * 8 + 1], a);
      a = fmaf(bf_lo(u.y), f[q * 8 + 2], a); a = fmaf(bf_hi(u.y), f[q * 8 + 3], a);
      a = fmaf(bf_lo(u.z), f[q * 8 + 4], a); a = fmaf(bf_hi(u.z), f[q * 8 + 5], a);
      a = fmaf(bf_lo(u.w), f[q * 8 + 6], a); a = fmaf(bf_hi(u.w), f[q * 8 + 7], a);
    }
    const float h = fmaxf(a, 0.0f);
    const uint4* r2 = reinterpret_cast<const uint4*>(m->w2t + i * GRNG_MLP_H);
#pragma unroll
    for (int q = 0; q < GRNG_MLP_H / 8; ++q) {
      const uint4 u = r2[q];
      z2[q * 8 + 0] = fmaf(bf_lo(u.x), h, z2[q * 8 + 0]); z2[q * 8 + 1] = fmaf(bf_hi(u.x), h, z2[q * 8 + 1]);
      z2[q * 8 + 2] = fmaf(bf_lo(u.y), h, z2[q * 8 + 2]); z2[q * 8 + 3] = fmaf(bf_hi(u.y), h, z2[q * 8 + 3]);
      z2[q * 8 + 4] = fmaf(bf_lo(u.z), h, z2[q * 8 + 4]); z2[q * 8 + 5] = fmaf(bf_hi(u.z), h, z2[q * 8 + 5]);
      z2[q * 8 + 6] = fmaf(bf_lo(u.w), h, z2[q * 8 + 6]); z2[q * 8 + 7] = fmaf(bf_hi(u.w), h, z2[q * 8 + 7]);
    }
  }
  float s = m->b3;
#pragma unroll
  for (int j = 0; j < GRNG_MLP_H; ++j) s = fmaf(m->w3[j], fmaxf(z2[j], 0.0f), s);
  return s;
}

__global__ void __launch_bounds__(256) mlp_score_kernel(const float* __restrict__ P, const float* __restrict__ X,
                                                        int64_t N, float* __restrict__ out) {
  extern __shared__ __align__(16) unsigned char smw[];
  MlpW* m = reinterpret_cast<MlpW*>(smw);
  mlp_load_w(m, P);
  __syncthreads();
  for (int64_t b = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; b < N; b += (int64_t)gridDim.x * blockDim.x) {
    float f[GRNG_MLP_IN];
#pragma unroll
    for (int k = 0; k < GRNG_MLP_IN; ++k) f[k] = X[b * GRNG_MLP_IN + k];
    out[b] = mlp_score(m, f);
  }
}

// ---- training (FP32) --------------------------------------------------------------------
// z1[b][j] = b1[j] + W1[j] . X[b]
__global__ void mlp_l1_kernel(const float* __restrict__ P, const float* __restrict__ X, int B,
                              float* __restrict__ z1) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * GRNG_MLP_H) return;
  const int b = t / GRNG_MLP_H, j = t % GRNG_MLP_H;
  float a = P[M_OFF_B1 + j];
  for (int k = 0; k < GRNG_MLP_IN; ++k) a = fmaf(P[M_OFF_W1 + j * GRNG_MLP_IN + k], X[b * GRNG_MLP_IN + k], a);
  z1[t] = a;
}
// z2[b][j] = b2[j] + W2[j] . relu(z1[b])
__global__ void mlp_l2_kernel(const float* __restrict__ P, const float* __restrict__ z1, int B,
                              float* __restrict__ z2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * GRNG_MLP_H) return;
  const int b = t / GRNG_MLP_H, j = t % GRNG_MLP_H;
  float a = P[M_OFF_B2 + j];
  for (int i = 0; i < GRNG_MLP_H; ++i)
    a = fmaf(P[M_OFF_W2 + j * GRNG_MLP_H + i], fmaxf(z1[b * GRNG_MLP_H + i], 0.0f), a);
  z2[t] = a;
}
// s[b], ds[b] = w_b (sigmoid(s) - y_b) / N, and the loss terms
__global__ void mlp_out_kernel(const float* __restrict__ P, const float* __restrict__ z2,
                               const float* __restrict__ y, const float* __restrict__ w, int B, float invN,
                               float* __restrict__ ds, float* __restrict__ lossb) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= B) return;
  float s = P[M_OFF_B3];
  for (int j = 0; j < GRNG_MLP_H; ++j) s = fmaf(P[M_OFF_W3 + j], fmaxf(z2[b * GRNG_MLP_H + j], 0.0f), s);
  const float wb = w ? w[b] : 1.0f;
  const float sp = s > 0.0f ? s + log1pf(expf(-s)) : log1pf(expf(s));
  lossb[b] = wb * (sp - y[b] * s);
  ds[b] = wb * (1.0f / (1.0f + expf(-s)) - y[b]) * invN;
}
// d2[b][j] = dL/dz2 = ds[b] w3[j] [z2 > 0]
__global__ void mlp_d2_kernel(const float* __restrict__ P, const float* __restrict__ z2,
                              const float* __restrict__ ds, int B, float* __restrict__ d2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * GRNG_MLP_H) return;
  const int b = t / GRNG_MLP_H, j = t % GRNG_MLP_H;
  d2[t] = z2[t] > 0.0f ? ds[b] * P[M_OFF_W3 + j] : 0.0f;
}
// d1[b][i] = dL/dz1 = (sum_j W2[j][i] d2[b][j]) [z1 > 0]
__global__ void mlp_d1_kernel(const float* __restrict__ P, const float* __restrict__ z1,
                              const float* __restrict__ d2, int B, float* __restrict__ d1) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= B * GRNG_MLP_H) return;
  const int b = t / GRNG_MLP_H, i = t % GRNG_MLP_H;
  float a = 0.0f;
  for (int j = 0; j < GRNG_MLP_H; ++j) a = fmaf(P[M_OFF_W2 + j * GRNG_MLP_H + i], d2[b * GRNG_MLP_H + j], a);
  d1[t] = z1[t] > 0.0f ? a : 0.0f;
}
// every parameter's gradient, one thread each, summed over the batch in order
__global__ void mlp_wgrad_kernel(const float* __restrict__ X, const float* __restrict__ z1,
                                 const float* __restrict__ z2, const float* __restrict__ ds,
                                 const float* __restrict__ d1, const float* __restrict__ d2, int B,
                                 float* __restrict__ G) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= GRNG_MLP_NPARAM) return;
  float a = 0.0f;
  if (t < M_OFF_B1) {
    const int j = t / GRNG_MLP_IN, k = t % GRNG_MLP_IN;
    for (int b = 0; b < B; ++b) a = fmaf(d1[b * GRNG_MLP_H + j], X[b * GRNG_MLP_IN + k], a);
  } else if (t < M_OFF_W2) {
    const int j = t - M_OFF_B1;
    for (int b = 0; b < B; ++b) a += d1[b * GRNG_MLP_H + j];
  } else if (t < M_OFF_B2) {
    const int j = (t - M_OFF_W2) / GRNG_MLP_H, i = (t - M_OFF_W2) % GRNG_MLP_H;
    for (int b = 0; b < B; ++b) a = fmaf(d2[b * GRNG_MLP_H + j], fmaxf(z1[b * GRNG_MLP_H + i], 0.0f), a);
  } else if (t < M_OFF_W3) {
    const int j = t - M_OFF_B2;
    for (int b = 0; b < B; ++b) a += d2[b * GRNG_MLP_H + j];
  } else if (t < M_OFF_B3) {
    const int j = t - M_OFF_W3;
    for (int b = 0; b < B; ++b) a = fmaf(ds[b], fmaxf(z2[b * GRNG_MLP_H + j], 0.0f), a);
  } else {
    for (int b = 0; b < B; ++b) a += ds[b];
  }
  G[t] = a;
}
// Adam (Kingma & Ba) with bias correction
__global__ void mlp_adam_kernel(float* __restrict__ P, const float* __restrict__ G, float* __restrict__ M,
                                float* __restrict__ V, float lr, float c1, float c2) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= GRNG_MLP_NPARAM) return;
  const float g = G[t];
  const float m = 0.9f * M[t] + 0.1f * g;
  const float v = 0.999f * V[t] + 0.001f * g * g;
  M[t] = m;
  V[t] = v;
  P[t] -= lr * (m / c1) / (sqrtf(v / c2) + 1e-8f);
}

namespace {
struct MlpBatchBufs {
  DevBuf z1, z2, d1, d2, ds, lb;
  void alloc(int B) {
    GRNG_CUDA(z1.alloc((size_t)B * GRNG_MLP_H * 4));
    GRNG_CUDA(z2.alloc((size_t)B * GRNG_MLP_H * 4));
    GRNG_CUDA(d1.alloc((size_t)B * GRNG_MLP_H * 4));
    GRNG_CUDA(d2.alloc((size_t)B * GRNG_MLP_H * 4));
    GRNG_CUDA(ds.alloc((size_t)B * 4));
    GRNG_CUDA(lb.alloc((size_t)B * 4));
  }
};
unsigned nb_(int64_t n) { return (unsigned)((n + 255) / 256); }

// gradient of the mean loss over the batch X[0..B) (divided by invN's N) into G
void mlp_batch_grad(const float* P, const float* X, const float* y, const float* w, int B, float invN,
                    MlpBatchBufs& t, float* G, cudaStream_t s) {
  const int BH = B * GRNG_MLP_H;
  mlp_l1_kernel<<<nb_(BH), 256, 0, s>>>(P, X, B, t.z1.as<float>()); note_launch();
  mlp_l2_kernel<<<nb_(BH), 256, 0, s>>>(P, t.z1.as<float>(), B, t.z2.as<float>()); note_launch();
  mlp_out_kernel<<<nb_(B), 256, 0, s>>>(P, t.z2.as<float>(), y, w, B, invN, t.ds.as<float>(), t.lb.as<float>()); note_launch();
  mlp_d2_kernel<<<nb_(BH), 256, 0, s>>>(P, t.z2.as<float>(), t.ds.as<float>(), B, t.d2.as<float>()); note_launch();
  mlp_d1_kernel<<<nb_(BH), 256, 0, s>>>(P, t.z1.as<float>(), t.d2.as<float>(), B, t.d1.as<float>()); note_launch();
  mlp_wgrad_kernel<<<nb_(GRNG_MLP_NPARAM), 256, 0, s>>>(X, t.z1.as<float>(), t.z2.as<float>(), t.ds.as<float>(),
                                                         t.d1.as<float>(), t.d2.as<float>(), B, G); note_launch();
  GRNG_CUDA(cudaGetLastError());
}
}  // namespace

// ---- candidate pool and its features ------------------------------------------------------
struct PoolCtx {
  const int32_t* knn_idx;
  const float* knn_key;
  int K, metric;
  const int32_t* parent;
  const float* pdist_hi;
  const float* prad;
};

__device__ __forceinline__ uint32_t mix32(uint32_t h) {  // integer finaliser (xorshift-multiply)
  h ^= h >> 16; h *= 0x7feb352du;
  h ^= h >> 15; h *= 0x846ca68bu;
  h ^= h >> 16;
  return h;
}

// Candidate q of pair (g, o) (q < 2 * GRNG_MLP_PW * K): returns the node z, or -1, and
// its features f.  Distances are divided by d(g, o) and clamped to [0, 8].
// node z of candidate q of pair (g, o), or -1
__device__ __forceinline__ int mlp_pool_z(const PoolCtx& c, int g, int o, int q) {
  const int K = c.K;
  const int side = q / (GRNG_MLP_PW * K);
  const int j = (q / K) % GRNG_MLP_PW;
  if (j >= K) return -1;
  const int w = c.knn_idx[(int64_t)(side ? o : g) * K + j];
  if (w < 0) return -1;
  const int z = c.knn_idx[(int64_t)w * K + q % K];
  return (z < 0 || z == g || z == o) ? -1 : z;
}

// c_other / c_same: how often z occurs in the pool of the other endpoint / again in its own
__device__ int mlp_candidate(const PoolCtx& c, int g, int o, float dxy, int q, int c_other, int c_same,
                             float (&f)[GRNG_MLP_IN]) {
  const int K = c.K;
  const int side = q / (GRNG_MLP_PW * K);
  const int j = (q / K) % GRNG_MLP_PW;
  const int t = q % K;
  if (j >= K) return -1;
  const int e = side ? o : g;
  const int w = c.knn_idx[(int64_t)e * K + j];
  if (w < 0) return -1;
  const int z = c.knn_idx[(int64_t)w * K + t];
  if (z < 0 || z == g || z == o) return -1;
  const float inv = 1.0f / fmaxf(dxy, 1e-30f);
  auto dn = [&](float k) {
    const float d = c.metric == L2 ? sqrtf(fmaxf(k, 0.0f)) : fmaxf(k, 0.0f);
    return fminf(d * inv, 8.0f);
  };
  auto cl = [](float v) { return fminf(fmaxf(v, 0.0f), 8.0f); };
  const float dew = dn(c.knn_key[(int64_t)e * K + j]), dwz = dn(c.knn_key[(int64_t)w * K + t]);
  const int az = c.parent ? c.parent[z] : 0, ag = c.parent ? c.parent[g] : 0, ao = c.parent ? c.parent[o] : 0;
  f[0] = (float)side;
  f[1] = (float)j / GRNG_MLP_PW;
  f[2] = (float)t / K;
  f[3] = dew;
  f[4] = dwz;
  f[5] = fabsf(dew - dwz);  // triangle bounds of d(e, z)
  f[6] = fminf(dew + dwz, 8.0f);
  f[7] = c.pdist_hi ? cl(c.pdist_hi[z] * inv) : 0.0f;
  f[8] = c.pdist_hi ? cl(c.pdist_hi[g] * inv) : 0.0f;
  f[9] = c.pdist_hi ? cl(c.pdist_hi[o] * inv) : 0.0f;
  f[10] = az == ag ? 1.0f : 0.0f;
  f[11] = az == ao ? 1.0f : 0.0f;
  f[12] = ag == ao ? 1.0f : 0.0f;
  f[13] = c.prad ? cl(c.prad[az] * inv) : 0.0f;
  f[14] = c.prad ? cl(c.prad[ag] * inv) : 0.0f;
  f[15] = c.prad ? cl(c.prad[ao] * inv) : 0.0f;
  f[16] = dn(c.knn_key[(int64_t)g * K + K - 1]);
  f[17] = dn(c.knn_key[(int64_t)o * K + K - 1]);
  f[18] = dn(c.knn_key[(int64_t)w * K + K - 1]);
  f[19] = (w == (side ? g : o)) ? 1.0f : 0.0f;
  f[20] = log2f(fmaxf(dxy, 1e-30f)) * 0.125f;
  const uint32_t h = mix32((uint32_t)az * 0x9E3779B1u ^ mix32((uint32_t)(side ? ao : ag)));
#pragma unroll
  for (int b = 0; b < 8; ++b) f[21 + b] = ((h >> b) & 1u) ? 1.0f : -1.0f;
  f[29] = c_other > 0 ? 1.0f : 0.0f;  // reached from both endpoints: near both
  f[30] = (float)min(c_other, 8) * 0.125f;
  f[31] = (float)min(c_same, 8) * 0.125f;
  return z;
}

// ---- the stage: one CTA per pair --------------------------------------------------------------
#define MLP_POOL_MAX (2 * GRNG_MLP_PW * GRNG_KMAX)

__global__ void __launch_bounds__(256, 1) mlp_stage_kernel(MlpStage p) {
  extern __shared__ __align__(16) unsigned char smm[];
  MlpW* W = reinterpret_cast<MlpW*>(smm);
  float* gs = reinterpret_cast<float*>(smm + (p.params ? MLPW_BYTES : 0));
  float* os = gs + p.Dp;
  __shared__ float s_score[MLP_POOL_MAX];
  __shared__ int s_z[MLP_POOL_MAX];
  __shared__ int s_sel[GRNG_MLP_KMAX];
  __shared__ unsigned long long s_best;
  __shared__ float s_v;
  __shared__ int s_block, s_nsel, s_pos;
  const int tid = threadIdx.x, lane = tid & 31;
  const Err e = err_fp32(p.Dp);
  const PoolCtx pc{p.knn_idx, p.knn_key, p.K, p.metric, p.parent, p.pdist_hi, p.prad};
  const int Q = 2 * GRNG_MLP_PW * p.K;
  unsigned long long n_scored = 0, n_test = 0, n_blk = 0;
  if (p.params) mlp_load_w(W, p.params);
  for (int64_t t = blockIdx.x; t < p.m; t += gridDim.x) {
    const int2 pr = p.pairs[t];
    const int g = pr.x, o = pr.y;
    __syncthreads();
    for (int d = tid; d < p.Dp; d += blockDim.x) {
      gs[d] = p.X[(int64_t)g * p.Dp + d];
      os[d] = p.X[(int64_t)o * p.Dp + d];
    }
    if (tid == 0) { s_block = 0; s_nsel = 0; }
    __syncthreads();
    if (tid == 0) s_v = key32(gs, os, p.Dp, p.metric);
    __syncthreads();
    const float v = s_v;
    const float dxy = p.metric == L2 ? sqrtf(fmaxf(v, 0.0f)) : v;
    const PairThr P = pair_thresholds(v, 0.0f, 0.0f, 0.0f, 0.0f, p.metric, e, 0);
    for (int q = tid; q < MLP_POOL_MAX; q += blockDim.x) s_z[q] = q < Q ? mlp_pool_z(pc, g, o, q) : -1;
    if (tid == 0) s_pos = 0;
    __syncthreads();
    const int half = GRNG_MLP_PW * p.K;
    for (int q = tid; q < MLP_POOL_MAX; q += blockDim.x) {
      float f[GRNG_MLP_IN];
      int z = s_z[q];
      if (z >= 0) {
        const int mine = q < half ? 0 : half, other = q < half ? half : 0;
        int c_other = 0, c_same = 0;
        for (int r = 0; r < half; ++r) {
          c_other += s_z[other + r] == z;
          c_same += s_z[mine + r] == z;
        }
        z = mlp_candidate(pc, g, o, dxy, q, c_other, c_same - 1, f);
      }
      if (p.rec_f && z >= 0) {
        // training sample: does z block (g, o)?  (FP32 keys; a label, not a decision)
        const float* pz = p.X + (int64_t)z * p.Dp;
        const float a = key32(pz, gs, p.Dp, p.metric), b = key32(pz, os, p.Dp, p.metric);
        const unsigned long long r = atomicAdd(p.rec_cnt, 1ull);
        if (r < p.rec_cap) {
          for (int k = 0; k < GRNG_MLP_IN; ++k) p.rec_f[r * GRNG_MLP_IN + k] = f[k];
          p.rec_y[r] = fmaxf(a, b) < v ? 1.0f : 0.0f;
        }
        if (fmaxf(a, b) < v) s_pos = 1;
      }
      if (p.params) {
        s_score[q] = z >= 0 ? mlp_score(W, f) : minf_();
        n_scored += z >= 0;
      }
    }
    __syncthreads();
    if (tid == 0 && s_pos) atomicAdd(p.stats + 4, 1ull);  // pairs with a blocker in the pool
    if (!p.params || P.quick) continue;
    // ---- the k best distinct candidates ----
    for (int r = 0; r < p.kshort; ++r) {
      __syncthreads();
      if (tid == 0) s_best = 0ull;
      __syncthreads();
      unsigned long long best = 0ull;  // (order-preserving bits of the score) << 32 | ~q
      for (int q = tid; q < MLP_POOL_MAX; q += blockDim.x) {
        const float sc = s_score[q];
        if (sc == minf_()) continue;
        const uint32_t u = __float_as_uint(sc);
        const uint32_t key = (u & 0x80000000u) ? ~u : (u | 0x80000000u);
        const unsigned long long k64 = ((unsigned long long)key << 32) | (uint32_t)(~q);
        best = k64 > best ? k64 : best;
      }
      for (int sh = 16; sh > 0; sh >>= 1) {
        const unsigned long long y = __shfl_xor_sync(FULLMASK, best, sh);
        best = y > best ? y : best;
      }
      if (lane == 0 && best) atomicMax(&s_best, best);
      __syncthreads();
      if (s_best == 0ull) break;  // uniform
      const int qb = (int)(~(uint32_t)(s_best & 0xffffffffu));
      const int zb = s_z[qb];
      if (tid == 0) s_sel[s_nsel++] = zb;
      __syncthreads();
      for (int q = tid; q < MLP_POOL_MAX; q += blockDim.x)
        if (s_z[q] == zb) s_score[q] = minf_();
    }
    __syncthreads();
    // ---- exact tests of the shortlist ----
    const int nsel = s_nsel;
    if (tid < nsel) {
      const int z = s_sel[tid];
      const float* pz = p.X + (int64_t)z * p.Dp;
      const float a = key32(pz, gs, p.Dp, p.metric), b = key32(pz, os, p.Dp, p.metric);
      const int stt = block_state(a, b, P, e);
      if (stt == 2) s_block = 1;
      else if (stt == 1) push_pair_(p.amb, p.amb_cnt, p.amb_cap, make_int2((int)(p.slot0 + t), z));
    }
    n_test += tid < nsel;
    __syncthreads();
    if (tid == 0 && s_block) {
      p.pflag[p.slot0 + t] = 3;
      ++n_blk;
    }
  }
  for (int sh = 16; sh > 0; sh >>= 1) {
    n_scored += __shfl_down_sync(FULLMASK, n_scored, sh);
    n_test += __shfl_down_sync(FULLMASK, n_test, sh);
  }
  if (lane == 0 && (n_scored || n_test)) {
    atomicAdd(p.stats + 0, n_scored);
    atomicAdd(p.stats + 1, n_test);
  }
  if (tid == 0 && n_blk) atomicAdd(p.stats + 2, n_blk);
}

void mlp_stage(const MlpStage& P, cudaStream_t s) {
  if (P.m <= 0) return;
  if (P.K < 1 || P.K > GRNG_KMAX || P.kshort < 0 || P.kshort > GRNG_MLP_KMAX)
    fail(GRNG_EINVAL, "shortlist length must be in [0, 16]");
  const size_t smem = (P.params ? MLPW_BYTES : 0) + (size_t)2 * P.Dp * 4;
  GRNG_CUDA(cudaFuncSetAttribute(mlp_stage_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0;
  GRNG_CUDA(cudaGetDevice(&dev));
  GRNG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  const int grid = (int)std::min<int64_t>(P.m, (int64_t)sms);
  mlp_stage_kernel<<<grid, 256, smem, s>>>(P); note_launch();
  GRNG_CUDA(cudaGetLastError());
}

}  // namespace grng

// ---- C ABI: training, scoring and the gradient check (see include/grng.h) ---------------------
using namespace grng;

namespace {
template <class F>
grng_status mlp_guard(F&& fn) {
  try {
    fn();
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
void to_dev(DevBuf& d, const void* src, size_t bytes, cudaStream_t s) {
  GRNG_CUDA(d.alloc(bytes));
  GRNG_CUDA(cudaMemcpyAsync(d.p, src, bytes, cudaMemcpyDefault, s));
}
}  // namespace

extern "C" int64_t grng_mlp_nparams(void) { return GRNG_MLP_NPARAM; }

extern "C" grng_status grng_mlp_score(const float* params, const float* feats, int64_t n, float* scores) {
  return mlp_guard([&] {
    if (!params || !feats || !scores || n < 1) fail(GRNG_EINVAL, "params, feats and scores must be given, n >= 1");
    cudaStream_t s = nullptr;
    DevBuf P, X, out;
    to_dev(P, params, (size_t)GRNG_MLP_NPARAM * 4, s);
    to_dev(X, feats, (size_t)n * GRNG_MLP_IN * 4, s);
    GRNG_CUDA(out.alloc((size_t)n * 4));
    const size_t smem = MLPW_BYTES;
    GRNG_CUDA(cudaFuncSetAttribute(mlp_score_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    mlp_score_kernel<<<(unsigned)std::min<int64_t>((n + 255) / 256, 1024), 256, smem, s>>>(
        P.as<float>(), X.as<float>(), n, out.as<float>()); note_launch();
    GRNG_CUDA(cudaGetLastError());
    GRNG_CUDA(cudaMemcpyAsync(scores, out.p, (size_t)n * 4, cudaMemcpyDefault, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
  });
}

extern "C" grng_status grng_mlp_loss_grad(const float* params, const float* feats, const float* labels,
                                          const float* weights, int64_t n, float* loss, float* grad) {
  return mlp_guard([&] {
    if (!params || !feats || !labels || n < 1 || n > (1 << 20))
      fail(GRNG_EINVAL, "params, feats and labels must be given, 1 <= n <= 2^20");
    cudaStream_t s = nullptr;
    DevBuf P, X, Y, Wt, G;
    to_dev(P, params, (size_t)GRNG_MLP_NPARAM * 4, s);
    to_dev(X, feats, (size_t)n * GRNG_MLP_IN * 4, s);
    to_dev(Y, labels, (size_t)n * 4, s);
    if (weights) to_dev(Wt, weights, (size_t)n * 4, s);
    GRNG_CUDA(G.alloc((size_t)GRNG_MLP_NPARAM * 4));
    MlpBatchBufs t;
    t.alloc((int)n);
    mlp_batch_grad(P.as<float>(), X.as<float>(), Y.as<float>(), weights ? Wt.as<float>() : nullptr, (int)n,
                   1.0f / (float)n, t, G.as<float>(), s);
    std::vector<float> lb((size_t)n);
    GRNG_CUDA(cudaMemcpyAsync(lb.data(), t.lb.p, (size_t)n * 4, cudaMemcpyDeviceToHost, s));
    if (grad) GRNG_CUDA(cudaMemcpyAsync(grad, G.p, (size_t)GRNG_MLP_NPARAM * 4, cudaMemcpyDefault, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    double acc = 0.0;
    for (float v : lb) acc += v;
    if (loss) *loss = (float)(acc / (double)n);
  });
}

extern "C" grng_status grng_mlp_train(const float* feats, const float* labels, const float* weights, int64_t n,
                                      int32_t epochs, int32_t batch, float lr, float* params, float* loss_out) {
  return mlp_guard([&] {
    if (!params || !feats || !labels || n < 1 || epochs < 1 || batch < 1 || batch > 65536 || !(lr > 0.0f))
      fail(GRNG_EINVAL, "need params, feats, labels, n >= 1, epochs >= 1, 1 <= batch <= 65536, lr > 0");
    cudaStream_t s = nullptr;
    DevBuf P, X, Y, Wt, G, M, V;
    to_dev(P, params, (size_t)GRNG_MLP_NPARAM * 4, s);
    to_dev(X, feats, (size_t)n * GRNG_MLP_IN * 4, s);
    to_dev(Y, labels, (size_t)n * 4, s);
    if (weights) to_dev(Wt, weights, (size_t)n * 4, s);
    GRNG_CUDA(G.alloc((size_t)GRNG_MLP_NPARAM * 4));
    GRNG_CUDA(M.alloc((size_t)GRNG_MLP_NPARAM * 4));
    GRNG_CUDA(V.alloc((size_t)GRNG_MLP_NPARAM * 4));
    GRNG_CUDA(cudaMemsetAsync(M.p, 0, (size_t)GRNG_MLP_NPARAM * 4, s));
    GRNG_CUDA(cudaMemsetAsync(V.p, 0, (size_t)GRNG_MLP_NPARAM * 4, s));
    const int B = (int)std::min<int64_t>(batch, n);
    MlpBatchBufs t;
    t.alloc(B);
    long step = 0;
    double last = 0.0;
    for (int ep = 0; ep < epochs; ++ep) {
      double acc = 0.0;
      for (int64_t b0 = 0; b0 < n; b0 += B) {
        const int nb = (int)std::min<int64_t>(B, n - b0);
        mlp_batch_grad(P.as<float>(), X.as<float>() + b0 * GRNG_MLP_IN, Y.as<float>() + b0,
                       weights ? Wt.as<float>() + b0 : nullptr, nb, 1.0f / (float)nb, t, G.as<float>(), s);
        ++step;
        const float c1 = 1.0f - powf(0.9f, (float)step), c2 = 1.0f - powf(0.999f, (float)step);
        mlp_adam_kernel<<<nb_(GRNG_MLP_NPARAM), 256, 0, s>>>(P.as<float>(), G.as<float>(), M.as<float>(),
                                                              V.as<float>(), lr, c1, c2); note_launch();
        GRNG_CUDA(cudaGetLastError());
        if (ep == epochs - 1) {
          std::vector<float> lb((size_t)nb);
          GRNG_CUDA(cudaMemcpyAsync(lb.data(), t.lb.p, (size_t)nb * 4, cudaMemcpyDeviceToHost, s));
          GRNG_CUDA(cudaStreamSynchronize(s));
          for (float v : lb) acc += v;
        }
      }
      last = acc / (double)n;
    }
    GRNG_CUDA(cudaMemcpyAsync(params, P.p, (size_t)GRNG_MLP_NPARAM * 4, cudaMemcpyDefault, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    if (loss_out) *loss_out = (float)last;
  });
}
