// tile.cuh -- FP32 CUDA-core distance tile (plain build): 128 x 128 keys per CTA.
//
// Each of the 256 threads owns an 8 x 8 sub-tile (rows {4ty..4ty+3, 64+4ty..}, columns
// {4tx..4tx+3, 64+4tx..}) so that the float4 shared-memory reads of one quarter-warp
// hit 8 distinct bank groups.  Coordinates stream through shared memory in chunks of
// KC dimensions, transposed to [KC][132]; the next chunk is prefetched into registers
// while the current one is consumed.  Keys accumulate over the dimensions in order,
// one FMA (L2) or one add of |a-b| (L1) per dimension, so T[x][y] and T[y][x] are
// bit-identical wherever they are computed.  L2 runs on packed pairs of columns (one packed
// subtraction and one packed FMA per pair), which round each half as the scalar forms do.
#pragma once
#include "common.cuh"

namespace grng {

#define GRNG_SSTRIDE 132

__device__ __forceinline__ float4 ldg4_or_zero(const float* p, bool ok) {
  return ok ? __ldg(reinterpret_cast<const float4*>(p)) : make_float4(0.f, 0.f, 0.f, 0.f);
}

// Packed pairs of FP32 values (sm_100 and later): each half is rounded exactly as the scalar
// operation rounds it, so a packed key equals the scalar one bit for bit.
__device__ __forceinline__ unsigned long long f2pack(float lo, float hi) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ void f2unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
// acc + (a - b)^2 per half: one packed subtraction, one packed FMA
__device__ __forceinline__ unsigned long long f2_sqdiff_acc(unsigned long long a, unsigned long long b,
                                                           unsigned long long acc) {
  unsigned long long t, r;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(t) : "l"(a), "l"(b));
  asm("fma.rn.f32x2 %0, %1, %1, %2;" : "=l"(r) : "l"(t), "l"(acc));
  return r;
}

__device__ __forceinline__ int tile_row(int i) {
  const int ty = threadIdx.x >> 4;
  return i < 4 ? ty * 4 + i : 64 + ty * 4 + (i - 4);
}
__device__ __forceinline__ int tile_col(int j) {
  const int tx = threadIdx.x & 15;
  return j < 4 ? tx * 4 + j : 64 + tx * 4 + (j - 4);
}

// acc[i][j] = key(row tile_row(i) of Xr, row tile_col(j) of Xc); rows beyond nr / nc
// are read as zeros (the caller masks them).  sA, sB: KC * GRNG_SSTRIDE floats each.
template <int KC, int METRIC>
__device__ __forceinline__ void tile_keys(const float* __restrict__ Xr, int nr,
                                          const float* __restrict__ Xc, int nc, int Dp,
                                          float* sA, float* sB, float (&acc)[8][8]) {
  constexpr int F4 = KC / 4;                               // float4 per row per chunk
  constexpr int LOADS = (GRNG_TILE * F4) / GRNG_THREADS;   // per thread per operand
  static_assert(LOADS >= 1, "chunk too small");
  const int tid = threadIdx.x;
  const int ty = tid >> 4, tx = tid & 15;
  float4 ra[LOADS], rb[LOADS];
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int j = 0; j < 8; ++j) acc[i][j] = 0.0f;
  unsigned long long acc2[8][4];  // L2: the accumulators as packed column pairs
#pragma unroll
  for (int i = 0; i < 8; ++i)
#pragma unroll
    for (int jp = 0; jp < 4; ++jp) acc2[i][jp] = 0ull;

  auto gload = [&](int k0) {
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      int idx = l * GRNG_THREADS + tid;
      int row = idx / F4, c4 = idx % F4;
      ra[l] = ldg4_or_zero(Xr + (int64_t)row * Dp + k0 + c4 * 4, row < nr);
      rb[l] = ldg4_or_zero(Xc + (int64_t)row * Dp + k0 + c4 * 4, row < nc);
    }
  };
  gload(0);
  for (int k0 = 0; k0 < Dp; k0 += KC) {
    __syncthreads();
#pragma unroll
    for (int l = 0; l < LOADS; ++l) {
      int idx = l * GRNG_THREADS + tid;
      int row = idx / F4, c4 = idx % F4;
      float* a = sA + (c4 * 4) * GRNG_SSTRIDE + row;
      float* b = sB + (c4 * 4) * GRNG_SSTRIDE + row;
      a[0] = ra[l].x; a[GRNG_SSTRIDE] = ra[l].y; a[2 * GRNG_SSTRIDE] = ra[l].z; a[3 * GRNG_SSTRIDE] = ra[l].w;
      b[0] = rb[l].x; b[GRNG_SSTRIDE] = rb[l].y; b[2 * GRNG_SSTRIDE] = rb[l].z; b[3 * GRNG_SSTRIDE] = rb[l].w;
    }
    __syncthreads();
    if (k0 + KC < Dp) gload(k0 + KC);
#pragma unroll
    for (int kk = 0; kk < KC; ++kk) {
      const float4 a0 = *reinterpret_cast<const float4*>(sA + kk * GRNG_SSTRIDE + ty * 4);
      const float4 a1 = *reinterpret_cast<const float4*>(sA + kk * GRNG_SSTRIDE + 64 + ty * 4);
      const float4 b0 = *reinterpret_cast<const float4*>(sB + kk * GRNG_SSTRIDE + tx * 4);
      const float4 b1 = *reinterpret_cast<const float4*>(sB + kk * GRNG_SSTRIDE + 64 + tx * 4);
      const float a[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
      if (METRIC == L2) {  // columns in packed pairs: half the instructions of the scalar loop
        const unsigned long long bp[4] = {f2pack(b0.x, b0.y), f2pack(b0.z, b0.w), f2pack(b1.x, b1.y),
                                          f2pack(b1.z, b1.w)};
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          const unsigned long long ap = f2pack(a[i], a[i]);
#pragma unroll
          for (int jp = 0; jp < 4; ++jp) acc2[i][jp] = f2_sqdiff_acc(ap, bp[jp], acc2[i][jp]);
        }
      } else {
        const float b[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
#pragma unroll
        for (int i = 0; i < 8; ++i)
#pragma unroll
          for (int j = 0; j < 8; ++j) acc[i][j] = acc[i][j] + fabsf(a[i] - b[j]);
      }
    }
  }
  if (METRIC == L2) {
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int jp = 0; jp < 4; ++jp) f2unpack(acc2[i][jp], acc[i][2 * jp], acc[i][2 * jp + 1]);
  }
}

}  // namespace grng
