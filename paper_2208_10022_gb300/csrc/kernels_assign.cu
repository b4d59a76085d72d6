// kernels_assign.cu -- one pivot layer (Eq. 2; relative pivot domain, Sec. 3):
// nearest pivot of every member (ties to the lowest pivot position, a pivot owns
// itself), FP64 member distance, radius = max(dist + member radius) and
// delta_max = max(dist).
//
// The member x pivot keys come from the FP32 distance tile, or, in the precision form for
// layers of 256 pivots or more, from split-BF16 Gram keys on the tensor cores
// (kernels_tc.cu), where each member keeps its four best candidates and a lower bound on
// the rest.  A member whose best key cannot be separated from the others under the error
// bound is re-decided in FP64 against every pivot whose key could tie the minimum.
#include <algorithm>
#include <mutex>
#include <string>

#include "../../include/grng.h"
#include "common.cuh"
#include "internal.h"
#include "tile.cuh"

namespace grng {

template <int KC, int METRIC>
__global__ void __launch_bounds__(GRNG_THREADS) assign_tile_kernel(const float* __restrict__ Xm, int64_t nmem,
                                                                   const float* __restrict__ Xp, int64_t m, int Dp,
                                                                   float* __restrict__ best1,
                                                                   int32_t* __restrict__ arg1,
                                                                   float* __restrict__ best2) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* sA = reinterpret_cast<float*>(sm_raw);
  float* sB = sA + KC * GRNG_SSTRIDE;
  float* T = sB + KC * GRNG_SSTRIDE;  // [128][129]
  const int64_t xb = (int64_t)blockIdx.x * GRNG_TILE;
  const int nr = (int)(nmem - xb < GRNG_TILE ? nmem - xb : GRNG_TILE);
  const int64_t npb = (m + GRNG_TILE - 1) / GRNG_TILE;
  const float inf = __int_as_float(0x7f800000);
  float m1 = inf, m2 = inf;
  int a1 = -1;
  for (int64_t pb = 0; pb < npb; ++pb) {
    const int nc = (int)(m - pb * GRNG_TILE < GRNG_TILE ? m - pb * GRNG_TILE : GRNG_TILE);
    float acc[8][8];
    tile_keys<KC, METRIC>(Xm + xb * Dp, nr, Xp + pb * GRNG_TILE * Dp, nc, Dp, sA, sB, acc);
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        int r = tile_row(i), c = tile_col(j);
        T[r * 129 + c] = (c < nc) ? acc[i][j] : inf;
      }
    __syncthreads();
    if (threadIdx.x < nr) {
      const float* Tr = T + threadIdx.x * 129;
      for (int c = 0; c < GRNG_TILE; ++c) {
        float v = Tr[c];
        if (v < m1) { m2 = m1; m1 = v; a1 = (int)(pb * GRNG_TILE + c); }
        else if (v < m2) m2 = v;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x < nr) {
    best1[xb + threadIdx.x] = m1;
    arg1[xb + threadIdx.x] = a1;
    best2[xb + threadIdx.x] = m2;
  }
}

// decide: self-assignment, certain argmin, or ambiguous (queued for FP64)
__global__ void assign_decide_kernel(const int32_t* __restrict__ mem_id, int64_t nmem,
                                     const int32_t* __restrict__ pivpos, const float* __restrict__ best1,
                                     const int32_t* __restrict__ arg1, const float* __restrict__ best2,
                                     int Dp, int32_t* __restrict__ assign, int32_t* __restrict__ amb,
                                     unsigned long long* __restrict__ amb_cnt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nmem) return;
  const int pp = pivpos[mem_id[t]];
  if (pp >= 0) { assign[t] = pp; return; }
  const Err e = err_fp32(Dp);
  if (hi_b(best1[t], e) < lo_b(best2[t], e)) {
    assign[t] = arg1[t];
  } else {
    assign[t] = -1;
    unsigned long long pos = atomicAdd(amb_cnt, 1ull);
    amb[pos] = (int32_t)t;
  }
}

// FP64 argmin over every pivot whose key could reach the FP32 minimum
__global__ void assign_recheck_kernel(const float* __restrict__ Xm, const float* __restrict__ Xp,
                                      int64_t m, int D, int Dp, int metric,
                                      const int32_t* __restrict__ amb, const float* __restrict__ best1,
                                      int32_t* __restrict__ assign, unsigned long long* __restrict__ n64) {
  __shared__ double sk[256];
  __shared__ int si[256];
  const int64_t t = amb[blockIdx.x];
  const float* x = Xm + t * Dp;
  const Err e = err_fp32(Dp);
  const float lim = hi_b(best1[t], e);
  double bk = 0.0;
  int bi = -1;
  unsigned long long cnt = 0;
  for (int64_t j = threadIdx.x; j < m; j += blockDim.x) {
    const float* pj = Xp + j * Dp;
    if (lo_b(key32(x, pj, Dp, metric), e) <= lim) {
      double k = key64(x, pj, D, metric);
      ++cnt;
      if (bi < 0 || k < bk) { bk = k; bi = (int)j; }  // j ascends per thread: ties keep the lowest
    }
  }
  sk[threadIdx.x] = bk;
  si[threadIdx.x] = bi;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      double k2 = sk[threadIdx.x + w];
      int i2 = si[threadIdx.x + w];
      if (i2 >= 0 && (si[threadIdx.x] < 0 || k2 < sk[threadIdx.x] ||
                      (k2 == sk[threadIdx.x] && i2 < si[threadIdx.x]))) {
        sk[threadIdx.x] = k2;
        si[threadIdx.x] = i2;
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) assign[t] = si[0];
  atomicAdd(n64, cnt);
}

// Tensor-core form: an undecided member whose four listed pivots include every pivot that
// could be nearest (every other pivot's key certainly above the smallest listed one's) is
// decided among those four -- FP32 keys with their brackets, canonical FP64 keys where the
// brackets overlap, ties to the lowest pivot position; the others go to the full recheck.
__global__ void assign_cand_kernel(const float* __restrict__ Xm, const float* __restrict__ Xp, int D, int Dp,
                                   int metric, const int32_t* __restrict__ amb, int64_t namb,
                                   const float* __restrict__ best1, const int32_t* __restrict__ cand,
                                   const float* __restrict__ rest, int32_t* __restrict__ assign,
                                   int32_t* __restrict__ amb2, unsigned long long* __restrict__ n2,
                                   unsigned long long* __restrict__ n64) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= namb) return;
  const int64_t t = amb[i];
  const Err e = err_fp32(Dp);
  const float lim = hi_b(best1[t], e);  // at least the smallest exact key
  if (!(rest[t] > lim)) {
    amb2[atomicAdd(n2, 1ull)] = (int32_t)t;
    return;
  }
  const float* x = Xm + t * Dp;
  float k32[4];
  float m32 = __int_as_float(0x7f800000);
  for (int k = 0; k < 4; ++k) {
    const int j = cand[t * 4 + k];
    k32[k] = j >= 0 ? key32(x, Xp + (int64_t)j * Dp, Dp, metric) : __int_as_float(0x7f800000);
    m32 = fminf(m32, hi_b(k32[k], e));
  }
  double bk = 0.0;
  int bi = -1;
  unsigned long long c64 = 0;
  for (int k = 0; k < 4; ++k) {
    const int j = cand[t * 4 + k];
    if (j < 0 || lo_b(k32[k], e) > m32) continue;  // certainly above another candidate's key
    const double kk = key64(x, Xp + (int64_t)j * Dp, D, metric);
    ++c64;
    if (bi < 0 || kk < bk || (kk == bk && j < bi)) { bk = kk; bi = j; }
  }
  assign[t] = bi;
  atomicAdd(n64, c64);
}

__global__ void member_dist_kernel(const float* __restrict__ Xm, const float* __restrict__ Xp,
                                   const double* __restrict__ mem_r, int64_t nmem, int D, int Dp,
                                   int metric, const int32_t* __restrict__ assign,
                                   double* __restrict__ dist, unsigned long long* __restrict__ radius,
                                   unsigned long long* __restrict__ delta) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nmem) return;
  const int p = assign[t];
  if (p < 0) return;  // cannot happen: the FP32 argmin always survives the recheck filter
  double d = dist_of_key64(key64(Xm + t * Dp, Xp + (int64_t)p * Dp, D, metric), metric);
  dist[t] = d;
  double rr = __dadd_rn(d, mem_r ? mem_r[t] : 0.0);
  atomicMax(radius + p, dbl_as_ull(rr));  // non-negative doubles order like their bits
  atomicMax(delta + p, dbl_as_ull(d));
}

__global__ void pivpos_kernel(const int32_t* __restrict__ piv_id, int64_t m, int32_t* __restrict__ pivpos) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j < m) pivpos[piv_id[j]] = (int32_t)j;
}

template <int KC>
static void launch_assign_tile(const float* Xm, int64_t nmem, const float* Xp, int64_t m, int Dp,
                               int metric, float* b1, int32_t* a1, float* b2, cudaStream_t s) {
  const size_t smem = (size_t)(2 * KC * GRNG_SSTRIDE + 128 * 129) * 4;
  const unsigned grid = (unsigned)((nmem + GRNG_TILE - 1) / GRNG_TILE);
  if (metric == L2) {
    GRNG_CUDA(cudaFuncSetAttribute(assign_tile_kernel<KC, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    assign_tile_kernel<KC, L2><<<grid, GRNG_THREADS, smem, s>>>(Xm, nmem, Xp, m, Dp, b1, a1, b2); note_launch();
  } else {
    GRNG_CUDA(cudaFuncSetAttribute(assign_tile_kernel<KC, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    assign_tile_kernel<KC, L1><<<grid, GRNG_THREADS, smem, s>>>(Xm, nmem, Xp, m, Dp, b1, a1, b2); note_launch();
  }
  GRNG_CUDA(cudaGetLastError());
}

void assign_layer(const float* Xmem, const int32_t* mem_id, const double* mem_r, int64_t nmem,
                  const float* Xpiv, const int32_t* piv_id, int64_t m, int64_t npoints, int D, int Dp,
                  int metric, const AssignOut& out, unsigned long long* stats, cudaStream_t s, bool tc,
                  long long spin) {
  if (nmem == 0 || m == 0) return;
  DevBuf pivpos, b1, a1, b2, amb, cnt, cand, rest, amb2;
  GRNG_CUDA(pivpos.alloc((size_t)npoints * 4));
  GRNG_CUDA(cudaMemsetAsync(pivpos.p, 0xff, (size_t)npoints * 4, s));
  pivpos_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(piv_id, m, pivpos.as<int32_t>()); note_launch();
  GRNG_CUDA(b1.alloc((size_t)nmem * 4));
  GRNG_CUDA(a1.alloc((size_t)nmem * 4));
  GRNG_CUDA(b2.alloc((size_t)nmem * 4));
  GRNG_CUDA(amb.alloc((size_t)nmem * 4));
  GRNG_CUDA(cnt.alloc(32));
  GRNG_CUDA(cudaMemsetAsync(cnt.p, 0, 32, s));
  const int KC = Dp % 32 == 0 ? 32 : (Dp % 16 == 0 ? 16 : 8);
  const bool use_tc = tc && metric == L2 && tc_supported(Dp) && m >= 256;  // two pivot blocks or more
  cudaEvent_t k0, k1;  // the member x pivot key kernel, on the launching stream
  GRNG_CUDA(cudaEventCreate(&k0));
  GRNG_CUDA(cudaEventCreate(&k1));
  if (!use_tc) GRNG_CUDA(cudaEventRecord(k0, s));
  if (use_tc) {
    GRNG_CUDA(cand.alloc((size_t)nmem * 16));
    GRNG_CUDA(rest.alloc((size_t)nmem * 4));
    tc_assign(Xmem, nmem, Xpiv, m, Dp, b1.as<float>(), a1.as<int32_t>(), b2.as<float>(), cand.as<int32_t>(),
              rest.as<float>(), spin, s, k0, k1);
  }
  else if (KC == 32) launch_assign_tile<32>(Xmem, nmem, Xpiv, m, Dp, metric, b1.as<float>(), a1.as<int32_t>(), b2.as<float>(), s);
  else if (KC == 16) launch_assign_tile<16>(Xmem, nmem, Xpiv, m, Dp, metric, b1.as<float>(), a1.as<int32_t>(), b2.as<float>(), s);
  else launch_assign_tile<8>(Xmem, nmem, Xpiv, m, Dp, metric, b1.as<float>(), a1.as<int32_t>(), b2.as<float>(), s);
  if (!use_tc) GRNG_CUDA(cudaEventRecord(k1, s));
  GRNG_CUDA(cudaEventSynchronize(k1));
  float kms = 0.0f;
  GRNG_CUDA(cudaEventElapsedTime(&kms, k0, k1));
  cudaEventDestroy(k0);
  cudaEventDestroy(k1);
  unsigned long long* dc = cnt.as<unsigned long long>();
  assign_decide_kernel<<<(unsigned)((nmem + 255) / 256), 256, 0, s>>>(
      mem_id, nmem, pivpos.as<int32_t>(), b1.as<float>(), a1.as<int32_t>(), b2.as<float>(), Dp, out.assign,
      amb.as<int32_t>(), dc); note_launch();
  GRNG_CUDA(cudaGetLastError());
  unsigned long long namb = 0;
  GRNG_CUDA(cudaMemcpyAsync(&namb, dc, 8, cudaMemcpyDeviceToHost, s));
  GRNG_CUDA(cudaStreamSynchronize(s));
  const int32_t* full = amb.as<int32_t>();  // members re-decided against every pivot
  if (namb && use_tc) {
    GRNG_CUDA(amb2.alloc((size_t)namb * 4));
    GRNG_CUDA(cudaMemsetAsync(dc + 2, 0, 8, s));
    assign_cand_kernel<<<(unsigned)((namb + 127) / 128), 128, 0, s>>>(
        Xmem, Xpiv, D, Dp, metric, amb.as<int32_t>(), (int64_t)namb, b1.as<float>(), cand.as<int32_t>(),
        rest.as<float>(), out.assign, amb2.as<int32_t>(), dc + 2, dc + 1); note_launch();
    GRNG_CUDA(cudaGetLastError());
    GRNG_CUDA(cudaMemcpyAsync(&namb, dc + 2, 8, cudaMemcpyDeviceToHost, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    full = amb2.as<int32_t>();
  }
  if (namb) {
    assign_recheck_kernel<<<(unsigned)namb, 256, 0, s>>>(Xmem, Xpiv, m, D, Dp, metric, full, b1.as<float>(),
                                                         out.assign, dc + 1); note_launch();
    GRNG_CUDA(cudaGetLastError());
  }
  GRNG_CUDA(cudaMemsetAsync(out.radius, 0, (size_t)m * 8, s));
  GRNG_CUDA(cudaMemsetAsync(out.delta_max, 0, (size_t)m * 8, s));
  member_dist_kernel<<<(unsigned)((nmem + 255) / 256), 256, 0, s>>>(
      Xmem, Xpiv, mem_r, nmem, D, Dp, metric, out.assign, out.dist,
      reinterpret_cast<unsigned long long*>(out.radius), reinterpret_cast<unsigned long long*>(out.delta_max)); note_launch();
  GRNG_CUDA(cudaGetLastError());
  if (stats) {
    unsigned long long h[2];
    GRNG_CUDA(cudaMemcpyAsync(h, dc, 16, cudaMemcpyDeviceToHost, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    stats[0] += h[0];  // ambiguous members
    stats[1] += h[1];  // FP64 member-pivot keys
    stats[2] += (unsigned long long)(kms * 1000.0f);  // key kernel, microseconds
    stats[3] = use_tc ? 1 : 0;
    unsigned long long hf = 0;
    if (use_tc) GRNG_CUDA(cudaMemcpyAsync(&hf, dc + 2, 8, cudaMemcpyDeviceToHost, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    stats[4] += hf;  // members re-decided against every pivot
  }
  GRNG_CUDA(cudaStreamSynchronize(s));
}

// ---------------------------------------------------------------------------------------
// Allocation-free nearest-pivot assignment (grng_assign_static in include/grng.h).
//
// Some callers cannot allocate device memory at all: code running inside a memory pool
// that forbids new allocations, plugins whose host owns every device allocation, or
// programs whose allocations must not change once they start.  For them the same
// assignment as grng_build_layer is available with every piece of scratch memory in one
// file-scope device array of fixed size.  That array lives in the library image, so
// every GPU that loads the library holds it until the process exits.
// ---------------------------------------------------------------------------------------
#define GRNG_STATIC_MAX_POINTS (1 << 18)         // members (points) per call
#define GRNG_STATIC_MAX_PIVOTS (1 << 16)         // pivots per call
#define GRNG_STATIC_MAX_PIVOT_FLOATS (1 << 21)   // pivots x dim
#define GRNG_STATIC_BYTES                                                                        \
  ((size_t)GRNG_STATIC_MAX_POINTS * 4 * 5 + (size_t)GRNG_STATIC_MAX_PIVOT_FLOATS * 4 +         \
   (size_t)GRNG_STATIC_MAX_PIVOTS * 8 * 2 + 256)

static __device__ __align__(256) unsigned char g_static_scratch[GRNG_STATIC_BYTES];

// pivot positions of the points; flags an index out of range or repeated
__global__ void static_pivpos_kernel(const int32_t* __restrict__ piv, int64_t m, int64_t n,
                                     int32_t* __restrict__ pivpos, int32_t* __restrict__ err) {
  const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const int32_t v = piv[j];
  if (v < 0 || v >= n) {
    atomicOr(err, 1);
    return;
  }
  if (atomicExch(pivpos + v, (int32_t)j) != -1) atomicOr(err, 2);
}

// as assign_decide_kernel, for members that are the points 0..n-1 themselves
__global__ void static_decide_kernel(int64_t n, const int32_t* __restrict__ pivpos, const float* __restrict__ best1,
                                     const int32_t* __restrict__ arg1, const float* __restrict__ best2, int Dp,
                                     int32_t* __restrict__ assign, int32_t* __restrict__ amb,
                                     unsigned long long* __restrict__ amb_cnt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= n) return;
  const int pp = pivpos[t];
  if (pp >= 0) { assign[t] = pp; return; }
  const Err e = err_fp32(Dp);
  if (hi_b(best1[t], e) < lo_b(best2[t], e)) {
    assign[t] = arg1[t];
  } else {
    assign[t] = -1;
    unsigned long long pos = atomicAdd(amb_cnt, 1ull);
    amb[pos] = (int32_t)t;
  }
}

// device address of the scratch array, looked up once per device (with that device current)
static void* static_scratch_address(int dev) {
  static std::mutex mu;
  static void* addr[64] = {nullptr};
  if (dev < 0 || dev >= 64) fail(1, "device ordinal out of range");
  std::lock_guard<std::mutex> lock(mu);
  if (!addr[dev]) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_static_scratch);
    if (e != cudaSuccess) {
      cudaGetLastError();
      fail(3, std::string("cudaGetSymbolAddress of the static scratch failed: ") + cudaGetErrorString(e));
    }
    addr[dev] = p;
  }
  return addr[dev];
}

// The kernels of the allocation-free call read and write the caller's buffers directly
// (float4 loads of the points, FP64 stores of the distances), so every buffer must be
// memory the device can address and must start on the boundary of its widest access.
static void check_device_buffer(const void* p, size_t align, const char* name) {
  if (reinterpret_cast<uintptr_t>(p) % align != 0)
    fail(1, std::string(name) + " must be aligned to " + std::to_string(align) + " bytes");
  cudaPointerAttributes at{};
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    fail(1, std::string(name) + " is not a pointer the CUDA runtime knows");
  }
  if (at.type != cudaMemoryTypeDevice && at.type != cudaMemoryTypeManaged)
    fail(1, std::string(name) + " must be device (or managed) memory");
  int dev = 0;
  GRNG_CUDA(cudaGetDevice(&dev));
  if (at.type == cudaMemoryTypeDevice && at.device != dev)
    fail(1, std::string(name) + " lives on another device than the current one");
}

void assign_static(const float* X, int64_t n, int dim, const int32_t* piv, int64_t m, int metric,
                   int32_t* assign, double* dist, cudaStream_t s) {
  if (!X || !piv || !assign || !dist) fail(1, "pointers must not be NULL");
  check_device_buffer(X, 16, "pts");
  check_device_buffer(piv, 4, "pivot_idx");
  check_device_buffer(assign, 4, "assign");
  check_device_buffer(dist, 8, "dist");
  if (metric != L2 && metric != L1) fail(1, "unknown metric");
  if (dim < 8 || dim % 8 != 0) fail(1, "dim must be a positive multiple of 8");
  if (n < 1 || n > GRNG_STATIC_MAX_POINTS) fail(1, "n must be in [1, 262144] for the allocation-free call");
  if (m < 1 || m > GRNG_STATIC_MAX_PIVOTS || m > n) fail(1, "m must be in [1, min(n, 65536)]");
  if (m * (int64_t)dim > GRNG_STATIC_MAX_PIVOT_FLOATS) fail(1, "m x dim must be at most 2097152");
  int dev = 0;
  GRNG_CUDA(cudaGetDevice(&dev));
  unsigned char* base = static_cast<unsigned char*>(static_scratch_address(dev));
  int32_t* pivpos = reinterpret_cast<int32_t*>(base);
  float* b1 = reinterpret_cast<float*>(pivpos + GRNG_STATIC_MAX_POINTS);
  int32_t* a1 = reinterpret_cast<int32_t*>(b1 + GRNG_STATIC_MAX_POINTS);
  float* b2 = reinterpret_cast<float*>(a1 + GRNG_STATIC_MAX_POINTS);
  int32_t* amb = reinterpret_cast<int32_t*>(b2 + GRNG_STATIC_MAX_POINTS);
  float* xp = reinterpret_cast<float*>(amb + GRNG_STATIC_MAX_POINTS);
  unsigned long long* radius = reinterpret_cast<unsigned long long*>(xp + GRNG_STATIC_MAX_PIVOT_FLOATS);
  unsigned long long* delta = radius + GRNG_STATIC_MAX_PIVOTS;
  unsigned long long* cnt = delta + GRNG_STATIC_MAX_PIVOTS;  // [0] ambiguous, [1] fp64 keys, [2] error
  int32_t* err = reinterpret_cast<int32_t*>(cnt + 2);
  // the array keeps the previous call's contents: clear what must start empty
  GRNG_CUDA(cudaMemsetAsync(pivpos, 0xff, (size_t)n * 4, s));
  GRNG_CUDA(cudaMemsetAsync(cnt, 0, 3 * sizeof(unsigned long long), s));
  static_pivpos_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(piv, m, n, pivpos, err); note_launch();
  GRNG_CUDA(cudaGetLastError());
  int32_t herr = 0;
  GRNG_CUDA(cudaMemcpyAsync(&herr, err, 4, cudaMemcpyDeviceToHost, s));
  GRNG_CUDA(cudaStreamSynchronize(s));
  if (herr & 1) fail(1, "pivot index out of range");
  if (herr & 2) fail(1, "duplicate pivot index");
  gather_rows(X, dim, piv, m, xp, s);
  const int KC = dim % 32 == 0 ? 32 : (dim % 16 == 0 ? 16 : 8);
  // members are the points 0..n-1 themselves: their ids are their positions, which the
  // decide kernel reads through mem_id; an identity map is not stored, so decide here
  if (KC == 32) launch_assign_tile<32>(X, n, xp, m, dim, metric, b1, a1, b2, s);
  else if (KC == 16) launch_assign_tile<16>(X, n, xp, m, dim, metric, b1, a1, b2, s);
  else launch_assign_tile<8>(X, n, xp, m, dim, metric, b1, a1, b2, s);
  static_decide_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(n, pivpos, b1, a1, b2, dim, assign, amb,
                                                                   cnt); note_launch();
  GRNG_CUDA(cudaGetLastError());
  unsigned long long namb = 0;
  GRNG_CUDA(cudaMemcpyAsync(&namb, cnt, 8, cudaMemcpyDeviceToHost, s));
  GRNG_CUDA(cudaStreamSynchronize(s));
  if (namb) {
    assign_recheck_kernel<<<(unsigned)namb, 256, 0, s>>>(X, xp, m, dim, dim, metric, amb, b1, assign, cnt + 1); note_launch();
    GRNG_CUDA(cudaGetLastError());
  }
  GRNG_CUDA(cudaMemsetAsync(radius, 0, (size_t)m * 8, s));
  GRNG_CUDA(cudaMemsetAsync(delta, 0, (size_t)m * 8, s));
  member_dist_kernel<<<(unsigned)((n + 255) / 256), 256, 0, s>>>(X, xp, nullptr, n, dim, dim, metric, assign, dist,
                                                                  radius, delta); note_launch();
  GRNG_CUDA(cudaGetLastError());
  GRNG_CUDA(cudaStreamSynchronize(s));
}

}  // namespace grng

extern "C" grng_status grng_assign_static(const float* pts, int64_t n, int32_t dim, const int32_t* pivot_idx,
                                          int32_t m, int32_t metric, int32_t* assign, double* dist,
                                          void* cuda_stream) {
  try {
    grng::assign_static(pts, n, dim, pivot_idx, m, metric, assign, dist, static_cast<cudaStream_t>(cuda_stream));
    grng::set_last_error("");
    return GRNG_OK;
  } catch (const grng::Failure& f) {
    grng::set_last_error(f.msg);
    return f.status;
  } catch (...) {
    grng::set_last_error("unexpected internal exception");
    return GRNG_EINTERNAL;
  }
}
