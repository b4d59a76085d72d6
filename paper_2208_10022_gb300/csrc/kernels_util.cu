// kernels_util.cu -- scans, grouping, sorting and adjacency extraction.
#include <algorithm>

#include "common.cuh"
#include "internal.h"

namespace grng {

#define FULLMASK 0xffffffffu

// ---- exclusive prefix sum of int64 (block scan + recursive block offsets) ----------
__global__ void scan_block_kernel(const int64_t* __restrict__ in, int64_t* __restrict__ out,
                                  int64_t n, int64_t* __restrict__ bsum) {
  __shared__ int64_t ws[32];
  const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
  const int64_t v = i < n ? in[i] : 0;
  int64_t x = v;
  for (int o = 1; o < 32; o <<= 1) {
    int64_t y = __shfl_up_sync(FULLMASK, x, o);
    if (lane >= o) x += y;
  }
  if (lane == 31) ws[w] = x;
  __syncthreads();
  if (w == 0) {
    int64_t s = ws[lane];
    for (int o = 1; o < 32; o <<= 1) {
      int64_t y = __shfl_up_sync(FULLMASK, s, o);
      if (lane >= o) s += y;
    }
    ws[lane] = s;
  }
  __syncthreads();
  const int64_t excl = x - v + (w > 0 ? ws[w - 1] : 0);
  if (i < n) out[i] = excl;
  if (threadIdx.x == 1023) bsum[blockIdx.x] = excl + v;
}
__global__ void scan_add_kernel(int64_t* __restrict__ out, int64_t n, const int64_t* __restrict__ boff) {
  const int64_t i = (int64_t)blockIdx.x * 1024 + threadIdx.x;
  if (i < n) out[i] += boff[blockIdx.x];
}
__global__ void scan_total_kernel(const int64_t* __restrict__ in, int64_t* __restrict__ out, int64_t n) {
  out[n] = n ? out[n - 1] + in[n - 1] : 0;
}

void exclusive_scan_i64(const int64_t* in, int64_t* out, int64_t n, cudaStream_t s) {
  if (n > 0) {
    const int64_t nb = (n + 1023) / 1024;
    DevBuf bs, bo;
    GRNG_CUDA(bs.alloc((size_t)(nb + 1) * 8));
    GRNG_CUDA(bo.alloc((size_t)(nb + 1) * 8));
    scan_block_kernel<<<(unsigned)nb, 1024, 0, s>>>(in, out, n, bs.as<int64_t>()); note_launch();
    GRNG_CUDA(cudaGetLastError());
    if (nb > 1) {
      exclusive_scan_i64(bs.as<int64_t>(), bo.as<int64_t>(), nb, s);
      scan_add_kernel<<<(unsigned)nb, 1024, 0, s>>>(out, n, bo.as<int64_t>()); note_launch();
      GRNG_CUDA(cudaGetLastError());
    }
    // the buffers must outlive the kernels that read them
    GRNG_CUDA(cudaStreamSynchronize(s));
  }
  scan_total_kernel<<<1, 1, 0, s>>>(in, out, n); note_launch();
  GRNG_CUDA(cudaGetLastError());
}

// ---- grouping of pairs by one component -------------------------------------------
__global__ void count_pairs_kernel(const int2* __restrict__ pr, int64_t m, int which,
                                   unsigned long long* __restrict__ cnt) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) atomicAdd(cnt + (which ? pr[i].y : pr[i].x), 1ull);
}
__global__ void scatter_pairs_kernel(const int2* __restrict__ pr, int64_t m, int which,
                                     unsigned long long* __restrict__ cur, int32_t* __restrict__ val) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    int2 p = pr[i];
    unsigned long long pos = atomicAdd(cur + (which ? p.y : p.x), 1ull);
    val[pos] = which ? p.x : p.y;
  }
}

void group_pairs(const int2* pairs, int64_t m, int which, int64_t nkeys, int64_t* off,
                 int32_t* val, DevBuf& tmp, cudaStream_t s) {
  GRNG_CUDA(tmp.alloc((size_t)(nkeys + 1) * 8));
  unsigned long long* cnt = tmp.as<unsigned long long>();
  GRNG_CUDA(cudaMemsetAsync(cnt, 0, (size_t)(nkeys + 1) * 8, s));
  if (m) {
    count_pairs_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(pairs, m, which, cnt); note_launch();
    GRNG_CUDA(cudaGetLastError());
  }
  exclusive_scan_i64(reinterpret_cast<const int64_t*>(cnt), off, nkeys, s);
  GRNG_CUDA(cudaMemcpyAsync(cnt, off, (size_t)nkeys * 8, cudaMemcpyDeviceToDevice, s));
  if (m) {
    scatter_pairs_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(pairs, m, which, cnt, val); note_launch();
    GRNG_CUDA(cudaGetLastError());
  }
  GRNG_CUDA(cudaStreamSynchronize(s));
}

// ---- bitonic sort of uint64 keys ------------------------------------------------------
__global__ void bitonic_global_kernel(uint64_t* __restrict__ a, int64_t n2, int64_t k, int64_t j) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;  // one per compared pair
  if (t >= n2 / 2) return;
  const int64_t i = (t / j) * 2 * j + (t % j);
  const int64_t l = i + j;
  const bool up = (i & k) == 0;
  uint64_t x = a[i], y = a[l];
  if ((x > y) == up) { a[i] = y; a[l] = x; }
}
// all steps with j < 1024 of one stage k, inside a 2048-element shared-memory block
__global__ void bitonic_shared_kernel(uint64_t* __restrict__ a, int64_t k, int64_t jstart) {
  __shared__ uint64_t s[2048];
  const int64_t base = (int64_t)blockIdx.x * 2048;
  s[threadIdx.x] = a[base + threadIdx.x];
  s[threadIdx.x + 1024] = a[base + threadIdx.x + 1024];
  __syncthreads();
  for (int64_t j = jstart; j > 0; j >>= 1) {
    const int t = threadIdx.x;
    const int i = (int)((t / j) * 2 * j + (t % j));
    const int l = i + (int)j;
    const bool up = ((base + i) & k) == 0;
    uint64_t x = s[i], y = s[l];
    if ((x > y) == up) { s[i] = y; s[l] = x; }
    __syncthreads();
  }
  a[base + threadIdx.x] = s[threadIdx.x];
  a[base + threadIdx.x + 1024] = s[threadIdx.x + 1024];
}
__global__ void fill_u64_kernel(uint64_t* a, int64_t from, int64_t to, uint64_t v) {
  const int64_t i = from + (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < to) a[i] = v;
}

void sort_u64(uint64_t* keys, int64_t m, DevBuf& tmp, cudaStream_t s) {
  if (m < 2) return;
  int64_t n2 = 2048;
  while (n2 < m) n2 <<= 1;
  GRNG_CUDA(tmp.alloc((size_t)n2 * 8));
  uint64_t* a = tmp.as<uint64_t>();
  GRNG_CUDA(cudaMemcpyAsync(a, keys, (size_t)m * 8, cudaMemcpyDeviceToDevice, s));
  if (n2 > m) {
    fill_u64_kernel<<<(unsigned)((n2 - m + 255) / 256), 256, 0, s>>>(a, m, n2, ~0ull); note_launch();
  }
  for (int64_t k = 2; k <= n2; k <<= 1) {
    int64_t j = k >> 1;
    for (; j >= 1024; j >>= 1) {
      bitonic_global_kernel<<<(unsigned)((n2 / 2 + 255) / 256), 256, 0, s>>>(a, n2, k, j); note_launch();
    }
    bitonic_shared_kernel<<<(unsigned)(n2 / 2048), 1024, 0, s>>>(a, k, j); note_launch();
  }
  GRNG_CUDA(cudaGetLastError());
  GRNG_CUDA(cudaMemcpyAsync(keys, a, (size_t)m * 8, cudaMemcpyDeviceToDevice, s));
  GRNG_CUDA(cudaStreamSynchronize(s));
}

// ---- stable order of items by key ------------------------------------------------------
__global__ void compose_keys_kernel(const int32_t* __restrict__ key, int64_t m, uint64_t* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) out[i] = ((uint64_t)(uint32_t)key[i] << 32) | (uint64_t)i;
}
__global__ void split_order_kernel(const uint64_t* __restrict__ k, int64_t m, int32_t* __restrict__ order,
                                   int32_t* __restrict__ rank) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < m) {
    int32_t item = (int32_t)(k[i] & 0xffffffffu);
    order[i] = item;
    rank[item] = (int32_t)i;
  }
}
void stable_order(const int32_t* key, int64_t m, int64_t nkeys, int32_t* order, int32_t* rank,
                  DevBuf& tmp, cudaStream_t s) {
  (void)nkeys;
  if (m == 0) return;
  DevBuf ks, t2;
  GRNG_CUDA(ks.alloc((size_t)m * 8));
  compose_keys_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(key, m, ks.as<uint64_t>()); note_launch();
  GRNG_CUDA(cudaGetLastError());
  sort_u64(ks.as<uint64_t>(), m, t2, s);
  split_order_kernel<<<(unsigned)((m + 255) / 256), 256, 0, s>>>(ks.as<uint64_t>(), m, order, rank); note_launch();
  GRNG_CUDA(cudaGetLastError());
  GRNG_CUDA(cudaStreamSynchronize(s));
  (void)tmp;
}

// ---- gathers and fills ---------------------------------------------------------------
__global__ void gather_rows_kernel(const float* __restrict__ X, int Dp, const int32_t* __restrict__ idx,
                                   int64_t m, float* __restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const int64_t tot = m * (Dp / 4);
  if (i < tot) {
    int64_t r = i / (Dp / 4), c = i % (Dp / 4);
    reinterpret_cast<float4*>(out)[i] = reinterpret_cast<const float4*>(X + (int64_t)idx[r] * Dp)[c];
  }
}
void gather_rows(const float* X, int Dp, const int32_t* idx, int64_t m, float* out, cudaStream_t s) {
  const int64_t tot = m * (Dp / 4);
  if (!tot) return;
  gather_rows_kernel<<<(unsigned)((tot + 255) / 256), 256, 0, s>>>(X, Dp, idx, m, out); note_launch();
  GRNG_CUDA(cudaGetLastError());
}
__global__ void fill_u32_kernel(uint32_t* p, uint32_t v, size_t count) {
  size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
  for (; i < count; i += (size_t)gridDim.x * blockDim.x) p[i] = v;
}
void fill_u32(uint32_t* p, uint32_t v, size_t count, cudaStream_t s) {
  if (!count) return;
  if (v == 0) {
    GRNG_CUDA(cudaMemsetAsync(p, 0, count * 4, s));
    return;
  }
  fill_u32_kernel<<<(unsigned)std::min<size_t>((count + 255) / 256, 65535), 256, 0, s>>>(p, v, count); note_launch();
  GRNG_CUDA(cudaGetLastError());
}

// ---- adjacency in original order from a triangular bitmask over sorted positions -----------
__device__ __forceinline__ bool tri_bit(const uint32_t* bits, int64_t words, int a, int b) {
  int lo = min(a, b), hi = max(a, b);
  return (__ldg(bits + (int64_t)lo * words + (hi >> 5)) >> (hi & 31)) & 1u;
}
__global__ void csr_count_kernel(const uint32_t* __restrict__ bits, int64_t words, const int32_t* __restrict__ rank,
                                 int64_t m, int64_t r0, int64_t r1, int64_t* __restrict__ cnt) {
  const int64_t row = r0 + (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= r1) return;
  const int si = rank[row];
  int64_t c = 0;
  for (int64_t j = lane; j < m; j += 32)
    if (j != row && tri_bit(bits, words, si, rank[j])) ++c;
  for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(FULLMASK, c, o);
  if (lane == 0) cnt[row - r0] = c;
}
__global__ void csr_write_kernel(const uint32_t* __restrict__ bits, int64_t words, const int32_t* __restrict__ rank,
                                 int64_t m, int64_t r0, int64_t r1, const int64_t* __restrict__ off,
                                 int32_t* __restrict__ adj) {
  const int64_t row = r0 + (int64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5);
  const int lane = threadIdx.x & 31;
  if (row >= r1) return;
  const int si = rank[row];
  int64_t pos = off[row - r0] - off[0];
  for (int64_t j0 = 0; j0 < m; j0 += 32) {
    const int64_t j = j0 + lane;
    const bool b = j < m && j != row && tri_bit(bits, words, si, rank[j]);
    const unsigned bm = __ballot_sync(FULLMASK, b);
    if (b) adj[pos + __popc(bm & ((1u << lane) - 1u))] = (int32_t)j;
    pos += __popc(bm);
  }
}
void bitmask_rows(const uint32_t* bits, int64_t words, const int32_t* rank, int64_t m, int64_t r0,
                  int64_t r1, int64_t* off, int32_t* adj, cudaStream_t s) {
  // off: device [r1-r0+1], relative offsets starting at off[0] = 0
  const int64_t rows = r1 - r0;
  if (rows <= 0) return;
  DevBuf cnt;
  GRNG_CUDA(cnt.alloc((size_t)rows * 8));
  csr_count_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(bits, words, rank, m, r0, r1, cnt.as<int64_t>()); note_launch();
  GRNG_CUDA(cudaGetLastError());
  exclusive_scan_i64(cnt.as<int64_t>(), off, rows, s);
  if (adj) {
    csr_write_kernel<<<(unsigned)((rows + 7) / 8), 256, 0, s>>>(bits, words, rank, m, r0, r1, off, adj); note_launch();
    GRNG_CUDA(cudaGetLastError());
  }
  GRNG_CUDA(cudaStreamSynchronize(s));
}
// cstart[c] = first s with parent[s] == c (parent non-decreasing); cstart[m] = n
__global__ void child_ranges_kernel(const int32_t* __restrict__ parent, int64_t n, int64_t m,
                                    int32_t* __restrict__ cstart) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s > n) return;
  const int64_t prev = s == 0 ? -1 : parent[s - 1];
  const int64_t cur = s == n ? m : parent[s];
  for (int64_t c = prev + 1; c <= cur; ++c) cstart[c] = (int32_t)s;
}
void child_ranges(const int32_t* parent, int64_t n, int64_t m, int32_t* cstart, cudaStream_t s) {
  child_ranges_kernel<<<(unsigned)((n + 1 + 255) / 256), 256, 0, s>>>(parent, n, m, cstart); note_launch();
  GRNG_CUDA(cudaGetLastError());
}

void bitmask_csr(const uint32_t* bits, int64_t words, const int32_t* rank, int64_t m, int64_t* off,
                 int32_t* adj, DevBuf& tmp, cudaStream_t s) {
  (void)tmp;
  bitmask_rows(bits, words, rank, m, 0, m, off, adj, s);
}

}  // namespace grng
