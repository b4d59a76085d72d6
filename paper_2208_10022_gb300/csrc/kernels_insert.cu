// kernels_insert.cu -- batched insertion (Algorithm 1 and Stage VII, Sec. 2): a batch of new
// points joins an index whose pivot layers, GRNGs and RNG are built, and only what the batch
// can change is recomputed.
//
//  - Radii.  Each new point joins its nearest finest pivot (Eq. 2); a finest radius grows when
//    the point lies beyond it, and a coarse radius R_c = max(d(c, pb) + rb) grows with its
//    members' radii (relative pivot domain, Sec. 3).  Radii never shrink.
//  - GRNGs.  Only the thresholds d - (2 r_i + r_j), d - (r_i + 2 r_j) of pairs with a grown
//    radius move, and they only fall, so a pair can only gain its link (definition, Sec. 2).
//    Re-tested: the pairs of every pivot whose radius grew that are not linked yet, and the
//    children of every coarse pair whose guidance link is new (Theorem 2 no longer excludes
//    them).  They go through the exhaustive tier; links are added, never removed.
//  - RNG.  New edges join a batch point: the batch rows are swept against every point in
//    distance tiles with the tier-1 filter of the build (Stage I candidates by Theorem 1,
//    select-group interceptors of Stage V) and keep their exact K nearest neighbours for
//    tier 2; what is left goes to the exhaustive tier.  Old edges lose their link when a
//    batch point lies strictly inside their lune (Stage VII): a point q can only enter the
//    lune of an edge (w, y) with key(q, w) < key(w, y), so only the old points w whose longest
//    edge reaches q are visited (the per-point maximum of Prop. 6), and each of their edges
//    is tested, in FP32 with the error bound and in canonical FP64 where the bound cannot
//    decide.
//
// RNG search (Algorithm 1 without Stage VII) shares the file: query rows are swept against
// every index point as batch rows are, but a query is not a point of the index, so no row
// ever blocks another row's pair and nothing of the index changes.
#include <algorithm>
#include <cstring>
#include <vector>

#include "common.cuh"
#include "internal.h"
#include "tile.cuh"

namespace grng {

#define FULLMASK 0xffffffffu
static __device__ __forceinline__ float inf_ins() { return __int_as_float(0x7f800000); }
static inline unsigned nblk_ins(int64_t m, int b = 256) { return (unsigned)((m + b - 1) / b); }

// ---- radii --------------------------------------------------------------------------------
// r = max(r, rb), dmax = max(dmax, db); changed[p] = 1 where r grew
__global__ void merge_radius_kernel(double* __restrict__ r, double* __restrict__ dmax, const double* __restrict__ rb,
                                    const double* __restrict__ db, int64_t m, uint8_t* __restrict__ changed) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= m) return;
  const double o = r[t], nb = rb[t];
  changed[t] = nb > o ? 1 : 0;
  if (nb > o) r[t] = nb;
  if (db[t] > dmax[t]) dmax[t] = db[t];
}

// R_c = max over members (d(c, member) + member radius), rounded as the build rounds it
__global__ void coarse_radius_kernel(const double* __restrict__ mdist, const double* __restrict__ mem_r,
                                     const int32_t* __restrict__ assign, int64_t nmem,
                                     unsigned long long* __restrict__ radius) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= nmem) return;
  const double rr = __dadd_rn(mdist[t], mem_r[t]);
  atomicMax(radius + assign[t], dbl_as_ull(rr));  // non-negative doubles order like their bits
}

__global__ void grew_kernel(const double* __restrict__ old_r, const double* __restrict__ new_r, int64_t m,
                            uint8_t* __restrict__ changed) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t < m) changed[t] = new_r[t] > old_r[t] ? 1 : 0;
}

// changed flags in sorted order, and the list of changed sorted positions
__global__ void changed_sorted_kernel(const uint8_t* __restrict__ changed, const int32_t* __restrict__ order,
                                      int64_t m, uint8_t* __restrict__ chg_s, int32_t* __restrict__ list,
                                      unsigned long long* __restrict__ cnt) {
  const int64_t s = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= m) return;
  const uint8_t c = changed[order[s]];
  chg_s[s] = c;
  if (c) list[atomicAdd(cnt, 1ull)] = (int32_t)s;
}

void merge_radii(double* r, double* dmax, const double* rb, const double* db, int64_t m, uint8_t* changed,
                 cudaStream_t s) {
  merge_radius_kernel<<<nblk_ins(m), 256, 0, s>>>(r, dmax, rb, db, m, changed); note_launch();
  GRNG_CUDA(cudaGetLastError());
}

void coarse_radii(const double* mdist, const double* mem_r, const int32_t* assign, int64_t nmem, double* radius,
                  const double* old_radius, int64_t m, uint8_t* changed, cudaStream_t s) {
  if (nmem)
    coarse_radius_kernel<<<nblk_ins(nmem), 256, 0, s>>>(mdist, mem_r, assign, nmem,
                                                        reinterpret_cast<unsigned long long*>(radius)); note_launch();
  grew_kernel<<<nblk_ins(m), 256, 0, s>>>(old_radius, radius, m, changed); note_launch();
  GRNG_CUDA(cudaGetLastError());
}

int64_t changed_sorted(const uint8_t* changed, const int32_t* order, int64_t m, uint8_t* chg_s, int32_t* list,
                       cudaStream_t s) {
  DevBuf c;
  GRNG_CUDA(c.alloc(8));
  GRNG_CUDA(cudaMemsetAsync(c.p, 0, 8, s));
  changed_sorted_kernel<<<nblk_ins(m), 256, 0, s>>>(changed, order, m, chg_s, list, c.as<unsigned long long>()); note_launch();
  GRNG_CUDA(cudaGetLastError());
  unsigned long long h = 0;
  GRNG_CUDA(cudaMemcpyAsync(&h, c.p, 8, cudaMemcpyDeviceToHost, s));
  GRNG_CUDA(cudaStreamSynchronize(s));
  return (int64_t)h;
}

// ---- GRNG pairs to re-test ------------------------------------------------------------------
__device__ __forceinline__ bool bit_of(const uint32_t* bits, int64_t words, int a, int b) {
  return (bits[(int64_t)a * words + (b >> 5)] >> (b & 31)) & 1u;
}

__device__ __forceinline__ void push_compact(bool keep, int2 v, int2* out, unsigned long long* cnt,
                                             unsigned long long cap) {
  const unsigned lane = threadIdx.x & 31;
  const unsigned bm = __ballot_sync(FULLMASK, keep);
  if (!bm) return;
  unsigned long long base = 0;
  if (lane == 0) base = atomicAdd(cnt, (unsigned long long)__popc(bm));
  base = __shfl_sync(FULLMASK, base, 0);
  if (keep) {
    const unsigned long long pos = base + __popc(bm & ((1u << lane) - 1u));
    if (pos < cap) out[pos] = v;
  }
}

// pairs (i, j) with i changed (one warp per i): not linked in both bitmasks yet, parents
// equal or linked in the coarser guidance graph; when both ends changed the lower one emits
__global__ void grng_changed_pairs_kernel(const int32_t* __restrict__ chg_list, int64_t nchg,
                                          const uint8_t* __restrict__ chg_s, int64_t m,
                                          const uint32_t* __restrict__ gx, const uint32_t* __restrict__ gg,
                                          int64_t words, const int32_t* __restrict__ parent,
                                          const uint32_t* __restrict__ gpar, int64_t gpar_words, int2* out,
                                          unsigned long long* cnt, unsigned long long cap) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = w0; w < nchg; w += nw) {
    const int i = chg_list[w];
    const int pi = parent ? parent[i] : 0;
    for (int64_t jb = 0; jb < m; jb += 32) {
      const int j = (int)(jb + lane);
      bool ok = j < m && j != i && !(j < m && chg_s[j] && j < i);
      const int a = min(i, j), b = max(i, j);
      if (ok) ok = !(bit_of(gx, words, a, b) && bit_of(gg, words, a, b));
      if (ok && parent) {
        const int pj = parent[j];
        if (pj != pi) ok = bit_of(gpar, gpar_words, min(pi, pj), max(pi, pj));
      }
      push_compact(ok, make_int2(a, b), out, cnt, cap);
    }
  }
}

// children pairs of coarse pairs whose guidance link is new (one warp per coarse pair)
__global__ void grng_child_pairs_kernel(const int2* __restrict__ newp, int64_t nnew,
                                        const int32_t* __restrict__ cstart, const uint32_t* __restrict__ gx,
                                        const uint32_t* __restrict__ gg, int64_t words, int2* out,
                                        unsigned long long* cnt, unsigned long long cap) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  for (int64_t w = w0; w < nnew; w += nw) {
    const int2 pp = newp[w];
    const int c0 = cstart[pp.x], c1 = cstart[pp.x + 1], d0 = cstart[pp.y], d1 = cstart[pp.y + 1];
    const int64_t nd = d1 - d0, tot = (int64_t)(c1 - c0) * nd;
    for (int64_t qb = 0; qb < tot; qb += 32) {
      const int64_t q = qb + lane;
      bool ok = q < tot;
      int a = 0, b = 0;
      if (ok) {
        const int i = c0 + (int)(q / nd), j = d0 + (int)(q % nd);
        a = min(i, j);
        b = max(i, j);
        ok = a != b && !(bit_of(gx, words, a, b) && bit_of(gg, words, a, b));
      }
      push_compact(ok, make_int2(a, b), out, cnt, cap);
    }
  }
}

int64_t grng_retest_pairs(const int32_t* chg_list, int64_t nchg, const uint8_t* chg_s, int64_t m, const uint32_t* gx,
                          const uint32_t* gg, int64_t words, const int32_t* parent, const uint32_t* gpar,
                          int64_t gpar_words, const int2* newp, int64_t nnew, const int32_t* cstart_par,
                          DevBuf& out, cudaStream_t s) {
  DevBuf c;
  GRNG_CUDA(c.alloc(8));
  unsigned long long cap = std::max<unsigned long long>(1 << 16, (unsigned long long)(nchg + nnew) * 64);
  for (int attempt = 0; attempt < 3; ++attempt) {
    GRNG_CUDA(out.alloc(cap * sizeof(int2)));
    GRNG_CUDA(cudaMemsetAsync(c.p, 0, 8, s));
    if (nchg) {
      grng_changed_pairs_kernel<<<(unsigned)std::min<int64_t>((nchg + 7) / 8, 4096), 256, 0, s>>>(
          chg_list, nchg, chg_s, m, gx, gg, words, parent, gpar, gpar_words, out.as<int2>(),
          c.as<unsigned long long>(), cap); note_launch();
    }
    if (nnew) {
      grng_child_pairs_kernel<<<(unsigned)std::min<int64_t>((nnew + 7) / 8, 4096), 256, 0, s>>>(
          newp, nnew, cstart_par, gx, gg, words, out.as<int2>(), c.as<unsigned long long>(), cap); note_launch();
    }
    GRNG_CUDA(cudaGetLastError());
    unsigned long long h = 0;
    GRNG_CUDA(cudaMemcpyAsync(&h, c.p, 8, cudaMemcpyDeviceToHost, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    if (h <= cap) return (int64_t)h;
    cap = h + h / 8;
  }
  fail(6, "re-test pair buffer overflow");
}

// ---- the batch rows against every point -----------------------------------------------------
struct InsertParams {
  const float* XB;          // [strips * 128][Dp] batch rows in sorted order, zero padded
  const int32_t* rowpos;    // [mb] sorted positions of the rows
  int64_t mb;
  const __half* AB;         // in-strip FP16 keys (rounded up) of the batch strips
  const uint8_t* nbrB_i;    // in-strip nearest neighbours of the rows
  const float* nbrB_k;
  const float* X;           // the level in sorted order [n][Dp]
  int64_t n;
  int Dp, K;
  const __half* A;          // in-block keys and neighbours of the level's 128-node blocks
  const uint8_t* nbr_i;
  const float* nbr_k;
  const uint8_t* is_new;    // [n] 1 for batch points
  const int32_t* parent;    // [n] finest pivot (sorted position)
  const uint32_t* gpar;     // finest layer's guidance bitmask
  int64_t gpar_words;
  const float* maxe;        // [n] FP32 upper bound of each old point's longest edge key (-1: none)
  int64_t bpc;              // column blocks per chunk
  int nchunks;
  float* knn_k;             // [mb_pad][nchunks][K] chunk-local lists of the rows
  int32_t* knn_i;
  int2* surv; unsigned long long* surv_cnt; unsigned long long surv_cap;
  int4* s7; unsigned long long* s7_cnt; unsigned long long s7_cap;  // (row pos, old pos, key bits, 0)
  unsigned long long* stats;  // [0] candidate pairs [1] Stage VII candidates
};

#define IS_U 66048  // max(2 * 32 * 132 * 4, 128 * 129 * 4): the operand chunks, then the key tile
static __host__ __device__ constexpr size_t is_bytes(int K) {
  return (size_t)IS_U + 2 * 32768 + (size_t)128 * (K + 1) * 8 + 128 * GRNG_KIN * 10 + 12 * 512 + 128;
}

template <int KC, int METRIC>
__global__ void __launch_bounds__(GRNG_THREADS, 1) insert_sweep_kernel(InsertParams p) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* sA = reinterpret_cast<float*>(sm_raw);
  float* sB = sA + KC * GRNG_SSTRIDE;
  float* T = reinterpret_cast<float*>(sm_raw);
  __half* AX = reinterpret_cast<__half*>(sm_raw + IS_U);
  __half* AY = AX + 128 * 128;
  const int K = p.K;
  float* knnK = reinterpret_cast<float*>(sm_raw + IS_U + 2 * 32768);
  int* knnI = reinterpret_cast<int*>(knnK + 128 * (K + 1));
  unsigned char* q = reinterpret_cast<unsigned char*>(knnI + 128 * (K + 1));
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
  int* rowp = reinterpret_cast<int*>(q); q += 512;
  int* newY = reinterpret_cast<int*>(q);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Dp = p.Dp;
  const int64_t xb = (int64_t)blockIdx.x * 128;  // first row of the strip
  const int nr = (int)(p.mb - xb < 128 ? p.mb - xb : 128);
  const int64_t nb = (p.n + 127) / 128;
  const int64_t by0 = (int64_t)blockIdx.y * p.bpc, by1 = min(nb, by0 + p.bpc);
  const Err e = err_fp32(Dp);
  unsigned long long st_cand = 0, st_s7 = 0;
  {
    const uint4* src = reinterpret_cast<const uint4*>(p.AB + blockIdx.x * 16384);
    uint4* dst = reinterpret_cast<uint4*>(AX);
    for (int i = tid; i < 16384 / 8; i += GRNG_THREADS) dst[i] = src[i];
    for (int i = tid; i < 128 * GRNG_KIN; i += GRNG_THREADS) {
      const bool ok = i / GRNG_KIN < nr;
      nbrXi[i] = ok ? p.nbrB_i[xb * GRNG_KIN + i] : (uint8_t)255;
      nbrXk[i] = ok ? p.nbrB_k[xb * GRNG_KIN + i] : inf_ins();
    }
    if (tid < 128) {
      rowp[tid] = tid < nr ? p.rowpos[xb + tid] : -1;
      parX[tid] = tid < nr ? p.parent[p.rowpos[xb + tid]] : 0;
    }
    for (int i = tid; i < 128 * (K + 1); i += GRNG_THREADS) {
      knnK[i] = inf_ins();
      knnI[i] = -1;
    }
  }
  for (int64_t by = by0; by < by1; ++by) {
    const int64_t yb = by * 128;
    const int nc = (int)(p.n - yb < 128 ? p.n - yb : 128);
    float acc[8][8];
    __syncthreads();
    tile_keys<KC, METRIC>(p.XB + xb * Dp, nr, p.X + yb * Dp, nc, Dp, sA, sB, acc);
    __syncthreads();  // every thread is done with sA/sB: T may overwrite them
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int r = tile_row(i), c = tile_col(j);
        float v = acc[i][j];
        if (r >= nr || c >= nc || rowp[r] == (int)(yb + c)) v = inf_ins();
        T[r * 129 + c] = v;
      }
    {
      const uint4* src = reinterpret_cast<const uint4*>(p.A + by * 16384);
      uint4* dst = reinterpret_cast<uint4*>(AY);
      for (int i = tid; i < 16384 / 8; i += GRNG_THREADS) dst[i] = src[i];
      for (int i = tid; i < 128 * GRNG_KIN; i += GRNG_THREADS) {
        const bool ok = i / GRNG_KIN < nc;
        nbrYi[i] = ok ? p.nbr_i[yb * GRNG_KIN + i] : (uint8_t)255;
        nbrYk[i] = ok ? p.nbr_k[yb * GRNG_KIN + i] : inf_ins();
      }
      if (tid < 128) {
        const bool ok = tid < nc;
        parY[tid] = ok ? p.parent[yb + tid] : 0;
        newY[tid] = ok ? p.is_new[yb + tid] : 1;
      }
    }
    __syncthreads();
    // ---- neighbour lists and row minima (thread = row), column minima (thread = column) ----
    if (tid < 128) {
      const int r = tid;
      if (r < nr) {
        float* kk = knnK + r * (K + 1);
        int* ki = knnI + r * (K + 1);
        float thr = kk[K - 1];
        float m1 = inf_ins(), m2 = inf_ins();
        int a1 = -1, a2 = -1;
        const float* Tr = T + r * 129;
        for (int c = 0; c < 128; ++c) {
          const float v = Tr[c];
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
    } else {
      const int c = tid - 128;
      float m1 = inf_ins(), m2 = inf_ins();
      int a1 = -1, a2 = -1;
      for (int r = 0; r < 128; ++r) {
        const float v = T[r * 129 + c];
        if (v < m2) {
          if (v < m1) { m2 = m1; a2 = a1; m1 = v; a1 = r; }
          else { m2 = v; a2 = r; }
        }
      }
      cmin1[c] = m1; cmin2[c] = m2; carg1[c] = a1; carg2[c] = a2;
    }
    __syncthreads();
    // ---- tier-1 filter of the candidate pairs (row x, column y); Stage VII candidates -------
    for (int rr = 0; rr < 16; ++rr) {
      const int r = warp * 16 + rr;
      if (r >= nr) break;
      const int x = rowp[r];
      const int px = parX[r];
      for (int cb = 0; cb < 4; ++cb) {
        if (cb * 32 >= nc) break;
        const int c = cb * 32 + lane;
        const int y = (int)(yb + c);
        const float v = c < nc ? T[r * 129 + c] : inf_ins();
        const bool valid = c < nc && v < inf_ins();
        // a pair of two batch points is taken from the row of its lower sorted position
        bool cand = valid && !(newY[c] && y < x);
        if (cand && p.gpar) {
          const int qy = parY[c];
          if (qy != px) {
            const int a = min(px, qy), b = max(px, qy);
            cand = (__ldg(p.gpar + (int64_t)a * p.gpar_words + (b >> 5)) >> (b & 31)) & 1u;
          }
        }
        bool surv = false;
        if (cand) {
          const PairThr P = pair_thresholds(v, 0.0f, 0.0f, 0.0f, 0.0f, METRIC, e, 0);
          bool blocked = false;
          {  // row minimum of x over the column block
            const int z = (rarg1[r] != c) ? rarg1[r] : rarg2[r];
            if (z >= 0) blocked = block_state(T[r * 129 + z], __half2float(AY[z * 128 + c]), P, e) == 2;
          }
          if (!blocked) {  // column minimum of y over the batch strip
            const int z = (carg1[c] != r) ? carg1[c] : carg2[c];
            if (z >= 0) blocked = block_state(__half2float(AX[r * 128 + z]), T[z * 129 + c], P, e) == 2;
          }
          for (int t = 0; t < GRNG_KIN && !blocked; ++t) {  // in-strip neighbours of x
            const int z = nbrXi[r * GRNG_KIN + t];
            if (z == 255) break;
            blocked = block_state(nbrXk[r * GRNG_KIN + t], T[z * 129 + c], P, e) == 2;
          }
          for (int t = 0; t < GRNG_KIN && !blocked; ++t) {  // in-block neighbours of y
            const int z = nbrYi[c * GRNG_KIN + t];
            if (z == 255) break;
            blocked = block_state(T[r * 129 + z], nbrYk[c * GRNG_KIN + t], P, e) == 2;
          }
          surv = !blocked;
        }
        st_cand += cand ? 1 : 0;
        {
          const unsigned sm = __ballot_sync(FULLMASK, surv);
          if (sm) {
            unsigned long long base = 0;
            if (lane == 0) base = atomicAdd(p.surv_cnt, (unsigned long long)__popc(sm));
            base = __shfl_sync(FULLMASK, base, 0);
            if (surv) {
              const unsigned long long pos = base + __popc(sm & ((1u << lane) - 1u));
              if (pos < p.surv_cap) p.surv[pos] = make_int2(x, y);
            }
          }
        }
        // Stage VII: x may lie in the lune of an old edge (y, w) only if key(x, y) < key(y, w)
        const bool s7 = valid && !newY[c] && lo_b(v, e) < p.maxe[y];
        st_s7 += s7 ? 1 : 0;
        const unsigned sm7 = __ballot_sync(FULLMASK, s7);
        if (sm7) {
          unsigned long long base = 0;
          if (lane == 0) base = atomicAdd(p.s7_cnt, (unsigned long long)__popc(sm7));
          base = __shfl_sync(FULLMASK, base, 0);
          if (s7) {
            const unsigned long long pos = base + __popc(sm7 & ((1u << lane) - 1u));
            if (pos < p.s7_cap) p.s7[pos] = make_int4(x, y, __float_as_int(v), 0);
          }
        }
      }
    }
  }
  __syncthreads();
  if (tid < nr) {
    const float* kk = knnK + tid * (K + 1);
    const int* ki = knnI + tid * (K + 1);
    const int64_t o = ((xb + tid) * p.nchunks + blockIdx.y) * K;
    for (int j = 0; j < K; ++j) {
      p.knn_k[o + j] = kk[j];
      p.knn_i[o + j] = ki[j];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    st_cand += __shfl_down_sync(FULLMASK, st_cand, o);
    st_s7 += __shfl_down_sync(FULLMASK, st_s7, o);
  }
  if (lane == 0) {
    atomicAdd(p.stats + 0, st_cand);
    atomicAdd(p.stats + 1, st_s7);
  }
}

// the rows' K nearest over all chunks, written at their sorted positions
__global__ void knn_merge_kernel(const float* __restrict__ ck, const int32_t* __restrict__ ci, int64_t mb,
                                 int nchunks, int K, const int32_t* __restrict__ rowpos, float* __restrict__ knn_k,
                                 int32_t* __restrict__ knn_i) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (r >= mb) return;
  float kk[GRNG_KMAX];
  int ki[GRNG_KMAX];
  for (int j = 0; j < K; ++j) { kk[j] = inf_ins(); ki[j] = -1; }
  for (int c = 0; c < nchunks; ++c) {
    const int64_t o = (r * nchunks + c) * K;
    for (int j = 0; j < K; ++j) {
      const float v = ck[o + j];
      if (!(v < kk[K - 1])) break;  // each chunk's list ascends
      int pos = K - 1;
      while (pos > 0 && kk[pos - 1] > v) { kk[pos] = kk[pos - 1]; ki[pos] = ki[pos - 1]; --pos; }
      kk[pos] = v;
      ki[pos] = ci[o + j];
    }
  }
  const int64_t d = (int64_t)rowpos[r] * K;
  for (int j = 0; j < K; ++j) {
    knn_k[d + j] = kk[j];
    knn_i[d + j] = ki[j];
  }
}

template <int KC>
static void launch_insert_kc(const InsertParams& p, int metric, unsigned strips, cudaStream_t s) {
  const size_t smem = is_bytes(p.K);
  dim3 grid(strips, (unsigned)p.nchunks);
  if (metric == L2) {
    GRNG_CUDA(cudaFuncSetAttribute(insert_sweep_kernel<KC, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    insert_sweep_kernel<KC, L2><<<grid, GRNG_THREADS, smem, s>>>(p); note_launch();
  } else {
    GRNG_CUDA(cudaFuncSetAttribute(insert_sweep_kernel<KC, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    insert_sweep_kernel<KC, L1><<<grid, GRNG_THREADS, smem, s>>>(p); note_launch();
  }
  GRNG_CUDA(cudaGetLastError());
}

void insert_sweep(const InsertSweep& S, DevBuf& surv, int64_t* nsurv, DevBuf& s7, int64_t* ns7, float* knn_k,
                  int32_t* knn_i, unsigned long long* stats, cudaStream_t s) {
  const int64_t nb = (S.n + 127) / 128;
  const unsigned strips = (unsigned)((S.mb + 127) / 128);
  int sms = 0, dev = 0;
  GRNG_CUDA(cudaGetDevice(&dev));
  GRNG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // enough CTAs to fill the GPU twice over, each with a contiguous range of column blocks
  const int64_t want = std::max<int64_t>(1, (2 * (int64_t)sms + strips - 1) / strips);
  const int64_t bpc = std::max<int64_t>(1, (nb + want - 1) / want);
  const int nchunks = (int)((nb + bpc - 1) / bpc);
  DevBuf ck, ci, ctr;
  GRNG_CUDA(ck.alloc((size_t)strips * 128 * nchunks * S.K * 4));
  GRNG_CUDA(ci.alloc((size_t)strips * 128 * nchunks * S.K * 4));
  GRNG_CUDA(ctr.alloc(4 * 8));
  unsigned long long scap = std::max<unsigned long long>(1 << 16, (unsigned long long)S.mb * 256);
  unsigned long long s7cap = std::max<unsigned long long>(1 << 16, (unsigned long long)S.mb * 64);
  for (int attempt = 0;; ++attempt) {
    GRNG_CUDA(surv.alloc(scap * sizeof(int2)));
    GRNG_CUDA(s7.alloc(s7cap * sizeof(int4)));
    GRNG_CUDA(cudaMemsetAsync(ctr.p, 0, 4 * 8, s));
    InsertParams p;
    p.XB = S.XB; p.rowpos = S.rowpos; p.mb = S.mb; p.AB = S.AB; p.nbrB_i = S.nbrB_i; p.nbrB_k = S.nbrB_k;
    p.X = S.X; p.n = S.n; p.Dp = S.Dp; p.K = S.K; p.A = S.A; p.nbr_i = S.nbr_i; p.nbr_k = S.nbr_k;
    p.is_new = S.is_new; p.parent = S.parent; p.gpar = S.gpar; p.gpar_words = S.gpar_words; p.maxe = S.maxe;
    p.bpc = bpc; p.nchunks = nchunks; p.knn_k = ck.as<float>(); p.knn_i = ci.as<int32_t>();
    unsigned long long* dc = ctr.as<unsigned long long>();
    p.surv = surv.as<int2>(); p.surv_cnt = dc; p.surv_cap = scap;
    p.s7 = s7.as<int4>(); p.s7_cnt = dc + 1; p.s7_cap = s7cap;
    p.stats = dc + 2;
    const int KC = S.Dp % 32 == 0 ? 32 : (S.Dp % 16 == 0 ? 16 : 8);
    if (KC == 32) launch_insert_kc<32>(p, S.metric, strips, s);
    else if (KC == 16) launch_insert_kc<16>(p, S.metric, strips, s);
    else launch_insert_kc<8>(p, S.metric, strips, s);
    unsigned long long h[4];
    GRNG_CUDA(cudaMemcpyAsync(h, dc, sizeof(h), cudaMemcpyDeviceToHost, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    if (h[0] <= scap && h[1] <= s7cap) {
      *nsurv = (int64_t)h[0];
      *ns7 = (int64_t)h[1];
      if (stats) { stats[0] += h[2]; stats[1] += h[3]; }
      break;
    }
    if (attempt >= 3) fail(6, "insertion sweep buffer overflow");
    scap = std::max(scap, h[0] + h[0] / 8);
    s7cap = std::max(s7cap, h[1] + h[1] / 8);
  }
  knn_merge_kernel<<<nblk_ins(S.mb), 256, 0, s>>>(ck.as<float>(), ci.as<int32_t>(), S.mb, nchunks, S.K, S.rowpos,
                                                   knn_k, knn_i); note_launch();
  GRNG_CUDA(cudaGetLastError());
  GRNG_CUDA(cudaStreamSynchronize(s));
}

// ---- search: query rows against every index point ---------------------------------------------
// One CTA takes a strip of 128 queries and a contiguous range of the index's 128-point column
// blocks.  Per tile: the FP32 keys (direct differences, as the build's tiles), then each
// query's two nearest points of the block and its K nearest so far (two threads per row, each
// with its own list over half the columns), then the tier-1 filter: Theorem 1 on the queries
// that lie in their pivot's ball, and a uniform test of every pair (q, y) against the block
// point nearest to q; the pairs it leaves are queued in shared memory and tested by all threads
// against the other of the two nearest points and y's in-block neighbours (Stage V's select
// group).  Only index points ever block: the queries are not points of the index.
struct SearchParams {
  const float* XQ;            // [strips * 128][Dp] query rows
  int64_t mq;
  int64_t row0;               // level position of query row 0
  const int32_t* qparent;     // [mq] sorted position of the query's finest pivot, or -1
  const float* X;             // index points in sorted order [n][Dp]
  int64_t n;
  int Dp, K;
  const __half* A;            // in-block FP16 keys (rounded up) and neighbours of the index blocks
  const uint8_t* nbr_i;
  const float* nbr_k;
  const int32_t* parent;      // [n] finest pivot (sorted position)
  const uint32_t* gpar;       // finest layer's guidance bitmask
  int64_t gpar_words;
  int64_t bpc;                // column blocks per chunk
  int nchunks;
  float* knn_k;               // [mq_pad][2 * nchunks][K] half-row lists per chunk
  int32_t* knn_i;
  int2* surv; unsigned long long* surv_cnt; unsigned long long surv_cap;
  unsigned long long* stats;  // [0] candidate pairs [1] queued pairs
};

#define SS_QCAP 4096
static __host__ __device__ constexpr size_t ss_bytes(int K) {
  return (size_t)IS_U + 32768 + 128 * GRNG_KIN * 5 + 128 * 6 * 4 + (size_t)128 * 2 * K * 8 + SS_QCAP * 4 + 16;
}

__device__ __forceinline__ void ss_cp16(void* dst, const void* src) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"((uint32_t)__cvta_generic_to_shared(dst)),
               "l"(src)
               : "memory");
}

template <int KC, int METRIC>
__global__ void __launch_bounds__(GRNG_THREADS, 1) search_sweep_kernel(SearchParams p) {
  extern __shared__ __align__(16) unsigned char sm_raw[];
  float* sA = reinterpret_cast<float*>(sm_raw);
  float* sB = sA + KC * GRNG_SSTRIDE;
  float* T = reinterpret_cast<float*>(sm_raw);
  unsigned char* q = sm_raw + IS_U;
  __half* AY = reinterpret_cast<__half*>(q); q += 32768;
  float* nbrYk = reinterpret_cast<float*>(q); q += 128 * GRNG_KIN * 4;
  uint8_t* nbrYi = q; q += 128 * GRNG_KIN;
  q += 512;
  int* ra1 = reinterpret_cast<int*>(q); q += 512;
  int* ra2 = reinterpret_cast<int*>(q); q += 512;
  int* parY = reinterpret_cast<int*>(q); q += 512;
  int* parX = reinterpret_cast<int*>(q); q += 512;
  q += 512;
  const int K = p.K;
  float* lk = reinterpret_cast<float*>(q); q += (size_t)128 * 2 * K * 4;  // [row][half][K]
  int* li = reinterpret_cast<int*>(q); q += (size_t)128 * 2 * K * 4;
  int* queue = reinterpret_cast<int*>(q); q += SS_QCAP * 4;
  int* s_qn = reinterpret_cast<int*>(q);

  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int Dp = p.Dp;
  const int64_t xb = (int64_t)blockIdx.x * 128;
  const int nr = (int)(p.mq - xb < 128 ? p.mq - xb : 128);
  const int64_t nb = (p.n + 127) / 128;
  const int64_t by0 = (int64_t)blockIdx.y * p.bpc, by1 = min(nb, by0 + p.bpc);
  const Err e = err_fp32(Dp);
  unsigned long long st_cand = 0, st_queued = 0;
  if (tid < 128) parX[tid] = tid < nr ? p.qparent[xb + tid] : -1;
  for (int i = tid; i < 128 * 2 * K; i += GRNG_THREADS) {
    lk[i] = inf_ins();
    li[i] = -1;
  }
  // the row pass: thread = (row, half); the odd half walks its columns rotated by 16 so that
  // the two threads of a row read different banks
  const int pr = tid >> 1, ph = tid & 1;
  for (int64_t by = by0; by < by1; ++by) {
    const int64_t yb = by * 128;
    const int nc = (int)(p.n - yb < 128 ? p.n - yb : 128);
    __syncthreads();  // the previous tile's filter and queue are done with T, AY, nbrY, parY
    {  // the block's in-block keys and neighbours arrive while the keys are computed
      const char* srcA = reinterpret_cast<const char*>(p.A + by * 16384);
      for (int i = tid; i < 2048; i += GRNG_THREADS) ss_cp16(reinterpret_cast<char*>(AY) + i * 16, srcA + i * 16);
      const char* srcK = reinterpret_cast<const char*>(p.nbr_k + yb * GRNG_KIN);
      for (int i = tid; i < 128 * GRNG_KIN / 4; i += GRNG_THREADS)
        ss_cp16(reinterpret_cast<char*>(nbrYk) + i * 16, srcK + i * 16);
      const char* srcI = reinterpret_cast<const char*>(p.nbr_i + yb * GRNG_KIN);
      for (int i = tid; i < 128 * GRNG_KIN / 16; i += GRNG_THREADS)
        ss_cp16(reinterpret_cast<char*>(nbrYi) + i * 16, srcI + i * 16);
      asm volatile("cp.async.commit_group;" ::: "memory");
    }
    float acc[8][8];
    tile_keys<KC, METRIC>(p.XQ + xb * Dp, nr, p.X + yb * Dp, nc, Dp, sA, sB, acc);
    __syncthreads();  // every thread is done with sA/sB: T may overwrite them
#pragma unroll
    for (int i = 0; i < 8; ++i)
#pragma unroll
      for (int j = 0; j < 8; ++j) {
        const int r = tile_row(i), c = tile_col(j);
        T[r * 129 + c] = (r < nr && c < nc) ? acc[i][j] : inf_ins();
      }
    if (tid < 128) parY[tid] = tid < nc ? p.parent[yb + tid] : 0;
    if (tid == 0) *s_qn = 0;
    asm volatile("cp.async.wait_all;" ::: "memory");
    __syncthreads();
    {  // ---- row pass: two nearest of the block, and the half-row's K nearest so far ----------
      float* kk = lk + (pr * 2 + ph) * K;
      int* ki = li + (pr * 2 + ph) * K;
      float thr = kk[K - 1];
      float m1 = inf_ins(), m2 = inf_ins();
      int a1 = -1, a2 = -1;
      const float* Tr = T + pr * 129;
      for (int i = 0; i < 64; ++i) {
        const int c = ph ? 64 + ((i + 16) & 63) : i;
        const float v = Tr[c];
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
      // merge the two halves' nearest pairs (lanes 2r and 2r+1 of one warp)
      const float o1 = __shfl_xor_sync(FULLMASK, m1, 1), o2 = __shfl_xor_sync(FULLMASK, m2, 1);
      const int b1 = __shfl_xor_sync(FULLMASK, a1, 1), b2 = __shfl_xor_sync(FULLMASK, a2, 1);
      if (ph == 0) {
        float n1, n2;
        int c1, c2;
        if (o1 < m1 || (o1 == m1 && b1 < a1)) {
          n1 = o1; c1 = b1;
          if (m1 < o2) { n2 = m1; c2 = a1; } else { n2 = o2; c2 = b2; }
        } else {
          n1 = m1; c1 = a1;
          if (o1 < m2) { n2 = o1; c2 = b1; } else { n2 = m2; c2 = a2; }
        }
        (void)n1;
        (void)n2;
        ra1[pr] = c1;
        ra2[pr] = c2;
      }
    }
    __syncthreads();
    // ---- tier-1 filter, uniform part: Theorem 1, then the block point nearest to q ----------
    // The guidance bits of the warp's 16 rows x the lane's 4 columns are loaded together
    // first: one memory latency per tile instead of one per row.
    unsigned long long link = ~0ull;  // bit rr * 4 + cb
    if (p.gpar) {
      unsigned wv[64];
#pragma unroll
      for (int t = 0; t < 64; ++t) {
        const int r = warp * 16 + (t >> 2), c = (t & 3) * 32 + lane;
        const int px = parX[r], qy = parY[c];
        wv[t] = ~0u;
        if (r < nr && c < nc && px >= 0 && qy != px) {
          const int a = min(px, qy), b = max(px, qy);
          wv[t] = __ldg(p.gpar + (int64_t)a * p.gpar_words + (b >> 5)) >> (b & 31);
        }
      }
#pragma unroll
      for (int t = 0; t < 64; ++t)
        if (!(wv[t] & 1u)) link &= ~(1ull << t);
    }
    for (int rr = 0; rr < 16; ++rr) {
      const int r = warp * 16 + rr;
      if (r >= nr) break;
      const int z1 = ra1[r], z2 = ra2[r];
      const float* Tr = T + r * 129;
      for (int cb = 0; cb < 4; ++cb) {
        if (cb * 32 >= nc) break;
        const int c = cb * 32 + lane;
        const float v = Tr[c];
        const bool cand = c < nc && v < inf_ins() && ((link >> (rr * 4 + cb)) & 1ull);
        st_cand += cand ? 1 : 0;
        bool open = false;
        if (cand) {
          const PairThr P = pair_thresholds(v, 0.0f, 0.0f, 0.0f, 0.0f, METRIC, e, 0);
          const int z = (z1 != c) ? z1 : z2;
          open = !(z >= 0 && block_state(Tr[z], __half2float(AY[z * 128 + c]), P, e) == 2);
        }
        const unsigned om = __ballot_sync(FULLMASK, open);
        if (om) {
          int base = 0;
          if (lane == 0) base = atomicAdd(s_qn, __popc(om));
          base = __shfl_sync(FULLMASK, base, 0);
          const int pos = base + __popc(om & ((1u << lane) - 1u));
          if (open && pos < SS_QCAP) queue[pos] = (r << 8) | c;
          st_queued += open ? 1 : 0;
        }
      }
    }
    __syncthreads();
    // ---- tier-1 filter, queued part (all threads): the other nearest point and the in-block
    // neighbours of y; the pairs none of them certainly blocks go on to tiers 2 and 3 ----------
    const int qn = *s_qn;
    auto full_test = [&](int r, int c) -> bool {
      const float v = T[r * 129 + c];
      const PairThr P = pair_thresholds(v, 0.0f, 0.0f, 0.0f, 0.0f, METRIC, e, 0);
      const int z1 = ra1[r], z2 = ra2[r];
      const int zo = (z1 != c) ? z2 : -1;  // the nearest was tested already, unless it was y
      if (zo >= 0 && zo != c && block_state(T[r * 129 + zo], __half2float(AY[zo * 128 + c]), P, e) == 2)
        return false;
      for (int t = 0; t < GRNG_KIN; ++t) {
        const int z = nbrYi[c * GRNG_KIN + t];
        if (z == 255) break;
        if (block_state(T[r * 129 + z], nbrYk[c * GRNG_KIN + t], P, e) == 2) return false;
      }
      return true;
    };
    auto push = [&](bool surv, int r, int c) {
      const unsigned sm = __ballot_sync(FULLMASK, surv);
      if (sm) {
        unsigned long long base = 0;
        if (lane == 0) base = atomicAdd(p.surv_cnt, (unsigned long long)__popc(sm));
        base = __shfl_sync(FULLMASK, base, 0);
        if (surv) {
          const unsigned long long pos = base + __popc(sm & ((1u << lane) - 1u));
          if (pos < p.surv_cap) p.surv[pos] = make_int2((int)(p.row0 + xb + r), (int)(yb + c));
        }
      }
    };
    if (qn <= SS_QCAP) {
      for (int b0 = 0; b0 < qn; b0 += GRNG_THREADS) {
        const int i = b0 + tid;
        bool surv = false;
        int r = 0, c = 0;
        if (i < qn) {
          r = queue[i] >> 8;
          c = queue[i] & 255;
          surv = full_test(r, c);
        }
        push(surv, r, c);
      }
    } else {  // the queue overflowed: every pair of the tile lane by lane instead (rare)
      for (int rr = 0; rr < 16; ++rr) {
        const int r = warp * 16 + rr;
        if (r >= nr) break;
        for (int cb = 0; cb < 4; ++cb) {
          if (cb * 32 >= nc) break;
          const int c = cb * 32 + lane;
          const float v = T[r * 129 + c];
          const bool cand = c < nc && v < inf_ins() && ((link >> (rr * 4 + cb)) & 1ull);
          bool surv = false;
          if (cand) {
            const PairThr P = pair_thresholds(v, 0.0f, 0.0f, 0.0f, 0.0f, METRIC, e, 0);
            const int z1 = ra1[r], z2 = ra2[r];
            const int z = (z1 != c) ? z1 : z2;
            surv = !(z >= 0 && block_state(T[r * 129 + z], __half2float(AY[z * 128 + c]), P, e) == 2) &&
                   full_test(r, c);
          }
          push(surv, r, c);
        }
      }
    }
  }
  __syncthreads();
  if (pr < nr) {
    const float* kk = lk + (pr * 2 + ph) * K;
    const int* ki = li + (pr * 2 + ph) * K;
    const int64_t o = ((xb + pr) * (2 * p.nchunks) + 2 * blockIdx.y + ph) * K;
    for (int j = 0; j < K; ++j) {
      p.knn_k[o + j] = kk[j];
      p.knn_i[o + j] = ki[j];
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    st_cand += __shfl_down_sync(FULLMASK, st_cand, o);
    st_queued += __shfl_down_sync(FULLMASK, st_queued, o);
  }
  if (lane == 0) {
    atomicAdd(p.stats + 0, st_cand);
    atomicAdd(p.stats + 1, st_queued);
  }
}

template <int KC>
static void launch_search_kc(const SearchParams& p, int metric, unsigned strips, cudaStream_t s) {
  const size_t smem = ss_bytes(p.K);
  dim3 grid(strips, (unsigned)p.nchunks);
  if (metric == L2) {
    GRNG_CUDA(cudaFuncSetAttribute(search_sweep_kernel<KC, L2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    search_sweep_kernel<KC, L2><<<grid, GRNG_THREADS, smem, s>>>(p); note_launch();
  } else {
    GRNG_CUDA(cudaFuncSetAttribute(search_sweep_kernel<KC, L1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    search_sweep_kernel<KC, L1><<<grid, GRNG_THREADS, smem, s>>>(p); note_launch();
  }
  GRNG_CUDA(cudaGetLastError());
}

void search_sweep(const SearchSweep& S, DevBuf& surv, int64_t* nsurv, float* knn_k, int32_t* knn_i,
                  unsigned long long* stats, cudaStream_t s) {
  const int64_t nb = (S.n + 127) / 128;
  const unsigned strips = (unsigned)((S.mq + 127) / 128);
  int sms = 0, dev = 0;
  GRNG_CUDA(cudaGetDevice(&dev));
  GRNG_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  // one CTA per SM (their shared memory allows no second), each with a contiguous range of
  // column blocks; a batch of more strips than SMs takes whole rows of blocks
  const int64_t want = std::max<int64_t>(1, (int64_t)sms / strips);
  const int64_t bpc = std::max<int64_t>(1, (nb + want - 1) / want);
  const int nchunks = (int)((nb + bpc - 1) / bpc);
  DevBuf ck, ci, ctr;
  GRNG_CUDA(ck.alloc((size_t)strips * 128 * 2 * nchunks * S.K * 4));
  GRNG_CUDA(ci.alloc((size_t)strips * 128 * 2 * nchunks * S.K * 4));
  GRNG_CUDA(ctr.alloc(4 * 8));
  // about 9,000 pairs per query leave tier 1 at intrinsic dimension 8; a first buffer of up to
  // 2^28 pairs (2 GB), and a larger batch that needs more is swept again with the exact size
  unsigned long long scap = S.small_buffers
                                ? 64ull
                                : std::min<unsigned long long>(
                                      1ull << 28, std::max<unsigned long long>(1 << 20, (unsigned long long)S.mq * 16384));
  for (int attempt = 0;; ++attempt) {
    GRNG_CUDA(surv.alloc(scap * sizeof(int2)));
    GRNG_CUDA(cudaMemsetAsync(ctr.p, 0, 4 * 8, s));
    SearchParams p;
    p.XQ = S.XQ; p.mq = S.mq; p.row0 = S.row0; p.qparent = S.qparent;
    p.X = S.X; p.n = S.n; p.Dp = S.Dp; p.K = S.K; p.A = S.A; p.nbr_i = S.nbr_i; p.nbr_k = S.nbr_k;
    p.parent = S.parent; p.gpar = S.gpar; p.gpar_words = S.gpar_words;
    p.bpc = bpc; p.nchunks = nchunks; p.knn_k = ck.as<float>(); p.knn_i = ci.as<int32_t>();
    unsigned long long* dc = ctr.as<unsigned long long>();
    p.surv = surv.as<int2>(); p.surv_cnt = dc; p.surv_cap = scap;
    p.stats = dc + 1;
    const int KC = S.Dp % 32 == 0 ? 32 : (S.Dp % 16 == 0 ? 16 : 8);
    if (KC == 32) launch_search_kc<32>(p, S.metric, strips, s);
    else if (KC == 16) launch_search_kc<16>(p, S.metric, strips, s);
    else launch_search_kc<8>(p, S.metric, strips, s);
    unsigned long long h[3];
    GRNG_CUDA(cudaMemcpyAsync(h, dc, sizeof(h), cudaMemcpyDeviceToHost, s));
    GRNG_CUDA(cudaStreamSynchronize(s));
    if (h[0] <= scap) {
      *nsurv = (int64_t)h[0];
      if (stats) { stats[0] += h[1]; stats[1] += h[2]; stats[2] += (unsigned long long)attempt; }
      break;
    }
    if (attempt >= 3) fail(6, "search sweep buffer overflow");
    scap = std::max(scap, h[0] + h[0] / 8);
  }
  knn_merge_kernel<<<nblk_ins(S.mq), 256, 0, s>>>(ck.as<float>(), ci.as<int32_t>(), S.mq, 2 * nchunks, S.K, S.rowpos,
                                                   knn_k, knn_i); note_launch();
  GRNG_CUDA(cudaGetLastError());
  GRNG_CUDA(cudaStreamSynchronize(s));
}

// ---- Stage VII ------------------------------------------------------------------------------
// per old point (sorted position): FP32 upper bound of its longest edge's key
__global__ void edge_maxkey_kernel(const uint64_t* __restrict__ edges, int64_t ne, const int32_t* __restrict__ rank,
                                   const float* __restrict__ X, int Dp, int metric, unsigned int* __restrict__ maxe) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne) return;
  const int i = rank[(int)(edges[t] >> 32)], j = rank[(int)(edges[t] & 0xffffffffu)];
  const float k = hi_b(key32(X + (int64_t)i * Dp, X + (int64_t)j * Dp, Dp, metric), err_fp32(Dp));
  atomicMax(maxe + i, __float_as_uint(k));  // non-negative floats order like their bits
  atomicMax(maxe + j, __float_as_uint(k));
}

__global__ void edge_degree_kernel(const uint64_t* __restrict__ edges, int64_t ne, int64_t* __restrict__ deg) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne) return;
  atomicAdd(reinterpret_cast<unsigned long long*>(deg + (edges[t] >> 32)), 1ull);
  atomicAdd(reinterpret_cast<unsigned long long*>(deg + (edges[t] & 0xffffffffu)), 1ull);
}

__global__ void edge_fill_kernel(const uint64_t* __restrict__ edges, int64_t ne, const int64_t* __restrict__ off,
                                 unsigned long long* __restrict__ cur, int32_t* __restrict__ other,
                                 int64_t* __restrict__ eidx) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= ne) return;
  const int a = (int)(edges[t] >> 32), b = (int)(edges[t] & 0xffffffffu);
  const unsigned long long pa = off[a] + atomicAdd(cur + a, 1ull);
  const unsigned long long pb = off[b] + atomicAdd(cur + b, 1ull);
  other[pa] = b; eidx[pa] = t;
  other[pb] = a; eidx[pb] = t;
}

// One warp per candidate (q, w): every old edge (w, y) of w; q removes it when it lies
// strictly inside its lune (Eq. 1), decided in FP32 with the error bound, else in FP64.
__global__ void stage7_kernel(const int4* __restrict__ s7, int64_t ns7, const float* __restrict__ X, int D, int Dp,
                              int metric, const int32_t* __restrict__ order, const int32_t* __restrict__ rank,
                              const int64_t* __restrict__ off, const int32_t* __restrict__ other,
                              const int64_t* __restrict__ eidx, uint8_t* __restrict__ removed,
                              unsigned long long* __restrict__ stats) {
  const int lane = threadIdx.x & 31;
  const int64_t w0 = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const Err e = err_fp32(Dp);
  unsigned long long c_test = 0, c_fp64 = 0;
  for (int64_t t = w0; t < ns7; t += nw) {
    const int4 c = s7[t];
    const int q = c.x, w = c.y;
    const float kqw = __int_as_float(c.z);
    const int wo = order[w];
    const float* pq = X + (int64_t)q * Dp;
    const float* pw = X + (int64_t)w * Dp;
    for (int64_t a = off[wo] + lane; a < off[wo + 1]; a += 32) {
      const int y = rank[other[a]];
      const float* py = X + (int64_t)y * Dp;
      const float kwy = key32(pw, py, Dp, metric);
      if (!(lo_b(kqw, e) < hi_b(kwy, e))) continue;  // q is not closer to w than y
      const float kqy = key32(pq, py, Dp, metric);
      if (lo_b(kqy, e) >= hi_b(kwy, e)) continue;    // q is not closer to y than w
      ++c_test;
      bool blocks;
      if (hi_b(kqw, e) < lo_b(kwy, e) && hi_b(kqy, e) < lo_b(kwy, e)) {
        blocks = true;
      } else {  // the canonical FP64 comparison
        ++c_fp64;
        const double d_wy = key64(pw, py, D, metric), d_qw = key64(pq, pw, D, metric), d_qy = key64(pq, py, D, metric);
        blocks = (d_qw > d_qy ? d_qw : d_qy) < d_wy;
      }
      if (blocks) removed[eidx[a]] = 1;
    }
  }
  for (int o = 16; o > 0; o >>= 1) {
    c_test += __shfl_down_sync(FULLMASK, c_test, o);
    c_fp64 += __shfl_down_sync(FULLMASK, c_fp64, o);
  }
  if (lane == 0) {
    atomicAdd(stats + 0, c_test);
    atomicAdd(stats + 1, c_fp64);
  }
}

__global__ void keep_edges_kernel(const uint64_t* __restrict__ edges, int64_t ne, const uint8_t* __restrict__ removed,
                                  uint64_t* __restrict__ out, unsigned long long* __restrict__ cnt) {
  const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  const bool keep = t < ne && !removed[t];
  const unsigned bm = __ballot_sync(FULLMASK, keep);
  unsigned long long base = 0;
  if ((threadIdx.x & 31) == 0 && bm) base = atomicAdd(cnt, (unsigned long long)__popc(bm));
  base = __shfl_sync(FULLMASK, base, 0);
  if (keep) out[base + __popc(bm & ((1u << (threadIdx.x & 31)) - 1u))] = edges[t];
}

void edge_max_keys(const uint64_t* edges, int64_t ne, const int32_t* rank, const float* X, int Dp, int metric,
                   float* maxe, int64_t n, cudaStream_t s) {
  GRNG_CUDA(cudaMemsetAsync(maxe, 0, (size_t)n * 4, s));  // 0.0f: a point without edges
  if (ne) {
    edge_maxkey_kernel<<<nblk_ins(ne), 256, 0, s>>>(edges, ne, rank, X, Dp, metric,
                                                    reinterpret_cast<unsigned int*>(maxe)); note_launch();
    GRNG_CUDA(cudaGetLastError());
  }
}

int64_t stage7_remove(const uint64_t* edges, int64_t ne, int64_t n_old, const int4* s7, int64_t ns7, const float* X,
                      int D, int Dp, int metric, const int32_t* order, const int32_t* rank, uint64_t* kept,
                      unsigned long long* stats, cudaStream_t s) {
  if (ne == 0) return 0;
  DevBuf deg, off, cur, oth, eid, rem, cnt;
  GRNG_CUDA(deg.alloc((size_t)(n_old + 1) * 8));
  GRNG_CUDA(off.alloc((size_t)(n_old + 1) * 8));
  GRNG_CUDA(cur.alloc((size_t)(n_old + 1) * 8));
  GRNG_CUDA(oth.alloc((size_t)2 * ne * 4));
  GRNG_CUDA(eid.alloc((size_t)2 * ne * 8));
  GRNG_CUDA(rem.alloc((size_t)ne));
  GRNG_CUDA(cnt.alloc(8));
  GRNG_CUDA(cudaMemsetAsync(deg.p, 0, (size_t)(n_old + 1) * 8, s));
  GRNG_CUDA(cudaMemsetAsync(cur.p, 0, (size_t)(n_old + 1) * 8, s));
  GRNG_CUDA(cudaMemsetAsync(rem.p, 0, (size_t)ne, s));
  GRNG_CUDA(cudaMemsetAsync(cnt.p, 0, 8, s));
  edge_degree_kernel<<<nblk_ins(ne), 256, 0, s>>>(edges, ne, deg.as<int64_t>()); note_launch();
  exclusive_scan_i64(deg.as<int64_t>(), off.as<int64_t>(), n_old, s);
  edge_fill_kernel<<<nblk_ins(ne), 256, 0, s>>>(edges, ne, off.as<int64_t>(), cur.as<unsigned long long>(),
                                                oth.as<int32_t>(), eid.as<int64_t>()); note_launch();
  if (ns7)
    stage7_kernel<<<(unsigned)std::min<int64_t>((ns7 + 7) / 8, 8192), 256, 0, s>>>(
        s7, ns7, X, D, Dp, metric, order, rank, off.as<int64_t>(), oth.as<int32_t>(), eid.as<int64_t>(),
        rem.as<uint8_t>(), stats); note_launch();
  keep_edges_kernel<<<nblk_ins(ne), 256, 0, s>>>(edges, ne, rem.as<uint8_t>(), kept, cnt.as<unsigned long long>()); note_launch();
  GRNG_CUDA(cudaGetLastError());
  unsigned long long h = 0;
  GRNG_CUDA(cudaMemcpyAsync(&h, cnt.p, 8, cudaMemcpyDeviceToHost, s));
  GRNG_CUDA(cudaStreamSynchronize(s));
  return (int64_t)h;
}

}  // namespace grng
