// common.cuh -- shared device definitions of the GRNG/RNG library (sm_103a).
//
// Decision model.  Every graph decision is, by definition, a comparison of canonical
// FP64 values (Eq. 1 and the GRNG definition, Sec. 2): keys
//     key_L2(a,b) = sum_k (a_k - b_k)^2   (left to right, round-to-nearest, no FMA)
//     key_L1(a,b) = sum_k |a_k - b_k|
// and, for GRNG thresholds, distances d = sqrt(key_L2) (resp. key_L1).
// The fast path computes keys in FP32 and brackets the canonical FP64 value:
//     lo(a) = a (1 - eps) - eta  <=  key64  <=  hi(a) = a (1 + eps) + eta
// with eps = (D + 8) 2^-24 and eta = 2 D 2^-126.  Derivation: each difference is
// rounded once, each square-and-add (an FMA) once, so the FP32 sum of D
// non-negative terms has relative error at most gamma_{D+2} = (D+2) u / (1-(D+2) u),
// u = 2^-24; the canonical FP64 value differs from the exact real by a relative
// (D+2) 2^-53; the bound computation itself rounds once more; eta covers squares
// that underflow.  A comparison whose bracketed values overlap is "ambiguous" and is
// re-decided with the canonical FP64 routine below, which reproduces the CPU
// definition operation for operation.
#pragma once
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <math.h>
#include <stdint.h>

#define GRNG_TILE 128      // nodes per block (rows and columns of a distance tile)
#define GRNG_THREADS 256   // threads of the tile kernels
#define GRNG_KIN 8         // in-block nearest neighbours kept per node (tier-1 interceptors)
#define GRNG_KMAX 32       // longest neighbour list (tier 2)

namespace grng {

enum Metric { L2 = 0, L1 = 1 };

struct Err {
  float eps;
  float eta;
};

__host__ __device__ inline Err err_fp32(int D) {
  Err e;
  e.eps = (float)(D + 8) * 5.9604644775390625e-8f;  // (D+8) 2^-24
  e.eta = (float)(2 * D) * 1.1754943508222875e-38f;  // 2 D 2^-126
  return e;
}
__device__ __forceinline__ float hi_b(float a, Err e) { return fmaf(a, 1.0f + e.eps, e.eta); }
__device__ __forceinline__ float lo_b(float a, Err e) { return fmaf(a, 1.0f - e.eps, -e.eta); }

// Guidance margin.  Theorems 1 and 2 prune the pairs below a non-linked pivot pair, and
// that pruning is exact in the reals; near a threshold, the FP64 rounding of the
// definition's distances could call a pair non-linked that exact arithmetic links.  So
// a pair counts as "safely" non-linked -- and may prune its descendants -- only when
// some blocker clears both G-lune thresholds by more than TAU_REL times the magnitude
// of the quantities involved; the FP64 rounding of those quantities is ~2^-46 relative,
// 64 times smaller than the margin for sums of up to 128 terms.
#define GRNG_TAU_REL 9.094947017729282e-13  // 2^-40

// ---- canonical FP64 key, the only FP64 arithmetic of the fast path --------------
__device__ __forceinline__ double key64(const float* __restrict__ a, const float* __restrict__ b,
                                        int D, int metric) {
  double acc = 0.0;
  if (metric == L2) {
    for (int k = 0; k < D; ++k) {
      double t = __dsub_rn((double)a[k], (double)b[k]);
      acc = __dadd_rn(acc, __dmul_rn(t, t));
    }
  } else {
    for (int k = 0; k < D; ++k) {
      double t = __dsub_rn((double)a[k], (double)b[k]);
      acc = __dadd_rn(acc, fabs(t));
    }
  }
  return acc;
}
__device__ __forceinline__ double dist_of_key64(double k, int metric) {
  return metric == L2 ? __dsqrt_rn(k) : k;
}

// FP32 key along the canonical order (used outside the tiles).
__device__ __forceinline__ float key32(const float* __restrict__ a, const float* __restrict__ b,
                                       int Dp, int metric) {
  float acc = 0.0f;
  if (metric == L2) {
    for (int k = 0; k < Dp; k += 4) {
      float4 x = *reinterpret_cast<const float4*>(a + k);
      float4 y = *reinterpret_cast<const float4*>(b + k);
      float t;
      t = x.x - y.x; acc = fmaf(t, t, acc);
      t = x.y - y.y; acc = fmaf(t, t, acc);
      t = x.z - y.z; acc = fmaf(t, t, acc);
      t = x.w - y.w; acc = fmaf(t, t, acc);
    }
  } else {
    for (int k = 0; k < Dp; k += 4) {
      float4 x = *reinterpret_cast<const float4*>(a + k);
      float4 y = *reinterpret_cast<const float4*>(b + k);
      acc += fabsf(x.x - y.x);
      acc += fabsf(x.y - y.y);
      acc += fabsf(x.z - y.z);
      acc += fabsf(x.w - y.w);
    }
  }
  return acc;
}

// ---- per-pair thresholds --------------------------------------------------------
// A pair (x, y) with radii (rx, ry) is blocked by k iff
//   cond1: d(k,x) < d(x,y) - (2 rx + ry)   and   cond2: d(k,y) < d(x,y) - (rx + 2 ry)
// (GRNG definition, Sec. 2); with rx = ry = 0 both conditions compare keys (Eq. 1).
// The fast path carries each condition as two key thresholds:
//   certainly true  if hi(key) <  c.lo      certainly false if lo(key) >= c.hi
struct PairThr {
  float t1lo, t1hi, t2lo, t2hi;
  int quick;  // 1: no k can satisfy one of the conditions (certainly linked)
  float lam;  // zero radii, L2: beta / 2 of a lune-based beta-skeleton (1: the lune of Eq. 1)
};

// v = FP32 key of (x, y); rx*/ry* = FP32 lower/upper bounds of the FP64 radii.
// guide = 1 applies the guidance margin to the "certainly true" side.  lam < 1 (zero radii,
// L2 only) asks for the beta-skeleton test: the thresholds stay those of Eq. 1, whose lune
// holds every beta-lune with beta <= 2, so every bound derived from them stays valid.
__device__ __forceinline__ PairThr pair_thresholds(float v, float rxlo, float rxhi, float rylo,
                                                   float ryhi, int metric, Err e, int guide,
                                                   float lam = 1.0f) {
  PairThr p;
  p.quick = 0;
  p.lam = (rxhi == 0.0f && ryhi == 0.0f) ? lam : 1.0f;
  const float u2 = 1.1920928955078125e-07f;  // 2 u
  if (rxhi == 0.0f && ryhi == 0.0f) {        // zero radii: key comparisons (Eq. 1)
    float vlo = lo_b(v, e), vhi = hi_b(v, e);
    if (guide) vlo -= (float)GRNG_TAU_REL * 2.0f * v;
    p.t1lo = p.t2lo = vlo;
    p.t1hi = p.t2hi = vhi;
    return p;
  }
  float vlo = fmaxf(lo_b(v, e), 0.0f), vhi = hi_b(v, e);
  float dlo, dhi;
  if (metric == L2) {
    dlo = sqrtf(vlo) * (1.0f - u2);
    dhi = sqrtf(vhi) * (1.0f + u2);
  } else {
    dlo = vlo;
    dhi = vhi;
  }
  float c1lo = 2.0f * rxlo + rylo, c1hi = 2.0f * rxhi + ryhi;
  float c2lo = rxlo + 2.0f * rylo, c2hi = rxhi + 2.0f * ryhi;
  float s1 = u2 * (dhi + c1hi), s2 = u2 * (dhi + c2hi);
  float tau = (float)GRNG_TAU_REL * 4.0f * (dhi + 2.0f * (rxhi + ryhi));
  float t1lo = dlo - c1hi - s1 - (guide ? tau : 0.0f), t1hi = dhi - c1lo + s1;
  float t2lo = dlo - c2hi - s2 - (guide ? tau : 0.0f), t2hi = dhi - c2lo + s2;
  // Quick accept (exact in the reals): a blocker k needs d(x,y) <= d(k,x) + d(k,y) <
  // t1 + t2, impossible once t1 + t2 <= d(x,y), i.e. d(x,y) <= 3 (rx + ry); likewise
  // once a threshold is not positive.  The margin dwarfs the FP64 rounding of the
  // canonical comparisons, so the FP64 definition agrees.
  if (t1hi <= 0.0f || t2hi <= 0.0f || t1hi + t2hi <= dlo * (1.0f - 2.0f * u2)) {
    p.quick = 1;
    p.t1lo = p.t2lo = -1.0f;
    p.t1hi = p.t2hi = 0.0f;
    return p;
  }
  if (metric == L2) {
    p.t1lo = t1lo > 0.0f ? t1lo * t1lo * (1.0f - u2) : -1.0f;
    p.t2lo = t2lo > 0.0f ? t2lo * t2lo * (1.0f - u2) : -1.0f;
    p.t1hi = t1hi * t1hi * (1.0f + u2);
    p.t2hi = t2hi * t2hi * (1.0f + u2);
  } else {
    p.t1lo = t1lo > 0.0f ? t1lo : -1.0f;
    p.t2lo = t2lo > 0.0f ? t2lo : -1.0f;
    p.t1hi = t1hi;
    p.t2hi = t2hi;
  }
  return p;
}

// Lune-based beta-skeleton (L2 keys a = |k-x|^2, b = |k-y|^2, v = |x-y|^2, lam = beta/2):
// k lies strictly inside both balls of the beta-lune iff (1-lam) a + lam b < lam v and
// lam a + (1-lam) b < lam v (Stewart's theorem for the distance to each centre).  The
// brackets of a, b and v carry their FP32 errors; 8u (a + b) and 4u of the threshold cover
// the rounding of the combinations and the FP32 rounding of lam.
__device__ __forceinline__ int beta_state(float a, float b, const PairThr& p, Err e) {
  const float u = 5.9604644775390625e-8f;
  const float lam = p.lam, mu = 1.0f - lam;
  const float ah = hi_b(a, e), bh = hi_b(b, e);
  const float al = fmaxf(lo_b(a, e), 0.0f), bl = fmaxf(lo_b(b, e), 0.0f);
  const float tlo = lam * p.t1lo * (1.0f - 4.0f * u), thi = lam * p.t1hi * (1.0f + 4.0f * u);
  const float sh = 8.0f * u * (ah + bh), sl = 8.0f * u * (al + bl);
  if (mu * ah + lam * bh + sh < tlo && lam * ah + mu * bh + sh < tlo) return 2;
  if (mu * al + lam * bl - sl >= thi || lam * al + mu * bl - sl >= thi) return 0;
  return 1;
}

// 2 = certainly blocks, 0 = certainly does not block, 1 = ambiguous.
// a = FP32 key(k, x), b = FP32 key(k, y).
__device__ __forceinline__ int block_state(float a, float b, const PairThr& p, Err e) {
  if (p.lam < 1.0f) return beta_state(a, b, p, e);
  if (hi_b(a, e) < p.t1lo && hi_b(b, e) < p.t2lo) return 2;
  if (lo_b(a, e) >= p.t1hi || lo_b(b, e) >= p.t2hi) return 0;
  return 1;
}

// Canonical FP64 decision for one triple, exactly as the CPU definition evaluates it.
// Returns bit0 = blocks (definition), bit1 = blocks with the guidance margin.  lam < 1 (zero
// radii): the beta-skeleton test, each side as the definition writes it (two products, then
// their sum), which is symmetric in x and y.
__device__ __forceinline__ int block64(const float* __restrict__ X, int D, int Dp, int metric,
                                       int64_t x, int64_t y, int64_t k, double rx, double ry,
                                       double lam = 1.0) {
  const float* px = X + x * Dp;
  const float* py = X + y * Dp;
  const float* pk = X + k * Dp;
  double kxy = key64(px, py, D, metric);
  double kkx = key64(pk, px, D, metric);
  double kky = key64(pk, py, D, metric);
  if (rx == 0.0 && ry == 0.0 && lam < 1.0) {
    const double mu = __dsub_rn(1.0, lam);
    const double t = __dmul_rn(lam, kxy);
    const double in1 = __dadd_rn(__dmul_rn(mu, kkx), __dmul_rn(lam, kky));
    const double in2 = __dadd_rn(__dmul_rn(lam, kkx), __dmul_rn(mu, kky));
    const int b = in1 < t && in2 < t;
    return b | (b << 1);
  }
  if (rx == 0.0 && ry == 0.0) {
    double m = kkx > kky ? kkx : kky;
    int b = m < kxy;
    int g = (kxy - m) > GRNG_TAU_REL * kxy;
    return b | (g << 1);
  }
  double dxy = dist_of_key64(kxy, metric);
  double dkx = dist_of_key64(kkx, metric);
  double dky = dist_of_key64(kky, metric);
  double t1 = __dsub_rn(dxy, __dadd_rn(__dmul_rn(2.0, rx), ry));
  double t2 = __dsub_rn(dxy, __dadd_rn(rx, __dmul_rn(2.0, ry)));
  int b = (dkx < t1) && (dky < t2);
  double m1 = t1 - dkx, m2 = t2 - dky;
  double m = m1 < m2 ? m1 : m2;
  double tau = GRNG_TAU_REL * (dxy + 2.0 * rx + 2.0 * ry);
  int g = b && (m > tau);
  return b | (g << 1);
}

__device__ __forceinline__ unsigned long long dbl_as_ull(double d) {
  return (unsigned long long)__double_as_longlong(d);
}

}  // namespace grng
