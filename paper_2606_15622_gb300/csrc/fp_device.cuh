// fp_device.cuh -- device helpers shared by the closure kernels (sm_103a).
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

#include "../../include/fpclosure.h"

namespace fpc {

// moment slots (layout documented in fpclosure.h)
constexpr int kN = 0, kU = 1, kTheta = 4, kU2 = 5, kU3 = 11, kW = 21, kZ = 27;
constexpr int kNSum = 26;   // gathered central sums: u2 (6), u3 (10), w (6), z (3), <|c|^6> (1)
constexpr int kNMomSum = 25;  // of those, the ones stored in the moment vector (from slot kU2)
constexpr int kM6Sum = 25;    // the sum slot of <|c|^6> (its own optional output array)

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): the counter-based
// generator of the noise variates and of the dropout masks.  The key
// schedule (k0 + r 0x9E3779B9, k1 + r 0xBB67AE85 for round r) depends on the
// seed only, so the host computes it once (philox_keys) and passes it as a
// kernel parameter.
struct PhiloxKeys {
  uint32_t k0[10], k1[10];
};

__device__ __forceinline__ uint4 philox4x32_10(uint4 x, const PhiloxKeys &key) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    // one 32x32 -> 64-bit multiply gives both halves of each product
    const uint64_t p0 = (uint64_t)0xD2511F53u * x.x, p1 = (uint64_t)0xCD9E8D57u * x.z;
    x = make_uint4((uint32_t)(p1 >> 32) ^ x.y ^ key.k0[r], (uint32_t)p1, (uint32_t)(p0 >> 32) ^ x.w ^ key.k1[r],
                   (uint32_t)p0);
  }
  return x;
}

inline PhiloxKeys philox_keys(uint64_t seed) {
  PhiloxKeys k;
  for (int r = 0; r < 10; ++r) {
    k.k0[r] = (uint32_t)seed + 0x9E3779B9u * (uint32_t)r;
    k.k1[r] = (uint32_t)(seed >> 32) + 0xBB67AE85u * (uint32_t)r;
  }
  return k;
}

// Conversions between binary64 and binary32 done with integer operations on
// the IEEE-754 bit layouts.  On this chip the FP64 pipe executes conversion
// instructions too, and it is the scarcest pipe; these keep per-cell
// bookkeeping off it.
//   f2d_exact:  float -> double, exact (below);
//   d2f_rn:     double -> float rounded to nearest, ties to even; results
//               below the smallest normal float are flushed to a signed zero,
//               beyond the largest give infinity, NaN stays NaN;
//   u2d_exact:  32-bit unsigned integer -> double, exact.
__device__ __forceinline__ float d2f_rn(double x) {
  const uint32_t hi = (uint32_t)__double2hiint(x), lo = (uint32_t)__double2loint(x);
  const uint32_t sign = hi & 0x80000000u;
  const int e = (int)((hi >> 20) & 0x7ffu);
  if (e == 0x7ff) return __uint_as_float(sign | 0x7f800000u | (((hi & 0xfffffu) | lo) ? 0x400000u : 0u));
  const int eb = e - 896;  // biased binary32 exponent
  if (eb >= 255) return __uint_as_float(sign | 0x7f800000u);
  if (eb <= 0) return __uint_as_float(sign);
  const uint32_t m = ((hi & 0xfffffu) << 3) | (lo >> 29);  // the top 23 of the 52 fraction bits
  const uint32_t rest = lo & 0x1fffffffu;                   // the 29 bits below them
  const uint32_t up = (rest > 0x10000000u || (rest == 0x10000000u && (m & 1u))) ? 1u : 0u;
  // a carry out of the fraction moves into the exponent (and to infinity at the top)
  return __uint_as_float(sign | ((((uint32_t)eb << 23) | m) + up));
}

__device__ __forceinline__ double u2d_exact(uint32_t n) {
  if (n == 0u) return 0.0;
  const int e = 31 - __clz(n);                                             // 2^e <= n < 2^(e+1)
  const uint64_t frac = ((uint64_t)n << (52 - e)) & 0xfffffffffffffull;  // drop the leading one
  return __longlong_as_double((long long)(((uint64_t)(e + 1023) << 52) | frac));
}

__device__ __forceinline__ uint64_t abs_bits(double x) {
  return (uint64_t)__double_as_longlong(x) & 0x7fffffffffffffffull;
}
__device__ __forceinline__ bool finite_d(double x) {
  return (abs_bits(x) & 0x7ff0000000000000ull) != 0x7ff0000000000000ull;
}

// x > 0 for a double (false for NaN), on its bits
__device__ __forceinline__ bool positive_d(double x) {
  const long long b = __double_as_longlong(x);
  return b > 0 && b <= 0x7ff0000000000000ll;
}

// Error-free transformation a + b = s + e (Knuth two-sum).
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
  s = a + b;
  float bb = s - a;
  e = (a - (s - bb)) + (b - bb);
}

// Order of the central moment held in gathered sum slot q (0..25).
__host__ __device__ constexpr int sum_order(int q) {
  return q < 6 ? 2 : (q < 16 ? 3 : (q < 22 ? 4 : (q < 25 ? 5 : 6)));
}

// Butterfly all-reduce over groups of G consecutive lanes (all 32 lanes call).
template <int G, typename T>
__device__ __forceinline__ T group_allreduce(T x) {
#pragma unroll
  for (int o = G / 2; o >= 1; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
  return x;
}

// Reduce-scatter of 32 slots over groups of G lanes: on return lane l of the
// group holds, in v[0 .. 32/G), the group sums of slots [l*32/G, (l+1)*32/G).
template <int G, typename T>
__device__ __forceinline__ void group_reduce_scatter(T (&v)[32], int lane) {
#pragma unroll
  for (int lvl = 0; (G >> (lvl + 1)) >= 1; ++lvl) {
    const int o = G >> (lvl + 1);
    const int half = 16 >> lvl;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      T send = up ? v[j] : v[j + half];
      T keep = up ? v[j + half] : v[j];
      v[j] = keep + __shfl_xor_sync(0xffffffffu, send, o);
    }
  }
}

// The same with (hi, lo) compensated pairs: hi sums by two-sum, errors and
// lo parts accumulated in lo.
template <int G>
__device__ __forceinline__ void group_reduce_scatter2(float (&hi)[32], float (&lo)[32], int lane) {
#pragma unroll
  for (int lvl = 0; (G >> (lvl + 1)) >= 1; ++lvl) {
    const int o = G >> (lvl + 1);
    const int half = 16 >> lvl;
    const bool up = (lane & o) != 0;
#pragma unroll
    for (int j = 0; j < half; ++j) {
      float sh = up ? hi[j] : hi[j + half];
      float sl = up ? lo[j] : lo[j + half];
      float kh = up ? hi[j + half] : hi[j];
      float kl = up ? lo[j + half] : lo[j];
      float rh = __shfl_xor_sync(0xffffffffu, sh, o);
      float rl = __shfl_xor_sync(0xffffffffu, sl, o);
      float s, e;
      two_sum(kh, rh, s, e);
      hi[j] = s;
      lo[j] = (kl + rl) + e;
    }
  }
}

template <typename VT>
__device__ __forceinline__ VT ldg_v(const VT *p) { return __ldg(p); }

// Exact float -> double by integer bit manipulation (no FP64-pipe work), with
// an optional power-of-two scale 2^exp_add folded into the exponent.
// Normal floats and zeros convert exactly; FP32 subnormals flush to zero;
// results outside the double range saturate to zero / infinity; inf and NaN
// pass through.
__device__ __forceinline__ double f2d_exact(float f, int exp_add = 0) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t sign = u & 0x80000000u;
  const int e = (int)((u >> 23) & 0xffu);
  const uint32_t man = u & 0x7fffffu;
  const int ed = e + (1023 - 127) + exp_add;
  uint32_t hi = sign | (man >> 3), lo = man << 29;
  if (e == 0 || ed <= 0) {
    hi = sign;
    lo = 0u;
  } else if (e == 255 || ed >= 2047) {
    hi |= 0x7ff00000u;
    if (e != 255) {
      hi = sign | 0x7ff00000u;
      lo = 0u;
    }
  } else {
    hi |= (uint32_t)ed << 20;
  }
  return __hiloint2double((int)hi, (int)lo);
}

// Double-float helpers (pairs of FP32 carrying ~46 significant bits).
// (rh, rl) ~ 1/n: rh the rounded reciprocal, rl its residual.
__device__ __forceinline__ void df_recip(float n, float &rh, float &rl) {
  rh = __frcp_rn(n);
  rl = fmaf(-rh, n, 1.f) * rh;
}
// (hi + lo) * (rh + rl) as a double-float (p, e)
__device__ __forceinline__ void df_scale(float hi, float lo, float rh, float rl, float &p, float &e) {
  p = hi * rh;
  e = fmaf(hi, rh, -p);
  e = fmaf(hi, rl, fmaf(lo, rh, e));
}

// Copy a per-cell constant row (NC entries, 16-byte aligned, NC a multiple of
// four) from shared memory into registers with 16-byte loads.
template <int NC>
__device__ __forceinline__ void load_row(const float *__restrict__ row, float (&K)[NC]) {
  static_assert(NC % 4 == 0, "row length");
  const float4 *r4 = reinterpret_cast<const float4 *>(row);
#pragma unroll
  for (int q = 0; q < NC / 4; ++q) {
    const float4 x = r4[q];
    K[4 * q] = x.x;
    K[4 * q + 1] = x.y;
    K[4 * q + 2] = x.z;
    K[4 * q + 3] = x.w;
  }
}
template <int NC>
__device__ __forceinline__ void load_row(const double *__restrict__ row, double (&K)[NC]) {
  static_assert(NC % 2 == 0, "row length");
  const double2 *r2 = reinterpret_cast<const double2 *>(row);
#pragma unroll
  for (int q = 0; q < NC / 2; ++q) {
    const double2 x = r2[q];
    K[2 * q] = x.x;
    K[2 * q + 1] = x.y;
  }
}

}  // namespace fpc
