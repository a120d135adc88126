// quads.cuh -- helpers of the kernels that stream particles in quads of four
// consecutive ones (velocity update, adjoint particle pass): vector loads and
// stores of a quad by the alignment class of its component array, and the
// half-warp search of a particle slice's first cell.
#pragma once

#include <cstdint>

namespace fpc {

// a quad of one component by its alignment class (2: one 16-byte access of
// floats or two of doubles, 1: two 8-byte float pairs, 0: four scalars)
template <typename T>
__device__ __forceinline__ void load_comp(const T *p, int cls, T (&x)[4]);
template <typename T>
__device__ __forceinline__ void store_comp(T *p, int cls, const T (&x)[4]);

// four consecutive values (16-byte aligned address) in and out
__device__ __forceinline__ void load4(const float *p, float (&x)[4]) {
  const float4 a = *reinterpret_cast<const float4 *>(p);
  x[0] = a.x, x[1] = a.y, x[2] = a.z, x[3] = a.w;
}
__device__ __forceinline__ void load4(const double *p, double (&x)[4]) {
  const double2 a = reinterpret_cast<const double2 *>(p)[0], b = reinterpret_cast<const double2 *>(p)[1];
  x[0] = a.x, x[1] = a.y, x[2] = b.x, x[3] = b.y;
}
__device__ __forceinline__ void store4(float *p, const float (&x)[4]) {
  *reinterpret_cast<float4 *>(p) = make_float4(x[0], x[1], x[2], x[3]);
}
__device__ __forceinline__ void store4(double *p, const double (&x)[4]) {
  reinterpret_cast<double2 *>(p)[0] = make_double2(x[0], x[1]);
  reinterpret_cast<double2 *>(p)[1] = make_double2(x[2], x[3]);
}

template <>
__device__ __forceinline__ void load_comp<float>(const float *p, int cls, float (&x)[4]) {
  if (cls == 2) {
    load4(p, x);
  } else if (cls == 1) {
    const float2 a = reinterpret_cast<const float2 *>(p)[0], b = reinterpret_cast<const float2 *>(p)[1];
    x[0] = a.x, x[1] = a.y, x[2] = b.x, x[3] = b.y;
  } else {
    x[0] = p[0], x[1] = p[1], x[2] = p[2], x[3] = p[3];
  }
}
template <>
__device__ __forceinline__ void load_comp<double>(const double *p, int cls, double (&x)[4]) {
  if (cls == 2)
    load4(p, x);
  else
    x[0] = p[0], x[1] = p[1], x[2] = p[2], x[3] = p[3];
}
template <>
__device__ __forceinline__ void store_comp<float>(float *p, int cls, const float (&x)[4]) {
  if (cls == 2) {
    store4(p, x);
  } else if (cls == 1) {
    reinterpret_cast<float2 *>(p)[0] = make_float2(x[0], x[1]);
    reinterpret_cast<float2 *>(p)[1] = make_float2(x[2], x[3]);
  } else {
    p[0] = x[0], p[1] = x[1], p[2] = x[2], p[3] = x[3];
  }
}
template <>
__device__ __forceinline__ void store_comp<double>(double *p, int cls, const double (&x)[4]) {
  if (cls == 2)
    store4(p, x);
  else
    p[0] = x[0], p[1] = x[1], p[2] = x[2], p[3] = x[3];
}

// The first cell c in [0, n] with off[c] >= t (off nondecreasing, off[n] >=
// t), found by the 16 lanes of the calling half warp together: each round
// probes 16 evenly spaced offsets and keeps the interval where the answer
// lies, so 2^17 cells take five dependent loads.
__device__ __forceinline__ int64_t lower_bound16(const int64_t *__restrict__ off, int64_t n, int64_t t, int lane) {
  const int h = lane & 15;
  const unsigned hmask = 0xffffu << (lane & 16);
  int64_t lo = 0, hi = n;  // the answer lies in [lo, hi]
  while (hi - lo > 15) {
    const int64_t step = (hi - lo + 15) / 16;
    const int64_t c = min(lo + step * h, hi);
    const unsigned b = (__ballot_sync(hmask, off[c] >= t) >> (lane & 16)) & 0xffffu;
    if (b == 0) {
      lo = min(lo + step * 15, hi) + 1;
    } else {
      const int f = __ffs(b) - 1;
      if (f == 0) {
        hi = lo;
      } else {
        hi = min(lo + step * f, hi);
        lo = lo + step * (f - 1) + 1;
      }
    }
  }
  const int64_t c = min(lo + h, hi);
  const unsigned b = (__ballot_sync(hmask, off[c] >= t) >> (lane & 16)) & 0xffffu;
  return lo + (__ffs(b) - 1);
}

}  // namespace fpc
