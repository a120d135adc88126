// mlp_common.cuh -- shapes and helpers of the surrogate network
// (32 -> 128 -> 128 -> 128 -> 128 -> 16, SiLU, BF16 operands, FP32
// accumulation) shared by the inference and training kernels.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

#include "fp_device.cuh"

namespace fpc {

constexpr int kIn = 32, kHid = 128, kOut = 16, kDepth = 4, kNFeat = 25, kNOut = 9;

// dropout of the hidden activations in one forward pass (sensitivity probe)
struct DropoutCfg {
  PhiloxKeys key;
  float rate, scale;  // drop probability, 1 / (1 - rate)
  uint32_t pass;
};

// device pointers of the network (weights W[l] are [out][in] row-major)
struct MlpDev {
  const __nv_bfloat16 *W[5];
  const float *b[5];
  const float *x_mu, *x_sigma, *y_mu, *y_sigma, *x_min, *x_max;
};

__device__ __forceinline__ uint32_t pack_bf16(float lo, float hi) {
  const __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);  // .x = lo (low half)
  return *reinterpret_cast<const uint32_t *>(&v);
}

__device__ __forceinline__ float silu(float z) { return __fdividef(z, 1.f + __expf(-z)); }

__device__ __forceinline__ float silu_grad(float z) {
  const float s = __fdividef(1.f, 1.f + __expf(-z));
  return s * (1.f + z * (1.f - s));
}

// D = A * B + C for one m16n8k16 tile (BF16 x BF16 -> FP32)
__device__ __forceinline__ void mma_bf16(float (&d)[4], uint32_t a0, uint32_t a1, uint32_t a2, uint32_t a3,
                                         uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}

// The 16 raw inputs of one cell from its LITE vector and tau, in FP32 (the
// entries narrowed on the integer pipe: d2f_rn).
__device__ __forceinline__ void lite_raw_features(const double *__restrict__ m, double tau, float (&f)[16]) {
  const float th = d2f_rn(m[4]);
  const float u00 = d2f_rn(m[5]), u01 = d2f_rn(m[6]), u02 = d2f_rn(m[7]), u11 = d2f_rn(m[8]), u12 = d2f_rn(m[9]),
              u22 = d2f_rn(m[10]);
  f[0] = d2f_rn(m[0]);
  f[1] = th;
  f[2] = d2f_rn(m[1]);
  f[3] = d2f_rn(m[2]);
  f[4] = d2f_rn(m[3]);
  f[5] = u00 - th;
  f[6] = u01;
  f[7] = u02;
  f[8] = u11 - th;
  f[9] = u12;
  f[10] = u22 - th;
  f[11] = 0.5f * d2f_rn(m[11]);
  f[12] = 0.5f * d2f_rn(m[12]);
  f[13] = 0.5f * d2f_rn(m[13]);
  f[14] = fmaf(u00, fmaf(u11, u22, -u12 * u12), fmaf(-u01, fmaf(u01, u22, -u12 * u02), u02 * fmaf(u01, u12, -u11 * u02)));
  f[15] = 1.f / d2f_rn(tau);
}

}  // namespace fpc
