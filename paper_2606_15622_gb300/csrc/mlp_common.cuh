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

// the learned closure fused around the inference pass: where the inputs
// come from and where the coefficients, flags and the list of cells for the
// exact fallback go (device pointers)
struct FusedIO {
  const double *src;  // moment vectors [n][FP_NMOM] or LITE vectors [n][FP_NLITE]
  const double *tau;  // [n]
  int min_particles;
  float margin;       // training box widened by margin x_sigma
  float eps2_hat, energy_tol;
  double *coeffs;     // [n][9]
  int32_t *flags;     // [n]
  int32_t *list;      // cells for the exact fallback (full inputs only)
  uint32_t *count;    // their number, zeroed before the launch
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

// FP64 moment -> FP32 network input, rounded to nearest even (the hardware
// conversion: the learned-closure kernels leave the FP64 pipe otherwise
// idle, so it costs one issue slot where the integer-pipe version takes
// about fifteen).
__device__ __forceinline__ float narrow(double x) { return __double2float_rn(x); }

// standardisation of the network's inputs: x = (f - mu) * (1 / sigma)
__device__ __forceinline__ float standardise(float f, float mu, float inv_sigma) { return (f - mu) * inv_sigma; }

// The 16 raw inputs of one cell from its LITE vector and tau, in FP32.
__device__ __forceinline__ void lite_raw_features(const double *__restrict__ m, double tau, float (&f)[16]) {
  const float th = narrow(m[4]);
  const float u00 = narrow(m[5]), u01 = narrow(m[6]), u02 = narrow(m[7]), u11 = narrow(m[8]), u12 = narrow(m[9]),
              u22 = narrow(m[10]);
  f[0] = narrow(m[0]);
  f[1] = th;
  f[2] = narrow(m[1]);
  f[3] = narrow(m[2]);
  f[4] = narrow(m[3]);
  f[5] = u00 - th;
  f[6] = u01;
  f[7] = u02;
  f[8] = u11 - th;
  f[9] = u12;
  f[10] = u22 - th;
  f[11] = 0.5f * narrow(m[11]);
  f[12] = 0.5f * narrow(m[12]);
  f[13] = 0.5f * narrow(m[13]);
  f[14] = fmaf(u00, fmaf(u11, u22, -u12 * u12), fmaf(-u01, fmaf(u01, u22, -u12 * u02), u02 * fmaf(u01, u12, -u11 * u02)));
  f[15] = 1.f / narrow(tau);
}

}  // namespace fpc
