// mlp.cu -- the learned closure's standalone input kernels (features and
// training rows), the exact per-cell fallback and the launchers of the
// network's passes (the kernels of the inference pass and of the fused
// closure are in mlp_tc.cu, those of training in mlp_train_tc.cu) (sm_103a).
//
// Features: the 25 moments of w = c / sqrt(theta) (u/theta, u3/theta^1.5,
// w/theta^2, z/theta^2.5), standardised, BF16, zero padded to 32.  The
// network maps them to the standardised dimensionless coefficients
// (tau C, tau sqrt(theta) G); the cubic-FP system of Eq. system9x9 is
// invariant under c -> c/sqrt(theta), so those depend on the features alone.
#include <cstdint>
#include <cuda_bf16.h>

#include "closure_math.cuh"
#include "fp_device.cuh"
#include "mlp_common.cuh"

namespace fpc {

// ---------------------------------------------------------------------------
// features
// ---------------------------------------------------------------------------
// (the moments narrowed to FP32 by `narrow`)
__device__ __forceinline__ void cell_features(const double *__restrict__ m, float (&f)[kNFeat]) {
  const float th = narrow(m[kTheta]);
  const float i1 = 1.f / th;
  const float ih = rsqrtf(th);
  const float i15 = i1 * ih, i2 = i1 * i1, i25 = i2 * ih;
#pragma unroll
  for (int a = 0; a < 6; ++a) f[a] = narrow(m[kU2 + a]) * i1;
#pragma unroll
  for (int a = 0; a < 10; ++a) f[6 + a] = narrow(m[kU3 + a]) * i15;
#pragma unroll
  for (int a = 0; a < 6; ++a) f[16 + a] = narrow(m[kW + a]) * i2;
#pragma unroll
  for (int a = 0; a < 3; ++a) f[22 + a] = narrow(m[kZ + a]) * i25;
}

__global__ void __launch_bounds__(256) features_kernel(MlpDev net, const double *__restrict__ mom,
                                                       const double *__restrict__ tau, int64_t n, int min_particles,
                                                       float margin, __nv_bfloat16 *__restrict__ x,
                                                       int32_t *__restrict__ flags) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double *m = mom + c * FP_NMOM;
  int fl = 0;
  bool fin = finite_d(tau[c]) && positive_d(tau[c]);
#pragma unroll
  for (int k = 0; k < FP_NMOM; ++k) fin = fin && finite_d(m[k]);
  if (!fin) fl |= FP_FLAG_NONFINITE;
  if (narrow(m[kN]) < (float)min_particles) fl |= FP_FLAG_FEW;  // N is a whole number
  if (!positive_d(m[kTheta])) fl |= FP_FLAG_SINGULAR;
  float f[kNFeat];
  cell_features(m, f);
  uint32_t packed[kIn / 2];
#pragma unroll
  for (int k = 0; k < kIn; k += 2) {
    float xs[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = k + h;
      if (q < kNFeat) {
        const float sg = net.x_sigma[q];
        const float lo = net.x_min[q] - margin * sg, hi = net.x_max[q] + margin * sg;
        if (!(f[q] >= lo && f[q] <= hi)) fl |= FP_FLAG_RANGE;
        xs[h] = standardise(f[q], net.x_mu[q], 1.f / sg);
      }
    }
    packed[k / 2] = pack_bf16(xs[0], xs[1]);
  }
  uint4 *dst = reinterpret_cast<uint4 *>(x + c * kIn);
#pragma unroll
  for (int q = 0; q < kIn / 8; ++q)
    dst[q] = make_uint4(packed[4 * q], packed[4 * q + 1], packed[4 * q + 2], packed[4 * q + 3]);
  flags[c] = fl;
}

// What training reads for each cell, by the arithmetic of the inference
// kernels: the unstandardised inputs (the full set from moment vectors, the
// LITE set from LITE vectors and tau), the dimensionless targets
// (tau C, tau sqrt(theta) G) of the exact coefficients, and the loss's
// auxiliary normalised moments (u^_ij, b^_i = u^_ikk, s4^ = w^_kk) of the full
// features.  Rows are zero padded to 32 / 16 / 16 floats.
__global__ void __launch_bounds__(256) training_rows_kernel(const double *__restrict__ mom,
                                                            const double *__restrict__ lite,
                                                            const double *__restrict__ coeffs,
                                                            const double *__restrict__ tau, int64_t n, int lite_inputs,
                                                            float *__restrict__ raw, float *__restrict__ targ,
                                                            float *__restrict__ aux) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  float f[kNFeat];
  if (mom) cell_features(mom + c * FP_NMOM, f);
  if (raw) {
    float r[kIn];
#pragma unroll
    for (int q = 0; q < kIn; ++q) r[q] = 0.f;
    if (lite_inputs) {
      float g[16];
      lite_raw_features(lite + c * FP_NLITE, tau[c], g);
#pragma unroll
      for (int q = 0; q < 16; ++q) r[q] = g[q];
    } else {
#pragma unroll
      for (int q = 0; q < kNFeat; ++q) r[q] = f[q];
    }
    float4 *dst = reinterpret_cast<float4 *>(raw + c * kIn);
#pragma unroll
    for (int q = 0; q < kIn / 4; ++q) dst[q] = make_float4(r[4 * q], r[4 * q + 1], r[4 * q + 2], r[4 * q + 3]);
  }
  if (targ) {
    const double tc = tau[c];
    const double gs = tc * sqrt(mom[c * FP_NMOM + kTheta]);
    float t[kOut];
#pragma unroll
    for (int a = 0; a < kOut; ++a) t[a] = 0.f;
#pragma unroll
    for (int a = 0; a < 6; ++a) t[a] = d2f_rn(coeffs[c * 9 + a] * tc);
#pragma unroll
    for (int a = 6; a < 9; ++a) t[a] = d2f_rn(coeffs[c * 9 + a] * gs);
    float4 *dst = reinterpret_cast<float4 *>(targ + c * kOut);
#pragma unroll
    for (int q = 0; q < kOut / 4; ++q) dst[q] = make_float4(t[4 * q], t[4 * q + 1], t[4 * q + 2], t[4 * q + 3]);
  }
  if (aux) {
    float x[kOut];
#pragma unroll
    for (int a = 0; a < kOut; ++a) x[a] = 0.f;
#pragma unroll
    for (int a = 0; a < 6; ++a) x[a] = f[a];
    x[6] = f[6 + 0] + f[6 + 3] + f[6 + 5];
    x[7] = f[6 + 1] + f[6 + 6] + f[6 + 8];
    x[8] = f[6 + 2] + f[6 + 7] + f[6 + 9];
    x[9] = f[16] + f[19] + f[21];
    float4 *dst = reinterpret_cast<float4 *>(aux + c * kOut);
#pragma unroll
    for (int q = 0; q < kOut / 4; ++q) dst[q] = make_float4(x[4 * q], x[4 * q + 1], x[4 * q + 2], x[4 * q + 3]);
  }
}

// ---------------------------------------------------------------------------
// fallback: the exact closure on the cells the fused kernel listed
// ---------------------------------------------------------------------------
// A short list (the usual case: a few hundred cells) is latency-bound: each
// cell goes to a half warp (closure_cell_group16), and consecutive entries go
// to consecutive blocks so that they spread over every SM.  A long list (an
// untrained or out-of-distribution network) is throughput-bound: one thread
// per cell (closure_cell).  Both give the same coefficients and flags.
constexpr int kFallbackThreads = 128;

__global__ void __launch_bounds__(kFallbackThreads) fallback_kernel(const int32_t *__restrict__ list,
                                                                    const uint32_t *__restrict__ count,
                                                                    const double *__restrict__ mom,
                                                                    const double *__restrict__ tau, SolveParams prm,
                                                                    double *__restrict__ coeffs,
                                                                    int32_t *__restrict__ flags) {
  const uint32_t cnt = *count;
  const uint32_t groups = gridDim.x * (kFallbackThreads / 16);  // half warps in the grid
  if (cnt <= 2 * groups) {
    const int r = threadIdx.x & 15;
    // a warp runs only while its first half holds a cell (the solve is
    // FP64-bound: idle warps must not compete for the pipe)
    const uint32_t first = (threadIdx.x >> 5) * 2 * gridDim.x + blockIdx.x;
    for (uint32_t base = 0; base + first < cnt; base += groups) {  // uniform over the warp
      const uint32_t i = base + (threadIdx.x >> 4) * gridDim.x + blockIdx.x;
      const bool valid = i < cnt;
      const int64_t c = valid ? list[i] : 0;
      double y[9];
      const int fe = closure_cell_group16(mom + c * FP_NMOM, valid ? tau[c] : 1.0, prm, valid, r, y);
      if (valid) {
        double *yc = coeffs + c * 9;
#pragma unroll
        for (int q = 0; q < 9; ++q)
          if (q == r) yc[q] = y[q];
        if (r == 0) flags[c] = fe | (flags[c] & (FP_FLAG_RANGE | FP_FLAG_ENERGY)) | FP_FLAG_FALLBACK;
      }
    }
    return;
  }
  for (uint32_t i = blockIdx.x * kFallbackThreads + threadIdx.x; i < cnt; i += gridDim.x * kFallbackThreads) {
    const int64_t c = list[i];
    double y[9];
    const int fe = closure_cell(mom + c * FP_NMOM, tau[c], prm, y);
    double *yc = coeffs + c * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) yc[q] = y[q];
    flags[c] = fe | (flags[c] & (FP_FLAG_RANGE | FP_FLAG_ENERGY)) | FP_FLAG_FALLBACK;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int mlp_sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

int launch_mlp_forward_tc(const MlpDev &net, const __nv_bfloat16 *x, int64_t n, int standardized_out, float *out,
                          cudaStream_t st);

MlpDev make_mlp_dev(const fp_mlp &m) {
  MlpDev d;
  for (int l = 0; l < 5; ++l) {
    d.W[l] = reinterpret_cast<const __nv_bfloat16 *>(m.W[l]);
    d.b[l] = m.b[l];
  }
  d.x_mu = m.x_mu;
  d.x_sigma = m.x_sigma;
  d.y_mu = m.y_mu;
  d.y_sigma = m.y_sigma;
  d.x_min = m.x_min;
  d.x_max = m.x_max;
  return d;
}

void launch_features(const fp_mlp &net, const double *mom, const double *tau, int64_t n, int min_particles,
                     double margin, void *x, int32_t *flags, cudaStream_t st) {
  const int64_t blocks = (n + 255) / 256;
  features_kernel<<<(unsigned)blocks, 256, 0, st>>>(make_mlp_dev(net), mom, tau, n, min_particles, (float)margin,
                                                     reinterpret_cast<__nv_bfloat16 *>(x), flags);
}

void launch_training_rows(const double *mom, const double *lite, const double *coeffs, const double *tau, int64_t n,
                          int lite_inputs, float *raw, float *targ, float *aux, cudaStream_t st) {
  const int64_t blocks = (n + 255) / 256;
  training_rows_kernel<<<(unsigned)blocks, 256, 0, st>>>(mom, lite, coeffs, tau, n, lite_inputs, raw, targ, aux);
}

int launch_mlp_forward_tc_dropout(const MlpDev &net, const __nv_bfloat16 *x, int64_t n, int standardized_out,
                                  float *out, const DropoutCfg &dc, cudaStream_t st);

// One inference pass with dropout masks (pass `pass` of the sensitivity
// probe); un-standardised outputs.
int launch_mlp_forward_dropout(const fp_mlp &net, const void *x, int64_t n, float *out, double rate, uint64_t seed,
                               uint32_t pass, cudaStream_t st) {
  DropoutCfg dc;
  dc.key = philox_keys(seed);
  dc.rate = (float)rate;
  dc.scale = (float)(1.0 / (1.0 - rate));
  dc.pass = pass;
  return launch_mlp_forward_tc_dropout(make_mlp_dev(net), reinterpret_cast<const __nv_bfloat16 *>(x), n, 0, out, dc,
                                       st);
}

int launch_mlp_forward_train_tc(const MlpDev &net, const void *x, int64_t n, int standardized_out, float *out,
                                void *h_save, float *z_save, cudaStream_t st);

int launch_mlp_forward(const fp_mlp &net, const void *x, int64_t n, int standardized_out, float *out, void *h_save,
                       float *z_save, cudaStream_t st) {
  const MlpDev d = make_mlp_dev(net);
  const __nv_bfloat16 *xb = reinterpret_cast<const __nv_bfloat16 *>(x);
  // inference: the persistent tcgen05 kernel; training (activations saved
  // for the backward pass): the tile-per-CTA tcgen05 kernel of mlp_train_tc.cu
  if (h_save == nullptr || z_save == nullptr) return launch_mlp_forward_tc(d, xb, n, standardized_out, out, st);
  return launch_mlp_forward_train_tc(d, xb, n, standardized_out, out, h_save, z_save, st);
}

int launch_closure_surrogate_tc(const MlpDev &net, const FusedIO &io, int64_t n, int lite, cudaStream_t st);

// The learned closure on full inputs: one fused kernel (inputs, network,
// coefficients, checks, fallback list), then the exact closure on the listed
// cells.  Returns -1 if the shared-memory limit could not be raised.
int launch_closure_surrogate(const fp_mlp &net, const double *mom, const double *tau, int64_t n, double eps2_hat,
                             const fp_params &p, int prec, double *coeffs, int32_t *flags, int32_t *list,
                             uint32_t *count, cudaStream_t st) {
  const FusedIO io{mom, tau, p.min_particles, (float)p.surr_range_margin, (float)eps2_hat, (float)p.surr_energy_tol,
                   coeffs, flags, list, count};
  cudaMemsetAsync(count, 0, sizeof(uint32_t), st);
  if (launch_closure_surrogate_tc(make_mlp_dev(net), io, n, 0, st)) return -1;
  double rtol = p.pivot_rtol;
  if (prec == FP_PREC_FP32_MOMENTS && rtol < FP_FP32_PIVOT_FLOOR) rtol = FP_FP32_PIVOT_FLOOR;
  SolveParams prm{p.eps2_hat, rtol, p.min_particles, prec == FP_PREC_FP32_MOMENTS ? FP_FP32_MIN_REGULAR : 0};
  // two blocks per SM: the occupancy the one-thread-per-cell path allows
  fallback_kernel<<<(unsigned)(mlp_sm_count() * 2), kFallbackThreads, 0, st>>>(list, count, mom, tau, prm, coeffs,
                                                                              flags);
  return 0;
}

// The learned closure on LITE inputs: one fused kernel, no fallback list.
int launch_closure_surrogate_lite(const fp_mlp &net, const double *lite, const double *tau, int64_t n,
                                  const fp_params &p, double *coeffs, int32_t *flags, cudaStream_t st) {
  const FusedIO io{lite, tau, p.min_particles, (float)p.surr_range_margin, 0.f, 0.f, coeffs, flags, nullptr, nullptr};
  return launch_closure_surrogate_tc(make_mlp_dev(net), io, n, 1, st);
}

}  // namespace fpc
