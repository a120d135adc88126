// sensitivity.cu -- the heuristic coefficient-sensitivity probe of the
// learned closure (the cylinder study's dropout probe): N forward passes with
// the hidden activations dropped at a given rate (each pass its own Philox
// masks, mlp_tc.cu), per cell the standard deviation over the passes of each
// predicted coefficient (1/N normalisation, Welford's update in FP64) and the
// aggregates sigma_Stress = |sigma over the six C entries| and sigma_Heat =
// |sigma over the three Gamma entries| (Euclidean norms).
#include <cstdint>

#include "fp_device.cuh"
#include "mlp_common.cuh"

namespace fpc {

// pass k (1-based) of the un-standardised network outputs tpred [n][16]
__global__ void __launch_bounds__(256) sens_accumulate_kernel(const float *__restrict__ tpred, int64_t n, double inv_k,
                                                              double *__restrict__ mean, double *__restrict__ m2) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
#pragma unroll
  for (int a = 0; a < kNOut; ++a) {
    const double y = (double)tpred[c * kOut + a];
    const double mo = mean[c * kNOut + a];
    const double d = y - mo;
    const double mn = fma(d, inv_k, mo);
    mean[c * kNOut + a] = mn;
    m2[c * kNOut + a] = fma(d, y - mn, m2[c * kNOut + a]);
  }
}

// sigma of the physical coefficients: C entries are t / tau, Gamma entries
// t / (tau sqrt(theta)); cells the features flag as degenerate get NaN
__global__ void __launch_bounds__(256) sens_finalize_kernel(const double *__restrict__ mean,
                                                            const double *__restrict__ m2,
                                                            const double *__restrict__ mom, int stride,
                                                            const double *__restrict__ tau, int64_t n,
                                                            double inv_n, const int32_t *__restrict__ flags,
                                                            double *__restrict__ out, double *__restrict__ mean_out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  double *o = out + c * FP_NSENS;
  if (flags[c] & (FP_FLAG_FEW | FP_FLAG_SINGULAR | FP_FLAG_NONFINITE)) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
    for (int a = 0; a < FP_NSENS; ++a) o[a] = nan;
    if (mean_out)
#pragma unroll
      for (int a = 0; a < kNOut; ++a) mean_out[c * kNOut + a] = nan;
    return;
  }
  const double itc = 1.0 / tau[c];
  const double ig = itc / sqrt(mom[c * stride + kTheta]);
  double ss = 0.0, sh = 0.0;
#pragma unroll
  for (int a = 0; a < kNOut; ++a) {
    const double f = a < 6 ? itc : ig;
    const double s = sqrt(fmax(m2[c * kNOut + a] * inv_n, 0.0)) * f;
    o[a] = s;
    if (a < 6)
      ss = fma(s, s, ss);
    else
      sh = fma(s, s, sh);
    if (mean_out) mean_out[c * kNOut + a] = mean[c * kNOut + a] * f;
  }
  o[9] = sqrt(ss);
  o[10] = sqrt(sh);
}

void launch_sens_accumulate(const float *tpred, int64_t n, int k, double *mean, double *m2, cudaStream_t st) {
  const int64_t blocks = (n + 255) / 256;
  sens_accumulate_kernel<<<(unsigned)blocks, 256, 0, st>>>(tpred, n, 1.0 / (double)k, mean, m2);
}

void launch_sens_finalize(const double *mean, const double *m2, const double *mom, int stride, const double *tau,
                          int64_t n, int n_passes, const int32_t *flags, double *out, double *mean_out,
                          cudaStream_t st) {
  const int64_t blocks = (n + 255) / 256;
  sens_finalize_kernel<<<(unsigned)blocks, 256, 0, st>>>(mean, m2, mom, stride, tau, n, 1.0 / (double)n_passes,
                                                         flags, out, mean_out);
}

}  // namespace fpc
