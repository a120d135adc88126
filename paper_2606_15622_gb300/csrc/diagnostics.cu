// diagnostics.cu -- per-cell high-order nonequilibrium diagnostics and the
// covariance-based entropy proxies of the paper's cavity and cylinder
// audits, from the gathered central moments and <|c|^6> (one thread per
// cell, FP64).  Definitions (c = v - U, theta = tr(Theta) / 3,
// Theta_ij = <c_i c_j>):
//   R_ij,norm   = <c_i c_j |c|^2> / theta^2       (local Maxwellian: 5 delta_ij)
//   Delta4,norm = <|c|^4> / theta^2 - 15            (Maxwellian: 0)
//   DM6,norm    = <|c|^6> / theta^3                 (Maxwellian: 105)
//   D_G         = -1/2 log det(Theta / theta)       (Eq. cyl_DG; >= 0)
//   D_q         = |q_hat|^2 / 5, q_hat = <c |c|^2> / (2 theta^1.5)
//   ds_eq       = 3/2 log(theta / theta_inf) - log(rho / rho_inf)  (Eq. cyl_entropy_eq)
//   ds_kin,G    = ds_eq - (D_G - D_G,inf)          (Eq. cyl_entropy_kinG)
// Cells with N < 2, theta <= 0, a non-finite moment or det(Theta) <= 0 get
// NaN in every entry.
#include <cstdint>

#include "closure_math.cuh"
#include "fp_device.cuh"

namespace fpc {

__global__ void __launch_bounds__(256) diagnostics_kernel(const double *__restrict__ mom,
                                                          const double *__restrict__ m6,
                                                          const double *__restrict__ rho, int64_t n_cells,
                                                          double theta_inf, double rho_inf, double dg_inf,
                                                          double *__restrict__ out) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n_cells) return;
  const double *m = mom + c * FP_NMOM;
  double *o = out + c * FP_NDIAG;
  const double th = m[kTheta];
  const double u00 = m[kU2 + 0], u01 = m[kU2 + 1], u02 = m[kU2 + 2], u11 = m[kU2 + 3], u12 = m[kU2 + 4],
               u22 = m[kU2 + 5];
  const double det = u00 * (u11 * u22 - u12 * u12) - u01 * (u01 * u22 - u12 * u02) + u02 * (u01 * u12 - u11 * u02);
  const double d = rho ? rho[c] : m[kN];
  bool ok = m[kN] >= 2.0 && th > 0.0 && det > 0.0 && finite_d(m6[c]) && d > 0.0;
#pragma unroll
  for (int k = 0; k < FP_NMOM; ++k) ok = ok && finite_d(m[k]);
  if (!ok) {
    const double nan = __longlong_as_double(0x7ff8000000000000ll);
#pragma unroll
    for (int k = 0; k < FP_NDIAG; ++k) o[k] = nan;
    return;
  }
  const double i2 = 1.0 / (th * th);
#pragma unroll
  for (int a = 0; a < 6; ++a) o[a] = m[kW + a] * i2;
  o[6] = (m[kW + 0] + m[kW + 3] + m[kW + 5]) * i2 - 15.0;
  o[7] = m6[c] * i2 / th;
  const double dg = -0.5 * log(det / (th * th * th));
  o[8] = dg;
  double qq = 0.0;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double b = m[kU3 + sym3(i, 0, 0)] + m[kU3 + sym3(i, 1, 1)] + m[kU3 + sym3(i, 2, 2)];
    qq += b * b;
  }
  o[9] = qq / (4.0 * th * th * th) / 5.0;
  const double ds_eq = 1.5 * log(th / theta_inf) - log(d / rho_inf);
  o[10] = ds_eq;
  o[11] = ds_eq - (dg - dg_inf);
}

void launch_diagnostics(const double *mom, const double *m6, const double *rho, int64_t n_cells, double theta_inf,
                        double rho_inf, double dg_inf, double *out, cudaStream_t st) {
  const int64_t blocks = (n_cells + 255) / 256;
  diagnostics_kernel<<<(unsigned)blocks, 256, 0, st>>>(mom, m6, rho, n_cells, theta_inf, rho_inf, dg_inf, out);
}

// Temporal under-relaxation of the coefficient field (the cylinder
// deployment of the learned closure): y = w y_new + (1 - w) y_prev, in place
// on y_prev, element by element.
__global__ void __launch_bounds__(256) relax_kernel(const double *__restrict__ y_new, double *__restrict__ y_prev,
                                                    int64_t n, double w) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) y_prev[i] = fma(w, y_new[i] - y_prev[i], y_prev[i]);
}

void launch_relax(const double *y_new, double *y_prev, int64_t n, double w, cudaStream_t st) {
  const int64_t blocks = (n + 255) / 256;
  relax_kernel<<<(unsigned)blocks, 256, 0, st>>>(y_new, y_prev, n, w);
}

}  // namespace fpc
