// train_math.cuh -- the training loss of the surrogate for one row and its
// gradient with respect to the standardised network outputs (shared by the
// loss kernel and the training forward that fuses it), and the Adam update of
// one parameter (shared by the Adam kernel and the gradient tile sum that
// fuses it).
//
// Loss per cell (dimensionless targets t, prediction t' = mu + sigma o):
//   sum_a w_a (o_a - (t_a - mu_a) / sigma_a)^2              coefficient MSE
//   + lam_d [tr(D u D) + 2 g.D b + |g|^2 (s4 - 9)]          induced drift
//   + lam_e e^2                                              energy residual
// with (D, g) = t' - t split into the symmetric C block and the G block and
// u, b, s4 the cell's normalised moments: tr(D u D) + ... is the mean square
// over the cell of the difference of the drifts of Eq. cubic_drift the two
// coefficient sets induce (times tau^2 / theta), and
// e = 1 + (sum_ij C'_ij u_ij + sum_i G'_i b_i - eps2_hat s4) / 3 the energy
// residual (zero for the exact closure: the trace of its stress rows).
#pragma once
#include <cuda_bf16.h>

#include "mlp_common.cuh"

namespace fpc {

struct LossParams {
  float w[kNOut];
  float lam_d, lam_e, eps2_hat, scale;  // scale multiplies the gradient (1 / batch)
};

// o: the row's standardised outputs (the first kNOut used); trow: its kNOut
// targets; x: its aux row (u_hat (6), b_hat (3), s4_hat); y_mu, y_sigma: the
// output scalers.  Returns the row's loss and writes dL/do (unscaled) to gr.
__device__ __forceinline__ float loss_row(const float *o_in, const float *trow, const float *x, const float *y_mu,
                                          const float *y_sigma, const LossParams &prm, float (&gr)[kNOut]) {
  float o[kNOut], d[kNOut];
#pragma unroll
  for (int a = 0; a < kNOut; ++a) {
    o[a] = o_in[a];
    const float tp = y_mu[a] + y_sigma[a] * o[a];
    d[a] = tp - trow[a];
  }
  const float U[3][3] = {{x[0], x[1], x[2]}, {x[1], x[3], x[4]}, {x[2], x[4], x[5]}};
  const float b[3] = {x[6], x[7], x[8]};
  const float s4 = x[9];
  const float D[3][3] = {{d[0], d[1], d[2]}, {d[1], d[3], d[4]}, {d[2], d[4], d[5]}};
  const float g[3] = {d[6], d[7], d[8]};
  // drift term and its gradient
  float DU[3][3], Db[3];
  float q = 0.f;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    Db[i] = D[i][0] * b[0] + D[i][1] * b[1] + D[i][2] * b[2];
#pragma unroll
    for (int j = 0; j < 3; ++j) DU[i][j] = D[i][0] * U[0][j] + D[i][1] * U[1][j] + D[i][2] * U[2][j];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j) q += DU[i][j] * D[j][i];
    q += 2.f * g[i] * Db[i] + g[i] * g[i] * (s4 - 9.f);
  }
  float full[3][3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) full[i][j] = 2.f * DU[i][j] + 2.f * g[i] * b[j];
  const int si[6] = {0, 0, 0, 1, 1, 2}, sj[6] = {0, 1, 2, 1, 2, 2};
  float gq[kNOut];
#pragma unroll
  for (int a = 0; a < 6; ++a) gq[a] = si[a] == sj[a] ? full[si[a]][sj[a]] : full[si[a]][sj[a]] + full[sj[a]][si[a]];
#pragma unroll
  for (int i = 0; i < 3; ++i) gq[6 + i] = 2.f * Db[i] + 2.f * (s4 - 9.f) * g[i];
  // energy residual of the prediction
  const float mult[6] = {1.f, 2.f, 2.f, 1.f, 2.f, 1.f};
  const float uh[6] = {x[0], x[1], x[2], x[3], x[4], x[5]};
  float e = 1.f - prm.eps2_hat * s4 / 3.f;
  float de[kNOut];
#pragma unroll
  for (int a = 0; a < 6; ++a) {
    const float tp = y_mu[a] + y_sigma[a] * o[a];
    de[a] = mult[a] * uh[a] / 3.f;
    e += tp * de[a];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const float tp = y_mu[6 + i] + y_sigma[6 + i] * o[6 + i];
    de[6 + i] = b[i] / 3.f;
    e += tp * de[6 + i];
  }
  float mse = 0.f;
#pragma unroll
  for (int a = 0; a < kNOut; ++a) {
    const float z = (trow[a] - y_mu[a]) / y_sigma[a];
    const float df = o[a] - z;
    mse += prm.w[a] * df * df;
    gr[a] = 2.f * prm.w[a] * df + y_sigma[a] * (prm.lam_d * gq[a] + prm.lam_e * 2.f * e * de[a]);
  }
  return mse + prm.lam_d * q + prm.lam_e * e * e;
}

// Adam (Kingma & Ba) on parameter i with gradient g: moments m, v, bias
// corrections bc1 = 1 - b1^t, bc2 = 1 - b2^t; the BF16 copy of the parameter
// is refreshed when shadow is not null
struct AdamParams {
  float *p, *m, *v;
  __nv_bfloat16 *shadow;
  float lr, b1, b2, eps, bc1, bc2;
};

__device__ __forceinline__ void adam_update(const AdamParams &a, int64_t i, float g) {
  const float mi = a.b1 * a.m[i] + (1.f - a.b1) * g;
  const float vi = a.b2 * a.v[i] + (1.f - a.b2) * g * g;
  a.m[i] = mi;
  a.v[i] = vi;
  const float pi = a.p[i] - a.lr * (mi / a.bc1) / (sqrtf(vi / a.bc2) + a.eps);
  a.p[i] = pi;
  if (a.shadow) a.shadow[i] = __float2bfloat16_rn(pi);
}

}  // namespace fpc
