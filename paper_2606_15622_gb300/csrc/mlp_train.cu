// mlp_train.cu -- training kernels of the surrogate: the loss and its
// gradient and Adam, for sm_103a (the backward pass on the tensor cores is
// in mlp_train_tc.cu).
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
#include <cstdint>
#include <cuda_bf16.h>

#include "fp_device.cuh"
#include "mlp_common.cuh"

namespace fpc {

// ---------------------------------------------------------------------------
// loss
// ---------------------------------------------------------------------------
struct LossParams {
  float w[kNOut];
  float lam_d, lam_e, eps2_hat, scale;  // scale multiplies the gradient (1 / batch)
};

// A warp takes 32 consecutive rows: their out, aux and t_true rows are
// copied into shared memory with coalesced loads (rows of 16 padded to 17
// floats, so that the lanes' row reads fall in different banks), each lane
// computes its row, and dout goes back the same way.
constexpr int kLossWarps = 2;
constexpr int kLS = kOut + 1;  // padded row stride (floats)

__global__ void __launch_bounds__(32 * kLossWarps)
    loss_kernel(const float *__restrict__ out, const float *__restrict__ t_true, const float *__restrict__ aux,
                const float *__restrict__ y_mu, const float *__restrict__ y_sigma, int64_t n, LossParams prm,
                float *__restrict__ dout, __nv_bfloat16 *__restrict__ dout_bf, float *__restrict__ loss_sum) {
  __shared__ float s_o[kLossWarps][32 * kLS], s_a[kLossWarps][32 * kLS], s_t[kLossWarps][32 * kNOut];
  const int lane = threadIdx.x & 31, wq = threadIdx.x >> 5;
  const int64_t row0 = ((int64_t)blockIdx.x * kLossWarps + wq) * 32, r = row0 + lane;
  const int nr = (int)(n - row0 < 32 ? (n - row0 > 0 ? n - row0 : 0) : 32);  // rows of this warp
  float *so = s_o[wq], *sa = s_a[wq], *sT = s_t[wq];
  for (int i = lane; i < nr * kOut; i += 32) {
    so[(i / kOut) * kLS + i % kOut] = out[row0 * kOut + i];
    sa[(i / kOut) * kLS + i % kOut] = aux[row0 * 16 + i];
  }
  for (int i = lane; i < nr * kNOut; i += 32) sT[i] = t_true[row0 * kNOut + i];
  __syncwarp();
  float lsum = 0.f;
  if (r < n) {
    const float *orow = so + lane * kLS, *trow = sT + lane * kNOut;
    float o[kNOut], d[kNOut], gr[kNOut];
#pragma unroll
    for (int a = 0; a < kNOut; ++a) {
      o[a] = orow[a];
      const float tp = y_mu[a] + y_sigma[a] * o[a];
      d[a] = tp - trow[a];
    }
    const float *x = sa + lane * kLS;  // u_hat (6), b_hat (3), s4_hat
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
    lsum = mse + prm.lam_d * q + prm.lam_e * e * e;
    float *drow = so + lane * kLS;  // this lane's out row is no longer needed
#pragma unroll
    for (int a = 0; a < kOut; ++a) drow[a] = a < kNOut ? gr[a] * prm.scale : 0.f;
  }
  __syncwarp();
  for (int i = lane; i < nr * kOut; i += 32) {
    const float v = so[(i / kOut) * kLS + i % kOut];
    dout[row0 * kOut + i] = v;
    dout_bf[row0 * kOut + i] = __float2bfloat16_rn(v);
  }
  // block sum of the loss
#pragma unroll
  for (int o2 = 16; o2 >= 1; o2 >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o2);
  __shared__ float ws[8];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = lsum;
  __syncthreads();
  if (threadIdx.x == 0) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += ws[i];
    atomicAdd(loss_sum, s);
  }
}

__global__ void adam_kernel(float *__restrict__ p, const float *__restrict__ gr, float *__restrict__ m,
                            float *__restrict__ v, int64_t n, float lr, float b1, float b2, float eps, float bc1,
                            float bc2, __nv_bfloat16 *__restrict__ shadow) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const float g = gr[i];
  const float mi = b1 * m[i] + (1.f - b1) * g;
  const float vi = b2 * v[i] + (1.f - b2) * g * g;
  m[i] = mi;
  v[i] = vi;
  const float pi = p[i] - lr * (mi / bc1) / (sqrtf(vi / bc2) + eps);
  p[i] = pi;
  if (shadow) shadow[i] = __float2bfloat16_rn(pi);
}

// ---------------------------------------------------------------------------
// host side
// ---------------------------------------------------------------------------
// flat parameter layout: W1 | b1 | W2 | b2 | W3 | b3 | W4 | b4 | W5 | b5
int64_t mlp_param_offset(int which, int layer) {
  const int64_t wsz[5] = {kHid * kIn, kHid * kHid, kHid * kHid, kHid * kHid, kOut * kHid};
  const int64_t bsz[5] = {kHid, kHid, kHid, kHid, kOut};
  int64_t off = 0;
  for (int l = 0; l < layer; ++l) off += wsz[l] + bsz[l];
  return which == 0 ? off : off + wsz[layer];
}
int64_t mlp_param_count() { return mlp_param_offset(1, 4) + kOut; }

size_t mlp_backward_tc_ws(int64_t n);
int launch_mlp_backward_tc(const MlpDev &net, const void *x, const void *h_save, const float *z_save,
                           const void *dout_bf, const float *dout, int64_t n, float *grads, void *ws,
                           cudaStream_t st);
MlpDev make_mlp_dev(const fp_mlp &m);

size_t mlp_backward_ws(int64_t n) { return mlp_backward_tc_ws(n); }

// the backward pass on the tensor cores (mlp_train_tc.cu); -1 if it could not be launched
int launch_mlp_backward(const fp_mlp &net, const void *x, const void *h_save, const float *z_save,
                        const void *dout_bf, const float *dout, int64_t n, float *grads, void *ws, cudaStream_t st) {
  return launch_mlp_backward_tc(make_mlp_dev(net), x, h_save, z_save, dout_bf, dout, n, grads, ws, st);
}

void launch_loss(const float *out, const float *t_true, const float *aux, const float *y_mu, const float *y_sigma,
                 int64_t n, const float *w, float lam_d, float lam_e, float eps2_hat, float scale, float *dout,
                 void *dout_bf, float *loss_sum, cudaStream_t st) {
  LossParams prm;
  for (int a = 0; a < kNOut; ++a) prm.w[a] = w[a];
  prm.lam_d = lam_d;
  prm.lam_e = lam_e;
  prm.eps2_hat = eps2_hat;
  prm.scale = scale;
  loss_kernel<<<(unsigned)((n + 32 * kLossWarps - 1) / (32 * kLossWarps)), 32 * kLossWarps, 0, st>>>(out, t_true, aux, y_mu, y_sigma, n, prm, dout,
                                                            reinterpret_cast<__nv_bfloat16 *>(dout_bf), loss_sum);
}

void launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, void *shadow, cudaStream_t st) {
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2,
                                                            reinterpret_cast<__nv_bfloat16 *>(shadow));
}

}  // namespace fpc
