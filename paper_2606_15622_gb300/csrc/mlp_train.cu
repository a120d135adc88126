// mlp_train.cu -- training kernels of the surrogate: the loss and its
// gradient (the per-row arithmetic is in train_math.cuh) and Adam, for sm_103a
// (the training forward and the backward pass on the tensor cores are in
// mlp_train_tc.cu).
#include <cstdint>
#include <cuda_bf16.h>

#include "fp_device.cuh"
#include "mlp_common.cuh"
#include "train_math.cuh"

namespace fpc {

// ---------------------------------------------------------------------------
// loss
// ---------------------------------------------------------------------------
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
    float gr[kNOut];
    lsum = loss_row(orow, trow, sa + lane * kLS, y_mu, y_sigma, prm, gr);
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

__global__ void adam_kernel(const float *__restrict__ gr, int64_t n, AdamParams a) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  adam_update(a, i, gr[i]);
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
int launch_mlp_backward_adam_tc(const MlpDev &net, const void *x, const void *h_save, const float *z_save,
                                const void *dout_bf, const float *dout, int64_t n, float *grads, void *ws,
                                const AdamParams *adam, cudaStream_t st);
int launch_mlp_forward_loss_tc(const MlpDev &net, const void *x, int64_t n, int standardized_out, float *out,
                               void *h_save, float *z_save, const float *t_true, const float *aux,
                               const LossParams *lp, float *dout, void *dout_bf, float *loss_sum, cudaStream_t st);
MlpDev make_mlp_dev(const fp_mlp &m);

size_t mlp_backward_ws(int64_t n) { return mlp_backward_tc_ws(n); }

// the backward pass on the tensor cores (mlp_train_tc.cu); -1 if it could not be launched
int launch_mlp_backward(const fp_mlp &net, const void *x, const void *h_save, const float *z_save,
                        const void *dout_bf, const float *dout, int64_t n, float *grads, void *ws, cudaStream_t st) {
  return launch_mlp_backward_tc(make_mlp_dev(net), x, h_save, z_save, dout_bf, dout, n, grads, ws, st);
}

// ---------------------------------------------------------------------------
// one training step: forward with the loss fused into its last layer, then
// the backward pass with Adam fused into the tile sum (two kernels each)
// ---------------------------------------------------------------------------
namespace {
constexpr size_t kTsAlign = 256;
size_t ts_round(size_t b) { return (b + kTsAlign - 1) / kTsAlign * kTsAlign; }
}  // namespace

// workspace: h_save | z_save | dout | dout_bf | the backward's tile slots
size_t train_step_ws(int64_t n) {
  const size_t rows = (size_t)n;
  return ts_round(rows * kDepth * kHid * 2) + ts_round(rows * kDepth * kHid * 4) + ts_round(rows * kOut * 4) +
         ts_round(rows * kOut * 2) + ts_round(mlp_backward_tc_ws(n));
}

int launch_train_step(const fp_mlp &net, const void *x, const float *t_true, const float *aux, int64_t n,
                      const float *w, float lam_d, float lam_e, float scale, float *grads, const AdamParams &adam,
                      float *loss_sum, void *ws, cudaStream_t st) {
  const size_t rows = (size_t)n;
  char *c = reinterpret_cast<char *>(ws);
  void *h_save = c;
  c += ts_round(rows * kDepth * kHid * 2);
  float *z_save = reinterpret_cast<float *>(c);
  c += ts_round(rows * kDepth * kHid * 4);
  float *dout = reinterpret_cast<float *>(c);
  c += ts_round(rows * kOut * 4);
  void *dout_bf = c;
  c += ts_round(rows * kOut * 2);
  LossParams prm;
  for (int a = 0; a < kNOut; ++a) prm.w[a] = w[a];
  prm.lam_d = lam_d;
  prm.lam_e = lam_e;
  prm.eps2_hat = (float)net.eps2_hat;
  prm.scale = scale;
  const MlpDev d = make_mlp_dev(net);
  if (launch_mlp_forward_loss_tc(d, x, n, 1, nullptr, h_save, z_save, t_true, aux, &prm, dout, dout_bf, loss_sum,
                                 st))
    return -1;
  return launch_mlp_backward_adam_tc(d, x, h_save, z_save, dout_bf, dout, n, grads, c, &adam, st);
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
  const AdamParams a{p, m, v, reinterpret_cast<__nv_bfloat16 *>(shadow), lr, b1, b2, eps, bc1, bc2};
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(g, n, a);
}

}  // namespace fpc
