// mlp_train.cu -- training kernels of the surrogate: the loss and its
// gradient, the backward pass (BF16 tensor-core GEMMs with FP32
// accumulation) and Adam, for sm_103a.
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

__global__ void __launch_bounds__(256) loss_kernel(const float *__restrict__ out, const float *__restrict__ t_true,
                                                   const float *__restrict__ aux, const float *__restrict__ y_mu,
                                                   const float *__restrict__ y_sigma, int64_t n, LossParams prm,
                                                   float *__restrict__ dout, __nv_bfloat16 *__restrict__ dout_bf,
                                                   float *__restrict__ loss_sum) {
  const int64_t r = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  float lsum = 0.f;
  if (r < n) {
    float o[kNOut], d[kNOut], gr[kNOut];
#pragma unroll
    for (int a = 0; a < kNOut; ++a) {
      o[a] = out[r * kOut + a];
      const float tp = y_mu[a] + y_sigma[a] * o[a];
      d[a] = tp - t_true[r * kNOut + a];
    }
    const float *x = aux + r * 16;  // u_hat (6), b_hat (3), s4_hat
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
      const float z = (t_true[r * kNOut + a] - y_mu[a]) / y_sigma[a];
      const float df = o[a] - z;
      mse += prm.w[a] * df * df;
      gr[a] = 2.f * prm.w[a] * df + y_sigma[a] * (prm.lam_d * gq[a] + prm.lam_e * 2.f * e * de[a]);
    }
    lsum = mse + prm.lam_d * q + prm.lam_e * e * e;
#pragma unroll
    for (int a = 0; a < kOut; ++a) {
      const float v = a < kNOut ? gr[a] * prm.scale : 0.f;
      dout[r * kOut + a] = v;
      dout_bf[r * kOut + a] = __float2bfloat16_rn(v);
    }
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

// ---------------------------------------------------------------------------
// generic BF16 GEMM (mma.sync m16n8k16, FP32 accumulation)
//   C(m, n) = sum_k A(m, k) B(k, n),  A(m,k) = A[m sam + k sak], B(k,n) = B[k sbk + n sbn]
// EPI 0: FP32 partial for K-split blockIdx.z at outf + z M ldo
// EPI 1: BF16 C(m, n) silu'(Z(m, n)) at outb (the next layer's dZ)
// ---------------------------------------------------------------------------
constexpr int kGT = 64, kGK = 32, kGS = kGK + 8;

template <int EPI>
__global__ void __launch_bounds__(128) gemm_kernel(int M, int N, int K, int k_chunk, const __nv_bfloat16 *__restrict__ A,
                                                   int64_t sam, int64_t sak, const __nv_bfloat16 *__restrict__ B,
                                                   int64_t sbk, int64_t sbn, float *__restrict__ outf,
                                                   __nv_bfloat16 *__restrict__ outb, int64_t ldo,
                                                   const float *__restrict__ Z, int64_t ldz) {
  __shared__ __align__(16) __nv_bfloat16 As[kGT][kGS], Bs[kGT][kGS];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int g = lane >> 2, t = lane & 3;
  const int m0 = blockIdx.y * kGT, n0 = blockIdx.x * kGT;
  const int kbeg = blockIdx.z * k_chunk;
  const int kend = min(K, kbeg + k_chunk);
  const int wm = (warp & 1) * 32, wn = (warp >> 1) * 32;
  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j) acc[i][j][0] = acc[i][j][1] = acc[i][j][2] = acc[i][j][3] = 0.f;
  const __nv_bfloat16 zero = __float2bfloat16_rn(0.f);
  for (int kk = kbeg; kk < kend; kk += kGK) {
    for (int e = tid; e < kGT * kGK; e += 128) {
      int m, k;
      if (sak == 1) {
        m = e / kGK;
        k = e % kGK;
      } else {
        k = e / kGT;
        m = e % kGT;
      }
      As[m][k] = (m0 + m < M && kk + k < kend) ? A[(int64_t)(m0 + m) * sam + (int64_t)(kk + k) * sak] : zero;
      int n2, k2;
      if (sbn == 1) {
        k2 = e / kGT;
        n2 = e % kGT;
      } else {
        n2 = e / kGK;
        k2 = e % kGK;
      }
      Bs[n2][k2] = (n0 + n2 < N && kk + k2 < kend) ? B[(int64_t)(kk + k2) * sbk + (int64_t)(n0 + n2) * sbn] : zero;
    }
    __syncthreads();
#pragma unroll
    for (int ks = 0; ks < kGK; ks += 16) {
      uint32_t a[2][4], b[4][2];
#pragma unroll
      for (int mt = 0; mt < 2; ++mt) {
        const int r = wm + mt * 16 + g;
        a[mt][0] = *reinterpret_cast<const uint32_t *>(&As[r][ks + 2 * t]);
        a[mt][1] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + 2 * t]);
        a[mt][2] = *reinterpret_cast<const uint32_t *>(&As[r][ks + 8 + 2 * t]);
        a[mt][3] = *reinterpret_cast<const uint32_t *>(&As[r + 8][ks + 8 + 2 * t]);
      }
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        const int cidx = wn + nt * 8 + g;
        b[nt][0] = *reinterpret_cast<const uint32_t *>(&Bs[cidx][ks + 2 * t]);
        b[nt][1] = *reinterpret_cast<const uint32_t *>(&Bs[cidx][ks + 8 + 2 * t]);
      }
#pragma unroll
      for (int mt = 0; mt < 2; ++mt)
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) mma_bf16(acc[mt][nt], a[mt][0], a[mt][1], a[mt][2], a[mt][3], b[nt][0], b[nt][1]);
    }
    __syncthreads();
  }
#pragma unroll
  for (int mt = 0; mt < 2; ++mt)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int m = m0 + wm + mt * 16 + g + 8 * h;
        const int n = n0 + wn + nt * 8 + 2 * t;
        if (m >= M) continue;
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          if (n + q >= N) continue;
          const float v = acc[mt][nt][2 * h + q];
          if (EPI == 0)
            outf[(int64_t)blockIdx.z * M * ldo + (int64_t)m * ldo + n + q] = v;
          else
            outb[(int64_t)m * ldo + n + q] = __float2bfloat16_rn(v * silu_grad(Z[(int64_t)m * ldz + n + q]));
        }
      }
}

// out[i] = sum_z part[z][i] over nz partial products of size cnt
__global__ void reduce_parts_kernel(const float *__restrict__ part, int nz, int64_t cnt, float *__restrict__ out) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  float s = 0.f;
  for (int z = 0; z < nz; ++z) s += part[z * cnt + i];
  out[i] = s;
}

// column sums of an [n][cols] matrix (FP32 accumulation)
template <typename T>
__global__ void colsum_kernel(const T *__restrict__ a, int64_t n, int cols, float *__restrict__ out) {
  const int cidx = blockIdx.x;
  float s = 0.f;
  for (int64_t r = threadIdx.x; r < n; r += blockDim.x) s += (float)a[r * cols + cidx];
#pragma unroll
  for (int o = 16; o >= 1; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
  __shared__ float ws[32];
  if ((threadIdx.x & 31) == 0) ws[threadIdx.x >> 5] = s;
  __syncthreads();
  if (threadIdx.x == 0) {
    float tot = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) tot += ws[i];
    out[cidx] = tot;
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

constexpr int kMaxSplit = 64;

size_t mlp_backward_ws(int64_t n) {
  const size_t dz = (size_t)2 * n * kHid * sizeof(__nv_bfloat16);
  const size_t parts = (size_t)kMaxSplit * kHid * kHid * sizeof(float);
  return ((dz + 255) / 256) * 256 + parts;
}

static void gemm(int epi, int M, int N, int K, const __nv_bfloat16 *A, int64_t sam, int64_t sak,
                 const __nv_bfloat16 *B, int64_t sbk, int64_t sbn, float *outf, __nv_bfloat16 *outb, int64_t ldo,
                 const float *Z, int64_t ldz, int nsplit, cudaStream_t st) {
  int k_chunk = (K + nsplit - 1) / nsplit;
  k_chunk = ((k_chunk + kGK - 1) / kGK) * kGK;
  nsplit = (K + k_chunk - 1) / k_chunk;
  if (nsplit < 1) nsplit = 1;
  dim3 grid((N + kGT - 1) / kGT, (M + kGT - 1) / kGT, nsplit);
  if (epi == 0)
    gemm_kernel<0><<<grid, 128, 0, st>>>(M, N, K, k_chunk, A, sam, sak, B, sbk, sbn, outf, outb, ldo, Z, ldz);
  else
    gemm_kernel<1><<<grid, 128, 0, st>>>(M, N, K, k_chunk, A, sam, sak, B, sbk, sbn, outf, outb, ldo, Z, ldz);
}

// dW = dZ^T H (K = n split over the batch), reduced into grads
static void weight_grad(const __nv_bfloat16 *dZ, int dcols, const __nv_bfloat16 *H, int hcols, int64_t n,
                        float *parts, float *gW, cudaStream_t st) {
  int nsplit = (int)((n + 255) / 256);
  if (nsplit > kMaxSplit) nsplit = kMaxSplit;
  if (nsplit < 1) nsplit = 1;
  int k_chunk = (int)((n + nsplit - 1) / nsplit);
  k_chunk = ((k_chunk + kGK - 1) / kGK) * kGK;
  nsplit = (int)((n + k_chunk - 1) / k_chunk);
  gemm(0, dcols, hcols, (int)n, dZ, 1, dcols, H, hcols, 1, parts, nullptr, hcols, nullptr, 0, nsplit, st);
  const int64_t cnt = (int64_t)dcols * hcols;
  reduce_parts_kernel<<<(unsigned)((cnt + 255) / 256), 256, 0, st>>>(parts, nsplit, cnt, gW);
}

void launch_mlp_backward(const fp_mlp &net, const void *x, const void *h_save, const float *z_save,
                         const void *dout_bf, const float *dout, int64_t n, float *grads, void *ws, cudaStream_t st) {
  const __nv_bfloat16 *X = reinterpret_cast<const __nv_bfloat16 *>(x);
  const __nv_bfloat16 *Hs = reinterpret_cast<const __nv_bfloat16 *>(h_save);
  const __nv_bfloat16 *dO = reinterpret_cast<const __nv_bfloat16 *>(dout_bf);
  __nv_bfloat16 *dz0 = reinterpret_cast<__nv_bfloat16 *>(ws);
  __nv_bfloat16 *dz1 = dz0 + (size_t)n * kHid;
  const size_t dz_bytes = (((size_t)2 * n * kHid * sizeof(__nv_bfloat16)) + 255) / 256 * 256;
  float *parts = reinterpret_cast<float *>(reinterpret_cast<char *>(ws) + dz_bytes);
  auto Hp = [&](int l) { return Hs + (size_t)(l - 1) * n * kHid; };     // H_l, l = 1..4
  auto Zp = [&](int l) { return z_save + (size_t)(l - 1) * n * kHid; };  // Z_l, l = 1..4
  auto Wb = [&](int l) { return reinterpret_cast<const __nv_bfloat16 *>(net.W[l - 1]); };
  // layer 5
  weight_grad(dO, kOut, Hp(4), kHid, n, parts, grads + mlp_param_offset(0, 4), st);
  colsum_kernel<float><<<kOut, 256, 0, st>>>(dout, n, kOut, grads + mlp_param_offset(1, 4));
  gemm(1, (int)n, kHid, kOut, dO, kOut, 1, Wb(5), kHid, 1, nullptr, dz0, kHid, Zp(4), kHid, 1, st);
  // layers 4..2: dz holds dZ_l
  __nv_bfloat16 *cur = dz0, *nxt = dz1;
  for (int l = 4; l >= 2; --l) {
    weight_grad(cur, kHid, Hp(l - 1), kHid, n, parts, grads + mlp_param_offset(0, l - 1), st);
    colsum_kernel<__nv_bfloat16><<<kHid, 256, 0, st>>>(cur, n, kHid, grads + mlp_param_offset(1, l - 1));
    gemm(1, (int)n, kHid, kHid, cur, kHid, 1, Wb(l), kHid, 1, nullptr, nxt, kHid, Zp(l - 1), kHid, 1, st);
    __nv_bfloat16 *tmp = cur;
    cur = nxt;
    nxt = tmp;
  }
  // layer 1
  weight_grad(cur, kHid, X, kIn, n, parts, grads + mlp_param_offset(0, 0), st);
  colsum_kernel<__nv_bfloat16><<<kHid, 256, 0, st>>>(cur, n, kHid, grads + mlp_param_offset(1, 0));
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
  loss_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(out, t_true, aux, y_mu, y_sigma, n, prm, dout,
                                                            reinterpret_cast<__nv_bfloat16 *>(dout_bf), loss_sum);
}

void launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, void *shadow, cudaStream_t st) {
  adam_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(p, g, m, v, n, lr, b1, b2, eps, bc1, bc2,
                                                            reinterpret_cast<__nv_bfloat16 *>(shadow));
}

}  // namespace fpc
