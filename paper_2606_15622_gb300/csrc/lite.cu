// lite.cu -- the paper's LITE path (Sec. 4, Phase 3 item 2): a moment pass
// that stops at the heat-flux vector, the 16 network inputs of Phase 1-2
// computed from it, and the learned closure on those inputs.
//
// LITE moment vector (FP_NLITE = 14 per cell): N, U (3), theta, u_ij (6, sym
// order 11,12,13,22,23,33), b_i = <c_i |c|^2> (3).  Its one-pass tiled gather
// accumulates 12 sums a particle (the full moment vector needs 29).
//
// Network inputs (16, then zero padding to 32): rho, T, U (3), Pi (6), q (3),
// DM2, nu, read as  rho = N (the cell's particle count: proportional to the
// density at fixed cell volume and particle weight), T = theta,
// Pi_ij = u_ij - theta delta_ij, q_i = b_i / 2 (per unit mass), DM2 = det u
// (the determinant of the second-moment tensor, positive for a
// non-degenerate cell), nu = 1 / tau.  They are standardised with the
// network's scalers and checked against its training box (FP_FLAG_RANGE).
// With only low-order moments there is no exact fallback: cells with too few
// particles, theta <= 0, non-finite inputs or a non-finite prediction take
// the linear drift C = -I/tau, G = 0.
#include <cstdint>
#include <cuda_bf16.h>

#include "fp_device.cuh"
#include "mlp_common.cuh"

namespace fpc {

constexpr int kNLiteSum = 9;  // u_ij (6, order 2), c_i |c|^2 (3, order 3)

__device__ __forceinline__ int lite_order(int q) { return q < 6 ? 2 : 3; }

template <typename VT, int G>
__global__ void __launch_bounds__(256) gather_lite_kernel(const VT *__restrict__ v, int64_t np,
                                                          const int64_t *__restrict__ off, int64_t n_cells,
                                                          double *__restrict__ lite) {
  constexpr int GPW = 32 / G;
  constexpr int K = 32 / G;
  constexpr int BLK = 16;  // particles per lane summed plainly before a two-sum fold
  const int lane = threadIdx.x & 31;
  const int lg = lane & (G - 1);
  const int g = lane / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const VT *vx = v, *vy = v + np, *vz = v + 2 * np;

  for (int64_t base = warp * GPW; base < n_cells; base += nwarps * GPW) {
    const int64_t c = base + g;
    const bool valid = c < n_cells;
    int64_t a = 0, e = 0;
    if (valid) {
      a = off[c];
      e = off[c + 1];
    }
    const int n = (int)(e - a);
    float v0x = 0.f, v0y = 0.f, v0z = 0.f;
    if (n > 0) {
      v0x = (float)vx[a];
      v0y = (float)vy[a];
      v0z = (float)vz[a];
    }
    const int itmax = __reduce_max_sync(0xffffffffu, (n + G - 1) / G);
    // pass A: mean offset and spread about the first particle
    float sx = 0.f, sy = 0.f, sz = 0.f, sq = 0.f;
    for (int it = 0; it < itmax; ++it) {
      const int64_t p = a + (int64_t)it * G + lg;
      if (p < e) {
        const float dx = (float)ldg_v(vx + p) - v0x, dy = (float)ldg_v(vy + p) - v0y, dz = (float)ldg_v(vz + p) - v0z;
        sx += dx;
        sy += dy;
        sz += dz;
        sq = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, sq)));
      }
    }
    sx = group_allreduce<G>(sx);
    sy = group_allreduce<G>(sy);
    sz = group_allreduce<G>(sz);
    sq = group_allreduce<G>(sq);
    const float inv_n = n > 0 ? 1.f / (float)n : 0.f;
    const float mx = sx * inv_n, my = sy * inv_n, mz = sz * inv_n;
    const float th_est = (sq * inv_n - (mx * mx + my * my + mz * mz)) * (1.f / 3.f);
    int ks = 0;  // power-of-two scale ~ 1/sqrt(theta): exact
    if (th_est > 0.f) {
      int ex;
      frexpf(th_est, &ex);
      ks = max(-20, min(20, -(ex / 2)));
    }
    const float s = ldexpf(1.f, ks);
    // pass B: the 9 centred, scaled sums; FP32 blocks folded by two-sum
    float hi[32], lo[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      hi[q] = 0.f;
      lo[q] = 0.f;
    }
    for (int it0 = 0; it0 < itmax; it0 += BLK) {
      float t[kNLiteSum];
#pragma unroll
      for (int q = 0; q < kNLiteSum; ++q) t[q] = 0.f;
      const int itend = min(it0 + BLK, itmax);
      for (int it = it0; it < itend; ++it) {
        const int64_t p = a + (int64_t)it * G + lg;
        if (p < e) {
          const float wx = (((float)ldg_v(vx + p) - v0x) - mx) * s;
          const float wy = (((float)ldg_v(vy + p) - v0y) - my) * s;
          const float wz = (((float)ldg_v(vz + p) - v0z) - mz) * s;
          const float xx = wx * wx, yy = wy * wy, zz = wz * wz;
          t[0] += xx;
          t[1] = fmaf(wx, wy, t[1]);
          t[2] = fmaf(wx, wz, t[2]);
          t[3] += yy;
          t[4] = fmaf(wy, wz, t[4]);
          t[5] += zz;
          const float r2 = xx + yy + zz;
          t[6] = fmaf(r2, wx, t[6]);
          t[7] = fmaf(r2, wy, t[7]);
          t[8] = fmaf(r2, wz, t[8]);
        }
      }
      if (it0 == 0) {
#pragma unroll
        for (int q = 0; q < kNLiteSum; ++q) hi[q] = t[q];
      } else {
#pragma unroll
        for (int q = 0; q < kNLiteSum; ++q) {
          float sum, err;
          two_sum(hi[q], t[q], sum, err);
          hi[q] = sum;
          lo[q] += err;
        }
      }
    }
    group_reduce_scatter2<G>(hi, lo, lane);
    // promote: means with the power-of-two scaling undone
    const double inv_nd = n > 0 ? 1.0 / (double)n : 0.0;
    double val[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int q = lg * K + j;
      const int ord = q < kNLiteSum ? lite_order(q) : 0;
      val[j] = ((double)hi[j] + (double)lo[j]) * ldexp(inv_nd, -ks * ord);
    }
    const int gbase = lane & ~(G - 1);
    const double u11 = __shfl_sync(0xffffffffu, val[0 % K], gbase + 0 / K);
    const double u22 = __shfl_sync(0xffffffffu, val[3 % K], gbase + 3 / K);
    const double u33 = __shfl_sync(0xffffffffu, val[5 % K], gbase + 5 / K);
    if (!valid) continue;
    double *o = lite + c * FP_NLITE;
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int q = lg * K + j;
      if (q < 6) o[5 + q] = val[j];
      else if (q < kNLiteSum) o[11 + (q - 6)] = val[j];
    }
    if (lg == 0) {
      o[0] = (double)n;
      o[1] = (double)v0x + (double)mx;
      o[2] = (double)v0y + (double)my;
      o[3] = (double)v0z + (double)mz;
      o[4] = (u11 + u22 + u33) * (1.0 / 3.0);
    }
  }
}


__global__ void __launch_bounds__(256) lite_features_kernel(MlpDev net, const double *__restrict__ lite,
                                                            const double *__restrict__ tau, int64_t n,
                                                            int min_particles, float margin,
                                                            __nv_bfloat16 *__restrict__ x,
                                                            int32_t *__restrict__ flags) {
  const int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= n) return;
  const double *m = lite + c * FP_NLITE;
  int fl = 0;
  bool fin = finite_d(tau[c]) && positive_d(tau[c]);
#pragma unroll
  for (int k = 0; k < FP_NLITE; ++k) fin = fin && finite_d(m[k]);
  if (!fin) fl |= FP_FLAG_NONFINITE;
  if (narrow(m[0]) < (float)min_particles) fl |= FP_FLAG_FEW;  // N is a whole number
  if (!positive_d(m[4])) fl |= FP_FLAG_SINGULAR;
  float f[16];
  lite_raw_features(m, tau[c], f);
  uint32_t packed[kIn / 2];
#pragma unroll
  for (int k = 0; k < kIn; k += 2) {
    float xs[2] = {0.f, 0.f};
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int q = k + h;
      if (q < 16) {
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

static int lite_sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

bool launch_gather_tile_lite(const float *v, int64_t np, const int64_t *off, int64_t n_cells, double *lite,
                             cudaStream_t st, int sm_count);

// FP32 velocities (16-byte aligned) take the shared-memory streamed gather;
// FP64 velocities the direct one below.
void launch_gather_lite(const void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, double *lite,
                        cudaStream_t st) {
  if (v_dtype == FP_V_F32 && launch_gather_tile_lite((const float *)v, np, off, n_cells, lite, st, lite_sm_count()))
    return;
  constexpr int G = 8;
  const int threads = 256;
  const int64_t cells_per_block = (threads / 32) * (32 / G);
  int64_t blocks = (n_cells + cells_per_block - 1) / cells_per_block;
  const int64_t cap = (int64_t)lite_sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (v_dtype == FP_V_F32)
    gather_lite_kernel<float, G><<<(unsigned)blocks, threads, 0, st>>>((const float *)v, np, off, n_cells, lite);
  else
    gather_lite_kernel<double, G><<<(unsigned)blocks, threads, 0, st>>>((const double *)v, np, off, n_cells, lite);
}

MlpDev make_mlp_dev(const fp_mlp &m);

void launch_lite_features(const fp_mlp &net, const double *lite, const double *tau, int64_t n, int min_particles,
                          double margin, void *x, int32_t *flags, cudaStream_t st) {
  const int64_t blocks = (n + 255) / 256;
  lite_features_kernel<<<(unsigned)blocks, 256, 0, st>>>(make_mlp_dev(net), lite, tau, n, min_particles,
                                                         (float)margin, reinterpret_cast<__nv_bfloat16 *>(x), flags);
}

}  // namespace fpc
