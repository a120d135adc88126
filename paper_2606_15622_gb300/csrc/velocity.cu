// velocity.cu -- the particle velocity update of the cubic-FP model
// (paper Sec. 3.9-3.10: Eq. update_vel with N from Eq. update_N and the
// energy factor alpha of Eq. update_alpha) for sm_103a.
//
// A group of G lanes per cell, static round-robin over cells:
//   pass 1  <N.N> and <M'.N> over the cell (for alpha);
//   pass 2  M^{n+1} = (M' a + (1-a) tau N + sqrt(theta (1-a^2)) xi) / alpha + U,
//           written in place.
// FP32 velocities are updated in FP32 arithmetic, FP64 velocities in FP64.
// The per-cell constants are read as FP64 and converted once per cell, one
// constant per lane, then spread over the group by shuffles, so the FP64 pipe
// sees ~1 instruction per cell on the FP32 path.
// Noise: the caller's variates, or Philox4x32-10 keyed by the seed on the
// counter (particle index, step), mapped to normals by Box-Muller in FP32.
#include <cstdint>

#include "fp_device.cuh"

namespace fpc {

constexpr int kVG = 8;  // lanes per cell

// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11).
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint32_t k0, uint32_t k1) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r > 0) {
      k0 += 0x9E3779B9u;
      k1 += 0xBB67AE85u;
    }
    const uint32_t hi0 = __umulhi(0xD2511F53u, x.x), lo0 = 0xD2511F53u * x.x;
    const uint32_t hi1 = __umulhi(0xCD9E8D57u, x.z), lo1 = 0xCD9E8D57u * x.z;
    x = make_uint4(hi1 ^ x.y ^ k0, lo1, hi0 ^ x.w ^ k1, lo0);
  }
  return x;
}

// Three standard normals for particle p at `step`: uniforms
// u = (floor(w / 2^8) + 1) 2^-24 (exact in FP32) from the four Philox words, Box-Muller on
// (u0, u1) and (u2, u3) in FP32.
__device__ __forceinline__ void philox_normals(uint64_t seed, uint64_t step, uint64_t p, float &x0, float &x1,
                                               float &x2) {
  const uint4 w = philox4x32_10(make_uint4((uint32_t)p, (uint32_t)(p >> 32), (uint32_t)step, (uint32_t)(step >> 32)),
                                (uint32_t)seed, (uint32_t)(seed >> 32));
  const float s24 = 5.9604644775390625e-08f;  // 2^-24
  const float u0 = ((float)(w.x >> 8) + 1.f) * s24, u1 = ((float)(w.y >> 8) + 1.f) * s24;
  const float u2 = ((float)(w.z >> 8) + 1.f) * s24, u3 = ((float)(w.w >> 8) + 1.f) * s24;
  const float r0 = sqrtf(-2.f * logf(u0)), r1 = sqrtf(-2.f * logf(u2));
  float s, c;
  sincospif(2.f * u1, &s, &c);
  x0 = r0 * c;
  x1 = r0 * s;
  x2 = r1 * cospif(2.f * u3);
}

template <typename T>
__device__ __forceinline__ T shfl_group(T x, int src_lane_in_group, int lane) {
  return __shfl_sync(0xffffffffu, x, (lane & ~(kVG - 1)) + src_lane_in_group);
}

struct VelParams {
  double dt, eps2_hat;
  uint64_t seed, step;
};

// Per-cell constants, slot order: U0..2, theta, u3[10] (for b), Y[9], tau = 24 slots
constexpr int kVConsts = 24;

template <typename VT>
__global__ void __launch_bounds__(256) velocity_kernel(VT *__restrict__ v, int64_t np, const int64_t *__restrict__ off,
                                                       int64_t n_cells, const double *__restrict__ mom,
                                                       const double *__restrict__ coeffs, const double *__restrict__ tau,
                                                       VelParams prm, const VT *__restrict__ xi,
                                                       double *__restrict__ alpha_out, int32_t *__restrict__ flags) {
  using T = VT;  // arithmetic type follows the storage type
  constexpr int G = kVG;
  constexpr int GPW = 32 / G;
  const int lane = threadIdx.x & 31;
  const int lg = lane & (G - 1);
  const int g = lane / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  VT *vx = v, *vy = v + np, *vz = v + 2 * np;

  for (int64_t base = warp * GPW; base < n_cells; base += nwarps * GPW) {
    const int64_t c = base + g;
    const bool valid = c < n_cells;
    int64_t a0 = 0, e = 0;
    int fl = 0;
    if (valid) {
      a0 = off[c];
      e = off[c + 1];
      fl = flags[c];
    }
    const int n = (int)(e - a0);
    // constants: lane lg fetches slots lg, lg + G, lg + 2G (converted once)
    T cv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int slot = lg + k * G;
      double x = 0.0;
      if (valid && slot < kVConsts) {
        if (slot < 4)
          x = mom[c * FP_NMOM + kU + slot];  // U0..2, theta (slots 1..4)
        else if (slot < 14)
          x = mom[c * FP_NMOM + kU3 + (slot - 4)];
        else if (slot < 23)
          x = coeffs[c * 9 + (slot - 14)];
        else
          x = tau[c];
      }
      cv[k] = (T)x;
    }
    auto cst = [&](int slot) -> T { return shfl_group(cv[slot / G], slot % G, lane); };
    const T U0 = cst(0), U1 = cst(1), U2 = cst(2), th = cst(3);
    // b_i = u_ikk from the third moments 111,112,113,122,123,133,222,223,233,333
    const T b0 = cst(4 + 0) + cst(4 + 3) + cst(4 + 5);
    const T b1 = cst(4 + 1) + cst(4 + 6) + cst(4 + 8);
    const T b2 = cst(4 + 2) + cst(4 + 7) + cst(4 + 9);
    const T tc = cst(23);
    const T itau = T(1) / tc;
    const T C00 = cst(14) + itau, C01 = cst(15), C02 = cst(16), C11 = cst(17) + itau, C12 = cst(18),
            C22 = cst(19) + itau;
    const T G0 = cst(20), G1 = cst(21), G2 = cst(22);
    const T eps2 = T(prm.eps2_hat) / (tc * th);
    const T x = T(prm.dt) * itau;
    T one_m_a, a;
    if (sizeof(T) == 4) {
      one_m_a = -expm1f((float)-x);
      a = expf((float)-x);
    } else {
      one_m_a = -expm1(-(double)x);
      a = exp(-(double)x);
    }
    const bool linear = (fl & (FP_FLAG_FEW | FP_FLAG_SINGULAR | FP_FLAG_NONFINITE)) != 0;
    auto drift = [&](T m0, T m1, T m2, T &n0, T &n1, T &n2) {
      const T m2s = m0 * m0 + m1 * m1 + m2 * m2;
      const T q = m2s - T(3) * th;
      n0 = C00 * m0 + C01 * m1 + C02 * m2 + G0 * q - eps2 * (m0 * m2s - b0);
      n1 = C01 * m0 + C11 * m1 + C12 * m2 + G1 * q - eps2 * (m1 * m2s - b1);
      n2 = C02 * m0 + C12 * m1 + C22 * m2 + G2 * q - eps2 * (m2 * m2s - b2);
    };
    const int itmax = __reduce_max_sync(0xffffffffu, (n + G - 1) / G);
    // pass 1: <N.N>, <M'.N>
    T snn = 0, smn = 0;
    const bool any_nonlinear = __any_sync(0xffffffffu, valid && !linear && n > 0);
    if (any_nonlinear) {
      for (int it = 0; it < itmax; ++it) {
        const int64_t p = a0 + (int64_t)it * G + lg;
        if (p < e && !linear) {
          const T m0 = vx[p] - U0, m1 = vy[p] - U1, m2 = vz[p] - U2;
          T n0, n1, n2;
          drift(m0, m1, m2, n0, n1, n2);
          snn += n0 * n0 + n1 * n1 + n2 * n2;
          smn += m0 * n0 + m1 * n1 + m2 * n2;
        }
      }
      snn = group_allreduce<G>(snn);
      smn = group_allreduce<G>(smn);
    }
    T alpha = 1;
    if (valid && !linear && n > 0) {
      const T inv_n = T(1) / T(n);
      const T alpha2 = T(1) + tc / (T(3) * th) * (tc * one_m_a * one_m_a * (snn * inv_n) + T(2) * (a * one_m_a) * (smn * inv_n));
      if (alpha2 > T(0) && alpha2 < T(INFINITY))
        alpha = sqrt(alpha2);
      else
        fl |= FP_FLAG_ALPHA;
    }
    const T ia = T(1) / alpha;
    const T drift_f = one_m_a * tc;
    const T noise = sqrt(th * one_m_a * (T(1) + a));
    // pass 2: the update
    for (int it = 0; it < itmax; ++it) {
      const int64_t p = a0 + (int64_t)it * G + lg;
      if (p < e) {
        const T m0 = vx[p] - U0, m1 = vy[p] - U1, m2 = vz[p] - U2;
        T n0 = 0, n1 = 0, n2 = 0;
        if (!linear) drift(m0, m1, m2, n0, n1, n2);
        T x0, x1, x2;
        if (xi) {
          x0 = xi[p];
          x1 = xi[np + p];
          x2 = xi[2 * np + p];
        } else {
          float f0, f1, f2;
          philox_normals(prm.seed, prm.step, (uint64_t)p, f0, f1, f2);
          x0 = f0;
          x1 = f1;
          x2 = f2;
        }
        vx[p] = (m0 * a + drift_f * n0 + noise * x0) * ia + U0;
        vy[p] = (m1 * a + drift_f * n1 + noise * x1) * ia + U1;
        vz[p] = (m2 * a + drift_f * n2 + noise * x2) * ia + U2;
      }
    }
    if (valid && lg == 0) {
      flags[c] = fl;
      if (alpha_out) alpha_out[c] = (double)alpha;
    }
  }
}

static int vel_sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

void launch_velocity(void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, const double *mom,
                     const double *coeffs, const double *tau, double dt, double eps2_hat, const void *xi, uint64_t seed,
                     uint64_t step, double *alpha_out, int32_t *flags, cudaStream_t st) {
  VelParams prm{dt, eps2_hat, seed, step};
  const int threads = 256;
  const int64_t groups_per_block = (threads / 32) * (32 / kVG);
  int64_t blocks = (n_cells + groups_per_block - 1) / groups_per_block;
  const int64_t cap = (int64_t)vel_sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (v_dtype == FP_V_F32)
    velocity_kernel<float><<<(unsigned)blocks, threads, 0, st>>>((float *)v, np, off, n_cells, mom, coeffs, tau, prm,
                                                                 (const float *)xi, alpha_out, flags);
  else
    velocity_kernel<double><<<(unsigned)blocks, threads, 0, st>>>((double *)v, np, off, n_cells, mom, coeffs, tau,
                                                                  prm, (const double *)xi, alpha_out, flags);
}

}  // namespace fpc
