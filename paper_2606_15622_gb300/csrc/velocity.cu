// velocity.cu -- the particle velocity update of the cubic-FP model
// (paper Sec. 3.9-3.10: Eq. update_vel with N from Eq. update_N and the
// energy factor alpha of Eq. update_alpha) for sm_103a.
//
//   M^{n+1} = (M' a + (1-a) tau N + sqrt(theta (1-a^2)) xi) / alpha + U,
// written in place or to a separate output array.  FP32 velocities are
// updated in FP32 arithmetic, FP64 velocities in FP64.  The per-cell
// constants (U, theta, b, C + I/tau, G, eps^2, a, (1-a) tau, the noise
// amplitude, 1/alpha) live in a shared-memory table read as float4.
//
// One pass (with <|c|^6>: velocity_chunk_kernel): alpha comes from the
// moments in closed form.  Every warp of a persistent grid takes an equal
// slice of the particles and walks its cells 32 at a time: each lane builds
// one cell's constants and alpha, then the warp streams the chunk's
// particles.  Two passes (velocity_kernel: no <|c|^6>, or LITE vectors): a
// warp takes whole cells, four at a time (an 8-lane group per cell builds
// its constants), sums <N.N> and <M'.N> over the particles, then updates.
// Both stream particles in quads of four consecutive ones per lane, with
// vector loads and stores where the arrays' alignment allows.
// Noise: the caller's variates, or one Philox4x32-10 word stream per step
// (keyed by the seed; particle g takes words 3g .. 3g + 2) mapped to normals
// by the inverse normal distribution function in FP32 (normal_quantile).
#include <climits>
#include <cstdint>

#include "fp_device.cuh"
#include "quads.cuh"

namespace fpc {

constexpr int kVG = 8;              // lanes per cell while building constants
constexpr int kVCells = 32 / kVG;   // consecutive cells per warp task
constexpr int kVWarps = 8;          // warps per block
constexpr int kVConst = 24;         // table entries per cell
constexpr int kVBatch = 4;          // particles per lane per round

// table slots
enum { VU0 = 0, VU1, VU2, VTH, VB0, VB1, VB2, VC00, VC01, VC02, VC11, VC12, VC22, VG0, VG1, VG2, VEPS, VA, VDRIFT,
       VNOISE, VIA, VLIN, VOMA, VTAU };

// Standard normal quantile of a Philox word w: u = (k + 1/2) 2^-23 with
// k = w >> 9, x = 2u - 1 = (2k + 1 - 2^23) 2^-23 (exact in FP32) and
// lg = log2(1 - x^2); z = Phi^-1(u) = sqrt(2) erfinv(x) = x P(lg + 4) for
// lg >= -8 and x Q(sqrt(-lg) - 3.75) below (0.2 % of the words), the form of
// Giles' erfinv approximation (GPU Computing Gems, 2011).  P and Q were fitted
// to scipy's ndtri for this kernel by normal_quantile_fit.py, which also
// evaluates this FP32 arithmetic for all 2^23 words: |dz| <= 1.3e-6 and
// |dz| / |z| <= 3.3e-7 with lg2.approx anywhere within its error bound.

// P (degree 9, in lg + 4) and Q (degree 8, in sqrt(-lg) - 3.75), leading
// coefficient first, evaluated by Horner's rule
__device__ constexpr float kQuantileP[10] = {3.862574705e-10f, 4.549878529e-10f, -5.210529963e-08f, -4.056917646e-07f,
                                             2.225996695e-06f, 6.797097012e-05f, 4.802460899e-04f, -3.469289979e-03f,
                                             -2.392821312e-01f, 2.217919827e+00f};
__device__ constexpr float kQuantileQ[9] = {-6.398928963e-05f, -6.059690350e-05f, 6.303846603e-04f,
                                            -1.477855956e-03f, 2.589873038e-03f, -4.353985656e-03f,
                                            6.956293248e-03f, 1.181739330e+00f, 4.179551601e+00f};

__device__ __forceinline__ float quantile_q(float v) {
  float p = kQuantileQ[0];
#pragma unroll
  for (int i = 1; i < 9; ++i) p = fmaf(p, v, kQuantileQ[i]);
  return p;
}

// x = (2k + 1 - 2^23) 2^-23 for k = w >> 9, from f = 1 + k 2^-23 (the bits
// of k under the exponent of 1): x = 2 (f - 1.5) + 2^-23, every step exact
__device__ __forceinline__ float quantile_x(uint32_t w) {
  return fmaf(2.0f, __uint_as_float((w >> 9) | 0x3f800000u) - 1.5f, 1.1920928955078125e-07f);
}

__device__ __forceinline__ float normal_quantile(uint32_t w) {
  const float x = quantile_x(w);
  const float t = fmaf(-x, x, 1.0f);  // 1 - x^2 in [2^-22, 1]
  float lg;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lg) : "f"(t));
  float p;
  if (__builtin_expect(t < 0.00390625f, 0)) {  // 2^-8: the tails, one word in 500
    p = quantile_q(sqrtf(-lg) - 3.75f);
  } else {
    const float v = lg + 4.0f;
    p = kQuantileP[0];
#pragma unroll
    for (int i = 1; i < 10; ++i) p = fmaf(p, v, kQuantileP[i]);
  }
  return x * p;
}

// Two normals at once: the same arithmetic as normal_quantile on a pair of
// words, with the polynomial's multiply-adds packed two to an instruction
// (each lane of fma.rn.f32x2 rounds as fmaf does, so the results are
// identical).
__device__ __forceinline__ float2 normal_quantile2(uint32_t wa, uint32_t wb) {
  const float2 x = __ffma2_rn(make_float2(2.0f, 2.0f),
                              __fadd2_rn(make_float2(__uint_as_float((wa >> 9) | 0x3f800000u),
                                                     __uint_as_float((wb >> 9) | 0x3f800000u)),
                                         make_float2(-1.5f, -1.5f)),
                              make_float2(1.1920928955078125e-07f, 1.1920928955078125e-07f));
  const float2 t = __ffma2_rn(make_float2(-x.x, -x.y), x, make_float2(1.0f, 1.0f));
  float la, lb;
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(la) : "f"(t.x));
  asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(lb) : "f"(t.y));
  const float2 v = __fadd2_rn(make_float2(la, lb), make_float2(4.0f, 4.0f));
  float2 p = make_float2(kQuantileP[0], kQuantileP[0]);
#pragma unroll
  for (int i = 1; i < 10; ++i) p = __ffma2_rn(p, v, make_float2(kQuantileP[i], kQuantileP[i]));
  if (__builtin_expect(t.x < 0.00390625f, 0)) p.x = quantile_q(sqrtf(-la) - 3.75f);
  if (__builtin_expect(t.y < 0.00390625f, 0)) p.y = quantile_q(sqrtf(-lb) - 3.75f);
  return __fmul2_rn(x, p);
}

// The noise of a step is one stream of Philox words: word j is word j % 4
// of the block on counter (j / 4, step); particle g (global index) takes
// words 3g .. 3g + 2, so the quad of particles 4Q .. 4Q + 3 takes exactly the
// blocks 3Q .. 3Q + 2.  Its twelve normals, particle u's component k at 3u + k.
__device__ __forceinline__ void quad_normals(const PhiloxKeys &key, uint64_t step, uint64_t Q, float (&z)[12]) {
  uint32_t w[12];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const uint64_t blk = 3 * Q + (uint64_t)k;
    const uint4 r = philox4x32_10(
        make_uint4((uint32_t)blk, (uint32_t)(blk >> 32), (uint32_t)step, (uint32_t)(step >> 32)), key);
    w[4 * k] = r.x;
    w[4 * k + 1] = r.y;
    w[4 * k + 2] = r.z;
    w[4 * k + 3] = r.w;
  }
#pragma unroll
  for (int k = 0; k < 6; ++k) {
    const float2 q = normal_quantile2(w[2 * k], w[2 * k + 1]);
    z[2 * k] = q.x;
    z[2 * k + 1] = q.y;
  }
}

struct VelParams {
  double dt, eps2_hat;
  uint64_t step;
  uint64_t particle_offset;  // global index of particle i (its Philox words): particle_offset + i
  PhiloxKeys key;
  // vector loads and stores of whole quads, per component (bits 2d, 2d + 1):
  // 2 = four values at once, 1 = two pairs, 0 = one at a time (the alignment
  // of element 4Q - particle_offset of component d)
  int vec;
};

template <typename T>
__device__ __forceinline__ void drift(const T *K, T m0, T m1, T m2, T &n0, T &n1, T &n2) {
  const T m2s = m0 * m0 + m1 * m1 + m2 * m2;
  const T q = m2s - T(3) * K[VTH];
  const T e = K[VEPS];
  n0 = K[VC00] * m0 + K[VC01] * m1 + K[VC02] * m2 + K[VG0] * q - e * (m0 * m2s - K[VB0]);
  n1 = K[VC01] * m0 + K[VC11] * m1 + K[VC12] * m2 + K[VG1] * q - e * (m1 * m2s - K[VB1]);
  n2 = K[VC02] * m0 + K[VC12] * m1 + K[VC22] * m2 + K[VG2] * q - e * (m2 * m2s - K[VB2]);
}

// v and vout may be the same array (in-place update): every particle is read
// before it is written, by the same lane.
// Cell averages of N.N and M'.N (Eq. update_N; M' = c = v - U, <c> = 0) in
// closed form from the central moments, with A = C + I/tau (vals[VC..]),
// Gamma, b, theta and eps^2 from the constant table:
//   <M'.N> = tr(A u) + Gamma.b - eps^2 s4
//   <N.N>  = tr(A^2 u) + |Gamma|^2 (s4 - 9 theta^2) + eps^4 (m6 - |b|^2)
//            + 2 Gamma.A b - 2 eps^2 tr(A w) - 2 eps^2 Gamma.(z - 3 theta b)
// (u_ij = <c_i c_j>, w_ij = <|c|^2 c_i c_j>, z_i = <|c|^4 c_i>, s4 = tr w,
// m6 = <|c|^6>, b_i = <|c|^2 c_i>); symmetric tensors in sym2 slot order.
template <typename T>
__device__ __forceinline__ void cell_drift_averages(const T (&vals)[kVConst], const T (&u)[6], const T (&w)[6],
                                                    const T (&z)[3], T m6, T &nn, T &mn) {
  const T A[6] = {vals[VC00], vals[VC01], vals[VC02], vals[VC11], vals[VC12], vals[VC22]};
  const T G[3] = {vals[VG0], vals[VG1], vals[VG2]};
  const T b[3] = {vals[VB0], vals[VB1], vals[VB2]};
  const T th = vals[VTH], e2 = vals[VEPS];
  auto tr = [](const T (&X)[6], const T (&Y)[6]) -> T {  // sum_ij X_ij Y_ij
    return X[0] * Y[0] + X[3] * Y[3] + X[5] * Y[5] + T(2) * (X[1] * Y[1] + X[2] * Y[2] + X[4] * Y[4]);
  };
  // A^2 (symmetric)
  const T A2[6] = {A[0] * A[0] + A[1] * A[1] + A[2] * A[2], A[0] * A[1] + A[1] * A[3] + A[2] * A[4],
                   A[0] * A[2] + A[1] * A[4] + A[2] * A[5], A[1] * A[1] + A[3] * A[3] + A[4] * A[4],
                   A[1] * A[2] + A[3] * A[4] + A[4] * A[5], A[2] * A[2] + A[4] * A[4] + A[5] * A[5]};
  const T Ab[3] = {A[0] * b[0] + A[1] * b[1] + A[2] * b[2], A[1] * b[0] + A[3] * b[1] + A[4] * b[2],
                   A[2] * b[0] + A[4] * b[1] + A[5] * b[2]};
  const T s4 = w[0] + w[3] + w[5];
  const T gb = G[0] * b[0] + G[1] * b[1] + G[2] * b[2];
  const T gg = G[0] * G[0] + G[1] * G[1] + G[2] * G[2];
  const T bb = b[0] * b[0] + b[1] * b[1] + b[2] * b[2];
  const T gAb = G[0] * Ab[0] + G[1] * Ab[1] + G[2] * Ab[2];
  const T gz = G[0] * z[0] + G[1] * z[1] + G[2] * z[2];
  mn = tr(A, u) + gb - e2 * s4;
  nn = tr(A2, u) + gg * (s4 - T(9) * th * th) + e2 * e2 * (m6 - bb) + T(2) * gAb - T(2) * e2 * tr(A, w) -
       T(2) * e2 * (gz - T(3) * th * gb);
}

// The two-pass update: without <|c|^6> (or from LITE vectors, kLite: U,
// theta and b_i stored directly, FP_NLITE per cell) the averages <N.N> and
// <M'.N> of Eq. update_alpha come from a first pass over the particles, so
// a warp takes whole cells: four at a time, the group of eight lanes of each
// building its constants.
template <typename VT, bool kLite = false>
__global__ void __launch_bounds__(32 * kVWarps, sizeof(VT) == 4 ? 3 : 2) velocity_kernel(const VT *v, VT *vout, int64_t np,
                                                                const int64_t *__restrict__ off, int64_t n_cells,
                                                                const double *__restrict__ mom,
                                                                const double *__restrict__ m6,
                                                                const double *__restrict__ coeffs,
                                                                const double *__restrict__ tau, VelParams prm,
                                                                const VT *__restrict__ xi,
                                                                double *__restrict__ alpha_out,
                                                                int32_t *__restrict__ flags) {
  using T = VT;  // arithmetic type follows the storage type
  __shared__ __align__(16) T table[kVWarps][kVCells][kVConst];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int lg = lane & (kVG - 1);
  const int g = lane / kVG;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const VT *vx = v, *vy = v + np, *vz = v + 2 * np;
  VT *wx = vout, *wy = vout + np, *wz = vout + 2 * np;
  T(*tab)[kVConst] = table[wib];

  // ---- this warp's share: the cells that start in an equal slice
  //      [tA, tB) of the particles ----
  const int64_t base0 = off[0], total = off[n_cells] - base0;
  auto slice = [&](int64_t k) {  // base0 + floor(total k / nwarps), exactly
    return base0 + (total / nwarps) * k + (total % nwarps) * k / nwarps;
  };
  const int64_t tA = slice(warp), tB = slice(warp + 1);
  const int64_t Lx = lower_bound16(off, n_cells, lane < 16 ? tA : tB, lane);
  const int64_t La = __shfl_sync(0xffffffffu, Lx, 0);
  const int64_t cb = warp + 1 == nwarps ? n_cells : __shfl_sync(0xffffffffu, Lx, 16);

  for (int64_t base = La; base < cb; base += kVCells) {
    const int64_t c = base + g;
    const bool valid = c < cb;
    const int64_t cc = valid ? c : cb;
    const int64_t a0 = off[cc];
    const int64_t e = valid ? off[c + 1] : a0;
    const int fl = valid ? flags[c] : FP_FLAG_FEW;
    const int n = (int)(e - a0);
    // ---- per-cell constants: lane lg converts slots lg, lg+8, lg+16 of
    //      [U0..2, theta, u3 (10), Y (9), tau] once; the group shares them
    T cv[3];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const int slot = lg + k * kVG;
      double x = 0.0;
      if (valid) {
        // (a LITE vector puts b_i in slot 4 + i and zeros in 7..13: the sums
        //  u_ikk below then give b_i as they do for the third moments)
        if (slot < 4)
          x = mom[c * (kLite ? FP_NLITE : FP_NMOM) + kU + slot];
        else if (slot < 14)
          x = kLite ? (slot < 7 ? mom[c * FP_NLITE + 11 + (slot - 4)] : 0.0) : mom[c * FP_NMOM + kU3 + (slot - 4)];
        else if (slot < 23)
          x = coeffs[c * 9 + (slot - 14)];
        else
          x = tau[c];
      }
      cv[k] = (T)x;
    }
    auto cst = [&](int slot) -> T {
      return __shfl_sync(0xffffffffu, cv[slot / kVG], (lane & ~(kVG - 1)) + slot % kVG);
    };
    const bool linear = (fl & (FP_FLAG_FEW | FP_FLAG_SINGULAR | FP_FLAG_NONFINITE)) != 0;
    {
      const T th = cst(3), tc = cst(23);
      const T itau = T(1) / tc;
      const T x = T(prm.dt) * itau;
      T one_m_a, a;
      if (sizeof(T) == 4) {
        one_m_a = -expm1f((float)-x);
        a = expf((float)-x);
      } else {
        one_m_a = -expm1(-(double)x);
        a = exp(-(double)x);
      }
      // b_i = u_ikk from the third moments 111,112,113,122,123,133,222,223,233,333
      const T vals[kVConst] = {cst(0), cst(1), cst(2), th,
                               cst(4 + 0) + cst(4 + 3) + cst(4 + 5), cst(4 + 1) + cst(4 + 6) + cst(4 + 8),
                               cst(4 + 2) + cst(4 + 7) + cst(4 + 9),
                               cst(14) + itau, cst(15), cst(16), cst(17) + itau, cst(18), cst(19) + itau,
                               cst(20), cst(21), cst(22),
                               T(prm.eps2_hat) / (tc * th), a, one_m_a * tc, sqrt(th * one_m_a * (T(1) + a)),
                               T(1), linear ? T(1) : T(0), one_m_a, tc};
      if (lg == 0) {
#pragma unroll
        for (int q = 0; q < kVConst; ++q) tab[g][q] = vals[q];
      }
    }
    // the warp's contiguous particle range and the inner boundaries,
    // relative to its first particle
    const int64_t o0 = __shfl_sync(0xffffffffu, a0, 0);
    const int i1 = (int)(__shfl_sync(0xffffffffu, a0, 8) - o0);
    const int i2 = (int)(__shfl_sync(0xffffffffu, a0, 16) - o0);
    const int i3 = (int)(__shfl_sync(0xffffffffu, a0, 24) - o0);
    const int i4 = (int)(__shfl_sync(0xffffffffu, e, 24) - o0);
    const VT *px = vx + o0, *py = vy + o0, *pz = vz + o0;
    VT *ox = wx + o0, *oy = wy + o0, *oz = wz + o0;
    __syncwarp();
    // ---- pass 1: <N.N>, <M'.N> per cell ----
    const unsigned nonlin = __ballot_sync(0xffffffffu, !linear && n > 0 && lg == 0);
    T s_nn[kVCells] = {}, s_mn[kVCells] = {};
    if (nonlin) {
      // kVBatch particles per lane per round, all loads issued first
      for (int q0 = lane; q0 < i4; q0 += 32 * kVBatch) {
        T mx[kVBatch], my[kVBatch], mz[kVBatch];
#pragma unroll
        for (int u = 0; u < kVBatch; ++u) {
          const int q = min(q0 + 32 * u, i4 - 1);
          mx[u] = px[q];
          my[u] = py[q];
          mz[u] = pz[q];
        }
#pragma unroll
        for (int u = 0; u < kVBatch; ++u) {
          const int q = q0 + 32 * u;
          const int cl = (q >= i1) + (q >= i2) + (q >= i3);
          T K[kVConst];
          load_row(tab[cl], K);
          if (q < i4 && K[VLIN] == T(0)) {
            const T m0 = mx[u] - K[VU0], m1 = my[u] - K[VU1], m2 = mz[u] - K[VU2];
            T n0, n1, n2;
            drift(K, m0, m1, m2, n0, n1, n2);
            const T nn = n0 * n0 + n1 * n1 + n2 * n2, mn = m0 * n0 + m1 * n1 + m2 * n2;
#pragma unroll
            for (int j = 0; j < kVCells; ++j) {
              s_nn[j] += cl == j ? nn : T(0);
              s_mn[j] += cl == j ? mn : T(0);
            }
          }
        }
      }
#pragma unroll
      for (int j = 0; j < kVCells; ++j) {
#pragma unroll
        for (int o = 16; o >= 1; o >>= 1) {
          s_nn[j] += __shfl_xor_sync(0xffffffffu, s_nn[j], o);
          s_mn[j] += __shfl_xor_sync(0xffffffffu, s_mn[j], o);
        }
      }
    }
    // ---- alpha per cell (group g, lane 0) ----
    {
      T snn = s_nn[0], smn = s_mn[0];
#pragma unroll
      for (int j = 1; j < kVCells; ++j) {
        snn = g == j ? s_nn[j] : snn;
        smn = g == j ? s_mn[j] : smn;
      }
      int flo = fl;
      T alpha = 1;
      if (valid && !linear && n > 0) {
        const T inv_n = T(1) / T(n);
        const T th = tab[g][VTH], tc = tab[g][VTAU], a = tab[g][VA], om = tab[g][VOMA];
        const T nn_avg = snn * inv_n, mn_avg = smn * inv_n;
        const T alpha2 = T(1) + tc / (T(3) * th) * (tc * om * om * nn_avg + T(2) * (a * om) * mn_avg);
        if (alpha2 > T(0) && alpha2 < T(INFINITY))
          alpha = sqrt(alpha2);
        else
          flo |= FP_FLAG_ALPHA;
      }
      __syncwarp();
      if (lg == 0) {
        tab[g][VIA] = T(1) / alpha;
        if (valid) {
          flags[c] = flo;
          if (alpha_out) alpha_out[c] = (double)alpha;
        }
      }
    }
    __syncwarp();
    // ---- pass 2: the update.  Lane l takes the quads Qs + l, Qs + l + 32, ..
    //      (quad Q = global particles 4Q .. 4Q + 3, the unit of the Philox
    //      stream); the quads at the ends of the range are partly masked.
    //      Loads go before stores, since the stores may alias later loads as
    //      far as the compiler can tell. ----
    const uint64_t g0 = prm.particle_offset + (uint64_t)o0;  // global index of the range's first particle
    const uint64_t Qs = g0 >> 2, Qe = i4 > 0 ? (g0 + (uint64_t)i4 + 3) >> 2 : Qs;
    for (uint64_t Q = Qs + (uint64_t)lane; Q < Qe; Q += 32) {
      const int qb = (int)((int64_t)(Q << 2) - (int64_t)g0);  // range index of the quad's first particle
      const bool whole = qb >= 0 && qb + 4 <= i4;
      T mx[4], my[4], mz[4];
      if (whole) {
        load_comp(px + qb, prm.vec & 3, mx);
        load_comp(py + qb, (prm.vec >> 2) & 3, my);
        load_comp(pz + qb, (prm.vec >> 4) & 3, mz);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = qb + u;
          mx[u] = my[u] = mz[u] = T(0);
          if ((unsigned)q < (unsigned)i4) {
            mx[u] = px[q];
            my[u] = py[q];
            mz[u] = pz[q];
          }
        }
      }
      T z[12];
      if (xi) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = qb + u;
          const bool in = q >= 0 && q < i4;
          const int64_t p = o0 + (in ? q : 0);
          z[3 * u] = in ? xi[p] : T(0);
          z[3 * u + 1] = in ? xi[np + p] : T(0);
          z[3 * u + 2] = in ? xi[2 * np + p] : T(0);
        }
      } else {
        float f[12];
        quad_normals(prm.key, prm.step, Q, f);
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = f[k];
      }
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        // (particles outside the range are computed on zeros and not stored)
        const int q = qb + u;
        const int cl = (q >= i1) + (q >= i2) + (q >= i3);
        T K[kVConst];
        load_row(tab[cl], K);
        const T m0 = mx[u] - K[VU0], m1 = my[u] - K[VU1], m2 = mz[u] - K[VU2];
        T n0 = 0, n1 = 0, n2 = 0;
        if (K[VLIN] == T(0)) drift(K, m0, m1, m2, n0, n1, n2);
        const T a = K[VA], df = K[VDRIFT], nz = K[VNOISE], ia = K[VIA];
        mx[u] = (m0 * a + df * n0 + nz * z[3 * u]) * ia + K[VU0];
        my[u] = (m1 * a + df * n1 + nz * z[3 * u + 1]) * ia + K[VU1];
        mz[u] = (m2 * a + df * n2 + nz * z[3 * u + 2]) * ia + K[VU2];
      }
      if (whole) {
        store_comp(ox + qb, prm.vec & 3, mx);
        store_comp(oy + qb, (prm.vec >> 2) & 3, my);
        store_comp(oz + qb, (prm.vec >> 4) & 3, mz);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = qb + u;
          if ((unsigned)q < (unsigned)i4) {
            ox[q] = mx[u];
            oy[q] = my[u];
            oz[q] = mz[u];
          }
        }
      }
    }
    __syncwarp();
  }
}

// ---------------------------------------------------------------------------
// One-pass update in chunks of 32 cells
// ---------------------------------------------------------------------------
// The constants of one cell (the table row of velocity_kernel) and alpha,
// computed by one lane from the FP64 moments, coefficients, tau and <|c|^6>
// (each entry narrowed once to T), with <N.N> and <M'.N> in closed form.
// flo: the cell's flags with FP_FLAG_ALPHA where alpha^2 is not a positive
// finite number (then alpha = 1).
template <typename T>
__device__ __forceinline__ void cell_constants(const double *__restrict__ mc, const double *__restrict__ yc,
                                               double tc_d, double m6_d, int fl, int n, const VelParams &prm,
                                               T (&vals)[kVConst], T &alpha, int &flo) {
  const bool linear = (fl & (FP_FLAG_FEW | FP_FLAG_SINGULAR | FP_FLAG_NONFINITE)) != 0;
  const T th = (T)mc[kTheta], tc = (T)tc_d;
  T u3[10], y[9];
#pragma unroll
  for (int q = 0; q < 10; ++q) u3[q] = (T)mc[kU3 + q];
#pragma unroll
  for (int q = 0; q < 9; ++q) y[q] = (T)yc[q];
  const T itau = T(1) / tc;
  const T x = T(prm.dt) * itau;
  T one_m_a, a;
  if (sizeof(T) == 4) {
    one_m_a = -expm1f((float)-x);
    a = expf((float)-x);
  } else {
    one_m_a = -expm1(-(double)x);
    a = exp(-(double)x);
  }
  // b_i = u_ikk from the third moments 111,112,113,122,123,133,222,223,233,333
  const T v[kVConst] = {(T)mc[kU], (T)mc[kU + 1], (T)mc[kU + 2], th,
                        u3[0] + u3[3] + u3[5], u3[1] + u3[6] + u3[8], u3[2] + u3[7] + u3[9],
                        y[0] + itau, y[1], y[2], y[3] + itau, y[4], y[5] + itau,
                        y[6], y[7], y[8],
                        T(prm.eps2_hat) / (tc * th), a, one_m_a * tc, sqrt(th * one_m_a * (T(1) + a)),
                        T(1), linear ? T(1) : T(0), one_m_a, tc};
#pragma unroll
  for (int q = 0; q < kVConst; ++q) vals[q] = v[q];
  T u[6], w[6], z[3];
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    u[q] = (T)mc[kU2 + q];
    w[q] = (T)mc[kW + q];
  }
#pragma unroll
  for (int q = 0; q < 3; ++q) z[q] = (T)mc[kZ + q];
  T nn, mn;
  cell_drift_averages<T>(vals, u, w, z, (T)m6_d, nn, mn);
  flo = fl;
  alpha = 1;
  if (!linear && n > 0) {
    const T alpha2 = T(1) + tc / (T(3) * th) * (tc * one_m_a * one_m_a * nn + T(2) * (a * one_m_a) * mn);
    if (alpha2 > T(0) && alpha2 < T(INFINITY))
      alpha = sqrt(alpha2);
    else
      flo |= FP_FLAG_ALPHA;
  }
  vals[VIA] = T(1) / alpha;
}

// One-pass velocity update (<|c|^6> given): every warp takes an equal slice
// of the particles (the tail of a cell that straddles the slice's start
// included; the cells that start in it are its own and write alpha and the
// flags) and walks its cells 32 at a time: lane l builds the constants of
// cell l of the chunk (table row in shared memory, alpha from the moments),
// then the warp streams the chunk's particles in quads of four consecutive
// ones (the unit of the Philox stream), finding each particle's cell among
// the chunk's 33 offsets.  A chunk's setup latency is paid once for about
// 32 cells' particles.
template <typename VT>
__global__ void __launch_bounds__(sizeof(VT) == 4 ? 256 : 128, sizeof(VT) == 4 ? 3 : 4)
    velocity_chunk_kernel(const VT *v, VT *vout, int64_t np, const int64_t *__restrict__ off, int64_t n_cells,
                          const double *__restrict__ mom, const double *__restrict__ m6,
                          const double *__restrict__ coeffs, const double *__restrict__ tau, VelParams prm,
                          const VT *__restrict__ xi, double *__restrict__ alpha_out, int32_t *__restrict__ flags) {
  using T = VT;
  constexpr int kW = sizeof(VT) == 4 ? 8 : 4;  // warps per block
  __shared__ __align__(16) T table[kW][32][kVConst];
  __shared__ int cofs[kW][33];  // the chunk's cell starts, relative to its first particle
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const VT *vx = v, *vy = v + np, *vz = v + 2 * np;
  VT *wx = vout, *wy = vout + np, *wz = vout + 2 * np;
  T(*tab)[kVConst] = table[wib];
  int *co = cofs[wib];

  // ---- the warp's slice [tA, tB) of the particles and its cells [ca, cb) ----
  const int64_t base0 = off[0], total = off[n_cells] - base0;
  auto slice = [&](int64_t k) {  // base0 + floor(total k / nwarps), exactly
    return base0 + (total / nwarps) * k + (total % nwarps) * k / nwarps;
  };
  const int64_t tA = slice(warp), tB = slice(warp + 1);
  const int64_t Lx = lower_bound16(off, n_cells, lane < 16 ? tA : tB, lane);
  const int64_t La = __shfl_sync(0xffffffffu, Lx, 0);
  const int64_t cb = warp + 1 == nwarps ? n_cells : __shfl_sync(0xffffffffu, Lx, 16);
  const int64_t ca = La > 0 && off[La] > tA ? La - 1 : La;

  for (int64_t cbase = ca; cbase < cb; cbase += 32) {
    const int64_t c = cbase + lane;
    const bool valid = c < cb;
    const int64_t a0 = off[valid ? c : cb];
    const int64_t a1 = valid ? off[c + 1] : a0;
    // the chunk's particle range, clipped to the slice
    const int64_t o0 = max(__shfl_sync(0xffffffffu, a0, 0), tA);
    const int64_t oe = min(__shfl_sync(0xffffffffu, a1, 31), tB);
    const int i4 = (int)max(oe - o0, (int64_t)0);
    co[lane] = (int)min(max(a0 - o0, (int64_t)0), (int64_t)i4);
    if (lane == 31) co[32] = i4;
    // ---- lane's cell: constants and alpha ----
    {
      T vals[kVConst];
      if (valid) {
        T alpha;
        int flo;
        cell_constants<T>(mom + c * FP_NMOM, coeffs + c * 9, tau[c], m6[c], flags[c], (int)(a1 - a0), prm, vals,
                          alpha, flo);
        if (c >= La) {  // the cell starts in this slice: its outputs are this warp's
          flags[c] = flo;
          if (alpha_out) alpha_out[c] = (double)alpha;
        }
      } else {
#pragma unroll
        for (int q = 0; q < kVConst; ++q) vals[q] = T(0);
      }
#pragma unroll
      for (int q = 0; q < kVConst; ++q) tab[lane][q] = vals[q];
    }
    __syncwarp();
    // ---- the chunk's particles, in quads ----
    const uint64_t g0 = prm.particle_offset + (uint64_t)o0;  // global index of the chunk's first particle
    const uint64_t Qs = g0 >> 2, Qe = i4 > 0 ? (g0 + (uint64_t)i4 + 3) >> 2 : Qs;
    const VT *px = vx + o0, *py = vy + o0, *pz = vz + o0;
    VT *ox = wx + o0, *oy = wy + o0, *oz = wz + o0;
    for (uint64_t Q = Qs + (uint64_t)lane; Q < Qe; Q += 32) {
      const int qb = (int)((int64_t)(Q << 2) - (int64_t)g0);  // chunk index of the quad's first particle
      const bool whole = qb >= 0 && qb + 4 <= i4;
      T mx[4], my[4], mz[4];
      if (whole) {
        load_comp(px + qb, prm.vec & 3, mx);
        load_comp(py + qb, (prm.vec >> 2) & 3, my);
        load_comp(pz + qb, (prm.vec >> 4) & 3, mz);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = qb + u;
          mx[u] = my[u] = mz[u] = T(0);
          if ((unsigned)q < (unsigned)i4) {
            mx[u] = px[q];
            my[u] = py[q];
            mz[u] = pz[q];
          }
        }
      }
      T z[12];
      if (xi) {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = qb + u;
          const bool in = (unsigned)q < (unsigned)i4;
          const int64_t p = o0 + (in ? q : 0);
          z[3 * u] = in ? xi[p] : T(0);
          z[3 * u + 1] = in ? xi[np + p] : T(0);
          z[3 * u + 2] = in ? xi[2 * np + p] : T(0);
        }
      } else {
        float f[12];
        quad_normals(prm.key, prm.step, Q, f);
#pragma unroll
        for (int k = 0; k < 12; ++k) z[k] = f[k];
      }
      // cell of the quad's first particle: the last cl with co[cl] <= max(qb, 0)
      const int q0 = max(qb, 0);
      int cl = 0;
#pragma unroll
      for (int st = 16; st >= 1; st >>= 1)
        if (co[cl + st] <= q0) cl += st;
      T K[kVConst];
      load_row(tab[cl], K);
      int next = cl < 31 ? co[cl + 1] : INT_MAX;  // where the next cell starts
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        // (particles outside the chunk are computed on zeros and not stored)
        const int q = qb + u;
        if (q >= next) {  // past a cell boundary (and any empty cells): the quad's rare case
          while (cl < 31 && co[cl + 1] <= q) ++cl;
          load_row(tab[cl], K);
          next = cl < 31 ? co[cl + 1] : INT_MAX;
        }
        const T m0 = mx[u] - K[VU0], m1 = my[u] - K[VU1], m2 = mz[u] - K[VU2];
        T n0 = 0, n1 = 0, n2 = 0;
        if (K[VLIN] == T(0)) drift(K, m0, m1, m2, n0, n1, n2);
        const T a = K[VA], df = K[VDRIFT], nz = K[VNOISE], ia = K[VIA];
        mx[u] = (m0 * a + df * n0 + nz * z[3 * u]) * ia + K[VU0];
        my[u] = (m1 * a + df * n1 + nz * z[3 * u + 1]) * ia + K[VU1];
        mz[u] = (m2 * a + df * n2 + nz * z[3 * u + 2]) * ia + K[VU2];
      }
      if (whole) {
        store_comp(ox + qb, prm.vec & 3, mx);
        store_comp(oy + qb, (prm.vec >> 2) & 3, my);
        store_comp(oz + qb, (prm.vec >> 4) & 3, mz);
      } else {
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int q = qb + u;
          if ((unsigned)q < (unsigned)i4) {
            ox[q] = mx[u];
            oy[q] = my[u];
            oz[q] = mz[u];
          }
        }
      }
    }
    __syncwarp();  // the table and offsets are rewritten by the next chunk
  }
}

static VelParams make_vel_params(double dt, double eps2_hat, uint64_t seed, uint64_t step, uint64_t poff,
                                 const void *v, const void *v_out, int64_t np, int v_dtype) {
  int vec = 0;
  if ((uintptr_t)v % 16 == 0 && (uintptr_t)v_out % 16 == 0) {
    for (int d = 0; d < 3; ++d) {
      const int e = (int)((((int64_t)d * np - (int64_t)(poff % 4)) % 4 + 4) % 4);  // element alignment
      int cls = 0;
      if (v_dtype == FP_V_F32)
        cls = e == 0 ? 2 : (e == 2 ? 1 : 0);
      else
        cls = e % 2 == 0 ? 2 : 0;  // two 16-byte pairs cover a quad of doubles
      vec |= cls << (2 * d);
    }
  }
  return VelParams{dt, eps2_hat, step, poff, philox_keys(seed), vec};
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

// A persistent grid: every warp takes an equal slice of the particles, so
// the grid is what the SMs hold at once (fewer blocks for small problems).
template <typename VT, bool kLite>
static int64_t vel_blocks(int64_t n_cells) {
  static int per_sm = 0;
  if (!per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, velocity_kernel<VT, kLite>, 32 * kVWarps, 0) !=
            cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  int64_t blocks = (int64_t)vel_sm_count() * per_sm;
  const int64_t by_cells = (n_cells + kVWarps - 1) / kVWarps;  // about one cell per warp at least
  if (blocks > by_cells) blocks = by_cells;
  return blocks < 1 ? 1 : blocks;
}

template <typename VT>
static int64_t vel_chunk_blocks(int64_t n_cells) {
  constexpr int kW = sizeof(VT) == 4 ? 8 : 4;
  static int per_sm = 0;
  if (!per_sm) {
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, velocity_chunk_kernel<VT>, 32 * kW, 0) != cudaSuccess ||
        per_sm < 1)
      per_sm = 1;
  }
  int64_t blocks = (int64_t)vel_sm_count() * per_sm;
  const int64_t by_cells = (n_cells + 4 * kW - 1) / (4 * kW);  // at least about four cells per warp
  if (blocks > by_cells) blocks = by_cells;
  return blocks < 1 ? 1 : blocks;
}

void launch_velocity(const void *v, void *v_out, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells,
                     const double *mom, const double *m6, const double *coeffs, const double *tau, double dt,
                     double eps2_hat, const void *xi, uint64_t seed, uint64_t step, uint64_t particle_offset,
                     double *alpha_out, int32_t *flags, cudaStream_t st) {
  const VelParams prm = make_vel_params(dt, eps2_hat, seed, step, particle_offset, v, v_out, np, v_dtype);
  const int threads = 32 * kVWarps;
#define FP_VEL_LAUNCH(VT)                                                                                         \
  velocity_kernel<VT><<<(unsigned)vel_blocks<VT, false>(n_cells), threads, 0, st>>>(                              \
      (const VT *)v, (VT *)v_out, np, off, n_cells, mom, m6, coeffs, tau, prm, (const VT *)xi, alpha_out, flags)
  // with <|c|^6> alpha comes from the moments: the chunked one-pass kernel
  if (m6 && v_dtype == FP_V_F32)
    velocity_chunk_kernel<float><<<(unsigned)vel_chunk_blocks<float>(n_cells), 256, 0, st>>>(
        (const float *)v, (float *)v_out, np, off, n_cells, mom, m6, coeffs, tau, prm, (const float *)xi, alpha_out,
        flags);
  else if (m6)
    velocity_chunk_kernel<double><<<(unsigned)vel_chunk_blocks<double>(n_cells), 128, 0, st>>>(
        (const double *)v, (double *)v_out, np, off, n_cells, mom, m6, coeffs, tau, prm, (const double *)xi,
        alpha_out, flags);
  else if (v_dtype == FP_V_F32)
    FP_VEL_LAUNCH(float);
  else
    FP_VEL_LAUNCH(double);
#undef FP_VEL_LAUNCH
}

// The update from LITE moment vectors (U, theta, b_i), alpha by a pass over
// the particles.
void launch_velocity_lite(const void *v, void *v_out, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells,
                          const double *lite, const double *coeffs, const double *tau, double dt, double eps2_hat,
                          const void *xi, uint64_t seed, uint64_t step, uint64_t particle_offset,
                          double *alpha_out, int32_t *flags, cudaStream_t st) {
  const VelParams prm = make_vel_params(dt, eps2_hat, seed, step, particle_offset, v, v_out, np, v_dtype);
  const int threads = 32 * kVWarps;
  if (v_dtype == FP_V_F32)
    velocity_kernel<float, true><<<(unsigned)vel_blocks<float, true>(n_cells), threads, 0, st>>>(
        (const float *)v, (float *)v_out, np, off, n_cells, lite, nullptr, coeffs, tau, prm, (const float *)xi,
        alpha_out, flags);
  else
    velocity_kernel<double, true><<<(unsigned)vel_blocks<double, true>(n_cells), threads, 0, st>>>(
        (const double *)v, (double *)v_out, np, off, n_cells, lite, nullptr, coeffs, tau, prm, (const double *)xi,
        alpha_out, flags);
}

}  // namespace fpc
