// adjoint.cu -- reverse mode through the exact closure (implicit function
// of Eq. system9x9) and through the moment gather, for sm_103a.
//
// With F(m, Y) = A(m) Y - r(m) = 0 defining the coefficients Y(m), a loss
// gradient gY = dL/dY pulls back to the moments as
//     lambda = A^-T gY,       dL/dm = -(dF/dm)^T lambda,
// and to the particle velocities through m_k = <psi_k(c)>, c = v - U:
//     dL/dv_p = (1/N) sum_k gm_k (grad psi_k(c_p) - <grad psi_k>) + gm_U / N.
//
// Kernel 1 (one thread per cell, FP64): lambda from the forward solve's
// stored factors (two triangular solves) or, without them, by re-assembling
// A and eliminating A^T with partial pivoting; then -lambda is propagated
// back through the assembly formulas by hand-written reverse mode.  Kernel 2 (four consecutive cells per warp, their particles
// walked flat by all lanes): the per-particle polynomial above, in the
// velocity's precision, one pass over the particles.
#include <cstdint>

#include "closure_math.cuh"
#include "fp_device.cuh"

namespace fpc {

// gm += -(dF/dm)^T lambda for F(m, Y) = A(m) Y - r(m) (the assembly of
// Eq. system9x9 differentiated by hand), with u, w, u3 adjoints kept per full
// index and folded onto the symmetric moment slots at the end.  Every factor
// that does not depend on the row's lambda is formed once per cell, so each
// term costs one FMA on the (scarce) FP64 pipe.
//   stress rows (ij): F = sum_k (C_ik u_kj + C_jk u_ki) + G_i b_j + G_j b_i
//                         + (2 / tau) u_ij - 2 e2 w_ij
//   heat rows (i):    F = sum_l C_il b_l + 2 sum_kl C_kl u_ikl + G_i (s4 - 9 th^2)
//                         + 2 sum_k G_k (w_ki - 3 th u_ki) + (4 / (3 tau)) b_i
//                         - e2 (3 z_i - 3 th b_i - 2 sum_k u_ik b_k)
// with b_i = sum_k u_ikk, s4 = sum_k w_kk, e2 = eps2_hat / (tau th).  With
// kAdd the results are added to gm, else they are stored in the 26 slots they
// fill (the N and U slots are left as they are).
template <bool kAdd>
__host__ __device__ __forceinline__ void assembly_vjp(const double (&m)[FP_NMOM], const double (&Y)[9],
                                                      const double (&lam)[9], double tc, double eps2_hat,
                                                      double (&gm)[FP_NMOM]) {
  double C[3][3], G[3], u[3][3], w[3][3], b[3], z[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    G[i] = Y[6 + i];
    z[i] = m[kZ + i];
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      C[i][j] = Y[sym2(i, j)];
      u[i][j] = m[kU2 + sym2(i, j)];
      w[i][j] = m[kW + sym2(i, j)];
    }
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) b[i] = m[kU3 + sym3(i, 0, 0)] + m[kU3 + sym3(i, 1, 1)] + m[kU3 + sym3(i, 2, 2)];
  const double th = m[kTheta];
  const double itau = 1.0 / tc, ith = 1.0 / th;
  const double e2 = eps2_hat * itau * ith;
  // per-cell factors of the row adjoints
  const double itau2 = 2.0 * itau, me2x2 = -2.0 * e2, e2x2 = 2.0 * e2, mz = -3.0 * e2;
  const double kb = fma(4.0 / 3.0, itau, 3.0 * e2 * th);  // heat row i on b_i
  const double m18th = -18.0 * th, m6th = -6.0 * th, e2x3 = 3.0 * e2, th3 = 3.0 * th;
  double G2[3], G6[3], eb2[3], P[3], E[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    G2[k] = 2.0 * G[k];
    G6[k] = m6th * G[k];
    eb2[k] = e2x2 * b[k];
  }
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    // heat row i on theta: -18 th G_i - 6 sum_k G_k u_ki + 3 e2 b_i;
    // on e2: -(3 z_i - 3 th b_i - 2 sum_k u_ik b_k)
    const double gu = fma(G[0], u[0][i], fma(G[1], u[1][i], G[2] * u[2][i]));
    const double ubs = fma(u[i][0], b[0], fma(u[i][1], b[1], u[i][2] * b[2]));
    P[i] = fma(m18th, G[i], fma(-6.0, gu, e2x3 * b[i]));
    E[i] = fma(2.0, ubs, fma(th3, b[i], -3.0 * z[i]));
  }
  double ub[3][3] = {}, wb[3][3] = {}, u3b[10] = {}, zb[3], bb[3] = {};
  double thb = 0.0, s4b = 0.0, e2b = 0.0, sw = 0.0;
  // stress rows
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const double f = -lam[sym2(i, j)];
#pragma unroll
      for (int k = 0; k < 3; ++k) {
        ub[k][j] = fma(f, C[i][k], ub[k][j]);
        ub[k][i] = fma(f, C[j][k], ub[k][i]);
      }
      bb[j] = fma(f, G[i], bb[j]);
      bb[i] = fma(f, G[j], bb[i]);
      ub[i][j] = fma(f, itau2, ub[i][j]);
      wb[i][j] = fma(f, me2x2, wb[i][j]);
      sw = fma(f, w[i][j], sw);  // e2 adjoint: -2 sum f w_ij
    }
  // heat-flux rows
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const double f = -lam[6 + i], f2 = 2.0 * f, f4 = 4.0 * f, fe = e2x2 * f;
#pragma unroll
    for (int l = 0; l < 3; ++l) bb[l] = fma(f, C[i][l], bb[l]);
    // 2 sum_kl C_kl u_ikl: a slot with k != l collects (k, l) and (l, k)
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      u3b[sym3(i, k, k)] = fma(f2, C[k][k], u3b[sym3(i, k, k)]);
#pragma unroll
      for (int l = k + 1; l < 3; ++l) u3b[sym3(i, k, l)] = fma(f4, C[k][l], u3b[sym3(i, k, l)]);
    }
    s4b = fma(f, G[i], s4b);
    thb = fma(f, P[i], thb);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      wb[k][i] = fma(f, G2[k], wb[k][i]);
      ub[k][i] = fma(f, G6[k], ub[k][i]);
      ub[i][k] = fma(f, eb2[k], ub[i][k]);
      bb[k] = fma(fe, u[i][k], bb[k]);
    }
    bb[i] = fma(f, kb, bb[i]);
    zb[i] = f * mz;
    e2b = fma(f, E[i], e2b);
  }
  // e2 = eps2_hat / (tau th);  b_i = sum_k u_ikk;  s4 = sum_k w_kk
  e2b = fma(-2.0, sw, e2b);
  thb = fma(e2b, -e2 * ith, thb);
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int k = 0; k < 3; ++k) u3b[sym3(i, k, k)] += bb[i];
#pragma unroll
  for (int k = 0; k < 3; ++k) wb[k][k] += s4b;
  // fold onto the moment slots
  auto put = [&](int k, double v) {
    if (kAdd)
      gm[k] += v;
    else
      gm[k] = v;
  };
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      put(kU2 + sym2(i, j), i != j ? ub[i][j] + ub[j][i] : ub[i][j]);
      put(kW + sym2(i, j), i != j ? wb[i][j] + wb[j][i] : wb[i][j]);
    }
#pragma unroll
  for (int q = 0; q < 10; ++q) put(kU3 + q, u3b[q]);
#pragma unroll
  for (int i = 0; i < 3; ++i) put(kZ + i, zb[i]);
  put(kTheta, thb);
}

template <bool kLU>
__device__ __forceinline__ void adjoint_cell(int64_t c, const double *__restrict__ mom,
                                             const double *__restrict__ coeffs, const int32_t *__restrict__ flags,
                                             const double *__restrict__ lu, const double *__restrict__ tau,
                                             const double *__restrict__ gY, const double *__restrict__ gm_in,
                                             double eps2_hat, double *__restrict__ gm_out) {
  double gm[FP_NMOM];
#pragma unroll
  for (int k = 0; k < FP_NMOM; ++k) gm[k] = gm_in ? gm_in[c * FP_NMOM + k] : 0.0;
  const int fl = flags[c];
  if (!(fl & (FP_FLAG_FEW | FP_FLAG_SINGULAR | FP_FLAG_NONFINITE))) {
    double m[FP_NMOM];
#pragma unroll
    for (int k = 0; k < FP_NMOM; ++k) m[k] = mom[c * FP_NMOM + k];
    const double tc = tau[c];
    // lambda = A^-T gY: with the forward's factors two triangular solves,
    // else eliminate the transposed augmented system
    double lam[9];
    if (kLU) {
      double g[9];
#pragma unroll
      for (int i = 0; i < 9; ++i) g[i] = gY[c * 9 + i];
      lu_solve_transposed(lu + lu_base(c), g, lam);
    } else {
      double a[9][10];
      assemble(m, tc, eps2_hat, a);
      double at[9][10];
#pragma unroll
      for (int i = 0; i < 9; ++i) {
#pragma unroll
        for (int j = 0; j < 9; ++j) at[i][j] = a[j][i];
        at[i][9] = gY[c * 9 + i];
      }
      pivoted_solve(at, 0.0, lam);
    }
    double Y[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) Y[q] = coeffs[c * 9 + q];
    if (gm_in)
      assembly_vjp<true>(m, Y, lam, tc, eps2_hat, gm);
    else
      assembly_vjp<false>(m, Y, lam, tc, eps2_hat, gm);
  }
#pragma unroll
  for (int k = 0; k < FP_NMOM; ++k) gm_out[c * FP_NMOM + k] = gm[k];
}

// One thread per cell, grid-stride, two 128-thread blocks per SM (FP64-bound:
// see solve_kernel), registers capped at 128 a thread (the rest spills to
// L1): half the register file stays free for the velocity update and the
// learned closure running beside it.
template <bool kLU>
__global__ void __launch_bounds__(128, 4) adjoint_cell_kernel(const double *__restrict__ mom,
                                                              const double *__restrict__ coeffs,
                                                              const int32_t *__restrict__ flags,
                                                              const double *__restrict__ lu,
                                                              const double *__restrict__ tau,
                                                              const double *__restrict__ gY,
                                                              const double *__restrict__ gm_in, int64_t n_cells,
                                                              double eps2_hat, double *__restrict__ gm_out) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells;
       c += (int64_t)gridDim.x * blockDim.x)
    adjoint_cell<kLU>(c, mom, coeffs, flags, lu, tau, gY, gm_in, eps2_hat, gm_out);
}

// ---------------------------------------------------------------------------
// particle gradient
// ---------------------------------------------------------------------------
constexpr int kAG = 8;              // lanes per cell while building constants
constexpr int kACells = 32 / kAG;   // consecutive cells per warp task
constexpr int kAWarps = 8;          // warps per block
constexpr int kAConst = 44;         // table entries per cell

// Per-cell table of the particle polynomial, every coefficient already
// multiplied by 1/N and by its constant factor:
//   dL/dv_d = Mu'_d.c + sum_{j<=k} A3'_{d,jk} c_j c_k
//             + c_d (c.W'c + |c|^2 gz'.c) + |c|^2 (W'c)_d + |c|^4 gz''_d + B_d
// with Mu' = Mu/N, A3'_{d,jk} = 3 m_jk A_{djk}/N (m = 1 on, 2 off the
// diagonal), W' = 2W/N, gz' = 4gz/N, gz'' = gz/N, B = (gm_U - <grad psi>)/N.
enum { AU = 0, AMU = 3, AA3 = 9, AW = 27, AGZ4 = 33, AGZ1 = 36, AB = 39 };

template <typename T>
__device__ __forceinline__ T shfl_g(T x, int src, int lane) {
  return __shfl_sync(0xffffffffu, x, (lane & ~(kAG - 1)) + src);
}

// multiplicity of a symmetric third-order slot (111: 1, 112: 3, 123: 6)
__host__ __device__ constexpr int mult3(int s) { return (s == 0 || s == 6 || s == 9) ? 1 : (s == 4 ? 6 : 3); }

// A warp takes four consecutive cells; an 8-lane group folds its cell's
// moments and moment gradients into the 35 coefficients of the per-particle
// polynomial (shared-memory table), then all 32 lanes walk the four cells'
// contiguous particle range.
template <typename VT>
__global__ void __launch_bounds__(32 * kAWarps, sizeof(VT) == 4 ? 3 : 1) adjoint_particle_kernel(const VT *__restrict__ v, int64_t np,
                                                                        const int64_t *__restrict__ off,
                                                                        int64_t n_cells,
                                                                        const double *__restrict__ mom,
                                                                        const double *__restrict__ gm,
                                                                        VT *__restrict__ gv) {
  using T = VT;
  constexpr int G = kAG;
  __shared__ __align__(16) T table[kAWarps][kACells][kAConst];
  const int lane = threadIdx.x & 31;
  const int wib = threadIdx.x >> 5;
  const int lg = lane & (G - 1);
  const int g = lane / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const VT *vx = v, *vy = v + np, *vz = v + 2 * np;
  VT *gx = gv, *gy = gv + np, *gz = gv + 2 * np;
  T(*tab)[kAConst] = table[wib];

  for (int64_t base = warp * kACells; base < n_cells; base += nwarps * kACells) {
    const int64_t c = base + g;
    const bool valid = c < n_cells;
    const int64_t a0 = off[valid ? c : n_cells];
    const int64_t e = valid ? off[c + 1] : a0;
    const int n = (int)(e - a0);
    // the cell's 30 moments and 30 moment gradients, converted once: lane lg
    // holds slots lg + 8 j of the concatenation [mom | gm] (60 values)
    T cv[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) {
      const int slot = lg + 8 * j;
      double x = 0.0;
      if (valid && slot < 60) x = slot < 30 ? mom[c * FP_NMOM + slot] : gm[c * FP_NMOM + slot - 30];
      cv[j] = (T)x;
    }
    {
      auto M_ = [&](int k) -> T { return shfl_g(cv[k / 8], k % 8, lane); };
      auto GM = [&](int k) -> T { return shfl_g(cv[(30 + k) / 8], (30 + k) % 8, lane); };
      // u-part: G_d += sum_j Mu_dj c_j with Mu_dj = gm_u(dj) (1 + delta_dj); theta adds 2/3 gm_theta c_d
      const T gth = GM(kTheta) * T(2.0 / 3.0);
      T Mu[6];
#pragma unroll
      for (int s = 0; s < 6; ++s) {
        const bool diag = s == 0 || s == 3 || s == 5;
        Mu[s] = GM(kU2 + s) * (diag ? T(2) : T(1)) + (diag ? gth : T(0));
      }
      // u3-part: G_d += 3 sum_jk A_djk c_j c_k with A = gm_u3(slot) / multiplicity
      T A3[10];
#pragma unroll
      for (int s = 0; s < 10; ++s) A3[s] = GM(kU3 + s) / T(mult3(s));
      // w-part: G_d += 2 c_d (c.W c) + 2 |c|^2 (W c)_d with W = gm_w(slot) / multiplicity
      T W[3][3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) W[i][j] = GM(kW + sym2(i, j)) * (i == j ? T(1) : T(0.5));
      // z-part: G_d += 4 |c|^2 c_d (gz.c) + |c|^4 gz_d
      const T gzv[3] = {GM(kZ), GM(kZ + 1), GM(kZ + 2)};
      // the cell mean of grad psi, from the moments
      T G0[3];
      {
        T u[3][3], w[3][3], b[3], u3[10];
#pragma unroll
        for (int s = 0; s < 10; ++s) u3[s] = M_(kU3 + s);
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = 0; j < 3; ++j) {
            u[i][j] = M_(kU2 + sym2(i, j));
            w[i][j] = M_(kW + sym2(i, j));
          }
#pragma unroll
        for (int i = 0; i < 3; ++i) b[i] = u3[sym3(i, 0, 0)] + u3[sym3(i, 1, 1)] + u3[sym3(i, 2, 2)];
        const T s4 = w[0][0] + w[1][1] + w[2][2];
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          T acc = 0;
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = 0; k < 3; ++k)
              acc += T(3) * A3[sym3(d, j, k)] * u[j][k] + T(2) * W[j][k] * u3[sym3(d, j, k)];
#pragma unroll
          for (int j = 0; j < 3; ++j) acc += T(2) * W[d][j] * b[j] + T(4) * gzv[j] * w[d][j];
          acc += s4 * gzv[d];
          G0[d] = acc;
        }
      }
      const T inv_n = n > 0 ? T(1) / T(n) : T(0);
      const T U0 = M_(kU), U1 = M_(kU + 1), U2 = M_(kU + 2);
      const T gU0 = GM(kU) * inv_n, gU1 = GM(kU + 1) * inv_n, gU2 = GM(kU + 2) * inv_n;
      if (lg == 0) {
        T *r = tab[g];
        r[AU] = U0;
        r[AU + 1] = U1;
        r[AU + 2] = U2;
#pragma unroll
        for (int s = 0; s < 6; ++s) r[AMU + s] = Mu[s] * inv_n;
#pragma unroll
        for (int d = 0; d < 3; ++d)
#pragma unroll
          for (int j = 0; j < 3; ++j)
#pragma unroll
            for (int k = j; k < 3; ++k)
              r[AA3 + 6 * d + sym2(j, k)] = A3[sym3(d, j, k)] * (j == k ? T(3) : T(6)) * inv_n;
#pragma unroll
        for (int i = 0; i < 3; ++i)
#pragma unroll
          for (int j = i; j < 3; ++j) r[AW + sym2(i, j)] = T(2) * W[i][j] * inv_n;
        const T gUv[3] = {gU0, gU1, gU2};
#pragma unroll
        for (int d = 0; d < 3; ++d) {
          r[AGZ4 + d] = T(4) * gzv[d] * inv_n;
          r[AGZ1 + d] = gzv[d] * inv_n;
          r[AB + d] = gUv[d] - G0[d] * inv_n;
        }
        r[AB + 3] = T(0);
        r[AB + 4] = T(0);
      }
    }
    const int64_t o0 = __shfl_sync(0xffffffffu, a0, 0);
    const int i1 = (int)(__shfl_sync(0xffffffffu, a0, 8) - o0);
    const int i2 = (int)(__shfl_sync(0xffffffffu, a0, 16) - o0);
    const int i3 = (int)(__shfl_sync(0xffffffffu, a0, 24) - o0);
    const int i4 = (int)(__shfl_sync(0xffffffffu, e, 24) - o0);
    const VT *px = vx + o0, *py = vy + o0, *pz = vz + o0;
    VT *qx = gx + o0, *qy = gy + o0, *qz = gz + o0;
    __syncwarp();
#pragma unroll 2
    for (int q = lane; q < i4; q += 32) {
      const int cl = (q >= i1) + (q >= i2) + (q >= i3);
      T K[kAConst];
      load_row(tab[cl], K);
      const T cc[3] = {px[q] - K[AU], py[q] - K[AU + 1], pz[q] - K[AU + 2]};
      // the six products c_j c_k (j <= k), in sym2 order
      const T pr[6] = {cc[0] * cc[0], cc[0] * cc[1], cc[0] * cc[2], cc[1] * cc[1], cc[1] * cc[2], cc[2] * cc[2]};
      const T r2 = pr[0] + pr[3] + pr[5];
      const T r4 = r2 * r2;
      T Wc[3];
#pragma unroll
      for (int i = 0; i < 3; ++i)
        Wc[i] = K[AW + sym2(i, 0)] * cc[0] + K[AW + sym2(i, 1)] * cc[1] + K[AW + sym2(i, 2)] * cc[2];
      const T t = cc[0] * Wc[0] + cc[1] * Wc[1] + cc[2] * Wc[2] +
                  r2 * (K[AGZ4] * cc[0] + K[AGZ4 + 1] * cc[1] + K[AGZ4 + 2] * cc[2]);
      T out[3];
#pragma unroll
      for (int d = 0; d < 3; ++d) {
        T gd = K[AMU + sym2(d, 0)] * cc[0] + K[AMU + sym2(d, 1)] * cc[1] + K[AMU + sym2(d, 2)] * cc[2];
#pragma unroll
        for (int s = 0; s < 6; ++s) gd += K[AA3 + 6 * d + s] * pr[s];
        out[d] = gd + cc[d] * t + r2 * Wc[d] + r4 * K[AGZ1 + d] + K[AB + d];
      }
      qx[q] = out[0];
      qy[q] = out[1];
      qz[q] = out[2];
    }
    __syncwarp();
  }
}

static int adj_sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

void launch_adjoint(const void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, const double *tau,
                    double eps2_hat, const double *mom, const double *coeffs, const int32_t *flags, const double *lu,
                    const double *gY, const double *gm_in, double *gm_out, void *gv, cudaStream_t st) {
  {
    const int threads = 128;
    int64_t blocks = (n_cells + threads - 1) / threads;
    if (blocks > 2 * adj_sm_count()) blocks = 2 * adj_sm_count();
    if (lu)
      adjoint_cell_kernel<true><<<(unsigned)blocks, threads, 0, st>>>(mom, coeffs, flags, lu, tau, gY, gm_in,
                                                                      n_cells, eps2_hat, gm_out);
    else
      adjoint_cell_kernel<false><<<(unsigned)blocks, threads, 0, st>>>(mom, coeffs, flags, nullptr, tau, gY, gm_in,
                                                                       n_cells, eps2_hat, gm_out);
  }
  if (!gv) return;
  const int threads = 32 * kAWarps;
  const int64_t cells_per_block = kAWarps * kACells;
  int64_t blocks = (n_cells + cells_per_block - 1) / cells_per_block;
  const int64_t cap = (int64_t)adj_sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (v_dtype == FP_V_F32)
    adjoint_particle_kernel<float><<<(unsigned)blocks, threads, 0, st>>>((const float *)v, np, off, n_cells, mom,
                                                                         gm_out, (float *)gv);
  else
    adjoint_particle_kernel<double><<<(unsigned)blocks, threads, 0, st>>>((const double *)v, np, off, n_cells, mom,
                                                                          gm_out, (double *)gv);
}

}  // namespace fpc
