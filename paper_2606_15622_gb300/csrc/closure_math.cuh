// closure_math.cuh -- per-cell FP64 assembly of the 9x9 moment-matching
// system (Eq. system9x9, Table 1 and its heat-flux rows) and the partial-pivot
// elimination, shared by the forward solve and the adjoint kernels.
#pragma once

#include <cstdint>

#include "fp_device.cuh"

namespace fpc {

__host__ __device__ __forceinline__ constexpr int sym2(int i, int j) {
  return (i < j ? i : j) == 0 ? (i > j ? i : j) : ((i < j ? i : j) == 1 ? 2 + (i > j ? i : j) : 5);
}
// (i,j,k) -> 0..9 in the order 111,112,113,122,123,133,222,223,233,333
__host__ __device__ __forceinline__ constexpr int sym3s(int i, int j, int k) {  // i <= j <= k
  return i == 0 ? (j == 0 ? k : (j == 1 ? 2 + k : 5)) : (i == 1 ? (j == 1 ? 5 + k : 8) : 9);
}
__host__ __device__ __forceinline__ constexpr int sym3(int i, int j, int k) {
  return sym3s(i < j ? (i < k ? i : k) : (j < k ? j : k),
               i + j + k - (i < j ? (i < k ? i : k) : (j < k ? j : k)) - (i > j ? (i > k ? i : k) : (j > k ? j : k)),
               i > j ? (i > k ? i : k) : (j > k ? j : k));
}
static_assert(sym2(2, 1) == 4 && sym2(1, 1) == 3 && sym2(0, 2) == 2, "sym2");
static_assert(sym3(2, 0, 1) == 4 && sym3(1, 2, 2) == 8 && sym3(2, 1, 1) == 7 && sym3(0, 2, 0) == 2, "sym3");


// fused multiply-add in the arithmetic of the operands
__device__ __forceinline__ double tfma(double a, double b, double c) { return fma(a, b, c); }
__device__ __forceinline__ float tfma(float a, float b, float c) { return fmaf(a, b, c); }

struct SolveParams {
  double eps2_hat;
  double pivot_rtol;
  int min_particles;
  int min_regular;  // cells with fewer particles are flagged singular without a solve
};

// Assemble the augmented system [A | r] (moment-matching rows for psi =
// c_i c_j and psi = c_i |c|^2; see fpclosure.h for the readings).
//   stress rows (ij):  sum_k (C_ik u_kj + C_jk u_ki) + G_i b_j + G_j b_i
//                      = -(2/tau) u_ij + 2 eps^2 w_ij
//   heat rows (i):     sum_l C_il b_l + 2 sum_kl C_kl u_ikl + G_i (s4 - 9 theta^2)
//                      + 2 sum_k G_k (w_ki - 3 theta u_ki)
//                      = -(4/(3 tau)) b_i + eps^2 (3 z_i - 3 theta b_i - 2 u_ik b_k)
// Every nonzero entry is handed to emit(row, col, value) as its own closed
// expression (a copy where a single moment is the coefficient): on this GPU
// each FP64 instruction is expensive, and accumulating into zeroed entries
// would cost an FP64 add per term.  Row and column are compile-time constants
// once the loops unroll; entries never emitted are zero.
template <typename T, class Emit>
__device__ __forceinline__ void assemble_emit(const T (&m)[FP_NMOM], T tau, T eps2_hat, Emit &&emit) {
  T u[3][3], w[3][3], b[3];
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j) {
      u[i][j] = m[kU2 + sym2(i, j)];
      w[i][j] = m[kW + sym2(i, j)];
    }
#pragma unroll
  for (int i = 0; i < 3; ++i)
    b[i] = m[kU3 + sym3(i, 0, 0)] + m[kU3 + sym3(i, 1, 1)] + m[kU3 + sym3(i, 2, 2)];
  const T theta = m[kTheta];
  const T s4 = w[0][0] + w[1][1] + w[2][2];
  const T eps2 = eps2_hat / (tau * theta);
  const T inv_tau = T(1) / tau;
  const T c_u = T(-2) * inv_tau, c_w = T(2) * eps2;  // stress right-hand side
  const T th3 = T(3) * theta;
  // stress rows
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = i; j < 3; ++j) {
      const int row = sym2(i, j);
      if (i == j) {
        // 2 sum_k C_ik u_ki + 2 G_i b_i
#pragma unroll
        for (int k = 0; k < 3; ++k) emit(row, sym2(i, k), T(2) * u[k][i]);
        emit(row, 6 + i, T(2) * b[i]);
      } else {
        // C_ii u_ij + C_jj u_ij + C_ij (u_ii + u_jj) + C_it u_tj + C_jt u_ti
        const int t = 3 - i - j;
        emit(row, sym2(i, i), u[i][j]);
        emit(row, sym2(j, j), u[i][j]);
        emit(row, sym2(i, j), u[i][i] + u[j][j]);
        emit(row, sym2(i, t), u[t][j]);
        emit(row, sym2(j, t), u[t][i]);
        emit(row, 6 + i, b[j]);
        emit(row, 6 + j, b[i]);
      }
      emit(row, 9, c_u * u[i][j] + c_w * w[i][j]);
    }
  // heat-flux rows
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    const int row = 6 + i;
#pragma unroll
    for (int p = 0; p < 3; ++p)
#pragma unroll
      for (int q = p; q < 3; ++q) {
        // C_pq: b from sum_l C_il b_l (if i is p or q), then 2 u_ipp or 4 u_ipq
        const T u3 = m[kU3 + sym3(i, p, q)];
        T bterm = T(0);
        bool has_b = false;
        if (p == i) {
          bterm = b[q];
          has_b = true;
        } else if (q == i) {
          bterm = b[p];
          has_b = true;
        }
        const T f = p == q ? T(2) : T(4);
        emit(row, sym2(p, q), has_b ? tfma(f, u3, bterm) : f * u3);
      }
#pragma unroll
    for (int k = 0; k < 3; ++k) {
      const T gk = T(2) * tfma(-th3, u[k][i], w[k][i]);
      emit(row, 6 + k, k == i ? (s4 - T(9) * theta * theta) + gk : gk);
    }
    const T ub = u[i][0] * b[0] + u[i][1] * b[1] + u[i][2] * b[2];
    emit(row, 9, T(-4.0 / 3.0) * inv_tau * b[i] + eps2 * (T(3) * m[kZ + i] - th3 * b[i] - T(2) * ub));
  }
}

__device__ __forceinline__ void assemble(const double (&m)[FP_NMOM], double tau, double eps2_hat,
                                         double (&a)[9][10]) {
#pragma unroll
  for (int r = 0; r < 9; ++r)
#pragma unroll
    for (int col = 0; col < 10; ++col) a[r][col] = 0.0;
  assemble_emit(m, tau, eps2_hat, [&](int row, int col, double v) { a[row][col] = v; });
}

// One elimination step for column K (a template so every index is static and
// the matrix stays in registers).  With kLU the whole rows are swapped and
// the multipliers are kept below the diagonal, so that afterwards P A = L U
// with L unit lower triangular in a[i][j < i], U in a[i][j >= i], and the
// row swapped with row K at step K in bits 4K..4K+3 of perm.
template <int K, bool kLU>
__device__ __forceinline__ void elim_step(double (&a)[9][10], uint64_t thr, int &flag, double (&rinv)[9],
                                          uint64_t &perm) {
  uint64_t best = abs_bits(a[K][K]);
  int bi = K;
#pragma unroll
  for (int i = K + 1; i < 9; ++i) {
    const uint64_t bb = abs_bits(a[i][K]);
    if (bb > best) {
      best = bb;
      bi = i;
    }
  }
  if (!(best > thr)) flag = FP_FLAG_SINGULAR;
  if (kLU) perm |= (uint64_t)bi << (4 * K);
#pragma unroll
  for (int i = K + 1; i < 9; ++i) {
    const bool sw = (bi == i);
#pragma unroll
    for (int j = kLU ? 0 : K; j < 10; ++j) {
      const double t = a[K][j];
      a[K][j] = sw ? a[i][j] : t;
      a[i][j] = sw ? t : a[i][j];
    }
  }
  rinv[K] = 1.0 / a[K][K];
#pragma unroll
  for (int i = K + 1; i < 9; ++i) {
    const double l = a[i][K] * rinv[K];
    if (kLU) a[i][K] = l;
#pragma unroll
    for (int j = K + 1; j < 10; ++j) a[i][j] = fma(-l, a[K][j], a[i][j]);
  }
}

// Partial-pivot elimination and back substitution on [A | r]; returns
// FP_FLAG_SINGULAR if a pivot is <= rtol * max|A| (y is then garbage).
// With kLU the factors stay in a (see elim_step), rinv holds the reciprocal
// pivots and perm the row swaps.
template <bool kLU = false>
__device__ __forceinline__ int pivoted_solve(double (&a)[9][10], double rtol, double (&y)[9], double (&rinv)[9],
                                             uint64_t &perm) {
  uint64_t amax = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i)
#pragma unroll
    for (int j = 0; j < 9; ++j) amax = max(amax, abs_bits(a[i][j]));
  const double amax_d = __longlong_as_double((long long)amax);
  int flag = 0;
  if (!(amax_d > 0.0) || !finite_d(amax_d)) flag = FP_FLAG_SINGULAR;
  const uint64_t thr = abs_bits(rtol * amax_d);
  perm = 0;
  elim_step<0, kLU>(a, thr, flag, rinv, perm);
  elim_step<1, kLU>(a, thr, flag, rinv, perm);
  elim_step<2, kLU>(a, thr, flag, rinv, perm);
  elim_step<3, kLU>(a, thr, flag, rinv, perm);
  elim_step<4, kLU>(a, thr, flag, rinv, perm);
  elim_step<5, kLU>(a, thr, flag, rinv, perm);
  elim_step<6, kLU>(a, thr, flag, rinv, perm);
  elim_step<7, kLU>(a, thr, flag, rinv, perm);
  elim_step<8, kLU>(a, thr, flag, rinv, perm);
#pragma unroll
  for (int k = 8; k >= 0; --k) {
    double s = a[k][9];
#pragma unroll
    for (int j = k + 1; j < 9; ++j) s = fma(-a[k][j], y[j], s);
    y[k] = s * rinv[k];
  }
  return flag;
}
__device__ __forceinline__ int pivoted_solve(double (&a)[9][10], double rtol, double (&y)[9]) {
  double rinv[9];
  uint64_t perm;
  return pivoted_solve<false>(a, rtol, y, rinv, perm);
}

// Stored factors: FP_LU_STRIDE doubles per cell -- L below / reciprocal
// pivots on / U above the diagonal (row-major 9 x 9), then the packed swaps
// as the bits of a double -- tiled by 32 cells: entry k of cell c lives at
// lu[(c / 32) * 32 * FP_LU_STRIDE + 32 k + c % 32], so the 32 cells of a warp
// write and read each entry as one contiguous 256-byte line.
__device__ __forceinline__ int64_t lu_base(int64_t c) { return (c >> 5) * 32 * FP_LU_STRIDE + (c & 31); }

// Solve A^T x = g with the stored factors of P A = L U: U^T z = g (forward),
// L^T w = z (backward), x = P^T w (the swaps undone in reverse order).
// lu points at the cell's first entry (lu_base); entries are 32 apart.
__device__ __forceinline__ void lu_solve_transposed(const double *__restrict__ lu, const double (&g)[9],
                                                    double (&x)[9]) {
  double z[9];
#pragma unroll
  for (int i = 0; i < 9; ++i) {
    double s = g[i];
#pragma unroll
    for (int k = 0; k < i; ++k) s = fma(-lu[32 * (k * 9 + i)], z[k], s);  // U^T[i][k] = U[k][i]
    z[i] = s * lu[32 * (i * 9 + i)];
  }
#pragma unroll
  for (int i = 8; i >= 0; --i) {
    double s = z[i];
#pragma unroll
    for (int k = i + 1; k < 9; ++k) s = fma(-lu[32 * (k * 9 + i)], x[k], s);  // L^T[i][k] = L[k][i]
    x[i] = s;
  }
  const uint64_t perm = (uint64_t)__double_as_longlong(lu[32 * 81]);
#pragma unroll
  for (int K = 8; K >= 0; --K) {
    const int bi = (int)((perm >> (4 * K)) & 15u);
    // swap x[K] and x[bi] (bi >= K) with selects: registers stay static
    double xk = x[K];
#pragma unroll
    for (int i = K + 1; i < 9; ++i) {
      const bool sw = bi == i;
      const double t = x[i];
      x[i] = sw ? xk : t;
      xk = sw ? t : xk;
    }
    x[K] = xk;
  }
}

// The closure of one cell from its moment vector: flags, and Y (the linear
// drift C = -I/tau, G = 0 for flagged cells).  With lu != nullptr the factors
// of an unflagged cell are written there (the cell's first entry, see
// lu_base; entries 32 apart).
template <bool kLU = false>
__device__ __forceinline__ int closure_cell(const double *__restrict__ mc, double tc, const SolveParams &prm,
                                            double (&y)[9], double *__restrict__ lu = nullptr) {
  double m[FP_NMOM];
#pragma unroll
  for (int k = 0; k < FP_NMOM; ++k) m[k] = mc[k];
  int fl = 0;
  bool fin = finite_d(tc) && tc > 0.0;
#pragma unroll
  for (int k = 0; k < FP_NMOM; ++k) fin = fin && finite_d(m[k]);
  if (!fin) fl |= FP_FLAG_NONFINITE;
  if (m[kN] < (double)prm.min_particles) fl |= FP_FLAG_FEW;
  if (!(m[kTheta] > 0.0)) fl |= FP_FLAG_SINGULAR;
  if (!fl && m[kN] < (double)prm.min_regular) fl |= FP_FLAG_SINGULAR;
  if (!fl) {
    double a[9][10], rinv[9];
    uint64_t perm;
    assemble(m, tc, prm.eps2_hat, a);
    fl |= pivoted_solve<kLU>(a, prm.pivot_rtol, y, rinv, perm);
    if (!fl) {
#pragma unroll
      for (int q = 0; q < 9; ++q)
        if (!finite_d(y[q])) fl |= FP_FLAG_NONFINITE;
    }
    if (kLU && !fl) {
#pragma unroll
      for (int i = 0; i < 9; ++i)
#pragma unroll
        for (int j = 0; j < 9; ++j) lu[32 * (i * 9 + j)] = i == j ? rinv[i] : a[i][j];
      lu[32 * 81] = __longlong_as_double((long long)perm);
    }
  }
  if (fl) {
    const double c0 = (finite_d(tc) && tc > 0.0) ? -1.0 / tc : 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) y[q] = 0.0;
    y[0] = c0;
    y[3] = c0;
    y[5] = c0;
  }
  return fl;
}

// ---------------------------------------------------------------------------
// Mixed-precision solve for FP32 moments: the system is factored in FP32 (on
// the FP32 pipe), the residual b - A x is formed in FP64 straight from the
// emitted entries (the FP64 matrix is never stored), and one correction solve
// with the FP32 factors refines x.  Each FP64 instruction costs this GPU ~64
// times an FP32 one, so this moves about three quarters of the FP64 work of
// the plain solve off the FP64 pipe.  The refinement converges at a rate of
// about kappa times the FP32 rounding of the system, and on an ill-conditioned
// cell a small correction does not mean a small error, so a cell is refined
// only if its smallest FP32 pivot is at least max(3e-3, 100 rtol) of max|A|
// (kappa of order 1e3 at most; 0.03 % of the cylinder's cells fail this) and
// its correction is at most 1e-4 of x; any other cell is solved again by the
// FP64 elimination, which then also decides its flags.
// ---------------------------------------------------------------------------
template <int K>
__device__ __forceinline__ void lu_step_f(float (&a)[9][10], float (&rinv)[9], uint64_t &perm, uint32_t &pmin) {
  uint32_t best = __float_as_uint(a[K][K]) & 0x7fffffffu;
  int bi = K;
#pragma unroll
  for (int i = K + 1; i < 9; ++i) {
    const uint32_t bb = __float_as_uint(a[i][K]) & 0x7fffffffu;
    if (bb > best) {
      best = bb;
      bi = i;
    }
  }
  pmin = min(pmin, best);
  perm |= (uint64_t)bi << (4 * K);
#pragma unroll
  for (int i = K + 1; i < 9; ++i) {
    const bool sw = (bi == i);
#pragma unroll
    for (int j = 0; j < 10; ++j) {
      const float t = a[K][j];
      a[K][j] = sw ? a[i][j] : t;
      a[i][j] = sw ? t : a[i][j];
    }
  }
  rinv[K] = 1.f / a[K][K];
#pragma unroll
  for (int i = K + 1; i < 9; ++i) {
    const float l = a[i][K] * rinv[K];
    a[i][K] = l;
#pragma unroll
    for (int j = K + 1; j < 10; ++j) a[i][j] = fmaf(-l, a[K][j], a[i][j]);
  }
}

// x = U^-1 (column 9 after the elimination), in FP32
__device__ __forceinline__ void back_sub_f(const float (&a)[9][10], const float (&rinv)[9], float (&x)[9]) {
#pragma unroll
  for (int k = 8; k >= 0; --k) {
    float t = a[k][9];
#pragma unroll
    for (int j = k + 1; j < 9; ++j) t = fmaf(-a[k][j], x[j], t);
    x[k] = t * rinv[k];
  }
}

// d = A^-1 r with the FP32 factors of P A = L U (whole rows were swapped, so
// L is in the final row order): all swaps first, then L, then U
__device__ __forceinline__ void lu_apply_f(const float (&a)[9][10], const float (&rinv)[9], uint64_t perm,
                                           float (&r)[9], float (&d)[9]) {
#pragma unroll
  for (int K = 0; K < 9; ++K) {
    const int bi = (int)((perm >> (4 * K)) & 15u);
    float rk = r[K];
#pragma unroll
    for (int i = K + 1; i < 9; ++i) {
      const bool sw = bi == i;
      const float t = r[i];
      r[i] = sw ? rk : t;
      rk = sw ? t : rk;
    }
    r[K] = rk;
  }
#pragma unroll
  for (int K = 0; K < 9; ++K)
#pragma unroll
    for (int i = K + 1; i < 9; ++i) r[i] = fmaf(-a[i][K], r[K], r[i]);
#pragma unroll
  for (int k = 8; k >= 0; --k) {
    float t = r[k];
#pragma unroll
    for (int j = k + 1; j < 9; ++j) t = fmaf(-a[k][j], d[j], t);
    d[k] = t * rinv[k];
  }
}

// closure_cell in FP64 as a separate function, so that the rare fallback does
// not add its registers to the mixed-precision path
static __device__ __noinline__ int closure_cell_fp64(const double *__restrict__ mc, double tc, const SolveParams &prm,
                                              double (&y)[9]) {
  return closure_cell<false>(mc, tc, prm, y);
}

// The closure of one cell from FP32-accurate moments by the mixed-precision
// solve; flags and Y as closure_cell (which it falls back to).
__device__ __forceinline__ int closure_cell_mixed(const double *__restrict__ mc, double tc, const SolveParams &prm,
                                                  double (&y)[9]) {
  int fl = 0;
  {
    double m[FP_NMOM];
#pragma unroll
    for (int k = 0; k < FP_NMOM; ++k) m[k] = mc[k];
    bool fin = finite_d(tc) && tc > 0.0;
#pragma unroll
    for (int k = 0; k < FP_NMOM; ++k) fin = fin && finite_d(m[k]);
    if (!fin) fl |= FP_FLAG_NONFINITE;
    if (m[kN] < (double)prm.min_particles) fl |= FP_FLAG_FEW;
    if (!(m[kTheta] > 0.0)) fl |= FP_FLAG_SINGULAR;
    if (!fl && m[kN] < (double)prm.min_regular) fl |= FP_FLAG_SINGULAR;
  }
  if (fl) return closure_cell_fp64(mc, tc, prm, y);  // the linear drift, as there
  // FP32 system from the moments rounded to FP32 (integer pipe)
  float af[9][10];
  {
    float mf[FP_NMOM];
#pragma unroll
    for (int k = 0; k < FP_NMOM; ++k) mf[k] = d2f_rn(mc[k]);
#pragma unroll
    for (int r = 0; r < 9; ++r)
#pragma unroll
      for (int c = 0; c < 10; ++c) af[r][c] = 0.f;
    assemble_emit(mf, d2f_rn(tc), d2f_rn(prm.eps2_hat), [&](int row, int col, float v) { af[row][col] = v; });
  }
  uint32_t amax = 0;
#pragma unroll
  for (int i = 0; i < 9; ++i)
#pragma unroll
    for (int j = 0; j < 9; ++j) amax = max(amax, __float_as_uint(af[i][j]) & 0x7fffffffu);
  float rinv[9], x0[9];
  uint64_t perm = 0;
  uint32_t pmin = 0x7f800000u;
  lu_step_f<0>(af, rinv, perm, pmin);
  lu_step_f<1>(af, rinv, perm, pmin);
  lu_step_f<2>(af, rinv, perm, pmin);
  lu_step_f<3>(af, rinv, perm, pmin);
  lu_step_f<4>(af, rinv, perm, pmin);
  lu_step_f<5>(af, rinv, perm, pmin);
  lu_step_f<6>(af, rinv, perm, pmin);
  lu_step_f<7>(af, rinv, perm, pmin);
  lu_step_f<8>(af, rinv, perm, pmin);
  const float accept = fmaxf(3e-3f, (float)(100.0 * prm.pivot_rtol));
  bool ok = amax < 0x7f800000u && __uint_as_float(pmin) > accept * __uint_as_float(amax);
  if (ok) {
    back_sub_f(af, rinv, x0);
    // residual b - A x0 in FP64 from the emitted entries
    double x[9], res[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      x[q] = f2d_exact(x0[q]);
      res[q] = 0.0;
    }
    {
      double m[FP_NMOM];
#pragma unroll
      for (int k = 0; k < FP_NMOM; ++k) m[k] = mc[k];
      assemble_emit(m, tc, prm.eps2_hat, [&](int row, int col, double v) {
        if (col == 9)
          res[row] += v;
        else
          res[row] = fma(-v, x[col], res[row]);
      });
    }
    float rf[9], d[9];
#pragma unroll
    for (int q = 0; q < 9; ++q) rf[q] = d2f_rn(res[q]);
    lu_apply_f(af, rinv, perm, rf, d);
    float dmax = 0.f, xmax = 0.f;
#pragma unroll
    for (int q = 0; q < 9; ++q) {
      dmax = fmaxf(dmax, fabsf(d[q]));
      xmax = fmaxf(xmax, fabsf(x0[q]));
      y[q] = x[q] + f2d_exact(d[q]);
    }
    ok = dmax <= 1e-4f * xmax;
#pragma unroll
    for (int q = 0; q < 9; ++q) ok = ok && finite_d(y[q]);
  }
  if (!ok) return closure_cell_fp64(mc, tc, prm, y);
  return 0;
}

// The closure of one cell by a group of 16 lanes (a half warp; all 32 lanes
// of the warp call this together, each half with its own cell, r = lane % 16).
// Lane r < 9 of the group holds row r of [A | r]: the pivot search is a
// max-reduction over the group, the swapped rows and the pivot row travel by
// shuffles, and each lane eliminates its own row; the back substitution
// broadcasts each y_k from lane k.  Every entry sees the operations of
// closure_cell in the same order (the same emitted expressions, multipliers
// a_iK * (1 / a_KK), fma updates, the sum over j ascending), so coefficients
// and flags are identical; what changes is the length of the dependent chain
// (FP64 instructions have a latency of about 64 cycles on this GPU, a
// division about 550), roughly halved, which is what a short fallback list
// waits for.  The division by each candidate pivot runs beside the pivot
// search.  The solve runs even for a flagged cell (the warp must stay
// converged for the shuffles) and its result is then discarded; valid =
// false makes the group a passenger: no loads, results meaningless.
__device__ __forceinline__ int closure_cell_group16(const double *__restrict__ mc, double tc, const SolveParams &prm,
                                                    bool valid, int r, double (&y)[9]) {
  constexpr unsigned kAll = 0xffffffffu;
  double m[FP_NMOM];
#pragma unroll
  for (int k = 0; k < FP_NMOM; ++k) m[k] = valid ? mc[k] : 1.0;
  int fl = 0;
  bool fin = finite_d(tc) && tc > 0.0;
#pragma unroll
  for (int k = 0; k < FP_NMOM; ++k) fin = fin && finite_d(m[k]);
  if (!fin) fl |= FP_FLAG_NONFINITE;
  if (m[kN] < (double)prm.min_particles) fl |= FP_FLAG_FEW;
  if (!(m[kTheta] > 0.0)) fl |= FP_FLAG_SINGULAR;
  if (!fl && m[kN] < (double)prm.min_regular) fl |= FP_FLAG_SINGULAR;

  double row[10];
#pragma unroll
  for (int col = 0; col < 10; ++col) row[col] = 0.0;
  assemble_emit(m, tc, prm.eps2_hat, [&](int rr, int col, double v) {
    if (rr == r) row[col] = v;
  });
  // max |A| over the group (rows 9.. are zero)
  uint64_t amax = 0;
#pragma unroll
  for (int j = 0; j < 9; ++j) amax = max(amax, abs_bits(row[j]));
#pragma unroll
  for (int o = 8; o >= 1; o >>= 1) amax = max(amax, (uint64_t)__shfl_xor_sync(kAll, (unsigned long long)amax, o, 16));
  const double amax_d = __longlong_as_double((long long)amax);
  int sfl = 0;
  if (!(amax_d > 0.0) || !finite_d(amax_d)) sfl = FP_FLAG_SINGULAR;
  const uint64_t thr = abs_bits(prm.pivot_rtol * amax_d);
  double rinv[9];
#pragma unroll
  for (int K = 0; K < 9; ++K) {
    const double inv_own = 1.0 / row[K];  // this lane's candidate reciprocal, beside the search
    // pivot: the largest |a_iK| over rows i >= K, the first such row on ties
    // (key 0 for lanes that are not candidates)
    const bool cand = r >= K && r < 9;
    uint64_t key = cand ? ((abs_bits(row[K]) << 1) | 1ull) : 0ull;
    int idx = r;
#pragma unroll
    for (int o = 8; o >= 1; o >>= 1) {
      const uint64_t k2 = __shfl_xor_sync(kAll, (unsigned long long)key, o, 16);
      const int i2 = __shfl_xor_sync(kAll, idx, o, 16);
      if (k2 > key || (k2 == key && i2 < idx)) {
        key = k2;
        idx = i2;
      }
    }
    const int bi = idx;
    if (!((key >> 1) > thr)) sfl = FP_FLAG_SINGULAR;
    // rows K and bi trade places; every lane reads the pivot row (old row bi)
    const int src = r == K ? bi : (r == bi ? K : r);
    double piv[10];
#pragma unroll
    for (int j = K; j < 10; ++j) {
      piv[j] = __shfl_sync(kAll, row[j], bi, 16);
      row[j] = __shfl_sync(kAll, row[j], src, 16);
    }
    rinv[K] = __shfl_sync(kAll, inv_own, bi, 16);
    if (r > K && r < 9) {
      const double l = row[K] * rinv[K];
#pragma unroll
      for (int j = K + 1; j < 10; ++j) row[j] = fma(-l, piv[j], row[j]);
    }
  }
#pragma unroll
  for (int k = 8; k >= 0; --k) {
    double s = row[9];
#pragma unroll
    for (int j = k + 1; j < 9; ++j) s = fma(-row[j], y[j], s);
    y[k] = __shfl_sync(kAll, s * rinv[k], k, 16);
  }
  if (!fl) {
    fl = sfl;
    if (!fl) {
#pragma unroll
      for (int q = 0; q < 9; ++q)
        if (!finite_d(y[q])) fl |= FP_FLAG_NONFINITE;
    }
  }
  if (fl) {
    const double c0 = (finite_d(tc) && tc > 0.0) ? -1.0 / tc : 0.0;
#pragma unroll
    for (int q = 0; q < 9; ++q) y[q] = 0.0;
    y[0] = c0;
    y[3] = c0;
    y[5] = c0;
  }
  return fl;
}

}  // namespace fpc
