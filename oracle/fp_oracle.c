/* oracle/fp_oracle.c
 *
 * TEST INFRASTRUCTURE ONLY.  A plain, slow, obviously-correct CPU reference
 * of the cubic Fokker-Planck moment closure and its particle velocity update,
 * in FP64, written from the paper's equations.  Only the tests, the smoke
 * check and the CPU-baseline and reference legs of the benchmark may load it;
 * the product path never does.  It shares no code, header or table with the CUDA library.
 *
 * What each entry point follows:
 *   oracle_moments            central moments, Sec. 3.6 (u^(p) definition)
 *   oracle_closure            Eq. system9x9 with Table 1 and the derived
 *                             heat-flux rows (closure_core.h), solved by
 *                             partial-pivot Gaussian elimination
 *   oracle_assemble           the 9x9 matrix and right-hand side alone
 *   oracle_closure_jacobian   dY/dm, by complex-step differentiation of the
 *                             same assembly + elimination
 *   oracle_closure_backward   vector-Jacobian products to the moments and to
 *                             the particle velocities (complex step through
 *                             the moments as well)
 *   oracle_velocity_update    Eq. update_vel with N from Eq. update_N and
 *                             alpha from Eq. update_alpha (Sec. 3.9-3.10)
 *   oracle_philox4x32_10      Philox4x32-10 (Salmon, Moraes, Dror, Shaw,
 *                             SC'11) -- the counter-based generator of the
 *                             noise variates xi
 *   oracle_normals            the inverse-distribution map of those words to xi
 *
 * Readings where the paper is silent (each stated where it is used):
 *   - diffusion D = 2 theta / tau (the noise amplitude of Sec. 3.8);
 *   - Table 1's V entries are second moments u_ij;
 *   - eps^2 = eps2_hat / (tau theta);
 *   - degenerate cells fall back to the linear drift C = -I/tau, G = 0.
 */
#include <complex.h>
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#define OR_NMOM 30
/* slots of the per-cell moment vector */
enum { M_N = 0, M_U = 1, M_THETA = 4, M_U2 = 5, M_U3 = 11, M_W = 21, M_Z = 27 };
enum {
  OR_FLAG_FEW = 1,
  OR_FLAG_SINGULAR = 2,
  OR_FLAG_NONFINITE = 4,
  OR_FLAG_ALPHA = 64
};

typedef struct {
  double eps2_hat;
  int32_t min_particles;
  double pivot_rtol;
} or_params;

/* symmetric index tables: (i,j) -> 0..5 in the order 11,12,13,22,23,33 and
 * (i,j,k) -> 0..9 in the order 111,112,113,122,123,133,222,223,233,333 */
static const int SYM2_I[6] = {0, 0, 0, 1, 1, 2};
static const int SYM2_J[6] = {0, 1, 2, 1, 2, 2};
static const int SYM2[3][3] = {{0, 1, 2}, {1, 3, 4}, {2, 4, 5}};
static const int SYM3_I[10] = {0, 0, 0, 0, 0, 0, 1, 1, 1, 2};
static const int SYM3_J[10] = {0, 0, 0, 1, 1, 2, 1, 1, 2, 2};
static const int SYM3_K[10] = {0, 1, 2, 1, 2, 2, 1, 2, 2, 2};
static int SYM3[3][3][3];
static int sym3_ready = 0;

static void init_sym3(void) {
  if (sym3_ready) return;
  for (int a = 0; a < 10; ++a) {
    int idx[3] = {SYM3_I[a], SYM3_J[a], SYM3_K[a]};
    /* every permutation of (i,j,k) maps to the same slot */
    int perms[6][3] = {{0, 1, 2}, {0, 2, 1}, {1, 0, 2}, {1, 2, 0}, {2, 0, 1}, {2, 1, 0}};
    for (int p = 0; p < 6; ++p) SYM3[idx[perms[p][0]]][idx[perms[p][1]]][idx[perms[p][2]]] = a;
  }
  sym3_ready = 1;
}

/* ---- real instantiation ---- */
#define REAL double
#define RE(x) (x)
#define SUFFIX(name) name##_d
#include "closure_core.h"
#undef REAL
#undef RE
#undef SUFFIX

/* ---- complex instantiation (complex-step derivatives) ---- */
#define REAL double complex
#define RE(x) creal(x)
#define SUFFIX(name) name##_z
#include "closure_core.h"
#undef REAL
#undef RE
#undef SUFFIX

/* complex step: d f / d x = Im f(x + i h) / h, exact to rounding for the
 * analytic arithmetic above (no subtractive cancellation) */
static const double CSTEP = 1e-40;

static or_params mkparams(double eps2_hat, int32_t min_particles, double pivot_rtol) {
  or_params p;
  p.eps2_hat = eps2_hat;
  p.min_particles = min_particles;
  p.pivot_rtol = pivot_rtol;
  return p;
}

/* ------------------------------------------------------------------------ */
int oracle_moments(const double *v, int64_t n_particles, const int64_t *offsets, int64_t n_cells,
                   double *moments) {
  init_sym3();
  const double *vx = v, *vy = v + n_particles, *vz = v + 2 * n_particles;
  for (int64_t c = 0; c < n_cells; ++c) {
    int64_t a = offsets[c], n = offsets[c + 1] - offsets[c];
    cell_moments_d(vx + a, vy + a, vz + a, n, moments + c * OR_NMOM);
  }
  return 0;
}

int oracle_assemble(const double *m, double tau, double eps2_hat, double *A81, double *r9) {
  init_sym3();
  double A[9][9], r[9];
  assemble_d(m, tau, eps2_hat, A, r);
  for (int i = 0; i < 9; ++i) {
    r9[i] = r[i];
    for (int j = 0; j < 9; ++j) A81[i * 9 + j] = A[i][j];
  }
  return 0;
}

/* Solve a given 9x9 system by the same elimination (rtol as in the closure).
 * Returns 0 or OR_FLAG_SINGULAR. */
int oracle_solve(const double *A81, const double *r9, double pivot_rtol, double *y9) {
  double A[9][9], r[9];
  for (int i = 0; i < 9; ++i) {
    r[i] = r9[i];
    for (int j = 0; j < 9; ++j) A[i][j] = A81[i * 9 + j];
  }
  return gauss_solve_d(A, r, pivot_rtol, y9, NULL);
}

/* Closure for every cell.  cond (nullable): infinity-norm condition number
 * of the assembled matrix (explicit inverse by the same elimination);
 * min_pivot (nullable): smallest |pivot| / max|A| met in the elimination. */
int oracle_closure(const double *moments, const double *tau, int64_t n_cells, double eps2_hat,
                   int32_t min_particles, double pivot_rtol, double *coeffs, int32_t *flags,
                   double *cond, double *min_pivot) {
  init_sym3();
  or_params prm = mkparams(eps2_hat, min_particles, pivot_rtol);
  for (int64_t c = 0; c < n_cells; ++c) {
    const double *m = moments + c * OR_NMOM;
    double mp = 0.0;
    flags[c] = closure_cell_d(m, tau[c], &prm, coeffs + c * 9, &mp);
    if (min_pivot) min_pivot[c] = mp;
    if (cond) {
      cond[c] = INFINITY;
      if (!flags[c]) {
        double A0[9][9], r0[9], inv[9][9];
        assemble_d(m, tau[c], eps2_hat, A0, r0);
        int ok = 1;
        for (int col = 0; col < 9 && ok; ++col) {
          double A[9][9], e[9], x[9];
          memcpy(A, A0, sizeof A);
          for (int i = 0; i < 9; ++i) e[i] = (i == col);
          ok = gauss_solve_d(A, e, 0.0, x, NULL) == 0;
          for (int i = 0; i < 9; ++i) inv[i][col] = x[i];
        }
        if (ok) {
          double na = 0, ni = 0;
          for (int i = 0; i < 9; ++i) {
            double sa = 0, si = 0;
            for (int j = 0; j < 9; ++j) {
              sa += fabs(A0[i][j]);
              si += fabs(inv[i][j]);
            }
            if (sa > na) na = sa;
            if (si > ni) ni = si;
          }
          cond[c] = na * ni;
        }
      }
    }
  }
  return 0;
}

/* dY/dm for one cell: J[a*OR_NMOM + k] = d Y_a / d m_k (zero columns for
 * flagged cells, whose coefficients do not depend on the moments). */
int oracle_closure_jacobian(const double *m, double tau, double eps2_hat, int32_t min_particles,
                            double pivot_rtol, double *J) {
  init_sym3();
  or_params prm = mkparams(eps2_hat, min_particles, pivot_rtol);
  double y0[9];
  int f0 = closure_cell_d(m, tau, &prm, y0, NULL);
  for (int k = 0; k < OR_NMOM; ++k) {
    double complex mz[OR_NMOM], yz[9];
    for (int q = 0; q < OR_NMOM; ++q) mz[q] = m[q];
    mz[k] += CSTEP * I;
    int f = closure_cell_z(mz, tau, &prm, yz, NULL);
    for (int a = 0; a < 9; ++a) J[a * OR_NMOM + k] = (f0 || f) ? 0.0 : cimag(yz[a]) / CSTEP;
  }
  return f0;
}

/* Reverse mode through the closure.
 *   grad_moments[c][k] = sum_a grad_coeffs[c][a] dY_a/dm_k  (+ grad_moments_in)
 *   grad_v[d][p]       = sum_k grad_moments[c][k] d m_k / d v_{d,p}
 * Both Jacobians come from complex steps of the forward arithmetic; the
 * second costs O(N^2) per cell, so callers pass small cells.  grad_moments,
 * grad_moments_in and grad_v are nullable. */
int oracle_closure_backward(const double *v, int64_t n_particles, const int64_t *offsets,
                            int64_t n_cells, const double *tau, double eps2_hat,
                            int32_t min_particles, double pivot_rtol, const double *moments,
                            const double *grad_coeffs, const double *grad_moments_in,
                            double *grad_moments, double *grad_v) {
  init_sym3();
  double *gm = (double *)malloc(sizeof(double) * OR_NMOM);
  double J[9 * OR_NMOM];
  for (int64_t c = 0; c < n_cells; ++c) {
    const double *m = moments + c * OR_NMOM;
    oracle_closure_jacobian(m, tau[c], eps2_hat, min_particles, pivot_rtol, J);
    for (int k = 0; k < OR_NMOM; ++k) {
      double s = grad_moments_in ? grad_moments_in[c * OR_NMOM + k] : 0.0;
      for (int a = 0; a < 9; ++a) s += grad_coeffs[c * 9 + a] * J[a * OR_NMOM + k];
      gm[k] = s;
      if (grad_moments) grad_moments[c * OR_NMOM + k] = s;
    }
    if (!grad_v) continue;
    int64_t a0 = offsets[c], n = offsets[c + 1] - offsets[c];
    if (n <= 0) continue;
    double complex *cv = (double complex *)malloc(sizeof(double complex) * 3 * (size_t)n);
    for (int d = 0; d < 3; ++d)
      for (int64_t p = 0; p < n; ++p) cv[d * n + p] = v[d * n_particles + a0 + p];
    for (int d = 0; d < 3; ++d)
      for (int64_t p = 0; p < n; ++p) {
        double complex mz[OR_NMOM];
        cv[d * n + p] += CSTEP * I;
        cell_moments_z(cv, cv + n, cv + 2 * n, n, mz);
        cv[d * n + p] = creal(cv[d * n + p]);
        double s = 0.0;
        for (int k = 0; k < OR_NMOM; ++k) s += gm[k] * (cimag(mz[k]) / CSTEP);
        grad_v[d * n_particles + a0 + p] = s;
      }
    free(cv);
  }
  free(gm);
  return 0;
}

/* ---- Philox4x32-10 (Salmon et al., SC'11) ------------------------------- *
 * Ten rounds of: (hi0,lo0) = M0 * x0, (hi1,lo1) = M1 * x2 (32x32 -> 64),
 * x = (hi1 ^ x1 ^ k0, lo1, hi0 ^ x3 ^ k1, lo0); the key is bumped by the
 * Weyl constants (W0, W1) between rounds. */
void oracle_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
  uint32_t x[4] = {ctr_in[0], ctr_in[1], ctr_in[2], ctr_in[3]};
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) {
      k0 += W0;
      k1 += W1;
    }
    uint64_t p0 = (uint64_t)M0 * x[0], p1 = (uint64_t)M1 * x[2];
    uint32_t hi0 = (uint32_t)(p0 >> 32), lo0 = (uint32_t)p0;
    uint32_t hi1 = (uint32_t)(p1 >> 32), lo1 = (uint32_t)p1;
    uint32_t y0 = hi1 ^ x[1] ^ k0, y1 = lo1, y2 = hi0 ^ x[3] ^ k1, y3 = lo0;
    x[0] = y0;
    x[1] = y1;
    x[2] = y2;
    x[3] = y3;
  }
  for (int i = 0; i < 4; ++i) out[i] = x[i];
}

/* Inverse of the standard normal distribution function
 * Phi(x) = erfc(-x / sqrt 2) / 2 for u in (0, 1): bisection on [-40, 40] to
 * a bracket of 1e-9, then Newton steps with the density
 * phi(x) = exp(-x^2 / 2) / sqrt(2 pi). */
static double inv_normal_cdf(double u) {
  const double rs2 = 0.70710678118654752440084436210485;   /* 1 / sqrt 2 */
  const double rs2pi = 0.39894228040143267793994605993438; /* 1 / sqrt(2 pi) */
  double lo = -40.0, hi = 40.0;
  for (int it = 0; it < 60 && hi - lo > 1e-9; ++it) {
    const double mid = 0.5 * (lo + hi);
    if (0.5 * erfc(-mid * rs2) < u)
      lo = mid;
    else
      hi = mid;
  }
  double x = 0.5 * (lo + hi);
  for (int it = 0; it < 3; ++it) x -= (0.5 * erfc(-x * rs2) - u) / (rs2pi * exp(-0.5 * x * x));
  return x;
}

/* The noise variates of particle p at a given step.  The variates of a step
 * are one stream of 32-bit words: word j is word (j mod 4) of the
 * Philox4x32-10 block with key (seed_lo, seed_hi) on counter
 * (floor(j/4)_lo, floor(j/4)_hi, step_lo, step_hi), and particle p takes words
 * 3p, 3p + 1, 3p + 2 (four consecutive particles use three whole blocks).
 * A word w gives the uniform u = (floor(w / 2^9) + 1/2) 2^-23 in (0, 1)
 * (exact in FP32 as well) and xi = Phi^-1(u), the inverse standard normal
 * distribution function.  Evaluated here in FP64. */
static void particle_normals(uint64_t seed, uint64_t step, uint64_t p, double xi[3]) {
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  uint64_t have = ~(uint64_t)0;  /* the block whose words w holds */
  uint32_t w[4];
  for (int i = 0; i < 3; ++i) {
    const uint64_t j = 3 * p + (uint64_t)i, blk = j >> 2;
    if (blk != have) {
      uint32_t ctr[4] = {(uint32_t)blk, (uint32_t)(blk >> 32), (uint32_t)step, (uint32_t)(step >> 32)};
      oracle_philox4x32_10(ctr, key, w);
      have = blk;
    }
    xi[i] = inv_normal_cdf(((double)(w[j & 3] >> 9) + 0.5) * (1.0 / 8388608.0));
  }
}

int oracle_normals(int64_t n, int64_t first_index, uint64_t seed, uint64_t step, double *xi) {
  for (int64_t p = 0; p < n; ++p) {
    double x[3];
    particle_normals(seed, step, (uint64_t)(first_index + p), x);
    for (int d = 0; d < 3; ++d) xi[d * n + p] = x[d];
  }
  return 0;
}

/* ---- velocity update, Sec. 3.9-3.10 ------------------------------------ *
 * For every particle of a cell (M' = M - U^n, a = exp(-dt/tau)):
 *   N_i = (C_ij + delta_ij/tau) M'_j + G_i (|M'|^2 - 3 theta)
 *         - eps^2 (M'_i |M'|^2 - b_i)                        (Eq. update_N,
 *         with 2 q_i / rho = b_i = <c_i |c|^2>)
 *   alpha^2 = 1 + tau/(3 theta) [ tau (1-a)^2 <N.N> + 2 (a - a^2) <M'.N> ]
 *                                                            (Eq. update_alpha)
 *   M^{n+1} = (1/alpha) [ M' a + (1-a) tau N + sqrt(theta (1-a^2)) xi ] + U
 *                                                            (Eq. update_vel)
 * Cells whose closure fell back to the linear drift (flags 1|2|4 on input)
 * take N = 0 and alpha = 1 (the exact Ornstein-Uhlenbeck step of the linear
 * model).  alpha^2 <= 0 or non-finite sets OR_FLAG_ALPHA and alpha = 1.
 * xi: caller's variates [3][n_particles], or NULL for the Philox ones.  v is
 * updated in place. */
int oracle_velocity_update(double *v, int64_t n_particles, const int64_t *offsets, int64_t n_cells,
                           const double *moments, const double *coeffs, const double *tau,
                           double dt, double eps2_hat, const double *xi, uint64_t seed,
                           uint64_t step, double *alpha_out, int32_t *flags) {
  init_sym3();
  double *vx = v, *vy = v + n_particles, *vz = v + 2 * n_particles;
  for (int64_t c = 0; c < n_cells; ++c) {
    const double *m = moments + c * OR_NMOM;
    const double *Y = coeffs + c * 9;
    int64_t a0 = offsets[c], n = offsets[c + 1] - offsets[c];
    double tc = tau[c], th = m[M_THETA];
    double U[3] = {m[M_U], m[M_U + 1], m[M_U + 2]};
    double Cm[3][3], G[3] = {Y[6], Y[7], Y[8]}, b[3];
    for (int i = 0; i < 3; ++i)
      for (int j = 0; j < 3; ++j) Cm[i][j] = Y[SYM2[i][j]] + (i == j ? 1.0 / tc : 0.0);
    for (int i = 0; i < 3; ++i)
      b[i] = m[M_U3 + SYM3[i][0][0]] + m[M_U3 + SYM3[i][1][1]] + m[M_U3 + SYM3[i][2][2]];
    double eps2 = eps2_hat / (tc * th);
    int linear = (flags[c] & (OR_FLAG_FEW | OR_FLAG_SINGULAR | OR_FLAG_NONFINITE)) != 0;
    double a = exp(-dt / tc);
    /* first pass: <N.N> and <M'.N> (compensated sums) */
    nsum_d snn = {0, 0}, smn = {0, 0};
    for (int64_t p = 0; p < n && !linear; ++p) {
      double Mp[3] = {vx[a0 + p] - U[0], vy[a0 + p] - U[1], vz[a0 + p] - U[2]};
      double m2 = Mp[0] * Mp[0] + Mp[1] * Mp[1] + Mp[2] * Mp[2];
      double N[3];
      for (int i = 0; i < 3; ++i)
        N[i] = Cm[i][0] * Mp[0] + Cm[i][1] * Mp[1] + Cm[i][2] * Mp[2] + G[i] * (m2 - 3.0 * th) -
               eps2 * (Mp[i] * m2 - b[i]);
      nsum_add_d(&snn, N[0] * N[0] + N[1] * N[1] + N[2] * N[2]);
      nsum_add_d(&smn, Mp[0] * N[0] + Mp[1] * N[1] + Mp[2] * N[2]);
    }
    double alpha = 1.0;
    if (!linear && n > 0) {
      double nn = nsum_get_d(&snn) / (double)n, mn = nsum_get_d(&smn) / (double)n;
      double alpha2 = 1.0 + tc / (3.0 * th) * (tc * (1.0 - a) * (1.0 - a) * nn + 2.0 * (a - a * a) * mn);
      if (alpha2 > 0.0 && isfinite(alpha2))
        alpha = sqrt(alpha2);
      else
        flags[c] |= OR_FLAG_ALPHA;
    }
    if (alpha_out) alpha_out[c] = alpha;
    double noise = sqrt(th * (1.0 - a * a));
    /* second pass: the update itself */
    for (int64_t p = 0; p < n; ++p) {
      double Mp[3] = {vx[a0 + p] - U[0], vy[a0 + p] - U[1], vz[a0 + p] - U[2]};
      double m2 = Mp[0] * Mp[0] + Mp[1] * Mp[1] + Mp[2] * Mp[2];
      double N[3] = {0, 0, 0};
      if (!linear)
        for (int i = 0; i < 3; ++i)
          N[i] = Cm[i][0] * Mp[0] + Cm[i][1] * Mp[1] + Cm[i][2] * Mp[2] + G[i] * (m2 - 3.0 * th) -
                 eps2 * (Mp[i] * m2 - b[i]);
      double x[3];
      if (xi) {
        for (int d = 0; d < 3; ++d) x[d] = xi[d * n_particles + a0 + p];
      } else {
        particle_normals(seed, step, (uint64_t)(a0 + p), x);
      }
      double out[3];
      for (int i = 0; i < 3; ++i)
        out[i] = (Mp[i] * a + (1.0 - a) * tc * N[i] + noise * x[i]) / alpha + U[i];
      vx[a0 + p] = out[0];
      vy[a0 + p] = out[1];
      vz[a0 + p] = out[2];
    }
  }
  return 0;
}
