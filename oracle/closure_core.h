/* oracle/closure_core.h -- test infrastructure only (see fp_oracle.c).
 *
 * The per-cell steps of the cubic Fokker-Planck closure written once for a
 * generic scalar type.  fp_oracle.c includes this file twice: with REAL =
 * double for the forward reference, and with REAL = double complex so that
 * complex-step differentiation gives exact derivatives of the very same
 * arithmetic (used as the reference gradient).
 *
 * Required macros: REAL, RE(x) (real part), SUFFIX(name) (name mangling).
 */

/* ---- moments of one cell (Sec. 3.6: u^(p)_{i1..in} = <|c|^p c_i1..c_in>) --
 * Two passes over the particles, every sum compensated (Neumaier):
 *   pass 1: U_i = <v_i>;
 *   pass 2: c = v - U and the central products listed in the slot table.
 * <.> is the plain mean over the N particles of the cell (the ensemble
 * average of Eq. update_alpha), i.e. 1/N, not 1/(N-1). */
typedef struct { REAL s, comp; } SUFFIX(nsum);

static inline void SUFFIX(nsum_add)(SUFFIX(nsum) * a, REAL x) {
  REAL t = a->s + x;
  if (fabs(RE(a->s)) >= fabs(RE(x)))
    a->comp += (a->s - t) + x;
  else
    a->comp += (x - t) + a->s;
  a->s = t;
}
static inline REAL SUFFIX(nsum_get)(const SUFFIX(nsum) * a) { return a->s + a->comp; }

static void SUFFIX(cell_moments)(const REAL *vx, const REAL *vy, const REAL *vz, int64_t n,
                                 REAL *m /* [OR_NMOM] */) {
  for (int k = 0; k < OR_NMOM; ++k) m[k] = 0;
  m[M_N] = (double)n;
  if (n <= 0) return;
  SUFFIX(nsum) su[3];
  memset(su, 0, sizeof su);
  for (int64_t p = 0; p < n; ++p) {
    SUFFIX(nsum_add)(&su[0], vx[p]);
    SUFFIX(nsum_add)(&su[1], vy[p]);
    SUFFIX(nsum_add)(&su[2], vz[p]);
  }
  REAL U[3];
  for (int i = 0; i < 3; ++i) U[i] = SUFFIX(nsum_get)(&su[i]) / (double)n;

  SUFFIX(nsum) s2[6], s3[10], s4[6], s5[3];
  memset(s2, 0, sizeof s2);
  memset(s3, 0, sizeof s3);
  memset(s4, 0, sizeof s4);
  memset(s5, 0, sizeof s5);
  for (int64_t p = 0; p < n; ++p) {
    REAL c[3] = {vx[p] - U[0], vy[p] - U[1], vz[p] - U[2]};
    REAL c2 = c[0] * c[0] + c[1] * c[1] + c[2] * c[2];
    for (int a = 0; a < 6; ++a) {
      REAL cc = c[SYM2_I[a]] * c[SYM2_J[a]];
      SUFFIX(nsum_add)(&s2[a], cc);          /* c_i c_j        */
      SUFFIX(nsum_add)(&s4[a], c2 * cc);     /* |c|^2 c_i c_j  */
    }
    for (int a = 0; a < 10; ++a)             /* c_i c_j c_k    */
      SUFFIX(nsum_add)(&s3[a], c[SYM3_I[a]] * c[SYM3_J[a]] * c[SYM3_K[a]]);
    for (int i = 0; i < 3; ++i)              /* |c|^4 c_i      */
      SUFFIX(nsum_add)(&s5[i], c2 * c2 * c[i]);
  }
  for (int i = 0; i < 3; ++i) m[M_U + i] = U[i];
  for (int a = 0; a < 6; ++a) m[M_U2 + a] = SUFFIX(nsum_get)(&s2[a]) / (double)n;
  for (int a = 0; a < 10; ++a) m[M_U3 + a] = SUFFIX(nsum_get)(&s3[a]) / (double)n;
  for (int a = 0; a < 6; ++a) m[M_W + a] = SUFFIX(nsum_get)(&s4[a]) / (double)n;
  for (int i = 0; i < 3; ++i) m[M_Z + i] = SUFFIX(nsum_get)(&s5[i]) / (double)n;
  /* theta = <c.c>/3 (Sec. 3.3: theta = kT/m) */
  m[M_THETA] = (m[M_U2 + 0] + m[M_U2 + 3] + m[M_U2 + 5]) / 3.0;
}

/* ---- assembly of the 9x9 system (Eq. system9x9, Table 1) ----------------
 * Unknowns Y = (C11, C12, C13, C22, C23, C33, G1, G2, G3) in the order of
 * Sec. 3.6, with C_ij = c^(1)_ij symmetric and G_i = c^(2)_i.
 *
 * Each row is the moment-matching condition Eq. moment_match for the cubic
 * drift Eq. cubic_drift.  For a test function psi(c) the FP production is
 *   <A_k d_k psi> + (1/2) <D_kl d_kl psi>,
 * with the isotropic diffusion D = (2 theta / tau) delta (the variance rate of
 * the noise sqrt(2 theta/tau) dW in Sec. 3.8).  The Boltzmann side is the
 * Maxwell-molecule relaxation with tau = 2 mu / p (Eq. tau): the stress
 * relaxes at p/mu = 2/tau and the heat flux at (2/3)(p/mu) = 4/(3 tau)
 * (Pr = 2/3, Sec. 2).
 *
 * Stress rows, psi = c_i c_j (i <= j):
 *   sum_k (C_ik u_kj + C_jk u_ki) + G_i b_j + G_j b_i
 *        = -(2/tau) u_ij + 2 eps^2 w_ij                     (V, W of Table 1)
 * Heat-flux rows, psi = c_i |c|^2:
 *   sum_l C_il b_l + 2 sum_kl C_kl u_ikl + G_i (s4 - 9 theta^2)
 *   + 2 sum_k G_k (w_ki - 3 theta u_ki)
 *        = -(4/(3 tau)) b_i + eps^2 (3 z_i - 3 theta b_i - 2 sum_k u_ik b_k)
 * where b_i = u_ikk = 2 q_i / rho, s4 = w_kk = <|c|^4> and, since C is
 * symmetric, a term in C_kl with k != l lands on the single unknown C_(kl).
 * eps^2 = eps2_hat / (tau theta) (the paper leaves the value open; this makes
 * eps2_hat dimensionless). */
static void SUFFIX(assemble)(const REAL *m, double tau, double eps2_hat, REAL A[9][9], REAL r[9]) {
  REAL u[3][3], u3[3][3][3], w[3][3], z[3], b[3];
  for (int i = 0; i < 3; ++i)
    for (int j = 0; j < 3; ++j) {
      u[i][j] = m[M_U2 + SYM2[i][j]];
      w[i][j] = m[M_W + SYM2[i][j]];
      for (int k = 0; k < 3; ++k) u3[i][j][k] = m[M_U3 + SYM3[i][j][k]];
    }
  for (int i = 0; i < 3; ++i) {
    z[i] = m[M_Z + i];
    b[i] = u3[i][0][0] + u3[i][1][1] + u3[i][2][2];
  }
  REAL theta = m[M_THETA];
  REAL s4 = w[0][0] + w[1][1] + w[2][2];
  REAL eps2 = eps2_hat / (tau * theta);
  for (int a = 0; a < 9; ++a) {
    r[a] = 0;
    for (int c = 0; c < 9; ++c) A[a][c] = 0;
  }
  /* stress rows */
  for (int row = 0; row < 6; ++row) {
    int i = SYM2_I[row], j = SYM2_J[row];
    for (int k = 0; k < 3; ++k) {
      A[row][SYM2[i][k]] += u[k][j];
      A[row][SYM2[j][k]] += u[k][i];
    }
    A[row][6 + i] += b[j];
    A[row][6 + j] += b[i];
    r[row] = -(2.0 / tau) * u[i][j] + 2.0 * eps2 * w[i][j];
  }
  /* heat-flux rows */
  for (int i = 0; i < 3; ++i) {
    int row = 6 + i;
    for (int l = 0; l < 3; ++l) A[row][SYM2[i][l]] += b[l];
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) A[row][SYM2[k][l]] += 2.0 * u3[i][k][l];
    A[row][6 + i] += s4 - 9.0 * theta * theta;
    for (int k = 0; k < 3; ++k) A[row][6 + k] += 2.0 * (w[k][i] - 3.0 * theta * u[k][i]);
    REAL ub = u[i][0] * b[0] + u[i][1] * b[1] + u[i][2] * b[2];
    r[row] = -(4.0 / (3.0 * tau)) * b[i] + eps2 * (3.0 * z[i] - 3.0 * theta * b[i] - 2.0 * ub);
  }
}

/* ---- Gaussian elimination with partial pivoting --------------------------
 * Row pivoting on the largest |a_ik| (first index on ties), elimination of
 * the augmented system, back substitution.  Returns 0, or OR_FLAG_SINGULAR
 * when a pivot is <= pivot_rtol * max_ij |A_ij| (the solution is then left
 * unset).  A and r are overwritten. */
static int SUFFIX(gauss_solve)(REAL A[9][9], REAL r[9], double pivot_rtol, REAL y[9],
                               double *min_pivot_ratio) {
  double amax = 0.0;
  for (int i = 0; i < 9; ++i)
    for (int j = 0; j < 9; ++j)
      if (fabs(RE(A[i][j])) > amax) amax = fabs(RE(A[i][j]));
  double minratio = INFINITY;
  if (!(amax > 0.0) || !isfinite(amax)) {
    if (min_pivot_ratio) *min_pivot_ratio = 0.0;
    return OR_FLAG_SINGULAR;
  }
  for (int k = 0; k < 9; ++k) {
    int p = k;
    for (int i = k + 1; i < 9; ++i)
      if (fabs(RE(A[i][k])) > fabs(RE(A[p][k]))) p = i;
    double ratio = fabs(RE(A[p][k])) / amax;
    if (ratio < minratio) minratio = ratio;
    if (!(ratio > pivot_rtol)) {
      if (min_pivot_ratio) *min_pivot_ratio = minratio;
      return OR_FLAG_SINGULAR;
    }
    if (p != k) {
      for (int j = 0; j < 9; ++j) {
        REAL t = A[k][j];
        A[k][j] = A[p][j];
        A[p][j] = t;
      }
      REAL t = r[k];
      r[k] = r[p];
      r[p] = t;
    }
    for (int i = k + 1; i < 9; ++i) {
      REAL l = A[i][k] / A[k][k];
      for (int j = k + 1; j < 9; ++j) A[i][j] -= l * A[k][j];
      A[i][k] = 0;
      r[i] -= l * r[k];
    }
  }
  for (int k = 8; k >= 0; --k) {
    REAL s = r[k];
    for (int j = k + 1; j < 9; ++j) s -= A[k][j] * y[j];
    y[k] = s / A[k][k];
  }
  if (min_pivot_ratio) *min_pivot_ratio = minratio;
  return 0;
}

/* ---- one cell of the closure -------------------------------------------- */
static int SUFFIX(closure_cell)(const REAL *m, double tau, const or_params *prm, REAL y[9],
                                double *min_pivot_ratio) {
  int flags = 0;
  int finite = isfinite(tau) && tau > 0.0;
  for (int k = 0; k < OR_NMOM; ++k) finite = finite && isfinite(RE(m[k]));
  if (!finite) flags |= OR_FLAG_NONFINITE;
  if (RE(m[M_N]) < (double)prm->min_particles) flags |= OR_FLAG_FEW;
  if (!(RE(m[M_THETA]) > 0.0)) flags |= OR_FLAG_SINGULAR;
  if (min_pivot_ratio) *min_pivot_ratio = 0.0;
  if (!flags) {
    REAL A[9][9], r[9];
    SUFFIX(assemble)(m, tau, prm->eps2_hat, A, r);
    flags |= SUFFIX(gauss_solve)(A, r, prm->pivot_rtol, y, min_pivot_ratio);
    if (!flags)
      for (int a = 0; a < 9; ++a)
        if (!isfinite(RE(y[a]))) flags |= OR_FLAG_NONFINITE;
  }
  if (flags) {
    /* linear (Langevin) drift, Eq. linear_drift: C = -I/tau, G = 0 */
    for (int a = 0; a < 9; ++a) y[a] = 0;
    double c0 = (isfinite(tau) && tau > 0.0) ? -1.0 / tau : 0.0;
    y[0] = c0;
    y[3] = c0;
    y[5] = c0;
  }
  return flags;
}
