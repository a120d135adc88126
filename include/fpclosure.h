/* fpclosure.h -- C ABI of the GB300 (sm_103a) cubic Fokker-Planck moment
 * closure library, libfpclosure.so.
 *
 * The closure (paper Sec. 3.4-3.7): for every cell, the particles' central
 * velocity moments up to fifth order are gathered, the 9x9 moment-matching
 * system of Eq. system9x9 (Table 1 and its heat-flux rows) is assembled, and
 * a partial-pivot solve gives the drift coefficients
 *     Y = (C11, C12, C13, C22, C23, C33, G1, G2, G3)
 * of the cubic drift Eq. cubic_drift (C_ij = c^(1)_ij, G_i = c^(2)_i).
 *
 * Conventions shared by every call
 * --------------------------------
 * - Array pointers are DEVICE pointers owned by the caller; the library keeps
 *   no reference after the call returns and allocates no device memory.
 *   Scratch space comes from a caller-provided workspace sized by
 *   fp_workspace_bytes() (a NULL workspace is allowed when the query says 0).
 * - Calls are asynchronous on the caller's stream (a cudaStream_t passed as
 *   fp_stream_t; NULL = legacy default stream).  The return code reports
 *   argument validation and launch errors only; numerical problems of a cell
 *   are reported in its flags, never as a call error.
 * - Velocities are structure-of-arrays: v[0..n) = x, v[n..2n) = y,
 *   v[2n..3n) = z, sorted by cell.  cell_offsets[n_cells+1] (int64) is
 *   non-decreasing with cell_offsets[0] = 0 and cell_offsets[n_cells] = n;
 *   cell c owns particles [cell_offsets[c], cell_offsets[c+1]).  Offsets live
 *   on the device and are not checked by the host.
 * - Moment vector of a cell (FP_NMOM = 30 doubles, row-major [n_cells][30]):
 *     0      N (particle count)
 *     1..3   U_i = <v_i>
 *     4      theta = <c.c>/3, c = v - U
 *     5..10  u_ij = <c_i c_j>            ij = 11,12,13,22,23,33
 *     11..20 u_ijk = <c_i c_j c_k>       ijk = 111,112,113,122,123,133,
 *                                               222,223,233,333
 *     21..26 w_ij = <|c|^2 c_i c_j>      ij as above
 *     27..29 z_i = <|c|^4 c_i>
 *   (<.> is the mean over the cell's N particles; the u^(p) of Sec. 3.6).
 * - Readings of the paper used throughout: the diffusion is D = 2 theta/tau
 *   (the noise amplitude of Sec. 3.8); eps^2 = eps2_hat / (tau theta);
 *   a cell that cannot be closed falls back to the linear drift of
 *   Eq. linear_drift, C = -I/tau, G = 0.
 */
#ifndef FPCLOSURE_H
#define FPCLOSURE_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct CUstream_st *fp_stream_t; /* same type as cudaStream_t */

#define FP_NMOM 30
#define FP_LU_STRIDE 82  /* entries per cell of stored factors (fp_closure_solve) */
#define FP_LU_DOUBLES(n) ((((n) + 31) / 32) * 32 * FP_LU_STRIDE) /* buffer size, doubles */
#define FP_NCOEF 9

/* return codes */
enum {
  FP_OK = 0,
  FP_ERR_ARG = -1,         /* invalid argument (size, pointer, enum)        */
  FP_ERR_CUDA = -2,        /* a CUDA launch or runtime call failed           */
  FP_ERR_WORKSPACE = -3,   /* workspace missing or smaller than required     */
  FP_ERR_UNSUPPORTED = -4  /* valid request the library does not implement  */
};

/* particle velocity storage type */
enum { FP_V_F32 = 0, FP_V_F64 = 1 };

/* moment precision:
 * FP_PREC_FP64          moments accumulated in FP64 from the given velocities
 * FP_PREC_FP32_MOMENTS  moments accumulated in FP32 with compensated
 *                       (two-sum) combination of partial sums and written in
 *                       FP64.  FP32 velocities in 16-byte aligned arrays take
 *                       one pass: velocities shifted by the mean of a
 *                       strided subset of up to 8 particles of the cell and
 *                       scaled by a power of two, the shifted sums turned
 *                       into central moments by the binomial expansion of
 *                       the shift (FP32); other inputs take two passes
 *                       (the cell mean, then sums centred on it and scaled
 *                       by a power of two ~1/sqrt(theta)).
 * The 9x9 system is assembled in FP64 in both modes and solved with partial
 * pivoting; the FP64 mode, and any call that keeps the factors for the
 * adjoint, eliminates in FP64.  Without factors the FP32-moment mode factors
 * the system in FP32 and refines the solution once against the FP64 residual
 * b - A x (agreeing with the FP64 elimination to ~1e-9 relative, far below
 * the moments' own error); cells whose FP32 pivots fall below
 * max(3e-3, 100 pivot_rtol) of max|A|, or whose correction exceeds 1e-4 of
 * the solution, are eliminated in FP64 instead, and that elimination decides
 * their flags.  With FP32
 * moments (relative error ~1e-7) a pivot below ~1e-6 max|A| cannot be told
 * from zero, so that mode flags a cell singular when a pivot is
 * <= max(pivot_rtol, FP_FP32_PIVOT_FLOOR) * max|A|.  A cell of four
 * particles gives a singular 9x9 system whatever its velocities (its pivot
 * ratio is ~1e-15 with exact moments), but with FP32 moments its smallest
 * pivot carries the moment noise (1e-7..1e-5 of max|A|), so that mode flags
 * cells with fewer than FP_FP32_MIN_REGULAR particles singular directly. */
#define FP_FP32_PIVOT_FLOOR 1e-6
#define FP_FP32_MIN_REGULAR 5
enum { FP_PREC_FP64 = 0, FP_PREC_FP32_MOMENTS = 1 };

/* per-cell flag bits */
enum {
  FP_FLAG_FEW = 1,        /* N < min_particles: linear-drift fallback        */
  FP_FLAG_SINGULAR = 2,   /* theta <= 0 or a pivot <= pivot_rtol max|A|      */
  FP_FLAG_NONFINITE = 4,  /* non-finite moment, tau or solution              */
  FP_FLAG_RANGE = 8,      /* surrogate feature outside its training box      */
  FP_FLAG_ENERGY = 16,    /* surrogate energy residual above tolerance       */
  FP_FLAG_FALLBACK = 32,  /* surrogate cell recomputed by the exact closure  */
  FP_FLAG_ALPHA = 64      /* velocity update: alpha^2 <= 0, alpha set to 1   */
};

typedef struct {
  double eps2_hat;          /* dimensionless cubic stabiliser (Sec. 3.4)     */
  int32_t min_particles;    /* cells with fewer particles take the fallback  */
  double pivot_rtol;        /* singular if |pivot| <= pivot_rtol * max|A|    */
  double surr_energy_tol;   /* surrogate: max |energy residual| accepted     */
  double surr_range_margin; /* surrogate: feature box widened by this margin
                               (in standard deviations)                      */
  uint64_t particle_offset; /* velocity update: the Philox counter of particle
                               i of a call is particle_offset + i; a run that
                               splits the particles over several calls or GPUs
                               passes each slice's first global index and draws
                               the variates of the unsplit run                */
} fp_params;

/* Defaults: eps2_hat 1e-3, min_particles 4, pivot_rtol 1e-13,
 * surr_energy_tol 0.05, surr_range_margin 0.5, particle_offset 0. */
void fp_default_params(fp_params *p);

/* Text for a return code; text of the last error of the calling thread. */
const char *fp_status_string(int status);
const char *fp_last_error(void);
int fp_version(void);

/* Workspace (bytes) that fp_closure_exact needs for n_cells cells when
 * moments_out is NULL (the moments are then kept in the workspace); 0 when
 * the caller provides moments_out.  Aligned to 256 bytes. */
size_t fp_workspace_bytes(int64_t n_cells, int64_t n_particles, int prec, int moments_out_given);

/* The exact closure (Sec. 3.6-3.7, Eq. system9x9).
 *   v             [3][n_particles], FP_V_F32 or FP_V_F64 (v_dtype)
 *   cell_offsets  [n_cells+1] int64
 *   tau           [n_cells] collision time tau = 2 mu / p (Eq. tau) per cell
 *   p             host pointer to parameters (NULL = defaults)
 *   prec          FP_PREC_FP64 or FP_PREC_FP32_MOMENTS
 *   moments_out   [n_cells][FP_NMOM] f64, or NULL (then ws is used)
 *   coeffs_out    [n_cells][9] f64
 *   flags_out     [n_cells] int32 (FP_FLAG_FEW | FP_FLAG_SINGULAR |
 *                 FP_FLAG_NONFINITE; flagged cells hold C = -I/tau, G = 0)
 *   ws, ws_bytes  device workspace, >= fp_workspace_bytes(...)
 * n_cells = 0 is a no-op; n_particles = 0 with n_cells > 0 gives empty
 * (FP_FLAG_FEW) cells. */
int fp_closure_exact(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                     int64_t n_cells, const double *tau, const fp_params *p, int prec,
                     double *moments_out, double *coeffs_out, int32_t *flags_out, void *ws,
                     size_t ws_bytes, fp_stream_t stream);

/* The two halves of fp_closure_exact, for callers that need the moments alone
 * (the surrogate's features, the velocity update) or hold them already.
 *
 * fp_moments: the per-cell moment vectors (Sec. 3.6), same arguments and
 * precision modes as fp_closure_exact; moments_out [n_cells][FP_NMOM] f64
 * required; m6_out [n_cells] f64 or NULL receives <|c|^6>, the sixth central
 * moment of the peculiar speed, which lets fp_velocity_update evaluate the
 * cell averages of Eq. update_alpha from moments (one particle pass).  No
 * workspace. */
int fp_moments(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets, int64_t n_cells,
               int prec, double *moments_out, double *m6_out, fp_stream_t stream);

/* fp_closure_solve: assembly of Eq. system9x9 from given moment vectors and
 * the pivoted solve (FP64, or with FP32 moments and no lu_out the
 * mixed-precision solve described above), one thread per cell.  moments [n_cells][FP_NMOM]
 * f64 (as fp_moments writes them), tau [n_cells]; prec = the precision the
 * moments were gathered in (selects the singularity threshold); outputs as
 * in fp_closure_exact.  lu_out: FP_LU_DOUBLES(n_cells) f64 or NULL; if
 * given, every unflagged cell's factors P A = L U of the elimination are
 * stored there for fp_closure_backward: FP_LU_STRIDE entries per cell (the
 * row-major 9 x 9 with L below the diagonal, the reciprocal pivots on it and
 * U above it, then the row swaps, 4 bits per step, in the bits of a double),
 * tiled by 32 cells so a warp's accesses coalesce: entry k of cell c (counted
 * from the call's first cell) at lu_out[(c / 32) * 32 * FP_LU_STRIDE + 32 k +
 * c % 32].  Entries of flagged cells are left as they were.  No workspace. */
int fp_closure_solve(const double *moments, const double *tau, int64_t n_cells, const fp_params *p, int prec,
                     double *coeffs_out, int32_t *flags_out, double *lu_out, fp_stream_t stream);

/* fp_velocity_update: one collision step of the particle velocities with the
 * mixed Ornstein-Uhlenbeck / Euler scheme (paper Sec. 3.9-3.10):
 *   N_i = (C_ij + delta_ij / tau) M'_j + G_i (|M'|^2 - 3 theta)
 *         - eps^2 (M'_i |M'|^2 - b_i)                        (Eq. update_N)
 *   alpha^2 = 1 + tau / (3 theta) [tau (1-a)^2 <N.N> + 2 (a - a^2) <M'.N>]
 *                                                            (Eq. update_alpha)
 *   M^{n+1} = (M' a + (1-a) tau N + sqrt(theta (1-a^2)) xi) / alpha + U
 *                                                            (Eq. update_vel)
 * with M' = M - U, a = exp(-dt/tau), b_i = <c_i |c|^2> = 2 q_i / rho and the
 * cell averages <.> over the cell's particles.
 *   v            [3][n_particles] f32 or f64, the velocities M^n; FP32
 *                velocities are updated in FP32 arithmetic, FP64 in FP64
 *   v_out        [3][n_particles] of v's dtype receiving M^{n+1}, or NULL (or
 *                v itself) to update v in place; a distinct v_out must not
 *                overlap v.  Writing out of place lets a caller keep M^n for
 *                a concurrent reader (e.g. the adjoint's particle pass)
 *   moments      [n_cells][FP_NMOM] of the same velocities (U, theta, u_ijk)
 *   m6           [n_cells] <|c|^6> of the same velocities (fp_moments), or
 *                NULL.  Given, <N.N> and <M'.N> are evaluated from the moments
 *                in closed form (N is a cubic in M' = c, so <N.N> needs
 *                moments up to the sixth) and the particles are read once;
 *                NULL, they are summed over the particles in a first pass.
 *                Both are the same cell averages up to rounding.
 *   coeffs       [n_cells][9] from the closure
 *   tau          [n_cells]; dt the time step
 *   p            eps2_hat is read (NULL = defaults)
 *   xi           [3][n_particles] standard normals of v's dtype, or NULL: then
 *                xi comes from Philox4x32-10 with key (seed lo, seed hi) on
 *                counter (particle index lo, hi, step lo, hi), the particle
 *                index counted from p->particle_offset; words 0..2 map to
 *                uniforms (floor(w / 2^9) + 1/2) 2^-23 and xi_k is the inverse
 *                standard normal distribution function of u_k, in FP32
 *                (a fitted approximation: |error| <= 1.3e-6 over all words)
 *   alpha_out    [n_cells] f64 or NULL
 *   flags        [n_cells] int32 IN/OUT: cells carrying FP_FLAG_FEW,
 *                FP_FLAG_SINGULAR or FP_FLAG_NONFINITE take the exact OU step
 *                of the linear model (N = 0, alpha = 1); alpha^2 <= 0 or
 *                non-finite sets FP_FLAG_ALPHA and alpha = 1.
 * No workspace. */
int fp_velocity_update(void *v, void *v_out, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                       int64_t n_cells, const double *moments, const double *m6, const double *coeffs,
                       const double *tau, double dt, const fp_params *p, const void *xi, uint64_t seed,
                       uint64_t step, double *alpha_out, int32_t *flags, fp_stream_t stream);

/* fp_closure_backward: the adjoint of fp_closure_exact (not in the paper; the
 * closure of Eq. system9x9 differentiated as an implicit function).  With
 * F(m, Y) = A(m) Y - r(m) = 0 and a loss gradient gY = dL/dY per cell:
 *   lambda = A^-T gY                    (two triangular solves with the
 *                                        forward's factors when lu is given,
 *                                        else a pivoted elimination of A^T)
 *   grad_moments = -(dF/dm)^T lambda + grad_moments_in
 *   grad_v[p] = (1/N) sum_k grad_moments_k (grad psi_k(c_p) - <grad psi_k>)
 *               + grad_moments_U / N    (c_p = v_p - U, m_k = <psi_k(c)>)
 * so the velocity gradient carries every moment gradient, including the
 * caller's grad_moments_in (for losses that also read the moments).
 *   v, cell_offsets, tau  as in fp_closure_exact (v only read when grad_v)
 *   p                     eps2_hat is read (NULL = defaults)
 *   moments, coeffs, flags  the forward outputs for the same v
 *   lu                    FP_LU_DOUBLES(n_cells) from fp_closure_solve for
 *                         the same moments and first cell, or NULL
 *                         (recomputed)
 *   grad_coeffs           [n_cells][9]
 *   grad_moments_in       [n_cells][FP_NMOM] or NULL (= 0)
 *   grad_moments          [n_cells][FP_NMOM] out, or NULL (then kept in ws)
 *   grad_v                [3][n_particles] out, v's dtype, or NULL; FP32
 *                         velocities get an FP32 particle pass, FP64 an FP64
 *                         one; the per-cell part is FP64 in both
 *   ws, ws_bytes          >= fp_workspace_bytes(n_cells, n_particles, prec,
 *                         grad_moments != NULL) when grad_v is requested
 * Cells flagged FP_FLAG_FEW | FP_FLAG_SINGULAR | FP_FLAG_NONFINITE hold the
 * constant linear drift: their coefficient gradient contributes nothing. */
int fp_closure_backward(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                        int64_t n_cells, const double *tau, const fp_params *p, const double *moments,
                        const double *coeffs, const int32_t *flags, const double *lu, const double *grad_coeffs,
                        const double *grad_moments_in, double *grad_moments, void *grad_v, void *ws,
                        size_t ws_bytes, fp_stream_t stream);

/* ---------------------------------------------------------------------------
 * The learned closure (the paper's neural surrogate, Sec. 4, Alg. 2): a small
 * MLP maps a cell's normalised moments to its drift coefficients; flagged
 * cells fall back to the exact closure.
 *
 * Features: the 25 moments of w = c / sqrt(theta): u_ij / theta (6),
 * u_ijk / theta^1.5 (10), w_ij / theta^2 (6), z_i / theta^2.5 (3), in the
 * slot order of the moment vector, standardised with (x_mu, x_sigma),
 * rounded to BF16 and zero padded to 32.  Targets: the dimensionless
 * coefficients t = (tau C_11, tau C_12, tau C_13, tau C_22, tau C_23,
 * tau C_33, tau sqrt(theta) G_1..3) standardised with (y_mu, y_sigma); the
 * cubic-FP system is invariant under c -> c / sqrt(theta), so t depends on
 * the features alone (for the eps2_hat the network was trained with).
 * Network: Linear(32,128) SiLU, 3 x [Linear(128,128) SiLU], Linear(128,16)
 * (outputs 9..15 unused); BF16 weights and activations, FP32 accumulation.
 * ------------------------------------------------------------------------- */
typedef struct {
  const void *W[5];             /* device, BF16 row-major [out][in], each
                                   16-byte aligned: 128x32, 128x128,
                                   128x128, 128x128, 16x128                  */
  const float *b[5];            /* device, FP32 [128] x 4, [16]              */
  const float *x_mu, *x_sigma;  /* device, FP32 [32] (padding: 0, 1)         */
  const float *y_mu, *y_sigma;  /* device, FP32 [16] (padding: 0, 1)         */
  const float *x_min, *x_max;   /* device, FP32 [32]: raw-feature box of the
                                   training set                              */
  int32_t in_dim, hidden, depth, out_dim; /* must be 32, 128, 4, 16          */
  double eps2_hat;              /* eps2_hat of the training targets          */
} fp_mlp;

/* Flat FP32 parameter vector used by training: W1 | b1 | W2 | b2 | W3 | b3 |
 * W4 | b4 | W5 | b5 (row-major W).  which = 0 for W_layer, 1 for b_layer;
 * layer = 0..4. */
int64_t fp_mlp_param_count(void);
int64_t fp_mlp_param_offset(int which, int layer);

/* fp_surrogate_training_rows: what training of the learned closure reads for
 * every cell (Sec. 4, Phases 1-2: the network is fit to coefficients of the
 * exact closure), computed by the arithmetic of the inference kernels so that
 * training and inference see the same inputs:
 *   raw_out     [n_cells][32] FP32 unstandardised network inputs, zero padded:
 *               lite_inputs = 0: the 25 normalised moments of `moments`, as
 *               fp_surrogate_features forms them before standardising;
 *               lite_inputs = 1: the 16 LITE inputs of `lite` and tau, as
 *               fp_surrogate_lite_features forms them
 *   target_out  [n_cells][16] FP32 dimensionless targets (tau C, tau sqrt(theta) G)
 *               of the coefficients `coeffs` [n_cells][9], zero padded
 *   aux_out     [n_cells][16] FP32 the loss's auxiliary moments (u^_ij (6),
 *               b^_i = u^_ikk (3), s4^ = w^_kk, zeros) of `moments`
 * moments [n_cells][FP_NMOM] is read unless only raw_out of LITE inputs is
 * wanted; lite [n_cells][FP_NLITE] only for lite_inputs = 1; coeffs only for
 * target_out.  Any output may be NULL; outputs 16-byte aligned.  Device
 * pointers owned by the caller; no workspace; FP_ERR_ARG on a bad argument. */
int fp_surrogate_training_rows(const double *moments, const double *lite, const double *coeffs, const double *tau,
                               int64_t n_cells, int lite_inputs, float *raw_out, float *target_out, float *aux_out,
                               fp_stream_t stream);

/* Workspace of fp_closure_surrogate for n_cells cells: the list of cells for
 * the exact fallback (4 bytes a cell) and its count. */
size_t fp_surrogate_workspace_bytes(int64_t n_cells);

/* Features of every cell: x_out [n_cells][32] BF16, and flags_out with
 * FP_FLAG_FEW | FP_FLAG_SINGULAR | FP_FLAG_NONFINITE (the exact closure's
 * preconditions) and FP_FLAG_RANGE when a raw feature lies outside
 * [x_min - m x_sigma, x_max + m x_sigma], m = p->surr_range_margin. */
int fp_surrogate_features(const fp_mlp *net, const double *moments, int64_t n_cells, const double *tau,
                          const fp_params *p, void *x_out, int32_t *flags_out, fp_stream_t stream);

/* The fused network on n rows of BF16 features x [n][32]:
 * out [n][16] FP32 -- standardised outputs when standardized_out != 0, else
 * y_mu + y_sigma * output.  For training, h_save (4 x n x 128 BF16, the
 * hidden activations) and z_save (4 x n x 128 FP32, their pre-activations)
 * are written when both are non-NULL, column-block-major so that the rows of
 * a warp are written and read back contiguously: columns 8k .. 8k + 7 of
 * row r of layer l at h_save + ((l * 16 + k) * n + r) * 8, columns
 * 4k .. 4k + 3 at z_save + ((l * 32 + k) * n + r) * 4.  No workspace. */
int fp_mlp_forward(const fp_mlp *net, const void *x, int64_t n, int standardized_out, float *out, void *h_save,
                   float *z_save, fp_stream_t stream);

/* The surrogate closure: features, network, coefficients C = t / tau,
 * G = t / (tau sqrt(theta)), all in one tcgen05 kernel (the inputs are formed
 * from the moment rows inside it, the predictions never leave it), followed
 * by the exact closure on the cells it lists; a cell is recomputed by the exact FP64 closure
 * from its moments (FP_FLAG_FALLBACK) when it fails the exact closure's
 * preconditions, a raw feature leaves the training box (FP_FLAG_RANGE),
 * the prediction is not finite, or the energy residual
 * e = 1 + (sum_ij C^_ij u^_ij + sum_i G^_i b^_i - eps2_hat s4^) / 3 of the
 * predicted drift exceeds p->surr_energy_tol (FP_FLAG_ENERGY).  prec: the
 * precision the moments were gathered in (fallback singularity threshold).
 *   moments [n_cells][FP_NMOM], tau [n_cells]; coeffs_out [n_cells][9],
 *   flags_out [n_cells]; ws >= fp_surrogate_workspace_bytes(n_cells). */
int fp_closure_surrogate(const fp_mlp *net, const double *moments, int64_t n_cells, const double *tau,
                         const fp_params *p, int prec, double *coeffs_out, int32_t *flags_out, void *ws,
                         size_t ws_bytes, fp_stream_t stream);

/* Training loss and its gradient w.r.t. the standardised outputs, per row:
 *   sum_a w_a (o_a - (t_a - y_mu_a) / y_sigma_a)^2
 *   + lam_drift [tr(D u D) + 2 g.D b + |g|^2 (s4 - 9)] + lam_energy e^2
 * with (D, g) = prediction - target in the symmetric C block and the G block,
 * (u, b, s4) the row's normalised moments u^_ij, b^_i = u^_ikk, s4^ = w^_kk
 * -- the first bracket is tau^2 / theta times the mean square, over the cell,
 * of the difference of the drifts (Eq. cubic_drift) the two coefficient sets
 * induce -- and e the energy residual above.
 *   out [n][16] standardised network outputs; t_true [n][9] dimensionless
 *   targets; aux [n][16] = (u^ (6), b^ (3), s4^, unused); w [9] host array;
 *   dout [n][16] FP32 and dout_bf16 [n][16] BF16: scale * dL/dout;
 *   loss_sum [1] FP32 += sum of the row losses. */
int fp_surrogate_loss(const float *out, const float *t_true, const float *aux, const float *y_mu,
                      const float *y_sigma, int64_t n, const float *w, float lam_drift, float lam_energy,
                      float eps2_hat, float scale, float *dout, void *dout_bf16, float *loss_sum, fp_stream_t stream);

/* Backward pass of fp_mlp_forward: grads (flat FP32, layout above) of
 * sum_rows dout . out given the forward's x, h_save, z_save and dout (FP32
 * for the last bias, BF16 for the GEMMs).  GEMMs: BF16 tensor cores, FP32
 * accumulation.  ws >= fp_mlp_backward_workspace_bytes(n). */
size_t fp_mlp_backward_workspace_bytes(int64_t n);
int fp_mlp_backward(const fp_mlp *net, const void *x, const void *h_save, const float *z_save,
                    const void *dout_bf16, const float *dout, int64_t n, float *grads, void *ws, size_t ws_bytes,
                    fp_stream_t stream);

/* One Adam step (Kingma & Ba) over n_params FP32 parameters with bias
 * corrections for step t >= 1; shadow_bf16 (or NULL) receives the BF16 copy
 * of the updated parameters (the forward's weights). */
int fp_adam_step(float *params, const float *grads, float *m, float *v, int64_t n_params, float lr, float beta1,
                 float beta2, float eps, int64_t t, void *shadow_bf16, fp_stream_t stream);

/* One training step of the learned closure (Sec. 4, Phase 2) in four kernel
 * launches: fp_mlp_forward (standardised outputs, activations saved) with the
 * loss of fp_surrogate_loss fused into its last layer, then fp_mlp_backward
 * with the Adam step of fp_adam_step fused into the sum of its per-tile
 * gradients.  It computes what those four calls compute in sequence, with
 * y_mu, y_sigma and eps2_hat taken from net (the loss's arithmetic is the
 * same code; results agree to FP32 rounding of the fused kernels' order).
 *   x [n][32] BF16 (16-byte aligned), t_true [n][9], aux [n][16] (as for
 *   fp_surrogate_loss); w [9] host array; scale multiplies dL/dout;
 *   params [n_params] FP32 (the flat layout, n_params = fp_mlp_param_count()),
 *   m, v: Adam moments; params, m, v updated in place; shadow_bf16 [n_params]
 *   BF16 copy of params written when non-NULL (net->W must point into it
 *   for the next step to see the update); t >= 1 the Adam step number;
 *   grads [n_params] FP32: the gradient (written); loss_sum [1] FP32 += sum
 *   of the row losses (non-finite, with non-finite gradients, if a tensor-core
 *   wait timed out);
 *   ws >= fp_surrogate_train_step_workspace_bytes(n), 256-byte aligned.
 * All arrays are device memory owned by the caller except w.  Returns
 * FP_ERR_ARG (n < 0, t < 1, n_params wrong, a null or misaligned pointer),
 * FP_ERR_UNSUPPORTED (network shape), FP_ERR_WORKSPACE, or FP_ERR_CUDA (launch);
 * every check precedes the first launch, and n = 0 launches nothing. */
size_t fp_surrogate_train_step_workspace_bytes(int64_t n);
int fp_surrogate_train_step(const fp_mlp *net, const void *x, const float *t_true, const float *aux, int64_t n,
                            const float *w, float lam_drift, float lam_energy, float scale, float *params,
                            float *grads, float *m, float *v, int64_t n_params, float lr, float beta1, float beta2,
                            float eps, int64_t t, void *shadow_bf16, float *loss_sum, void *ws, size_t ws_bytes,
                            fp_stream_t stream);

/* fp_closure_exact_static: fp_closure_exact for callers that cannot allocate
 * device memory.  (The paper has no counterpart; this is a deployment
 * convenience of this library.)
 *
 * Some callers may not allocate GPU memory at all -- a solver plugin inside a
 * host application that owns the device memory budget, or a time-critical
 * step loop where cudaMalloc, which may synchronise the device, is not
 * allowed.  fp_closure_exact needs scratch for the per-cell moments when the
 * caller does not take them; this call keeps that scratch in a fixed array
 * built into the library instead and allocates nothing (no cudaMalloc,
 * cudaFree or allocating library routine).  The caller passes its inputs and
 * outputs exactly as to fp_closure_exact with moments_out = NULL and no
 * workspace; the results are the same.
 *   - At most FP_STATIC_MAX_CELLS cells per call; larger n_cells is rejected
 *     with FP_ERR_ARG (message via fp_closure_exact_static_error()).
 *   - The array (FP_STATIC_MAX_CELLS x FP_NMOM doubles, 7.9 MB) is a
 *     file-scope __device__ array: every GPU that loads the library holds it
 *     until the process exits.
 *   - The first call on each device looks up the array's device address
 *     (cudaGetSymbolAddress, with that device current); make that first call
 *     before any stream capture.  The address is kept for the process:
 *     after cudaDeviceReset on a device (or from a second driver-API context
 *     on it) the library's module may load at another address, so do not
 *     call this entry point on that device again in the same process.
 *   - If the moment gather fails to launch, the call returns FP_ERR_CUDA
 *     before the solve runs, leaving coeffs_out and flags_out untouched.
 *   - Every call on a device shares the one array and it keeps the last
 *     call's contents; nothing needs clearing (each call overwrites every
 *     slot it reads).  Calls whose executions overlap on the GPU (different
 *     streams, no ordering between them) race on the array: serialise them. */
#define FP_STATIC_MAX_CELLS 32768
int fp_closure_exact_static(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                            int64_t n_cells, const double *tau, const fp_params *p, int prec, double *coeffs_out,
                            int32_t *flags_out, fp_stream_t stream);
const char *fp_closure_exact_static_error(void);

/* ------------------------------------------------------------------------
 * The LITE path (Sec. 4, Phase 3 item 2, and Phase 1-2 item 1): the moment
 * pass stops at the heat flux, and the network reads the paper's 16 low-order
 * inputs rho, T, U (3), Pi (6), q (3), DM2, nu.  Read here as rho = N (the
 * cell's particle count), T = theta, Pi_ij = u_ij - theta delta_ij,
 * q_i = <c_i |c|^2> / 2, DM2 = det(u) (determinant of the second-moment
 * tensor), nu = 1 / tau; inputs 16..31 of the network are zero.  A network
 * trained on these inputs (same fp_mlp shape as the full-moment one) maps
 * them to the same dimensionless targets (tau C, tau sqrt(theta) G).
 * ------------------------------------------------------------------------ */
#define FP_NLITE 14  /* LITE moment vector: N, U1..3, theta, u11,u12,u13,u22,u23,u33, b1..3 (b_i = <c_i |c|^2>) */

/* fp_moments_lite: the LITE moment vectors [n_cells][FP_NLITE] f64 (required)
 * of the velocities (FP32 compensated sums as in FP_PREC_FP32_MOMENTS, any
 * velocity dtype).  No workspace. */
int fp_moments_lite(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets, int64_t n_cells,
                    double *lite_out, fp_stream_t stream);

/* fp_surrogate_lite_features: the network inputs [n_cells][32] BF16
 * (standardised with net's scalers, zero padded) and flags (FP_FLAG_FEW,
 * FP_FLAG_SINGULAR for theta <= 0, FP_FLAG_NONFINITE, FP_FLAG_RANGE outside
 * the training box widened by p->surr_range_margin sigma) from LITE vectors
 * and tau.  x_out 16-byte aligned.  No workspace. */
int fp_surrogate_lite_features(const fp_mlp *net, const double *lite, int64_t n_cells, const double *tau,
                               const fp_params *p, void *x_out, int32_t *flags_out, fp_stream_t stream);

/* fp_velocity_update_lite: fp_velocity_update from LITE vectors
 * [n_cells][FP_NLITE] (U, theta and b_i are all the update reads; the cell
 * averages of Eq. update_alpha are summed over the particles in a first
 * pass).  Other arguments as fp_velocity_update (without m6). */
int fp_velocity_update_lite(void *v, void *v_out, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                            int64_t n_cells, const double *lite, const double *coeffs, const double *tau, double dt,
                            const fp_params *p, const void *xi, uint64_t seed, uint64_t step, double *alpha_out,
                            int32_t *flags, fp_stream_t stream);

/* Workspace of fp_closure_surrogate_lite: 0 bytes (the call is one fused
 * kernel); kept so that callers size every call the same way. */
size_t fp_surrogate_lite_workspace_bytes(int64_t n_cells);

/* fp_closure_surrogate_lite: the learned closure on the LITE inputs:
 * features, the network and coefficients in one tcgen05 kernel, C = t_C / tau,
 * G = t_G / (tau sqrt(theta)).  There are no high-order moments to fall back
 * on: cells flagged FP_FLAG_FEW, FP_FLAG_SINGULAR or FP_FLAG_NONFINITE (also
 * for a non-finite prediction) take the linear drift C = -I/tau, G = 0;
 * FP_FLAG_RANGE is reported and the prediction kept.  ws and ws_bytes are
 * not read (ws may be NULL). */
int fp_closure_surrogate_lite(const fp_mlp *net, const double *lite, int64_t n_cells, const double *tau,
                              const fp_params *p, double *coeffs_out, int32_t *flags_out, void *ws, size_t ws_bytes,
                              fp_stream_t stream);

/* ------------------------------------------------------------------------
 * Heuristic coefficient-sensitivity probe of the learned closure (the
 * cylinder study's dropout probe): n_passes forward passes with the hidden
 * activations dropped at `rate` (kept ones scaled by 1 / (1 - rate)); per
 * cell sigma_i = sqrt(1/N sum_k (y_i^(k) - mean_i)^2) of each predicted
 * coefficient y_i (C11, C12, C13, C22, C23, C33, Gamma1..3, in physical
 * units: the network's tau C and tau sqrt(theta) Gamma divided back), and
 * sigma_Stress = sqrt(sum over the six C entries of sigma_i^2), sigma_Heat =
 * sqrt(sum over the three Gamma entries).  The masks of pass k come from
 * Philox4x32-10 keyed by `seed`: activation j of hidden layer l (0..3) of
 * cell r is dropped when word j % 4 of the generator on counter (r lo, r hi,
 * k, 32 l + j / 4) gives (floor(w / 2^8) + 1) 2^-24 <= rate.
 *   moments        [n_cells][moment_stride] f64: moment_stride FP_NMOM for a
 *                  network on the full inputs (fp_moments), FP_NLITE for one
 *                  on the LITE inputs (fp_moments_lite)
 *   tau            [n_cells]; p: min_particles and surr_range_margin are read
 *   n_passes >= 1, 0 <= rate < 1
 *   sens_out       [n_cells][FP_NSENS] f64: sigma_1..9, sigma_Stress,
 *                  sigma_Heat; NaN for cells flagged FP_FLAG_FEW,
 *                  FP_FLAG_SINGULAR or FP_FLAG_NONFINITE
 *   mean_out       [n_cells][9] f64 mean coefficients over the passes, or NULL
 *   flags_out      [n_cells] int32 input flags (as fp_surrogate_features), or
 *                  NULL
 *   ws             >= fp_surrogate_sensitivity_workspace_bytes(n_cells),
 *                  256-byte aligned */
#define FP_NSENS 11
size_t fp_surrogate_sensitivity_workspace_bytes(int64_t n_cells);
int fp_surrogate_sensitivity(const fp_mlp *net, const double *moments, int moment_stride, int64_t n_cells,
                             const double *tau, const fp_params *p, int n_passes, double rate, uint64_t seed,
                             double *sens_out, double *mean_out, int32_t *flags_out, void *ws, size_t ws_bytes,
                             fp_stream_t stream);

/* ------------------------------------------------------------------------
 * Cell sort and the collision step (Alg. 1 and Alg. 2: particles sorted by
 * cell, moments, closure, velocity update).
 *
 * fp_sort_by_cell: the stable permutation that orders particles by cell
 * index, the CSR offsets and (optionally) the velocities in that order.
 *   cell_of      [n_particles] int32 cell index per particle; an index outside
 *                [0, n_cells) puts the particle behind the last cell, in no
 *                cell (cell_offsets_out[n_cells] < n_particles counts them)
 *   v            [3][n_particles] SoA (FP_V_F32 / FP_V_F64), or NULL
 *   v_sorted     [3][n_particles] (same dtype; required when v is given, must
 *                not alias v): v_sorted[d][i] = v[d][perm_out[i]]
 *   perm_out     [n_particles] int32: input index of the particle at sorted
 *                position i; equal cell indices keep their input order
 *   cell_offsets_out [n_cells + 1] int64: first sorted position of each cell,
 *                offsets[n_cells] = particles inside the cells
 *   ws           >= fp_sort_workspace_bytes(n_particles, n_cells), 256-byte
 *                aligned (keys and indices twice, digit counts)
 * n_particles <= 2^31 - 1 and n_cells <= 2^31 - 2, else FP_ERR_UNSUPPORTED.
 * Result identical on every run (integer work only). */
size_t fp_sort_workspace_bytes(int64_t n_particles, int64_t n_cells);
int fp_sort_by_cell(const int32_t *cell_of, int64_t n_particles, int64_t n_cells, const void *v, int v_dtype,
                    void *v_sorted, int32_t *perm_out, int64_t *cell_offsets_out, void *ws, size_t ws_bytes,
                    fp_stream_t stream);

/* fp_collision_step: one collision step of unsorted particles in one call:
 * fp_sort_by_cell, then either the exact cubic-FP closure (net_lite NULL:
 * moments in `prec` with <|c|^6>, FP64 assembly and solve, the velocity update
 * with alpha from the moments) or the learned closure on LITE inputs (net_lite
 * a network trained on them: LITE moment pass, fp_closure_surrogate_lite,
 * the velocity update with alpha from a pass over the particles), with
 * Philox noise keyed by (seed, step) on the sorted particle index.
 *   v          [3][n_particles] input velocities, any order
 *   v_out      [3][n_particles] updated velocities in sorted order (may alias
 *              v; particles in no cell are copied unchanged)
 *   perm_out, cell_offsets_out   as fp_sort_by_cell (reorder other particle
 *              arrays of the caller with perm_out)
 *   tau        [n_cells] f64; coeffs_out [n_cells][9] f64; flags_out
 *              [n_cells] int32 (closure flags | FP_FLAG_ALPHA)
 *   moments_out  [n_cells][FP_NMOM] (exact) or [n_cells][FP_NLITE] (LITE)
 *              f64, or NULL (kept in the workspace)
 *   ws         >= fp_collision_step_workspace_bytes(n_particles, n_cells,
 *              v_dtype, net_lite != NULL), 256-byte aligned */
size_t fp_collision_step_workspace_bytes(int64_t n_particles, int64_t n_cells, int v_dtype, int lite);
int fp_collision_step(const int32_t *cell_of, const void *v, int v_dtype, int64_t n_particles, int64_t n_cells,
                      const double *tau, const fp_params *p, int prec, const fp_mlp *net_lite, double dt,
                      uint64_t seed, uint64_t step, void *v_out, int32_t *perm_out, int64_t *cell_offsets_out,
                      double *coeffs_out, int32_t *flags_out, double *moments_out, void *ws, size_t ws_bytes,
                      fp_stream_t stream);

/* ------------------------------------------------------------------------
 * Diagnostics and deployment options of the learned closure.
 *
 * fp_diagnostics: per-cell high-order nonequilibrium diagnostics (the
 * normalised fields of the paper's cavity study: R_ij = <c_i c_j c_k c_k>,
 * Delta_4 = <(c_k c_k)^2> - 15 theta^2, DM6 = <(c_k c_k)^3>, each divided by
 * the local Maxwellian scale theta^2 or theta^3) and the covariance-based
 * entropy proxies of its cylinder audit (Eqs. cyl_theta_def, cyl_entropy_eq,
 * cyl_DG, cyl_entropy_kinG and the supplemental heat-flux term D_q).
 *   moments   [n_cells][FP_NMOM] f64, m6 [n_cells] f64 (fp_moments' m6_out)
 *   rho       [n_cells] f64 cell densities, or NULL: the particle count N
 *   theta_inf, rho_inf, dg_inf   the reference (upstream) theta, rho, D_G
 *   out       [n_cells][FP_NDIAG] f64:
 *     0..5  R_ij / theta^2 (sym order 11,12,13,22,23,33; Maxwellian 5 delta_ij)
 *     6     <|c|^4> / theta^2 - 15                   (Maxwellian 0)
 *     7     <|c|^6> / theta^3                        (Maxwellian 105)
 *     8     D_G = -1/2 log det(Theta / theta), Theta_ij = <c_i c_j>  (>= 0)
 *     9     D_q = |q_hat|^2 / 5, q_hat = <c |c|^2> / (2 theta^1.5)
 *     10    Delta s_eq / k_B = 3/2 log(theta / theta_inf) - log(rho / rho_inf)
 *     11    Delta s_kin,G / k_B = Delta s_eq / k_B - (D_G - dg_inf)
 *   Cells with N < 2, theta <= 0, det Theta <= 0, rho <= 0 or a non-finite
 *   input get NaN in every entry.  No workspace. */
#define FP_NDIAG 12
int fp_diagnostics(const double *moments, const double *m6, const double *rho, int64_t n_cells, double theta_inf,
                   double rho_inf, double dg_inf, double *out, fp_stream_t stream);

/* fp_coeffs_relax: temporal under-relaxation of the coefficient field (the
 * paper's cylinder deployment couples the network's prediction with w = 0.2):
 * coeffs_prev <- w coeffs_new + (1 - w) coeffs_prev, [n_cells][9] f64 each,
 * in place on coeffs_prev; w in [0, 1]. */
int fp_coeffs_relax(const double *coeffs_new, double *coeffs_prev, int64_t n_cells, double w, fp_stream_t stream);

/* ------------------------------------------------------------------------
 * Host-resident step (a runtime layer; the paper has no counterpart).
 *
 * fp_step_host runs one step of the hot path -- the exact closure (gather +
 * solve), optionally the learned closure and the adjoint, and the velocity
 * update -- for velocities held in HOST memory, and returns the coefficients,
 * flags and updated velocities to host memory.  The cells are split into
 * n_chunks contiguous chunks; each chunk's host -> device copies, compute and
 * device -> host copies run on separate streams of the pipeline, so the
 * copies of one chunk overlap the compute of its neighbours.  The results
 * equal those of the separate calls on the whole population (the Philox
 * counter of a particle is its global index).  Host buffers must be
 * page-locked for the copies to overlap.  Device buffers are caller-owned and
 * full size; the call allocates nothing.  The call is ordered after work
 * already queued on `stream`, and `stream` waits for all of its work; it
 * returns once everything is queued.
 * ------------------------------------------------------------------------ */
typedef struct fp_pipeline fp_pipeline;  /* streams and events of the pipeline */

/* Creates the pipeline's streams (one at the highest priority) and events.
 * FP_ERR_CUDA if they cannot be created; *out is NULL then. */
int fp_pipeline_create(fp_pipeline **out);
/* Waits for the pipeline's streams and releases them. NULL is ignored. */
void fp_pipeline_destroy(fp_pipeline *pl);

typedef struct {
  /* host */
  const void *h_v;          /* [3][n_particles] velocities M^n (v_dtype)        */
  void *h_v_out;            /* [3][n_particles] receives M^{n+1}                */
  const int64_t *h_offsets; /* [n_cells + 1], 0 .. n_particles                  */
  const double *h_tau;      /* [n_cells]                                        */
  double *h_coeffs;         /* [n_cells][9] receives the exact closure          */
  int32_t *h_flags;         /* [n_cells] receives the flags after the update    */
  /* device, full size */
  void *d_v, *d_v_out;      /* [3][n_particles] each; distinct                  */
  int64_t *d_offsets;       /* [n_cells + 1]                                    */
  double *d_tau;            /* [n_cells]                                        */
  double *d_moments;        /* [n_cells][FP_NMOM]                               */
  double *d_m6;             /* [n_cells] <|c|^6> for a one-pass update, or NULL */
  double *d_coeffs;         /* [n_cells][9]                                     */
  int32_t *d_flags;         /* [n_cells] closure flags                          */
  int32_t *d_flags_v;       /* [n_cells] the update's flags (closure flags plus
                               FP_FLAG_ALPHA), copied to h_flags                */
  /* learned closure with exact fallback: skipped if net is NULL */
  const fp_mlp *net;
  double *d_coeffs_s;       /* [n_cells][9]                                     */
  int32_t *d_flags_s;       /* [n_cells]                                        */
  void *d_surrogate_ws;     /* fp_surrogate_workspace_bytes(n_cells) bytes      */
  size_t surrogate_ws_bytes;
  /* adjoint: skipped if d_grad_coeffs is NULL */
  double *d_lu;                /* FP_LU_DOUBLES(n_cells): factors kept by the
                                  solve for the adjoint, or NULL (recomputed);
                                  chunks start on multiples of 32 cells      */
  const double *d_grad_coeffs; /* [n_cells][9] dL/dY                            */
  double *d_grad_moments;      /* [n_cells][FP_NMOM] receives dL/dm             */
  void *d_grad_v;              /* [3][n_particles] receives dL/dv, or NULL      */
} fp_step_io;

/* n_chunks in [1, 64] (clamped to n_cells); dt, seed, step as for
 * fp_velocity_update (Philox noise), p and prec as for fp_closure_exact.
 * FP_ERR_ARG for null buffers, d_v_out == d_v, offsets not running from 0 to
 * n_particles; otherwise the first error of a chunk's call. */
int fp_step_host(fp_pipeline *pl, const fp_step_io *io, int v_dtype, int64_t n_particles, int64_t n_cells,
                 const fp_params *p, int prec, double dt, uint64_t seed, uint64_t step, int n_chunks,
                 fp_stream_t stream);

/* ------------------------------------------------------------------------
 * Self-test of the bounded waits (a runtime check; the paper has no
 * counterpart).  Every kernel that consumes bulk copies waits on mbarriers
 * with a limit on the global timer and reports a wait that runs out in band
 * instead of spinning.  fp_selftest_wait_timeout launches one CTA that waits
 * on an mbarrier nothing completes, with limit_ns in (0, 1e9]:
 *   status_out     device int32: 0 when the wait gave up (the expected
 *                  answer), 1 if the barrier had completed
 *   waited_ns_out  device uint64: the time the wait took (>= limit_ns)
 * Asynchronous on `stream`; FP_ERR_ARG for a null pointer or a limit out of
 * range. */
int fp_selftest_wait_timeout(uint64_t limit_ns, int32_t *status_out, uint64_t *waited_ns_out, fp_stream_t stream);

#ifdef __cplusplus
}
#endif

#endif /* FPCLOSURE_H */
