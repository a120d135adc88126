// api.cu -- the C ABI of libfpclosure.so (declarations and contracts in
// include/fpclosure.h): argument validation, workspace carving, launches.
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "fp_device.cuh"
#include "train_math.cuh"

namespace fpc {
void launch_gather(const void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, int prec,
                   double *mom, double *m6, cudaStream_t st);
void launch_solve(const double *mom, const double *tau, int64_t n_cells, const fp_params &p, int prec,
                  double *coeffs, int32_t *flags, double *lu, cudaStream_t st);
void launch_velocity(const void *v, void *v_out, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells,
                     const double *mom, const double *m6, const double *coeffs, const double *tau, double dt,
                     double eps2_hat, const void *xi, uint64_t seed, uint64_t step, uint64_t particle_offset,
                     double *alpha_out, int32_t *flags, cudaStream_t st);
void launch_adjoint(const void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, const double *tau,
                    double eps2_hat, const double *mom, const double *coeffs, const int32_t *flags, const double *lu,
                    const double *gY, const double *gm_in, double *gm_out, void *gv, cudaStream_t st);
void launch_training_rows(const double *mom, const double *lite, const double *coeffs, const double *tau, int64_t n,
                          int lite_inputs, float *raw, float *targ, float *aux, cudaStream_t st);
void launch_features(const fp_mlp &net, const double *mom, const double *tau, int64_t n, int min_particles,
                     double margin, void *x, int32_t *flags, cudaStream_t st);
int launch_mlp_forward(const fp_mlp &net, const void *x, int64_t n, int standardized_out, float *out, void *h_save,
                       float *z_save, cudaStream_t st);
int launch_closure_surrogate(const fp_mlp &net, const double *mom, const double *tau, int64_t n, double eps2_hat,
                             const fp_params &p, int prec, double *coeffs, int32_t *flags, int32_t *list,
                             uint32_t *count, cudaStream_t st);
int launch_closure_surrogate_lite(const fp_mlp &net, const double *lite, const double *tau, int64_t n,
                                  const fp_params &p, double *coeffs, int32_t *flags, cudaStream_t st);
void launch_gather_lite(const void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, double *lite,
                        cudaStream_t st);
void launch_lite_features(const fp_mlp &net, const double *lite, const double *tau, int64_t n, int min_particles,
                          double margin, void *x, int32_t *flags, cudaStream_t st);
int launch_mlp_forward_dropout(const fp_mlp &net, const void *x, int64_t n, float *out, double rate, uint64_t seed,
                               uint32_t pass, cudaStream_t st);
void launch_sens_accumulate(const float *tpred, int64_t n, int k, double *mean, double *m2, cudaStream_t st);
void launch_sens_finalize(const double *mean, const double *m2, const double *mom, int stride, const double *tau,
                          int64_t n, int n_passes, const int32_t *flags, double *out, double *mean_out,
                          cudaStream_t st);
size_t sort_workspace_bytes(int64_t n, int64_t n_cells);
void launch_sort_by_cell(const int32_t *cell_of, int64_t n, int64_t n_cells, int32_t *perm, int64_t *offsets,
                         void *ws, cudaStream_t st, const uint32_t **sorted_keys);
void launch_gather_sorted(const void *v, int v_dtype, int64_t n, const int32_t *perm, void *v_sorted,
                          cudaStream_t st);
void launch_copy_tail(const void *v, void *v_out, int v_dtype, int64_t n, const int64_t *first, cudaStream_t st);
void launch_velocity_lite(const void *v, void *v_out, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells,
                          const double *lite, const double *coeffs, const double *tau, double dt, double eps2_hat,
                          const void *xi, uint64_t seed, uint64_t step, uint64_t particle_offset,
                          double *alpha_out, int32_t *flags, cudaStream_t st);
void launch_diagnostics(const double *mom, const double *m6, const double *rho, int64_t n_cells, double theta_inf,
                        double rho_inf, double dg_inf, double *out, cudaStream_t st);
void launch_relax(const double *y_new, double *y_prev, int64_t n, double w, cudaStream_t st);
int64_t mlp_param_offset(int which, int layer);
void launch_wait_timeout(uint64_t limit_ns, int32_t *status, uint64_t *waited_ns, cudaStream_t st);
int64_t mlp_param_count();
size_t mlp_backward_ws(int64_t n);
int launch_mlp_backward(const fp_mlp &net, const void *x, const void *h_save, const float *z_save,
                         const void *dout_bf, const float *dout, int64_t n, float *grads, void *ws, cudaStream_t st);
void launch_loss(const float *out, const float *t_true, const float *aux, const float *y_mu, const float *y_sigma,
                 int64_t n, const float *w, float lam_d, float lam_e, float eps2_hat, float scale, float *dout,
                 void *dout_bf, float *loss_sum, cudaStream_t st);
void launch_adam(float *p, const float *g, float *m, float *v, int64_t n, float lr, float b1, float b2, float eps,
                 float bc1, float bc2, void *shadow, cudaStream_t st);
size_t train_step_ws(int64_t n);
int launch_train_step(const fp_mlp &net, const void *x, const float *t_true, const float *aux, int64_t n,
                      const float *w, float lam_d, float lam_e, float scale, float *grads, const AdamParams &adam,
                      float *loss_sum, void *ws, cudaStream_t st);
}  // namespace fpc


namespace {
thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof g_err, fmt, ap);
  va_end(ap);
  return code;
}

int check_launch(const char *what) {
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fail(FP_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
  return FP_OK;
}

constexpr size_t kAlign = 256;
size_t align_up(size_t x) { return (x + kAlign - 1) / kAlign * kAlign; }
int check_net(const fp_mlp *net) {
  if (!net) return fail(FP_ERR_ARG, "null network");
  if (net->in_dim != 32 || net->hidden != 128 || net->depth != 4 || net->out_dim != 16)
    return fail(FP_ERR_UNSUPPORTED, "network shape %d-%dx%d-%d (32-128x4-16 supported)", net->in_dim, net->hidden,
                net->depth, net->out_dim);
  for (int l = 0; l < 5; ++l) {
    if (!net->W[l] || !net->b[l]) return fail(FP_ERR_ARG, "null weight or bias %d", l);
    if ((uintptr_t)net->W[l] % 16) return fail(FP_ERR_ARG, "weight %d not 16-byte aligned", l);
  }
  if (!net->x_mu || !net->x_sigma || !net->y_mu || !net->y_sigma || !net->x_min || !net->x_max)
    return fail(FP_ERR_ARG, "null scaler");
  return FP_OK;
}
// fallback list [n] int32, then its count
size_t surrogate_ws_parts(int64_t n, size_t *off_count) {
  *off_count = align_up((size_t)n * 4);
  return *off_count + 256;
}
}  // namespace

namespace fpc {
// error reporting for the other translation units of the C ABI
int report(int code, const char *msg) { return fail(code, "%s", msg); }
}  // namespace fpc

extern "C" {

void fp_default_params(fp_params *p) {
  if (!p) return;
  p->eps2_hat = 1e-3;
  p->min_particles = 4;
  p->pivot_rtol = 1e-13;
  p->surr_energy_tol = 0.05;
  p->surr_range_margin = 0.5;
  p->particle_offset = 0;
}

const char *fp_status_string(int status) {
  switch (status) {
    case FP_OK: return "ok";
    case FP_ERR_ARG: return "invalid argument";
    case FP_ERR_CUDA: return "CUDA error";
    case FP_ERR_WORKSPACE: return "workspace missing or too small";
    case FP_ERR_UNSUPPORTED: return "unsupported request";
    default: return "unknown status";
  }
}

const char *fp_last_error(void) { return g_err; }

int fp_version(void) { return 100; }

size_t fp_workspace_bytes(int64_t n_cells, int64_t n_particles, int prec, int moments_out_given) {
  (void)n_particles;
  (void)prec;
  if (n_cells <= 0 || moments_out_given) return 0;
  return align_up((size_t)n_cells * FP_NMOM * sizeof(double));
}

int fp_closure_exact(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                     int64_t n_cells, const double *tau, const fp_params *p, int prec, double *moments_out,
                     double *coeffs_out, int32_t *flags_out, void *ws, size_t ws_bytes, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0 || n_particles < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return fail(FP_ERR_ARG, "v_dtype %d", v_dtype);
  if (prec != FP_PREC_FP64 && prec != FP_PREC_FP32_MOMENTS) return fail(FP_ERR_ARG, "prec %d", prec);
  if (!cell_offsets || !tau || !coeffs_out || !flags_out) return fail(FP_ERR_ARG, "null array pointer");
  if (n_particles > 0 && !v) return fail(FP_ERR_ARG, "null velocity pointer");
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  if (prm.min_particles < 1) prm.min_particles = 1;
  double *mom = moments_out;
  if (!mom) {
    const size_t need = fp_workspace_bytes(n_cells, n_particles, prec, 0);
    if (!ws || ws_bytes < need)
      return fail(FP_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
    if ((uintptr_t)ws % kAlign) return fail(FP_ERR_ARG, "workspace not 256-byte aligned");
    mom = (double *)ws;
  }
  cudaStream_t st = (cudaStream_t)stream;
  fpc::launch_gather(v, v_dtype, n_particles, cell_offsets, n_cells, prec, mom, nullptr, st);
  if (int rc = check_launch("gather")) return rc;
  fpc::launch_solve(mom, tau, n_cells, prm, prec, coeffs_out, flags_out, nullptr, st);
  return check_launch("solve");
}

int fp_moments(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets, int64_t n_cells,
               int prec, double *moments_out, double *m6_out, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0 || n_particles < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return fail(FP_ERR_ARG, "v_dtype %d", v_dtype);
  if (prec != FP_PREC_FP64 && prec != FP_PREC_FP32_MOMENTS) return fail(FP_ERR_ARG, "prec %d", prec);
  if (!cell_offsets || !moments_out) return fail(FP_ERR_ARG, "null array pointer");
  if (n_particles > 0 && !v) return fail(FP_ERR_ARG, "null velocity pointer");
  fpc::launch_gather(v, v_dtype, n_particles, cell_offsets, n_cells, prec, moments_out, m6_out,
                     (cudaStream_t)stream);
  return check_launch("gather");
}

int fp_closure_solve(const double *moments, const double *tau, int64_t n_cells, const fp_params *p, int prec,
                     double *coeffs_out, int32_t *flags_out, double *lu_out, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (prec != FP_PREC_FP64 && prec != FP_PREC_FP32_MOMENTS) return fail(FP_ERR_ARG, "prec %d", prec);
  if (!moments || !tau || !coeffs_out || !flags_out) return fail(FP_ERR_ARG, "null array pointer");
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  if (prm.min_particles < 1) prm.min_particles = 1;
  fpc::launch_solve(moments, tau, n_cells, prm, prec, coeffs_out, flags_out, lu_out, (cudaStream_t)stream);
  return check_launch("solve");
}

namespace {
int check_update_args(const void *v, const void *v_out, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                      int64_t n_cells, const double *moments, const double *coeffs, const double *tau, double dt,
                      const int32_t *flags) {
  if (n_cells < 0 || n_particles < 0) return fail(FP_ERR_ARG, "negative size");
  if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return fail(FP_ERR_ARG, "v_dtype %d", v_dtype);
  if (!cell_offsets || !moments || !coeffs || !tau || !flags) return fail(FP_ERR_ARG, "null array pointer");
  if (n_particles > 0 && !v) return fail(FP_ERR_ARG, "null velocity pointer");
  if (!(dt >= 0.0)) return fail(FP_ERR_ARG, "dt must be >= 0");
  if (v_out && v_out != v && n_particles > 0) {
    const size_t bytes = (size_t)3 * (size_t)n_particles * (v_dtype == FP_V_F32 ? 4 : 8);
    const char *a = (const char *)v, *b = (const char *)v_out;
    if (a < b + bytes && b < a + bytes) return fail(FP_ERR_ARG, "v_out overlaps v without being v");
  }
  return FP_OK;
}
}  // namespace

int fp_velocity_update(void *v, void *v_out, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                       int64_t n_cells, const double *moments, const double *m6, const double *coeffs,
                       const double *tau, double dt, const fp_params *p, const void *xi, uint64_t seed,
                       uint64_t step, double *alpha_out, int32_t *flags, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells == 0 && n_particles >= 0) return FP_OK;
  if (int rc = check_update_args(v, v_out, v_dtype, n_particles, cell_offsets, n_cells, moments, coeffs, tau, dt,
                                 flags))
    return rc;
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  fpc::launch_velocity(v, v_out ? v_out : v, v_dtype, n_particles, cell_offsets, n_cells, moments, m6, coeffs, tau,
                       dt, prm.eps2_hat, xi, seed, step, prm.particle_offset, alpha_out, flags, (cudaStream_t)stream);
  return check_launch("velocity");
}

int fp_velocity_update_lite(void *v, void *v_out, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                            int64_t n_cells, const double *lite, const double *coeffs, const double *tau, double dt,
                            const fp_params *p, const void *xi, uint64_t seed, uint64_t step, double *alpha_out,
                            int32_t *flags, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells == 0 && n_particles >= 0) return FP_OK;
  if (int rc = check_update_args(v, v_out, v_dtype, n_particles, cell_offsets, n_cells, lite, coeffs, tau, dt, flags))
    return rc;
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  fpc::launch_velocity_lite(v, v_out ? v_out : v, v_dtype, n_particles, cell_offsets, n_cells, lite, coeffs, tau, dt,
                            prm.eps2_hat, xi, seed, step, prm.particle_offset, alpha_out, flags,
                            (cudaStream_t)stream);
  return check_launch("velocity_lite");
}

int fp_closure_backward(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                        int64_t n_cells, const double *tau, const fp_params *p, const double *moments,
                        const double *coeffs, const int32_t *flags, const double *lu, const double *grad_coeffs,
                        const double *grad_moments_in, double *grad_moments, void *grad_v, void *ws,
                        size_t ws_bytes, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0 || n_particles < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0 || (!grad_moments && !grad_v)) return FP_OK;
  if (!tau || !moments || !coeffs || !flags || !grad_coeffs) return fail(FP_ERR_ARG, "null array pointer");
  if (grad_v) {
    if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return fail(FP_ERR_ARG, "v_dtype %d", v_dtype);
    if (!cell_offsets) return fail(FP_ERR_ARG, "null offsets");
    if (n_particles > 0 && !v) return fail(FP_ERR_ARG, "null velocity pointer");
  }
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  double *gm = grad_moments;
  if (!gm) {
    const size_t need = fp_workspace_bytes(n_cells, n_particles, FP_PREC_FP64, 0);
    if (!ws || ws_bytes < need)
      return fail(FP_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
    if ((uintptr_t)ws % kAlign) return fail(FP_ERR_ARG, "workspace not 256-byte aligned");
    gm = (double *)ws;
  }
  fpc::launch_adjoint(v, v_dtype, n_particles, cell_offsets, n_cells, tau, prm.eps2_hat, moments, coeffs, flags, lu,
                      grad_coeffs, grad_moments_in, gm, grad_v, (cudaStream_t)stream);
  return check_launch("adjoint");
}

int64_t fp_mlp_param_count(void) { return fpc::mlp_param_count(); }

int64_t fp_mlp_param_offset(int which, int layer) {
  if (which < 0 || which > 1 || layer < 0 || layer > 4) return -1;
  return fpc::mlp_param_offset(which, layer);
}

size_t fp_surrogate_workspace_bytes(int64_t n_cells) {
  if (n_cells <= 0) return 0;
  size_t c;
  return surrogate_ws_parts(n_cells, &c);
}

int fp_surrogate_features(const fp_mlp *net, const double *moments, int64_t n_cells, const double *tau,
                          const fp_params *p, void *x_out, int32_t *flags_out, fp_stream_t stream) {
  g_err[0] = 0;
  if (int rc = check_net(net)) return rc;
  if (n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (!moments || !tau || !x_out || !flags_out) return fail(FP_ERR_ARG, "null array pointer");
  if ((uintptr_t)x_out % 16) return fail(FP_ERR_ARG, "features not 16-byte aligned");
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  fpc::launch_features(*net, moments, tau, n_cells, prm.min_particles, prm.surr_range_margin, x_out, flags_out,
                       (cudaStream_t)stream);
  return check_launch("features");
}

int fp_surrogate_training_rows(const double *moments, const double *lite, const double *coeffs, const double *tau,
                               int64_t n_cells, int lite_inputs, float *raw_out, float *target_out, float *aux_out,
                               fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (lite_inputs != 0 && lite_inputs != 1) return fail(FP_ERR_ARG, "lite_inputs %d", lite_inputs);
  if (n_cells == 0) return FP_OK;
  const bool need_mom = target_out || aux_out || (raw_out && !lite_inputs);
  if (!tau) return fail(FP_ERR_ARG, "null tau");
  if (need_mom && !moments) return fail(FP_ERR_ARG, "null moments");
  if (raw_out && lite_inputs && !lite) return fail(FP_ERR_ARG, "null lite vectors");
  if (target_out && !coeffs) return fail(FP_ERR_ARG, "null coefficients");
  if (((uintptr_t)raw_out | (uintptr_t)target_out | (uintptr_t)aux_out) % 16)
    return fail(FP_ERR_ARG, "outputs not 16-byte aligned");
  fpc::launch_training_rows(need_mom ? moments : nullptr, lite, coeffs, tau, n_cells, lite_inputs, raw_out, target_out,
                            aux_out, (cudaStream_t)stream);
  return check_launch("training rows");
}

int fp_mlp_forward(const fp_mlp *net, const void *x, int64_t n, int standardized_out, float *out, void *h_save,
                   float *z_save, fp_stream_t stream) {
  g_err[0] = 0;
  if (int rc = check_net(net)) return rc;
  if (n < 0) return fail(FP_ERR_ARG, "negative size");
  if (n == 0) return FP_OK;
  if (!x || !out) return fail(FP_ERR_ARG, "null array pointer");
  if ((uintptr_t)x % 16 || (uintptr_t)out % 8) return fail(FP_ERR_ARG, "misaligned x or out");
  if (fpc::launch_mlp_forward(*net, x, n, standardized_out, out, h_save, z_save, (cudaStream_t)stream))
    return fail(FP_ERR_CUDA, "could not raise the shared-memory limit of the MLP kernel");
  return check_launch("mlp_forward");
}

int fp_closure_surrogate(const fp_mlp *net, const double *moments, int64_t n_cells, const double *tau,
                         const fp_params *p, int prec, double *coeffs_out, int32_t *flags_out, void *ws,
                         size_t ws_bytes, fp_stream_t stream) {
  g_err[0] = 0;
  if (int rc = check_net(net)) return rc;
  if (n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (prec != FP_PREC_FP64 && prec != FP_PREC_FP32_MOMENTS) return fail(FP_ERR_ARG, "prec %d", prec);
  if (!moments || !tau || !coeffs_out || !flags_out) return fail(FP_ERR_ARG, "null array pointer");
  size_t off_count;
  const size_t need = surrogate_ws_parts(n_cells, &off_count);
  if (!ws || ws_bytes < need) return fail(FP_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
  if ((uintptr_t)ws % kAlign) return fail(FP_ERR_ARG, "workspace not 256-byte aligned");
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  if (prm.min_particles < 1) prm.min_particles = 1;
  char *w = (char *)ws;
  if (fpc::launch_closure_surrogate(*net, moments, tau, n_cells, net->eps2_hat, prm, prec, coeffs_out, flags_out,
                                    (int32_t *)w, (uint32_t *)(w + off_count), (cudaStream_t)stream))
    return fail(FP_ERR_CUDA, "could not raise the shared-memory limit of the MLP kernel");
  return check_launch("closure_surrogate");
}

int fp_surrogate_loss(const float *out, const float *t_true, const float *aux, const float *y_mu,
                      const float *y_sigma, int64_t n, const float *w, float lam_drift, float lam_energy,
                      float eps2_hat, float scale, float *dout, void *dout_bf16, float *loss_sum,
                      fp_stream_t stream) {
  g_err[0] = 0;
  if (n < 0) return fail(FP_ERR_ARG, "negative size");
  if (n == 0) return FP_OK;
  if (!out || !t_true || !aux || !y_mu || !y_sigma || !w || !dout || !dout_bf16 || !loss_sum)
    return fail(FP_ERR_ARG, "null array pointer");
  fpc::launch_loss(out, t_true, aux, y_mu, y_sigma, n, w, lam_drift, lam_energy, eps2_hat, scale, dout, dout_bf16,
                   loss_sum, (cudaStream_t)stream);
  return check_launch("loss");
}

size_t fp_mlp_backward_workspace_bytes(int64_t n) { return n > 0 ? fpc::mlp_backward_ws(n) : 0; }

int fp_mlp_backward(const fp_mlp *net, const void *x, const void *h_save, const float *z_save,
                    const void *dout_bf16, const float *dout, int64_t n, float *grads, void *ws, size_t ws_bytes,
                    fp_stream_t stream) {
  g_err[0] = 0;
  if (int rc = check_net(net)) return rc;
  if (n < 0) return fail(FP_ERR_ARG, "negative size");
  if (n == 0) return FP_OK;
  if (!x || !h_save || !z_save || !dout_bf16 || !dout || !grads) return fail(FP_ERR_ARG, "null array pointer");
  const size_t need = fpc::mlp_backward_ws(n);
  if (!ws || ws_bytes < need) return fail(FP_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
  if ((uintptr_t)ws % kAlign) return fail(FP_ERR_ARG, "workspace not 256-byte aligned");
  if (fpc::launch_mlp_backward(*net, x, h_save, z_save, dout_bf16, dout, n, grads, ws, (cudaStream_t)stream))
    return fail(FP_ERR_CUDA, "mlp_backward: shared-memory limit could not be raised");
  return check_launch("mlp_backward");
}

int fp_adam_step(float *params, const float *grads, float *m, float *v, int64_t n_params, float lr, float beta1,
                 float beta2, float eps, int64_t t, void *shadow_bf16, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_params < 0 || t < 1) return fail(FP_ERR_ARG, "n_params < 0 or t < 1");
  if (n_params == 0) return FP_OK;
  if (!params || !grads || !m || !v) return fail(FP_ERR_ARG, "null array pointer");
  const float bc1 = (float)(1.0 - pow((double)beta1, (double)t));
  const float bc2 = (float)(1.0 - pow((double)beta2, (double)t));
  fpc::launch_adam(params, grads, m, v, n_params, lr, beta1, beta2, eps, bc1, bc2, shadow_bf16, (cudaStream_t)stream);
  return check_launch("adam");
}

size_t fp_surrogate_train_step_workspace_bytes(int64_t n) { return n > 0 ? fpc::train_step_ws(n) : 0; }

int fp_surrogate_train_step(const fp_mlp *net, const void *x, const float *t_true, const float *aux, int64_t n,
                            const float *w, float lam_drift, float lam_energy, float scale, float *params,
                            float *grads, float *m, float *v, int64_t n_params, float lr, float beta1, float beta2,
                            float eps, int64_t t, void *shadow_bf16, float *loss_sum, void *ws, size_t ws_bytes,
                            fp_stream_t stream) {
  g_err[0] = 0;
  if (int rc = check_net(net)) return rc;
  if (n < 0 || t < 1) return fail(FP_ERR_ARG, "n < 0 or t < 1");
  if (n_params != fpc::mlp_param_count())
    return fail(FP_ERR_ARG, "n_params %lld is not fp_mlp_param_count()", (long long)n_params);
  if (n == 0) return FP_OK;
  if (!x || !t_true || !aux || !w || !params || !grads || !m || !v || !loss_sum)
    return fail(FP_ERR_ARG, "null array pointer");
  if ((uintptr_t)x % 16) return fail(FP_ERR_ARG, "misaligned x");
  const size_t need = fpc::train_step_ws(n);
  if (!ws || ws_bytes < need) return fail(FP_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
  if ((uintptr_t)ws % kAlign) return fail(FP_ERR_ARG, "workspace not 256-byte aligned");
  const float bc1 = (float)(1.0 - pow((double)beta1, (double)t));
  const float bc2 = (float)(1.0 - pow((double)beta2, (double)t));
  const fpc::AdamParams adam{params, m, v, reinterpret_cast<__nv_bfloat16 *>(shadow_bf16), lr, beta1, beta2, eps,
                             bc1, bc2};
  if (fpc::launch_train_step(*net, x, t_true, aux, n, w, lam_drift, lam_energy, scale, grads, adam, loss_sum, ws,
                             (cudaStream_t)stream))
    return fail(FP_ERR_CUDA, "train_step: shared-memory limit could not be raised");
  return check_launch("train_step");
}

int fp_diagnostics(const double *moments, const double *m6, const double *rho, int64_t n_cells, double theta_inf,
                   double rho_inf, double dg_inf, double *out, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (!moments || !m6 || !out) return fail(FP_ERR_ARG, "null array pointer");
  if (!(theta_inf > 0.0) || !(rho_inf > 0.0)) return fail(FP_ERR_ARG, "theta_inf and rho_inf must be positive");
  fpc::launch_diagnostics(moments, m6, rho, n_cells, theta_inf, rho_inf, dg_inf, out, (cudaStream_t)stream);
  return check_launch("diagnostics");
}

int fp_coeffs_relax(const double *coeffs_new, double *coeffs_prev, int64_t n_cells, double w, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (!coeffs_new || !coeffs_prev) return fail(FP_ERR_ARG, "null array pointer");
  if (!(w >= 0.0 && w <= 1.0)) return fail(FP_ERR_ARG, "w must lie in [0, 1]");
  fpc::launch_relax(coeffs_new, coeffs_prev, n_cells * 9, w, (cudaStream_t)stream);
  return check_launch("relax");
}

int fp_moments_lite(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets, int64_t n_cells,
                    double *lite_out, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0 || n_particles < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return fail(FP_ERR_ARG, "v_dtype %d", v_dtype);
  if (!cell_offsets || !lite_out) return fail(FP_ERR_ARG, "null array pointer");
  if (n_particles > 0 && !v) return fail(FP_ERR_ARG, "null velocity pointer");
  fpc::launch_gather_lite(v, v_dtype, n_particles, cell_offsets, n_cells, lite_out, (cudaStream_t)stream);
  return check_launch("gather_lite");
}

int fp_surrogate_lite_features(const fp_mlp *net, const double *lite, int64_t n_cells, const double *tau,
                               const fp_params *p, void *x_out, int32_t *flags_out, fp_stream_t stream) {
  g_err[0] = 0;
  if (int rc = check_net(net)) return rc;
  if (n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (!lite || !tau || !x_out || !flags_out) return fail(FP_ERR_ARG, "null array pointer");
  if ((uintptr_t)x_out % 16) return fail(FP_ERR_ARG, "features not 16-byte aligned");
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  fpc::launch_lite_features(*net, lite, tau, n_cells, prm.min_particles, prm.surr_range_margin, x_out, flags_out,
                            (cudaStream_t)stream);
  return check_launch("lite_features");
}

size_t fp_surrogate_lite_workspace_bytes(int64_t n_cells) {
  (void)n_cells;
  return 0;  // the fused kernel needs none
}

int fp_closure_surrogate_lite(const fp_mlp *net, const double *lite, int64_t n_cells, const double *tau,
                              const fp_params *p, double *coeffs_out, int32_t *flags_out, void *ws, size_t ws_bytes,
                              fp_stream_t stream) {
  g_err[0] = 0;
  (void)ws;
  (void)ws_bytes;
  if (int rc = check_net(net)) return rc;
  if (n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (!lite || !tau || !coeffs_out || !flags_out) return fail(FP_ERR_ARG, "null array pointer");
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  if (fpc::launch_closure_surrogate_lite(*net, lite, tau, n_cells, prm, coeffs_out, flags_out, (cudaStream_t)stream))
    return fail(FP_ERR_CUDA, "could not raise the shared-memory limit of the MLP kernel");
  return check_launch("surrogate_lite");
}

size_t fp_sort_workspace_bytes(int64_t n_particles, int64_t n_cells) {
  if (n_particles < 0 || n_cells < 0) return 0;
  return fpc::sort_workspace_bytes(n_particles, n_cells);
}

namespace {
int check_sort_args(const int32_t *cell_of, int64_t n_particles, int64_t n_cells, const void *v, int v_dtype,
                    const void *v_sorted, const int32_t *perm, const int64_t *offsets) {
  if (n_particles < 0 || n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_particles > 2147483647ll || n_cells > 2147483646ll)
    return fail(FP_ERR_UNSUPPORTED, "sort limited to 2^31 - 1 particles and 2^31 - 2 cells");
  if (!offsets) return fail(FP_ERR_ARG, "null offsets pointer");
  if (n_particles > 0 && (!cell_of || !perm)) return fail(FP_ERR_ARG, "null array pointer");
  if (v) {
    if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return fail(FP_ERR_ARG, "v_dtype %d", v_dtype);
    if (!v_sorted) return fail(FP_ERR_ARG, "null sorted-velocity pointer");
    if (v_sorted == v && n_particles > 0) return fail(FP_ERR_ARG, "v_sorted aliases v");
  }
  return FP_OK;
}
}  // namespace

int fp_sort_by_cell(const int32_t *cell_of, int64_t n_particles, int64_t n_cells, const void *v, int v_dtype,
                    void *v_sorted, int32_t *perm_out, int64_t *cell_offsets_out, void *ws, size_t ws_bytes,
                    fp_stream_t stream) {
  g_err[0] = 0;
  if (int rc = check_sort_args(cell_of, n_particles, n_cells, v, v_dtype, v_sorted, perm_out, cell_offsets_out))
    return rc;
  const size_t need = fpc::sort_workspace_bytes(n_particles, n_cells);
  if (!ws || ws_bytes < need) return fail(FP_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", need, ws_bytes);
  if ((uintptr_t)ws % kAlign) return fail(FP_ERR_ARG, "workspace not 256-byte aligned");
  const cudaStream_t st = (cudaStream_t)stream;
  fpc::launch_sort_by_cell(cell_of, n_particles, n_cells, perm_out, cell_offsets_out, ws, st, nullptr);
  if (v) fpc::launch_gather_sorted(v, v_dtype, n_particles, perm_out, v_sorted, st);
  return check_launch("sort_by_cell");
}

namespace {
struct StepLayout {
  size_t sort, vs, mom, m6, total;
};
StepLayout step_layout(int64_t n_particles, int64_t n_cells, int v_dtype, int lite) {
  StepLayout L{};
  size_t o = align_up(fpc::sort_workspace_bytes(n_particles, n_cells));
  L.vs = o;
  o += align_up((size_t)n_particles * 3 * (v_dtype == FP_V_F64 ? 8 : 4));
  L.mom = o;
  o += align_up((size_t)n_cells * (lite ? FP_NLITE : FP_NMOM) * 8);
  L.m6 = o;
  if (!lite) o += align_up((size_t)n_cells * 8);
  L.total = o;
  return L;
}
}  // namespace

size_t fp_collision_step_workspace_bytes(int64_t n_particles, int64_t n_cells, int v_dtype, int lite) {
  if (n_particles < 0 || n_cells < 0) return 0;
  return step_layout(n_particles, n_cells, v_dtype, lite).total;
}

int fp_collision_step(const int32_t *cell_of, const void *v, int v_dtype, int64_t n_particles, int64_t n_cells,
                      const double *tau, const fp_params *p, int prec, const fp_mlp *net_lite, double dt,
                      uint64_t seed, uint64_t step, void *v_out, int32_t *perm_out, int64_t *cell_offsets_out,
                      double *coeffs_out, int32_t *flags_out, double *moments_out, void *ws, size_t ws_bytes,
                      fp_stream_t stream) {
  g_err[0] = 0;
  if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return fail(FP_ERR_ARG, "v_dtype %d", v_dtype);
  if (n_particles > 0 && !v) return fail(FP_ERR_ARG, "null velocity pointer");
  if (n_particles > 0 && !v_out) return fail(FP_ERR_ARG, "null output velocity pointer");
  if (int rc = check_sort_args(cell_of, n_particles, n_cells, nullptr, v_dtype, nullptr, perm_out, cell_offsets_out))
    return rc;
  if (prec != FP_PREC_FP64 && prec != FP_PREC_FP32_MOMENTS) return fail(FP_ERR_ARG, "prec %d", prec);
  if (n_cells > 0 && (!tau || !coeffs_out || !flags_out)) return fail(FP_ERR_ARG, "null array pointer");
  if (!(dt >= 0.0) || !std::isfinite(dt)) return fail(FP_ERR_ARG, "dt %g", dt);
  const int lite = net_lite != nullptr;
  if (lite)
    if (int rc = check_net(net_lite)) return rc;
  const StepLayout L = step_layout(n_particles, n_cells, v_dtype, lite);
  if (!ws || ws_bytes < L.total)
    return fail(FP_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", L.total, ws_bytes);
  if ((uintptr_t)ws % kAlign) return fail(FP_ERR_ARG, "workspace not 256-byte aligned");
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  if (prm.min_particles < 1) prm.min_particles = 1;
  const cudaStream_t st = (cudaStream_t)stream;
  char *w = (char *)ws;
  void *vs = w + L.vs;
  double *mom = moments_out ? moments_out : (double *)(w + L.mom);
  fpc::launch_sort_by_cell(cell_of, n_particles, n_cells, perm_out, cell_offsets_out, ws, st, nullptr);
  fpc::launch_gather_sorted(v, v_dtype, n_particles, perm_out, vs, st);
  if (int rc = check_launch("sort_by_cell")) return rc;
  if (n_cells > 0) {
    if (!lite) {
      double *m6 = (double *)(w + L.m6);
      fpc::launch_gather(vs, v_dtype, n_particles, cell_offsets_out, n_cells, prec, mom, m6, st);
      fpc::launch_solve(mom, tau, n_cells, prm, prec, coeffs_out, flags_out, nullptr, st);
      fpc::launch_velocity(vs, v_out, v_dtype, n_particles, cell_offsets_out, n_cells, mom, m6, coeffs_out, tau, dt,
                           prm.eps2_hat, nullptr, seed, step, prm.particle_offset, nullptr, flags_out, st);
    } else {
      fpc::launch_gather_lite(vs, v_dtype, n_particles, cell_offsets_out, n_cells, mom, st);
      if (fpc::launch_closure_surrogate_lite(*net_lite, mom, tau, n_cells, prm, coeffs_out, flags_out, st))
        return fail(FP_ERR_CUDA, "could not raise the shared-memory limit of the MLP kernel");
      fpc::launch_velocity_lite(vs, v_out, v_dtype, n_particles, cell_offsets_out, n_cells, mom, coeffs_out, tau, dt,
                                prm.eps2_hat, nullptr, seed, step, prm.particle_offset, nullptr, flags_out, st);
    }
  }
  fpc::launch_copy_tail(vs, v_out, v_dtype, n_particles, cell_offsets_out + n_cells, st);
  return check_launch("collision_step");
}

namespace {
struct SensLayout {
  size_t x, fl, tp, mean, m2, total;
};
SensLayout sens_layout(int64_t n) {
  SensLayout L{};
  size_t o = 0;
  L.x = o;
  o += align_up((size_t)n * 32 * 2);
  L.fl = o;
  o += align_up((size_t)n * 4);
  L.tp = o;
  o += align_up((size_t)n * 16 * 4);
  L.mean = o;
  o += align_up((size_t)n * 9 * 8);
  L.m2 = o;
  o += align_up((size_t)n * 9 * 8);
  L.total = o;
  return L;
}
}  // namespace

size_t fp_surrogate_sensitivity_workspace_bytes(int64_t n_cells) {
  if (n_cells < 0) return 0;
  return sens_layout(n_cells).total;
}

int fp_surrogate_sensitivity(const fp_mlp *net, const double *moments, int moment_stride, int64_t n_cells,
                             const double *tau, const fp_params *p, int n_passes, double rate, uint64_t seed,
                             double *sens_out, double *mean_out, int32_t *flags_out, void *ws, size_t ws_bytes,
                             fp_stream_t stream) {
  g_err[0] = 0;
  if (int rc = check_net(net)) return rc;
  if (n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (moment_stride != FP_NMOM && moment_stride != FP_NLITE)
    return fail(FP_ERR_ARG, "moment_stride %d (FP_NMOM or FP_NLITE)", moment_stride);
  if (n_passes < 1) return fail(FP_ERR_ARG, "n_passes %d", n_passes);
  if (!(rate >= 0.0 && rate < 1.0)) return fail(FP_ERR_ARG, "rate %g", rate);
  if (n_cells == 0) return FP_OK;
  if (!moments || !tau || !sens_out) return fail(FP_ERR_ARG, "null array pointer");
  const SensLayout L = sens_layout(n_cells);
  if (!ws || ws_bytes < L.total) return fail(FP_ERR_WORKSPACE, "workspace of %zu bytes needed, %zu given", L.total, ws_bytes);
  if ((uintptr_t)ws % kAlign) return fail(FP_ERR_ARG, "workspace not 256-byte aligned");
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  if (prm.min_particles < 1) prm.min_particles = 1;
  const cudaStream_t st = (cudaStream_t)stream;
  char *w = (char *)ws;
  void *x = w + L.x;
  int32_t *fl = flags_out ? flags_out : (int32_t *)(w + L.fl);
  float *tp = (float *)(w + L.tp);
  double *mean = (double *)(w + L.mean), *m2 = (double *)(w + L.m2);
  if (moment_stride == FP_NMOM)
    fpc::launch_features(*net, moments, tau, n_cells, prm.min_particles, prm.surr_range_margin, x, fl, st);
  else
    fpc::launch_lite_features(*net, moments, tau, n_cells, prm.min_particles, prm.surr_range_margin, x, fl, st);
  cudaMemsetAsync(mean, 0, (size_t)n_cells * 9 * 8, st);
  cudaMemsetAsync(m2, 0, (size_t)n_cells * 9 * 8, st);
  for (int k = 0; k < n_passes; ++k) {
    if (fpc::launch_mlp_forward_dropout(*net, x, n_cells, tp, rate, seed, (uint32_t)k, st))
      return fail(FP_ERR_CUDA, "could not raise the shared-memory limit of the MLP kernel");
    fpc::launch_sens_accumulate(tp, n_cells, k + 1, mean, m2, st);
  }
  fpc::launch_sens_finalize(mean, m2, moments, moment_stride, tau, n_cells, n_passes, fl, sens_out, mean_out, st);
  return check_launch("surrogate_sensitivity");
}

int fp_selftest_wait_timeout(uint64_t limit_ns, int32_t *status_out, uint64_t *waited_ns_out, fp_stream_t stream) {
  if (!status_out || !waited_ns_out) return fail(FP_ERR_ARG, "null pointer");
  if (limit_ns == 0 || limit_ns > 1000000000ull) return fail(FP_ERR_ARG, "limit %llu ns outside (0, 1 s]",
                                                             (unsigned long long)limit_ns);
  fpc::launch_wait_timeout(limit_ns, status_out, waited_ns_out, (cudaStream_t)stream);
  return check_launch("selftest_wait_timeout");
}

}  // extern "C"
