// api.cu -- the C ABI of libfpclosure.so (declarations and contracts in
// include/fpclosure.h): argument validation, workspace carving, launches.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "fp_device.cuh"

namespace fpc {
void launch_gather(const void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, int prec,
                   double *mom, cudaStream_t st);
void launch_solve(const double *mom, const double *tau, int64_t n_cells, const fp_params &p, int prec,
                  double *coeffs, int32_t *flags, cudaStream_t st);
void launch_velocity(void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, const double *mom,
                     const double *coeffs, const double *tau, double dt, double eps2_hat, const void *xi, uint64_t seed,
                     uint64_t step, double *alpha_out, int32_t *flags, cudaStream_t st);
void launch_adjoint(const void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, const double *tau,
                    double eps2_hat, const double *mom, const double *coeffs, const int32_t *flags, const double *gY,
                    const double *gm_in, double *gm_out, void *gv, cudaStream_t st);
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
}  // namespace

extern "C" {

void fp_default_params(fp_params *p) {
  if (!p) return;
  p->eps2_hat = 1e-3;
  p->min_particles = 4;
  p->pivot_rtol = 1e-13;
  p->surr_energy_tol = 0.05;
  p->surr_range_margin = 0.5;
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
  fpc::launch_gather(v, v_dtype, n_particles, cell_offsets, n_cells, prec, mom, st);
  if (int rc = check_launch("gather")) return rc;
  fpc::launch_solve(mom, tau, n_cells, prm, prec, coeffs_out, flags_out, st);
  return check_launch("solve");
}

int fp_moments(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets, int64_t n_cells,
               int prec, double *moments_out, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0 || n_particles < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return fail(FP_ERR_ARG, "v_dtype %d", v_dtype);
  if (prec != FP_PREC_FP64 && prec != FP_PREC_FP32_MOMENTS) return fail(FP_ERR_ARG, "prec %d", prec);
  if (!cell_offsets || !moments_out) return fail(FP_ERR_ARG, "null array pointer");
  if (n_particles > 0 && !v) return fail(FP_ERR_ARG, "null velocity pointer");
  fpc::launch_gather(v, v_dtype, n_particles, cell_offsets, n_cells, prec, moments_out, (cudaStream_t)stream);
  return check_launch("gather");
}

int fp_closure_solve(const double *moments, const double *tau, int64_t n_cells, const fp_params *p, int prec,
                     double *coeffs_out, int32_t *flags_out, fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (prec != FP_PREC_FP64 && prec != FP_PREC_FP32_MOMENTS) return fail(FP_ERR_ARG, "prec %d", prec);
  if (!moments || !tau || !coeffs_out || !flags_out) return fail(FP_ERR_ARG, "null array pointer");
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  if (prm.min_particles < 1) prm.min_particles = 1;
  fpc::launch_solve(moments, tau, n_cells, prm, prec, coeffs_out, flags_out, (cudaStream_t)stream);
  return check_launch("solve");
}

int fp_velocity_update(void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets, int64_t n_cells,
                       const double *moments, const double *coeffs, const double *tau, double dt, const fp_params *p,
                       const void *xi, uint64_t seed, uint64_t step, double *alpha_out, int32_t *flags,
                       fp_stream_t stream) {
  g_err[0] = 0;
  if (n_cells < 0 || n_particles < 0) return fail(FP_ERR_ARG, "negative size");
  if (n_cells == 0) return FP_OK;
  if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return fail(FP_ERR_ARG, "v_dtype %d", v_dtype);
  if (!cell_offsets || !moments || !coeffs || !tau || !flags) return fail(FP_ERR_ARG, "null array pointer");
  if (n_particles > 0 && !v) return fail(FP_ERR_ARG, "null velocity pointer");
  if (!(dt >= 0.0)) return fail(FP_ERR_ARG, "dt must be >= 0");
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  fpc::launch_velocity(v, v_dtype, n_particles, cell_offsets, n_cells, moments, coeffs, tau, dt, prm.eps2_hat, xi,
                       seed, step, alpha_out, flags, (cudaStream_t)stream);
  return check_launch("velocity");
}

int fp_closure_backward(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                        int64_t n_cells, const double *tau, const fp_params *p, const double *moments,
                        const double *coeffs, const int32_t *flags, const double *grad_coeffs,
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
  fpc::launch_adjoint(v, v_dtype, n_particles, cell_offsets, n_cells, tau, prm.eps2_hat, moments, coeffs, flags,
                      grad_coeffs, grad_moments_in, gm, grad_v, (cudaStream_t)stream);
  return check_launch("adjoint");
}

}  // extern "C"
