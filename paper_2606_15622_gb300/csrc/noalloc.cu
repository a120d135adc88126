// noalloc.cu -- fp_closure_exact_static: the exact closure for callers that
// cannot allocate device memory.
//
// Some callers are not allowed to allocate GPU memory at all: a solver plugin
// living inside a host application that owns the device memory budget, or a
// time-critical step loop where cudaMalloc (which may synchronise the device
// and has unbounded latency) is forbidden.  fp_closure_exact needs scratch
// for the per-cell moments whenever the caller does not want them returned;
// this variant keeps that scratch in a fixed array compiled into the library
// instead, so the caller passes only its inputs and outputs.
//
// The array holds the moment vectors of at most FP_STATIC_MAX_CELLS cells
// (7.9 MB).  It is a file-scope __device__ array: every GPU that loads the
// library keeps it for the life of the process.  Host code cannot use the
// symbol itself as a device address, so its address is looked up with
// cudaGetSymbolAddress once per device, with that device current, on the
// first call made on it.
#include <cstdint>
#include <cstdio>
#include <mutex>

#include "fp_device.cuh"

namespace fpc {
void launch_gather(const void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, int prec,
                   double *mom, double *m6, cudaStream_t st);
void launch_solve(const double *mom, const double *tau, int64_t n_cells, const fp_params &p, int prec,
                  double *coeffs, int32_t *flags, double *lu, cudaStream_t st);
}  // namespace fpc

namespace {

static __device__ __align__(256) double g_static_moments[(size_t)FP_STATIC_MAX_CELLS * FP_NMOM];

constexpr int kMaxDevices = 64;
std::mutex g_lookup_mutex;
double *g_scratch_of_device[kMaxDevices] = {};

thread_local char g_static_err[256] = "";

int static_fail(int code, const char *msg) {
  snprintf(g_static_err, sizeof g_static_err, "%s", msg);
  return code;
}

// Device address of the scratch array on the current device (looked up on
// the first call per device).  The address belongs to the device's primary
// context.  cudaDeviceReset ends that context; the library's module is then
// loaded again, possibly at another address, and the cached one is stale.
// The header therefore states that a process which resets a device must not
// call this entry point on that device afterwards.
int scratch_address(double **out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices)
    return static_fail(FP_ERR_CUDA, "fp_closure_exact_static: no usable current device");
  std::lock_guard<std::mutex> lock(g_lookup_mutex);
  if (!g_scratch_of_device[dev]) {
    void *ptr = nullptr;
    const cudaError_t e = cudaGetSymbolAddress(&ptr, g_static_moments);
    if (e != cudaSuccess || !ptr)
      return static_fail(FP_ERR_CUDA, "fp_closure_exact_static: cudaGetSymbolAddress of the scratch array failed");
    g_scratch_of_device[dev] = static_cast<double *>(ptr);
  }
  *out = g_scratch_of_device[dev];
  return FP_OK;
}

}  // namespace

extern "C" {

const char *fp_closure_exact_static_error(void) { return g_static_err; }

int fp_closure_exact_static(const void *v, int v_dtype, int64_t n_particles, const int64_t *cell_offsets,
                            int64_t n_cells, const double *tau, const fp_params *p, int prec, double *coeffs_out,
                            int32_t *flags_out, fp_stream_t stream) {
  g_static_err[0] = 0;
  if (n_cells < 0 || n_particles < 0) return static_fail(FP_ERR_ARG, "negative size");
  if (n_cells > FP_STATIC_MAX_CELLS)
    return static_fail(FP_ERR_ARG,
                       "fp_closure_exact_static: n_cells exceeds FP_STATIC_MAX_CELLS (32768); split the call or "
                       "use fp_closure_exact with a workspace");
  if (n_cells == 0) return FP_OK;
  if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return static_fail(FP_ERR_ARG, "bad v_dtype");
  if (prec != FP_PREC_FP64 && prec != FP_PREC_FP32_MOMENTS) return static_fail(FP_ERR_ARG, "bad prec");
  if (!cell_offsets || !tau || !coeffs_out || !flags_out) return static_fail(FP_ERR_ARG, "null array pointer");
  if (n_particles > 0 && !v) return static_fail(FP_ERR_ARG, "null velocity pointer");
  double *scratch = nullptr;
  if (int rc = scratch_address(&scratch)) return rc;
  fp_params prm;
  fp_default_params(&prm);
  if (p) prm = *p;
  if (prm.min_particles < 1) prm.min_particles = 1;
  const cudaStream_t st = (cudaStream_t)stream;
  // the gather writes every slot of cells [0, n_cells) before the solve
  // reads them, so the scratch needs no clearing between calls
  fpc::launch_gather(v, v_dtype, n_particles, cell_offsets, n_cells, prec, scratch, nullptr, st);
  // a gather that failed to launch left another call's moments in the array:
  // stop before the solve reads them into the caller's outputs
  cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(FP_ERR_CUDA, cudaGetErrorString(e));
  fpc::launch_solve(scratch, tau, n_cells, prm, prec, coeffs_out, flags_out, nullptr, st);
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_fail(FP_ERR_CUDA, cudaGetErrorString(e));
  return FP_OK;
}

}  // extern "C"
