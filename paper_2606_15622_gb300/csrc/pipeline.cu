// pipeline.cu -- fp_step_host: one step of the hot path on velocities held
// in host memory, with the host <-> device copies overlapped with the work.
//
// The cells are split into contiguous chunks (cells are independent, so a
// chunk is the closure problem of its own cells).  The offsets and tau of all
// cells go first (two copies), the coefficients and flags of all cells last;
// for every chunk, on five streams ordered by events:
//   copy-in  (H2D)   velocities of the chunk's particles (the three
//                    components in one strided copy)
//   main     (high priority) gather -> solve (keeping its factors for the
//            adjoint when asked)
//   adjoint  [adjoint]                                after the solve
//   learned  [surrogate closure]                    after the gather
//   update   flags copy, velocity update M^n -> M^{n+1}  after the solve
//   copy-out (D2H)   updated velocities (one strided copy)
// so chunk k's copies overlap the compute of its neighbours.  Few large
// copies keep the host link busy in both directions: every copy costs a
// few microseconds of setup on its engine.  Each chunk's
// calls are the public entry points on slices of caller-owned, full-size
// device arrays: offsets stay absolute particle indices, the Philox counter
// of a particle is its global index, and the results are those of the
// unchunked calls.
#include <cstdint>
#include <new>

#include "fp_device.cuh"

namespace fpc {
int report(int code, const char *msg);
}

struct fp_pipeline {
  static constexpr int kMaxChunks = 64;
  cudaStream_t h2d = nullptr, main = nullptr, sur = nullptr, vel = nullptr, d2h = nullptr, adj = nullptr;
  cudaEvent_t start = nullptr;
  cudaEvent_t ev_h2d[kMaxChunks] = {}, ev_mom[kMaxChunks] = {}, ev_solve[kMaxChunks] = {}, ev_vel[kMaxChunks] = {};
  cudaEvent_t done_main = nullptr, done_sur = nullptr, done_vel = nullptr, done_d2h = nullptr, done_adj = nullptr;
};

namespace {

int destroy_all(fp_pipeline *pl) {
  cudaStream_t *ss[6] = {&pl->h2d, &pl->main, &pl->sur, &pl->vel, &pl->d2h, &pl->adj};
  for (cudaStream_t *s : ss)
    if (*s) cudaStreamDestroy(*s);
  cudaEvent_t *es[6] = {&pl->start, &pl->done_main, &pl->done_sur, &pl->done_vel, &pl->done_d2h, &pl->done_adj};
  for (cudaEvent_t *e : es)
    if (*e) cudaEventDestroy(*e);
  for (int k = 0; k < fp_pipeline::kMaxChunks; ++k) {
    if (pl->ev_h2d[k]) cudaEventDestroy(pl->ev_h2d[k]);
    if (pl->ev_mom[k]) cudaEventDestroy(pl->ev_mom[k]);
    if (pl->ev_solve[k]) cudaEventDestroy(pl->ev_solve[k]);
    if (pl->ev_vel[k]) cudaEventDestroy(pl->ev_vel[k]);
  }
  delete pl;
  return 0;
}

inline size_t vbytes(int v_dtype) { return v_dtype == FP_V_F32 ? 4 : 8; }

}  // namespace

extern "C" {

int fp_pipeline_create(fp_pipeline **out) {
  if (!out) return fpc::report(FP_ERR_ARG, "fp_pipeline_create: null output pointer");
  *out = nullptr;
  fp_pipeline *pl = new (std::nothrow) fp_pipeline;
  if (!pl) return fpc::report(FP_ERR_CUDA, "fp_pipeline_create: out of host memory");
  int lo = 0, hi = 0;
  bool ok = cudaDeviceGetStreamPriorityRange(&lo, &hi) == cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&pl->main, cudaStreamNonBlocking, hi) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&pl->h2d, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&pl->sur, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&pl->vel, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithFlags(&pl->d2h, cudaStreamNonBlocking) == cudaSuccess;
  ok = ok && cudaStreamCreateWithPriority(&pl->adj, cudaStreamNonBlocking, hi) == cudaSuccess;
  cudaEvent_t *es[6] = {&pl->start, &pl->done_main, &pl->done_sur, &pl->done_vel, &pl->done_d2h, &pl->done_adj};
  for (cudaEvent_t *e : es) ok = ok && cudaEventCreateWithFlags(e, cudaEventDisableTiming) == cudaSuccess;
  for (int k = 0; ok && k < fp_pipeline::kMaxChunks; ++k) {
    ok = ok && cudaEventCreateWithFlags(&pl->ev_h2d[k], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&pl->ev_mom[k], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&pl->ev_solve[k], cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&pl->ev_vel[k], cudaEventDisableTiming) == cudaSuccess;
  }
  if (!ok) {
    cudaGetLastError();
    destroy_all(pl);
    return fpc::report(FP_ERR_CUDA, "fp_pipeline_create: could not create streams or events");
  }
  *out = pl;
  return FP_OK;
}

void fp_pipeline_destroy(fp_pipeline *pl) {
  if (!pl) return;
  // the handle's streams may still hold work: wait for it first
  cudaStreamSynchronize(pl->h2d);
  cudaStreamSynchronize(pl->main);
  cudaStreamSynchronize(pl->sur);
  cudaStreamSynchronize(pl->vel);
  cudaStreamSynchronize(pl->d2h);
  cudaStreamSynchronize(pl->adj);
  destroy_all(pl);
}

int fp_step_host(fp_pipeline *pl, const fp_step_io *io, int v_dtype, int64_t n_particles, int64_t n_cells,
                 const fp_params *p, int prec, double dt, uint64_t seed, uint64_t step, int n_chunks,
                 fp_stream_t stream) {
  if (!pl || !io) return fpc::report(FP_ERR_ARG, "fp_step_host: null pipeline or io");
  if (n_cells < 0 || n_particles < 0) return fpc::report(FP_ERR_ARG, "fp_step_host: negative size");
  if (n_cells == 0) return FP_OK;
  if (v_dtype != FP_V_F32 && v_dtype != FP_V_F64) return fpc::report(FP_ERR_ARG, "fp_step_host: bad v_dtype");
  if (n_chunks < 1 || n_chunks > fp_pipeline::kMaxChunks)
    return fpc::report(FP_ERR_ARG, "fp_step_host: n_chunks must lie in [1, 64]");
  if (!io->h_v || !io->h_v_out || !io->h_offsets || !io->h_tau || !io->h_coeffs || !io->h_flags)
    return fpc::report(FP_ERR_ARG, "fp_step_host: null host buffer");
  if (!io->d_v || !io->d_v_out || !io->d_offsets || !io->d_tau || !io->d_moments || !io->d_coeffs ||
      !io->d_flags || !io->d_flags_v)
    return fpc::report(FP_ERR_ARG, "fp_step_host: null device buffer");
  if (io->d_v == io->d_v_out) return fpc::report(FP_ERR_ARG, "fp_step_host: d_v_out must differ from d_v");
  if (io->net && (!io->d_coeffs_s || !io->d_flags_s || !io->d_surrogate_ws))
    return fpc::report(FP_ERR_ARG, "fp_step_host: learned closure requested without its buffers");
  if (io->d_grad_coeffs && !io->d_grad_moments)
    return fpc::report(FP_ERR_ARG, "fp_step_host: adjoint requested without d_grad_moments");
  if (io->h_offsets[0] != 0 || io->h_offsets[n_cells] != n_particles)
    return fpc::report(FP_ERR_ARG, "fp_step_host: offsets must run from 0 to n_particles");
  if (n_chunks > n_cells) n_chunks = (int)n_cells;

  const size_t sv = vbytes(v_dtype);
  const cudaStream_t caller = (cudaStream_t)stream;
  // everything already queued on the caller's stream comes first
  if (cudaEventRecord(pl->start, caller) != cudaSuccess) return fpc::report(FP_ERR_CUDA, "fp_step_host: event");
  cudaStreamWaitEvent(pl->h2d, pl->start, 0);
  cudaStreamWaitEvent(pl->main, pl->start, 0);
  cudaStreamWaitEvent(pl->sur, pl->start, 0);
  cudaStreamWaitEvent(pl->vel, pl->start, 0);
  cudaStreamWaitEvent(pl->d2h, pl->start, 0);
  cudaStreamWaitEvent(pl->adj, pl->start, 0);

  const char *hv = (const char *)io->h_v;
  char *hvo = (char *)io->h_v_out;
  char *dv = (char *)io->d_v, *dvo = (char *)io->d_v_out;
  const size_t pitch = (size_t)n_particles * sv;  // bytes between velocity components
  cudaMemcpyAsync(io->d_offsets, io->h_offsets, (size_t)(n_cells + 1) * sizeof(int64_t), cudaMemcpyHostToDevice,
                  pl->h2d);
  cudaMemcpyAsync(io->d_tau, io->h_tau, (size_t)n_cells * sizeof(double), cudaMemcpyHostToDevice, pl->h2d);
  int rc = FP_OK;
  for (int k = 0; k < n_chunks && rc == FP_OK; ++k) {
    // chunk boundaries on multiples of 32 cells (the tiles of stored factors)
    const int64_t c0 = k == 0 ? 0 : (n_cells * k / n_chunks) & ~(int64_t)31;
    const int64_t c1 = k == n_chunks - 1 ? n_cells : (n_cells * (k + 1) / n_chunks) & ~(int64_t)31;
    const int64_t nc = c1 - c0;
    if (nc <= 0) continue;
    const int64_t p0 = io->h_offsets[c0], p1 = io->h_offsets[c1];
    if (p0 < 0 || p1 < p0 || p1 > n_particles) {
      rc = fpc::report(FP_ERR_ARG, "fp_step_host: offsets are not non-decreasing");
      break;
    }
    const size_t vb = (size_t)(p1 - p0) * sv;
    // ---- copy in ----
    if (vb) {
      const size_t o = (size_t)p0 * sv;
      cudaMemcpy2DAsync(dv + o, pitch, hv + o, pitch, vb, 3, cudaMemcpyHostToDevice, pl->h2d);
    }
    cudaEventRecord(pl->ev_h2d[k], pl->h2d);
    // ---- closure ----
    cudaStreamWaitEvent(pl->main, pl->ev_h2d[k], 0);
    double *mom = io->d_moments + c0 * FP_NMOM;
    double *m6 = io->d_m6 ? io->d_m6 + c0 : nullptr;
    if ((rc = fp_moments(io->d_v, v_dtype, n_particles, io->d_offsets + c0, nc, prec, mom, m6, pl->main))) break;
    // ---- the learned closure (moments only) beside the FP64 solve ----
    if (io->net) {
      cudaEventRecord(pl->ev_mom[k], pl->main);
      cudaStreamWaitEvent(pl->sur, pl->ev_mom[k], 0);
      if ((rc = fp_closure_surrogate(io->net, mom, nc, io->d_tau + c0, p, prec, io->d_coeffs_s + c0 * 9,
                                     io->d_flags_s + c0, io->d_surrogate_ws, io->surrogate_ws_bytes, pl->sur)))
        break;
    }
    double *lu = io->d_lu ? io->d_lu + (c0 / 32) * 32 * FP_LU_STRIDE : nullptr;
    if ((rc = fp_closure_solve(mom, io->d_tau + c0, nc, p, prec, io->d_coeffs + c0 * 9, io->d_flags + c0,
                               io->d_grad_coeffs ? lu : nullptr, pl->main)))
      break;
    cudaEventRecord(pl->ev_solve[k], pl->main);
    // ---- velocity update and adjoint side by side ----
    cudaStreamWaitEvent(pl->vel, pl->ev_solve[k], 0);
    cudaMemcpyAsync(io->d_flags_v + c0, io->d_flags + c0, (size_t)nc * sizeof(int32_t), cudaMemcpyDeviceToDevice,
                    pl->vel);
    if ((rc = fp_velocity_update(io->d_v, io->d_v_out, v_dtype, n_particles, io->d_offsets + c0, nc, mom, m6,
                                 io->d_coeffs + c0 * 9, io->d_tau + c0, dt, p, nullptr, seed, step, nullptr,
                                 io->d_flags_v + c0, pl->vel)))
      break;
    cudaEventRecord(pl->ev_vel[k], pl->vel);
    if (io->d_grad_coeffs) {  // on its own stream: the next chunk's gather and solve need not wait for it
      cudaStreamWaitEvent(pl->adj, pl->ev_solve[k], 0);
      if ((rc = fp_closure_backward(io->d_v, v_dtype, n_particles, io->d_offsets + c0, nc, io->d_tau + c0, p, mom,
                                    io->d_coeffs + c0 * 9, io->d_flags + c0, lu, io->d_grad_coeffs + c0 * 9, nullptr,
                                    io->d_grad_moments + c0 * FP_NMOM, io->d_grad_v, nullptr, 0, pl->adj)))
        break;
    }
    // ---- copy out ----
    cudaStreamWaitEvent(pl->d2h, pl->ev_vel[k], 0);
    if (vb) {
      const size_t o = (size_t)p0 * sv;
      cudaMemcpy2DAsync(hvo + o, pitch, dvo + o, pitch, vb, 3, cudaMemcpyDeviceToHost, pl->d2h);
    }
  }
  if (rc == FP_OK) {  // every chunk's update has been waited for on the copy-out stream
    cudaMemcpyAsync(io->h_coeffs, io->d_coeffs, (size_t)n_cells * 9 * sizeof(double), cudaMemcpyDeviceToHost,
                    pl->d2h);
    cudaMemcpyAsync(io->h_flags, io->d_flags_v, (size_t)n_cells * sizeof(int32_t), cudaMemcpyDeviceToHost, pl->d2h);
  }
  // the caller's stream resumes after all of it (also after an error, so no
  // queued work outlives the call unordered)
  cudaEventRecord(pl->done_main, pl->main);
  cudaEventRecord(pl->done_sur, pl->sur);
  cudaEventRecord(pl->done_vel, pl->vel);
  cudaEventRecord(pl->done_d2h, pl->d2h);
  cudaEventRecord(pl->done_adj, pl->adj);
  cudaStreamWaitEvent(caller, pl->done_main, 0);
  cudaStreamWaitEvent(caller, pl->done_sur, 0);
  cudaStreamWaitEvent(caller, pl->done_vel, 0);
  cudaStreamWaitEvent(caller, pl->done_d2h, 0);
  cudaStreamWaitEvent(caller, pl->done_adj, 0);
  if (rc) return rc;
  const cudaError_t e = cudaGetLastError();
  if (e != cudaSuccess) return fpc::report(FP_ERR_CUDA, cudaGetErrorString(e));
  return FP_OK;
}

}  // extern "C"
