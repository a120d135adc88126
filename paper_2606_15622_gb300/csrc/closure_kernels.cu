// closure_kernels.cu -- moment gather and 9x9 assembly + pivoted solve
// (paper Sec. 3.6-3.7) for sm_103a.
//
// Kernel 1 (gather): a group of G lanes per cell, static round-robin over the
// cells.  Each group makes two passes over its cell's particles (contiguous,
// coalesced loads of the SoA arrays):
//   pass A  mean offset m and spread from the first particle v0;
//   pass B  the 25 central sums (u_ij, u_ijk, |c|^2 c_i c_j, |c|^4 c_i) and
//           <|c|^6> (which the velocity update's <N.N> needs).
// FP32 mode centres on v0 + m and scales by a power of two s ~ 1/sqrt(theta)
// (exact scaling), accumulates short blocks in FP32 and folds the blocks with
// two-sum; the group reduction is a compensated reduce-scatter.  FP64 mode
// accumulates plain FP64 sums about the exact mean.  The second pass re-reads
// the cell from L1/L2, so DRAM traffic stays one read of the velocities.
//
// Kernel 2 (solve): one THREAD per cell.  GB300's FP64 pipe issues one warp
// instruction every ~16 cycles per SM whatever the active mask, so idle lanes
// of a warp-per-cell layout would waste FP64 issue slots; a thread per cell
// keeps every FP64 lane busy.  The augmented 9x10 matrix lives in registers;
// partial pivoting compares |a| as integers (bit patterns of non-negative
// doubles order like the values) and swaps rows with selects, so the FP64
// pipe only sees the elimination itself.
#include <cstdint>

#include "closure_math.cuh"
#include "fp_device.cuh"

namespace fpc {

// ---------------------------------------------------------------------------
// gather
// ---------------------------------------------------------------------------
__device__ __forceinline__ void accumulate26(float (&t)[kNSum], float wx, float wy, float wz) {
  const float xx = wx * wx, xy = wx * wy, xz = wx * wz, yy = wy * wy, yz = wy * wz, zz = wz * wz;
  t[0] += xx; t[1] += xy; t[2] += xz; t[3] += yy; t[4] += yz; t[5] += zz;
  t[6] = fmaf(xx, wx, t[6]);  t[7] = fmaf(xx, wy, t[7]);   t[8] = fmaf(xx, wz, t[8]);
  t[9] = fmaf(xy, wy, t[9]);  t[10] = fmaf(xy, wz, t[10]); t[11] = fmaf(xz, wz, t[11]);
  t[12] = fmaf(yy, wy, t[12]); t[13] = fmaf(yy, wz, t[13]); t[14] = fmaf(yz, wz, t[14]);
  t[15] = fmaf(zz, wz, t[15]);
  const float r2 = xx + yy + zz;
  t[16] = fmaf(r2, xx, t[16]); t[17] = fmaf(r2, xy, t[17]); t[18] = fmaf(r2, xz, t[18]);
  t[19] = fmaf(r2, yy, t[19]); t[20] = fmaf(r2, yz, t[20]); t[21] = fmaf(r2, zz, t[21]);
  const float r4 = r2 * r2;
  t[22] = fmaf(r4, wx, t[22]); t[23] = fmaf(r4, wy, t[23]); t[24] = fmaf(r4, wz, t[24]);
  t[25] = fmaf(r4, r2, t[25]);
}

__device__ __forceinline__ void accumulate26d(double (&t)[32], double cx, double cy, double cz) {
  const double xx = cx * cx, xy = cx * cy, xz = cx * cz, yy = cy * cy, yz = cy * cz, zz = cz * cz;
  t[0] += xx; t[1] += xy; t[2] += xz; t[3] += yy; t[4] += yz; t[5] += zz;
  t[6] = fma(xx, cx, t[6]);  t[7] = fma(xx, cy, t[7]);   t[8] = fma(xx, cz, t[8]);
  t[9] = fma(xy, cy, t[9]);  t[10] = fma(xy, cz, t[10]); t[11] = fma(xz, cz, t[11]);
  t[12] = fma(yy, cy, t[12]); t[13] = fma(yy, cz, t[13]); t[14] = fma(yz, cz, t[14]);
  t[15] = fma(zz, cz, t[15]);
  const double r2 = xx + yy + zz;
  t[16] = fma(r2, xx, t[16]); t[17] = fma(r2, xy, t[17]); t[18] = fma(r2, xz, t[18]);
  t[19] = fma(r2, yy, t[19]); t[20] = fma(r2, yz, t[20]); t[21] = fma(r2, zz, t[21]);
  const double r4 = r2 * r2;
  t[22] = fma(r4, cx, t[22]); t[23] = fma(r4, cy, t[23]); t[24] = fma(r4, cz, t[24]);
  t[25] = fma(r4, r2, t[25]);
}

template <typename VT>
__device__ __forceinline__ float as_f32(VT x) { return (float)x; }

// Lane-held slots -> moments[5 + q] (q < 25) and m6[c] (q = 25, if m6 is
// given); lane lg of the group owns slots [lg*K, lg*K + K).  theta needs u11,
// u22, u33 (slots 0, 3, 5): fetched from their owners by shuffles executed by
// every lane.
template <int G>
__device__ __forceinline__ void store_moments(double (&val)[32 / G], bool valid, int lane, int64_t c, int n,
                                              double U0, double U1, double U2, double *__restrict__ mom,
                                              double *__restrict__ m6) {
  constexpr int K = 32 / G;
  const int lg = lane & (G - 1);
  const int gbase = lane & ~(G - 1);
  const double u11 = __shfl_sync(0xffffffffu, val[0 % K], gbase + 0 / K);
  const double u22 = __shfl_sync(0xffffffffu, val[3 % K], gbase + 3 / K);
  const double u33 = __shfl_sync(0xffffffffu, val[5 % K], gbase + 5 / K);
  if (!valid) return;
  double *mo = mom + c * FP_NMOM;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int q = lg * K + j;
    if (q < kNMomSum) mo[kU2 + q] = val[j];
    if (q == kM6Sum && m6) m6[c] = val[j];
  }
  if (lg == 0) {
    mo[kN] = (double)n;
    mo[kU + 0] = U0;
    mo[kU + 1] = U1;
    mo[kU + 2] = U2;
    mo[kTheta] = (u11 + u22 + u33) * (1.0 / 3.0);
  }
}

template <typename VT, int G>
__global__ void __launch_bounds__(256) gather_fp32_kernel(const VT *__restrict__ v, int64_t np,
                                                          const int64_t *__restrict__ off, int64_t n_cells,
                                                          double *__restrict__ mom, double *__restrict__ m6) {
  constexpr int GPW = 32 / G;
  constexpr int K = 32 / G;
  constexpr int BLK = 8;  // particles per lane accumulated plainly before a two-sum fold
  const int lane = threadIdx.x & 31;
  const int lg = lane & (G - 1);
  const int g = lane / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const VT *vx = v, *vy = v + np, *vz = v + 2 * np;

  for (int64_t base = warp * GPW; base < n_cells; base += nwarps * GPW) {
    const int64_t c = base + g;
    const bool valid = c < n_cells;
    int64_t a = 0, e = 0;
    if (valid) {
      a = off[c];
      e = off[c + 1];
    }
    const int n = (int)(e - a);
    float v0x = 0.f, v0y = 0.f, v0z = 0.f;
    if (n > 0) {
      v0x = as_f32(vx[a]);
      v0y = as_f32(vy[a]);
      v0z = as_f32(vz[a]);
    }
    const int itmax = __reduce_max_sync(0xffffffffu, (n + G - 1) / G);

    // pass A: offsets from v0
    float sx = 0.f, sy = 0.f, sz = 0.f, sq = 0.f;
    for (int it = 0; it < itmax; ++it) {
      const int64_t p = a + (int64_t)it * G + lg;
      if (p < e) {
        const float dx = as_f32(ldg_v(vx + p)) - v0x;
        const float dy = as_f32(ldg_v(vy + p)) - v0y;
        const float dz = as_f32(ldg_v(vz + p)) - v0z;
        sx += dx;
        sy += dy;
        sz += dz;
        sq = fmaf(dx, dx, fmaf(dy, dy, fmaf(dz, dz, sq)));
      }
    }
    sx = group_allreduce<G>(sx);
    sy = group_allreduce<G>(sy);
    sz = group_allreduce<G>(sz);
    sq = group_allreduce<G>(sq);
    const float inv_n = n > 0 ? 1.f / (float)n : 0.f;
    const float mx = sx * inv_n, my = sy * inv_n, mz = sz * inv_n;
    const float th_est = (sq * inv_n - (mx * mx + my * my + mz * mz)) * (1.f / 3.f);
    // power-of-two scale s = 2^ks ~ 1/sqrt(theta): exact in floating point
    int ks = 0;
    if (th_est > 0.f) {
      int ex;
      frexpf(th_est, &ex);
      ks = -(ex / 2);
    }
    const float s = ldexpf(1.f, ks);

    // pass B: centred, scaled sums; FP32 blocks folded by two-sum
    float hi[32], lo[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) {
      hi[q] = 0.f;
      lo[q] = 0.f;
    }
    for (int it0 = 0; it0 < itmax; it0 += BLK) {
      float t[kNSum];
#pragma unroll
      for (int q = 0; q < kNSum; ++q) t[q] = 0.f;
      const int itend = min(it0 + BLK, itmax);
      for (int it = it0; it < itend; ++it) {
        const int64_t p = a + (int64_t)it * G + lg;
        if (p < e) {
          const float wx = ((as_f32(ldg_v(vx + p)) - v0x) - mx) * s;
          const float wy = ((as_f32(ldg_v(vy + p)) - v0y) - my) * s;
          const float wz = ((as_f32(ldg_v(vz + p)) - v0z) - mz) * s;
          accumulate26(t, wx, wy, wz);
        }
      }
      if (it0 == 0) {
#pragma unroll
        for (int q = 0; q < kNSum; ++q) hi[q] = t[q];
      } else {
#pragma unroll
        for (int q = 0; q < kNSum; ++q) {
          float sum, err;
          two_sum(hi[q], t[q], sum, err);
          hi[q] = sum;
          lo[q] += err;
        }
      }
    }
    group_reduce_scatter2<G>(hi, lo, lane);

    // promote to FP64 and undo the scaling: order-k sums carry s^k
    const double inv_nd = n > 0 ? 1.0 / (double)n : 0.0;
    double val[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      const int q = lg * K + j;
      const int ord = q < kNSum ? sum_order(q) : 0;
      const double fac = ldexp(inv_nd, -ks * ord);
      val[j] = ((double)hi[j] + (double)lo[j]) * fac;
    }
    const double U0 = (double)v0x + (double)mx, U1 = (double)v0y + (double)my, U2 = (double)v0z + (double)mz;
    store_moments<G>(val, valid, lane, c, n, U0, U1, U2, mom, m6);
  }
}

template <typename VT, int G>
__global__ void __launch_bounds__(256) gather_fp64_kernel(const VT *__restrict__ v, int64_t np,
                                                          const int64_t *__restrict__ off, int64_t n_cells,
                                                          double *__restrict__ mom, double *__restrict__ m6) {
  constexpr int GPW = 32 / G;
  constexpr int K = 32 / G;
  const int lane = threadIdx.x & 31;
  const int lg = lane & (G - 1);
  const int g = lane / G;
  const int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  const int64_t nwarps = ((int64_t)gridDim.x * blockDim.x) >> 5;
  const VT *vx = v, *vy = v + np, *vz = v + 2 * np;

  for (int64_t base = warp * GPW; base < n_cells; base += nwarps * GPW) {
    const int64_t c = base + g;
    const bool valid = c < n_cells;
    int64_t a = 0, e = 0;
    if (valid) {
      a = off[c];
      e = off[c + 1];
    }
    const int n = (int)(e - a);
    const int itmax = __reduce_max_sync(0xffffffffu, (n + G - 1) / G);
    double sx = 0.0, sy = 0.0, sz = 0.0;
    for (int it = 0; it < itmax; ++it) {
      const int64_t p = a + (int64_t)it * G + lg;
      if (p < e) {
        sx += (double)ldg_v(vx + p);
        sy += (double)ldg_v(vy + p);
        sz += (double)ldg_v(vz + p);
      }
    }
    sx = group_allreduce<G>(sx);
    sy = group_allreduce<G>(sy);
    sz = group_allreduce<G>(sz);
    const double inv_nd = n > 0 ? 1.0 / (double)n : 0.0;
    const double Ux = sx * inv_nd, Uy = sy * inv_nd, Uz = sz * inv_nd;
    double t[32];
#pragma unroll
    for (int q = 0; q < 32; ++q) t[q] = 0.0;
    for (int it = 0; it < itmax; ++it) {
      const int64_t p = a + (int64_t)it * G + lg;
      if (p < e)
        accumulate26d(t, (double)ldg_v(vx + p) - Ux, (double)ldg_v(vy + p) - Uy, (double)ldg_v(vz + p) - Uz);
    }
    group_reduce_scatter<G>(t, lane);
    double val[K];
#pragma unroll
    for (int j = 0; j < K; ++j) val[j] = t[j] * inv_nd;
    store_moments<G>(val, valid, lane, c, n, Ux, Uy, Uz, mom, m6);
  }
}

// ---------------------------------------------------------------------------
// assembly + solve (closure_math.cuh)
// ---------------------------------------------------------------------------
// One thread per cell, grid-stride over two resident 128-thread blocks per SM;
// two warps per SM sub-partition keep its FP64 unit busy through each
// other's dependency stalls.  The registers are capped at 168 a thread (some
// of the 9 x 10 system spills to L1): alone the kernel is as fast as with
// the whole register file, and the third of the file it leaves free lets the
// learned closure's kernels run beside it in the step.  With kLU the factors
// of P A = L U of every unflagged cell go to lu for the adjoint.
template <bool kLU, bool kMixed = false>
__global__ void __launch_bounds__(128, 3) solve_kernel(const double *__restrict__ mom, const double *__restrict__ tau,
                                                       int64_t n_cells, SolveParams prm, double *__restrict__ coeffs,
                                                       int32_t *__restrict__ flags, double *__restrict__ lu) {
  for (int64_t c = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; c < n_cells;
       c += (int64_t)gridDim.x * blockDim.x) {
    double y[9];
    const int fl = kMixed ? closure_cell_mixed(mom + c * FP_NMOM, tau[c], prm, y)
                          : closure_cell<kLU>(mom + c * FP_NMOM, tau[c], prm, y, kLU ? lu + lu_base(c) : nullptr);
    double *yc = coeffs + c * 9;
#pragma unroll
    for (int q = 0; q < 9; ++q) yc[q] = y[q];
    flags[c] = fl;
  }
}

// ---------------------------------------------------------------------------
// launchers
// ---------------------------------------------------------------------------
static int sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

template <int G>
static void launch_gather_t(const void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, int prec,
                            double *mom, double *m6, cudaStream_t st) {
  const int threads = 256;
  const int64_t groups_per_block = (threads / 32) * (32 / G);
  int64_t blocks = (n_cells + groups_per_block - 1) / groups_per_block;
  const int64_t cap = (int64_t)sm_count() * 8;
  if (blocks > cap) blocks = cap;
  if (blocks < 1) blocks = 1;
  if (prec == FP_PREC_FP32_MOMENTS) {
    if (v_dtype == FP_V_F32)
      gather_fp32_kernel<float, G><<<(unsigned)blocks, threads, 0, st>>>((const float *)v, np, off, n_cells, mom, m6);
    else
      gather_fp32_kernel<double, G><<<(unsigned)blocks, threads, 0, st>>>((const double *)v, np, off, n_cells, mom,
                                                                          m6);
  } else {
    if (v_dtype == FP_V_F32)
      gather_fp64_kernel<float, G><<<(unsigned)blocks, threads, 0, st>>>((const float *)v, np, off, n_cells, mom, m6);
    else
      gather_fp64_kernel<double, G><<<(unsigned)blocks, threads, 0, st>>>((const double *)v, np, off, n_cells, mom,
                                                                          m6);
  }
}

bool launch_gather_tile(const float *v, int64_t np, const int64_t *off, int64_t n_cells, double *mom, double *m6,
                        cudaStream_t st, int sm_count);

void launch_gather(const void *v, int v_dtype, int64_t np, const int64_t *off, int64_t n_cells, int prec,
                   double *mom, double *m6, cudaStream_t st) {
  // FP32 moments of FP32 velocities: shared-memory staged tiles (16-byte
  // aligned velocity arrays); every other combination: direct loads.
  if (prec == FP_PREC_FP32_MOMENTS && v_dtype == FP_V_F32 &&
      launch_gather_tile((const float *)v, np, off, n_cells, mom, m6, st, sm_count()))
    return;
  launch_gather_t<8>(v, v_dtype, np, off, n_cells, prec, mom, m6, st);
}

void launch_solve(const double *mom, const double *tau, int64_t n_cells, const fp_params &p, int prec,
                  double *coeffs, int32_t *flags, double *lu, cudaStream_t st) {
  double rtol = p.pivot_rtol;
  if (prec == FP_PREC_FP32_MOMENTS && rtol < FP_FP32_PIVOT_FLOOR) rtol = FP_FP32_PIVOT_FLOOR;
  SolveParams prm{p.eps2_hat, rtol, p.min_particles, prec == FP_PREC_FP32_MOMENTS ? FP_FP32_MIN_REGULAR : 0};
  const int threads = 128;
  int64_t blocks = (n_cells + threads - 1) / threads;
  if (blocks > 2 * sm_count()) blocks = 2 * sm_count();
  if (lu)
    solve_kernel<true><<<(unsigned)blocks, threads, 0, st>>>(mom, tau, n_cells, prm, coeffs, flags, lu);
  else if (prec == FP_PREC_FP32_MOMENTS)  // FP32-accurate moments: the mixed-precision solve
    solve_kernel<false, true><<<(unsigned)blocks, threads, 0, st>>>(mom, tau, n_cells, prm, coeffs, flags, nullptr);
  else
    solve_kernel<false><<<(unsigned)blocks, threads, 0, st>>>(mom, tau, n_cells, prm, coeffs, flags, nullptr);
}

}  // namespace fpc
