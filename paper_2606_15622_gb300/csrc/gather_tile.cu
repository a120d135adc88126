// gather_tile.cu -- FP32-moment gather from FP32 velocities, streamed through
// shared memory by bulk asynchronous copies (paper Sec. 3.6 moments).
//
// Work is cut into chunks of kChunkCells consecutive cells, dealt round-robin
// to persistent CTAs.  Each CTA is warp-specialised:
//   * a producer warp reads the chunk's cell offsets (one coalesced load),
//     splits the chunk into sub-tiles of whole cells holding at most kSubP
//     particles, and streams each sub-tile's three SoA component ranges
//     (widened to 16-byte boundaries) into a ring of kSlots shared-memory
//     slots with cp.async.bulk, completing on the slot's `full` mbarrier;
//   * four consumer warps take the sub-tiles in the same order, reduce two
//     cells per warp (16 lanes per cell) from shared memory, and release the
//     slot on its `empty` mbarrier.
// A cell larger than a sub-tile is reduced by one group straight from global
// memory.  No global-memory round trip sits on a consumer's path; the
// producer runs up to kSlots sub-tiles ahead.
//
// Moments leave through FP32 double-float arithmetic and an integer
// float->double conversion: the FP64 pipe (one warp instruction per ~16 SM
// cycles on GB300) sees ~3 instructions per cell.
#include <cstdint>

#include "fp_device.cuh"
#include "tma.cuh"

namespace fpc {

constexpr int kChunkCells = 64;
constexpr int kSubP = 2048;                  // particles per sub-tile (max)
constexpr int kCapF = kSubP + 8;             // floats per component slot (alignment slack)
constexpr int kSlots = 4;
constexpr int kConsumerWarps = 4;
constexpr int kTileThreads = 32 * (1 + kConsumerWarps);
constexpr int kTileG = 16;                   // lanes per cell
constexpr int kSlotFloats = 3 * kCapF;
constexpr size_t kTileSmem = (size_t)kSlots * kSlotFloats * sizeof(float);

struct SlotMeta {
  int64_t cs, ce;                 // cells [cs, ce) of the sub-tile
  int64_t pa;                     // first particle (offset of cell cs)
  int lead[3];                    // slot index of particle pa, per component
  int big;                        // 1: the single cell cs is reduced from global memory
  int done;                       // 1: no more sub-tiles for this CTA
  int64_t offs[kChunkCells + 1];  // off[cs .. ce]
};

// One cell per 16-lane group, both groups of the warp in lockstep; px/py/pz
// point at the cell's first particle (shared or global memory).
template <bool kShared>
__device__ __forceinline__ void reduce_cell_pair(bool valid, int n, const float *px, const float *py,
                                                 const float *pz, int64_t c, double *__restrict__ mom, int lane) {
  constexpr int G = kTileG;
  constexpr int K = 32 / G;
  constexpr int BLK = 8;
  const int lg = lane & (G - 1);
  auto ld = [](const float *p, int i) -> float {
    if (kShared) return p[i];
    return __ldg(p + i);
  };
  if (!valid) n = 0;
  float v0x = 0.f, v0y = 0.f, v0z = 0.f;
  if (n > 0) {
    v0x = ld(px, 0);
    v0y = ld(py, 0);
    v0z = ld(pz, 0);
  }
  const int itmax = __reduce_max_sync(0xffffffffu, (n + G - 1) / G);
  // pass A: offsets from the first particle
  float sx = 0.f, sy = 0.f, sz = 0.f, sq = 0.f;
  for (int it = 0; it < itmax; ++it) {
    const int i = it * G + lg;
    if (i < n) {
      const float dx = ld(px, i) - v0x, dy = ld(py, i) - v0y, dz = ld(pz, i) - v0z;
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
  float rh = 0.f, rl = 0.f;
  if (n > 0) df_recip((float)n, rh, rl);
  const float mx = sx * rh, my = sy * rh, mz = sz * rh;
  const float th_est = (sq * rh - (mx * mx + my * my + mz * mz)) * (1.f / 3.f);
  int ks = 0;  // power-of-two scale s = 2^ks ~ 1/sqrt(theta): exact
  if (th_est > 0.f) {
    int ex;
    frexpf(th_est, &ex);
    ks = -(ex / 2);
  }
  const float s = ldexpf(1.f, ks);

  // pass B: centred, scaled sums; FP32 blocks of BLK particles per lane folded by two-sum
  float hi[32], lo[32];
#pragma unroll
  for (int q = 0; q < 32; ++q) {
    hi[q] = 0.f;
    lo[q] = 0.f;
  }
  for (int it0 = 0; it0 < itmax; it0 += BLK) {
    float t[25];
#pragma unroll
    for (int q = 0; q < 25; ++q) t[q] = 0.f;
    const int itend = min(it0 + BLK, itmax);
    for (int it = it0; it < itend; ++it) {
      const int i = it * G + lg;
      if (i < n) {
        const float wx = ((ld(px, i) - v0x) - mx) * s;
        const float wy = ((ld(py, i) - v0y) - my) * s;
        const float wz = ((ld(pz, i) - v0z) - mz) * s;
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
      }
    }
    if (it0 == 0) {
#pragma unroll
      for (int q = 0; q < 25; ++q) hi[q] = t[q];
    } else {
#pragma unroll
      for (int q = 0; q < 25; ++q) {
        float sum, err;
        two_sum(hi[q], t[q], sum, err);
        hi[q] = sum;
        lo[q] += err;
      }
    }
  }
  group_reduce_scatter<G>(hi, lane);
  if (itmax > BLK) group_reduce_scatter<G>(lo, lane);  // warp-uniform branch

  // promote: mean = (hi + lo) / n, then undo the 2^(ks * order) scaling
  double val[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int q = lg * K + j;
    const int ord = q < kNSum ? sum_order(q) : 0;
    float p, e;
    df_scale(hi[j], lo[j], rh, rl, p, e);
    val[j] = f2d_exact(p, -ks * ord) + f2d_exact(e, -ks * ord);
  }
  const int gbase = lane & ~(G - 1);
  const double u11 = __shfl_sync(0xffffffffu, val[0 % K], gbase + 0 / K);
  const double u22 = __shfl_sync(0xffffffffu, val[3 % K], gbase + 3 / K);
  const double u33 = __shfl_sync(0xffffffffu, val[5 % K], gbase + 5 / K);
  if (!valid) return;
  double *mo = mom + c * FP_NMOM;
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int q = lg * K + j;
    if (q < kNSum) mo[kU2 + q] = val[j];
  }
  if (lg >= 1 && lg <= 3) {
    const float v0 = lg == 1 ? v0x : (lg == 2 ? v0y : v0z);
    const float m = lg == 1 ? mx : (lg == 2 ? my : mz);
    mo[kU + lg - 1] = f2d_exact(v0) + f2d_exact(m);
  }
  if (lg == 0) {
    mo[kN] = n < (1 << 24) ? f2d_exact((float)n) : (double)n;
    mo[kTheta] = (u11 + u22 + u33) * (1.0 / 3.0);
  }
}

// Mark every cell of this CTA's chunks non-finite (theta = NaN): used when a
// bounded wait ran out, so the closure flags the cells FP_FLAG_NONFINITE.
__device__ void mark_failed(int64_t n_cells, int64_t n_chunks, double *__restrict__ mom, int tid) {
  for (int64_t j = blockIdx.x; j < n_chunks; j += gridDim.x) {
    const int64_t c0 = j * kChunkCells;
    const int64_t c1 = c0 + kChunkCells < n_cells ? c0 + kChunkCells : n_cells;
    for (int64_t c = c0 + tid; c < c1; c += kTileThreads) mom[c * FP_NMOM + kTheta] = __longlong_as_double(-1ll);
  }
}

__global__ void __launch_bounds__(kTileThreads, 2)
    gather_tile_kernel(const float *__restrict__ v, int64_t np, const int64_t *__restrict__ off, int64_t n_cells,
                       double *__restrict__ mom, int64_t n_chunks) {
  extern __shared__ __align__(128) float slot_buf[];
  __shared__ __align__(8) uint64_t full_bar[kSlots], empty_bar[kSlots];
  __shared__ SlotMeta meta[kSlots];
  __shared__ int task_ctr[kSlots];
  __shared__ int failed;
  const int tid = threadIdx.x;
  const int lane = tid & 31;
  const int warp = tid >> 5;
  if (tid == 0) {
    for (int s = 0; s < kSlots; ++s) {
      mbar_init(&full_bar[s], 1);
      mbar_init(&empty_bar[s], kConsumerWarps);
      task_ctr[s] = 0;
    }
    failed = 0;
    fence_barrier_init();
  }
  __syncthreads();

  if (warp == 0) {
    // ---------------- producer ----------------
    int64_t sub = 0;
    const uintptr_t vend = ((uintptr_t)(v + 3 * np)) & ~(uintptr_t)15;
    bool ok = true;
    auto acquire_slot = [&](int64_t sidx) -> int {
      const int s = (int)(sidx % kSlots);
      const int64_t use = sidx / kSlots;
      if (use > 0 && !mbar_wait_bounded(&empty_bar[s], (uint32_t)((use - 1) & 1))) ok = false;
      return s;
    };
    for (int64_t j = blockIdx.x; ok && j < n_chunks; j += gridDim.x) {
      const int64_t c0 = j * kChunkCells;
      const int64_t c1 = c0 + kChunkCells < n_cells ? c0 + kChunkCells : n_cells;
      // this lane's two offsets: off[c0 + lane], off[c0 + 32 + lane] (clamped to c1)
      const int64_t i0 = c0 + lane, i1 = c0 + 32 + lane;
      const int64_t o0 = off[i0 < c1 ? i0 : c1];
      const int64_t o1 = off[i1 < c1 ? i1 : c1];
      const int64_t oend = off[c1];
      int64_t cs = c0;
      while (ok && cs < c1) {
        // offset of cell cs (lanes hold off[c0..c0+63])
        const int rs = (int)(cs - c0);
        const int64_t start = rs < 32 ? __shfl_sync(0xffffffffu, o0, rs) : __shfl_sync(0xffffffffu, o1, rs - 32);
        // ce = last c in (cs, c1] with off[c] - start <= kSubP
        const bool f0 = (i0 > cs && i0 <= c1) && (o0 - start <= kSubP);
        const bool f1 = (i1 > cs && i1 <= c1) && (o1 - start <= kSubP);
        const unsigned m0 = __ballot_sync(0xffffffffu, f0), m1 = __ballot_sync(0xffffffffu, f1);
        int64_t ce;
        if (c1 - c0 == kChunkCells && oend - start <= kSubP)
          ce = c1;
        else if (m1)
          ce = c0 + 32 + (31 - __clz(m1));
        else if (m0)
          ce = c0 + (31 - __clz(m0));
        else
          ce = cs;  // the single cell cs exceeds a sub-tile
        const int big = ce == cs;
        if (big) ce = cs + 1;
        const int s = acquire_slot(sub);
        if (!ok) break;
        const int re = (int)(ce - c0);
        const int64_t pend = re < 32 ? __shfl_sync(0xffffffffu, o0, re)
                                     : (re < 64 ? __shfl_sync(0xffffffffu, o1, re - 32) : oend);
        SlotMeta &M = meta[s];
        // offsets of the sub-tile's cells
        if (i0 >= cs && i0 <= ce) M.offs[i0 - cs] = o0;
        if (i1 >= cs && i1 <= ce) M.offs[i1 - cs] = o1;
        if (lane == 0 && ce == c1 && c1 - c0 == kChunkCells) M.offs[ce - cs] = oend;
        float *buf = slot_buf + s * kSlotFloats;
        uint32_t bytes[3] = {0u, 0u, 0u};
        const float *src[3] = {nullptr, nullptr, nullptr};
        int lead[3] = {0, 0, 0};
        int64_t tail_from = pend;
        if (!big) {
#pragma unroll
          for (int d = 0; d < 3; ++d) {
            const float *base = v + d * np;
            const uintptr_t a = (uintptr_t)(base + start);
            const uintptr_t al = a & ~(uintptr_t)15;
            uintptr_t ae = ((uintptr_t)(base + pend) + 15) & ~(uintptr_t)15;
            if (d == 2 && ae > vend) {
              ae = vend > al ? vend : al;
              tail_from = (int64_t)((ae - (uintptr_t)base) / 4);
              if (tail_from < start) tail_from = start;
            }
            lead[d] = (int)((a - al) / 4);
            bytes[d] = (uint32_t)(ae - al);
            src[d] = (const float *)al;
          }
          // the last particles of the z array when its end is not 16-byte aligned
          for (int64_t i = tail_from + lane; i < pend; i += 32)
            buf[2 * kCapF + lead[2] + (i - start)] = v[2 * np + i];
        }
        __syncwarp();
        if (lane == 0) {
          M.cs = cs;
          M.ce = ce;
          M.pa = start;
          M.lead[0] = lead[0];
          M.lead[1] = lead[1];
          M.lead[2] = lead[2];
          M.big = big;
          M.done = 0;
          task_ctr[s] = 0;
          fence_proxy_async_smem();
          mbar_arrive_expect_tx(&full_bar[s], bytes[0] + bytes[1] + bytes[2]);
#pragma unroll
          for (int d = 0; d < 3; ++d)
            if (bytes[d]) bulk_g2s(buf + d * kCapF, src[d], bytes[d], &full_bar[s]);
        }
        ++sub;
        cs = ce;
      }
    }
    if (ok) {
      const int s = acquire_slot(sub);
      if (ok && lane == 0) {
        meta[s].done = 1;
        mbar_arrive_expect_tx(&full_bar[s], 0u);
      }
    }
    if (!ok) {
      if (lane == 0) atomicExch(&failed, 1);
      // wait (bounded) for copies still in flight into the ring, then stop
      for (int64_t q = sub - 1; q >= 0 && q >= sub - kSlots; --q)
        mbar_wait_bounded(&full_bar[q % kSlots], (uint32_t)((q / kSlots) & 1), 100000000ull);
    }
  } else {
    // ---------------- consumers ----------------
    constexpr int GPW = 32 / kTileG;
    bool ok = true;
    for (int64_t sub = 0;; ++sub) {
      const int s = (int)(sub % kSlots);
      if (!mbar_wait_bounded(&full_bar[s], (uint32_t)((sub / kSlots) & 1))) {
        ok = false;
        break;
      }
      const SlotMeta &M = meta[s];
      if (M.done) break;
      const float *bx = slot_buf + s * kSlotFloats;
      while (true) {
        int task = 0;
        if (lane == 0) task = atomicAdd(&task_ctr[s], 1);
        task = __shfl_sync(0xffffffffu, task, 0);
        const int64_t cbase = M.cs + (int64_t)task * GPW;
        if (cbase >= M.ce) break;
        const int64_t c = cbase + lane / kTileG;
        const bool valid = c < M.ce;
        const int64_t a = valid ? M.offs[c - M.cs] : M.pa;
        const int n = valid ? (int)(M.offs[c - M.cs + 1] - a) : 0;
        if (M.big) {
          reduce_cell_pair<false>(valid, n, v + a, v + np + a, v + 2 * np + a, c, mom, lane);
        } else {
          const int64_t rel = a - M.pa;
          reduce_cell_pair<true>(valid, n, bx + M.lead[0] + rel, bx + kCapF + M.lead[1] + rel,
                                 bx + 2 * kCapF + M.lead[2] + rel, c, mom, lane);
        }
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty_bar[s])) : "memory");
    }
    if (!ok && lane == 0) atomicExch(&failed, 1);
  }
  __syncthreads();
  if (failed) mark_failed(n_cells, n_chunks, mom, tid);
}

static int g_tile_attr_done[64];

bool launch_gather_tile(const float *v, int64_t np, const int64_t *off, int64_t n_cells, double *mom,
                        cudaStream_t st, int sm_count) {
  if (((uintptr_t)v & 15) != 0) return false;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !g_tile_attr_done[dev]) {
    if (cudaFuncSetAttribute(gather_tile_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTileSmem) !=
        cudaSuccess)
      return false;
    g_tile_attr_done[dev] = 1;
  }
  const int64_t n_chunks = (n_cells + kChunkCells - 1) / kChunkCells;
  int64_t grid = (int64_t)sm_count * 2;
  if (grid > n_chunks) grid = n_chunks;
  if (grid < 1) grid = 1;
  gather_tile_kernel<<<(unsigned)grid, kTileThreads, kTileSmem, st>>>(v, np, off, n_cells, mom, n_chunks);
  return true;
}

}  // namespace fpc
