// gather_tile.cu -- FP32-moment gather from FP32 velocities, streamed through
// shared memory by bulk asynchronous copies (paper Sec. 3.6 moments).
//
// Work is cut into chunks of kChunkCells consecutive cells, dealt round-robin
// to persistent CTAs.  Each CTA is warp-specialised:
//   * a producer warp reads the chunk's cell offsets (one coalesced load),
//     splits the chunk into sub-tiles of whole cells holding at most kSubP
//     particles, ranks the sub-tile's cells by size, and streams the three SoA
//     component ranges (widened to 16-byte boundaries) into a ring of kSlots
//     shared-memory slots with cp.async.bulk, completing on the slot's `full`
//     mbarrier;
//   * consumer warps take the sub-tiles in the same order and reduce four
//     cells per warp task (eight lanes per cell, the four cells of a task
//     consecutive in size order so their loops have similar trip counts)
//     from shared memory, then release the slot on its `empty` mbarrier.
// A cell larger than a sub-tile is reduced straight from global memory.  No
// global-memory round trip sits on a consumer's path; the producer runs up
// to kSlots sub-tiles ahead.
//
// A lane takes two steps of its group at once (particles i and i + 8) and does
// their arithmetic packed as FP32x2 (__fadd2_rn / __fmul2_rn / __ffma2_rn: one
// instruction for both); steps whose particles all lie in their cells skip the
// masking.  Per lane the sums are plain FP32 over blocks of 16 pair steps;
// each block is reduced over the group's eight lanes through a swizzled
// shared-memory transpose (a lane writes its row, the owner of four sums adds
// eight float4s), and owners fold the blocks with two-sum.  Promotion to FP64
// scales by the power of two in FP32 (exact), widens hi and lo parts on the
// integer pipe with the scale folded into the exponent and adds them: one
// FP64-pipe instruction per moment.
//
// The same kernel, instantiated with kLite, serves the LITE moment pass:
// only the 9 sums of u_ij and b_i = <c_i |c|^2> a particle, written as the
// FP_NLITE vector (N, U, theta, u_ij, b_i).
#include <cstdint>

#include "fp_device.cuh"
#include "tma.cuh"

namespace fpc {

constexpr int kChunkCells = 64;
constexpr int kSubP = 2048;                  // particles per sub-tile (max)
constexpr int kCapF = kSubP + 8;             // floats per component slot (alignment slack)
constexpr int kSlots = 3;
constexpr int kConsumerWarps = 7;          // 8 warps a CTA, 2 CTAs per SM: the register cap of 128 still holds the sums
constexpr int kTileThreads = 32 * (1 + kConsumerWarps);
constexpr int kTileG = 8;                    // lanes per cell (measured best of 4, 8, 16, 32)
constexpr int kCellsPerTask = 32 / kTileG;   // cells per warp task
constexpr int kSlotFloats = 3 * kCapF;
constexpr int kScratchFloats = 32 * 32;  // transpose scratch per consumer warp
constexpr size_t kTileSmem = (size_t)kSlots * kSlotFloats * sizeof(float) + (size_t)kConsumerWarps * kScratchFloats * 4;

struct SlotMeta {
  int64_t cs, ce;                 // cells [cs, ce) of the sub-tile
  int64_t pa;                     // first particle (offset of cell cs)
  int lead[3];                    // slot index of particle pa, per component
  int big;                        // 1: the single cell cs is reduced from global memory
  int done;                       // 1: no more sub-tiles for this CTA
  int64_t offs[kChunkCells + 1];  // off[cs .. ce]
  uint8_t order[kChunkCells];     // sub-tile cells (relative to cs), largest first
};

// One cell per kTileG-lane group, the warp's groups in lockstep; px/py/pz
// point at the cell's first particle (shared or global memory).
constexpr int kLiteSum = 9;  // u_ij (6, order 2), c_i |c|^2 (3, order 3)

template <bool kLite>
__device__ __forceinline__ int tile_order(int q) {
  if (kLite) return q < 6 ? 2 : 3;
  return sum_order(q);
}

// physical float4 chunk of logical chunk c in transpose-scratch row r: the
// eight rows of a quarter-warp put a given chunk on eight different bank groups
__device__ __forceinline__ int swz(int c, int r) { return c ^ (((r & 3) << 1) | ((r >> 2) & 1)); }

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// The monomials of one pair of particles (w packed as FP32x2) added to the
// packed sums T (sum slot order of sum_order; the LITE set is u_ij, c_i |c|^2).
template <bool kLite, int NS>
__device__ __forceinline__ void accumulate2(float2 (&T)[NS], float2 wx, float2 wy, float2 wz) {
  const float2 xx = __fmul2_rn(wx, wx), xy = __fmul2_rn(wx, wy), xz = __fmul2_rn(wx, wz);
  const float2 yy = __fmul2_rn(wy, wy), yz = __fmul2_rn(wy, wz), zz = __fmul2_rn(wz, wz);
  T[0] = __fadd2_rn(T[0], xx); T[1] = __fadd2_rn(T[1], xy); T[2] = __fadd2_rn(T[2], xz);
  T[3] = __fadd2_rn(T[3], yy); T[4] = __fadd2_rn(T[4], yz); T[5] = __fadd2_rn(T[5], zz);
  const float2 r2 = __fadd2_rn(__fadd2_rn(xx, yy), zz);
  if constexpr (kLite) {
    T[6] = __ffma2_rn(r2, wx, T[6]); T[7] = __ffma2_rn(r2, wy, T[7]); T[8] = __ffma2_rn(r2, wz, T[8]);
  } else {
    T[6] = __ffma2_rn(xx, wx, T[6]);   T[7] = __ffma2_rn(xx, wy, T[7]);   T[8] = __ffma2_rn(xx, wz, T[8]);
    T[9] = __ffma2_rn(xy, wy, T[9]);   T[10] = __ffma2_rn(xy, wz, T[10]); T[11] = __ffma2_rn(xz, wz, T[11]);
    T[12] = __ffma2_rn(yy, wy, T[12]); T[13] = __ffma2_rn(yy, wz, T[13]); T[14] = __ffma2_rn(yz, wz, T[14]);
    T[15] = __ffma2_rn(zz, wz, T[15]);
    T[16] = __ffma2_rn(r2, xx, T[16]); T[17] = __ffma2_rn(r2, xy, T[17]); T[18] = __ffma2_rn(r2, xz, T[18]);
    T[19] = __ffma2_rn(r2, yy, T[19]); T[20] = __ffma2_rn(r2, yz, T[20]); T[21] = __ffma2_rn(r2, zz, T[21]);
    const float2 r4 = __fmul2_rn(r2, r2);
    T[22] = __ffma2_rn(r4, wx, T[22]); T[23] = __ffma2_rn(r4, wy, T[23]); T[24] = __ffma2_rn(r4, wz, T[24]);
    T[25] = __ffma2_rn(r4, r2, T[25]);
  }
}

// Exact float -> double times 2^e_add (|e_add| < 700) on the integer pipe:
// zeros and FP32 subnormals give 0, inf and NaN stay inf and NaN.
__device__ __forceinline__ double f2d_scaled(float f, int e_add) {
  const uint32_t u = __float_as_uint(f);
  const uint32_t a = u & 0x7fffffffu;
  uint32_t hi = (a >> 3) + ((uint32_t)(896 + e_add) << 20);
  uint32_t lo = u << 29;
  if (a < 0x00800000u) hi = lo = 0u;
  if (a >= 0x7f800000u) {
    hi = 0x7ff00000u | (a > 0x7f800000u ? 0x80000u : 0u);
    lo = 0u;
  }
  return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)lo);
}

template <bool kShared, bool kLite>
__device__ __forceinline__ void reduce_cells(bool valid, int n, const float *px, const float *py, const float *pz,
                                             int64_t c, double *__restrict__ mom, double *__restrict__ m6,
                                             float *scratch, const float *zeros, int lane) {
  constexpr int G = kTileG;
  constexpr int NS = kLite ? kLiteSum : kNSum;
  constexpr int K = 32 / G;             // sums a lane owns after the reduction (one float4 chunk)
  constexpr int NCH = (NS + K - 1) / K;  // chunks in use
  constexpr int BLK = 16;               // pair steps per lane summed plainly before a two-sum fold
  static_assert(K == 4, "one float4 chunk per lane");
  const int lg = lane & (G - 1);
  const int gbase = lane & ~(G - 1);
  auto ld = [](const float *p, int i) -> float {
    if (kShared) return p[i];
    return __ldg(p + i);
  };
  if (!valid) n = 0;
  // an empty staged cell reads zeros (its offsets from v0 are then exactly 0);
  // the groups of a huge cell read that cell's data, in range
  if (kShared && n == 0) px = py = pz = zeros;
  const float v0x = ld(px, 0), v0y = ld(py, 0), v0z = ld(pz, 0);
  const int itmax = __reduce_max_sync(0xffffffffu, (n + G - 1) / G);
  const int npair = (itmax + 1) >> 1;
  // pair steps below pfull have both particles in range for every group
  const int pfull = (int)__reduce_min_sync(0xffffffffu, (unsigned)(n / G)) >> 1;
  const float2 nv0x = f2(-v0x), nv0y = f2(-v0y), nv0z = f2(-v0z);
  // pass A on pairs of steps (it, it + 1): out-of-range particles read particle
  // 0, whose offset from v0 is exactly zero
  float2 SDx = f2(0.f), SDy = f2(0.f), SDz = f2(0.f), SQx = f2(0.f), SQy = f2(0.f), SQz = f2(0.f);
#pragma unroll 2
  for (int pp = 0; pp < pfull; ++pp) {
    const int j0 = 2 * pp * G + lg, j1 = j0 + G;
    const float2 dx = __fadd2_rn(make_float2(ld(px, j0), ld(px, j1)), nv0x);
    const float2 dy = __fadd2_rn(make_float2(ld(py, j0), ld(py, j1)), nv0y);
    const float2 dz = __fadd2_rn(make_float2(ld(pz, j0), ld(pz, j1)), nv0z);
    SDx = __fadd2_rn(SDx, dx);
    SDy = __fadd2_rn(SDy, dy);
    SDz = __fadd2_rn(SDz, dz);
    SQx = __ffma2_rn(dx, dx, SQx);
    SQy = __ffma2_rn(dy, dy, SQy);
    SQz = __ffma2_rn(dz, dz, SQz);
  }
  for (int pp = pfull; pp < npair; ++pp) {
    const int i0 = 2 * pp * G + lg, i1 = i0 + G;
    const int j0 = i0 < n ? i0 : 0, j1 = i1 < n ? i1 : 0;
    const float2 dx = __fadd2_rn(make_float2(ld(px, j0), ld(px, j1)), nv0x);
    const float2 dy = __fadd2_rn(make_float2(ld(py, j0), ld(py, j1)), nv0y);
    const float2 dz = __fadd2_rn(make_float2(ld(pz, j0), ld(pz, j1)), nv0z);
    SDx = __fadd2_rn(SDx, dx);
    SDy = __fadd2_rn(SDy, dy);
    SDz = __fadd2_rn(SDz, dz);
    SQx = __ffma2_rn(dx, dx, SQx);
    SQy = __ffma2_rn(dy, dy, SQy);
    SQz = __ffma2_rn(dz, dz, SQz);
  }
  float sx = SDx.x + SDx.y, sy = SDy.x + SDy.y, sz = SDz.x + SDz.y;
  float sq = (SQx.x + SQx.y) + (SQy.x + SQy.y) + (SQz.x + SQz.y);
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
    ks = max(-20, min(20, -(ex / 2)));
  }
  const float s = ldexpf(1.f, ks);
  const float2 nmx = f2(-mx), nmy = f2(-my), nmz = f2(-mz);
  // full steps: ((v - v0) - m) s as one fused multiply-add, exact because s
  // is a power of two (d s and m s are exact, one rounding as before)
  const float2 S2f = f2(s), nmsx = f2(-mx * s), nmsy = f2(-my * s), nmsz = f2(-mz * s);

  // pass B: centred, scaled sums w = ((v - v0) - m) s, pairs of steps packed
  // FP32x2, blocks of BLK pair steps; each block is reduced over the group's
  // lanes through a swizzled shared-memory transpose, and the owner of a sum
  // folds the blocks with two-sum
  float hi[K], lo[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    hi[j] = 0.f;
    lo[j] = 0.f;
  }
  float4 *sc4 = reinterpret_cast<float4 *>(scratch);
  for (int b0 = 0; b0 < npair; b0 += BLK) {  // warp-uniform
    float2 T[NS];
#pragma unroll
    for (int q = 0; q < NS; ++q) T[q] = f2(0.f);
    const int b1 = min(b0 + BLK, npair);
    const int bf = min(b1, max(b0, pfull));
#pragma unroll 2
    for (int pp = b0; pp < bf; ++pp) {
      const int j0 = 2 * pp * G + lg, j1 = j0 + G;
      const float2 wx = __ffma2_rn(__fadd2_rn(make_float2(ld(px, j0), ld(px, j1)), nv0x), S2f, nmsx);
      const float2 wy = __ffma2_rn(__fadd2_rn(make_float2(ld(py, j0), ld(py, j1)), nv0y), S2f, nmsy);
      const float2 wz = __ffma2_rn(__fadd2_rn(make_float2(ld(pz, j0), ld(pz, j1)), nv0z), S2f, nmsz);
      accumulate2<kLite, NS>(T, wx, wy, wz);
    }
    for (int pp = bf; pp < b1; ++pp) {
      const int i0 = 2 * pp * G + lg, i1 = i0 + G;
      const bool in0 = i0 < n, in1 = i1 < n;
      const int j0 = in0 ? i0 : 0, j1 = in1 ? i1 : 0;
      const float2 S2 = make_float2(in0 ? s : 0.f, in1 ? s : 0.f);
      const float2 wx = __fmul2_rn(__fadd2_rn(__fadd2_rn(make_float2(ld(px, j0), ld(px, j1)), nv0x), nmx), S2);
      const float2 wy = __fmul2_rn(__fadd2_rn(__fadd2_rn(make_float2(ld(py, j0), ld(py, j1)), nv0y), nmy), S2);
      const float2 wz = __fmul2_rn(__fadd2_rn(__fadd2_rn(make_float2(ld(pz, j0), ld(pz, j1)), nv0z), nmz), S2);
      accumulate2<kLite, NS>(T, wx, wy, wz);
    }
#pragma unroll
    for (int ch = 0; ch < NCH; ++ch) {
      float t4[4];
#pragma unroll
      for (int k = 0; k < 4; ++k) t4[k] = 4 * ch + k < NS ? T[4 * ch + k].x + T[4 * ch + k].y : 0.f;
      sc4[lane * 8 + swz(ch, lane)] = make_float4(t4[0], t4[1], t4[2], t4[3]);
    }
    __syncwarp();
    float bs[K] = {0.f, 0.f, 0.f, 0.f};
    if (lg < NCH) {
#pragma unroll
      for (int i = 0; i < G; ++i) {
        const int rr = gbase + i;
        const float4 t = sc4[rr * 8 + swz(lg, rr)];
        bs[0] += t.x;
        bs[1] += t.y;
        bs[2] += t.z;
        bs[3] += t.w;
      }
    }
    __syncwarp();
    if (b0 == 0) {
#pragma unroll
      for (int j = 0; j < K; ++j) hi[j] = bs[j];
    } else {
#pragma unroll
      for (int j = 0; j < K; ++j) {
        float sum, err;
        two_sum(hi[j], bs[j], sum, err);
        hi[j] = sum;
        lo[j] += err;
      }
    }
  }

  // promote: mean = (hi + lo) / n as a double-float, the 2^(ks * order)
  // scaling undone in the exponent (exact), one FP64 add
  double val[K];
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int q = lg * K + j;
    const int ord = q < NS ? tile_order<kLite>(q) : 0;
    float p, e;
    df_scale(hi[j], lo[j], rh, rl, p, e);
    val[j] = q < NS ? f2d_scaled(p, -ks * ord) + f2d_scaled(e, -ks * ord) : 0.0;
  }
  const double u11 = __shfl_sync(0xffffffffu, val[0 % K], gbase + 0 / K);
  const double u22 = __shfl_sync(0xffffffffu, val[3 % K], gbase + 3 / K);
  const double u33 = __shfl_sync(0xffffffffu, val[5 % K], gbase + 5 / K);
  if (!valid) return;
  double *mo = mom + c * (kLite ? FP_NLITE : FP_NMOM);
#pragma unroll
  for (int j = 0; j < K; ++j) {
    const int q = lg * K + j;
    if (kLite) {
      if (q < kLiteSum) mo[kU2 + q] = val[j];  // u_ij at 5..10, b_i at 11..13
    } else {
      if (q < kNMomSum) mo[kU2 + q] = val[j];
      if (q == kM6Sum && m6) m6[c] = val[j];
    }
  }
  if (lg >= 1 && lg <= 3) {
    const float v0 = n > 0 ? (lg == 1 ? v0x : (lg == 2 ? v0y : v0z)) : 0.f;
    const float m = lg == 1 ? mx : (lg == 2 ? my : mz);
    mo[kU + lg - 1] = f2d_exact(v0) + f2d_exact(m);
  }
  if (lg == 0) {
    mo[kN] = u2d_exact((uint32_t)n);
    mo[kTheta] = (u11 + u22 + u33) * (1.0 / 3.0);
  }
}

// Mark every cell of this CTA's chunks non-finite (theta = NaN): used when a
// bounded wait ran out, so the closure flags the cells FP_FLAG_NONFINITE.
__device__ void mark_failed(int64_t n_cells, int64_t n_chunks, double *__restrict__ mom, int stride, int tid) {
  for (int64_t j = blockIdx.x; j < n_chunks; j += gridDim.x) {
    const int64_t c0 = j * kChunkCells;
    const int64_t c1 = c0 + kChunkCells < n_cells ? c0 + kChunkCells : n_cells;
    for (int64_t c = c0 + tid; c < c1; c += kTileThreads) mom[c * stride + kTheta] = __longlong_as_double(-1ll);
  }
}

// Order the sub-tile's cells by size, largest first (ties: lower index
// first), with a 64-element bitonic network: lane l holds elements l and
// l + 32; keys pack ((size + 1) << 6) | (63 - index), 0 for absent cells.
__device__ __forceinline__ void rank_cells(int ncell, int na, int nb, uint8_t *order, int lane) {
  uint32_t ka = lane < ncell ? ((uint32_t)(na + 1) << 6) | (uint32_t)(63 - lane) : 0u;
  uint32_t kb = lane + 32 < ncell ? ((uint32_t)(nb + 1) << 6) | (uint32_t)(31 - lane) : 0u;
#pragma unroll
  for (int k = 2; k <= 64; k <<= 1) {
#pragma unroll
    for (int j = k >> 1; j >= 1; j >>= 1) {
      // element indices ea = lane, eb = lane + 32; max goes to the lower index
      // of a pair inside blocks with (e & k) == 0, to the higher one otherwise
      const int ea = lane, eb = lane + 32;
      if (j == 32) {
        const uint32_t hi = ka > kb ? ka : kb, lo = ka > kb ? kb : ka;
        const bool up = (ea & k) == 0;  // same block for ea and eb when k = 64
        ka = up ? hi : lo;
        kb = up ? lo : hi;
      } else {
        const uint32_t pa = __shfl_xor_sync(0xffffffffu, ka, j);
        const uint32_t pb = __shfl_xor_sync(0xffffffffu, kb, j);
        const bool lower = (lane & j) == 0;
        const bool upa = (ea & k) == 0, upb = (eb & k) == 0;
        ka = (lower == upa) ? (ka > pa ? ka : pa) : (ka > pa ? pa : ka);
        kb = (lower == upb) ? (kb > pb ? kb : pb) : (kb > pb ? pb : kb);
      }
    }
  }
  if (lane < ncell) order[lane] = (uint8_t)(63 - (ka & 63u));
  if (lane + 32 < ncell) order[lane + 32] = (uint8_t)(63 - (kb & 63u));
}

template <bool kLite>
__global__ void __launch_bounds__(kTileThreads, 2)
    gather_tile_kernel(const float *__restrict__ v, int64_t np, const int64_t *__restrict__ off, int64_t n_cells,
                       double *__restrict__ mom, double *__restrict__ m6, int64_t n_chunks) {
  extern __shared__ __align__(128) float slot_buf[];
  float *scratch_all = slot_buf + kSlots * kSlotFloats;
  __shared__ __align__(16) float zeros[4];
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
    zeros[0] = zeros[1] = zeros[2] = zeros[3] = 0.f;
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
    // lanes hold off[c0 + lane] and off[c0 + 32 + lane] (indices clamped to
    // c1); the next chunk's offsets are loaded while this one is streamed
    auto load_chunk = [&](int64_t jj, int64_t &q0, int64_t &q1, int64_t &qe) {
      if (jj >= n_chunks) return;
      const int64_t b0 = jj * kChunkCells;
      const int64_t b1 = b0 + kChunkCells < n_cells ? b0 + kChunkCells : n_cells;
      q0 = off[b0 + lane < b1 ? b0 + lane : b1];
      q1 = off[b0 + 32 + lane < b1 ? b0 + 32 + lane : b1];
      qe = off[b1];
    };
    int64_t nx0 = 0, nx1 = 0, nxe = 0;
    load_chunk(blockIdx.x, nx0, nx1, nxe);
    for (int64_t j = blockIdx.x; ok && j < n_chunks; j += gridDim.x) {
      const int64_t c0 = j * kChunkCells;
      const int64_t c1 = c0 + kChunkCells < n_cells ? c0 + kChunkCells : n_cells;
      const int64_t i0 = c0 + lane, i1 = c0 + 32 + lane;
      const int64_t o0 = nx0, o1 = nx1, oend = nxe;
      load_chunk(j + gridDim.x, nx0, nx1, nxe);
      // per-cell sizes of the lane's two cells (cell i0 and i1)
      const int64_t o0n = __shfl_down_sync(0xffffffffu, o0, 1);
      const int64_t o1f = __shfl_sync(0xffffffffu, o1, 0);
      const int64_t o1n = __shfl_down_sync(0xffffffffu, o1, 1);
      const int64_t e0 = lane < 31 ? o0n : o1f;           // off[i0 + 1]
      const int64_t e1 = lane < 31 ? o1n : oend;          // off[i1 + 1]
      int64_t cs = c0;
      while (ok && cs < c1) {
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
        if (i0 >= cs && i0 <= ce) M.offs[i0 - cs] = o0;
        if (i1 >= cs && i1 <= ce) M.offs[i1 - cs] = o1;
        if (lane == 0 && ce == c1 && c1 - c0 == kChunkCells) M.offs[ce - cs] = oend;
        // size ranking of the sub-tile's cells (cell cs + r held by lane r or r - 32)
        {
          const int ncell = (int)(ce - cs);
          const int la = (int)(i0 - cs), lb = (int)(i1 - cs);  // this lane's cells, relative
          // gather sizes so that lane r holds cell cs + r (and cs + r + 32)
          const int64_t sa_abs = (i0 >= cs && i0 < ce) ? e0 - o0 : 0;
          const int64_t sb_abs = (i1 >= cs && i1 < ce) ? e1 - o1 : 0;
          (void)la;
          (void)lb;
          // cell cs + r lives at absolute index c0 + rs + r
          const int src_a = rs + lane, src_b = rs + lane + 32;
          const int64_t na_a = __shfl_sync(0xffffffffu, sa_abs, src_a & 31);
          const int64_t na_b = __shfl_sync(0xffffffffu, sb_abs, src_a & 31);
          const int64_t nb_a = __shfl_sync(0xffffffffu, sa_abs, src_b & 31);
          const int64_t nb_b = __shfl_sync(0xffffffffu, sb_abs, src_b & 31);
          const int na = (int)(src_a < 32 ? na_a : na_b);
          const int nb = (int)(src_b < 32 ? nb_a : (src_b < 64 ? nb_b : 0));
          rank_cells(ncell, na, nb, M.order, lane);
        }
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
    bool ok = true;
    const int g = lane / kTileG;
    float *scratch = scratch_all + (warp - 1) * kScratchFloats;
    for (int64_t sub = 0;; ++sub) {
      const int s = (int)(sub % kSlots);
      if (!mbar_wait_bounded(&full_bar[s], (uint32_t)((sub / kSlots) & 1))) {
        ok = false;
        break;
      }
      const SlotMeta &M = meta[s];
      if (M.done) break;
      const float *bx = slot_buf + s * kSlotFloats;
      const int ncell = (int)(M.ce - M.cs);
      while (true) {
        int task = 0;
        if (lane == 0) task = atomicAdd(&task_ctr[s], 1);
        task = __shfl_sync(0xffffffffu, task, 0);
        const int r0 = task * kCellsPerTask;
        if (r0 >= ncell) break;
        const int r = r0 + g;
        const bool valid = r < ncell;
        const int rc = valid ? (int)M.order[r] : 0;
        const int64_t c = M.cs + rc;
        const int64_t a = M.offs[rc];
        const int n = valid ? (int)(M.offs[rc + 1] - a) : 0;
        if (M.big) {
          reduce_cells<false, kLite>(valid, n, v + a, v + np + a, v + 2 * np + a, c, mom, m6, scratch, zeros, lane);
        } else {
          const int64_t rel = a - M.pa;
          reduce_cells<true, kLite>(valid, n, bx + M.lead[0] + rel, bx + kCapF + M.lead[1] + rel,
                             bx + 2 * kCapF + M.lead[2] + rel, c, mom, m6, scratch, zeros, lane);
        }
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty_bar[s])) : "memory");
    }
    if (!ok && lane == 0) atomicExch(&failed, 1);
  }
  __syncthreads();
  if (failed) mark_failed(n_cells, n_chunks, mom, kLite ? FP_NLITE : FP_NMOM, tid);
}

static int g_tile_attr_done[2][64];

template <bool kLite>
static bool launch_tile(const float *v, int64_t np, const int64_t *off, int64_t n_cells, double *mom, double *m6,
                        cudaStream_t st, int sm_count) {
  if (((uintptr_t)v & 15) != 0) return false;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !g_tile_attr_done[kLite][dev]) {
    if (cudaFuncSetAttribute(gather_tile_kernel<kLite>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTileSmem) != cudaSuccess)
      return false;
    g_tile_attr_done[kLite][dev] = 1;
  }
  const int64_t n_chunks = (n_cells + kChunkCells - 1) / kChunkCells;
  int64_t grid = (int64_t)sm_count * 2;
  if (grid > n_chunks) grid = n_chunks;
  if (grid < 1) grid = 1;
  gather_tile_kernel<kLite><<<(unsigned)grid, kTileThreads, kTileSmem, st>>>(v, np, off, n_cells, mom, m6,
                                                                              n_chunks);
  return true;
}

bool launch_gather_tile(const float *v, int64_t np, const int64_t *off, int64_t n_cells, double *mom, double *m6,
                        cudaStream_t st, int sm_count) {
  return launch_tile<false>(v, np, off, n_cells, mom, m6, st, sm_count);
}

// LITE vectors [n_cells][FP_NLITE] from FP32 velocities
bool launch_gather_tile_lite(const float *v, int64_t np, const int64_t *off, int64_t n_cells, double *lite,
                             cudaStream_t st, int sm_count) {
  return launch_tile<true>(v, np, off, n_cells, lite, nullptr, st, sm_count);
}

}  // namespace fpc
