// gather_tile.cu -- FP32-moment gather from FP32 velocities (paper Sec. 3.6
// moments): one pass over the particles, streamed through shared memory by
// bulk asynchronous copies.
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
//     consecutive in size order so their loops have similar trip counts),
//     then release the slot on its `empty` mbarrier.
// When the CTA's sub-tiles are done, all its threads finish its cells, one
// thread a cell (the records they read are in global memory, not in a slot).
// A cell larger than a sub-tile is reduced straight from global memory.
//
// One pass over the particles.  A cell's velocities are shifted by
// v0 + delta, v0 its first particle and delta the mean offset from v0 of a
// strided subset of m = min(n, 8) particles (particle floor(k n / m) for
// k < m: the whole cell when n <= 8), and scaled by the power of two s that
// brings the subset's largest offset from the shift into [1/2, 1) (exact).
// With w = ((v - v0) - delta) s the eight lanes of a cell sum, in one sweep,
// the monomials the central moments expand into -- w_i w_j, w_i w_j w_k,
// |w|^2 w_i w_j, |w|^4 w_i, |w|^6 and w_i (29 sums; the LITE set w_i w_j,
// |w|^2 w_i, w_i: 12).  A lane takes two steps of its group at once
// (particles i and i + 8) packed as FP32x2 (__fadd2_rn / __fmul2_rn /
// __ffma2_rn); steps whose particles all lie in their cells skip the masking;
// blocks of 16 pair steps are reduced over the group's lanes through a
// swizzled shared-memory transpose and folded with two-sum.  The group then
// writes the 29 means (FP32) with v0, delta, the scale and n into the cell's
// own output row as a staging record.
//
// The finishing lane reads the record and turns the shifted means into
// central moments by the binomial expansion of c = w - d, d = <w>:
//   u_ij   = <w_i w_j> - d_i d_j
//   u_ijk  = <w_i w_j w_k> - d_i <w_j w_k> - d_j <w_i w_k> - d_k <w_i w_j>
//            + 2 d_i d_j d_k
// and, with R = |w|^2, L = w.d, Q = |d|^2 and |c|^2 = R - 2L + Q, the
// contractions <c_i c_j |c|^2>, <c_i |c|^4>, <|c|^6> from the same 29 means
// (the set is closed under the shift).  The arithmetic is FP32: the subset
// mean leaves |d| near sigma / sqrt(8), so the expansion cancels little.  The
// scale is undone in the exponent (exact) and the row is written in FP64.
// With the per-cell work on one lane per cell, the eight lanes of a group
// only stream particles, and there is no second sweep for the mean.
#include <cstdint>

#include "fp_device.cuh"
#include "tma.cuh"

namespace fpc {

constexpr int kChunkCells = 64;
constexpr int kSubP = 2048;                  // particles per sub-tile (max)
constexpr int kCapF = kSubP + 8;             // floats per component slot (alignment slack)
constexpr int kSlots = 2;
constexpr int kConsumerWarps = 4;            // 5 warps a CTA, 3 CTAs per SM (measured best)
constexpr int kCtasPerSm = 3;
constexpr int kTileThreads = 32 * (1 + kConsumerWarps);
constexpr int kTileG = 8;                    // lanes per cell
constexpr int kCellsPerTask = 32 / kTileG;   // cells per warp task
constexpr int kSlotFloats = 3 * kCapF;
constexpr int kScratchFloats = 32 * 32;      // transpose scratch per consumer warp
constexpr size_t kTileSmem = (size_t)kSlots * kSlotFloats * sizeof(float) + (size_t)kConsumerWarps * kScratchFloats * 4;
static_assert(kTileG == 8, "one subset particle a lane");
static_assert((size_t)(kTileThreads / 32) * 32 * FP_NMOM * 8 <= (size_t)kSlots * kSlotFloats * 4, "finishing stage fits the slots");

// sums a particle: full set (w_i w_j 0..5, w_i w_j w_k 6..15, |w|^2 w_i w_j
// 16..21, |w|^4 w_i 22..24, |w|^6 25, w_i 26..28); LITE set (w_i w_j 0..5,
// |w|^2 w_i 6..8, w_i 9..11).  Symmetric index pairs in the order 11, 12,
// 13, 22, 23, 33; triples 111, 112, 113, 122, 123, 133, 222, 223, 233, 333.
constexpr int kFullSum = 29;
constexpr int kLiteSum = 12;
// staging record (floats) at the start of a cell's output row: the means at
// [0, kRecX), then v0 (3), delta (3), the scale exponent and n (as ints)
template <bool kLite>
__host__ __device__ constexpr int rec_x() { return kLite ? 16 : 32; }
static_assert(rec_x<false>() + 8 <= 2 * FP_NMOM && rec_x<true>() + 8 <= 2 * FP_NLITE, "record fits its row");

struct SlotMeta {
  int64_t cs, ce;                 // cells [cs, ce) of the sub-tile
  int64_t pa;                     // first particle (offset of cell cs)
  int lead[3];                    // slot index of particle pa, per component
  int big;                        // 1: the single cell cs is reduced from global memory
  int done;                       // 1: no more sub-tiles for this CTA
  int64_t offs[kChunkCells + 1];  // off[cs .. ce]
  uint8_t order[kChunkCells];     // sub-tile cells (relative to cs), largest first
};

// physical float4 chunk of logical chunk c in transpose-scratch row r: the
// eight rows of a quarter-warp put a given chunk on eight different bank groups
__device__ __forceinline__ int swz(int c, int r) { return c ^ (((r & 3) << 1) | ((r >> 2) & 1)); }

__device__ __forceinline__ float2 f2(float a) { return make_float2(a, a); }

// The monomials of one pair of particles (w packed as FP32x2) added to the
// packed sums T, in the slot order above.
template <bool kLite, int NS>
__device__ __forceinline__ void accumulate2(float2 (&T)[NS], float2 wx, float2 wy, float2 wz) {
  const float2 xx = __fmul2_rn(wx, wx), xy = __fmul2_rn(wx, wy), xz = __fmul2_rn(wx, wz);
  const float2 yy = __fmul2_rn(wy, wy), yz = __fmul2_rn(wy, wz), zz = __fmul2_rn(wz, wz);
  T[0] = __fadd2_rn(T[0], xx); T[1] = __fadd2_rn(T[1], xy); T[2] = __fadd2_rn(T[2], xz);
  T[3] = __fadd2_rn(T[3], yy); T[4] = __fadd2_rn(T[4], yz); T[5] = __fadd2_rn(T[5], zz);
  const float2 r2 = __fadd2_rn(__fadd2_rn(xx, yy), zz);
  if constexpr (kLite) {
    T[6] = __ffma2_rn(r2, wx, T[6]); T[7] = __ffma2_rn(r2, wy, T[7]); T[8] = __ffma2_rn(r2, wz, T[8]);
    T[9] = __fadd2_rn(T[9], wx); T[10] = __fadd2_rn(T[10], wy); T[11] = __fadd2_rn(T[11], wz);
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
    T[26] = __fadd2_rn(T[26], wx); T[27] = __fadd2_rn(T[27], wy); T[28] = __fadd2_rn(T[28], wz);
  }
}

// Exact float -> double times 2^e_add (|e_add| <= 120) on the integer pipe:
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

// Power-of-two exponent ks with |x| 2^ks in [1/2, 1) for a positive normal
// x, clamped to [-20, 20]; 0 for x = 0, 20 for an FP32 subnormal.
__device__ __forceinline__ int scale_exponent(float x) {
  if (!(x > 0.f)) return 0;
  const int e = (int)((__float_as_uint(x) >> 23) & 0xffu);
  if (e == 0) return 20;
  return max(-20, min(20, 126 - e));
}

// One cell per kTileG-lane group, the warp's groups in lockstep; px/py/pz
// point at the cell's first particle (shared or global memory).  Writes the
// cell's staging record to rec (its output row) when valid.
template <bool kShared, bool kLite>
__device__ __forceinline__ void gather_cells(bool valid, int n, const float *px, const float *py, const float *pz,
                                             float *__restrict__ rec, float *scratch, const float *zeros, int lane) {
  constexpr int G = kTileG;
  constexpr int NS = kLite ? kLiteSum : kFullSum;
  constexpr int K = 32 / G;              // sums a lane owns after the reduction (one float4 chunk)
  constexpr int NCH = (NS + K - 1) / K;  // chunks in use
  constexpr int BLK = 16;                // pair steps per lane summed plainly before a two-sum fold
  constexpr int RX = rec_x<kLite>();
  static_assert(K == 4 && NCH <= G, "one float4 chunk per lane");
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

  // the shift: lane lg holds subset particle floor(lg n / m), m = min(n, G)
  const int m = n < G ? n : G;
  const bool in_sub = lg < m;
  const int si = !in_sub ? 0 : (n <= (1 << 28) ? (lg * n) / m : (int)(((int64_t)lg * n) / m));
  const float ex = ld(px, si) - v0x, ey = ld(py, si) - v0y, ez = ld(pz, si) - v0z;
  float sx = in_sub ? ex : 0.f, sy = in_sub ? ey : 0.f, sz = in_sub ? ez : 0.f;
  sx = group_allreduce<G>(sx);
  sy = group_allreduce<G>(sy);
  sz = group_allreduce<G>(sz);
  const float rm = m > 0 ? __frcp_rn((float)m) : 0.f;
  const float dx = sx * rm, dy = sy * rm, dz = sz * rm;
  float mx = in_sub ? fmaxf(fabsf(ex - dx), fmaxf(fabsf(ey - dy), fabsf(ez - dz))) : 0.f;
#pragma unroll
  for (int o = G / 2; o >= 1; o >>= 1) mx = fmaxf(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  const int ks = scale_exponent(mx);
  const float s = __uint_as_float((uint32_t)(127 + ks) << 23);
  const float2 nv0x = f2(-v0x), nv0y = f2(-v0y), nv0z = f2(-v0z);
  const float2 ndx = f2(-dx), ndy = f2(-dy), ndz = f2(-dz);
  // full steps: ((v - v0) - delta) s as one fused multiply-add, exact because
  // s is a power of two (d s and delta s are exact, one rounding as before)
  const float2 S2f = f2(s), ndsx = f2(-dx * s), ndsy = f2(-dy * s), ndsz = f2(-dz * s);

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
      const float2 wx = __ffma2_rn(__fadd2_rn(make_float2(ld(px, j0), ld(px, j1)), nv0x), S2f, ndsx);
      const float2 wy = __ffma2_rn(__fadd2_rn(make_float2(ld(py, j0), ld(py, j1)), nv0y), S2f, ndsy);
      const float2 wz = __ffma2_rn(__fadd2_rn(make_float2(ld(pz, j0), ld(pz, j1)), nv0z), S2f, ndsz);
      accumulate2<kLite, NS>(T, wx, wy, wz);
    }
    // out-of-range particles read particle 0 and are scaled by zero
    for (int pp = bf; pp < b1; ++pp) {
      const int i0 = 2 * pp * G + lg, i1 = i0 + G;
      const bool in0 = i0 < n, in1 = i1 < n;
      const int j0 = in0 ? i0 : 0, j1 = in1 ? i1 : 0;
      const float2 S2 = make_float2(in0 ? s : 0.f, in1 ? s : 0.f);
      const float2 wx = __fmul2_rn(__fadd2_rn(__fadd2_rn(make_float2(ld(px, j0), ld(px, j1)), nv0x), ndx), S2);
      const float2 wy = __fmul2_rn(__fadd2_rn(__fadd2_rn(make_float2(ld(py, j0), ld(py, j1)), nv0y), ndy), S2);
      const float2 wz = __fmul2_rn(__fadd2_rn(__fadd2_rn(make_float2(ld(pz, j0), ld(pz, j1)), nv0z), ndz), S2);
      accumulate2<kLite, NS>(T, wx, wy, wz);
    }
    // the block's sums over the group's lanes: each lane writes its row, the
    // owner of a float4 chunk adds the group's eight rows
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
  if (!valid) return;
  // the means (hi + lo) / n rounded to FP32
  float rh = 0.f, rl = 0.f;
  if (n > 0) df_recip((float)n, rh, rl);
  float4 *r4 = reinterpret_cast<float4 *>(rec);
  if (lg < NCH) {
    float mean[K];
#pragma unroll
    for (int j = 0; j < K; ++j) {
      float p, e;
      df_scale(hi[j], lo[j], rh, rl, p, e);
      mean[j] = p + e;
    }
    r4[lg] = make_float4(mean[0], mean[1], mean[2], mean[3]);
  }
  if (lg == 0) {
    r4[RX / 4] = make_float4(v0x, v0y, v0z, dx);
    r4[RX / 4 + 1] = make_float4(dy, dz, __int_as_float(ks), __int_as_float(n));
  }
}

// Finish one cell: read its staging record from its row (a copy in shared
// memory), convert the shifted means to central moments (FP32), undo the
// scale in the exponent and write the FP64 row over the record; <|c|^6> is
// returned in m6v.  One lane per cell.
template <bool kLite>
__device__ __forceinline__ void finish_row(double *row, double &m6v) {
  constexpr int NS = kLite ? kLiteSum : kFullSum;
  constexpr int RX = rec_x<kLite>();
  constexpr uint8_t kPairI[6] = {0, 0, 0, 1, 1, 2}, kPairJ[6] = {0, 1, 2, 1, 2, 2};  // 11,12,13,22,23,33
  const float4 *r4 = reinterpret_cast<const float4 *>(row);
  float M[4 * ((NS + 3) / 4)];
#pragma unroll
  for (int q = 0; q < (NS + 3) / 4; ++q) {
    const float4 t = r4[q];
    M[4 * q] = t.x;
    M[4 * q + 1] = t.y;
    M[4 * q + 2] = t.z;
    M[4 * q + 3] = t.w;
  }
  const float4 x0 = r4[RX / 4], x1 = r4[RX / 4 + 1];
  const float v0[3] = {x0.x, x0.y, x0.z}, dl[3] = {x0.w, x1.x, x1.y};
  const int ks = __float_as_int(x1.z), n = __float_as_int(x1.w);

  // symmetric second moments B_ij = <w_i w_j> and the mean offset d = <w>
  const int DA = kLite ? 9 : 26;
  const float d[3] = {M[DA], M[DA + 1], M[DA + 2]};
  float B[3][3];
  B[0][0] = M[0]; B[0][1] = B[1][0] = M[1]; B[0][2] = B[2][0] = M[2];
  B[1][1] = M[3]; B[1][2] = B[2][1] = M[4]; B[2][2] = M[5];
  const float Q = fmaf(d[0], d[0], fmaf(d[1], d[1], d[2] * d[2]));
  const float trB = (B[0][0] + B[1][1]) + B[2][2];
  float Bd[3], wR[3];
#pragma unroll
  for (int i = 0; i < 3; ++i) Bd[i] = fmaf(B[i][0], d[0], fmaf(B[i][1], d[1], B[i][2] * d[2]));

  double out[30];  // the row: N, U (3), theta, then the central moments
  out[0] = u2d_exact((uint32_t)n);
#pragma unroll
  for (int i = 0; i < 3; ++i) out[1 + i] = (f2d_scaled(v0[i], 0) + f2d_scaled(dl[i], 0)) + f2d_scaled(d[i], -ks);
#pragma unroll
  for (int q = 0; q < 6; ++q) {
    const int i = kPairI[q], j = kPairJ[q];
    out[kU2 + q] = f2d_scaled(fmaf(-d[i], d[j], B[i][j]), -2 * ks);
  }
  out[kTheta] = (out[kU2 + 0] + out[kU2 + 3] + out[kU2 + 5]) * (1.0 / 3.0);

  if constexpr (kLite) {
    // b_i = <c_i |c|^2> = <w_i R> - 2 (B d)_i - d_i tr B + 2 Q d_i
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      wR[i] = M[6 + i];
      const float b = fmaf(2.f * Q, d[i], fmaf(-d[i], trB, fmaf(-2.f, Bd[i], wR[i])));
      out[kU2 + 6 + i] = f2d_scaled(b, -3 * ks);
    }
    double2 *o2 = reinterpret_cast<double2 *>(row);
#pragma unroll
    for (int k = 0; k < FP_NLITE / 2; ++k) o2[k] = make_double2(out[2 * k], out[2 * k + 1]);
  } else {
    // third moments C_ijk (slot 6 + index of the sorted triple)
    float C[3][3][3];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
      for (int j = 0; j < 3; ++j)
#pragma unroll
        for (int k = 0; k < 3; ++k) {
          // sort (i, j, k) and map to 111,112,113,122,123,133,222,223,233,333
          const int a = min(i, min(j, k)), cc = max(i, max(j, k)), b = i + j + k - a - cc;
          const int t = a == 0 ? (b == 0 ? cc : (b == 1 ? 2 + cc : 5)) : (a == 1 ? (b == 1 ? 5 + cc : 8) : 9);
          C[i][j][k] = M[6 + t];
        }
    float D[3][3];
    D[0][0] = M[16]; D[0][1] = D[1][0] = M[17]; D[0][2] = D[2][0] = M[18];
    D[1][1] = M[19]; D[1][2] = D[2][1] = M[20]; D[2][2] = M[21];
    const float E[3] = {M[22], M[23], M[24]}, F = M[25];
    float Cd[3][3], Dd[3], dCd[3], t[3];
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      wR[i] = (C[i][0][0] + C[i][1][1]) + C[i][2][2];
#pragma unroll
      for (int j = 0; j < 3; ++j) Cd[i][j] = fmaf(C[i][j][0], d[0], fmaf(C[i][j][1], d[1], C[i][j][2] * d[2]));
      Dd[i] = fmaf(D[i][0], d[0], fmaf(D[i][1], d[1], D[i][2] * d[2]));
    }
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      dCd[i] = fmaf(Cd[i][0], d[0], fmaf(Cd[i][1], d[1], Cd[i][2] * d[2]));
      t[i] = fmaf(Q, d[i], fmaf(-2.f, Bd[i], wR[i]));  // <w_i |c|^2>
    }
    // u_ijk = C_ijk - d_i B_jk - d_j B_ik - d_k B_ij + 2 d_i d_j d_k
    constexpr uint8_t I3[10][3] = {{0, 0, 0}, {0, 0, 1}, {0, 0, 2}, {0, 1, 1}, {0, 1, 2},
                                   {0, 2, 2}, {1, 1, 1}, {1, 1, 2}, {1, 2, 2}, {2, 2, 2}};
#pragma unroll
    for (int q = 0; q < 10; ++q) {
      const int i = I3[q][0], j = I3[q][1], k = I3[q][2];
      float u = fmaf(-d[i], B[j][k], C[i][j][k]);
      u = fmaf(-d[j], B[i][k], u);
      u = fmaf(-d[k], B[i][j], u);
      u = fmaf(2.f * d[i] * d[j], d[k], u);
      out[kU3 + q] = f2d_scaled(u, -3 * ks);
    }
    // <c_i c_j |c|^2> = (D_ij - 2 (C d)_ij + Q B_ij) - d_i t_j - d_j t_i + d_i d_j (tr B - Q)
    const float t0 = trB - Q;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const int i = kPairI[q], j = kPairJ[q];
      float w = fmaf(Q, B[i][j], fmaf(-2.f, Cd[i][j], D[i][j]));
      w = fmaf(-d[i], t[j], w);
      w = fmaf(-d[j], t[i], w);
      w = fmaf(d[i] * d[j], t0, w);
      out[kW + q] = f2d_scaled(w, -4 * ks);
    }
    // <c_i |c|^4> = <w_i |c|^4> - d_i <|c|^4>, with |c|^4 = R^2 - 4RL + 2RQ + 4L^2 - 4LQ + Q^2
    const float RR = (D[0][0] + D[1][1]) + D[2][2];
    const float RL = fmaf(d[0], wR[0], fmaf(d[1], wR[1], d[2] * wR[2]));
    const float LL = fmaf(d[0], Bd[0], fmaf(d[1], Bd[1], d[2] * Bd[2]));
    const float QQ = Q * Q;
    const float s4 = fmaf(-3.f, QQ, fmaf(4.f, LL, fmaf(2.f * Q, trB, fmaf(-4.f, RL, RR))));
#pragma unroll
    for (int i = 0; i < 3; ++i) {
      float z = fmaf(-4.f, Dd[i], E[i]);
      z = fmaf(2.f * Q, wR[i], z);
      z = fmaf(4.f, dCd[i], z);
      z = fmaf(-4.f * Q, Bd[i], z);
      z = fmaf(QQ, d[i], z);
      z = fmaf(-d[i], s4, z);
      out[kZ + i] = f2d_scaled(z, -5 * ks);
    }
    double2 *o2 = reinterpret_cast<double2 *>(row);
#pragma unroll
    for (int k = 0; k < FP_NMOM / 2; ++k) o2[k] = make_double2(out[2 * k], out[2 * k + 1]);
    {
      // <|c|^6> = <R^3> - 6<R^2 L> + 3Q<R^2> + 12<R L^2> - 12Q<R L> + 3Q^2<R>
      //           - 8<L^3> + 12Q<L^2> - 6Q^2<L> + Q^3, with <L> = Q
      const float R2L = fmaf(d[0], E[0], fmaf(d[1], E[1], d[2] * E[2]));
      const float RLL = fmaf(d[0], Dd[0], fmaf(d[1], Dd[1], d[2] * Dd[2]));
      const float LLL = fmaf(d[0], dCd[0], fmaf(d[1], dCd[1], d[2] * dCd[2]));
      float s6 = fmaf(-6.f, R2L, F);
      s6 = fmaf(3.f * Q, RR, s6);
      s6 = fmaf(12.f, RLL, s6);
      s6 = fmaf(-12.f * Q, RL, s6);
      s6 = fmaf(3.f * QQ, trB, s6);
      s6 = fmaf(-8.f, LLL, s6);
      s6 = fmaf(12.f * Q, LL, s6);
      s6 = fmaf(-5.f * QQ, Q, s6);
      m6v = f2d_scaled(s6, -6 * ks);
    }
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
  if (ncell <= 32) {  // warp-uniform: one element a lane, a 32-element network
    uint32_t k1 = lane < ncell ? ((uint32_t)(na + 1) << 6) | (uint32_t)(63 - lane) : 0u;
#pragma unroll
    for (int k = 2; k <= 32; k <<= 1) {
#pragma unroll
      for (int j = k >> 1; j >= 1; j >>= 1) {
        const uint32_t p = __shfl_xor_sync(0xffffffffu, k1, j);
        const bool lower = (lane & j) == 0, up = (lane & k) == 0;
        k1 = (lower == up) ? (k1 > p ? k1 : p) : (k1 > p ? p : k1);
      }
    }
    if (lane < ncell) order[lane] = (uint8_t)(63 - (k1 & 63u));
    return;
  }
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
__global__ void __launch_bounds__(kTileThreads, kCtasPerSm)
    gather_tile_kernel(const float *__restrict__ v, int64_t np, const int64_t *__restrict__ off, int64_t n_cells,
                       double *__restrict__ mom, double *__restrict__ m6, int64_t n_chunks) {
  extern __shared__ __align__(128) float slot_buf[];
  float *scratch_all = slot_buf + kSlots * kSlotFloats;
  __shared__ __align__(16) float zeros[4];
  __shared__ __align__(8) uint64_t full_bar[kSlots], empty_bar[kSlots];
  __shared__ SlotMeta meta[kSlots];
  __shared__ int task_ctr[kSlots];
  __shared__ int failed;
  constexpr int kStride = kLite ? FP_NLITE : FP_NMOM;
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
      const int64_t cs = M.cs, ce = M.ce;
      const int ncell = (int)(ce - cs);
      while (true) {
        int task = 0;
        if (lane == 0) task = atomicAdd(&task_ctr[s], 1);
        task = __shfl_sync(0xffffffffu, task, 0);
        const int r0 = task * kCellsPerTask;
        if (r0 >= ncell) break;
        const int r = r0 + g;
        const bool valid = r < ncell;
        const int rc = valid ? (int)M.order[r] : 0;
        const int64_t c = cs + rc;
        const int64_t a = M.offs[rc];
        const int n = valid ? (int)(M.offs[rc + 1] - a) : 0;
        float *rec = reinterpret_cast<float *>(mom + c * kStride);
        if (M.big) {
          gather_cells<false, kLite>(valid, n, v + a, v + np + a, v + 2 * np + a, rec, scratch, zeros, lane);
        } else {
          const int64_t rel = a - M.pa;
          gather_cells<true, kLite>(valid, n, bx + M.lead[0] + rel, bx + kCapF + M.lead[1] + rel,
                                    bx + 2 * kCapF + M.lead[2] + rel, rec, scratch, zeros, lane);
        }
      }
      __syncwarp();
      if (lane == 0) asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(smem_u32(&empty_bar[s])) : "memory");
    }
    if (!ok && lane == 0) atomicExch(&failed, 1);
  }
  __syncthreads();
  if (failed) {
    mark_failed(n_cells, n_chunks, mom, kStride, tid);
    return;
  }
  // finish this CTA's cells (their records were written by this CTA's
  // consumers, ordered by the barrier above): a warp takes 32 consecutive
  // rows, copies them into shared memory (the idle slots) with coalesced
  // 16-byte loads, finishes one row a lane there and copies them back
  constexpr int kBlk = 32;
  double *stage = reinterpret_cast<double *>(slot_buf) + (size_t)warp * kBlk * kStride;
  float4 *st4 = reinterpret_cast<float4 *>(stage);
  const int64_t my_chunks = n_chunks > blockIdx.x ? (n_chunks - blockIdx.x + gridDim.x - 1) / gridDim.x : 0;
  for (int64_t b = warp; b < my_chunks * (kChunkCells / kBlk); b += kTileThreads / 32) {
    const int64_t c0 = (blockIdx.x + (b / (kChunkCells / kBlk)) * (int64_t)gridDim.x) * kChunkCells +
                       (b % (kChunkCells / kBlk)) * kBlk;
    if (c0 >= n_cells) continue;  // warp-uniform
    const int nc = (int)(n_cells - c0 < kBlk ? n_cells - c0 : kBlk);
    const int nv = nc * kStride / 2;  // float4s of the block's rows
    const float4 *src = reinterpret_cast<const float4 *>(mom + c0 * kStride);
    for (int k = lane; k < nv; k += 32) st4[k] = src[k];
    __syncwarp();
    double m6v = 0.0;
    if (lane < nc) finish_row<kLite>(stage + lane * kStride, m6v);
    __syncwarp();
    float4 *dst = reinterpret_cast<float4 *>(mom + c0 * kStride);
    for (int k = lane; k < nv; k += 32) dst[k] = st4[k];
    if (!kLite && m6 && lane < nc) m6[c0 + lane] = m6v;
    __syncwarp();
  }
}

static int g_tile_attr_done[2][64];

template <bool kLite>
static bool launch_tile(const float *v, int64_t np, const int64_t *off, int64_t n_cells, double *mom, double *m6,
                        cudaStream_t st, int sm_count) {
  if (((uintptr_t)v & 15) != 0 || ((uintptr_t)mom & 15) != 0) return false;  // 16-byte record stores
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !g_tile_attr_done[kLite][dev]) {
    if (cudaFuncSetAttribute(gather_tile_kernel<kLite>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTileSmem) != cudaSuccess)
      return false;
    g_tile_attr_done[kLite][dev] = 1;
  }
  const int64_t n_chunks = (n_cells + kChunkCells - 1) / kChunkCells;
  int64_t grid = (int64_t)sm_count * kCtasPerSm;
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
