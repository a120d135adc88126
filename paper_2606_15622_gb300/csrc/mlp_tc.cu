// mlp_tc.cu -- inference forward pass of the learned closure's network
// (32 -> 4 x [128, SiLU] -> 16, BF16 operands, FP32 accumulation) on the
// fifth-generation tensor cores of sm_103a.
//
// One persistent CTA per SM keeps all five weight matrices in shared memory.
// Its two groups of eight warps each stream their own 128-row tiles; two
// threads (warps w and w + 4 of the group, which share TMEM lanes 32 (w % 4)
// ..) own each row and split every 32 columns.  Per tile and layer:
//   - the layer's accumulators D[l] (128 x 128 FP32, tensor memory) are read
//     32 columns at a time with tcgen05.ld; bias, SiLU (through tanh) and
//     BF16 rounding turn them into 32 columns of the next layer's A operand
//     in shared memory;
//   - after each 32-column chunk the group's leader issues the next layer's
//     tcgen05.mma instructions over those 32 K-columns (M = 128, K = 16 each,
//     N = 128, or 16 for the output layer) into the other accumulator buffer
//     D[l + 1], so the tensor cores work while the epilogue continues, and
//     commits the layer to the group's mbarrier after the last chunk;
//   - the input tile of the next tile is staged in its own buffer as soon as
//     the first layer's MMAs have consumed the current one.
// The output layer adds its bias, undoes the target standardisation if asked
// and stores 16 FP32 per row.
// Operands use the canonical K-major layout without swizzle: 8-row x 16-byte
// "core matrices", adjacent along K at 128 bytes (leading byte offset) and
// along M/N at K * 16 bytes (stride byte offset); enumerating (8-row group,
// K-chunk, row) makes that layout linear, so the staging copies (cp.async,
// all in flight at once) write contiguous shared memory.
// With kDrop (the coefficient-sensitivity probe) every hidden activation is
// kept with probability 1 - rate and scaled by 1 / (1 - rate), or set to
// zero, after the SiLU and before the BF16 rounding.  The decision for row
// r, pass k, layer l, column j uses word j % 4 of Philox4x32-10 (key = the
// probe's seed) on counter (r lo, r hi, k, 32 l + j / 4): dropped when
// (floor(w / 2^8) + 1) 2^-24 <= rate.
// The learned closure runs as one instance of this kernel: the group's two
// threads per row form the row's inputs from its moment (or LITE) vector
// straight into the input tile -- the next tile's rows are bulk-prefetched
// into L2 while the current tile runs, and formed once its last layer is
// done -- and the output threads turn the predictions into coefficients,
// check the energy residual, write the flags and append the cells that need
// the exact closure to a list (one atomic per warp), so the inputs and the
// predictions never travel through HBM.
// Only the group's leader waits on the mbarrier, with a bound, and passes its
// outcome to the group through shared memory at the next group barrier; a
// wait that runs out marks the group's remaining rows (NaN outputs, or
// non-finite cells that the exact fallback or the linear drift serves), and
// the CTA frees its tensor memory before returning.
#include <cstdint>
#include <cuda_bf16.h>

#include "fp_device.cuh"
#include "mlp_common.cuh"
#include "tc_common.cuh"
#include "tma.cuh"

namespace fpc {

namespace {

constexpr int kTcRows = 128;                 // rows per tile = TMEM lanes
constexpr int kTcGroups = 2;                 // tiles in flight per CTA
constexpr int kTcGroupThreads = 256;         // two threads per row: 16 of every 32 columns each
constexpr int kTcThreads = kTcGroupThreads * kTcGroups;
constexpr uint32_t kTmemCols = 512;          // two 128-column accumulators per group

// shared-memory carve-up (bytes from a 1024-byte aligned base)
constexpr uint32_t kOffW1 = 0;                                 // [128][32]  8 KB
constexpr uint32_t kOffWH = kOffW1 + kHid * kIn * 2;           // 3 x [128][128]
constexpr uint32_t kOffW5 = kOffWH + 3 * kHid * kHid * 2;      // [16][128]
constexpr uint32_t kOffA = kOffW5 + kOut * kHid * 2;           // 2 x [128][128] activations
constexpr uint32_t kOffX = kOffA + kTcGroups * kTcRows * kHid * 2;  // 2 x [128][32] input tiles
constexpr uint32_t kOffBias = kOffX + kTcGroups * kTcRows * kIn * 2;
constexpr uint32_t kNBias = 4 * kHid + 3 * kOut;               // b1..b4 / 2, b5, y_mu, y_sigma
constexpr uint32_t kOffBar = kOffBias + kNBias * 4;            // 2 mbarriers
constexpr uint32_t kOffTmemSlot = kOffBar + 8 * kTcGroups;       // TMEM address + two outcomes
constexpr uint32_t kOffScal = kOffTmemSlot + 16;               // [32] float4 input scalers (closure variants)
constexpr uint32_t kOffFlags = kOffScal + 4 * kIn * 4;         // [2 groups][2 parities][128] part-1 input flags
constexpr uint32_t kTcSmemUsed = kOffFlags + kTcGroups * 2 * kTcRows * 4;
constexpr size_t kTcSmem = kTcSmemUsed + 1024;                 // room to align the base
static_assert(kOffBar % 8 == 0, "mbarrier alignment");
static_assert(kOffScal % 16 == 0, "float4 scalers");
static_assert(kTcSmem <= 227 * 1024, "shared memory");

__device__ __forceinline__ void group_sync(int g) {
  asm volatile("bar.sync %0, %1;" ::"r"(1 + g), "r"(kTcGroupThreads) : "memory");
}

// SiLU(z) = z sigma(z) with sigma(z) = (1 + tanh(z / 2)) / 2: one hardware
// tanh (relative error about 2^-11, below the 2^-9 of the BF16 rounding
// that follows) instead of an exponential and a reciprocal.  Called with
// the accumulator a and the halved bias hb: z / 2 = a / 2 + hb.
__device__ __forceinline__ float silu_tanh(float a, float hb) {
  const float hz = fmaf(a, 0.5f, hb);
  float t;
  asm("tanh.approx.f32 %0, %1;" : "=f"(t) : "f"(hz));
  return fmaf(hz, t, hz);
}

// bias + SiLU (+ dropout) of 16 accumulators (columns 16 h16 .. 16 h16 + 15)
// -> two 16-byte chunks of BF16 in the next layer's A operand (row `row`)
template <bool kDrop>
__device__ __forceinline__ void epilogue16(const uint32_t (&r)[16], const float *__restrict__ hb, unsigned char *A,
                                           int row, int h16, const DropoutCfg &dc, int64_t cell, int layer) {
  float keep[16];
  if (kDrop) {
#pragma unroll
    for (int g4 = 0; g4 < 4; ++g4) {
      const uint32_t ctr3 = (uint32_t)(32 * layer + (h16 * 16 + 4 * g4) / 4);
      const uint4 w = philox4x32_10(make_uint4((uint32_t)cell, (uint32_t)((uint64_t)cell >> 32), dc.pass, ctr3),
                                    dc.key);
      const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const float u = ((float)(ws[e] >> 8) + 1.f) * 5.9604644775390625e-08f;  // (0, 1], exact
        keep[4 * g4 + e] = u <= dc.rate ? 0.f : dc.scale;
      }
    }
  }
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    const float4 b0 = *reinterpret_cast<const float4 *>(hb + h16 * 16 + q * 8);
    const float4 b1 = *reinterpret_cast<const float4 *>(hb + h16 * 16 + q * 8 + 4);
    const float bq[8] = {b0.x, b0.y, b0.z, b0.w, b1.x, b1.y, b1.z, b1.w};
    uint32_t pk[4];
#pragma unroll
    for (int e = 0; e < 4; ++e) {
      float a0 = silu_tanh(__uint_as_float(r[q * 8 + 2 * e]), bq[2 * e]);
      float a1 = silu_tanh(__uint_as_float(r[q * 8 + 2 * e + 1]), bq[2 * e + 1]);
      if (kDrop) {
        a0 *= keep[q * 8 + 2 * e];
        a1 *= keep[q * 8 + 2 * e + 1];
      }
      pk[e] = pack_bf16(a0, a1);
    }
    *reinterpret_cast<uint4 *>(A + cm_off(row, h16 * 2 + q, kHid)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  }
}

// ---------------------------------------------------------------------------
// learned closure fused around the network: inputs formed from the moment
// rows in the prologue, coefficients and checks in the output epilogue
// ---------------------------------------------------------------------------
constexpr int kSrcX = 0;     // BF16 inputs given (standalone forward pass)
constexpr int kSrcFull = 1;  // full inputs from moment vectors [n][FP_NMOM]
constexpr int kSrcLite = 2;  // LITE inputs from LITE vectors [n][FP_NLITE]

constexpr int kPreMask = FP_FLAG_FEW | FP_FLAG_SINGULAR | FP_FLAG_NONFINITE;  // the exact closure's preconditions
constexpr int kFallbackMask = kPreMask | FP_FLAG_RANGE | FP_FLAG_ENERGY;

// what the epilogue of one row needs from its inputs, held by the row's
// output thread (half 0) from the end of the previous tile to the output
// layer: the normalised u^_ij, b^_i = u^_ikk and s4^ = w^_kk of the energy
// check (full inputs), tau, 1 / tau and 1 / (tau sqrt(theta)), and the flags
// of the inputs this thread formed
struct RowState {
  float u[6], b[3], s4, itc, ig;
  double tc;
  int fl;
};

// FP_NMOM or FP_NLITE doubles per row
template <int kSrc>
constexpr int src_stride() {
  return kSrc == kSrcFull ? FP_NMOM : FP_NLITE;
}

// Bulk prefetch into L2 of rows [r0, r1) of the row-major source and of
// tau[r0, r1): the byte ranges are trimmed to 16-byte boundaries and cut
// into 4 KB pieces, one per thread t < pieces (the ranges lie inside the
// caller's arrays; a prefetch completes nothing and is waited for by no one).
template <int kSrc>
__device__ __forceinline__ void prefetch_rows(const FusedIO &io, int64_t r0, int64_t r1, int t) {
  const uintptr_t a0 = (uintptr_t)(io.src + r0 * src_stride<kSrc>()), a1 = (uintptr_t)(io.src + r1 * src_stride<kSrc>());
  const uintptr_t s = (a0 + 15) & ~(uintptr_t)15, e = a1 & ~(uintptr_t)15;
  const int pieces = e > s ? (int)((e - s + 4095) / 4096) : 0;
  if (t < pieces) {
    const uintptr_t p = s + 4096 * (uintptr_t)t;
    const uint32_t bytes = (uint32_t)(e - p < 4096 ? e - p : 4096);
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(p), "r"(bytes) : "memory");
  } else if (t == pieces) {
    const uintptr_t b0 = ((uintptr_t)(io.tau + r0) + 15) & ~(uintptr_t)15, b1 = (uintptr_t)(io.tau + r1) & ~(uintptr_t)15;
    if (b1 > b0) asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;" ::"l"(b0), "r"((uint32_t)(b1 - b0)) : "memory");
  }
}

// standardise features f[0, cnt) (feature indices q0 + k), check them
// against the widened training box, round to BF16 and pack 16 of them (the
// rest zero) into two 16-byte chunks
__device__ __forceinline__ int standardise16(const float *f, int q0, int cnt, const float4 *__restrict__ scal,
                                             uint32_t (&pk)[8]) {
  int fl = 0;
  float xs[16];
#pragma unroll
  for (int k = 0; k < 16; ++k) {
    xs[k] = 0.f;
    if (k < cnt) {
      const float4 sc = scal[q0 + k];  // mu, 1 / sigma, box low, box high
      if (!(f[k] >= sc.z && f[k] <= sc.w)) fl |= FP_FLAG_RANGE;
      xs[k] = standardise(f[k], sc.x, sc.y);
    }
  }
#pragma unroll
  for (int k = 0; k < 8; ++k) pk[k] = pack_bf16(xs[2 * k], xs[2 * k + 1]);
  return fl;
}

// Inputs of row `row` (cell c) of the next tile, formed by its two threads:
// part 0 the normalised u_ij / theta and u_ijk / theta^1.5 (features 0..15),
// the preconditions and the epilogue's state; part 1 w_ij / theta^2 and
// z_i / theta^2.5 (features 16..24).  Arithmetic as fp_surrogate_features
// (moments narrowed to FP32, FP32 powers of 1 / theta).
// Each part writes two 16-byte chunks of the row in X (zeros past n) and its
// flags (part 0 to `st`, part 1 to `fl_part1`).
__device__ __forceinline__ void form_full_inputs(const FusedIO &io, const float4 *__restrict__ scal, int64_t c,
                                                 int64_t n, int part, unsigned char *X, int row, int *fl_part1,
                                                 RowState &st) {
  uint32_t pk[8];
  int fl = 0;
  if (c < n) {
    const double *m = io.src + c * FP_NMOM;
    const double thd = m[kTheta];
    const float th = narrow(thd);
    const float i1 = 1.f / th;
    const float ih = rsqrtf(th);
    const float i15 = i1 * ih, i2 = i1 * i1, i25 = i2 * ih;
    float f[16];
    if (part == 0) {
      const double tc = io.tau[c], nd = m[kN];
      bool fin = finite_d(tc) && positive_d(tc) && finite_d(nd) && finite_d(thd);
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const double v = m[kU2 + a];
        fin = fin && finite_d(v);
        f[a] = narrow(v) * i1;
      }
#pragma unroll
      for (int a = 0; a < 10; ++a) {
        const double v = m[kU3 + a];
        fin = fin && finite_d(v);
        f[6 + a] = narrow(v) * i15;
      }
      if (!fin) fl |= FP_FLAG_NONFINITE;
      if (narrow(nd) < (float)io.min_particles) fl |= FP_FLAG_FEW;  // N is a whole number
      if (!positive_d(thd)) fl |= FP_FLAG_SINGULAR;
#pragma unroll
      for (int a = 0; a < 6; ++a) st.u[a] = f[a];
      st.b[0] = f[6 + 0] + f[6 + 3] + f[6 + 5];
      st.b[1] = f[6 + 1] + f[6 + 6] + f[6 + 8];
      st.b[2] = f[6 + 2] + f[6 + 7] + f[6 + 9];
      st.s4 = narrow(m[kW + 0]) * i2 + narrow(m[kW + 3]) * i2 + narrow(m[kW + 5]) * i2;
      st.itc = 1.f / narrow(tc);
      st.ig = st.itc / sqrtf(th);
      st.tc = tc;
      fl |= standardise16(f, 0, 16, scal, pk);
    } else {
      bool fin = true;
#pragma unroll
      for (int a = 0; a < 3; ++a) fin = fin && finite_d(m[kU + a]);
#pragma unroll
      for (int a = 0; a < 6; ++a) {
        const double v = m[kW + a];
        fin = fin && finite_d(v);
        f[a] = narrow(v) * i2;
      }
#pragma unroll
      for (int a = 0; a < 3; ++a) {
        const double v = m[kZ + a];
        fin = fin && finite_d(v);
        f[6 + a] = narrow(v) * i25;
      }
      if (!fin) fl |= FP_FLAG_NONFINITE;
      fl |= standardise16(f, 16, kNFeat - 16, scal, pk);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) pk[k] = 0u;
  }
  *reinterpret_cast<uint4 *>(X + cm_off(row, 2 * part, kIn)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  *reinterpret_cast<uint4 *>(X + cm_off(row, 2 * part + 1, kIn)) = make_uint4(pk[4], pk[5], pk[6], pk[7]);
  if (part == 0)
    st.fl = fl;
  else
    *fl_part1 = fl;
}

// LITE inputs of row `row` (cell c): both threads form the 16 raw inputs
// (arithmetic of fp_surrogate_lite_features); part p standardises inputs
// 8p .. 8p + 7 into chunk p and zeroes chunk 2 + p.
__device__ __forceinline__ void form_lite_inputs(const FusedIO &io, const float4 *__restrict__ scal, int64_t c,
                                                 int64_t n, int part, unsigned char *X, int row, int *fl_part1,
                                                 RowState &st) {
  uint32_t pk[8];
  int fl = 0;
  if (c < n) {
    const double *m = io.src + c * FP_NLITE;
    const double tc = io.tau[c];
    bool fin = finite_d(tc) && positive_d(tc);
#pragma unroll
    for (int k = 0; k < FP_NLITE; ++k) fin = fin && finite_d(m[k]);
    float f[16];
    lite_raw_features(m, tc, f);
    if (part == 0) {
      if (!fin) fl |= FP_FLAG_NONFINITE;
      if (narrow(m[0]) < (float)io.min_particles) fl |= FP_FLAG_FEW;  // N is a whole number
      if (!positive_d(m[4])) fl |= FP_FLAG_SINGULAR;
      st.tc = tc;
      st.itc = 1.f / narrow(tc);
      st.ig = st.itc / sqrtf(narrow(m[4]));
      fl |= standardise16(f, 0, 8, scal, pk);
    } else {
      fl |= standardise16(f + 8, 8, 8, scal, pk);
    }
  } else {
#pragma unroll
    for (int k = 0; k < 8; ++k) pk[k] = 0u;
  }
  *reinterpret_cast<uint4 *>(X + cm_off(row, part, kIn)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
  *reinterpret_cast<uint4 *>(X + cm_off(row, 2 + part, kIn)) = make_uint4(0u, 0u, 0u, 0u);
  if (part == 0)
    st.fl = fl;
  else
    *fl_part1 = fl;
}

// Append cell c to the fallback list when `pick` (warp-aggregated: one
// atomic per warp; all 32 lanes call this together).
__device__ __forceinline__ void append_fallback(const FusedIO &io, bool pick, int64_t c, int lane) {
  const unsigned m = __ballot_sync(0xffffffffu, pick);
  if (!m) return;
  uint32_t base = 0;
  if (lane == 0) base = atomicAdd(io.count, (uint32_t)__popc(m));
  base = __shfl_sync(0xffffffffu, base, 0);
  if (pick) io.list[base + __popc(m & ((1u << lane) - 1u))] = (int32_t)c;
}

// Output epilogue of the full-input learned closure for cell c (v: the
// un-standardised predictions tau C, tau sqrt(theta) G): cells failing the
// exact closure's preconditions are left to the fallback; otherwise the
// energy residual e = 1 + (sum_ij C^_ij u^_ij + sum_i G^_i b^_i
// - eps2_hat s4^) / 3 of the predicted drift is checked and, for a cell that
// passes every check, C = t / tau and G = t / (tau sqrt(theta)) are scaled in
// FP32 and widened exactly.  Returns whether the cell goes to the fallback.
__device__ __forceinline__ bool full_epilogue(const FusedIO &io, const float (&v)[kOut], const RowState &st,
                                              int fl, int64_t c) {
  if (!(fl & kPreMask)) {
    bool fin = true;
#pragma unroll
    for (int a = 0; a < kNOut; ++a) fin = fin && isfinite(v[a]);
    const float cu = v[0] * st.u[0] + 2.f * v[1] * st.u[1] + 2.f * v[2] * st.u[2] + v[3] * st.u[3] +
                     2.f * v[4] * st.u[4] + v[5] * st.u[5];
    const float e = 1.f + (cu + v[6] * st.b[0] + v[7] * st.b[1] + v[8] * st.b[2] - io.eps2_hat * st.s4) * (1.f / 3.f);
    if (!fin) fl |= FP_FLAG_NONFINITE;
    if (!(fabsf(e) <= io.energy_tol)) fl |= FP_FLAG_ENERGY;
    if (!(fl & kFallbackMask)) {
      double *y = io.coeffs + c * 9;
#pragma unroll
      for (int a = 0; a < 6; ++a) y[a] = f2d_exact(v[a] * st.itc);
#pragma unroll
      for (int a = 6; a < 9; ++a) y[a] = f2d_exact(v[a] * st.ig);
    }
  }
  io.flags[c] = fl;
  return (fl & kFallbackMask) != 0;
}

// the linear drift C = -I / tau, G = 0 (zero for a tau that is not a
// positive finite number)
__device__ __forceinline__ void linear_drift(double *y, double tc) {
  const double c0 = (finite_d(tc) && positive_d(tc)) ? -1.0 / tc : 0.0;
#pragma unroll
  for (int q = 0; q < 9; ++q) y[q] = 0.0;
  y[0] = c0;
  y[3] = c0;
  y[5] = c0;
}

// Output epilogue of the LITE closure: degenerate cells and non-finite
// predictions take the linear drift, the others the scaled predictions.
__device__ __forceinline__ void lite_epilogue(const FusedIO &io, const float (&v)[kOut], const RowState &st, int fl,
                                              int64_t c) {
  bool fin = true;
#pragma unroll
  for (int a = 0; a < kNOut; ++a) fin = fin && isfinite(v[a]);
  if (!fin) fl |= FP_FLAG_NONFINITE;
  double *y = io.coeffs + c * 9;
  if (fl & kPreMask) {
    linear_drift(y, st.tc);
  } else {
#pragma unroll
    for (int a = 0; a < 6; ++a) y[a] = f2d_exact(v[a] * st.itc);
#pragma unroll
    for (int a = 6; a < 9; ++a) y[a] = f2d_exact(v[a] * st.ig);
  }
  io.flags[c] = fl;
}

}  // namespace

// kSrc = kSrcX: the forward pass on given BF16 inputs x (with kDrop, the
// dropout masks of the sensitivity probe).  kSrc = kSrcFull / kSrcLite: the
// learned closure from moment / LITE vectors (io), the inputs formed by the
// group's threads into the input tile and the coefficients written by the
// output epilogue; x and out are unused.
template <bool kDrop, int kSrc>
__global__ void __launch_bounds__(kTcThreads, 1)
    mlp_forward_tc_kernel(MlpDev net, const __nv_bfloat16 *__restrict__ x, int64_t n, int standardized_out,
                          float *__restrict__ out, DropoutCfg dc, FusedIO io) {
  static_assert(kSrc == kSrcX || !kDrop, "dropout only on given inputs");
  extern __shared__ unsigned char smem_raw[];
  unsigned char *sm = smem_raw + ((1024u - (smem_u32(smem_raw) & 1023u)) & 1023u);
  float *bias = reinterpret_cast<float *>(sm + kOffBias);
  float4 *scal = reinterpret_cast<float4 *>(sm + kOffScal);
  int *fl_part1 = reinterpret_cast<int *>(sm + kOffFlags);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kOffBar);
  uint32_t *tmem_slot = reinterpret_cast<uint32_t *>(sm + kOffTmemSlot);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = warp >> 3;                      // group
  const int half = (warp >> 2) & 1;             // which 16 of every 32 columns
  const int row = (warp & 3) * 32 + lane;       // = TMEM lane (warps may use lanes 32 (warp % 4) ..)

  const int gt = tid & (kTcGroupThreads - 1);  // thread index within the group
  const int64_t n_tiles = (n + kTcRows - 1) / kTcRows;
  const int64_t tile_step = (int64_t)gridDim.x * kTcGroups;
  int64_t tile = (int64_t)blockIdx.x * kTcGroups + g;
  // the rows of the group's first tile head for L2 while the weights load
  if (kSrc != kSrcX && tile < n_tiles)
    prefetch_rows<kSrc>(io, tile * kTcRows, tile * kTcRows + kTcRows < n ? tile * kTcRows + kTcRows : n, gt);

  // ---- one-time setup: weights, biases, scalers, barriers, tensor memory ----
  stage_rows_async(sm + kOffW1, net.W[0], kHid, kIn, kHid, tid, kTcThreads);
  for (int l = 0; l < 3; ++l)
    stage_rows_async(sm + kOffWH + l * kHid * kHid * 2, net.W[1 + l], kHid, kHid, kHid, tid, kTcThreads);
  stage_rows_async(sm + kOffW5, net.W[4], kOut, kHid, kOut, tid, kTcThreads);
  // (the parameter arrays indexed by constants only: no local-memory copy)
  if (tid < kHid) {
#pragma unroll
    for (int l = 0; l < 4; ++l) bias[l * kHid + tid] = 0.5f * net.b[l][tid];  // hidden biases halved (see silu_tanh)
  } else if (tid < kHid + kOut) {
    const int j = tid - kHid;
    bias[4 * kHid + j] = net.b[4][j];
    bias[4 * kHid + kOut + j] = net.y_mu[j];
    bias[4 * kHid + 2 * kOut + j] = net.y_sigma[j];
  }
  if (kSrc != kSrcX && tid < kIn) {
    // mu, 1 / sigma and the widened training box [x_min - m sigma, x_max + m sigma]
    const int nf = kSrc == kSrcFull ? kNFeat : 16;
    if (tid < nf) {
      const float sg = net.x_sigma[tid];
      scal[tid] = make_float4(net.x_mu[tid], 1.f / sg, net.x_min[tid] - io.margin * sg,
                              net.x_max[tid] + io.margin * sg);
    } else {
      scal[tid] = make_float4(0.f, 1.f, 0.f, 0.f);
    }
  }
  if (tid == 0) {
    for (int q = 0; q < kTcGroups; ++q) mbar_init(&bar[q], 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(tmem_slot)),
                 "r"(kTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  __syncthreads();  // scalers and the tensor-memory address are visible; the weights may still be in flight

  unsigned char *A = sm + kOffA + g * (kTcRows * kHid * 2);
  unsigned char *X = sm + kOffX + g * (kTcRows * kIn * 2);
  int *flp = fl_part1 + g * 2 * kTcRows;  // part-1 flags of the group, by tile parity
  RowState st;
  // the first tile's inputs while the weight copies land
  if (tile < n_tiles) {
    if constexpr (kSrc == kSrcX)
      stage_rows_async(X, x + tile * kTcRows * kIn, kTcRows, kIn, n - tile * kTcRows, gt, kTcGroupThreads);
    else if constexpr (kSrc == kSrcFull)
      form_full_inputs(io, scal, tile * kTcRows + row, n, half, X, row, flp + row, st);
    else
      form_lite_inputs(io, scal, tile * kTcRows + row, n, half, X, row, flp + row, st);
  }
  cp_async_wait();
  fence_proxy_async_smem();  // weights written through the generic proxy, read by the MMA
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = *tmem_slot + (uint32_t)(g * 2 * kHid);  // the group's two accumulators
  const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;   // this warp's TMEM lanes
  const uint32_t a_addr = smem_u32(A), x_addr = smem_u32(X);
  const uint32_t w1_addr = smem_u32(sm + kOffW1), wh_addr = smem_u32(sm + kOffWH), w5_addr = smem_u32(sm + kOffW5);
  const bool leader = gt == 0;
  volatile uint32_t *group_ok = tmem_slot + 1 + g;  // the leader's outcome on the last wait
  uint32_t phase = 0;
  bool failed = false;

  // the leader waits for the group's last commit; the group learns the outcome
  auto wait_layer = [&]() -> bool {
    if (leader) *group_ok = mma_wait(&bar[g], phase) ? 1u : 0u;
    phase ^= 1u;
    group_sync(g);
    tc_fence_after();
    return *group_ok != 0u;
  };

  for (int it = 0; tile < n_tiles; tile += tile_step, ++it) {
    const int64_t row0 = tile * kTcRows;
    const int64_t next = tile + tile_step;
    if (!failed) {
      // layer 1: D[0] = X W1^T
      if constexpr (kSrc == kSrcX) cp_async_wait();  // this thread's part of the input tile has landed
      fence_proxy_async_smem();
      tc_fence_before();
      group_sync(g);
      if (leader) {
        tc_fence_after();
        for (int s = 0; s < kIn / 16; ++s)
          tc_mma(tmem, smem_desc(x_addr + 256 * s, 128, kIn * 16), smem_desc(w1_addr + 256 * s, 128, kIn * 16),
                 idesc_bf16(kTcRows, kHid), s > 0 ? 1u : 0u);
        tc_commit(&bar[g]);
      }
      if (kSrc != kSrcX && next < n_tiles) {
        const int64_t r1 = next * kTcRows + kTcRows < n ? next * kTcRows + kTcRows : n;
        prefetch_rows<kSrc>(io, next * kTcRows, r1, gt);
      }
      // hidden layers l = 0..3: epilogue of D[l & 1], MMAs of layer l + 1
#pragma unroll 1
      for (int l = 0; l < 4; ++l) {
        if (!wait_layer()) {
          failed = true;
          break;
        }
        if constexpr (kSrc == kSrcX)
          if (l == 0 && next < n_tiles)  // X is free: stage the next input tile
            stage_rows_async(X, x + next * kTcRows * kIn, kTcRows, kIn, n - next * kTcRows, gt, kTcGroupThreads);
        const uint32_t d_in = tmem + (uint32_t)((l & 1) * kHid), d_out = tmem + (uint32_t)(((l + 1) & 1) * kHid);
        const int n_next = l == 3 ? kOut : kHid;
        const uint32_t w_next = l == 3 ? w5_addr : wh_addr + (uint32_t)(l * kHid * kHid * 2);
        const float *hb = bias + l * kHid;
        // TMEM loads run one chunk ahead of the arithmetic (two register sets)
        uint32_t ra[16], rb[16];
        tc_ld16(d_in + lane_off + (uint32_t)(half * 16), ra);
        tc_wait16(ra);
#pragma unroll
        for (int c32 = 0; c32 < kHid / 32; ++c32) {
          uint32_t(&cur)[16] = (c32 & 1) ? rb : ra;
          uint32_t(&nxt)[16] = (c32 & 1) ? ra : rb;
          if (c32 + 1 < kHid / 32) tc_ld16(d_in + lane_off + (uint32_t)((c32 + 1) * 32 + half * 16), nxt);
          epilogue16<kDrop>(cur, hb, A, row, c32 * 2 + half, dc, row0 + row, l);
          if (c32 & 1) {
            // these 64 columns are the next layer's K-steps 2 c32 - 2 .. 2 c32 + 1
            fence_proxy_async_smem();
            tc_fence_before();
            group_sync(g);
            if (leader) {
              tc_fence_after();
              for (int s = 2 * c32 - 2; s < 2 * c32 + 2; ++s)
                tc_mma(d_out, smem_desc(a_addr + 256 * s, 128, kHid * 16),
                       smem_desc(w_next + 256 * s, 128, kHid * 16), idesc_bf16(kTcRows, n_next), s > 0 ? 1u : 0u);
              if (c32 == kHid / 32 - 1) tc_commit(&bar[g]);
            }
          }
          if (c32 + 1 < kHid / 32) tc_wait16(nxt);
        }
      }
      // output layer: D[0] columns 0..15
      if (!failed && !wait_layer()) failed = true;
      if (!failed && half == 0) {
        uint32_t r16[16];
        tc_ld16(tmem + lane_off, r16);
        tc_wait16(r16);
        float v[16];
        const float *b5 = bias + 4 * kHid, *ymu = b5 + kOut, *ysg = ymu + kOut;
        const bool std_out = kSrc == kSrcX && standardized_out;
#pragma unroll
        for (int j = 0; j < kOut; ++j) {
          v[j] = __uint_as_float(r16[j]) + b5[j];
          if (!std_out) v[j] = fmaf(v[j], ysg[j], ymu[j]);
        }
        const int64_t c = row0 + row;
        if constexpr (kSrc == kSrcX) {
          if (c < n) {
            float2 *o = reinterpret_cast<float2 *>(out + c * kOut);
#pragma unroll
            for (int q = 0; q < kOut / 2; ++q) o[q] = make_float2(v[2 * q], v[2 * q + 1]);
          }
        } else if constexpr (kSrc == kSrcFull) {
          const bool pick = c < n && full_epilogue(io, v, st, st.fl | flp[(it & 1) * kTcRows + row], c);
          append_fallback(io, pick, c, lane);
        } else {
          if (c < n) lite_epilogue(io, v, st, st.fl | flp[(it & 1) * kTcRows + row], c);
        }
      }
    }
    if (failed) {
      // the group's MMAs stopped answering: this tile and the group's later
      // ones are marked (NaN outputs; for the closures non-finite, which the
      // full inputs' fallback recomputes exactly and LITE answers with the
      // linear drift)
      if (half == 0) {
        const int64_t c = row0 + row;
        if constexpr (kSrc == kSrcX) {
          if (c < n) {
            float2 *o = reinterpret_cast<float2 *>(out + c * kOut);
            const float nan = __int_as_float(0x7fc00000);
#pragma unroll
            for (int q = 0; q < kOut / 2; ++q) o[q] = make_float2(nan, nan);
          }
        } else if constexpr (kSrc == kSrcFull) {
          if (c < n) io.flags[c] = FP_FLAG_NONFINITE;
          append_fallback(io, c < n, c, lane);
        } else {
          if (c < n) {
            linear_drift(io.coeffs + c * 9, io.tau[c]);
            io.flags[c] = FP_FLAG_NONFINITE;
          }
        }
      }
    } else if (kSrc != kSrcX && next < n_tiles) {
      // the next tile's inputs: X is free since the first layer's MMAs of
      // this tile completed; part-1 flags go to the other parity slot
      if constexpr (kSrc == kSrcFull)
        form_full_inputs(io, scal, next * kTcRows + row, n, half, X, row, flp + ((it + 1) & 1) * kTcRows + row, st);
      else if constexpr (kSrc == kSrcLite)
        form_lite_inputs(io, scal, next * kTcRows + row, n, half, X, row, flp + ((it + 1) & 1) * kTcRows + row, st);
    }
  }
  // ---- teardown ----
  // Normally every MMA batch of this CTA has been waited for.  A group whose
  // wait ran out may still have the batch it gave up on in flight: its
  // leader waits for that commit once more, bounded, before the tensor memory
  // is released.  Should that wait run out too, the release below precedes
  // the MMA's completion, which leaves the tensor memory's state undefined;
  // the marked rows tell the caller to treat the context as suspect.
  if (failed && leader) (void)mbar_wait_bounded(&bar[g], phase ^ 1u, 200000000ull);
  cp_async_wait();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(*tmem_slot), "r"(kTmemCols)
                 : "memory");
}

static int g_tc_attr_done[4][64];

static int tc_sm_count() {
  static int n = 0;
  if (!n) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    if (n <= 0) n = 152;
  }
  return n;
}

template <bool kDrop, int kSrc>
static int launch_tc(const MlpDev &net, const __nv_bfloat16 *x, int64_t n, int standardized_out, float *out,
                     const DropoutCfg &dc, const FusedIO &io, cudaStream_t st) {
  constexpr int variant = kDrop ? 3 : kSrc;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !g_tc_attr_done[variant][dev]) {
    if (cudaFuncSetAttribute(mlp_forward_tc_kernel<kDrop, kSrc>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kTcSmem) != cudaSuccess)
      return -1;
    g_tc_attr_done[variant][dev] = 1;
  }
  const int64_t n_tiles = (n + kTcRows - 1) / kTcRows;
  int64_t grid = (n_tiles + kTcGroups - 1) / kTcGroups;
  if (grid > tc_sm_count()) grid = tc_sm_count();
  if (grid < 1) grid = 1;
  mlp_forward_tc_kernel<kDrop, kSrc><<<(unsigned)grid, kTcThreads, kTcSmem, st>>>(net, x, n, standardized_out, out,
                                                                                   dc, io);
  return 0;
}

// Returns -1 if the shared-memory limit could not be raised.
int launch_mlp_forward_tc(const MlpDev &net, const __nv_bfloat16 *x, int64_t n, int standardized_out, float *out,
                          cudaStream_t st) {
  return launch_tc<false, kSrcX>(net, x, n, standardized_out, out, DropoutCfg{}, FusedIO{}, st);
}

// The forward pass with the dropout masks of pass `dc.pass` (sensitivity probe).
int launch_mlp_forward_tc_dropout(const MlpDev &net, const __nv_bfloat16 *x, int64_t n, int standardized_out,
                                  float *out, const DropoutCfg &dc, cudaStream_t st) {
  return launch_tc<true, kSrcX>(net, x, n, standardized_out, out, dc, FusedIO{}, st);
}

// The learned closure in one kernel: io.src holds moment vectors (lite = 0;
// cells to recompute exactly are appended to io.list, io.count zeroed by the
// caller) or LITE vectors (lite = 1).  Returns -1 if the shared-memory limit
// could not be raised.
int launch_closure_surrogate_tc(const MlpDev &net, const FusedIO &io, int64_t n, int lite, cudaStream_t st) {
  if (lite) return launch_tc<false, kSrcLite>(net, nullptr, n, 0, nullptr, DropoutCfg{}, io, st);
  return launch_tc<false, kSrcFull>(net, nullptr, n, 0, nullptr, DropoutCfg{}, io, st);
}

}  // namespace fpc
