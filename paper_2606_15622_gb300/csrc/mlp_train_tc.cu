// mlp_train_tc.cu -- backward pass of the network for training, on the
// fifth-generation tensor cores of sm_103a (tcgen05, BF16 x BF16 -> FP32).
//
// One CTA per 128-row tile of the batch, four threads per row (= TMEM lane),
// each with a quarter of the row's columns.
// Going down the layers l = 5 .. 1 with dZ_5 = dout:
//   weight gradient  dW_l = dZ_l^T H_(l-1)   (M = out, N = in, K = the
//                    tile's 128 rows; layer 5 as dW_5^T = H_4^T dZ_5 so that
//                    M = 128; layer 1 with H_0 = X, N = 32)
//   data gradient    dA_(l-1) = dZ_l W_l    (M = 128 rows, N = in, K = out)
//   next dZ          dZ_(l-1) = dA_(l-1) silu'(Z_(l-1)), rounded to BF16
//   bias gradient    db_l = column sums of dZ_l (BF16 values, FP32 sums;
//                    db_5 from the FP32 dout)
// Every operand is K-major in the no-swizzle core-matrix layout (as the
// inference kernel's): W_l^T is staged transposed once per CTA, dZ_l is
// written by the epilogue both row-major (the A operand of the data
// gradient) and transposed (the A operand of the weight gradient), and
// H_(l-1) is staged transposed from the forward's saved activations.  The
// weight gradient and the data gradient of a layer are issued together into
// two 128-column TMEM accumulators and committed to one mbarrier.  Each tile
// writes its complete gradient (the flat parameter layout) to its own slot
// of the workspace, and a second kernel sums the slots in a fixed order, so
// the result does not depend on scheduling.
// The one thread that waits on the mbarrier does so with a bound; a wait
// that runs out fills the tile's slot with NaN (the caller sees non-finite
// gradients) and the CTA waits once more, bounded, for the batch it gave up
// on before releasing its tensor memory.
#include <cstdint>
#include <cuda_bf16.h>

#include "fp_device.cuh"
#include "mlp_common.cuh"
#include "tc_common.cuh"
#include "train_math.cuh"

namespace fpc {

int64_t mlp_param_offset(int which, int layer);
int64_t mlp_param_count();

namespace {

constexpr int kBR = 128;               // rows per tile = TMEM lanes
constexpr int kPart = 4;               // threads per row, each with a quarter of the row's columns
constexpr int kBT = kPart * kBR;
constexpr int kZB = kHid / 4 / kPart;  // a thread's 4-column blocks of Z
constexpr int kHB = kHid / 8 / kPart;  // a thread's 8-column blocks of H
constexpr int kXB = kIn / 8 / kPart;   // a thread's 8-column blocks of X
static_assert(kZB % 4 == 0 && kXB >= 1, "a thread's columns are whole 16-column chunks");
constexpr uint32_t kBTmemCols = 256;   // data gradient [0, 128), weight gradient [128, 256)

// shared-memory carve-up (bytes from a 1024-byte aligned base)
constexpr uint32_t kBOffWT = 0;                                // W2^T, W3^T, W4^T: 3 x [128 in][128 out]
constexpr uint32_t kBOffWT5 = kBOffWT + 3 * kHid * kHid * 2;   // W5^T: [128 in][16 out]
constexpr uint32_t kBOffDZ = kBOffWT5 + kHid * kOut * 2;       // dZ: [128 rows][K = out]
constexpr uint32_t kBOffDZT = kBOffDZ + kBR * kHid * 2;        // dZ^T: [out][K = 128 rows]
constexpr uint32_t kBOffHT = kBOffDZT + kHid * kBR * 2;        // H^T: [in][K = 128 rows]
constexpr uint32_t kBOffBar = kBOffHT + kHid * kBR * 2;         // one mbarrier
constexpr uint32_t kBOffSlot = kBOffBar + 8;                   // TMEM address, outcome
constexpr uint32_t kBOffRed = kBOffSlot + 16;                  // db_5 partial sums: [16 row groups][16]
constexpr uint32_t kBSmemUsed = kBOffRed + kBT * 4;
constexpr size_t kBSmem = kBSmemUsed + 1024;
static_assert(kBSmem <= 227 * 1024, "shared memory");

// element (row r, column k) of a K-major operand with K columns
__device__ __forceinline__ uint32_t cm_elem(int r, int k, int K) { return cm_off(r, k >> 3, K) + (uint32_t)(k & 7) * 2; }

// the flat parameter layout W1 | b1 | W2 | b2 | ... | W5 | b5 (as mlp_param_offset)
__host__ __device__ constexpr int64_t poff(int which, int layer) {
  int64_t off = 0;
  for (int l = 0; l < layer; ++l)
    off += (l == 0 ? kHid * kIn : (l == 4 ? kOut * kHid : kHid * kHid)) + (l == 4 ? kOut : kHid);
  return which == 0 ? off : off + (layer == 0 ? kHid * kIn : (layer == 4 ? kOut * kHid : kHid * kHid));
}

// w rotated left by r (0 .. N - 1) places, with selects (no local memory)
template <int N>
__device__ __forceinline__ void rotate_words(uint32_t (&w)[N], int r) {
#pragma unroll
  for (int b = 1; b < N; b <<= 1) {
    uint32_t u[N];
#pragma unroll
    for (int k = 0; k < N; ++k) u[k] = (r & b) ? w[(k + b) % N] : w[k];
#pragma unroll
    for (int k = 0; k < N; ++k) w[k] = u[k];
  }
}

// row t's values at columns i0 .. i0 + 7 (packed BF16 pairs, i0 a multiple
// of 8) stored transposed: element (i0 + j, t) of a K-major operand with
// K = 128 rows.  Elements (i, t) and (i, t ^ 1) share a 32-bit word, so lanes
// t and t ^ 1 swap their values and each writes four whole words (the even
// lane the even columns); the start is rotated by the lane's 8-row group so
// that the 32 stores of one instruction fall in 32 different banks.  Called
// by all lanes of a warp, with t = the row = a multiple of 32 plus the lane.
__device__ __forceinline__ void st_col8(unsigned char *base, int i0, int t, uint4 q) {
  const uint32_t mine[4] = {q.x, q.y, q.z, q.w};
  const bool odd = t & 1;
  uint32_t w[4];
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const uint32_t nb = __shfl_xor_sync(0xffffffffu, mine[k], 1);
    // word of column i0 + 2k + odd: low half row t & ~1, high half row t | 1
    w[k] = odd ? __byte_perm(nb, mine[k], 0x7632) : __byte_perm(mine[k], nb, 0x5410);
  }
  const int g = (t >> 3) & 3;
  rotate_words(w, g);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    const int i = i0 + 2 * ((k + g) & 3) + (odd ? 1 : 0);
    *reinterpret_cast<uint32_t *>(base + cm_elem(i, t & ~1, kBR)) = w[k];
  }
}

// values 8 v0 .. 8 (v0 + NV) - 1 of a BF16 row, loaded with 16-byte loads
// (all issued first) and stored transposed (zeros past the batch)
template <int NV>
__device__ __forceinline__ void stage_row_t(unsigned char *base, const __nv_bfloat16 *row, bool live, int t, int v0) {
  uint4 q[NV];
#pragma unroll
  for (int v = 0; v < NV; ++v)
    q[v] = live ? reinterpret_cast<const uint4 *>(row)[v0 + v] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
  for (int v = 0; v < NV; ++v) st_col8(base, 8 * (v0 + v), t, q[v]);
}

// 16 accumulator columns of this thread's lane, as floats
__device__ __forceinline__ void ld_cols16(uint32_t taddr, float (&v)[16]) {
  uint32_t r[16];
  tc_ld16(taddr, r);
  tc_wait16(r);
#pragma unroll
  for (int j = 0; j < 16; ++j) v[j] = __uint_as_float(r[j]);
}

}  // namespace

__global__ void __launch_bounds__(kBT, 1)
    mlp_backward_tc_kernel(MlpDev net, const __nv_bfloat16 *__restrict__ x, const __nv_bfloat16 *__restrict__ h_save,
                           const float *__restrict__ z_save, const __nv_bfloat16 *__restrict__ dout_bf,
                           const float *__restrict__ dout, int64_t n, int64_t n_params, float *__restrict__ parts) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kBOffBar);
  volatile uint32_t *slot = reinterpret_cast<volatile uint32_t *>(sm + kBOffSlot);
  unsigned char *DZ = sm + kBOffDZ, *DZT = sm + kBOffDZT, *HT = sm + kBOffHT;
  const int tid = threadIdx.x, t = tid & (kBR - 1), qd = tid >> 7, warp = tid >> 5;  // row t, part qd
  const int64_t row0 = (int64_t)blockIdx.x * kBR, r = row0 + t;
  const bool live = r < n;
  float *part = parts + (int64_t)blockIdx.x * n_params;

  // W_l^T (l = 2..4) and W_5^T, transposed into the B layout once.  Element
  // (i, o) and (i, o + 1) share a 32-bit word: a thread takes inputs
  // 8 ib .. 8 ib + 7 of an output pair and writes eight words, starting at an
  // input rotated by its block, so that a warp's 32 stores (four output pairs
  // by eight input blocks) fall in 32 different banks
#pragma unroll
  for (int l = 0; l < 3; ++l) {
    const uint4 *W = reinterpret_cast<const uint4 *>(net.W[1 + l]);  // [out][in], 8 inputs a vector
    unsigned char *WT = sm + kBOffWT + (uint32_t)l * kHid * kHid * 2;
#pragma unroll 1
    for (int e = tid; e < (kHid / 2) * (kHid / 8); e += kBT) {
      const int lane = e & 31, grp = e >> 5, jb = lane >> 2;
      const int o = 2 * (4 * (grp % 16) + (lane & 3)), ib = 8 * (grp / 16) + jb;
      const uint4 qa = W[o * (kHid / 8) + ib], qb = W[(o + 1) * (kHid / 8) + ib];
      const uint32_t a4[4] = {qa.x, qa.y, qa.z, qa.w}, b4[4] = {qb.x, qb.y, qb.z, qb.w};
      uint32_t w[8];
#pragma unroll
      for (int k = 0; k < 4; ++k) {
        w[2 * k] = __byte_perm(a4[k], b4[k], 0x5410);
        w[2 * k + 1] = __byte_perm(a4[k], b4[k], 0x7632);
      }
      rotate_words(w, jb);
#pragma unroll
      for (int k = 0; k < 8; ++k)
        *reinterpret_cast<uint32_t *>(WT + cm_elem(8 * ib + ((k + jb) & 7), o, kHid)) = w[k];
    }
  }
  for (int e = tid; e < kOut * kHid; e += kBT) {
    const int o = e / kHid, i = e % kHid;
    *reinterpret_cast<__nv_bfloat16 *>(sm + kBOffWT5 + cm_elem(i, o, kOut)) = net.W[4][e];
  }
  // layer 5 operands: dout (A of dA_4, K = 16), dout^T (B of dW_5^T), H_4^T
  // (A of dW_5^T); rows past the batch are zero
  stage_rows_async(DZ, dout_bf + row0 * kOut, kBR, kOut, n - row0, tid, kBT);
  if (qd == 0) stage_row_t<kOut / 8>(DZT, dout_bf + r * kOut, live, t, 0);
  {
    const uint4 *h4 = reinterpret_cast<const uint4 *>(h_save) + ((size_t)3 * (kHid / 8) + qd * kHB) * n + r;
    uint4 q[kHB];
#pragma unroll
    for (int v = 0; v < kHB; ++v) q[v] = live ? h4[(size_t)v * n] : make_uint4(0u, 0u, 0u, 0u);
#pragma unroll
    for (int v = 0; v < kHB; ++v) st_col8(HT, 8 * (qd * kHB + v), t, q[v]);
  }
  // db_5, first half: column tid % 16 of the FP32 dout summed over rows
  // tid / 16 + G k, G = kBT / 16 row groups (coalesced loads, all issued at once)
  {
    constexpr int G = kBT / kOut;
    static_assert(kBR % G == 0, "db_5 row groups");
    float d[kBR / G];
#pragma unroll
    for (int k = 0; k < kBR / G; ++k) {
      const int64_t q = (tid >> 4) + G * k;
      d[k] = row0 + q < n ? dout[(row0 + q) * kOut + (tid & 15)] : 0.f;
    }
    float s = 0.f;
#pragma unroll
    for (int k = 0; k < kBR / G; ++k) s += d[k];
    reinterpret_cast<float *>(sm + kBOffRed)[tid] = s;
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void *)slot)),
                 "r"(kBTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  cp_async_wait();
  fence_proxy_async_smem();  // operands written through the generic proxy, read by the MMA
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = slot[0];
  const uint32_t d_a = tmem, d_w = tmem + (uint32_t)kHid;
  const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;  // warps w, w + 4, w + 8, w + 12 share lanes
  const uint32_t dz_addr = smem_u32(DZ), dzt_addr = smem_u32(DZT), ht_addr = smem_u32(HT);
  uint32_t phase = 0;
  bool failed = false;

  // the leader waits for the layer's commit; everybody learns the outcome
  auto wait_layer = [&]() -> bool {
    if (tid == 0) slot[1] = mma_wait(bar, phase) ? 1u : 0u;
    phase ^= 1u;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return slot[1] != 0u;
  };
  // after the operands of the next MMAs were written by this CTA's threads
  auto operands_ready = [&]() {
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
  };

  // ---- layer 5: dW_5^T = H_4^T dout (N = 16), dA_4 = dout W_5 (K = 16) ----
  if (tid == 0) {
    for (int s = 0; s < kBR / 16; ++s)
      tc_mma(d_w, smem_desc(ht_addr + 256 * s, 128, kBR * 16), smem_desc(dzt_addr + 256 * s, 128, kBR * 16),
             idesc_bf16(kBR, kOut), s > 0 ? 1u : 0u);
    tc_mma(d_a, smem_desc(dz_addr, 128, kOut * 16), smem_desc(smem_u32(sm + kBOffWT5), 128, kOut * 16),
           idesc_bf16(kBR, kHid), 0u);
    tc_commit(bar);
  }
  // layers l = 5 .. 1: epilogue of layer l's MMAs, then the MMAs of layer l - 1
#pragma unroll 1
  for (int l = 5; l >= 1; --l) {
    // this thread's part of row t of Z_(l-1) and of H_(l-2) (X for layer 1),
    // loaded while the layer's MMAs run
    float4 zr[kZB];
    uint4 hr[kHB];
    if (l >= 2) {
      const float4 *z4 = reinterpret_cast<const float4 *>(z_save) + ((size_t)(l - 2) * (kHid / 4) + qd * kZB) * n + r;
#pragma unroll
      for (int q = 0; q < kZB; ++q) zr[q] = live ? z4[(size_t)q * n] : make_float4(0.f, 0.f, 0.f, 0.f);
      // X rows are row-major, the saved H column-block-major
      const uint4 *h4 = l - 1 == 1 ? reinterpret_cast<const uint4 *>(x + r * kIn) + qd * kXB
                                   : reinterpret_cast<const uint4 *>(h_save) + ((size_t)(l - 3) * (kHid / 8) + qd * kHB) * n + r;
      const int nh = l - 1 == 1 ? kXB : kHB;
      const size_t hstride = l - 1 == 1 ? 1 : (size_t)n;
#pragma unroll
      for (int v = 0; v < kHB; ++v) hr[v] = live && v < nh ? h4[v * hstride] : make_uint4(0u, 0u, 0u, 0u);
    }
    if (!wait_layer()) {
      failed = true;
      break;
    }
    // weight gradient of layer l: lane t holds row t of dW_l (out t), or for
    // layer 5 row t of dW_5^T (in t)
    if (l == 5) {
      // db_5, second half: the 16 row groups in order
      if (tid < kOut) {
        const float *red = reinterpret_cast<const float *>(sm + kBOffRed);
        float s = 0.f;
#pragma unroll
        for (int g = 0; g < kBT / kOut; ++g) s += red[g * kOut + tid];
        part[poff(1, 4) + tid] = s;
      }
      if (qd == 0) {
      float v[16];
      ld_cols16(d_w + lane_off, v);
      float *g = part + poff(0, 4);  // W5 [16][128]
#pragma unroll
      for (int o = 0; o < kOut; ++o) g[o * kHid + t] = v[o];
      }
    } else {
      // kept in blocks of four inputs ([in / 4][out][4], coalesced; the
      // tile sum restores the flat layout)
      const int in = l == 1 ? kIn : kHid;
      float4 *g = reinterpret_cast<float4 *>(part + poff(0, l - 1)) + t;
      const int nch = in / 16;  // 16-column chunks, split over the row's threads
      for (int c = qd * nch / kPart; c < (qd + 1) * nch / kPart; ++c) {
        float v[16];
        ld_cols16(d_w + lane_off + (uint32_t)(16 * c), v);
#pragma unroll
        for (int q = 0; q < 4; ++q)
          g[(4 * c + q) * kHid] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
      }
    }
    if (l == 1) break;
    // dZ_(l-1) = dA_(l-1) silu'(Z_(l-1)) -> DZ (row t) and DZT (column t)
    {
      const int c0 = qd * (kZB / 4);  // this thread's 16-column chunks
#pragma unroll
      for (int cc = 0; cc < kZB / 4; ++cc) {
        const int c = c0 + cc;
        float v[16];
        ld_cols16(d_a + lane_off + (uint32_t)(16 * c), v);
        const float zz[16] = {zr[4 * cc].x,     zr[4 * cc].y,     zr[4 * cc].z,     zr[4 * cc].w,
                              zr[4 * cc + 1].x, zr[4 * cc + 1].y, zr[4 * cc + 1].z, zr[4 * cc + 1].w,
                              zr[4 * cc + 2].x, zr[4 * cc + 2].y, zr[4 * cc + 2].z, zr[4 * cc + 2].w,
                              zr[4 * cc + 3].x, zr[4 * cc + 3].y, zr[4 * cc + 3].z, zr[4 * cc + 3].w};
        uint32_t pk[8];
#pragma unroll
        for (int j = 0; j < 16; j += 2) {
          const float g0 = live ? v[j] * silu_grad(zz[j]) : 0.f, g1 = live ? v[j + 1] * silu_grad(zz[j + 1]) : 0.f;
          pk[j / 2] = pack_bf16(g0, g1);
        }
        const uint4 lo = make_uint4(pk[0], pk[1], pk[2], pk[3]), hi = make_uint4(pk[4], pk[5], pk[6], pk[7]);
        *reinterpret_cast<uint4 *>(DZ + cm_off(t, 2 * c, kHid)) = lo;
        *reinterpret_cast<uint4 *>(DZ + cm_off(t, 2 * c + 1, kHid)) = hi;
        st_col8(DZT, 16 * c, t, lo);
        st_col8(DZT, 16 * c + 8, t, hi);
      }
    }
    // H_(l-2)^T for the weight gradient of layer l - 1 (X^T for layer 1)
    if (l - 1 == 1) {
#pragma unroll
      for (int v = 0; v < kXB; ++v) st_col8(HT, 8 * (qd * kXB + v), t, hr[v]);
    } else {
#pragma unroll
      for (int v = 0; v < kHB; ++v) st_col8(HT, 8 * (qd * kHB + v), t, hr[v]);
    }
    operands_ready();
    // MMAs of layer l - 1: dW_(l-1) = dZ^T H^T^T, dA_(l-2) = dZ W_(l-1)
    if (tid == 0) {
      const int nw = l - 1 == 1 ? kIn : kHid;
      for (int s = 0; s < kBR / 16; ++s)
        tc_mma(d_w, smem_desc(dzt_addr + 256 * s, 128, kBR * 16), smem_desc(ht_addr + 256 * s, 128, kBR * 16),
               idesc_bf16(kBR, nw), s > 0 ? 1u : 0u);
      if (l - 1 >= 2) {
        const uint32_t wt = smem_u32(sm + kBOffWT + (uint32_t)(l - 3) * kHid * kHid * 2);  // W_(l-1)^T
        for (int s = 0; s < kHid / 16; ++s)
          tc_mma(d_a, smem_desc(dz_addr + 256 * s, 128, kHid * 16), smem_desc(wt + 256 * s, 128, kHid * 16),
                 idesc_bf16(kBR, kHid), s > 0 ? 1u : 0u);
      }
      tc_commit(bar);
    }
    // db_(l-1): column t of dZ_(l-1) summed over the tile's rows (row t of DZT)
    if (qd == 0) {
      float s = 0.f;
#pragma unroll
      for (int k8 = 0; k8 < kBR / 8; ++k8) {
        const uint4 q = *reinterpret_cast<const uint4 *>(DZT + cm_off(t, k8, kBR));
        const uint32_t w4[4] = {q.x, q.y, q.z, q.w};
#pragma unroll
        for (int e = 0; e < 4; ++e)
          s += __uint_as_float(w4[e] << 16) + __uint_as_float(w4[e] & 0xffff0000u);
      }
      part[poff(1, l - 2) + t] = s;
    }
  }
  if (failed) {
    // the tile's gradient is unusable: NaN in its whole slot
    for (int64_t i = tid; i < n_params; i += kBT) part[i] = __int_as_float(0x7fc00000);
    if (tid == 0) (void)mbar_wait_bounded(bar, phase ^ 1u, 200000000ull);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(slot[0]), "r"(kBTmemCols) : "memory");
}

// ---------------------------------------------------------------------------
// training forward: the network on a 128-row tile per CTA, four threads per
// row (a quarter of its columns each; the warps w, w + 4, w + 8, w + 12 share
// TMEM lanes), saving every hidden layer's pre-activations Z (FP32) and activations
// H = SiLU(Z) (BF16, the exponential form the backward pass differentiates)
// ---------------------------------------------------------------------------
namespace {
constexpr uint32_t kFOffW1 = 0;                               // W1 [128 out][K = 32 in]
constexpr uint32_t kFOffWH = kFOffW1 + kHid * kIn * 2;        // W2..W4 [128][K = 128]
constexpr uint32_t kFOffW5 = kFOffWH + 3 * kHid * kHid * 2;   // W5 [16][K = 128]
constexpr uint32_t kFOffA = kFOffW5 + kOut * kHid * 2;        // activations [128 rows][K = 128]
constexpr uint32_t kFOffX = kFOffA + kBR * kHid * 2;          // inputs [128 rows][K = 32]
constexpr uint32_t kFOffBias = kFOffX + kBR * kIn * 2;        // b1..b4 (4 x 128), b5, y_mu, y_sigma (3 x 16)
constexpr uint32_t kFOffLT = kFOffBias + (4 * kHid + 3 * kOut) * 4;  // loss: the tile's targets [128][9]
constexpr int kLA = 17;                                               // loss: padded aux row stride (floats)
constexpr uint32_t kFOffLA = kFOffLT + kBR * kNOut * 4;              // loss: the tile's aux rows [128][17]
constexpr uint32_t kFOffBar = kFOffLA + kBR * kLA * 4;
constexpr uint32_t kFOffSlot = kFOffBar + 8;
constexpr uint32_t kFSmemUsed = kFOffSlot + 16;
constexpr size_t kFSmem = kFSmemUsed + 1024;
constexpr uint32_t kFTmemCols = 128;
constexpr int kFT = 4 * kBR;  // threads: four per row, each with a quarter of the row's columns
static_assert(kFSmem <= 227 * 1024, "shared memory");
static_assert(kFOffBar % 8 == 0, "mbarrier alignment");
}  // namespace

__global__ void __launch_bounds__(kFT, 1)
    mlp_forward_train_tc_kernel(MlpDev net, const __nv_bfloat16 *__restrict__ x, int64_t n, int standardized_out,
                                float *__restrict__ out, __nv_bfloat16 *__restrict__ h_save,
                                float *__restrict__ z_save, const float *__restrict__ t_true,
                                const float *__restrict__ aux, LossParams prm, float *__restrict__ dout,
                                __nv_bfloat16 *__restrict__ dout_bf, float *__restrict__ loss_sum) {
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  unsigned char *sm = reinterpret_cast<unsigned char *>(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
  uint64_t *bar = reinterpret_cast<uint64_t *>(sm + kFOffBar);
  volatile uint32_t *slot = reinterpret_cast<volatile uint32_t *>(sm + kFOffSlot);
  float *bias = reinterpret_cast<float *>(sm + kFOffBias);
  unsigned char *A = sm + kFOffA, *X = sm + kFOffX;
  float *sLT = reinterpret_cast<float *>(sm + kFOffLT), *sLA = reinterpret_cast<float *>(sm + kFOffLA);
  const int tid = threadIdx.x, t = tid & (kBR - 1), qd = tid >> 7, warp = tid >> 5;
  const int64_t row0 = (int64_t)blockIdx.x * kBR, r = row0 + t;
  const bool live = r < n;
  const bool with_loss = t_true != nullptr;  // the loss of the standardised outputs, fused
  if (with_loss) {  // the tile's targets and aux rows, coalesced
    const int nr = (int)(n - row0 < kBR ? n - row0 : kBR);
    for (int i = tid; i < nr * kNOut; i += kFT) sLT[i] = t_true[row0 * kNOut + i];
    for (int i = tid; i < nr * 16; i += kFT) sLA[(i >> 4) * kLA + (i & 15)] = aux[row0 * 16 + i];
  }

  stage_rows_async(sm + kFOffW1, net.W[0], kHid, kIn, kHid, tid, kFT);
  for (int l = 0; l < 3; ++l)
    stage_rows_async(sm + kFOffWH + (uint32_t)l * kHid * kHid * 2, net.W[1 + l], kHid, kHid, kHid, tid, kFT);
  stage_rows_async(sm + kFOffW5, net.W[4], kOut, kHid, kOut, tid, kFT);
  stage_rows_async(X, x + row0 * kIn, kBR, kIn, n - row0, tid, kFT);
  if (tid < kHid) {
#pragma unroll
    for (int l = 0; l < 4; ++l) bias[l * kHid + tid] = net.b[l][tid];
  } else if (tid < kHid + kOut) {
    const int j = tid - kHid;
    bias[4 * kHid + j] = net.b[4][j];
    bias[4 * kHid + kOut + j] = net.y_mu[j];
    bias[4 * kHid + 2 * kOut + j] = net.y_sigma[j];
  }
  if (tid == 0) {
    mbar_init(bar, 1);
    fence_barrier_init();
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32((const void *)slot)),
                 "r"(kFTmemCols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
  }
  cp_async_wait();
  fence_proxy_async_smem();
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  const uint32_t tmem = slot[0];
  const uint32_t lane_off = (uint32_t)((warp & 3) * 32) << 16;  // warps w, w + 4, w + 8, w + 12 share lanes
  const uint32_t a_addr = smem_u32(A), x_addr = smem_u32(X);
  uint32_t phase = 0;
  bool failed = false;
  auto wait_layer = [&]() -> bool {
    if (tid == 0) slot[1] = mma_wait(bar, phase) ? 1u : 0u;
    phase ^= 1u;
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    return slot[1] != 0u;
  };

  // layer 1
  if (tid == 0) {
    for (int s = 0; s < kIn / 16; ++s)
      tc_mma(tmem, smem_desc(x_addr + 256 * s, 128, kIn * 16), smem_desc(smem_u32(sm + kFOffW1) + 256 * s, 128, kIn * 16),
             idesc_bf16(kBR, kHid), s > 0 ? 1u : 0u);
    tc_commit(bar);
  }
#pragma unroll 1
  for (int l = 0; l < 4; ++l) {
    if (!wait_layer()) {
      failed = true;
      break;
    }
    // z = acc + b, H = SiLU(z): saved, and the next layer's A operand
    const float *bl = bias + l * kHid;
    // saved column-block-major (Z in blocks of four columns, H of eight), so
    // that the 32 rows of a warp write 512 contiguous bytes
    float4 *zs = reinterpret_cast<float4 *>(z_save) + (size_t)l * (kHid / 4) * n + r;
    uint4 *hs = reinterpret_cast<uint4 *>(h_save) + (size_t)l * (kHid / 8) * n + r;
#pragma unroll 1
    for (int c = qd * (kHid / 64); c < (qd + 1) * (kHid / 64); ++c) {  // this thread's quarter of the columns
      float v[16];
      ld_cols16(tmem + lane_off + (uint32_t)(16 * c), v);
      uint32_t pk[8];
#pragma unroll
      for (int j = 0; j < 16; ++j) v[j] += bl[16 * c + j];
#pragma unroll
      for (int j = 0; j < 16; j += 2) pk[j / 2] = pack_bf16(silu(v[j]), silu(v[j + 1]));
      const uint4 lo = make_uint4(pk[0], pk[1], pk[2], pk[3]), hi = make_uint4(pk[4], pk[5], pk[6], pk[7]);
      *reinterpret_cast<uint4 *>(A + cm_off(t, 2 * c, kHid)) = lo;
      *reinterpret_cast<uint4 *>(A + cm_off(t, 2 * c + 1, kHid)) = hi;
      if (live) {
#pragma unroll
        for (int q = 0; q < 4; ++q)
          zs[(size_t)(4 * c + q) * n] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
        hs[(size_t)(2 * c) * n] = lo;
        hs[(size_t)(2 * c + 1) * n] = hi;
      }
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    if (tid == 0) {
      const int n_next = l == 3 ? kOut : kHid;
      const uint32_t w = l == 3 ? smem_u32(sm + kFOffW5) : smem_u32(sm + kFOffWH + (uint32_t)l * kHid * kHid * 2);
      for (int s = 0; s < kHid / 16; ++s)
        tc_mma(tmem, smem_desc(a_addr + 256 * s, 128, kHid * 16), smem_desc(w + 256 * s, 128, kHid * 16),
               idesc_bf16(kBR, n_next), s > 0 ? 1u : 0u);
      tc_commit(bar);
    }
  }
  if (!failed && !wait_layer()) failed = true;
  if (!failed && qd == 0) {
    float v[16];
    ld_cols16(tmem + lane_off, v);
    const float *b5 = bias + 4 * kHid, *ymu = b5 + kOut, *ysg = ymu + kOut;
#pragma unroll
    for (int j = 0; j < kOut; ++j) {
      v[j] += b5[j];
      if (!standardized_out) v[j] = fmaf(ysg[j], v[j], ymu[j]);
    }
    if (live && out) {
      float4 *o4 = reinterpret_cast<float4 *>(out + r * kOut);
#pragma unroll
      for (int q = 0; q < 4; ++q) o4[q] = make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
    }
    if (with_loss) {
      // the row's loss and scale * dL/dout (FP32 and BF16), the loss summed
      // over the warp and added to loss_sum
      float lrow = 0.f;
      if (live) {
        float gr[kNOut];
        lrow = loss_row(v, sLT + t * kNOut, sLA + t * kLA, ymu, ysg, prm, gr);
        float gs[kOut];
#pragma unroll
        for (int a = 0; a < kOut; ++a) gs[a] = a < kNOut ? gr[a] * prm.scale : 0.f;
        float4 *d4 = reinterpret_cast<float4 *>(dout + r * kOut);
#pragma unroll
        for (int q = 0; q < 4; ++q) d4[q] = make_float4(gs[4 * q], gs[4 * q + 1], gs[4 * q + 2], gs[4 * q + 3]);
        uint4 *b4 = reinterpret_cast<uint4 *>(dout_bf + r * kOut);
        b4[0] = make_uint4(pack_bf16(gs[0], gs[1]), pack_bf16(gs[2], gs[3]), pack_bf16(gs[4], gs[5]),
                           pack_bf16(gs[6], gs[7]));
        b4[1] = make_uint4(pack_bf16(gs[8], gs[9]), pack_bf16(gs[10], gs[11]), pack_bf16(gs[12], gs[13]),
                           pack_bf16(gs[14], gs[15]));
      }
#pragma unroll
      for (int o2 = 16; o2 >= 1; o2 >>= 1) lrow += __shfl_xor_sync(0xffffffffu, lrow, o2);
      if ((tid & 31) == 0) atomicAdd(loss_sum, lrow);
    }
  } else if (failed) {
    if (live && qd == 0) {
      for (int j = 0; j < kOut; ++j) {
        if (out) out[r * kOut + j] = __int_as_float(0x7fc00000);
        if (with_loss) {
          dout[r * kOut + j] = __int_as_float(0x7fc00000);
          dout_bf[r * kOut + j] = __float2bfloat16_rn(__int_as_float(0x7fc00000));
        }
      }
    }
    if (with_loss && tid == 0) atomicAdd(loss_sum, __int_as_float(0x7fc00000));
    if (tid == 0) (void)mbar_wait_bounded(bar, phase ^ 1u, 200000000ull);
  }
  tc_fence_before();
  __syncthreads();
  tc_fence_after();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(slot[0]), "r"(kFTmemCols) : "memory");
}

// Returns -1 if the shared-memory limit could not be raised.
// With t_true non-null the loss (lp, over the standardised outputs) is fused
// into the last layer: dout, dout_bf and loss_sum are written, out may be null.
int launch_mlp_forward_loss_tc(const MlpDev &net, const void *x, int64_t n, int standardized_out, float *out,
                               void *h_save, float *z_save, const float *t_true, const float *aux,
                               const LossParams *lp, float *dout, void *dout_bf, float *loss_sum, cudaStream_t st) {
  static int attr_done[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    if (cudaFuncSetAttribute(mlp_forward_train_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)kFSmem) != cudaSuccess)
      return -1;
    attr_done[dev] = 1;
  }
  const int64_t tiles = (n + kBR - 1) / kBR;
  LossParams prm{};
  if (lp) prm = *lp;
  mlp_forward_train_tc_kernel<<<(unsigned)tiles, kFT, kFSmem, st>>>(
      net, reinterpret_cast<const __nv_bfloat16 *>(x), n, standardized_out, out,
      reinterpret_cast<__nv_bfloat16 *>(h_save), z_save, t_true, aux, prm, dout,
      reinterpret_cast<__nv_bfloat16 *>(dout_bf), loss_sum);
  return 0;
}

int launch_mlp_forward_train_tc(const MlpDev &net, const void *x, int64_t n, int standardized_out, float *out,
                                void *h_save, float *z_save, cudaStream_t st) {
  return launch_mlp_forward_loss_tc(net, x, n, standardized_out, out, h_save, z_save, nullptr, nullptr, nullptr,
                                    nullptr, nullptr, nullptr, st);
}

// The gradient summed over the tiles' slots into out (the flat layout); with
// adam.p non-null the Adam step of that parameter follows.
__global__ void sum_tiles_kernel(const float *__restrict__ parts, int ntiles, int64_t cnt, float *__restrict__ out,
                                 AdamParams adam) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= cnt) return;
  // tile order (the result does not depend on scheduling), loads eight at a time
  float s = 0.f;
  int z = 0;
  for (; z + 8 <= ntiles; z += 8) {
    float v[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) v[k] = parts[(int64_t)(z + k) * cnt + i];
#pragma unroll
    for (int k = 0; k < 8; ++k) s += v[k];
  }
  for (; z < ntiles; ++z) s += parts[(int64_t)z * cnt + i];
  // the hidden layers' weight gradients are kept in blocks of four inputs
  // ([in / 4][out][4]); everything else is in the flat layout
  int64_t dst = i;
#pragma unroll
  for (int l = 0; l < 4; ++l) {
    const int64_t off = poff(0, l), in = l == 0 ? kIn : kHid;
    if (i >= off && i < off + kHid * in) {
      const int64_t loc = i - off;
      dst = off + ((loc >> 2) % kHid) * in + 4 * (loc / (4 * kHid)) + (loc & 3);
    }
  }
  out[dst] = s;
  if (adam.p) adam_update(adam, dst, s);
}

size_t mlp_backward_tc_ws(int64_t n) {
  const int64_t tiles = (n + kBR - 1) / kBR;
  return (size_t)tiles * (size_t)mlp_param_count() * sizeof(float);
}

// Returns -1 if the shared-memory limit could not be raised.
// With adam non-null, the Adam step of every parameter follows its gradient
// in the tile sum.
int launch_mlp_backward_adam_tc(const MlpDev &net, const void *x, const void *h_save, const float *z_save,
                                const void *dout_bf, const float *dout, int64_t n, float *grads, void *ws,
                                const AdamParams *adam, cudaStream_t st) {
  static int attr_done[64];
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev >= 0 && dev < 64 && !attr_done[dev]) {
    if (cudaFuncSetAttribute(mlp_backward_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kBSmem) !=
        cudaSuccess)
      return -1;
    attr_done[dev] = 1;
  }
  const int64_t tiles = (n + kBR - 1) / kBR;
  const int64_t np = mlp_param_count();
  float *parts = reinterpret_cast<float *>(ws);
  mlp_backward_tc_kernel<<<(unsigned)tiles, kBT, kBSmem, st>>>(
      net, reinterpret_cast<const __nv_bfloat16 *>(x), reinterpret_cast<const __nv_bfloat16 *>(h_save), z_save,
      reinterpret_cast<const __nv_bfloat16 *>(dout_bf), dout, n, np, parts);
  AdamParams a{};
  if (adam) a = *adam;
  sum_tiles_kernel<<<(unsigned)((np + 255) / 256), 256, 0, st>>>(parts, (int)tiles, np, grads, a);
  return 0;
}

int launch_mlp_backward_tc(const MlpDev &net, const void *x, const void *h_save, const float *z_save,
                           const void *dout_bf, const float *dout, int64_t n, float *grads, void *ws,
                           cudaStream_t st) {
  return launch_mlp_backward_adam_tc(net, x, h_save, z_save, dout_bf, dout, n, grads, ws, nullptr, st);
}

}  // namespace fpc
