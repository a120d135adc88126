// tc_common.cuh -- fifth-generation tensor-core helpers (tcgen05, sm_103a)
// shared by the network's inference and training kernels: the no-swizzle
// K-major core-matrix operand layout, shared-memory and instruction
// descriptors of kind::f16 (BF16 x BF16 -> FP32), MMA issue and commit,
// tensor-memory loads, the bounded MMA wait and cp.async staging of
// row-major matrices into the operand layout.
#pragma once

#include <cstdint>
#include <cuda_bf16.h>

#include "tma.cuh"

namespace fpc {

// byte offset of the 16-byte chunk (row r, k-chunk c) of a K-major operand
// with K columns, in the no-swizzle core-matrix layout
__device__ __forceinline__ uint32_t cm_off(int r, int c, int K) {
  return (uint32_t)((r >> 3) * (K * 16) + c * 128 + (r & 7) * 16);
}

// shared-memory matrix descriptor (no swizzle): start address, leading byte
// offset (K direction), stride byte offset (M/N direction), descriptor
// version 1 at bit 46
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
  return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
         (1ull << 46);
}

// instruction descriptor of kind::f16: D = FP32 (bit 4), A = B = BF16
// (bits 7, 10), both K-major, N >> 3 at bit 17, M >> 4 at bit 24
__host__ __device__ constexpr uint32_t idesc_bf16(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) | ((uint32_t)(m >> 4) << 24);
}

__device__ __forceinline__ void tc_mma(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}" ::"r"(d_tmem),
      "l"(a), "l"(b), "r"(idesc), "r"(acc)
      : "memory");
}

__device__ __forceinline__ void tc_commit(uint64_t *bar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(smem_u32(bar))
               : "memory");
}

__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// 16 consecutive FP32 columns of this thread's TMEM lane.  The load is
// asynchronous: tc_wait16 completes it and names the registers as operands,
// so the compiler cannot read them before the wait.
__device__ __forceinline__ void tc_ld16(uint32_t taddr, uint32_t (&r)[16]) {
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
      "%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
        "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
}
__device__ __forceinline__ void tc_wait16(uint32_t (&r)[16]) {
  asm volatile("tcgen05.wait::ld.sync.aligned;"
               : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                 "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                 "+r"(r[15])
               :
               : "memory");
}

// Spin on the group's mbarrier (MMAs finish within microseconds, so no
// sleeping back-off at first); false after ~2 s.
__device__ __forceinline__ bool mma_wait(uint64_t *bar, uint32_t parity) {
#pragma unroll 1
  for (int i = 0; i < 4096; ++i)
    if (mbar_test_wait(bar, parity)) return true;
  return mbar_wait_bounded(bar, parity);
}

// Asynchronous copy of rows [0, N) of a row-major [N][K] BF16 matrix into the
// core-matrix layout (cp.async, 16 bytes per copy, all in flight at once);
// chunk i = (8-row group, K-chunk, row in group) lands at byte 16 i.  Rows
// at or beyond `valid` are zero-filled (source size 0).  Complete with
// cp_async_wait().
__device__ __forceinline__ void stage_rows_async(unsigned char *dst, const __nv_bfloat16 *__restrict__ src, int N,
                                                 int K, int64_t valid, int t0, int nt) {
  const int chunks = N * K / 8;
  for (int i = t0; i < chunks; i += nt) {
    const int rg = i / K, c = (i >> 3) % (K / 8), r = rg * 8 + (i & 7);
    const bool ok = r < valid;
    const __nv_bfloat16 *g = ok ? src + (int64_t)r * K + c * 8 : src;
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(dst + 16 * i)), "l"(g),
                 "r"(ok ? 16 : 0)
                 : "memory");
  }
  asm volatile("cp.async.commit_group;" ::: "memory");
}
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group 0;" ::: "memory"); }


}  // namespace fpc
