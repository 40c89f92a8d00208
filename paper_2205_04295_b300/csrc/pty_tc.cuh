// 5th-generation tensor cores on sm_103a (tcgen05), written as inline PTX:
// tensor-memory (TMEM) allocation, shared-memory matrix descriptors, the
// single-thread MMA issue, its completion on an mbarrier and the TMEM ->
// register loads of the accumulator.
//
// Operand layout used here: K-major, no swizzle.  The unit is the "core
// matrix" of 8 rows x 16 bytes (4 TF32 values along K), stored as 128
// contiguous bytes, row r at byte 16 r.  A descriptor names the first core
// matrix of the operand and two strides: LBO, between core matrices adjacent
// along K, and SBO, between core matrices adjacent along M (or N).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "pty_copy.cuh"

namespace pty {

// Shared-memory matrix descriptor: start address, LBO and SBO (bytes, each a
// multiple of 16 below 256 KB), descriptor version 1 (bits 46-48 = 0b001),
// base offset 0, relative LBO, no swizzle.
__device__ __forceinline__ uint64_t tc_smem_desc(const void* start, uint32_t lbo, uint32_t sbo) {
  const uint32_t a = smem_u32(start);
  return (uint64_t)((a & 0x3FFFFu) >> 4) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
         ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46);
}

// Instruction descriptor of kind::tf32: D in FP32, A and B in TF32, both
// K-major, shape M x N (M = 128, N a multiple of 8 up to 256); neg_b
// negates B.
__host__ __device__ constexpr uint32_t tc_idesc_tf32(int M, int N, bool neg_b) {
  return (1u << 4)                        // D format: F32
         | (2u << 7)                      // A format: TF32
         | (2u << 10)                     // B format: TF32
         | ((neg_b ? 1u : 0u) << 14)      // negate B
         | ((uint32_t)(N >> 3) << 17)     // N / 8
         | ((uint32_t)(M >> 4) << 24);    // M / 16
}

// TMEM allocation of ncols columns (a power of two, 32..512) by one whole
// warp; the TMEM address is written to *slot (shared memory).
__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t ncols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(ncols)
               : "memory");
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols)
               : "memory");
}

// D (TMEM) = A B (accumulate = 0) or D += A B, issued by one thread.
__device__ __forceinline__ void tc_mma_tf32(uint32_t d_tmem, uint64_t adesc, uint64_t bdesc,
                                            uint32_t idesc, uint32_t accumulate) {
  asm volatile(
      "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
      " tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n}\n" ::"r"(d_tmem),
      "l"(adesc), "l"(bdesc), "r"(idesc), "r"(accumulate)
      : "memory");
}
// The mbarrier receives one arrival when every MMA this thread issued so far
// has completed.
__device__ __forceinline__ void tc_commit(unsigned long long* mbar) {
  asm volatile(
      "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
          smem_u32(mbar))
      : "memory");
}
__device__ __forceinline__ void tc_fence_before_sync() {
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after_sync() {
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (shape 32x32b: the
// warp reads lanes 32 (warp % 4) .. + 31, thread t lane + t), then the wait.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float* v) {
  uint32_t r[32];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, "
      "%11, %12, %13, %14, %15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, "
      "%28, %29, %30, %31}, [%32];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]),
        "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]),
        "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// x = hi + lo with hi = x cut to a TF32 value (its low 13 mantissa bits
// cleared) and lo = x - hi, exact in FP32 and itself taken as TF32 by the
// MMA: the three products hi hi + hi lo + lo hi carry about 21 bits of each
// operand.
__device__ __forceinline__ void tf32_split(float x, float& hi, float& lo) {
  hi = __uint_as_float(__float_as_uint(x) & 0xFFFFE000u);
  lo = x - hi;
}

}  // namespace pty
