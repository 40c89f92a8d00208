// Asynchronous global -> shared copies (cp.async, the LDGSTS path): a CTA
// requests the next patch's data while it transforms the current one, and no
// registers are held for the data in flight.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pty {

// Copy B bytes (4, 8 or 16; both addresses B-aligned) from global to shared.
template <int B>
__device__ __forceinline__ void cp_async(void* smem, const void* gmem) {
  static_assert(B == 4 || B == 8 || B == 16, "cp.async sizes are 4, 8 or 16 bytes");
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  if (B == 16)
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
  else
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(B)
                 : "memory");
}
__device__ __forceinline__ void cp_async_commit() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
}
// Wait until at most N of this thread's committed groups are still pending.
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

}  // namespace pty
