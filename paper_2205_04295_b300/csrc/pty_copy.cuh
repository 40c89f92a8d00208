// Asynchronous global -> shared copies: cp.async (LDGSTS) for small or
// unaligned pieces, and tensor-map TMA loads (cp.async.bulk.tensor) that
// complete on an mbarrier.  A CTA requests the next patch's data while it
// transforms the current one, and no registers are held for data in flight.
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

// ---- tensor-map (TMA) copies completing on an mbarrier
__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return (unsigned)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(unsigned long long* mb, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(mb)), "r"(count)
               : "memory");
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
// Order this thread's earlier generic-proxy shared-memory accesses before
// the async proxy's (a TMA write into a buffer the CTA has just read).
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* mb, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(mb)),
               "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* mb, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(smem_u32(mb)), "r"(parity)
      : "memory");
  return ok != 0;
}
// Wait for phase `parity` of the mbarrier, giving up after `limit_ns` of the
// global timer; returns false on time-out.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* mb, unsigned parity,
                                                  unsigned long long limit_ns) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (!mbar_try_wait(mb, parity)) {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > limit_ns) return false;
  }
  return true;
}
// The library's status words: err[0] is set by a wait that gave up; err[1]
// (0 or 1, written only by the host between calls) is a test hook that gives
// a staged pass's mbarrier one more expected arrival, which no copy makes, so
// that its bounded waits run out while every copy still completes.
__device__ __forceinline__ int stalled_arrivals(const int* err) {
  return err ? *reinterpret_cast<const volatile int*>(err + 1) : 0;
}
// Bulk (TMA, no tensor map) copy of `bytes` (a multiple of 16; both
// addresses 16-byte aligned) from global to shared memory, completing on mb.
__device__ __forceinline__ void bulk_load(void* dst, const void* src, unsigned bytes,
                                          unsigned long long* mb) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
      ::"r"(smem_u32(dst)), "l"(src), "r"(bytes), "r"(smem_u32(mb))
      : "memory");
}
// 3-D tiled TMA load of the box at (x, y, z) of tensor map `tm` into dst.
__device__ __forceinline__ void tma_load_3d(void* dst, const void* tm, int x, int y, int z,
                                            unsigned long long* mb) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(smem_u32(dst)),
      "l"(reinterpret_cast<unsigned long long>(tm)), "r"(x), "r"(y), "r"(z), "r"(smem_u32(mb))
      : "memory");
}

}  // namespace pty
