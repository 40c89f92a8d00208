// Thread-block clusters on sm_103a, as inline PTX: a CTA's rank in its
// cluster, the cluster-wide barrier and the generic address of a shared
// variable in another CTA of the cluster (distributed shared memory).  Loads
// and stores through such an address are ordinary C++ accesses; the barrier's
// release/acquire orders them against the other CTAs' accesses.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

namespace pty {

__device__ __forceinline__ unsigned cluster_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}

// Every thread of every CTA of the cluster arrives (release) and waits
// (acquire); called by all threads at the same point of uniform control flow.
__device__ __forceinline__ void cluster_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}

// Generic address of `p` (a shared-memory address of this CTA) in the CTA of
// cluster rank `rank`.  No side effects: repeated calls fold together.
template <typename T>
__device__ __forceinline__ T* cluster_map(T* p, unsigned rank) {
  uint64_t r;
  asm("mapa.u64 %0, %1, %2;" : "=l"(r) : "l"(reinterpret_cast<uint64_t>(p)), "r"(rank));
  return reinterpret_cast<T*>(r);
}

}  // namespace pty
