// Programmatic dependent launch (Hopper and later; used on sm_103a): a kernel
// of a dependent chain lets the next kernel start its independent prologue
// while it drains (pdl_trigger), and each kernel waits for the previous one
// (its completion and its memory) before touching that kernel's results or
// any caller data (pdl_wait).  Both are no-ops in a launch without the
// programmatic attribute, so the same device code serves plain launches.
#pragma once
#include <cuda_runtime.h>

namespace pty {

__device__ __forceinline__ void pdl_trigger() {
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Launch with programmatic stream serialisation allowed.
template <typename... KArgs, typename... Args>
cudaError_t launch_pdl(void (*kern)(KArgs...), dim3 g, dim3 b, size_t sm, cudaStream_t s,
                       Args... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = g;
  cfg.blockDim = b;
  cfg.dynamicSmemBytes = sm;
  cfg.stream = s;
  cudaLaunchAttribute at[1];
  at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
  at[0].val.programmaticStreamSerializationAllowed = 1;
  cfg.attrs = at;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, static_cast<KArgs>(args)...);
}

}  // namespace pty
