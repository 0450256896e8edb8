// Programmatic dependent launch (PDL) for the solver's iteration chain.
//
// A kernel launched with the programmatic-stream-serialization attribute may be
// scheduled while its predecessor in the stream is still running, once every
// CTA of the predecessor has signalled griddepcontrol.launch_dependents (or
// exited).  Its own griddepcontrol.wait then blocks until the predecessor grid
// has completed and its memory operations are visible, so the successor's
// launch latency and CTA rasterisation overlap the predecessor's tail instead
// of following it.
//
// Rule kept by every kernel launched through launch_k: pdl_begin() is its first
// statement, before any global-memory access (griddepcontrol.wait is a no-op for
// a kernel launched without the attribute).  Because the signal is given only
// after the wait, a grid can be scheduled early only behind a predecessor whose
// CTAs are all resident, and never before the grid two steps back has finished.
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace dda {

#ifdef __CUDACC__
__device__ __forceinline__ void pdl_begin() {
  asm volatile("griddepcontrol.wait;" ::: "memory");
  asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}
#endif

// Launches made by this host thread use the attribute while the flag is set
// (the solver sets it around its iteration chain).
bool pdl_enabled();
void set_pdl(bool on);

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st, Args&&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  if (pdl_enabled()) {
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
  }
  return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace dda
