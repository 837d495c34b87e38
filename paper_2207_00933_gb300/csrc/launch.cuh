// Kernel launches with programmatic dependent launch (PDL).
//
// A step of the reconstruction is a chain of short, dependent kernels on
// one stream (attribution, merge, contraction steps, selection), each a few
// microseconds long at the usual sizes, so the gap between one kernel's
// end and the next one's start is a large share of the step.  With PDL the
// next kernel is launched while the previous one is still running: its CTAs
// are scheduled as soon as every CTA of the previous kernel has started (or
// resources free up) and wait in griddepcontrol.wait until the previous
// kernel has completed and its memory is visible.
//
// Contract of every kernel launched through launch_k: it calls
// pdl_wait() before its first global-memory access (a no-op when the
// launch carried no programmatic dependency), then pdl_trigger().
#pragma once
#include <cuda_runtime.h>

namespace sqc {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// Whether launches from this host thread carry the programmatic
// dependency (set per API call from the context's configuration).
bool& pdl_flag();

struct PdlScope {
  bool prev;
  explicit PdlScope(bool on) : prev(pdl_flag()) { pdl_flag() = on; }
  ~PdlScope() { pdl_flag() = prev; }
};

template <typename... KArgs, typename... Args>
cudaError_t launch_k(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                     bool cooperative, const Args&... args) {
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = grid;
  cfg.blockDim = block;
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[2];
  int na = 0;
  if (pdl_flag()) {
    attr[na].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[na].val.programmaticStreamSerializationAllowed = 1;
    ++na;
  }
  if (cooperative) {
    attr[na].id = cudaLaunchAttributeCooperative;
    attr[na].val.cooperative = 1;
    ++na;
  }
  cfg.attrs = na ? attr : nullptr;
  cfg.numAttrs = na;
  cudaError_t e = cudaLaunchKernelEx(&cfg, kernel, args...);
  if (e != cudaSuccess && pdl_flag()) {
    // a launch form that does not take the programmatic dependency: plain
    cudaGetLastError();
    cfg.attrs = cooperative ? attr + (na - 1) : nullptr;
    cfg.numAttrs = cooperative ? 1 : 0;
    e = cudaLaunchKernelEx(&cfg, kernel, args...);
  }
  return e;
}

}  // namespace sqc
