// pdl.cuh -- programmatic dependent launch between consecutive iterations.
//
// An iteration's kernel is launched with programmatic stream serialization:
// the next kernel of the stream (the next iteration, or the second kernel of
// this one) may then be scheduled while this one is still running, and waits
// in pdl_wait() until this one has completed and its writes are visible. The
// launch latency between the kernels of a captured chain is hidden; the
// synchronous semantics are unchanged. Without the attribute both calls do
// nothing.
#pragma once

#include <cuda_runtime.h>

namespace cupso {

// Wait for the preceding kernel of the stream (completed, writes visible).
__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

// Let the following kernel of the stream begin launching.
__device__ __forceinline__ void pdl_launch_next() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t st,
                              Args... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace cupso
