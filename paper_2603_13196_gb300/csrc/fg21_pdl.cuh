// Programmatic dependent launch for the likelihood's kernel chain (prep ->
// tensor or SIMT kernel -> reduction).  A kernel launched with
// launch_dependent() is scheduled as the blocks of the kernel before it in the
// stream exit, without the full kernel boundary in between, so its launch
// latency overlaps that kernel's tail (about 1 us per edge).  Every such
// kernel calls pdl_wait() before it reads or writes anything the earlier
// kernels touch: the wait returns once the preceding grid has completed and
// its memory operations are visible (and, through that grid's own wait,
// everything before it).  The wait is a no-op for a kernel launched the
// ordinary way.  No kernel triggers its dependents early: measured, the
// dependents' blocks then sit on the SMs beside the running kernel and cost
// more than the overlap gains.
#pragma once
#include <cuda_runtime.h>
#include <utility>

namespace fg21 {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }

template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kernel)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t stream,
                             Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = stream;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    at[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kernel, std::forward<Args>(args)...);
}

}  // namespace fg21
