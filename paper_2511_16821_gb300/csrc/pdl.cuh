// pdl.cuh -- programmatic dependent launch between kernels of one stream (sm_90 and later).
//
// A kernel launched with programmatic stream serialisation may be scheduled before its predecessor
// in the stream has finished: as soon as every block of the predecessor has signalled
// launch_dependents (or exited). Its blocks are then resident when the predecessor ends, instead
// of being launched after it. Every kernel launched this way calls pdl_wait() before it reads
// anything its predecessor wrote (the wait returns once the predecessor has completed and its
// memory is visible); it calls pdl_trigger() to let its own successor be scheduled. Without a
// programmatic predecessor the wait returns at once. A successor is scheduled only after every
// block of its predecessor has started, so waiting blocks never hold resources the predecessor
// still needs. Problems stepped in a batch launch normally (their step graphs run many streams
// at once, where programmatic launch measured slower).
#pragma once

#include <cuda_runtime.h>

#include <utility>

namespace hyb {

__device__ __forceinline__ void pdl_wait() { asm volatile("griddepcontrol.wait;" ::: "memory"); }
__device__ __forceinline__ void pdl_trigger() { asm volatile("griddepcontrol.launch_dependents;" ::: "memory"); }

// pdl = false: an ordinary launch (the kernel's wait and trigger are then no-ops)
template <typename... KArgs, typename... Args>
static cudaError_t launch_pdl(bool pdl, void (*kern)(KArgs...), dim3 grid, dim3 block, size_t smem, cudaStream_t s,
                              Args&&... args) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = pdl ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

}  // namespace hyb
