// lb_pdl.cuh -- programmatic dependent launch for the kernel pairs of a
// timestep.
//
// A kernel launched with the stream attribute ProgrammaticStreamSerialization
// may have its CTAs scheduled while the previous kernel on the stream drains.
// Each such kernel first executes griddepcontrol.wait, which returns once the
// previous kernel has completed and its writes are visible, and only then
// touches memory; it then executes griddepcontrol.launch_dependents, so the
// next kernel's launch and CTA start-up overlap its own last wave.  Both
// instructions are no-ops for a launch without the attribute.  Every kernel
// in the chain waits for its predecessor before it can complete, so kernels
// complete in plain stream order.  Measured on the FP32 two-pass step: +0.6 %
// at 256^3, +4 % at 128^3, +33 % at 64^3 (an L2-resident lattice, bound by
// the gaps between launches).
#pragma once

#include <cuda_runtime.h>

#ifndef LBK_PDL
#define LBK_PDL 1
#endif

namespace lbk {

__device__ __forceinline__ void pdl_wait_then_release()
{
    asm volatile("griddepcontrol.wait;" ::: "memory");
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
}

template <typename... KArgs, typename... Args>
inline cudaError_t launch_pdl(void (*kernel)(KArgs...), dim3 grid, dim3 block, cudaStream_t stream, Args... args)
{
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = block;
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = LBK_PDL ? 1 : 0;
    return cudaLaunchKernelEx(&cfg, kernel, args...);
}

}  // namespace lbk
