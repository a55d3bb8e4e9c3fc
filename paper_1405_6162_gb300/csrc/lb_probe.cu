// lb_probe.cu -- FP64 fused multiply-add throughput probe.
//
// The FP64 timestep is bound by GB300's FP64 pipe rather than by HBM, so its
// roofline needs the pipe's peak: this kernel issues nothing but FP64 fused
// multiply-adds (kChains independent chains per thread, enough warps per SM
// to cover their latency) and the caller times it with CUDA events.
#include <cuda_runtime.h>

#include "lb_internal.cuh"

namespace {

constexpr int kChains = 16;
constexpr int kUnroll = 4;

__global__ void __launch_bounds__(256) k_fma_fp64(int iters, double a, double b, double *__restrict__ sink)
{
    double acc[kChains];
#pragma unroll
    for (int k = 0; k < kChains; k++) acc[k] = (double)(threadIdx.x + k);
    // iters is a multiple of kUnroll: kUnroll x kChains independent FMAs per
    // trip, so the loop's own instructions are a few percent of the issue
#pragma unroll 1
    for (int it = 0; it < iters; it += kUnroll) {
#pragma unroll
        for (int u = 0; u < kUnroll; u++)
#pragma unroll
            for (int k = 0; k < kChains; k++) acc[k] = fma(acc[k], a, b);
    }
    double s = 0.0;
#pragma unroll
    for (int k = 0; k < kChains; k++) s += acc[k];
    // a is chosen by the caller so that the sum stays finite; the store
    // keeps the chains alive without writing more than one value per CTA
    if (s == -1.0) sink[blockIdx.x] = s;
}

}  // namespace

extern "C" int lb_probe_fp64_fma(int blocks, long long iters, double *sink, void *cuda_stream,
                                 double *flops_out)
{
    if (blocks < 1 || iters < kUnroll || iters > (1LL << 30) || iters % kUnroll || !sink || !flops_out)
        return LB_ERR_INVALID;
    k_fma_fp64<<<blocks, 256, 0, (cudaStream_t)cuda_stream>>>((int)iters, 0.999999, 1e-7, sink);
    *flops_out = 2.0 * kChains * (double)iters * 256.0 * (double)blocks;
    return lbk::check_launch();
}
