// lb_internal.cuh -- context layout and launcher declarations shared by the
// translation units of liblb (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "lb.h"

#ifndef LBK_COMPONENT_PAD
#define LBK_COMPONENT_PAD 0
#endif

namespace lbk {

// Component stride of the SoA distribution arrays: N rounded up to 64
// elements, plus LBK_COMPONENT_PAD elements.
inline long long component_stride(long long N) { return ((N + 63) / 64) * 64 + LBK_COMPONENT_PAD; }

struct Buffers {
    void *f[2] = {nullptr, nullptr};  // SoA [19][N] in storage type, two time levels
    void *g[2] = {nullptr, nullptr};
    int cur = 0;                      // index of the buffer holding the state
};

}  // namespace lbk

struct lb_ctx {
    lb_params p;
    cudaStream_t stream;
    int device;
    long long N;
    long long S;           // elements between distribution components (>= N, padded)
    size_t esize;          // 8 (FP64) or 4 (FP32 shifted)
    lbk::Buffers buf;      // post-collision (pre-streaming) distributions
    void *phi = nullptr;   // [N] storage type: order parameter of the two-pass kernel
    double *io = nullptr;  // [4N] FP64 staging for host transfers (lazy)
    double *partial = nullptr;  // reduction partials [kReduceBlocks][5]
    double *dev_out = nullptr;  // [8] reduction result
    int kernel = LB_KERNEL_AUTO;
    int block_x = 0, block_y = 0, z_chunk = 0;
    lb_alloc_fn alloc = nullptr;
    lb_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
};

namespace lbk {

constexpr int kReduceBlocks = 608;   // 4 x 152 SMs; fixed so sums are reproducible
constexpr int kReduceThreads = 256;

// status helpers (lb_api.cu)
int cuda_status(cudaError_t e);
int check_launch();

// launchers (lb_kernels.cu); each returns an LB_* code
int launch_init(lb_ctx *c, const double *phi0_d, const double *u0_d);
int launch_step_two_pass(lb_ctx *c, int nsteps);
int launch_moments(lb_ctx *c, double *rho, double *u, double *phi);
int launch_get_state(lb_ctx *c, double *f, double *g);
int launch_set_state(lb_ctx *c, const double *f, const double *g);
// rows [i0, i1) of f (which = 0) or g (which = 1): dir 0 = out of the state, 1 = into it
int launch_rows(lb_ctx *c, int which, int i0, int i1, double *buf, int dir);
int launch_reduce(lb_ctx *c, double *dev_out5);

// fused kernel (lb_fused.cu)
int launch_step_fused(lb_ctx *c, int nsteps);
int fused_validate(int precision, int block_x, int block_y, int z_chunk);

// staged kernel (lb_staged.cu)
int launch_step_staged(lb_ctx *c, int nsteps);
int staged_validate(int precision, int block_x, int block_y, int z_chunk);

}  // namespace lbk
