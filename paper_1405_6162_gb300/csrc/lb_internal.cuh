// lb_internal.cuh -- context layout and launcher declarations shared by the
// translation units of liblb (not part of the ABI).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>

#include "d3q19.cuh"
#include "df64.cuh"
#include "lb.h"
#include "lb_coll.cuh"

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
    // lagged kernel: [0] = CTA ticket counter, [1 + z] = phi-done counter of plane z
    unsigned long long *lag_counters = nullptr;
    unsigned int *err_flag = nullptr;         // set by a device-side wait that timed out
    unsigned long long lag_target_skew = 0;   // test hook: makes the waits unsatisfiable
    long long wait_timeout_ns = 1000000000LL; // bound of every device-side wait
    double *adj = nullptr;        // [6N] adjoint scratch (lazy): phi_bar, d_bar (3), lap_bar, phi
    double *adj_part = nullptr;   // per-CTA partial dJ/dkappa
    int batch_owned = 0;  // member of an lb_batch: stepped and freed by it
    int reduced = 0;      // tau_g = 1 form: g kept as phi and (gmh, u), see lb_taug1.cu
    int m_valid = 0;      // reduced form: the previous step's (gmh, u) are present
    int npts = 7;         // points of the phi stencil: 7, 19 or 27 (lb_set_stencil)
    int collision = LB_COLLISION_BGK;       // collision of f (lb_set_collision)
    double tau_bulk = 1.0, tau_ghost = 1.0; // MRT relaxation times
    double force[3] = {0.0, 0.0, 0.0};      // Guo body force density (lb_set_force)
    unsigned char *mask_buf = nullptr;      // [N] device copy of a host mask (lazy)
    int *mask_scratch = nullptr;            // compaction counts and offsets (lazy)
    int kernel = LB_KERNEL_AUTO;
    int block_x = 0, block_y = 0, z_chunk = 0;
    lb_alloc_fn alloc = nullptr;
    lb_free_fn free_fn = nullptr;
    void *alloc_user = nullptr;
};

namespace lbk {

// the f collision needs the MRT / forced kernel
inline bool uses_mrt(const lb_ctx *c)
{
    return c->collision == LB_COLLISION_MRT || c->force[0] != 0.0 || c->force[1] != 0.0 || c->force[2] != 0.0;
}

// storage / arithmetic type of a context and whether f is stored shifted
template <typename T_, bool SH_>
struct Prec {
    using T = T_;
    static constexpr bool SH = SH_;
};

// f(Prec<T, SH>{}) for the context's precision
template <typename F>
inline int by_precision(const lb_ctx *c, F &&f)
{
    switch (c->p.precision) {
    case LB_FP64: return f(Prec<double, false>{});
    case LB_FP64_DF: return f(Prec<df64, false>{});
    default: return f(Prec<float, true>{});
    }
}

// MRT rates and force of the context in the arithmetic type T
template <typename T>
inline Mrt<T> make_mrt(const lb_ctx *c)
{
    return make_mrt<T>(c->p, c->collision == LB_COLLISION_MRT, c->tau_bulk, c->tau_ghost, c->force);
}

constexpr int kLagBlock = 256;       // sites per block of the lagged kernel
constexpr long long kLagSlack = 128;  // extra lag (blocks) beyond the stencil reach
constexpr int kReduceBlocks = 304;   // 2 x 152 SMs, one wave; fixed so sums are reproducible
constexpr int kReduceThreads = 256;

// ensemble membership (lb_api.cu): the member shares the batch's error flag
void adopt_into_batch(lb_ctx *c, unsigned int *shared_err);
void release_from_batch(lb_ctx *c);

// status helpers (lb_api.cu)
int cuda_status(cudaError_t e);
int check_launch();

// launchers (lb_kernels.cu); each returns an LB_* code
int launch_init(lb_ctx *c, const double *phi0_d, const double *u0_d);
int launch_step_two_pass(lb_ctx *c, int nsteps);
int two_pass_validate(int block_x, int block_y, int z_chunk);   // threads per CTA, phi sites per thread
// one FP64 two-pass timestep on raw buffers (component stride S, phi scratch
// of N doubles supplied by the caller)
int launch_two_pass_fp64_raw(const lb_params &p, const double *fa, const double *ga, double *phi, double *fb,
                             double *gb, long long S, cudaStream_t stream);
int launch_moments(lb_ctx *c, double *rho, double *u, double *phi);
int launch_get_state(lb_ctx *c, double *f, double *g);
int launch_set_state(lb_ctx *c, const double *f, const double *g);
// rows [i0, i1) of f (which = 0) or g (which = 1): dir 0 = out of the state, 1 = into it
int launch_rows(lb_ctx *c, int which, int i0, int i1, double *buf, int dir);
int launch_reduce(lb_ctx *c, double *dev_out5);   // reduced form: phi from component 0

// fused kernel (lb_fused.cu)
int launch_step_fused(lb_ctx *c, int nsteps);
int fused_validate(int precision, int block_x, int block_y, int z_chunk);

// staged kernel (lb_staged.cu)
int launch_step_staged(lb_ctx *c, int nsteps);
int staged_validate(int precision, int block_x, int block_y, int z_chunk);

// adjoint (lb_adjoint.cu)
int adjoint_blocks(long long N);
int launch_adjoint_step(lb_ctx *c, const double *f, const double *g, const double *af_in, const double *ag_in,
                        double *af_out, double *ag_out, double *dkappa, double *aux, double *kpart);
int launch_adjoint_seed(lb_ctx *c, const double *phi_bar, double *af, double *ag);
int launch_adjoint_init(lb_ctx *c, const double *phi0, const double *u0, const double *af0, const double *ag0,
                        double *phi0_bar, double *dkappa, double *aux, double *kpart);

// tau_g = 1 reduced form (lb_taug1.cu)
int launch_step_taug1(lb_ctx *c, int nsteps);
// y rows per warp (0 = by precision; 1, 2, 4), warps per block (0 = 4; 1..8),
// z run of the phi pass (0 = sized for about three waves)
int taug1_validate(const lb_params &p, int block_x, int block_y, int z_chunk);
int taug1_convert(lb_ctx *c, int to_reduced);
int taug1_g_rows(lb_ctx *c, int i0, int i1, double *out);
int taug1_phi_out(lb_ctx *c, double *out);

// masked copies (lb_masked.cu)
size_t masked_scratch_ints(long long N);
int masked_total_offset(long long N);
int launch_mask_scan(lb_ctx *c, const unsigned char *mask_d, int *scratch);
int launch_masked_moments(lb_ctx *c, long long total, const int *scratch, double *rho, double *u, double *phi);
int launch_masked_rows(lb_ctx *c, long long total, const int *scratch, int which, int i0, int i1, double *io,
                       int to_device_state);

// lagged kernel (lb_lag.cu)
int launch_step_lag(lb_ctx *c, int nsteps);
int lag_validate(int block_x, int block_y, int z_chunk);

// bulk-copy single-pass kernel (lb_bulk.cu)
int launch_step_bulk(lb_ctx *c, int nsteps);
int bulk_validate(const lb_params &p, int block_x, int block_y, int z_chunk);
// LB_KERNEL_AUTO: the bulk kernel in its fastest measured shape where it
// applies (FP32-shifted, 7-point BGK, a shape it takes), else the two-pass step
bool auto_uses_bulk(const lb_ctx *c);
int launch_step_bulk_auto(lb_ctx *c, int nsteps);

// slab kernel (lb_slab.cu)
int launch_step_slab(lb_ctx *c, int nsteps);
int slab_validate(int precision, int block_x, int block_y, int z_chunk);

}  // namespace lbk
