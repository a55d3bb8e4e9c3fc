// lb_kernels.cu -- the default two-pass timestep (phi pass, then the fused
// pull-collide-stream pass).
//
// Storage convention: the context keeps the post-collision, pre-streaming
// distributions A_i(x).  The post-streaming state of the model is the pull
// f_i(x, t) = A_i(x - c_i), so one timestep is "pull, collide at x, write
// A'_i(x)": every store is aligned to its own site and every load is a
// shifted, still coalesced read (targetDP Sec. III.B: SoA so consecutive
// sites are consecutive in memory).
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lb_internal.cuh"
#include "lb_pdl.cuh"
#include "lb_site.cuh"

namespace lbk {

// ------------------------------------------------------------------ two-pass step
// (both kernels launched with programmatic dependent launch, lb_pdl.cuh)

// phi = sum_i g_i(x - c_i) of V sites per thread (the paper's virtual vector
// length): the thread's sites are blockDim.x apart, their 19 V loads are
// issued before any sum
template <typename T, int V>
__global__ void __launch_bounds__(256) k_phi_pull(const T *__restrict__ ga, T *__restrict__ phi,
                                                  int nx, int ny, int nz, long long S)
{
    pdl_wait_then_release();
    const int N = nx * ny * nz;
    const int s0 = blockIdx.x * blockDim.x * V + threadIdx.x;
    T g[V][Q];
#pragma unroll
    for (int v = 0; v < V; v++) {
        const int s = s0 + v * (int)blockDim.x;
        if (s < N) {
            const Nbr n(s, nx, ny, nz);
#pragma unroll
            for (int i = 0; i < Q; i++) g[v][i] = ga[(size_t)i * S + n.src(i)];
        }
    }
#pragma unroll
    for (int v = 0; v < V; v++) {
        const int s = s0 + v * (int)blockDim.x;
        if (s < N) phi[s] = sum19(g[v]);
    }
}

// CTAs per SM the register budget of the collide/stream kernel must allow
// (measured: FP64 is bound by the FP64 pipe at 2 or 3; an allowance of 1
// lets ptxas spend 152 registers and loses 11 %; FP32 is DRAM-bound)
#ifndef LBK_K2_MINB64
#define LBK_K2_MINB64 2
#endif
#ifndef LBK_K2_MINB32
#define LBK_K2_MINB32 3
#endif
#ifndef LBK_K2_MINBDF
#define LBK_K2_MINBDF 2
#endif
#ifndef LBK_K2_MINB32W
#define LBK_K2_MINB32W 3   // FP32 with the 19- / 27-point stencils
#endif
#define LBK_K2_MINB(T, NP) \
    (is_df64<T>::value ? LBK_K2_MINBDF : sizeof(T) == 8 ? LBK_K2_MINB64 : NP > 7 ? LBK_K2_MINB32W : LBK_K2_MINB32)

template <typename T, bool SH, int NP = 7>
__global__ void __launch_bounds__(256, LBK_K2_MINB(T, NP)) k_collide_pull(const T *__restrict__ fa, const T *__restrict__ ga,
                                                      const T *__restrict__ phi,
                                                      T *__restrict__ fb, T *__restrict__ gb,
                                                      Coll<T> p, int nx, int ny, int nz, long long S)
{
    pdl_wait_then_release();
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n(s, nx, ny, nz);
    collide_site<T, SH, NP>(fa, ga, phi, fb, gb, p, n, s, S);
}

// multiple-relaxation-time collision of f with a Guo body force (collide_mrt)
template <typename T, bool SH, int NP>
__global__ void __launch_bounds__(256, LBK_K2_MINB(T, NP))
k_collide_pull_mrt(const T *__restrict__ fa, const T *__restrict__ ga, const T *__restrict__ phi,
                   T *__restrict__ fb, T *__restrict__ gb, Coll<T> p, Mrt<T> m, int nx, int ny, int nz,
                   long long S)
{
    pdl_wait_then_release();
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n(s, nx, ny, nz);
    T f[Q], g[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const size_t o = (size_t)i * S + n.src(i);
        f[i] = fa[o];
        g[i] = ga[o];
    }
    const T ph = phi[s];
    T dx, dy, dz, lap;
    stencil_np<NP, T>(phi, n, ph, dx, dy, dz, lap);
    collide_mrt<T, SH>(p, m, f, g, ph, dx, dy, dz, lap);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        fb[(size_t)i * S + s] = f[i];
        gb[(size_t)i * S + s] = g[i];
    }
}

// ------------------------------------------------------------------ launchers

static inline unsigned grid_for(long long N, int tpb) { return (unsigned)((N + tpb - 1) / tpb); }

// the phi pass with V sites per thread
template <typename T>
static cudaError_t launch_phi(lb_ctx *c, const T *ga, int tpb, int vvl)
{
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const unsigned grid = grid_for(c->N, tpb * vvl);
    if (vvl == 4) return launch_pdl(k_phi_pull<T, 4>, grid, tpb, c->stream, ga, (T *)c->phi, nx, ny, nz, c->S);
    if (vvl == 2) return launch_pdl(k_phi_pull<T, 2>, grid, tpb, c->stream, ga, (T *)c->phi, nx, ny, nz, c->S);
    return launch_pdl(k_phi_pull<T, 1>, grid, tpb, c->stream, ga, (T *)c->phi, nx, ny, nz, c->S);
}

template <typename T, bool SH, int NP>
static int two_pass(lb_ctx *c, int nsteps)
{
    const auto p = make_coll<T>(c->p);
    const bool mrt = uses_mrt(c);
    const auto m = make_mrt<T>(c);
    // launch shape: threads per CTA of both passes, sites per thread of the
    // phi pass (lb_set_kernel's block_x, block_y; 0 = 256 and 1)
    const int tpb = c->block_x ? c->block_x : 256;
    const int vvl = c->block_y ? c->block_y : 1;
    const unsigned grid = grid_for(c->N, tpb);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    for (int t = 0; t < nsteps; t++) {
        const int a = c->buf.cur, b = 1 - a;
        const T *fa = (const T *)c->buf.f[a], *ga = (const T *)c->buf.g[a];
        T *fb = (T *)c->buf.f[b], *gb = (T *)c->buf.g[b];
        cudaError_t e = launch_phi<T>(c, ga, tpb, vvl);
        if (e == cudaSuccess) {
            if (mrt)
                e = launch_pdl(k_collide_pull_mrt<T, SH, NP>, grid, tpb, c->stream, fa, ga, (const T *)c->phi, fb, gb,
                               p, m, nx, ny, nz, c->S);
            else
                e = launch_pdl(k_collide_pull<T, SH, NP>, grid, tpb, c->stream, fa, ga, (const T *)c->phi, fb, gb, p,
                               nx, ny, nz, c->S);
        }
        int rc = e != cudaSuccess ? cuda_status(e) : check_launch();
        if (rc) return rc;
        c->buf.cur = b;
    }
    return LB_OK;
}

int launch_two_pass_fp64_raw(const lb_params &prm, const double *fa, const double *ga, double *phi, double *fb,
                             double *gb, long long S, cudaStream_t stream)
{
    const auto p = make_coll<double>(prm);
    const long long N = (long long)prm.nx * prm.ny * prm.nz;
    const unsigned grid = grid_for(N, 256);
    k_phi_pull<double, 1><<<grid, 256, 0, stream>>>(ga, phi, prm.nx, prm.ny, prm.nz, S);
    k_collide_pull<double, false><<<grid, 256, 0, stream>>>(fa, ga, phi, fb, gb, p, prm.nx, prm.ny, prm.nz, S);
    return check_launch();
}

template <typename T, bool SH>
static int two_pass_t(lb_ctx *c, int nsteps)
{
    if (c->npts == 19) return two_pass<T, SH, 19>(c, nsteps);
    if (c->npts == 27) return two_pass<T, SH, 27>(c, nsteps);
    return two_pass<T, SH, 7>(c, nsteps);
}

int two_pass_validate(int block_x, int block_y, int z_chunk)
{
    if (block_x != 0 && (block_x % 32 != 0 || block_x < 32 || block_x > 256)) return LB_ERR_INVALID;
    if (block_y != 0 && block_y != 1 && block_y != 2 && block_y != 4) return LB_ERR_INVALID;
    return z_chunk == 0 ? LB_OK : LB_ERR_INVALID;
}

int launch_step_two_pass(lb_ctx *c, int nsteps)
{
    return by_precision(c, [&](auto P) { return two_pass_t<typename decltype(P)::T, decltype(P)::SH>(c, nsteps); });
}

}  // namespace lbk
