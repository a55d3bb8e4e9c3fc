// lb_io.cu -- initialisation, moments, state I/O and the FP64 conservation
// reductions of a lattice (everything but the timestep itself).
//
// The context keeps the post-collision, pre-streaming distributions A_i(x);
// the post-streaming state is the pull f_i(x, t) = A_i(x - c_i), so every
// per-site quantity here gathers A_i from x - c_i.
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "df64.cuh"
#include "lb_internal.cuh"
#include "lb_moments.cuh"
#include "lb_site.cuh"

namespace lbk {

// ------------------------------------------------------------------ init

// A_i(x - c_i) = feq_i(x), so that the first pull yields the equilibrium of
// phi0 (its stencils taken in double) and u0.  Double storage evaluates the
// equilibria in double.  Float and double-float storage evaluate them in
// double-float arithmetic on the FP32 units (df64.cuh, ~48 bits; the double
// pipe runs at 1/64 of the float rate): double-float storage keeps the
// value, float storage its high part -- the float nearest to it, the same
// float as rounding a double result except at a near tie.
__device__ __forceinline__ void init_store(float *a, size_t o, df64 v) { a[o] = v.hi; }
__device__ __forceinline__ void init_store(df64 *a, size_t o, df64 v) { a[o] = v; }

template <typename T, bool SH, int NP>
__global__ void __launch_bounds__(256) k_init(const double *__restrict__ phi0,
                                              const double *__restrict__ u0,
                                              T *__restrict__ fa, T *__restrict__ ga,
                                              Coll<double> p, Coll<df64> pd, int nx, int ny, int nz, long long S)
{
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n(s, nx, ny, nz);
    const double ph = phi0[s];
    double dx, dy, dz, lap;
    stencil_np<NP, double>(phi0, n, ph, dx, dy, dz, lap);
    const double jx = u0 ? p.rho0 * u0[s] : 0.0;
    const double jy = u0 ? p.rho0 * u0[N + s] : 0.0;
    const double jz = u0 ? p.rho0 * u0[2 * N + s] : 0.0;
    const double R = SH ? 0.0 : p.rho0;
    if constexpr (sizeof(T) == 8 && !is_df64<T>::value) {
        equilibria<double, SH>(p, R, jx, jy, jz, ph, dx, dy, dz, lap, [&](int i, double fe, double ge) {
            const size_t o = (size_t)i * S + n.src(i);
            fa[o] = fe;
            ga[o] = ge;
        });
    } else {
        const df64 zero(0.0f, 0.0f);
        equilibria<df64, SH>(pd, df64(R), u0 ? df64(jx) : zero, u0 ? df64(jy) : zero, u0 ? df64(jz) : zero,
                             df64(ph), df64(dx), df64(dy), df64(dz), df64(lap), [&](int i, df64 fe, df64 ge) {
                                 const size_t o = (size_t)i * S + n.src(i);
                                 init_store(fa, o, fe);
                                 init_store(ga, o, ge);
                             });
    }
}

// ------------------------------------------------------------------ moments / state

template <typename T, bool SH>
__global__ void __launch_bounds__(256) k_moments(const T *__restrict__ fa, const T *__restrict__ ga,
                                                 double *__restrict__ rho, double *__restrict__ u,
                                                 double *__restrict__ phi, double rho0, double hFx,
                                                 double hFy, double hFz, int nx, int ny, int nz, long long S)
{
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n(s, nx, ny, nz);
    if (rho || u) {
        double r, v[3];
        site_rho_u<T, SH>(fa, n, S, rho0, hFx, hFy, hFz, r, v);
        if (rho) rho[s] = r;
        if (u) {
            u[s] = v[0];
            u[N + s] = v[1];
            u[2 * N + s] = v[2];
        }
    }
    if (phi) phi[s] = site_phi(ga, n, S);
}

// out[(i - i0)*N + s] = A_i(x - c_i) + shift_i, for i in [i0, i1)
template <typename T>
__global__ void __launch_bounds__(256) k_get_state(const T *__restrict__ a, double *__restrict__ out,
                                                   int i0, int i1, double shift_rho0,
                                                   int nx, int ny, int nz, long long S)
{
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n(s, nx, ny, nz);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        if (i < i0 || i >= i1) continue;
        out[(size_t)(i - i0) * N + s] = double(a[(size_t)i * S + n.src(i)]) + weight(i) * shift_rho0;
    }
}

// A_i(x - c_i) = in[(i - i0)*N + s] - shift_i, for i in [i0, i1)
template <typename T>
__global__ void __launch_bounds__(256) k_set_state(T *__restrict__ a, const double *__restrict__ in,
                                                   int i0, int i1, double shift_rho0,
                                                   int nx, int ny, int nz, long long S)
{
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n(s, nx, ny, nz);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        if (i < i0 || i >= i1) continue;
        a[(size_t)i * S + n.src(i)] = T(in[(size_t)(i - i0) * N + s] - weight(i) * shift_rho0);
    }
}

// ------------------------------------------------------------------ reductions
// Totals over all sites need no pull: sum_x f_i(x, t) = sum_x A_i(x - c_i)
// = sum_x A_i(x) on the periodic lattice.

__device__ __forceinline__ double warp_sum(double v)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    return v;
}

template <int K>
__device__ __forceinline__ void block_sum(double (&acc)[K], double *out)
{
    __shared__ double sh[kReduceThreads / 32][K];
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
#pragma unroll
    for (int k = 0; k < K; k++) acc[k] = warp_sum(acc[k]);
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < K; k++) sh[wid][k] = acc[k];
    __syncthreads();
    if (wid == 0) {
#pragma unroll
        for (int k = 0; k < K; k++) {
            double v = lane < kReduceThreads / 32 ? sh[lane][k] : 0.0;
            v = warp_sum(v);
            if (lane == 0) out[k] = v;
        }
    }
}

// A stored value widened to FP64 exactly.  float: from the IEEE 754
// binary32 and binary64 layouts -- sign and fraction kept (the fraction
// moved up 29 bits), the exponent rebiased by 1023 - 127 = 896; a subnormal
// is first scaled by 2^64 (exact in FP32, and normal) and rebiased by 64
// less; zero keeps its sign, infinity stays infinite and NaN becomes a quiet
// NaN.  Integer and FP32 operations only: on GB300 the conversion
// instruction runs on the FP64 pipe (about 2 lanes a clock per SM), where it
// would double this kernel's FP64 work.
__device__ __forceinline__ double widen(float x)
{
    const unsigned u = __float_as_uint(x), a = u & 0x7fffffffu;
    const bool sub = a < 0x00800000u;   // zero or subnormal
    const unsigned v = sub ? (__float_as_uint(x * 0x1p64f) & 0x7fffffffu) : a;
    unsigned hi = (v >> 3) + (sub ? 0x34000000u : 0x38000000u);
    hi = v ? hi : 0u;
    if (a >= 0x7f800000u) hi = (a >> 3) | 0x7ff00000u | (a > 0x7f800000u ? 0x00080000u : 0u);
    return __hiloint2double((int)(hi | (u & 0x80000000u)), (int)(v << 29));
}
__device__ __forceinline__ double widen(double x) { return x; }
// hi + lo of a double-float is exact in FP64 (|lo| <= ulp(hi) / 2)
__device__ __forceinline__ double widen(df64 x) { return widen(x.hi) + widen(x.lo); }

// Per-block partial totals.  A thread sums each of the 19 f rows over its
// sites in FP64 (sum_x A_i(x)), and the g rows (G rows: 19, or 1 in the
// tau_g = 1 reduced form, whose row 0 holds phi) into four FP64 partial
// sums, as only their total, sum phi, is wanted; R and j = sum_i c_i F_i are
// formed from the 19 row totals once per thread.  That is 38 FP64 additions
// a site (plus one per float of a double-float) against the 68 that forming
// every site's moments takes.  The order of every addition is fixed by the
// launch shape, so the totals are bitwise reproducible.
template <typename T, int G_ROWS>
__global__ void __launch_bounds__(kReduceThreads, 2) k_reduce_partial(const T *__restrict__ fa,
                                                                      const T *__restrict__ ga, long long N,
                                                                      long long S, double *__restrict__ partial)
{
    double F[Q], G[4] = {0.0, 0.0, 0.0, 0.0};
#pragma unroll
    for (int i = 0; i < Q; i++) F[i] = 0.0;
    for (long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x; s < N;
         s += (long long)gridDim.x * blockDim.x) {
        T f[Q], g[G_ROWS];
#pragma unroll
        for (int i = 0; i < Q; i++) f[i] = fa[(size_t)i * S + s];
#pragma unroll
        for (int i = 0; i < G_ROWS; i++) g[i] = ga[(size_t)i * S + s];
#pragma unroll
        for (int i = 0; i < Q; i++) F[i] += widen(f[i]);
#pragma unroll
        for (int i = 0; i < G_ROWS; i++) G[i & 3] += widen(g[i]);
    }
    double acc[5];
    density_moments(F, acc[0], acc[1], acc[2], acc[3]);
    acc[4] = (G[0] + G[1]) + (G[2] + G[3]);
    block_sum<5>(acc, partial + 5 * blockIdx.x);
}

__global__ void __launch_bounds__(kReduceThreads) k_reduce_final(const double *__restrict__ partial,
                                                                 int nblocks, double offset0,
                                                                 double *__restrict__ out)
{
    double acc[5] = {0.0, 0.0, 0.0, 0.0, 0.0};
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x)
#pragma unroll
        for (int k = 0; k < 5; k++) acc[k] += partial[5 * b + k];
    __shared__ double res[5];
    block_sum<5>(acc, res);
    __syncthreads();
    if (threadIdx.x == 0) {
        out[0] = res[0] + offset0;
        for (int k = 1; k < 5; k++) out[k] = res[k];
    }
}

// ------------------------------------------------------------------ launchers

static inline unsigned grid_for(long long N, int tpb) { return (unsigned)((N + tpb - 1) / tpb); }

template <typename T, bool SH, int NP>
static void init_np(lb_ctx *c, const double *phi0_d, const double *u0_d)
{
    const int cur = c->buf.cur;
    k_init<T, SH, NP><<<grid_for(c->N, 256), 256, 0, c->stream>>>(phi0_d, u0_d, (T *)c->buf.f[cur],
                                                                  (T *)c->buf.g[cur], make_coll<double>(c->p),
                                                                  make_coll<df64>(c->p), c->p.nx, c->p.ny,
                                                                  c->p.nz, c->S);
}

template <typename T, bool SH>
static void init_t(lb_ctx *c, const double *phi0_d, const double *u0_d)
{
    if (c->npts == 19)
        init_np<T, SH, 19>(c, phi0_d, u0_d);
    else if (c->npts == 27)
        init_np<T, SH, 27>(c, phi0_d, u0_d);
    else
        init_np<T, SH, 7>(c, phi0_d, u0_d);
}

int launch_init(lb_ctx *c, const double *phi0_d, const double *u0_d)
{
    return by_precision(c, [&](auto P) {
        init_t<typename decltype(P)::T, decltype(P)::SH>(c, phi0_d, u0_d);
        return check_launch();
    });
}

int launch_moments(lb_ctx *c, double *rho, double *u, double *phi)
{
    const int cur = c->buf.cur;
    const double hF[3] = {0.5 * c->force[0], 0.5 * c->force[1], 0.5 * c->force[2]};
    const unsigned grid = grid_for(c->N, 256);
    return by_precision(c, [&](auto P) {
        using T = typename decltype(P)::T;
        k_moments<T, decltype(P)::SH><<<grid, 256, 0, c->stream>>>((const T *)c->buf.f[cur], (const T *)c->buf.g[cur],
                                                                  rho, u, phi, c->p.rho0, hF[0], hF[1], hF[2],
                                                                  c->p.nx, c->p.ny, c->p.nz, c->S);
        return check_launch();
    });
}

// f or g, components [i0, i1), to out (i1 - i0 rows of N)
static int get_rows(lb_ctx *c, int which, int i0, int i1, double *out)
{
    const int cur = c->buf.cur;
    const unsigned grid = grid_for(c->N, 256);
    const double shift = (which == 0 && c->p.precision == LB_FP32_SHIFTED) ? c->p.rho0 : 0.0;
    const void *a = which == 0 ? c->buf.f[cur] : c->buf.g[cur];
    return by_precision(c, [&](auto P) {
        using T = typename decltype(P)::T;
        k_get_state<T><<<grid, 256, 0, c->stream>>>((const T *)a, out, i0, i1, shift, c->p.nx, c->p.ny, c->p.nz,
                                                     c->S);
        return check_launch();
    });
}

static int set_rows(lb_ctx *c, int which, int i0, int i1, const double *in)
{
    const int cur = c->buf.cur;
    const unsigned grid = grid_for(c->N, 256);
    const double shift = (which == 0 && c->p.precision == LB_FP32_SHIFTED) ? c->p.rho0 : 0.0;
    void *a = which == 0 ? c->buf.f[cur] : c->buf.g[cur];
    return by_precision(c, [&](auto P) {
        using T = typename decltype(P)::T;
        k_set_state<T><<<grid, 256, 0, c->stream>>>((T *)a, in, i0, i1, shift, c->p.nx, c->p.ny, c->p.nz, c->S);
        return check_launch();
    });
}

int launch_get_state(lb_ctx *c, double *f, double *g)
{
    int rc = LB_OK;
    if (f) rc = get_rows(c, 0, 0, Q, f);
    if (!rc && g) rc = get_rows(c, 1, 0, Q, g);
    return rc;
}

int launch_set_state(lb_ctx *c, const double *f, const double *g)
{
    int rc = LB_OK;
    if (f) rc = set_rows(c, 0, 0, Q, f);
    if (!rc && g) rc = set_rows(c, 1, 0, Q, g);
    return rc;
}

int launch_rows(lb_ctx *c, int which, int i0, int i1, double *buf, int dir)
{
    return dir == 0 ? get_rows(c, which, i0, i1, buf) : set_rows(c, which, i0, i1, buf);
}

int launch_reduce(lb_ctx *c, double *dev_out5)
{
    const int cur = c->buf.cur;
    const double off = c->p.precision == LB_FP32_SHIFTED ? double(c->N) * c->p.rho0 : 0.0;
    int rc = by_precision(c, [&](auto P) {
        using T = typename decltype(P)::T;
        const T *fa = (const T *)c->buf.f[cur], *ga = (const T *)c->buf.g[cur];
        if (c->reduced)
            k_reduce_partial<T, 1><<<kReduceBlocks, kReduceThreads, 0, c->stream>>>(fa, ga, c->N, c->S, c->partial);
        else
            k_reduce_partial<T, Q><<<kReduceBlocks, kReduceThreads, 0, c->stream>>>(fa, ga, c->N, c->S, c->partial);
        return check_launch();
    });
    if (rc) return rc;
    k_reduce_final<<<1, kReduceThreads, 0, c->stream>>>(c->partial, kReduceBlocks, off, dev_out5);
    return check_launch();
}

}  // namespace lbk
