// lb_taug1.cu -- the timestep for tau_g = 1, keeping g as its moments.
//
// With tau_g = 1 the collision of g returns its equilibrium exactly,
// g*_i = geq_i(phi, mu, u), so after streaming g_i(x, t+1) = geq_i evaluated
// with (phi, mu, u) of site x - c_i at time t, and phi(x, t+1) is the sum of
// those 19 values.  The context then keeps, instead of 19 values of g, five
// per site in its g buffers:
//     level a: component 0      phi(t)  (the stencil's input)
//              components 1..4  the quad (gmh, u_x, u_y, u_z) of each site,
//                               interleaved (one 16 B / 32 B vector per
//                               site), gmh = 9/2 (Gamma mu - phi/3)
// With P = phi (1 - 3/2 u^2) the equilibrium is then
//     geq_i = w_i [P + gmh (c_i^2 - 1) + c_i.u (3 phi + 9/2 phi c_i.u)].
// One step is two passes:
//   k_t1_collide  pull f, 7-point stencil of phi(t), collide f; write f* and
//                 gmh(t), u(t) next to phi(t)        (19+1 r, 19+4 w words)
//   k_t1_phi      phi(x, t+1) = sum_i geq_i(moments at x - c_i) into the
//                 other level's component 0          (5 r, 1 w words)
// -- 49 words per site instead of the 97 of the general two-pass step.
// k_t1_phi streams along z so that each source site's moments are loaded and
// expanded about once: a warp covers 32 consecutive x columns of which the
// 30 inner ones are outputs (the outer two only feed their neighbours); each
// lane walks a run of z planes for KY rows of its column, holding the
// partial sums of the three output planes a source plane reaches.  Sources
// in the lane's own column (c_x = 0) add to its own outputs; those with
// c_x = +-1 add to per-output partial sums that one shuffle each hands to
// lane +-1 once the output plane is complete.
// The per-site arithmetic is the general collision's (the g relaxation is
// simply not needed); results agree with the general step to rounding.
//
// Flag m_valid: (mu, u) of the previous step are present.  After lb_init or
// lb_set_state only phi(t) is known; g is then reported as the equilibrium at
// each site (exact after lb_init, which starts from that equilibrium).
#include <cuda_runtime.h>

#include <atomic>

#include "d3q19.cuh"
#include "lb_internal.cuh"
#include "lb_pdl.cuh"
#include "lb_site.cuh"
#include "lb_t1.cuh"

namespace lbk {

namespace {

constexpr int kT1Threads = 256;

template <typename T, bool SH, int NP>
__global__ void __launch_bounds__(kT1Threads, sizeof(T) == 8 ? 2 : 3)
k_t1_collide(const T *__restrict__ fa, T *__restrict__ ga /* level a: phi in, (gmh, u) out */, T *__restrict__ fb,
             Coll<T> p, int nx, int ny, int nz, long long S)
{
    pdl_wait_then_release();
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    t1_collide_site<T, SH, NP>(fa, ga, fb, p, nx, ny, nz, S, s);
}

constexpr int kPhiWarps = 4;      // default warps per block, stacked in y
constexpr int kPhiMaxWarps = 8;

template <typename T, int KY>
__global__ void __launch_bounds__(32 * kPhiMaxWarps) k_t1_phi(const T *__restrict__ ga, T *__restrict__ gb, int nx,
                                                               int ny, int nz, int kzc, long long S)
{
    pdl_wait_then_release();
    t1_phi_tile<T, KY>(ga, gb, nx, ny, nz, kzc, S, blockIdx.x, (blockIdx.y * blockDim.y + threadIdx.y) * KY,
                       blockIdx.z, threadIdx.x);
}

// g state of the reduced form as post-streaming FP64 rows [i0, i1):
// streamed equilibria of the previous step's moments (m_valid), else the
// equilibrium at each site from phi(t), its stencil and u from f.
template <typename T, bool SH, int NP>
__global__ void __launch_bounds__(kT1Threads) k_t1_g_state(const T *__restrict__ fa, const T *__restrict__ gcur,
                                                            const T *__restrict__ gprev, int m_valid, Coll<T> p,
                                                            double *__restrict__ out, int i0, int i1, int nx,
                                                            int ny, int nz, long long S)
{
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n(s, nx, ny, nz);
    if (m_valid) {
#pragma unroll
        for (int i = 0; i < Q; i++) {
            if (i < i0 || i >= i1) continue;
            out[(size_t)(i - i0) * N + s] = double(geq_eq(i, load_eq(gprev, S, n.src(i))));
        }
        return;
    }
    double f[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = double(fa[(size_t)i * S + n.src(i)]);
    double R, jx, jy, jz;
    density_moments(f, R, jx, jy, jz);
    const double rho = SH ? double(p.rho0) + R : R;
    const double ph = double(gcur[s]);
    double dx, dy, dz, lap;
    stencil_np<NP, double>(gcur, n, ph, dx, dy, dz, lap);
    const double mu = ph * (double(p.A) + double(p.B) * ph * ph) - double(p.kappa) * lap;
    const Eq<double> e = make_eq(ph, gmh_of(ph, mu, double(p.gamma)), jx / rho, jy / rho, jz / rho);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        if (i < i0 || i >= i1) continue;
        out[(size_t)(i - i0) * N + s] = geq_eq(i, e);
    }
}

// phi(t) of a full-form state (pull sum of g) into component 0 of level b
template <typename T>
__global__ void __launch_bounds__(kT1Threads) k_t1_from_full(const T *__restrict__ ga, T *__restrict__ phi_out,
                                                              int nx, int ny, int nz, long long S)
{
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n(s, nx, ny, nz);
    phi_out[s] = phi_site(ga, n, S);
}

// full-form g (post-collision storage) from the reduced form: A_i(x - c_i) =
// the g state at x.  gcur is phi(t) (a copy: gout is the current level)
template <typename T, bool SH, int NP>
__global__ void __launch_bounds__(kT1Threads) k_t1_to_full(const T *__restrict__ fa, const T *__restrict__ gcur,
                                                            const T *__restrict__ gprev, int m_valid, Coll<T> p,
                                                            T *__restrict__ gout, int nx, int ny, int nz, long long S)
{
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n(s, nx, ny, nz);
    double f[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = double(fa[(size_t)i * S + n.src(i)]);
    double R, jx, jy, jz;
    density_moments(f, R, jx, jy, jz);
    const double rho = SH ? double(p.rho0) + R : R;
    const double ph = double(gcur[s]);
    double dx, dy, dz, lap;
    stencil_np<NP, double>(gcur, n, ph, dx, dy, dz, lap);
    const double mu = ph * (double(p.A) + double(p.B) * ph * ph) - double(p.kappa) * lap;
    const Eq<double> own = make_eq(ph, gmh_of(ph, mu, double(p.gamma)), jx / rho, jy / rho, jz / rho);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        double v;
        if (m_valid)
            v = double(geq_eq(i, load_eq(gprev, S, n.src(i))));
        else
            v = geq_eq(i, own);
        gout[(size_t)i * S + n.src(i)] = T(v);
    }
}

template <typename T>
__global__ void __launch_bounds__(kT1Threads) k_t1_copy_phi(const T *__restrict__ phi_src, T *__restrict__ dst,
                                                            long long N)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < N) dst[s] = phi_src[s];
}

inline unsigned grid_of(long long N) { return (unsigned)((N + kT1Threads - 1) / kT1Threads); }

// resident CTAs per SM of a phi-pass kernel and block size
template <typename K>
int blocks_per_sm(K kernel, int threads, int smem, std::atomic<int> &cache, int *bps)
{
    int b = cache.load(std::memory_order_relaxed);
    if (!b) {
        const int rc = cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, kernel, threads, smem));
        if (rc) return rc;
        b = b > 0 ? b : 1;
        cache.store(b, std::memory_order_relaxed);
    }
    *bps = b;
    return LB_OK;
}

// z run of the phi pass: the launch's choice, else 8..64 planes, as long as
// about three waves of resident blocks remain
int phi_z_run(lb_ctx *c, long long columns, int bps, int *kzc)
{
    int z = c->z_chunk;
    if (!z) {
        int dev = 0, sms = 0;
        int rc = cuda_status(cudaGetDevice(&dev));
        if (!rc) rc = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
        if (rc) return rc;
        const long long want = 3LL * sms * bps;
        const long long zz = (long long)c->p.nz * columns / (want > 0 ? want : 1);
        z = zz < 8 ? 8 : (zz > 64 ? 64 : (int)zz);
    }
    *kzc = z > c->p.nz ? c->p.nz : z;
    return LB_OK;
}

template <typename T, bool SH, int NP, int KY>
int run_t1(lb_ctx *c, int nsteps)
{
    const auto p = make_coll<T>(c->p);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const unsigned grid = grid_of(c->N);
    const int warps = c->block_y ? c->block_y : kPhiWarps;
    const unsigned gx = (nx + kPhiOut - 1) / kPhiOut, gy = (ny + KY * warps - 1) / (KY * warps);
    static std::atomic<int> cache[kPhiMaxWarps + 1];
    int bps = 0, kzc = 0;
    int rc = blocks_per_sm(k_t1_phi<T, KY>, 32 * warps, 0, cache[warps], &bps);
    if (!rc) rc = phi_z_run(c, (long long)gx * gy, bps, &kzc);
    if (rc) return rc;
    const dim3 pgrid(gx, gy, (nz + kzc - 1) / kzc), pblock(32, warps);
    for (int t = 0; t < nsteps; t++) {
        const int a = c->buf.cur, b = 1 - a;
        cudaError_t e = launch_pdl(k_t1_collide<T, SH, NP>, grid, kT1Threads, c->stream, (const T *)c->buf.f[a],
                                   (T *)c->buf.g[a], (T *)c->buf.f[b], p, nx, ny, nz, c->S);
        if (e == cudaSuccess)
            e = launch_pdl(k_t1_phi<T, KY>, pgrid, pblock, c->stream, (const T *)c->buf.g[a], (T *)c->buf.g[b], nx,
                           ny, nz, kzc, c->S);
        rc = e != cudaSuccess ? cuda_status(e) : check_launch();
        if (rc) return rc;
        c->buf.cur = b;
        c->m_valid = 1;
    }
    return LB_OK;
}

template <typename T, bool SH, int NP>
int run_t1_ky(lb_ctx *c, int nsteps)
{
    switch (c->block_x ? c->block_x : PhiTile<T>::KY) {
    case 1: return run_t1<T, SH, NP, 1>(c, nsteps);
    case 2: return run_t1<T, SH, NP, 2>(c, nsteps);
    case 4:
        if constexpr (is_df64<T>::value) return LB_ERR_INVALID;   // spills at four rows
        else return run_t1<T, SH, NP, 4>(c, nsteps);
    default: return LB_ERR_INVALID;
    }
}

}  // namespace

template <typename T, bool SH>
int run_t1_t(lb_ctx *c, int nsteps)
{
    if (c->npts == 19) return run_t1_ky<T, SH, 19>(c, nsteps);
    if (c->npts == 27) return run_t1_ky<T, SH, 27>(c, nsteps);
    return run_t1_ky<T, SH, 7>(c, nsteps);
}

template <typename T, bool SH, int NP>
void to_full(lb_ctx *c)
{
    const int cur = c->buf.cur, oth = 1 - cur;
    k_t1_copy_phi<T><<<grid_of(c->N), kT1Threads, 0, c->stream>>>((const T *)c->buf.g[cur], (T *)c->phi, c->N);
    k_t1_to_full<T, SH, NP><<<grid_of(c->N), kT1Threads, 0, c->stream>>>(
        (const T *)c->buf.f[cur], (const T *)c->phi, (const T *)c->buf.g[oth], c->m_valid,
        make_coll<T>(c->p), (T *)c->buf.g[cur], c->p.nx, c->p.ny, c->p.nz, c->S);
}

template <typename T, bool SH>
void to_full_t(lb_ctx *c)
{
    if (c->npts == 19)
        to_full<T, SH, 19>(c);
    else if (c->npts == 27)
        to_full<T, SH, 27>(c);
    else
        to_full<T, SH, 7>(c);
}

template <typename T, bool SH, int NP>
void g_rows(lb_ctx *c, int i0, int i1, double *out)
{
    const int cur = c->buf.cur, oth = 1 - cur;
    k_t1_g_state<T, SH, NP><<<grid_of(c->N), kT1Threads, 0, c->stream>>>(
        (const T *)c->buf.f[cur], (const T *)c->buf.g[cur], (const T *)c->buf.g[oth], c->m_valid,
        make_coll<T>(c->p), out, i0, i1, c->p.nx, c->p.ny, c->p.nz, c->S);
}

template <typename T, bool SH>
void g_rows_t(lb_ctx *c, int i0, int i1, double *out)
{
    if (c->npts == 19)
        g_rows<T, SH, 19>(c, i0, i1, out);
    else if (c->npts == 27)
        g_rows<T, SH, 27>(c, i0, i1, out);
    else
        g_rows<T, SH, 7>(c, i0, i1, out);
}

int taug1_validate(const lb_params &p, int block_x, int block_y, int z_chunk)
{
    if (p.tau_g != 1.0) return LB_ERR_INVALID;
    if (block_x != 0 && block_x != 1 && block_x != 2 && block_x != 4) return LB_ERR_INVALID;
    if (block_x == 4 && p.precision == LB_FP64_DF) return LB_ERR_INVALID;
    if (block_y < 0 || block_y > kPhiMaxWarps || z_chunk < 0) return LB_ERR_INVALID;
    return LB_OK;
}

int launch_step_taug1(lb_ctx *c, int nsteps)
{
    return by_precision(c, [&](auto P) { return run_t1_t<typename decltype(P)::T, decltype(P)::SH>(c, nsteps); });
}

// convert the stored state between the full and the reduced form
int taug1_convert(lb_ctx *c, int to_reduced)
{
    const int cur = c->buf.cur;
    const unsigned grid = grid_of(c->N);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    return by_precision(c, [&](auto P) {
        using T = typename decltype(P)::T;
        if (to_reduced) {
            // phi(t) into the phi scratch, then into component 0 of level cur
            k_t1_from_full<T><<<grid, kT1Threads, 0, c->stream>>>((const T *)c->buf.g[cur], (T *)c->phi, nx, ny, nz,
                                                                  c->S);
            k_t1_copy_phi<T><<<grid, kT1Threads, 0, c->stream>>>((const T *)c->phi, (T *)c->buf.g[cur], c->N);
            c->m_valid = 0;
        } else {
            // back to the full form: phi(t) into the phi scratch, then the 19
            // values of g rebuilt into the current level (the previous step's
            // moments are read from the other level)
            to_full_t<T, decltype(P)::SH>(c);
        }
        return check_launch();
    });
}

template <typename T>
__global__ void __launch_bounds__(kT1Threads) k_t1_phi_out(const T *__restrict__ phi, double *__restrict__ out,
                                                           long long N)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s < N) out[s] = double(phi[s]);
}

int taug1_phi_out(lb_ctx *c, double *out)
{
    const unsigned grid = grid_of(c->N);
    const int cur = c->buf.cur;
    return by_precision(c, [&](auto P) {
        using T = typename decltype(P)::T;
        k_t1_phi_out<T><<<grid, kT1Threads, 0, c->stream>>>((const T *)c->buf.g[cur], out, c->N);
        return check_launch();
    });
}

int taug1_g_rows(lb_ctx *c, int i0, int i1, double *out)
{
    return by_precision(c, [&](auto P) {
        g_rows_t<typename decltype(P)::T, decltype(P)::SH>(c, i0, i1, out);
        return check_launch();
    });
}

}  // namespace lbk
