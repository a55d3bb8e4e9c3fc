// lb_taug1.cu -- the timestep for tau_g = 1, keeping g as its moments.
//
// With tau_g = 1 the collision of g returns its equilibrium exactly,
// g*_i = geq_i(phi, mu, u), so after streaming g_i(x, t+1) = geq_i evaluated
// with (phi, mu, u) of site x - c_i at time t, and phi(x, t+1) is the sum of
// those 19 values.  The context then keeps, instead of 19 values of g, five
// per site in the first five components of its g buffers:
//     level a: [0] phi(t)   [1] mu(t)   [2..4] u(t)
// and one step is two passes:
//   k_t1_collide  pull f, 7-point stencil of phi(t), collide f; write f* and
//                 mu(t), u(t) next to phi(t)          (19+1 r, 19+4 w words)
//   k_t1_phi      phi(x, t+1) = sum_i geq_i(phi, mu, u at x - c_i) into the
//                 other level's component 0         (~5 r, 1 w words)
// -- about 49 words per site instead of the 97 of the general two-pass step.
// The per-site arithmetic is the general collision's (the g relaxation is
// simply not needed); results agree with the general step to rounding.
//
// Flag m_valid: (mu, u) of the previous step are present.  After lb_init or
// lb_set_state only phi(t) is known; g is then reported as the equilibrium at
// each site (exact after lb_init, which starts from that equilibrium).
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lb_internal.cuh"
#include "lb_site.cuh"

namespace lbk {

namespace {

constexpr int kT1Threads = 256;

// geq_i at a site with moments (phi, Gamma mu - phi/3, u); i a literal after
// inlining
template <typename T>
__device__ __forceinline__ T geq_dir(int i, T phi, T gm, T ux, T uy, T uz)
{
    const T cu = T(cx(i)) * ux + T(cy(i)) * uy + T(cz(i)) * uz;
    const T u2 = ux * ux + uy * uy + uz * uz;
    const T c2 = T(cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i));
    return T(weight(i)) * (phi + T(3) * phi * cu + T(4.5) * (phi * cu * cu - phi * u2 * T(1.0 / 3.0) + gm * (c2 - T(1))));
}

template <typename T, bool SH>
__global__ void __launch_bounds__(kT1Threads, sizeof(T) == 8 ? 2 : 3)
k_t1_collide(const T *__restrict__ fa, T *__restrict__ ga /* level a: phi in, mu/u out */, T *__restrict__ fb,
             Coll<T> p, int nx, int ny, int nz, long long S)
{
    const long long N = (long long)nx * ny * nz;
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n(s, nx, ny, nz);
    const T *phi = ga;
    T f[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = fa[(size_t)i * S + n.src(i)];
    const T ph = phi[s];
    T dx, dy, dz, lap;
    stencil(phi, n, ph, dx, dy, dz, lap);
    // the general collision's f part; g's result is its equilibrium, kept as moments
    T g[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) g[i] = T(0);
    T R, jx, jy, jz;
    density_moments(f, R, jx, jy, jz);
    collide<T, SH>(p, f, g, ph, dx, dy, dz, lap);
#pragma unroll
    for (int i = 0; i < Q; i++) fb[(size_t)i * S + s] = f[i];
    const T rho = SH ? p.rho0 + R : R;
    const T rinv = T(1) / rho;
    ga[1 * S + s] = ph * (p.A + p.B * ph * ph) - p.kappa * lap;   // mu
    ga[2 * S + s] = jx * rinv;
    ga[3 * S + s] = jy * rinv;
    ga[4 * S + s] = jz * rinv;
}

// Moments of one site, and the equilibria of the (up to three) directions
// that share a source row, i.e. the same (c_y, c_z): c_x = 0, +1, -1.
template <typename T>
struct SrcM {
    T ph, gmh, ux, uy, uz;   // phi, 9/2 (Gamma mu - phi/3), u
};

template <typename T>
__device__ __forceinline__ SrcM<T> load_m(const T *__restrict__ ga, long long S, long long src, T gamma)
{
    SrcM<T> m;
    m.ph = ga[src];
    m.gmh = T(4.5) * (gamma * ga[S + src] - m.ph * T(1.0 / 3.0));
    m.ux = ga[2 * S + src];
    m.uy = ga[3 * S + src];
    m.uz = ga[4 * S + src];
    return m;
}

// geq for direction (cx, cy, cz) at a source with moments m:
//   w [phi (1 - 3/2 u^2) + 3 phi c.u + 9/2 phi (c.u)^2 + gmh (c^2 - 1)]
template <typename T>
__device__ __forceinline__ T geq_m(const SrcM<T> &m, int cxv, int cyv, int czv, T w)
{
    const T cu = T(cxv) * m.ux + T(cyv) * m.uy + T(czv) * m.uz;
    const T base = m.ph * (T(1) - T(1.5) * (m.ux * m.ux + m.uy * m.uy + m.uz * m.uz));
    const T c2m1 = T(cxv * cxv + cyv * cyv + czv * czv - 1);
    return w * (base + m.gmh * c2m1 + cu * (T(3) * m.ph + T(4.5) * m.ph * cu));
}

template <typename T>
__global__ void __launch_bounds__(kT1Threads) k_t1_phi(const T *__restrict__ ga, T *__restrict__ gb, Coll<T> p,
                                                        int nx, int ny, int nz, long long S)
{
    const long long N = (long long)nx * ny * nz;
    const int s0 = blockIdx.x * blockDim.x + threadIdx.x;
    const bool live = s0 < N;
    const int s = live ? s0 : (int)(N - 1);           // dead lanes mirror the last site
    const Nbr n(s, nx, ny, nz);
    const int lane = threadIdx.x & 31;
    const int x = n.X[1];
    // the lane below / above holds x - 1 / x + 1 of the same row
    const bool from_below = lane > 0 && x > 0 && live;
    const bool from_above = lane < 31 && x + 1 < nx && s0 + 1 < N;
    T acc = T(0);
    // (c_y, c_z) of the 9 source rows; dirs with that (c_y, c_z) and c_x = 0, +1, -1
#pragma unroll
    for (int r = 0; r < 9; r++) {
        const int cyv = r == 0 ? 0 : (r == 1 ? 1 : (r == 2 ? -1 : (r == 3 || r == 4 ? 0 : (r == 5 || r == 7 ? 1 : -1))));
        const int czv = r < 3 ? 0 : (r == 3 ? 1 : (r == 4 ? -1 : (r == 5 || r == 8 ? 1 : -1)));
        const bool three = r < 5;                    // rows with c_x = 0, +1, -1 (else c_x = 0 only)
        const T w0 = T(r == 0 ? 1.0 / 3.0 : (r < 5 ? 1.0 / 18.0 : 1.0 / 36.0));
        const T w1 = T(r == 0 ? 1.0 / 18.0 : 1.0 / 36.0);
        // pull: the source of direction c is x - c; own column of this row
        const long long row = (long long)n.Y[1 - cyv] + n.Z[1 - czv];
        const SrcM<T> m = load_m(ga, S, row + x, p.gamma);
        acc += geq_m(m, 0, cyv, czv, w0);
        if (three) {
            // direction (+1, cy, cz) takes its value from x - 1: computed by the lane below
            const T vp = geq_m(m, 1, cyv, czv, w1);
            const T vm = geq_m(m, -1, cyv, czv, w1);
            const T up = __shfl_up_sync(0xffffffffu, vp, 1);
            const T dn = __shfl_down_sync(0xffffffffu, vm, 1);
            acc += from_below ? up : geq_m(load_m(ga, S, row + n.X[0], p.gamma), 1, cyv, czv, w1);
            acc += from_above ? dn : geq_m(load_m(ga, S, row + n.X[2], p.gamma), -1, cyv, czv, w1);
        }
    }
    if (live) gb[s] = acc;
}

// g state of the reduced form as post-streaming FP64 rows [i0, i1):
// streamed equilibria of the previous step's moments (m_valid), else the
// equilibrium at each site from phi(t), its stencil and u from f.
template <typename T, bool SH>
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
            const int src = n.src(i);
            const double ph = double(gprev[src]), mu = double(gprev[S + src]);
            out[(size_t)(i - i0) * N + s] = geq_dir<double>(i, ph, double(p.gamma) * mu - ph / 3.0, double(gprev[2 * S + src]),
                                                            double(gprev[3 * S + src]), double(gprev[4 * S + src]));
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
    const double xp = gcur[n.at(1, 0, 0)], xm = gcur[n.at(-1, 0, 0)], yp = gcur[n.at(0, 1, 0)];
    const double ym = gcur[n.at(0, -1, 0)], zp = gcur[n.at(0, 0, 1)], zm = gcur[n.at(0, 0, -1)];
    const double lap = ((xp + xm) + (yp + ym)) + (zp + zm) - 6.0 * ph;
    const double mu = ph * (double(p.A) + double(p.B) * ph * ph) - double(p.kappa) * lap;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        if (i < i0 || i >= i1) continue;
        out[(size_t)(i - i0) * N + s] = geq_dir<double>(i, ph, double(p.gamma) * mu - ph / 3.0, jx / rho, jy / rho, jz / rho);
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
template <typename T, bool SH>
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
    const double xp = gcur[n.at(1, 0, 0)], xm = gcur[n.at(-1, 0, 0)], yp = gcur[n.at(0, 1, 0)];
    const double ym = gcur[n.at(0, -1, 0)], zp = gcur[n.at(0, 0, 1)], zm = gcur[n.at(0, 0, -1)];
    const double lap = ((xp + xm) + (yp + ym)) + (zp + zm) - 6.0 * ph;
    const double mu = ph * (double(p.A) + double(p.B) * ph * ph) - double(p.kappa) * lap;
#pragma unroll
    for (int i = 0; i < Q; i++) {
        double v;
        if (m_valid) {
            const int src = n.src(i);
            const double q = double(gprev[src]), m = double(gprev[S + src]);
            v = geq_dir<double>(i, q, double(p.gamma) * m - q / 3.0, double(gprev[2 * S + src]),
                                double(gprev[3 * S + src]), double(gprev[4 * S + src]));
        } else {
            v = geq_dir<double>(i, ph, double(p.gamma) * mu - ph / 3.0, jx / rho, jy / rho, jz / rho);
        }
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

template <typename T, bool SH>
int run_t1(lb_ctx *c, int nsteps)
{
    const auto p = make_coll<T>(c->p);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const unsigned grid = grid_of(c->N);
    for (int t = 0; t < nsteps; t++) {
        const int a = c->buf.cur, b = 1 - a;
        k_t1_collide<T, SH><<<grid, kT1Threads, 0, c->stream>>>((const T *)c->buf.f[a], (T *)c->buf.g[a],
                                                                (T *)c->buf.f[b], p, nx, ny, nz, c->S);
        k_t1_phi<T><<<grid, kT1Threads, 0, c->stream>>>((const T *)c->buf.g[a], (T *)c->buf.g[b], p, nx, ny, nz,
                                                        c->S);
        const int rc = check_launch();
        if (rc) return rc;
        c->buf.cur = b;
        c->m_valid = 1;
    }
    return LB_OK;
}

}  // namespace

int launch_step_taug1(lb_ctx *c, int nsteps)
{
    return c->p.precision == LB_FP64 ? run_t1<double, false>(c, nsteps) : run_t1<float, true>(c, nsteps);
}

// convert the stored state between the full and the reduced form
int taug1_convert(lb_ctx *c, int to_reduced)
{
    const int cur = c->buf.cur, oth = 1 - cur;
    const unsigned grid = grid_of(c->N);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    if (to_reduced) {
        // phi(t) into the phi scratch, then into component 0 of level cur
        if (c->p.precision == LB_FP64) {
            k_t1_from_full<double><<<grid, kT1Threads, 0, c->stream>>>((const double *)c->buf.g[cur], (double *)c->phi,
                                                                       nx, ny, nz, c->S);
            k_t1_copy_phi<double><<<grid, kT1Threads, 0, c->stream>>>((const double *)c->phi,
                                                                      (double *)c->buf.g[cur], c->N);
        } else {
            k_t1_from_full<float><<<grid, kT1Threads, 0, c->stream>>>((const float *)c->buf.g[cur], (float *)c->phi,
                                                                      nx, ny, nz, c->S);
            k_t1_copy_phi<float><<<grid, kT1Threads, 0, c->stream>>>((const float *)c->phi, (float *)c->buf.g[cur],
                                                                     c->N);
        }
        c->m_valid = 0;
        return check_launch();
    }
    // back to the full form: phi(t) into the phi scratch, then the 19 values
    // of g rebuilt into the current level (the previous step's moments are
    // read from the other level)
    if (c->p.precision == LB_FP64) {
        k_t1_copy_phi<double><<<grid, kT1Threads, 0, c->stream>>>((const double *)c->buf.g[cur], (double *)c->phi,
                                                                  c->N);
        k_t1_to_full<double, false><<<grid, kT1Threads, 0, c->stream>>>(
            (const double *)c->buf.f[cur], (const double *)c->phi, (const double *)c->buf.g[oth], c->m_valid,
            make_coll<double>(c->p), (double *)c->buf.g[cur], nx, ny, nz, c->S);
    } else {
        k_t1_copy_phi<float><<<grid, kT1Threads, 0, c->stream>>>((const float *)c->buf.g[cur], (float *)c->phi,
                                                                 c->N);
        k_t1_to_full<float, true><<<grid, kT1Threads, 0, c->stream>>>(
            (const float *)c->buf.f[cur], (const float *)c->phi, (const float *)c->buf.g[oth], c->m_valid,
            make_coll<float>(c->p), (float *)c->buf.g[cur], nx, ny, nz, c->S);
    }
    return check_launch();
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
    if (c->p.precision == LB_FP64)
        k_t1_phi_out<double><<<grid, kT1Threads, 0, c->stream>>>((const double *)c->buf.g[cur], out, c->N);
    else
        k_t1_phi_out<float><<<grid, kT1Threads, 0, c->stream>>>((const float *)c->buf.g[cur], out, c->N);
    return check_launch();
}

int taug1_g_rows(lb_ctx *c, int i0, int i1, double *out)
{
    const int cur = c->buf.cur, oth = 1 - cur;
    const unsigned grid = grid_of(c->N);
    if (c->p.precision == LB_FP64)
        k_t1_g_state<double, false><<<grid, kT1Threads, 0, c->stream>>>(
            (const double *)c->buf.f[cur], (const double *)c->buf.g[cur], (const double *)c->buf.g[oth], c->m_valid,
            make_coll<double>(c->p), out, i0, i1, c->p.nx, c->p.ny, c->p.nz, c->S);
    else
        k_t1_g_state<float, true><<<grid, kT1Threads, 0, c->stream>>>(
            (const float *)c->buf.f[cur], (const float *)c->buf.g[cur], (const float *)c->buf.g[oth], c->m_valid,
            make_coll<float>(c->p), out, i0, i1, c->p.nx, c->p.ny, c->p.nz, c->S);
    return check_launch();
}

}  // namespace lbk
