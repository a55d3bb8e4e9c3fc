// lb_adjoint.cu -- reverse mode of the FP64 timestep (a kernel pair) and of
// the initialisation, for gradients of a loss on phi_T.
//
// States are in the ABI (post-streaming) convention, so the forward
// quantities of F(t) are local to each site.  Per reverse step:
//   k_phi_local   phi(x) = sum_i g_i(x, t)
//   k_adj_collide at x: recompute rho, j, u, mu, the stress; gather the
//                 adjoint after streaming, fs_bar_i(x) = f_bar_i(x + c_i, t+1);
//                 apply the collision's vector-Jacobian product; write
//                 f_bar(x, t), the direct part of g_bar, and the adjoints of
//                 phi, grad phi and lap phi at x; per-CTA partial dJ/dkappa
//   k_adj_stencil phi_bar(x) = local part + transposed 7-point stencils;
//                 g_bar_i(x, t) += phi_bar(x)
// The equilibrium VJP sums each opposite pair (i+, i-) once: its even part
// feeds rho and the stress, its odd part the momentum.
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lb_internal.cuh"
#include "lb_site.cuh"

namespace lbk {

namespace {

struct AdjP {
    double omega, omega_g, rho0, gamma, A, B, kappa;
};

// c of the + member of pair k (k = 0..8: faces x, y, z; edges 7, 9, 11, 13, 15, 17)
__device__ __forceinline__ int pc(int k, int a)
{
    const int ip = k < 3 ? 2 * k + 1 : 7 + 2 * (k - 3);
    return a == 0 ? cx(ip) : (a == 1 ? cy(ip) : cz(ip));
}
__device__ __forceinline__ int pplus(int k) { return k < 3 ? 2 * k + 1 : 7 + 2 * (k - 3); }
__device__ __forceinline__ double pw(int k) { return k < 3 ? 1.0 / 18.0 : 1.0 / 36.0; }

// Adjoint of (rho, j, phi, d, lap, kappa) -> (feq, geq) at one site, given
// the weights Fe_i on feq_i and Ge_i on geq_i.  INIT: rho and j are inputs
// (no adjoint flows into them).
template <bool INIT>
__device__ __forceinline__ void equilibrium_vjp(const AdjP &p, double rho, const double (&j)[3], double phi,
                                                const double (&d)[3], double lap, const double (&Fe)[Q],
                                                const double (&Ge)[Q], double &rho_b, double (&j_b)[3],
                                                double &phi_b, double (&d_b)[3], double &lap_b, double &kap_b)
{
    const double u[3] = {j[0] / rho, j[1] / rho, j[2] / rho};
    // pair sums: even parts (s) and odd parts (o)
    double Wf = Fe[0] / 3.0, Wg = Ge[0] / 3.0;
    double Tf[3][3] = {{0}}, Tg[3][3] = {{0}}, Of[3] = {0, 0, 0}, Og[3] = {0, 0, 0};
#pragma unroll
    for (int k = 0; k < 9; k++) {
        const int ip = pplus(k);
        const double w = pw(k);
        const double sf = w * (Fe[ip] + Fe[ip + 1]), of = w * (Fe[ip] - Fe[ip + 1]);
        const double sg = w * (Ge[ip] + Ge[ip + 1]), og = w * (Ge[ip] - Ge[ip + 1]);
        Wf += sf;
        Wg += sg;
#pragma unroll
        for (int a = 0; a < 3; a++) {
            const int ca = pc(k, a);
            Of[a] += of * ca;
            Og[a] += og * ca;
#pragma unroll
            for (int b = 0; b < 3; b++) {
                Tf[a][b] += sf * ca * pc(k, b);
                Tg[a][b] += sg * ca * pc(k, b);
            }
        }
    }
    // feq_i = w_i [rho + 3 c.j + 9/2 c S c - 3/2 tr S]
    double Sb[3][3], Gb[3][3];
#pragma unroll
    for (int a = 0; a < 3; a++)
#pragma unroll
        for (int b = 0; b < 3; b++) {
            Sb[a][b] = 4.5 * Tf[a][b] - (a == b ? 1.5 * Wf : 0.0);
            Gb[a][b] = 4.5 * Tg[a][b] - (a == b ? 1.5 * Wg : 0.0);
        }
    rho_b += Wf;
    double u_b[3];
#pragma unroll
    for (int a = 0; a < 3; a++) {
        j_b[a] += 3.0 * Of[a];
        u_b[a] = 3.0 * phi * Og[a];
    }
    // geq_i = w_i [phi + 3 phi c.u + 9/2 c G c - 3/2 tr G],  G = (Gamma mu - phi/3) I + phi u u
    phi_b += Wg + 3.0 * (u[0] * Og[0] + u[1] * Og[1] + u[2] * Og[2]);
    const double trG = Gb[0][0] + Gb[1][1] + Gb[2][2];
    const double mu_b = p.gamma * trG;
    double uGu = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        double Gu = 0.0;
#pragma unroll
        for (int b = 0; b < 3; b++) Gu += Gb[a][b] * u[b];
        uGu += u[a] * Gu;
        u_b[a] += 2.0 * phi * Gu;
    }
    phi_b += uGu - trG / 3.0;
    // S = pb I + kappa d d + j j / rho
    const double pb_b = Sb[0][0] + Sb[1][1] + Sb[2][2];
    double dSd = 0.0, jSj = 0.0;
#pragma unroll
    for (int a = 0; a < 3; a++) {
        double Sd = 0.0, Sj = 0.0;
#pragma unroll
        for (int b = 0; b < 3; b++) {
            Sd += Sb[a][b] * d[b];
            Sj += Sb[a][b] * j[b];
        }
        d_b[a] += 2.0 * p.kappa * Sd;
        dSd += d[a] * Sd;
        jSj += j[a] * Sj;
        if (!INIT) j_b[a] += 2.0 * Sj / rho;
    }
    kap_b += dSd;
    if (!INIT) rho_b -= jSj / (rho * rho);
    // pb = A/2 phi^2 + 3B/4 phi^4 - kappa phi lap - kappa/2 |d|^2
    const double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    phi_b += pb_b * (p.A * phi + 3.0 * p.B * phi * phi * phi - p.kappa * lap);
    lap_b -= p.kappa * phi * pb_b;
#pragma unroll
    for (int a = 0; a < 3; a++) d_b[a] -= p.kappa * d[a] * pb_b;
    kap_b -= pb_b * (phi * lap + 0.5 * dd);
    // mu = A phi + B phi^3 - kappa lap
    phi_b += mu_b * (p.A + 3.0 * p.B * phi * phi);
    lap_b -= p.kappa * mu_b;
    kap_b -= lap * mu_b;
    // u = j / rho
    if (!INIT) {
        const double uj = u_b[0] * j[0] + u_b[1] * j[1] + u_b[2] * j[2];
#pragma unroll
        for (int a = 0; a < 3; a++) j_b[a] += u_b[a] / rho;
        rho_b -= uj / (rho * rho);
    }
}

__device__ __forceinline__ double block_sum_d(double v, double *sh)
{
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double r = 0.0;
    if (threadIdx.x == 0)
        for (int w = 0; w < (int)(blockDim.x >> 5); w++) r += sh[w];
    return r;
}

constexpr int kAdjThreads = 256;

// phi(x) = sum_i g_i(x) of a post-streaming state
__global__ void __launch_bounds__(kAdjThreads) k_phi_local(const double *__restrict__ g, double *__restrict__ phi,
                                                           long long N)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    double v[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) v[i] = g[(size_t)i * N + s];
    phi[s] = sum19(v);
}

// Collision VJP per site.  INIT: the initial state (f_bar of the equilibria
// in af_in/ag_in, no streaming, phi given by phi0, j = rho0 u0).
template <bool INIT>
__global__ void __launch_bounds__(kAdjThreads) k_adj_collide(const double *__restrict__ f, const double *__restrict__ g,
                                                             const double *__restrict__ phi,
                                                             const double *__restrict__ u0,
                                                             const double *__restrict__ af_in,
                                                             const double *__restrict__ ag_in,
                                                             double *__restrict__ af_out, double *__restrict__ ag_out,
                                                             double *__restrict__ aux, double *__restrict__ kpart,
                                                             AdjP p, int nx, int ny, int nz)
{
    __shared__ double sh[kAdjThreads / 32];
    const long long N = (long long)nx * ny * nz;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    double kap_b = 0.0;
    if (s < N) {
        const Nbr n((int)s, nx, ny, nz);
        const double ph = phi[s];
        double dx, dy, dz, lap;
        stencil(phi, n, ph, dx, dy, dz, lap);
        double rho, j[3];
        if (INIT) {
            rho = p.rho0;
            j[0] = u0 ? p.rho0 * u0[s] : 0.0;
            j[1] = u0 ? p.rho0 * u0[N + s] : 0.0;
            j[2] = u0 ? p.rho0 * u0[2 * N + s] : 0.0;
        } else {
            double fv[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) fv[i] = f[(size_t)i * N + s];
            density_moments(fv, rho, j[0], j[1], j[2]);
        }
        // adjoint after the streaming transpose: value of (x + c_i) at t+1
        double Fe[Q], Ge[Q], fsb[Q], gsb[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const size_t o = (size_t)i * N + (INIT ? s : n.at(cx(i), cy(i), cz(i)));
            fsb[i] = af_in[o];
            gsb[i] = ag_in[o];
            Fe[i] = (INIT ? 1.0 : p.omega) * fsb[i];
            Ge[i] = (INIT ? 1.0 : p.omega_g) * gsb[i];
        }
        const double d[3] = {dx, dy, dz};
        double rho_b = 0.0, j_b[3] = {0.0, 0.0, 0.0}, phi_b = 0.0, d_b[3] = {0.0, 0.0, 0.0}, lap_b = 0.0;
        equilibrium_vjp<INIT>(p, rho, j, ph, d, lap, Fe, Ge, rho_b, j_b, phi_b, d_b, lap_b, kap_b);
        if (!INIT) {
#pragma unroll
            for (int i = 0; i < Q; i++) {
                af_out[(size_t)i * N + s] = (1.0 - p.omega) * fsb[i] + rho_b + (j_b[0] * cx(i) + j_b[1] * cy(i) + j_b[2] * cz(i));
                ag_out[(size_t)i * N + s] = (1.0 - p.omega_g) * gsb[i];
            }
        }
        aux[s] = phi_b;
        aux[N + s] = d_b[0];
        aux[2 * N + s] = d_b[1];
        aux[3 * N + s] = d_b[2];
        aux[4 * N + s] = lap_b;
    }
    const double tot = block_sum_d(kap_b, sh);
    if (threadIdx.x == 0) kpart[blockIdx.x] = tot;
}

// phi_bar = local part + transposed stencils; g_bar_i += phi_bar (or, for the
// initialisation, phi0_bar = phi_bar)
template <bool INIT>
__global__ void __launch_bounds__(kAdjThreads) k_adj_stencil(const double *__restrict__ aux, double *__restrict__ out,
                                                             int nx, int ny, int nz)
{
    const long long N = (long long)nx * ny * nz;
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const Nbr n((int)s, nx, ny, nz);
    const double *db0 = aux + N, *db1 = aux + 2 * N, *db2 = aux + 3 * N, *lb = aux + 4 * N;
    const int xp = n.at(1, 0, 0), xm = n.at(-1, 0, 0), yp = n.at(0, 1, 0), ym = n.at(0, -1, 0);
    const int zp = n.at(0, 0, 1), zm = n.at(0, 0, -1);
    const double pb = aux[s] + 0.5 * ((db0[xm] - db0[xp]) + (db1[ym] - db1[yp]) + (db2[zm] - db2[zp]))
                    + ((lb[xm] + lb[xp]) + (lb[ym] + lb[yp]) + (lb[zm] + lb[zp])) - 6.0 * lb[s];
    if (INIT) {
        out[s] = pb;
    } else {
#pragma unroll
        for (int i = 0; i < Q; i++) out[(size_t)i * N + s] += pb;
    }
}

// Adjoint of the read-out phi_T = sum_i g_i(T): f_bar = 0 and every
// g_bar_i = dJ/dphi_T at the same site
__global__ void __launch_bounds__(kAdjThreads) k_adj_seed(const double *__restrict__ phi_bar,
                                                          double *__restrict__ af, double *__restrict__ ag,
                                                          long long N)
{
    const long long s = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= N) return;
    const double pb = phi_bar[s];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        af[(size_t)i * N + s] = 0.0;
        ag[(size_t)i * N + s] = pb;
    }
}

// dkappa += sum of the per-CTA partials (one CTA, fixed order)
__global__ void k_adj_kappa(const double *__restrict__ kpart, int nb, double *__restrict__ dkappa)
{
    __shared__ double sh[kAdjThreads / 32];
    double v = 0.0;
    for (int b = threadIdx.x; b < nb; b += blockDim.x) v += kpart[b];
    const double tot = block_sum_d(v, sh);
    if (threadIdx.x == 0) *dkappa += tot;
}

AdjP adj_params(const lb_params &q)
{
    AdjP p;
    p.omega = 1.0 / q.tau;
    p.omega_g = 1.0 / q.tau_g;
    p.rho0 = q.rho0;
    p.gamma = q.gamma;
    p.A = q.A;
    p.B = q.B;
    p.kappa = q.kappa;
    return p;
}

}  // namespace

int adjoint_blocks(long long N) { return (int)((N + kAdjThreads - 1) / kAdjThreads); }

int launch_adjoint_step(lb_ctx *c, const double *f, const double *g, const double *af_in, const double *ag_in,
                        double *af_out, double *ag_out, double *dkappa, double *aux, double *kpart)
{
    const int nb = adjoint_blocks(c->N);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    double *phi = aux + 5 * c->N;
    k_phi_local<<<nb, kAdjThreads, 0, c->stream>>>(g, phi, c->N);
    k_adj_collide<false><<<nb, kAdjThreads, 0, c->stream>>>(f, g, phi, nullptr, af_in, ag_in, af_out, ag_out, aux,
                                                            kpart, adj_params(c->p), nx, ny, nz);
    k_adj_stencil<false><<<nb, kAdjThreads, 0, c->stream>>>(aux, ag_out, nx, ny, nz);
    k_adj_kappa<<<1, kAdjThreads, 0, c->stream>>>(kpart, nb, dkappa);
    return check_launch();
}

int launch_adjoint_seed(lb_ctx *c, const double *phi_bar, double *af, double *ag)
{
    k_adj_seed<<<adjoint_blocks(c->N), kAdjThreads, 0, c->stream>>>(phi_bar, af, ag, c->N);
    return check_launch();
}

int launch_adjoint_init(lb_ctx *c, const double *phi0, const double *u0, const double *af0, const double *ag0,
                        double *phi0_bar, double *dkappa, double *aux, double *kpart)
{
    const int nb = adjoint_blocks(c->N);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    k_adj_collide<true><<<nb, kAdjThreads, 0, c->stream>>>(nullptr, nullptr, phi0, u0, af0, ag0, nullptr, nullptr,
                                                           aux, kpart, adj_params(c->p), nx, ny, nz);
    k_adj_stencil<true><<<nb, kAdjThreads, 0, c->stream>>>(aux, phi0_bar, nx, ny, nz);
    k_adj_kappa<<<1, kAdjThreads, 0, c->stream>>>(kpart, nb, dkappa);
    return check_launch();
}

}  // namespace lbk
