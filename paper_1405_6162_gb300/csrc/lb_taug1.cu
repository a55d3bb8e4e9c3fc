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

#include "d3q19.cuh"
#include "lb_internal.cuh"
#include "lb_site.cuh"

namespace lbk {

namespace {

constexpr int kT1Threads = 256;

// a source site's moments expanded for geq: base by c^2 (0, 1, 2), 3 phi, 9/2 phi, u
template <typename T>
struct Eq {
    T b0, b1, b2, a3, a45, ux, uy, uz;
};

template <typename T>
__device__ __forceinline__ Eq<T> make_eq(T phi, T gmh, T ux, T uy, T uz)
{
    Eq<T> e;
    const T u2 = ux * ux + uy * uy + uz * uz;
    e.b1 = phi - T(1.5) * phi * u2;
    e.b0 = e.b1 - gmh;
    e.b2 = e.b1 + gmh;
    e.a3 = T(3) * phi;
    e.a45 = T(4.5) * phi;
    e.ux = ux;
    e.uy = uy;
    e.uz = uz;
    return e;
}

template <typename T>
__device__ __forceinline__ T gmh_of(T phi, T mu, T gamma)
{
    return T(4.5) * (gamma * mu - phi * T(1.0 / 3.0));
}

// c_i . u with the zero components left out; i a literal after inlining
template <typename T>
__device__ __forceinline__ T cdot(int i, T ux, T uy, T uz)
{
    T r = cx(i) > 0 ? ux : -ux;
    if (cx(i) == 0) r = cy(i) > 0 ? uy : -uy;
    else if (cy(i) != 0) r = cy(i) > 0 ? r + uy : r - uy;
    if (cx(i) == 0 && cy(i) == 0) r = cz(i) > 0 ? uz : -uz;
    else if (cz(i) != 0) r = cz(i) > 0 ? r + uz : r - uz;
    return r;
}

// geq_i from expanded moments; i a literal after inlining
template <typename T>
__device__ __forceinline__ T geq_eq(int i, const Eq<T> &e)
{
    const int c2 = cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i);
    if (c2 == 0) {
        if constexpr (sizeof(T) == 4) {
            // the float weights sum to 1 + e1 and their (c^2 - 1) moment is e2
            // instead of 0 (e1, e2 from the rounded values); the rest term
            // removes the bias e1 P + e2 gmh they would give sum_i geq_i
            constexpr double w0f = double(float(1.0 / 3.0)), w1f = double(float(1.0 / 18.0)),
                             w2f = double(float(1.0 / 36.0));
            constexpr float e1 = float(w0f + 6.0 * w1f + 12.0 * w2f - 1.0);
            constexpr float e2 = float(12.0 * w2f - w0f);
            return T(weight(0)) * e.b0 - (e1 * e.b1 + e2 * (e.b1 - e.b0));
        }
        return T(weight(0)) * e.b0;
    }
    const T cu = cdot(i, e.ux, e.uy, e.uz);
    const T base = c2 == 1 ? e.b1 : e.b2;
    return T(weight(i)) * (base + cu * (e.a3 + e.a45 * cu));
}

// the quad (gmh, u) of a site: one vector access
template <typename T>
struct Quad;
template <>
struct Quad<float> {
    static __device__ __forceinline__ void load(const float *__restrict__ q, long long s, float (&v)[4])
    {
        const float4 a = reinterpret_cast<const float4 *>(q)[s];
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
    }
    static __device__ __forceinline__ void store(float *__restrict__ q, long long s, float a, float b, float c,
                                                 float d)
    {
        reinterpret_cast<float4 *>(q)[s] = make_float4(a, b, c, d);
    }
};
template <>
struct Quad<double> {
    static __device__ __forceinline__ void load(const double *__restrict__ q, long long s, double (&v)[4])
    {
        const double2 a = reinterpret_cast<const double2 *>(q)[2 * s], b = reinterpret_cast<const double2 *>(q)[2 * s + 1];
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    }
    static __device__ __forceinline__ void store(double *__restrict__ q, long long s, double a, double b, double c,
                                                 double d)
    {
        reinterpret_cast<double2 *>(q)[2 * s] = make_double2(a, b);
        reinterpret_cast<double2 *>(q)[2 * s + 1] = make_double2(c, d);
    }
};

// the quads start at component 1 (S is a multiple of 64 elements, so they are aligned)
template <typename T>
__device__ __forceinline__ const T *quads(const T *g, long long S) { return g + S; }
template <typename T>
__device__ __forceinline__ T *quads(T *g, long long S) { return g + S; }

// moments of site src stored in the reduced form
template <typename T>
__device__ __forceinline__ Eq<T> load_eq(const T *__restrict__ g, long long S, long long src)
{
    T v[4];
    Quad<T>::load(quads(g, S), src, v);
    return make_eq(g[src], v[0], v[1], v[2], v[3]);
}

template <typename T, bool SH, int NP>
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
    stencil_np<NP, T>(phi, n, ph, dx, dy, dz, lap);
    // the general collision's f part; g's result is its equilibrium, kept as moments
    T ux, uy, uz, mu;
    collide_f<T, SH>(p, f, ph, dx, dy, dz, lap, ux, uy, uz, mu);
#pragma unroll
    for (int i = 0; i < Q; i++) fb[(size_t)i * S + s] = f[i];
    Quad<T>::store(quads(ga, S), s, gmh_of(ph, mu, p.gamma), ux, uy, uz);
}

constexpr int kPhiWarps = 4;   // warps per block, stacked in y
constexpr int kPhiOut = 30;    // output columns per warp

#ifndef LBK_T1_KY32
#define LBK_T1_KY32 1
#endif
#ifndef LBK_T1_KY64
#define LBK_T1_KY64 2
#endif
template <typename T>
struct PhiTile {
    static constexpr int KY = sizeof(T) == 8 ? LBK_T1_KY64 : LBK_T1_KY32;   // y rows per lane
};

__device__ __forceinline__ int wrap_up(int v, int n)
{
    while (v >= n) v -= n;   // v < 2n + 32: a few iterations at most
    return v;
}

template <typename T, int KY>
__global__ void __launch_bounds__(32 * kPhiWarps) k_t1_phi(const T *__restrict__ ga, T *__restrict__ gb, int nx,
                                                            int ny, int nz, int kzc, long long S)
{
    const int lane = threadIdx.x;
    const int y0 = (blockIdx.y * kPhiWarps + threadIdx.y) * KY;
    if (y0 >= ny) return;   // uniform over the warp
    const int z0 = blockIdx.z * kzc;
    const int nzc = min(kzc, nz - z0);   // output planes z0 .. z0 + nzc - 1
    const int xu = blockIdx.x * kPhiOut + lane - 1;   // unwrapped column, -1 .. nx + 30
    const int x = wrap_up(xu + nx, nx);
    const bool out_x = lane >= 1 && lane <= kPhiOut && xu < nx;
    const long long plane = (long long)nx * ny;
    int yoff[KY + 2];
#pragma unroll
    for (int k = 0; k < KY + 2; k++) yoff[k] = wrap_up(y0 - 1 + k + ny, ny) * nx;
    // partial sums of output plane oz live in slot oz mod 3
    T acc[3][KY], acc_r[3][KY], acc_l[3][KY];
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
        for (int a = 0; a < KY; a++) acc[q][a] = acc_r[q][a] = acc_l[q][a] = T(0);
    // raw moments of the next source plane, loaded one plane ahead
    int zr = wrap_up(z0 - 1 + nz, nz);   // source plane of step j: z0 + j - 1
    const T *q0 = quads(ga, S);
    T nxt[KY + 2][5];
#pragma unroll
    for (int r = 0; r < KY + 2; r++) {
        const long long o = x + zr * plane + yoff[r];
        T v[4];
        Quad<T>::load(q0, o, v);
        nxt[r][0] = ga[o], nxt[r][1] = v[0], nxt[r][2] = v[1], nxt[r][3] = v[2], nxt[r][4] = v[3];
    }
    for (int j0 = 0; j0 < nzc + 2; j0 += 3) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int j = j0 + k;
            if (j >= nzc + 2) break;   // uniform over the block
            T cur[KY + 2][5];
#pragma unroll
            for (int r = 0; r < KY + 2; r++)
#pragma unroll
                for (int m = 0; m < 5; m++) cur[r][m] = nxt[r][m];
            zr = zr + 1 == nz ? 0 : zr + 1;
            const long long zo = zr * plane;   // one plane past the last is still in range
#pragma unroll
            for (int r = 0; r < KY + 2; r++) {
                const long long o = x + zo + yoff[r];
                T v[4];
                Quad<T>::load(q0, o, v);
                nxt[r][0] = ga[o], nxt[r][1] = v[0], nxt[r][2] = v[1], nxt[r][3] = v[2], nxt[r][4] = v[3];
            }
#pragma unroll
            for (int ry = -1; ry <= KY; ry++) {
                const T *c5 = cur[ry + 1];
                const Eq<T> e = make_eq(c5[0], c5[1], c5[2], c5[3], c5[4]);
#pragma unroll
                for (int i = 0; i < Q; i++) {
                    const int oy = ry + cy(i);
                    if (oy < 0 || oy >= KY) continue;
                    const int q = (k + 2 + cz(i)) % 3;   // slot of output plane j - 1 + c_z
                    const T v = geq_eq(i, e);
                    if (cx(i) == 0)
                        acc[q][oy] += v;
                    else if (cx(i) > 0)
                        acc_r[q][oy] += v;   // to column x + 1
                    else
                        acc_l[q][oy] += v;   // to column x - 1
                }
            }
            // output plane j - 2 (slot (k + 1) mod 3) is complete
            const int qd = (k + 1) % 3;
            const int oz = j - 2;
#pragma unroll
            for (int a = 0; a < KY; a++) {
                const T from_left = __shfl_up_sync(0xffffffffu, acc_r[qd][a], 1);
                const T from_right = __shfl_down_sync(0xffffffffu, acc_l[qd][a], 1);
                if (out_x && oz >= 0 && y0 + a < ny)
                    gb[x + yoff[a + 1] + (z0 + oz) * plane] = acc[qd][a] + (from_left + from_right);
                acc[qd][a] = acc_r[qd][a] = acc_l[qd][a] = T(0);
            }
        }
    }
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

template <typename T, bool SH, int NP>
int run_t1(lb_ctx *c, int nsteps)
{
    const auto p = make_coll<T>(c->p);
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const unsigned grid = grid_of(c->N);
    constexpr int KY = PhiTile<T>::KY;
    const unsigned gx = (nx + kPhiOut - 1) / kPhiOut, gy = (ny + KY * kPhiWarps - 1) / (KY * kPhiWarps);
    // z runs of 8..64 planes: as long as about three waves of resident blocks remain
    static int per_sm[2] = {0, 0};
    int &bps = per_sm[sizeof(T) == 8];
    if (!bps) {
        int b = 0;
        const int rc1 = cuda_status(
            cudaOccupancyMaxActiveBlocksPerMultiprocessor(&b, k_t1_phi<T, KY>, 32 * kPhiWarps, 0));
        if (rc1) return rc1;
        bps = b > 0 ? b : 1;
    }
    int dev = 0, sms = 0;
    int rc0 = cuda_status(cudaGetDevice(&dev));
    if (!rc0) rc0 = cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (rc0) return rc0;
    const long long want = 3LL * sms * bps;
    int kzc = (int)((long long)nz * gx * gy / (want > 0 ? want : 1));
    kzc = kzc < 8 ? 8 : (kzc > 64 ? 64 : kzc);
    if (kzc > nz) kzc = nz;
    const dim3 pgrid(gx, gy, (nz + kzc - 1) / kzc);
    const dim3 pblock(32, kPhiWarps);
    for (int t = 0; t < nsteps; t++) {
        const int a = c->buf.cur, b = 1 - a;
        k_t1_collide<T, SH, NP><<<grid, kT1Threads, 0, c->stream>>>((const T *)c->buf.f[a], (T *)c->buf.g[a],
                                                                (T *)c->buf.f[b], p, nx, ny, nz, c->S);
        k_t1_phi<T, KY><<<pgrid, pblock, 0, c->stream>>>((const T *)c->buf.g[a], (T *)c->buf.g[b], nx, ny, nz, kzc,
                                                          c->S);
        const int rc = check_launch();
        if (rc) return rc;
        c->buf.cur = b;
        c->m_valid = 1;
    }
    return LB_OK;
}

}  // namespace

template <typename T, bool SH>
int run_t1_t(lb_ctx *c, int nsteps)
{
    if (c->npts == 19) return run_t1<T, SH, 19>(c, nsteps);
    if (c->npts == 27) return run_t1<T, SH, 27>(c, nsteps);
    return run_t1<T, SH, 7>(c, nsteps);
}

template <typename T, bool SH, int NP>
void to_full(lb_ctx *c)
{
    const int cur = c->buf.cur, oth = 1 - cur;
    k_t1_copy_phi<T><<<grid_of(c->N), kT1Threads, 0, c->stream>>>((const T *)c->buf.g[cur], (T *)c->phi, c->N);
    k_t1_to_full<T, SH, NP><<<grid_of(c->N), kT1Threads, 0, c->stream>>>(
        (const T *)c->buf.f[cur], (const T *)c->phi, (const T *)c->buf.g[oth], c->m_valid, make_coll<T>(c->p),
        (T *)c->buf.g[cur], c->p.nx, c->p.ny, c->p.nz, c->S);
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

int launch_step_taug1(lb_ctx *c, int nsteps)
{
    return c->p.precision == LB_FP64 ? run_t1_t<double, false>(c, nsteps) : run_t1_t<float, true>(c, nsteps);
}

// convert the stored state between the full and the reduced form
int taug1_convert(lb_ctx *c, int to_reduced)
{
    const int cur = c->buf.cur;
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
    if (c->p.precision == LB_FP64)
        to_full_t<double, false>(c);
    else
        to_full_t<float, true>(c);
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
    if (c->p.precision == LB_FP64)
        g_rows_t<double, false>(c, i0, i1, out);
    else
        g_rows_t<float, true>(c, i0, i1, out);
    return check_launch();
}

}  // namespace lbk
