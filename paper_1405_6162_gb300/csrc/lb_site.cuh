// lb_site.cuh -- per-site pieces of the pull timestep shared by the
// one-lattice kernels and the batched persistent kernel.
#pragma once

#include "d3q19.cuh"

namespace lbk {

// Periodic neighbourhood of site s: X[k], Y[k], Z[k] are the coordinates
// x + k - 1 (wrapped), pre-multiplied by the row and plane strides.
struct Nbr {
    int X[3], Y[3], Z[3];
    __device__ __forceinline__ Nbr(int s, int nx, int ny, int nz)
    {
        const int x = s % nx;
        const int r = s / nx;
        const int y = r % ny;
        const int z = r / ny;
        X[0] = (x == 0 ? nx : x) - 1; X[1] = x; X[2] = (x + 1 == nx) ? 0 : x + 1;
        Y[0] = ((y == 0 ? ny : y) - 1) * nx; Y[1] = y * nx; Y[2] = ((y + 1 == ny) ? 0 : y + 1) * nx;
        const int pl = nx * ny;
        Z[0] = ((z == 0 ? nz : z) - 1) * pl; Z[1] = z * pl; Z[2] = ((z + 1 == nz) ? 0 : z + 1) * pl;
    }
    __device__ __forceinline__ int at(int ox, int oy, int oz) const
    {
        return X[ox + 1] + Y[oy + 1] + Z[oz + 1];
    }
    // site the pull of direction i reads from: x - c_i
    __device__ __forceinline__ int src(int i) const { return at(-cx(i), -cy(i), -cz(i)); }
};

// The phi stencil of NP points: 7 = nearest faces, d_a phi = (phi(x + e_a) -
// phi(x - e_a))/2, lap phi = sum of the 6 faces - 6 phi(x); 19 / 27 =
// the isotropic lattice-weighted differences over the D3Q19 / D3Q27
// neighbourhoods, d_a phi = 3 sum_c W_c c_a phi(x + c) and
// lap phi = 6 sum_c W_c (phi(x + c) - phi(x)), with W the D3Q19 weights
// (1/18 faces, 1/36 edges) or the D3Q27 ones (2/27, 1/54, 1/216 corners).
// Loads T, computes in R.
template <int NP, typename R, typename T>
__device__ __forceinline__ void stencil_np(const T *__restrict__ phi, const Nbr &n, R ph,
                                           R &dx, R &dy, R &dz, R &lap)
{
    static_assert(NP == 7 || NP == 19 || NP == 27, "stencil of 7, 19 or 27 points");
    if constexpr (NP == 7) {
        const R xp = R(phi[n.at(1, 0, 0)]), xm = R(phi[n.at(-1, 0, 0)]);
        const R yp = R(phi[n.at(0, 1, 0)]), ym = R(phi[n.at(0, -1, 0)]);
        const R zp = R(phi[n.at(0, 0, 1)]), zm = R(phi[n.at(0, 0, -1)]);
        dx = half(xp - xm);
        dy = half(yp - ym);
        dz = half(zp - zm);
        lap = ((xp + xm) + (yp + ym)) + (zp + zm) - R(6) * ph;
    } else {
        // per weight class k (1 faces, 2 edges, 3 corners): sum of phi and the
        // signed sums sum c_a phi
        R sum[4] = {}, da[4] = {}, db[4] = {}, dc[4] = {};
#pragma unroll
        for (int a = -1; a <= 1; a++)
#pragma unroll
            for (int b = -1; b <= 1; b++)
#pragma unroll
                for (int c = -1; c <= 1; c++) {
                    const int k = a * a + b * b + c * c;
                    if (k == 0 || (NP == 19 && k == 3)) continue;
                    const R v = R(phi[n.at(a, b, c)]);
                    sum[k] += v;
                    if (a) da[k] += a > 0 ? v : -v;
                    if (b) db[k] += b > 0 ? v : -v;
                    if (c) dc[k] += c > 0 ? v : -v;
                }
        if constexpr (NP == 19) {
            const R gf = R(1.0 / 6.0), ge = R(1.0 / 12.0);
            dx = gf * da[1] + ge * da[2];
            dy = gf * db[1] + ge * db[2];
            dz = gf * dc[1] + ge * dc[2];
            lap = R(1.0 / 3.0) * sum[1] + R(1.0 / 6.0) * sum[2] - R(4) * ph;
        } else {
            const R gf = R(2.0 / 9.0), ge = R(1.0 / 18.0), gc = R(1.0 / 72.0);
            dx = gf * da[1] + ge * da[2] + gc * da[3];
            dy = gf * db[1] + ge * db[2] + gc * db[3];
            dz = gf * dc[1] + ge * dc[2] + gc * dc[3];
            lap = R(4.0 / 9.0) * sum[1] + R(1.0 / 9.0) * sum[2] + R(1.0 / 36.0) * sum[3] - R(38.0 / 9.0) * ph;
        }
    }
}

// the 7-point stencil in the storage type
template <typename T>
__device__ __forceinline__ void stencil(const T *__restrict__ phi, const Nbr &n, T ph,
                                        T &dx, T &dy, T &dz, T &lap)
{
    stencil_np<7, T>(phi, n, ph, dx, dy, dz, lap);
}

// phi = sum of the 19 pulled g values at the site of n (component stride S)
template <typename T>
__device__ __forceinline__ T phi_site(const T *__restrict__ ga, const Nbr &n, long long S)
{
    T g[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) g[i] = ga[(size_t)i * S + n.src(i)];
    return sum19(g);
}

// Pull f and g to site s, collide with the NP-point phi stencil, write the
// post-collision values at s.
template <typename T, bool SH, int NP = 7>
__device__ __forceinline__ void collide_site(const T *__restrict__ fa, const T *__restrict__ ga,
                                             const T *__restrict__ phi, T *__restrict__ fb,
                                             T *__restrict__ gb, const Coll<T> &p, const Nbr &n, long long s,
                                             long long S)
{
    T f[Q], g[Q];
    const T ph = phi[s];
    T dx, dy, dz, lap;
    // the 27-point stencil first, so that its temporaries are dead before the
    // 38 distribution values arrive (measured: +7 % for it in FP32, -2 % for
    // the 19-point one, which stays after the loads)
    if constexpr (NP == 27) stencil_np<NP, T>(phi, n, ph, dx, dy, dz, lap);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const size_t o = (size_t)i * S + n.src(i);
        f[i] = fa[o];
        g[i] = ga[o];
    }
    if constexpr (NP != 27) stencil_np<NP, T>(phi, n, ph, dx, dy, dz, lap);
    collide<T, SH>(p, f, g, ph, dx, dy, dz, lap);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        fb[(size_t)i * S + s] = f[i];
        gb[(size_t)i * S + s] = g[i];
    }
}

}  // namespace lbk
