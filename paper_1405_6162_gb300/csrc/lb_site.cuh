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

template <typename T>
__device__ __forceinline__ void stencil(const T *__restrict__ phi, const Nbr &n, T ph,
                                        T &dx, T &dy, T &dz, T &lap)
{
    const T xp = phi[n.at(1, 0, 0)], xm = phi[n.at(-1, 0, 0)];
    const T yp = phi[n.at(0, 1, 0)], ym = phi[n.at(0, -1, 0)];
    const T zp = phi[n.at(0, 0, 1)], zm = phi[n.at(0, 0, -1)];
    dx = T(0.5) * (xp - xm);
    dy = T(0.5) * (yp - ym);
    dz = T(0.5) * (zp - zm);
    lap = ((xp + xm) + (yp + ym)) + (zp + zm) - T(6) * ph;
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

// Pull f and g to site s, collide with the phi stencil, write the
// post-collision values at s.
template <typename T, bool SH>
__device__ __forceinline__ void collide_site(const T *__restrict__ fa, const T *__restrict__ ga,
                                             const T *__restrict__ phi, T *__restrict__ fb,
                                             T *__restrict__ gb, const Coll<T> &p, const Nbr &n, long long s,
                                             long long S)
{
    T f[Q], g[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) {
        const size_t o = (size_t)i * S + n.src(i);
        f[i] = fa[o];
        g[i] = ga[o];
    }
    const T ph = phi[s];
    T dx, dy, dz, lap;
    stencil(phi, n, ph, dx, dy, dz, lap);
    collide<T, SH>(p, f, g, ph, dx, dy, dz, lap);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        fb[(size_t)i * S + s] = f[i];
        gb[(size_t)i * S + s] = g[i];
    }
}

}  // namespace lbk
