// lb_fused.cu -- single-pass timestep: phi, stencil, collision and streaming
// in one kernel.
//
// The order parameter phi(x) = sum_i g_i(x) of the post-streaming state is
// the sum of 19 pulled values A_i(x - c_i); the stencil at x needs phi on the
// 6 face neighbours, i.e. pulled values up to two sites away.  A CTA owns a
// block_x x block_y tile of an x-y plane and marches through z_chunk planes
// (2.5-D blocking).  It keeps phi for planes z-1 .. z+2 over the tile plus a
// one-site ring in a 4-slot shared-memory ring buffer; each step of the march
// computes phi two planes ahead (ring sites included) and, in the same phase,
// pulls f and g for plane z, collides and writes the post-collision values at
// their own sites, so one barrier per plane separates the phases.
// Every value of f and g is read from HBM once per timestep and written once
// (76 words per site); the second pull of g and the ring sites' pulls are
// L1/L2 hits.  This replaces targetDP's flat TARGET_TLP/VVL strip-mining
// (Sec. III.C) with a tile the hardware caches can reuse.
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lb_internal.cuh"

namespace lbk {

namespace {

#ifndef LBK_FUSED_MAXT32
#define LBK_FUSED_MAXT32 512  // FP32 CTA size limit
#endif
#ifndef LBK_FUSED_MINB32
#define LBK_FUSED_MINB32 1    // FP32 CTAs per SM the register budget must allow
#endif
constexpr int kMaxThreads = LBK_FUSED_MAXT32;
constexpr int kMaxThreads64 = 256;    // FP64: more registers per thread

struct Geo {
    int nx, ny, nz;
    int bx, by, zc;      // tile extents and z-chunk length
    int tiles_x;         // tiles along x
    long long N;
    long long S;         // component stride
};

__device__ __forceinline__ int wrap_lo(int v, int n) { return v < 0 ? v + n : v; }
__device__ __forceinline__ int wrap_hi(int v, int n) { return v >= n ? v - n : v; }

// Sum of the 19 pulled g values at (x, y, zp): phi of the post-streaming state.
template <typename T>
__device__ __forceinline__ T pulled_phi(const T *__restrict__ ga, const Geo &G, int x, int y, int zp)
{
    const int X[3] = {wrap_lo(x - 1, G.nx), x, wrap_hi(x + 1, G.nx)};
    const int Y[3] = {wrap_lo(y - 1, G.ny) * G.nx, y * G.nx, wrap_hi(y + 1, G.ny) * G.nx};
    const int pl = G.nx * G.ny;
    const int Z[3] = {wrap_lo(zp - 1, G.nz) * pl, zp * pl, wrap_hi(zp + 1, G.nz) * pl};
    T g[Q];
#pragma unroll
    for (int i = 0; i < Q; i++)
        g[i] = ga[(size_t)i * G.S + (X[1 - cx(i)] + Y[1 - cy(i)] + Z[1 - cz(i)])];
    return sum19(g);
}

template <typename T, bool SH>
__global__ void __launch_bounds__(sizeof(T) == 8 ? kMaxThreads64 : kMaxThreads,
                                  sizeof(T) == 8 ? 1 : LBK_FUSED_MINB32) k_fused(const T *__restrict__ fa, const T *__restrict__ ga,
                                                       T *__restrict__ fb, T *__restrict__ gb,
                                                       Coll<T> p, Geo G)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *ring = reinterpret_cast<T *>(smem_raw);
    const int pw = G.bx + 2;                    // padded row width
    const int psz = pw * (G.by + 2);            // padded plane size

    const int tile = blockIdx.x;
    const int x0 = (tile % G.tiles_x) * G.bx;
    const int y0 = (tile / G.tiles_x) * G.by;
    const int z0 = blockIdx.y * G.zc;
    const int ex = min(G.bx, G.nx - x0);
    const int ey = min(G.by, G.ny - y0);
    const int ez = min(G.zc, G.nz - z0);

    const int lx = threadIdx.x, ly = threadIdx.y;
    const int tid = ly * G.bx + lx;
    const int nthr = G.bx * G.by;
    const bool active = lx < ex && ly < ey;
    const int x = x0 + lx, y = y0 + ly;
    const int nhalo = 2 * (ex + ey);

    // phi of the ring sites of plane zp into ring slot `slot`
    auto ring_phi = [&](int zp, T *pl) {
        for (int h = tid; h < nhalo; h += nthr) {
            int hx, hy;
            if (h < ex) { hx = h; hy = -1; }
            else if (h < 2 * ex) { hx = h - ex; hy = ey; }
            else if (h < 2 * ex + ey) { hx = -1; hy = h - 2 * ex; }
            else { hx = ex; hy = h - 2 * ex - ey; }
            const int gx = wrap_hi(wrap_lo(x0 + hx, G.nx), G.nx);
            const int gy = wrap_hi(wrap_lo(y0 + hy, G.ny), G.ny);
            pl[(hy + 1) * pw + hx + 1] = pulled_phi(ga, G, gx, gy, zp);
        }
    };
    const int c0 = (ly + 1) * pw + lx + 1;

    // ring slot of plane z0 - 1 + m is m % 4; prologue: planes z0-1, z0, z0+1
    for (int m = 0; m < 3; m++) {
        int zp = z0 - 1 + m;
        zp = zp < 0 ? zp + G.nz : (zp >= G.nz ? zp - G.nz : zp);
        zp = zp >= G.nz ? zp - G.nz : zp;
        T *pl = ring + m * psz;
        if (active) pl[c0] = pulled_phi(ga, G, x, y, zp);
        ring_phi(zp, pl);
    }
    __syncthreads();

    const int X[3] = {wrap_lo(x - 1, G.nx), x, wrap_hi(x + 1, G.nx)};
    const int Y[3] = {wrap_lo(y - 1, G.ny) * G.nx, y * G.nx, wrap_hi(y + 1, G.ny) * G.nx};
    const int plane = G.nx * G.ny;

    // one barrier per plane: phi of plane z+2 and the collision of plane z
    // are computed in the same phase (their loads are in flight together)
    for (int k = 0; k < ez; k++) {
        const int z = z0 + k;
        const bool ahead = k + 1 < ez;                 // plane z+1 is collided next
        int z2 = z + 2;
        z2 = z2 >= G.nz ? z2 - G.nz : z2;
        z2 = z2 >= G.nz ? z2 - G.nz : z2;
        T *pn = ring + ((k + 3) & 3) * psz;
        if (ahead) ring_phi(z2, pn);
        if (active) {
            const T phn = ahead ? pulled_phi(ga, G, x, y, z2) : T(0);
            const T *cm = ring + (k & 3) * psz;
            const T *cc = ring + ((k + 1) & 3) * psz;
            const T *cp = ring + ((k + 2) & 3) * psz;
            const T ph = cc[c0];
            const T xp = cc[c0 + 1], xm = cc[c0 - 1], yp = cc[c0 + pw], ym = cc[c0 - pw];
            const T zp = cp[c0], zm = cm[c0];
            const T dx = T(0.5) * (xp - xm), dy = T(0.5) * (yp - ym), dz = T(0.5) * (zp - zm);
            const T lap = ((xp + xm) + (yp + ym)) + (zp + zm) - T(6) * ph;

            const int Z[3] = {wrap_lo(z - 1, G.nz) * plane, z * plane, wrap_hi(z + 1, G.nz) * plane};
            T f[Q], g[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const size_t o = (size_t)i * G.S + (X[1 - cx(i)] + Y[1 - cy(i)] + Z[1 - cz(i)]);
                f[i] = fa[o];
                g[i] = ga[o];
            }
            collide<T, SH>(p, f, g, ph, dx, dy, dz, lap);
            const size_t s = (size_t)(X[1] + Y[1] + Z[1]);
#pragma unroll
            for (int i = 0; i < Q; i++) {
                store(fb + (size_t)i * G.S + s, f[i]);
                store(gb + (size_t)i * G.S + s, g[i]);
            }
            if (ahead) pn[c0] = phn;
        }
        __syncthreads();
    }
}

void defaults(int precision, int &bx, int &by, int &zc)
{
    if (bx == 0) bx = 32;
    if (by == 0) by = precision == LB_FP64 ? 4 : 8;
    if (zc == 0) zc = 32;
}

template <typename T, bool SH>
int run(lb_ctx *c, int nsteps)
{
    Geo G;
    G.nx = c->p.nx;
    G.ny = c->p.ny;
    G.nz = c->p.nz;
    G.N = c->N;
    G.S = c->S;
    int bx = c->block_x, by = c->block_y, zc = c->z_chunk;
    defaults(c->p.precision, bx, by, zc);
    if ((G.nz + zc - 1) / zc > 65535) zc = (G.nz + 65534) / 65535;   // grid.y limit
    G.bx = bx;
    G.by = by;
    G.zc = zc;
    G.tiles_x = (G.nx + bx - 1) / bx;
    const int tiles_y = (G.ny + by - 1) / by;
    const dim3 grid((unsigned)(G.tiles_x * tiles_y), (unsigned)((G.nz + zc - 1) / zc));
    const dim3 block((unsigned)bx, (unsigned)by);
    const size_t shm = 4 * (size_t)(bx + 2) * (by + 2) * sizeof(T);
    const auto p = make_coll<T>(c->p);
    for (int t = 0; t < nsteps; t++) {
        const int a = c->buf.cur, b = 1 - a;
        k_fused<T, SH><<<grid, block, shm, c->stream>>>((const T *)c->buf.f[a], (const T *)c->buf.g[a],
                                                        (T *)c->buf.f[b], (T *)c->buf.g[b], p, G);
        const int rc = check_launch();
        if (rc) return rc;
        c->buf.cur = b;
    }
    return LB_OK;
}

}  // namespace

int fused_validate(int precision, int block_x, int block_y, int z_chunk)
{
    defaults(precision, block_x, block_y, z_chunk);
    if (block_x % 32 != 0 || block_x > 512) return LB_ERR_INVALID;
    const int maxt = precision == LB_FP64 ? kMaxThreads64 : kMaxThreads;
    if (block_y < 1 || block_x * block_y > maxt) return LB_ERR_INVALID;
    if (z_chunk < 1 || z_chunk > 65535) return LB_ERR_INVALID;
    return LB_OK;
}

int launch_step_fused(lb_ctx *c, int nsteps)
{
    const int rc = fused_validate(c->p.precision, c->block_x, c->block_y, c->z_chunk);
    if (rc) return rc;
    return c->p.precision == LB_FP64 ? run<double, false>(c, nsteps) : run<float, true>(c, nsteps);
}

}  // namespace lbk
