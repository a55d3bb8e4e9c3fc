// lb_slab.cu -- single-pass timestep, phi pass and collision pass per z-slab.
//
// A CTA owns a block_x x block_y tile of the x-y plane and a slab of z_chunk
// planes.  Phase 1 computes phi (sum of the 19 pulled g values) for every
// plane of the slab plus one plane above and below, over the tile and a
// one-site ring, into shared memory.  After one barrier, phase 2 collides the
// slab plane by plane with one thread per site and no further barriers,
// exactly like a plain pull kernel, taking the stencil from shared memory.
// Phase 2 reads the same g values phase 1 just read; with slabs a few planes
// deep the slabs of all resident CTAs fit in the 129 MB L2, so g comes from
// HBM once per timestep and the DRAM traffic stays near the 76 words per site
// of the algorithm, without the phi buffer pass of the two-pass form.
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lb_internal.cuh"

namespace lbk {

namespace {

#ifndef LBK_SLAB_MAXT32
#define LBK_SLAB_MAXT32 512   // FP32 CTA size limit
#endif
#ifndef LBK_SLAB_MINB32
#define LBK_SLAB_MINB32 1     // FP32 CTAs per SM the register budget must allow
#endif
constexpr int kSlabMaxThreads = LBK_SLAB_MAXT32;
constexpr int kSlabMaxThreads64 = 256;

struct BGeo {
    int nx, ny, nz;
    int bx, by, zc;
    int tiles_x;
    long long S;
};

__device__ __forceinline__ int wrap_lo(int v, int n) { return v < 0 ? v + n : v; }
__device__ __forceinline__ int wrap_hi(int v, int n) { return v >= n ? v - n : v; }

template <typename T>
__device__ __forceinline__ T pulled_phi(const T *__restrict__ ga, const BGeo &G, int x, int y, int zp)
{
    const int X[3] = {wrap_lo(x - 1, G.nx), x, wrap_hi(x + 1, G.nx)};
    const int Y[3] = {wrap_lo(y - 1, G.ny) * G.nx, y * G.nx, wrap_hi(y + 1, G.ny) * G.nx};
    const int pl = G.nx * G.ny;
    const int Z[3] = {wrap_lo(zp - 1, G.nz) * pl, zp * pl, wrap_hi(zp + 1, G.nz) * pl};
    T g[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) g[i] = ga[(size_t)i * G.S + (X[1 - cx(i)] + Y[1 - cy(i)] + Z[1 - cz(i)])];
    return sum19(g);
}

template <typename T, bool SH>
__global__ void __launch_bounds__(sizeof(T) == 8 ? kSlabMaxThreads64 : kSlabMaxThreads,
                                  sizeof(T) == 8 ? 1 : LBK_SLAB_MINB32)
k_slab(const T *__restrict__ fa, const T *__restrict__ ga, T *__restrict__ fb, T *__restrict__ gb,
       Coll<T> p, BGeo G)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *phs = reinterpret_cast<T *>(smem_raw);   // [zc + 2][by + 2][bx + 2]
    const int pw = G.bx + 2;
    const int psz = pw * (G.by + 2);

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
    const int plane = G.nx * G.ny;

    // phase 1: phi of planes z0-1 .. z0+ez (slot k holds plane z0 + k - 1)
    for (int k = 0; k < ez + 2; k++) {
        int zp = z0 + k - 1;
        zp = zp < 0 ? zp + G.nz : (zp >= G.nz ? zp - G.nz : zp);
        T *pl = phs + k * psz;
        if (active) pl[(ly + 1) * pw + lx + 1] = pulled_phi(ga, G, x, y, zp);
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
    }
    __syncthreads();
    if (!active) return;

    // phase 2: collide every plane of the slab
    const int X[3] = {wrap_lo(x - 1, G.nx), x, wrap_hi(x + 1, G.nx)};
    const int Y[3] = {wrap_lo(y - 1, G.ny) * G.nx, y * G.nx, wrap_hi(y + 1, G.ny) * G.nx};
    const int c0 = (ly + 1) * pw + lx + 1;
    for (int k = 0; k < ez; k++) {
        const int z = z0 + k;
        const T *cm = phs + k * psz;
        const T *cc = cm + psz;
        const T *cp = cc + psz;
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
    }
}

void slab_defaults(int precision, int &bx, int &by, int &zc)
{
    if (bx == 0) bx = 32;
    if (by == 0) by = precision == LB_FP64 ? 4 : 8;
    if (zc == 0) zc = 8;
}

size_t slab_smem(int precision, int bx, int by, int zc)
{
    return (size_t)(zc + 2) * (bx + 2) * (by + 2) * (precision == LB_FP64 ? 8 : 4);
}

template <typename T, bool SH>
int run_slab(lb_ctx *c, int nsteps)
{
    BGeo G;
    G.nx = c->p.nx;
    G.ny = c->p.ny;
    G.nz = c->p.nz;
    G.S = c->S;
    int bx = c->block_x, by = c->block_y, zc = c->z_chunk;
    slab_defaults(c->p.precision, bx, by, zc);
    if ((G.nz + zc - 1) / zc > 65535) return LB_ERR_INVALID;
    G.bx = bx;
    G.by = by;
    G.zc = zc;
    G.tiles_x = (G.nx + bx - 1) / bx;
    const int tiles_y = (G.ny + by - 1) / by;
    const dim3 grid((unsigned)(G.tiles_x * tiles_y), (unsigned)((G.nz + zc - 1) / zc));
    const dim3 block((unsigned)bx, (unsigned)by);
    const size_t shm = slab_smem(c->p.precision, bx, by, zc);
    int rc = cuda_status(cudaFuncSetAttribute(k_slab<T, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    if (rc) return rc;
    const auto p = make_coll<T>(c->p);
    for (int t = 0; t < nsteps; t++) {
        const int a = c->buf.cur, b = 1 - a;
        k_slab<T, SH><<<grid, block, shm, c->stream>>>((const T *)c->buf.f[a], (const T *)c->buf.g[a],
                                                       (T *)c->buf.f[b], (T *)c->buf.g[b], p, G);
        rc = check_launch();
        if (rc) return rc;
        c->buf.cur = b;
    }
    return LB_OK;
}

}  // namespace

int slab_validate(int precision, int block_x, int block_y, int z_chunk)
{
    slab_defaults(precision, block_x, block_y, z_chunk);
    const int maxt = precision == LB_FP64 ? kSlabMaxThreads64 : kSlabMaxThreads;
    if (block_x % 32 != 0 || block_x > 512) return LB_ERR_INVALID;
    if (block_y < 1 || block_x * block_y > maxt) return LB_ERR_INVALID;
    if (z_chunk < 1 || z_chunk > 65535) return LB_ERR_INVALID;
    if (slab_smem(precision, block_x, block_y, z_chunk) > 227 * 1024) return LB_ERR_INVALID;
    return LB_OK;
}

int launch_step_slab(lb_ctx *c, int nsteps)
{
    const int rc = slab_validate(c->p.precision, c->block_x, c->block_y, c->z_chunk);
    if (rc) return rc;
    return c->p.precision == LB_FP64 ? run_slab<double, false>(c, nsteps) : run_slab<float, true>(c, nsteps);
}

}  // namespace lbk
