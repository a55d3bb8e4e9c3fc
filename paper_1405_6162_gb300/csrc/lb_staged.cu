// lb_staged.cu -- single-pass timestep with asynchronous plane staging.
//
// Same tile / z-march decomposition as lb_fused.cu, but the pulled values of
// each plane are not loaded into registers: every thread issues cp.async
// copies of its site's 38 pulled values (and ring sites' 19 pulled g values)
// straight into one of three shared-memory plane buffers.  While plane z is
// collided from its buffer, the copies of planes z+1 and z+2 are in flight,
// so the memory system always holds two planes of requests regardless of
// register pressure.  The pulled g of a plane serves both phi (ring included)
// and the collision, so g is read once per timestep.
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lb_internal.cuh"

namespace lbk {

namespace {

constexpr int kStagedMaxThreads = 512;

struct SGeo {
    int nx, ny, nz;
    int bx, by, zc;
    int tiles_x;
    long long N;
    long long S;         // component stride
};

__device__ __forceinline__ int wrap_lo(int v, int n) { return v < 0 ? v + n : v; }
__device__ __forceinline__ int wrap_hi(int v, int n) { return v >= n ? v - n : v; }

template <int BYTES>
__device__ __forceinline__ void cp_async(void *smem, const void *gmem)
{
    const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(s), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory"); }

// Shared-memory layout of one plane buffer (T elements):
//   f[19][nt], g[19][nt]: pulled values of the tile's sites (nt = bx*by)
//   h[19][nh]:            pulled g of the ring sites (nh = 2*(bx+by))
struct Layout {
    int nt, nh, buf;   // elements per array / per buffer
    int ring;          // one padded phi plane
};

__host__ __device__ inline Layout layout_of(int bx, int by)
{
    Layout L;
    L.nt = bx * by;
    L.nh = 2 * (bx + by);
    L.buf = 2 * Q * L.nt + Q * L.nh;
    L.ring = (bx + 2) * (by + 2);
    return L;
}

template <typename T>
size_t smem_bytes(int bx, int by)
{
    const Layout L = layout_of(bx, by);
    return (size_t)(3 * L.buf + 3 * L.ring) * sizeof(T);
}

template <typename T, bool SH>
__global__ void __launch_bounds__(kStagedMaxThreads, 1) k_staged(const T *__restrict__ fa, const T *__restrict__ ga,
                                                                  T *__restrict__ fb, T *__restrict__ gb,
                                                                  Coll<T> p, SGeo G)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const Layout Lo = layout_of(G.bx, G.by);
    T *bufs = reinterpret_cast<T *>(smem_raw);
    T *ring = bufs + 3 * Lo.buf;
    const int pw = G.bx + 2;

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

    const int X[3] = {wrap_lo(x - 1, G.nx), x, wrap_hi(x + 1, G.nx)};
    const int Y[3] = {wrap_lo(y - 1, G.ny) * G.nx, y * G.nx, wrap_hi(y + 1, G.ny) * G.nx};

    // ring site h -> tile-local coordinates (hx, hy)
    auto ring_xy = [&](int h, int &hx, int &hy) {
        if (h < ex) { hx = h; hy = -1; }
        else if (h < 2 * ex) { hx = h - ex; hy = ey; }
        else if (h < 2 * ex + ey) { hx = -1; hy = h - 2 * ex; }
        else { hx = ex; hy = h - 2 * ex - ey; }
    };

    // queue the copies of plane zp (wrapped) into buffer b
    auto issue = [&](int zp, int b, bool with_f) {
        T *B = bufs + b * Lo.buf;
        const int Z[3] = {wrap_lo(zp - 1, G.nz) * plane, zp * plane, wrap_hi(zp + 1, G.nz) * plane};
        if (active) {
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const size_t o = (size_t)i * G.S + (X[1 - cx(i)] + Y[1 - cy(i)] + Z[1 - cz(i)]);
                cp_async<sizeof(T)>(B + Q * Lo.nt + i * Lo.nt + tid, ga + o);
                if (with_f) cp_async<sizeof(T)>(B + i * Lo.nt + tid, fa + o);
            }
        }
        for (int h = tid; h < nhalo; h += nthr) {
            int hx, hy;
            ring_xy(h, hx, hy);
            const int gx = wrap_hi(wrap_lo(x0 + hx, G.nx), G.nx);
            const int gy = wrap_hi(wrap_lo(y0 + hy, G.ny), G.ny);
            const int HX[3] = {wrap_lo(gx - 1, G.nx), gx, wrap_hi(gx + 1, G.nx)};
            const int HY[3] = {wrap_lo(gy - 1, G.ny) * G.nx, gy * G.nx, wrap_hi(gy + 1, G.ny) * G.nx};
#pragma unroll
            for (int i = 0; i < Q; i++) {
                const size_t o = (size_t)i * G.S + (HX[1 - cx(i)] + HY[1 - cy(i)] + Z[1 - cz(i)]);
                cp_async<sizeof(T)>(B + 2 * Q * Lo.nt + i * Lo.nh + h, ga + o);
            }
        }
    };

    // phi of the plane held in buffer b (tile + ring) into ring slot b
    auto phi_from = [&](int b) {
        const T *B = bufs + b * Lo.buf;
        T *R = ring + b * Lo.ring;
        if (active) {
            T g[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) g[i] = B[Q * Lo.nt + i * Lo.nt + tid];
            R[(ly + 1) * pw + lx + 1] = sum19(g);
        }
        for (int h = tid; h < nhalo; h += nthr) {
            int hx, hy;
            ring_xy(h, hx, hy);
            T g[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) g[i] = B[2 * Q * Lo.nt + i * Lo.nh + h];
            R[(hy + 1) * pw + hx + 1] = sum19(g);
        }
    };

    // buffer / ring slot of plane z0 + k - 1 is k % 3
    issue(wrap_lo(z0 - 1, G.nz), 0, false);
    cp_async_commit();
    issue(z0, 1, true);
    cp_async_commit();
    issue(wrap_hi(z0 + 1, G.nz), 2, 1 < ez);
    cp_async_commit();
    cp_async_wait<2>();
    __syncthreads();
    phi_from(0);
    cp_async_wait<1>();
    __syncthreads();
    phi_from(1);
    __syncthreads();

    for (int k = 0; k < ez; k++) {
        const int z = z0 + k;
        // plane z+2 is needed for phi if z+2 <= z0+ez, for f if z+2 < z0+ez
        if (k + 2 <= ez) {
            int zp = z + 2;
            zp = zp >= G.nz ? zp - G.nz : zp;
            zp = zp >= G.nz ? zp - G.nz : zp;
            issue(zp, k % 3, k + 2 < ez);
        }
        cp_async_commit();
        cp_async_wait<1>();
        __syncthreads();
        phi_from((k + 2) % 3);
        __syncthreads();
        if (active) {
            const T *cm = ring + (k % 3) * Lo.ring;
            const T *cc = ring + ((k + 1) % 3) * Lo.ring;
            const T *cp = ring + ((k + 2) % 3) * Lo.ring;
            const int c0 = (ly + 1) * pw + lx + 1;
            const T ph = cc[c0];
            const T xp = cc[c0 + 1], xm = cc[c0 - 1], yp = cc[c0 + pw], ym = cc[c0 - pw];
            const T zp = cp[c0], zm = cm[c0];
            const T dx = T(0.5) * (xp - xm), dy = T(0.5) * (yp - ym), dz = T(0.5) * (zp - zm);
            const T lap = ((xp + xm) + (yp + ym)) + (zp + zm) - T(6) * ph;
            const T *B = bufs + ((k + 1) % 3) * Lo.buf;
            T f[Q], g[Q];
#pragma unroll
            for (int i = 0; i < Q; i++) {
                f[i] = B[i * Lo.nt + tid];
                g[i] = B[Q * Lo.nt + i * Lo.nt + tid];
            }
            collide<T, SH>(p, f, g, ph, dx, dy, dz, lap);
            const size_t s = (size_t)(X[1] + Y[1] + z * plane);
#pragma unroll
            for (int i = 0; i < Q; i++) {
                store(fb + (size_t)i * G.S + s, f[i]);
                store(gb + (size_t)i * G.S + s, g[i]);
            }
        }
        __syncthreads();
    }
    cp_async_wait<0>();
}

void staged_defaults(int precision, int &bx, int &by, int &zc)
{
    if (bx == 0) bx = 32;
    if (by == 0) by = precision == LB_FP64 ? 4 : 8;
    if (zc == 0) zc = 64;
}

template <typename T, bool SH>
int run_staged(lb_ctx *c, int nsteps)
{
    SGeo G;
    G.nx = c->p.nx;
    G.ny = c->p.ny;
    G.nz = c->p.nz;
    G.N = c->N;
    G.S = c->S;
    int bx = c->block_x, by = c->block_y, zc = c->z_chunk;
    staged_defaults(c->p.precision, bx, by, zc);
    if ((G.nz + zc - 1) / zc > 65535) zc = (G.nz + 65534) / 65535;
    G.bx = bx;
    G.by = by;
    G.zc = zc;
    G.tiles_x = (G.nx + bx - 1) / bx;
    const int tiles_y = (G.ny + by - 1) / by;
    const dim3 grid((unsigned)(G.tiles_x * tiles_y), (unsigned)((G.nz + zc - 1) / zc));
    const dim3 block((unsigned)bx, (unsigned)by);
    const size_t shm = smem_bytes<T>(bx, by);
    int rc = cuda_status(cudaFuncSetAttribute(k_staged<T, SH>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    if (rc) return rc;
    const auto p = make_coll<T>(c->p);
    for (int t = 0; t < nsteps; t++) {
        const int a = c->buf.cur, b = 1 - a;
        k_staged<T, SH><<<grid, block, shm, c->stream>>>((const T *)c->buf.f[a], (const T *)c->buf.g[a],
                                                         (T *)c->buf.f[b], (T *)c->buf.g[b], p, G);
        rc = check_launch();
        if (rc) return rc;
        c->buf.cur = b;
    }
    return LB_OK;
}

}  // namespace

int staged_validate(int precision, int block_x, int block_y, int z_chunk)
{
    staged_defaults(precision, block_x, block_y, z_chunk);
    if (block_x % 32 != 0 || block_x > 512) return LB_ERR_INVALID;
    if (block_y < 1 || block_x * block_y > kStagedMaxThreads) return LB_ERR_INVALID;
    if (z_chunk < 1 || z_chunk > 65535) return LB_ERR_INVALID;
    const size_t shm = precision == LB_FP64 ? smem_bytes<double>(block_x, block_y)
                                            : smem_bytes<float>(block_x, block_y);
    if (shm > 227 * 1024) return LB_ERR_INVALID;
    return LB_OK;
}

int launch_step_staged(lb_ctx *c, int nsteps)
{
    const int rc = staged_validate(c->p.precision, c->block_x, c->block_y, c->z_chunk);
    if (rc) return rc;
    return c->p.precision == LB_FP64 ? run_staged<double, false>(c, nsteps) : run_staged<float, true>(c, nsteps);
}

}  // namespace lbk
