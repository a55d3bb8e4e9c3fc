// lb_lag.cu -- single-pass timestep with a lagged phi / collision pipeline.
//
// Sites are cut into blocks of kLagBlock consecutive indices (one CTA each).
// The CTA holding ticket c (tickets are taken from a global counter when the
// CTA starts, so a lower ticket always belongs to a CTA that has already
// started) computes phi = sum of the 19 pulled g values for block c and, in
// the same phase, collides block c - D; it publishes block c's phi at its
// end.  D exceeds the distance in blocks
// between a site and its farthest stencil neighbour (one plane up), so every
// phi a collision needs was produced by a CTA with a lower ticket; completion
// is published per plane with a counter and awaited with a time-bounded spin
// (on timeout the CTA records an error flag and returns).  Each CTA issues
// one release fence (after its phi stores) and one acquire fence (after its
// wait), both by a single thread behind a CTA barrier.  Between the two
// uses of a g value lie only about D blocks of traffic (~16 MB at 256^3), so
// the collision's g reads hit L2: DRAM traffic stays near the 76 words per
// site of the algorithm while every thread keeps the simple one-site,
// barrier-free access pattern of a plain pull kernel.
//
// The lattice's first plane wraps onto the last, so blocks touching plane 0
// are collided last (collision order b = (q + b0) mod nblocks).
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lb_internal.cuh"

namespace lbk {

namespace {

struct LGeo {
    int nx, ny, nz;
    long long N, S;
    long long plane;          // nx * ny
    long long nblocks;        // ceil(N / kLagBlock)
    long long D;              // lag in blocks
    long long b0;             // blocks touching plane 0
    unsigned long long ticket_base;
    unsigned long long target;   // plane counter value meaning "done this launch"
    long long timeout_ns;
};

__device__ __forceinline__ unsigned long long global_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

template <typename T>
__device__ __forceinline__ T ldcg(const T *p) { return __ldcg(p); }

__device__ __forceinline__ void coords(long long s, const LGeo &G, int &x, int &y, int &z)
{
    const long long r = s / G.nx;
    x = (int)(s - r * G.nx);
    z = (int)(r / G.ny);
    y = (int)(r - (long long)z * G.ny);
}

__device__ __forceinline__ unsigned long long load_relaxed(const unsigned long long *p)
{
    unsigned long long v;
    asm volatile("ld.relaxed.gpu.global.u64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
    return v;
}

// Periodic neighbourhood of site s, pre-multiplied by the row/plane strides.
struct LNbr {
    int X[3];
    long long Y[3], Z[3];
    __device__ __forceinline__ LNbr(long long s, const LGeo &G)
    {
        int x, y, z;
        coords(s, G, x, y, z);
        X[0] = x == 0 ? G.nx - 1 : x - 1; X[1] = x; X[2] = x + 1 == G.nx ? 0 : x + 1;
        Y[0] = (long long)(y == 0 ? G.ny - 1 : y - 1) * G.nx; Y[1] = (long long)y * G.nx;
        Y[2] = (long long)(y + 1 == G.ny ? 0 : y + 1) * G.nx;
        Z[0] = (z == 0 ? G.nz - 1 : z - 1) * G.plane; Z[1] = z * G.plane;
        Z[2] = (z + 1 == G.nz ? 0 : z + 1) * G.plane;
    }
    __device__ __forceinline__ long long src(int i) const { return X[1 - cx(i)] + Y[1 - cy(i)] + Z[1 - cz(i)]; }
};

template <typename T, bool SH>
__global__ void __launch_bounds__(kLagBlock) k_lag(const T *__restrict__ fa, const T *__restrict__ ga,
                                                   T *__restrict__ fb, T *__restrict__ gb, T *phi,
                                                   Coll<T> p, LGeo G, unsigned long long *ticket,
                                                   unsigned long long *plane_done, unsigned int *err)
{
    __shared__ long long s_c;
    __shared__ int s_fail;
    if (threadIdx.x == 0) {
        s_c = (long long)(atomicAdd(ticket, 1ULL) - G.ticket_base);
        s_fail = 0;
    }
    __syncthreads();
    const long long c = s_c;
    const long long q = c - G.D;
    long long b = q + G.b0;
    if (b >= G.nblocks) b -= G.nblocks;
    const bool produce = c < G.nblocks, consume = q >= 0;

    // wait until every plane the collision of block b reads phi from is done
    if (consume && threadIdx.x == 0) {
        const long long first = b * kLagBlock;
        const long long last = min(first + kLagBlock, G.N) - 1;
        const long long p0 = first / G.plane, p1 = last / G.plane;
        const unsigned long long t0 = global_ns();
        int fail = (*(volatile unsigned int *)err) != 0;   // an earlier wait already gave up
        for (long long k = p0 - 1; k <= p1 + 1 && k - (p0 - 1) < G.nz && !fail; k++) {
            const long long pl = k < 0 ? k + G.nz : (k >= G.nz ? k - G.nz : k);
            while (load_relaxed(plane_done + pl) < G.target) {
                if ((long long)(global_ns() - t0) > G.timeout_ns) {
                    atomicOr(err, 1u);
                    fail = 1;
                    break;
                }
                __nanosleep(64);
            }
        }
        // acquire: the phi reads below are ordered after the counts seen
        asm volatile("fence.acq_rel.gpu;" ::: "memory");
        s_fail = fail;
    }
    __syncthreads();

    // phi of block c and the collision of block b in one phase: the 19 phi
    // loads and the 38 + 7 collision loads of a thread are in flight together
    const long long sp = c * kLagBlock + threadIdx.x;
    const long long sb = b * kLagBlock + threadIdx.x;
    const bool do_phi = produce && sp < G.N;
    const bool do_col = consume && !s_fail && sb < G.N;
    T phv = T(0);
    if (do_phi) {
        const LNbr n(sp, G);
        T g[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) g[i] = ga[(size_t)i * G.S + n.src(i)];
        phv = sum19(g);
    }
    if (do_col) {
        const LNbr n(sb, G);
        // phi was written during this launch by other CTAs: read it from L2
        const long long sc = n.X[1] + n.Y[1] + n.Z[1];
        const T ph = ldcg(phi + sc);
        const T xp = ldcg(phi + (n.X[2] + n.Y[1] + n.Z[1])), xm = ldcg(phi + (n.X[0] + n.Y[1] + n.Z[1]));
        const T yp = ldcg(phi + (n.X[1] + n.Y[2] + n.Z[1])), ym = ldcg(phi + (n.X[1] + n.Y[0] + n.Z[1]));
        const T zp = ldcg(phi + (n.X[1] + n.Y[1] + n.Z[2])), zm = ldcg(phi + (n.X[1] + n.Y[1] + n.Z[0]));
        T f[Q], g[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) {
            const size_t o = (size_t)i * G.S + n.src(i);
            f[i] = fa[o];
            g[i] = ga[o];
        }
        const T dx = T(0.5) * (xp - xm), dy = T(0.5) * (yp - ym), dz = T(0.5) * (zp - zm);
        const T lap = ((xp + xm) + (yp + ym)) + (zp + zm) - T(6) * ph;
        collide<T, SH>(p, f, g, ph, dx, dy, dz, lap);
#pragma unroll
        for (int i = 0; i < Q; i++) {
            store(fb + (size_t)i * G.S + sc, f[i]);
            store(gb + (size_t)i * G.S + sc, g[i]);
        }
    }
    if (do_phi) phi[sp] = phv;

    // publish block c: the barrier orders every thread's phi store before
    // thread 0's release fence (fences are cumulative), then the counts
    if (produce) {
        __syncthreads();
        if (threadIdx.x == 0) {
            asm volatile("fence.acq_rel.gpu;" ::: "memory");
            const long long first = c * kLagBlock;
            const long long last = min(first + kLagBlock, G.N) - 1;
            for (long long pl = first / G.plane; pl <= last / G.plane; pl++) {
                const long long lo = max(first, pl * G.plane), hi = min(last, (pl + 1) * G.plane - 1);
                atomicAdd(plane_done + pl, (unsigned long long)(hi - lo + 1));
            }
        }
    }
}

template <typename T, bool SH>
int run_lag(lb_ctx *c, int nsteps)
{
    LGeo G;
    G.nx = c->p.nx;
    G.ny = c->p.ny;
    G.nz = c->p.nz;
    G.N = c->N;
    G.S = c->S;
    G.plane = (long long)c->p.nx * c->p.ny;
    G.nblocks = (c->N + kLagBlock - 1) / kLagBlock;
    const long long bpp = (G.plane + kLagBlock - 1) / kLagBlock;   // blocks per plane (rounded up)
    G.b0 = bpp;
    const long long slack = c->z_chunk > 0 ? c->z_chunk : kLagSlack;
    G.D = 3 * bpp + 4 + slack;
    if (G.D > G.nblocks) G.D = G.nblocks;
    G.timeout_ns = c->wait_timeout_ns;
    const long long grid = G.nblocks + G.D;
    if (grid > 0x7fffffffLL) return LB_ERR_INVALID;
    const auto p = make_coll<T>(c->p);
    // every launch starts from zeroed counters (a stream-ordered memset), so
    // a launch is self-contained and can be captured in a graph and replayed
    G.ticket_base = 0;
    G.target = (unsigned long long)G.plane + c->lag_target_skew;
    const size_t cbytes = (size_t)(G.nz + 1) * sizeof(unsigned long long);
    for (int t = 0; t < nsteps; t++) {
        const int a = c->buf.cur, b = 1 - a;
        int rc = cuda_status(cudaMemsetAsync(c->lag_counters, 0, cbytes, c->stream));
        if (rc) return rc;
        k_lag<T, SH><<<(unsigned)grid, kLagBlock, 0, c->stream>>>(
            (const T *)c->buf.f[a], (const T *)c->buf.g[a], (T *)c->buf.f[b], (T *)c->buf.g[b], (T *)c->phi, p, G,
            c->lag_counters, c->lag_counters + 1, c->err_flag);
        rc = check_launch();
        if (rc) return rc;
        c->buf.cur = b;
    }
    return LB_OK;
}

}  // namespace

int lag_validate(int block_x, int block_y, int z_chunk)
{
    if ((block_x != 0 && block_x != kLagBlock) || (block_y != 0 && block_y != 1)) return LB_ERR_INVALID;
    if (z_chunk < 0 || z_chunk > (1 << 20)) return LB_ERR_INVALID;
    return LB_OK;
}

int launch_step_lag(lb_ctx *c, int nsteps)
{
    const int rc = lag_validate(c->block_x, c->block_y, c->z_chunk);
    if (rc) return rc;
    return c->p.precision == LB_FP64 ? run_lag<double, false>(c, nsteps) : run_lag<float, true>(c, nsteps);
}

}  // namespace lbk
