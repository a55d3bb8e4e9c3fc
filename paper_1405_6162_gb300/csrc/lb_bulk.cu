// lb_bulk.cu -- single-pass timestep: whole x-rows of g staged in shared
// memory by asynchronous copies, the phi halo shared across a cluster of CTAs
// along y.
//
// One CTA owns one row y of the lattice (all nx sites, one thread per site)
// and marches through a chunk of z planes.  For output plane z the pulled
// order-parameter distribution g_i(x - c_i) of the row is 19 whole x-rows of
// the stored (post-collision) array -- component i from row y - cy_i of plane
// z - cz_i -- shifted by -cx_i inside the row.  Per plane the CTA
//
//  * copies those 19 rows into a ring of shared-memory slots ahead of use
//    (16-byte cp.async from every warp, one commit group per plane), so g is
//    read from HBM once per timestep;
//  * forms phi = sum_i g_i of the row from the slot (the phi of the
//    order-parameter pass, targetDP Sec. II.A), keeps it in a 4-plane ring and
//    pushes it into the halo rings of the CTAs that own rows y - 1 and y + 1
//    in the same cluster (asynchronous stores to distributed shared memory
//    that complete bytes of the receiving CTA's mbarrier);
//  * collides the row with f taken straight from global memory (loaded one
//    plane ahead into registers), g from its slot and phi and its 7-point
//    stencil from the rings, and writes f*, g* of the row.
//
// The cluster's outer rows have a neighbour outside the cluster: the CTA
// copies that row's 19 pulled g rows too (in the same commit group) and sums
// them with the same code as its own row, so every site's phi has the same
// bits wherever it is formed.  Every warp takes part in every role: measured
// on GB300, single warps that only issued copies or summed halo rows were
// latency-bound (~0.2 us per 1 KB row issued, ~0.8 us per halo row summed)
// and set the pace of the whole kernel.
//
// The only wait on other CTAs -- for the peers' phi rows -- is bounded (the
// context's wait timeout): a CTA that gives up sets the context's error flag,
// stops its loop once all its threads agree, lets its copies in flight land,
// and meets the other CTAs of its cluster at the final cluster barrier before
// it exits (no CTA exits while a peer may still write its shared memory).
// Shapes it cannot take (nx not a whole number of 16-byte rows, nx > 256, ny
// not a multiple of the cluster, double-float, shared memory beyond 227 KB)
// are refused by bulk_validate.
#include <cuda_runtime.h>
#include <stdint.h>

#include "d3q19.cuh"
#include "lb_internal.cuh"

namespace lbk {

namespace {

constexpr int kBulkMaxRow = 256;   // sites per row (one thread each)
constexpr int kRing = 4;           // planes held in the phi and halo-phi rings

struct BGeo {
    int nx, ny, nz;
    int zc;                 // planes per CTA
    int cy;                 // CTAs per cluster (along y)
    int ng;                 // own-row g slots (planes copied ahead = ng - 2)
    int nsl;                // local halo sides a slot holds (1, or 2 without a cluster)
    long long S;            // component stride (elements)
    long long timeout_ns;
    int stall;              // test hook: the wait for the peers' phi never completes
};

// ------------------------------------------------------------------ PTX helpers

__device__ __forceinline__ uint32_t saddr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

__device__ __forceinline__ unsigned long long now_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}

// this CTA's arrival on its own barrier, announcing `bytes` still to come
// in the current phase
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

// true once the phase of `bar` with `parity` has completed; the thread may
// sleep in hardware until then, for at most ~0.1 ms
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(100000u)
        : "memory");
    return ok != 0;
}

// One row of `bytes` (a multiple of 16) from global to this CTA's shared
// memory in 16-byte asynchronous copies by the lanes of a warp.
__device__ __forceinline__ void copy_row(uint32_t dst, const void *src, uint32_t bytes, int lane)
{
    const char *s = static_cast<const char *>(src);
    for (uint32_t off = (uint32_t)lane * 16u; off < bytes; off += 512u)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(dst + off), "l"(s + off) : "memory");
}
__device__ __forceinline__ void copies_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void copies_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
__device__ __forceinline__ void copies_drain() { asm volatile("cp.async.wait_all;" ::: "memory"); }

// this thread's copies have landed except those of its newest `pending`
// commit groups
__device__ __forceinline__ void copies_wait_pending(int pending)
{
    if (pending <= 0) copies_wait<0>();
    else if (pending == 1) copies_wait<1>();
    else if (pending == 2) copies_wait<2>();
    else if (pending == 3) copies_wait<3>();
    else if (pending == 4) copies_wait<4>();
    else if (pending == 5) copies_wait<5>();
    else copies_wait<6>();
}

__device__ __forceinline__ uint32_t map_rank(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}

// Store v into another CTA's shared memory at cluster address `addr`; the
// store completes `sizeof v` bytes of the current phase of that CTA's
// barrier at cluster address `bar` (no fence: the barrier's phase makes the
// data visible to the threads that wait on it)
__device__ __forceinline__ void st_peer(uint32_t addr, float v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b32 [%0], %1, [%2];" ::"r"(addr),
                 "r"(__float_as_uint(v)), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_peer(uint32_t addr, double v, uint32_t bar)
{
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.b64 [%0], %1, [%2];" ::"r"(addr),
                 "l"((unsigned long long)__double_as_longlong(v)), "r"(bar)
                 : "memory");
}

__device__ __forceinline__ uint32_t cluster_rank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}

__device__ __forceinline__ void cluster_sync_all()
{
    asm volatile("barrier.cluster.arrive.release;\n barrier.cluster.wait.acquire;" ::: "memory");
}

// barrier of the CTA's threads (id 1); returns whether any of them passed
// pred = true (the same answer in every thread)
__device__ __forceinline__ bool cta_sync_or(int nthreads, bool pred)
{
    uint32_t r;
    asm volatile(
        "{\n .reg .pred p, q;\n setp.ne.u32 p, %1, 0;\n bar.red.or.pred q, 1, %2, p;\n selp.u32 %0, 1, 0, q;\n}\n"
        : "=r"(r)
        : "r"((uint32_t)pred), "r"(nthreads)
        : "memory");
    return r != 0;
}

// v mod n for v in [-n, 2n) (every use: an index plus or minus one, or a
// chunk's planes z0 - 1 .. z0 + ez): no integer division
__device__ __forceinline__ int wrapm(int v, int n) { return v < 0 ? v + n : (v >= n ? v - n : v); }

// Wait (bounded) for the phase of `bar` with `parity`.  False once the
// deadline passes or another thread of the CTA has given up.
__device__ __forceinline__ bool wait_peers(uint32_t bar, uint32_t parity, long long timeout_ns, volatile int *abort)
{
    unsigned long long t0 = 0;
    while (!mbar_wait(bar, parity)) {
        if (*abort) return false;
        const unsigned long long t = now_ns();
        if (t0 == 0) {
            t0 = t;
        } else if ((long long)(t - t0) > timeout_ns) {
            *abort = 1;
            return false;
        }
    }
    return true;
}

// ------------------------------------------------------------------ shared-memory layout

struct Smem {
    size_t bars;     // halo_full[4]
    size_t flag;     // int: a wait of this CTA gave up
    size_t rtab;     // [3 * 19] long long row offsets, then [3 * 19] int plane selectors
    size_t own;      // [ng][19][nx]: pulled g rows of the own row
    size_t loc;      // [ng - 1][nsl][19][nx]: pulled g rows of the local halo rows
    size_t phi;      // [4][nx]: phi of the own row
    size_t halo;     // [4][2][nx]: phi of rows y - 1 (side 0) and y + 1 (side 1)
    size_t total;
};

__host__ __device__ inline size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

__host__ __device__ inline Smem smem_layout(int nx, int ng, int nsl, size_t esize)
{
    Smem L;
    L.bars = 0;
    L.flag = (size_t)kRing * 8;
    L.rtab = align_up(L.flag + 16, 16);
    const size_t row = (size_t)nx * esize;
    L.own = align_up(L.rtab + (size_t)3 * Q * 12, 128);
    L.loc = align_up(L.own + (size_t)ng * Q * row, 128);
    L.phi = align_up(L.loc + (size_t)(ng - 1) * nsl * Q * row, 128);
    L.halo = align_up(L.phi + (size_t)kRing * row, 128);
    L.total = align_up(L.halo + (size_t)kRing * 2 * row, 128);
    return L;
}

#ifndef LBK_BULK_MINB32
#define LBK_BULK_MINB32 2
#endif

// NXC: the row length as a compile-time constant (every shared-memory offset
// an immediate), or 0 for any row length.  LEAN: two own-row slots (ng = 2)
// and one local halo slot, refilled while the row collides; three CTAs per SM.
template <typename T, bool SH, int NXC, bool LEAN>
__global__ void __launch_bounds__(kBulkMaxRow, LEAN ? 3 : (sizeof(T) == 4 ? LBK_BULK_MINB32 : 1))
k_bulk(const T *__restrict__ fa, const T *__restrict__ ga, T *__restrict__ fb, T *__restrict__ gb, Coll<T> p,
       BGeo G, unsigned int *err_flag)
{
    extern __shared__ __align__(128) unsigned char sm[];
    const Smem L = smem_layout(NXC ? NXC : G.nx, G.ng, G.nsl, sizeof(T));
    const uint32_t halo_full = saddr(sm + L.bars);
    volatile int *abort = reinterpret_cast<volatile int *>(sm + L.flag);
    T *own = reinterpret_cast<T *>(sm + L.own);
    T *loc = reinterpret_cast<T *>(sm + L.loc);
    T *phir = reinterpret_cast<T *>(sm + L.phi);
    T *halo = reinterpret_cast<T *>(sm + L.halo);

    const int nx = NXC ? NXC : G.nx, ny = G.ny, nz = G.nz;
    const int nct = blockDim.x, nw = nct >> 5;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int y = blockIdx.x;
    const int z0 = blockIdx.y * G.zc;
    const int ez = min(G.zc, nz - z0);
    const int nplanes = ez + 2;           // phi of planes z0 - 1 .. z0 + ez: j = 0 .. ez + 1
    const int D = G.ng - 2;               // commit groups in flight beyond the one awaited
    const uint32_t rank = G.cy > 1 ? cluster_rank() : 0;
    // sides (0: row y - 1, 1: row y + 1) whose phi a peer pushes; the others
    // are formed here from copied rows
    const bool peer_lo = rank > 0, peer_hi = (int)rank + 1 < G.cy;
    const int npeer = (int)peer_lo + (int)peer_hi;
    const int nloc = 2 - npeer;
    const int loc_side0 = peer_lo ? 1 : 0;   // the first local side
    const uint32_t row_bytes = (uint32_t)(nx * sizeof(T));
    const int plane = nx * ny;

    // halo_full[(j - 1) % 4] completes the phase of collision plane j once
    // this CTA has armed it (its one arrival, announcing the bytes of the
    // peers' phi rows) and those bytes have arrived; the test hook asks for
    // a second arrival that never comes
    const uint32_t peer_bytes = (uint32_t)(npeer * nx * sizeof(T));
    if (tid == 0) {
        for (int s = 0; s < kRing; s++) mbar_init(halo_full + 8 * s, (uint32_t)(1 + G.stall));
        *abort = 0;
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        for (int j = 1; j <= kRing && j <= ez; j++) mbar_expect_tx(halo_full + 8 * (j - 1), peer_bytes);
    }
    __syncthreads();
    cluster_sync_all();   // every peer's barriers exist before any remote arrival

    // plane index j = 0 .. nplanes-1 is lattice plane z0 - 1 + j (wrapped)
    auto plane_of = [&](int j) { return wrapm(z0 - 1 + j, nz); };

    // --- copies.  Commit group s (s = 0 .. nplanes-1) holds the own rows of
    // plane s and the local halo rows of plane s - 1 (when 1 <= s - 1 <= ez).
    // Own rows of plane s go to slot s % ng; local halo rows of plane m to
    // slot m % (ng - 1).  Row list of a group: 19 own rows, then 19 per local
    // side; warp w copies rows w, w + nw, ...  rtab[r] holds row r's source
    // offset without its plane part (component and row in the plane); rcz[r]
    // holds 1 - cz of the row's component, which picks its source plane
    // p - cz among p - 1, p, p + 1 of the group's own or halo plane p.
    long long *rtab = reinterpret_cast<long long *>(sm + L.rtab);
    int *rcz = reinterpret_cast<int *>(sm + L.rtab + 8 * 3 * Q);
    for (int r = tid; r < Q * (1 + nloc); r += nct) {
        const int k = r / Q, i = r - k * Q;
        const int yr = k == 0 ? y : wrapm(y + ((k == 1 ? loc_side0 : 1) ? 1 : -1), ny);
        rtab[r] = (long long)i * G.S + (long long)wrapm(yr - cy(i), ny) * nx;
        rcz[r] = 1 - cz(i);
    }
    __syncthreads();
    auto issue_group = [&](int s) {
        if (s < nplanes) {
            const int nrows = Q + ((s - 1 >= 1 && s - 1 <= ez) ? Q * nloc : 0);
            // source planes p - cz: index 1 - cz = 0, 1, 2 is plane p - 1, p, p + 1
            // of the own plane (o) and of the halo plane (h)
            const int po = plane_of(s), ph = plane_of(s > 0 ? s - 1 : 0);
            const long long zo[3] = {(long long)wrapm(po - 1, nz) * plane, (long long)po * plane,
                                     (long long)wrapm(po + 1, nz) * plane};
            const long long zh[3] = {(long long)wrapm(ph - 1, nz) * plane, (long long)ph * plane,
                                     (long long)wrapm(ph + 1, nz) * plane};
            const uint32_t own_dst = saddr(own + (size_t)(s % G.ng) * Q * nx);
            const uint32_t loc_dst = saddr(loc + (size_t)((s > 0 ? s - 1 : 0) % (G.ng - 1)) * G.nsl * Q * nx);
            for (int r = warp; r < nrows; r += nw) {
                const int c = rcz[r];
                const long long zp = r < Q ? (c == 0 ? zo[0] : c == 1 ? zo[1] : zo[2])
                                           : (c == 0 ? zh[0] : c == 1 ? zh[1] : zh[2]);
                const uint32_t dst = r < Q ? own_dst + (uint32_t)r * row_bytes : loc_dst + (uint32_t)(r - Q) * row_bytes;
                copy_row(dst, ga + rtab[r] + zp, row_bytes, lane);
            }
        }
        copies_commit();   // one group per s, empty or not, so the counts stay uniform
    };

    const int x = tid;
    const bool active = x < nx;
    const int xc = active ? x : 0;
    const int X[3] = {xc == 0 ? nx - 1 : xc - 1, xc, xc + 1 == nx ? 0 : xc + 1};
    const int Y[3] = {wrapm(y - 1, ny) * nx, y * nx, wrapm(y + 1, ny) * nx};
    // remote halo addresses: our row is side 1 of rank - 1 and side 0 of rank + 1
    uint32_t r_lo = 0, r_hi = 0, rb_lo = 0, rb_hi = 0;
    if (peer_lo) {
        r_lo = map_rank(saddr(halo + nx + xc), rank - 1);
        rb_lo = map_rank(halo_full, rank - 1);
    }
    if (peer_hi) {
        r_hi = map_rank(saddr(halo + xc), rank + 1);
        rb_hi = map_rank(halo_full, rank + 1);
    }

    T fr[Q];
    auto load_f = [&](int z) {
        if (!active) return;
        const int Z[3] = {wrapm(z - 1, nz) * plane, z * plane, wrapm(z + 1, nz) * plane};
#pragma unroll
        for (int i = 0; i < Q; i++)
            fr[i] = fa[(size_t)i * G.S + (size_t)(unsigned)(X[1 - cx(i)] + Y[1 - cy(i)] + Z[1 - cz(i)])];
    };
    // phi = sum_i g_i(x - c_i) of the 19 rows at `rows` (one order everywhere)
    auto sum_rows = [&](const T *rows) {
        T g[Q];
#pragma unroll
        for (int i = 0; i < Q; i++) g[i] = rows[i * nx + X[1 - cx(i)]];
        return sum19(g);
    };
    // phi of plane j (own row) into the own ring and, for a collision
    // plane, into the peers' halo rings
    auto form_phi = [&](int j) {
        const bool share = j >= 1 && j <= ez;
        const int h = (j - 1) & (kRing - 1);
        if (active) {
            const T ph = sum_rows(own + (size_t)(j % G.ng) * Q * nx);
            phir[(j % kRing) * nx + x] = ph;
            if (share) {
                const uint32_t off = (uint32_t)(h * 2 * nx * sizeof(T));
                if (peer_lo) st_peer(r_lo + off, ph, rb_lo + 8 * h);
                if (peer_hi) st_peer(r_hi + off, ph, rb_hi + 8 * h);
            }
        }
    };
    // phi of the local halo rows of collision plane j into the halo ring
    auto form_local_halo = [&](int j) {
        if (!active || nloc == 0) return;
        const int h = (j - 1) & (kRing - 1);
        const T *base = loc + (size_t)(j % (G.ng - 1)) * G.nsl * Q * nx;
        halo[h * 2 * nx + loc_side0 * nx + x] = sum_rows(base);
        if (nloc == 2) halo[h * 2 * nx + nx + x] = sum_rows(base + (size_t)Q * nx);
    };

    // the g values of collision plane jc from its slot
    auto load_g = [&](int jc, T (&g)[Q]) {
        const T *gs = own + (size_t)(jc % G.ng) * Q * nx;
#pragma unroll
        for (int i = 0; i < Q; i++) g[i] = gs[i * nx + X[1 - cx(i)]];
    };
    // the collision of plane jc (index k = jc - 1 of the chunk) with its g
    auto collide_row = [&](int k, T (&g)[Q]) {
        const int jc = k + 1, jn = k + 2;
        const int hc = (jc - 1) & (kRing - 1);
        const T *pc = phir + (jc % kRing) * nx;
        const T ph = pc[x];
        const T xp = pc[X[2]], xm = pc[X[0]];
        const T ym = halo[hc * 2 * nx + x], yp = halo[hc * 2 * nx + nx + x];
        const T zp = phir[(jn % kRing) * nx + x], zm = phir[(k % kRing) * nx + x];
        const T dx = T(0.5) * (xp - xm), dy = T(0.5) * (yp - ym), dz = T(0.5) * (zp - zm);
        const T lap = ((xp + xm) + (yp + ym)) + (zp + zm) - T(6) * ph;
        collide<T, SH>(p, fr, g, ph, dx, dy, dz, lap);
        const size_t o = (size_t)(z0 + k) * plane + (size_t)y * nx + x;
        T *pf = fb + o, *pg = gb + o;
#pragma unroll
        for (int i = 0; i < Q; i++, pf += G.S, pg += G.S) {
            store(pf, fr[i]);
            store(pg, g[i]);
        }
    };
    // every thread has read the halo ring slot of plane k (collided in the
    // previous iteration): arm it for plane k + 4
    auto rearm = [&](int k) {
        if (tid == 0 && k >= 1 && k + kRing <= ez) mbar_expect_tx(halo_full + 8 * ((k - 1) & (kRing - 1)), peer_bytes);
    };
    auto wait_halo = [&](int jc) {
        if (npeer + G.stall == 0) return true;
        return wait_peers(halo_full + 8 * ((jc - 1) & (kRing - 1)), (uint32_t)(((jc - 1) / kRing) & 1), G.timeout_ns,
                          abort);
    };

    bool ok = true;
    if constexpr (!LEAN) {
        // prologue: groups 0 .. D + 1 in flight, phi of planes 0 and 1
        load_f(z0);
        for (int s = 0; s <= D + 1; s++) issue_group(s);
        copies_wait_pending(D + 1);   // group 0
        cta_sync_or(nct, false);
        form_phi(0);
        copies_wait_pending(D);       // group 1
        cta_sync_or(nct, false);
        form_phi(1);
        for (int k = 0; k < ez; k++) {
            const int jc = k + 1, jn = k + 2;   // collision plane, next phi plane
            copies_wait_pending(D - 1);         // group jn: own rows of jn, local halo rows of jc
            // the copies of group jn are visible CTA-wide, and every thread is
            // past the previous collision, so the slots of plane k are free
            if (cta_sync_or(nct, !ok || *abort)) break;
            rearm(k);
            issue_group(jn + D);
            form_phi(jn);
            form_local_halo(jc);
            // No barrier here: the collision below reads, of what this
            // iteration wrote, only the values at its own site (phi of jn, the
            // local halo of jc); the x-neighbours' phi of jn are read in the
            // next iteration, after its barrier, and the peers' halo rows
            // through their barrier.
            ok = wait_halo(jc);
            if (ok && active) {
                T g[Q];
                load_g(jc, g);
                collide_row(k, g);
            }
            if (k + 1 < ez) load_f(z0 + k + 1);
        }
    } else {
        // Two own slots and one local halo slot, so that three CTAs fit an
        // SM.  The slot of collision plane jc is free once every thread has
        // its g values in registers: the copy of plane jc + 2 goes into it
        // then and lands while the row collides.
        issue_group(0);
        copies_wait<0>();
        cta_sync_or(nct, false);
        form_phi(0);
        issue_group(1);
        copies_wait<0>();
        cta_sync_or(nct, false);
        form_phi(1);
        issue_group(2);   // into plane 0's slot, whose phi is formed
        for (int k = 0; k < ez; k++) {
            const int jc = k + 1, jn = k + 2;
            copies_wait<0>();   // group jn: own rows of jn, local halo rows of jc
            // the copies of group jn are visible CTA-wide, every thread is
            // past the previous collision
            if (cta_sync_or(nct, !ok || *abort)) break;
            rearm(k);
            load_f(z0 + k);
            form_phi(jn);
            form_local_halo(jc);
            ok = wait_halo(jc);
            T g[Q];
            load_g(jc, g);
            // every thread has its g of jc and has formed the local halo of jc:
            // jc's slot and the local halo slot take group jc + 2
            cta_sync_or(nct, false);
            issue_group(jc + 2);
            if (ok && active) collide_row(k, g);
        }
    }
    copies_drain();   // nothing in flight when the CTA exits
    if (tid == 0 && *abort) atomicExch(err_flag, 1u);
    cluster_sync_all();   // no CTA leaves while a peer may still write its shared memory
}

void bulk_defaults(int &ng, int &cy, int &zc)
{
    if (ng == 0) ng = 3;
    if (cy == 0) cy = 4;
    if (zc == 0) zc = 32;
}

}  // namespace

size_t bulk_smem_bytes(int nx, int ng, int cy, size_t esize)
{
    return smem_layout(nx, ng, cy == 1 ? 2 : 1, esize).total;
}

int bulk_validate(const lb_params &p, int block_x, int block_y, int z_chunk)
{
    int ng = block_x, cy = block_y, zc = z_chunk;
    bulk_defaults(ng, cy, zc);
    if (p.precision != LB_FP64 && p.precision != LB_FP32_SHIFTED) return LB_ERR_INVALID;
    const size_t es = p.precision == LB_FP64 ? 8 : 4;
    if (p.nx > kBulkMaxRow || ((size_t)p.nx * es) % 16 != 0) return LB_ERR_INVALID;
    if (ng < 2 || ng > 8 || (ng == 2 && p.precision != LB_FP32_SHIFTED)) return LB_ERR_INVALID;
    if (cy != 1 && cy != 2 && cy != 4 && cy != 8) return LB_ERR_INVALID;
    if (p.ny % cy != 0) return LB_ERR_INVALID;
    if (zc < 1 || (p.nz + zc - 1) / zc > 65535) return LB_ERR_INVALID;
    if (bulk_smem_bytes(p.nx, ng, cy, es) > 227 * 1024) return LB_ERR_INVALID;
    return LB_OK;
}

template <typename T, bool SH>
static int run_bulk(lb_ctx *c, int nsteps)
{
    BGeo G;
    G.nx = c->p.nx;
    G.ny = c->p.ny;
    G.nz = c->p.nz;
    int ng = c->block_x, cy = c->block_y, zc = c->z_chunk;
    bulk_defaults(ng, cy, zc);
    G.zc = zc;
    G.cy = cy;
    G.ng = ng;
    G.nsl = cy == 1 ? 2 : 1;
    G.S = c->S;
    G.timeout_ns = c->wait_timeout_ns;
    G.stall = c->lag_target_skew != 0;
    const size_t shm = bulk_smem_bytes(G.nx, G.ng, cy, sizeof(T));
    // the lean form only in FP32 (validated), so only its FP32 copies exist
    constexpr bool kLean = sizeof(T) == 4;
    auto kern = (kLean && G.ng == 2) ? (G.nx == 256 ? k_bulk<T, SH, 256, kLean> : k_bulk<T, SH, 0, kLean>)
                                     : (G.nx == 256 ? k_bulk<T, SH, 256, false> : k_bulk<T, SH, 0, false>);
    int rc = cuda_status(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)shm));
    if (rc) return rc;
    const auto p = make_coll<T>(c->p);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)G.ny, (unsigned)((G.nz + zc - 1) / zc));
    cfg.blockDim = dim3((unsigned)(32 * ((G.nx + 31) / 32)));
    cfg.dynamicSmemBytes = shm;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = (unsigned)cy;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    for (int t = 0; t < nsteps; t++) {
        const int a = c->buf.cur, b = 1 - a;
        const cudaError_t e = cudaLaunchKernelEx(&cfg, kern, (const T *)c->buf.f[a], (const T *)c->buf.g[a],
                                                 (T *)c->buf.f[b], (T *)c->buf.g[b], p, G, c->err_flag);
        rc = e != cudaSuccess ? cuda_status(e) : check_launch();
        if (rc) return rc;
        c->buf.cur = b;
    }
    return LB_OK;
}

// the shape the library default uses: 3 slots, clusters of 2, 16 planes per
// CTA (the fastest measured at 256^3 FP32-shifted on GB300), on rows of 256
// sites (eight warps a CTA; at 128^3, four warps a CTA, the two-pass step is
// faster: 17.4 against 14.2 GLUPS)
constexpr int kAutoSlots = 3, kAutoCluster = 2, kAutoPlanes = 16;

bool auto_uses_bulk(const lb_ctx *c)
{
    return c->p.precision == LB_FP32_SHIFTED && c->npts == 7 && !uses_mrt(c) && c->p.nx == kBulkMaxRow &&
           bulk_validate(c->p, kAutoSlots, kAutoCluster, kAutoPlanes) == LB_OK;
}

int launch_step_bulk_auto(lb_ctx *c, int nsteps)
{
    const int bx = c->block_x, by = c->block_y, zc = c->z_chunk;
    c->block_x = kAutoSlots;
    c->block_y = kAutoCluster;
    c->z_chunk = kAutoPlanes;
    const int rc = c->p.precision == LB_FP64 ? run_bulk<double, false>(c, nsteps) : run_bulk<float, true>(c, nsteps);
    c->block_x = bx;
    c->block_y = by;
    c->z_chunk = zc;
    return rc;
}

int launch_step_bulk(lb_ctx *c, int nsteps)
{
    const int rc = bulk_validate(c->p, c->block_x, c->block_y, c->z_chunk);
    if (rc) return rc;
    return c->p.precision == LB_FP64 ? run_bulk<double, false>(c, nsteps) : run_bulk<float, true>(c, nsteps);
}

}  // namespace lbk
