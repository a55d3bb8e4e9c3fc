// lb_masked.cu -- masked copies between the lattice and compact arrays: the
// sites whose mask byte is non-zero, in site order (targetDP Sec. III.B,
// copyFromTargetMasked / copyToTargetMasked).
//
// A stream compaction: per-CTA counts of selected sites (16 mask bytes per
// thread, one vector load when aligned), one CTA's exclusive scan of the
// counts (offsets[nb] = total), then the list of selected sites, each thread
// placing its 16 sites after the CTA offset and the counts of the threads
// before it (a block scan).  The gather / scatter kernels then run one thread per selected
// site, so every thread has work whatever the mask's density.  The order is
// the site order, so the result is unique and bit-exact.
#include <cuda_runtime.h>

#include "d3q19.cuh"
#include "lb_internal.cuh"
#include "lb_moments.cuh"
#include "lb_site.cuh"

namespace lbk {

namespace {

constexpr int kMaskThreads = 512;               // threads of the one-CTA scan
constexpr int kMaskWarps = kMaskThreads / 32;
constexpr unsigned kFull = 0xffffffffu;
static_assert(kMaskThreads % 32 == 0 && kMaskWarps <= 32, "CTA of whole warps, at most 32");

constexpr int kTileThreads = 256;                 // compaction CTAs
constexpr int kPerThread = 16;                    // mask bytes per thread
constexpr int kTile = kTileThreads * kPerThread;  // sites per compaction CTA

// the 16 mask bytes of a thread as non-zero flags (bit k = site base + k);
// one 16-byte load when the chunk is aligned and inside the mask
template <bool VEC>
__device__ __forceinline__ unsigned mask_bits(const unsigned char *__restrict__ mask, long long base, long long N)
{
    unsigned bits = 0;
    if (VEC && base + kPerThread <= N) {
        const uint4 v = *reinterpret_cast<const uint4 *>(mask + base);
        const unsigned w[4] = {v.x, v.y, v.z, v.w};
#pragma unroll
        for (int q = 0; q < 4; q++)
#pragma unroll
            for (int k = 0; k < 4; k++)
                if ((w[q] >> (8 * k)) & 0xffu) bits |= 1u << (4 * q + k);
    } else {
#pragma unroll
        for (int k = 0; k < kPerThread; k++)
            if (base + k < N && mask[base + k] != 0) bits |= 1u << k;
    }
    return bits;
}

template <bool VEC>
__global__ void __launch_bounds__(kTileThreads) k_mask_count(const unsigned char *__restrict__ mask, long long N,
                                                             int *__restrict__ counts)
{
    __shared__ int warp_cnt[kTileThreads / 32];
    const long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kPerThread;
    int c = __popc(mask_bits<VEC>(mask, base, N));
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) c += __shfl_down_sync(0xffffffffu, c, o);
    if ((threadIdx.x & 31) == 0) warp_cnt[threadIdx.x >> 5] = c;
    __syncthreads();
    if (threadIdx.x == 0) {
        int t = 0;
#pragma unroll
        for (int w = 0; w < kTileThreads / 32; w++) t += warp_cnt[w];
        counts[blockIdx.x] = t;
    }
}

// inclusive scan over a warp
__device__ __forceinline__ int warp_incl(int x)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int y = __shfl_up_sync(kFull, x, o);
        if (lane >= o) x += y;
    }
    return x;
}

// offsets[i] = counts[0] + ... + counts[i - 1] for i < nb, offsets[nb] = total
__global__ void __launch_bounds__(kMaskThreads) k_mask_scan(const int *__restrict__ counts, int nb,
                                                            int *__restrict__ offsets)
{
    __shared__ int warp_tot[32];
    __shared__ int carry_s;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    if (threadIdx.x == 0) carry_s = 0;
    __syncthreads();
    for (int base = 0; base < nb; base += kMaskThreads) {
        const int i = base + threadIdx.x;
        const int v = i < nb ? counts[i] : 0;
        const int x = warp_incl(v);
        if (lane == 31) warp_tot[warp] = x;
        __syncthreads();
        if (warp == 0) {
            const int t = warp_incl(lane < kMaskWarps ? warp_tot[lane] : 0);
            if (lane < kMaskWarps) warp_tot[lane] = t;
        }
        __syncthreads();
        const int carry = carry_s;
        if (i < nb) offsets[i] = carry + (warp ? warp_tot[warp - 1] : 0) + x - v;
        __syncthreads();
        if (threadIdx.x == 0) carry_s = carry + warp_tot[kMaskWarps - 1];
        __syncthreads();
    }
    if (threadIdx.x == 0) offsets[nb] = carry_s;
}

// idx[k] = site of the k-th selected site (site order): each thread's 16
// sites are placed after the selected sites of the CTAs before it (offsets)
// and of the threads before it in its CTA (a block scan of the counts)
template <bool VEC>
__global__ void __launch_bounds__(kTileThreads) k_mask_index(const unsigned char *__restrict__ mask, long long N,
                                                             const int *__restrict__ offsets, int *__restrict__ idx)
{
    __shared__ int warp_tot[kTileThreads / 32];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const long long base = (long long)blockIdx.x * kTile + (long long)threadIdx.x * kPerThread;
    const unsigned bits = mask_bits<VEC>(mask, base, N);
    const int c = __popc(bits);
    const int incl = warp_incl(c);
    if (lane == 31) warp_tot[warp] = incl;
    __syncthreads();
    int before = offsets[blockIdx.x] + incl - c;
    for (int w = 0; w < warp; w++) before += warp_tot[w];
#pragma unroll
    for (int k = 0; k < kPerThread; k++)
        if (bits & (1u << k)) idx[before++] = (int)(base + k);
}

constexpr int kGatherThreads = 256;   // one selected site per thread

// rho, u = (sum f c + F/2)/rho, phi of the selected sites; u as [3][total].
// REDUCED: phi is component 0 of the g level (the tau_g = 1 form).
template <typename T, bool SH, bool REDUCED>
__global__ void __launch_bounds__(kGatherThreads) k_masked_moments(
    const T *__restrict__ fa, const T *__restrict__ ga, const int *__restrict__ idx, int total, double rho0,
    double hFx, double hFy, double hFz, double *__restrict__ rho, double *__restrict__ u, double *__restrict__ phi,
    int nx, int ny, int nz, long long S)
{
    const int k = blockIdx.x * kGatherThreads + threadIdx.x;
    if (k >= total) return;
    const int s = idx[k];
    const Nbr n(s, nx, ny, nz);
    if (rho || u) {
        double r, v[3];
        site_rho_u<T, SH>(fa, n, S, rho0, hFx, hFy, hFz, r, v);
        if (rho) rho[k] = r;
        if (u) {
            u[k] = v[0];
            u[(size_t)total + k] = v[1];
            u[2 * (size_t)total + k] = v[2];
        }
    }
    if (phi) phi[k] = REDUCED ? double(ga[s]) : site_phi(ga, n, S);
}

// rows [i0, i1) of the post-streaming state A_i(x - c_i) + w_i shift at the
// selected sites, out[(i - i0) * total + k]
template <typename T>
__global__ void __launch_bounds__(kGatherThreads) k_masked_get(const T *__restrict__ a, const int *__restrict__ idx,
                                                               int total, int i0, int i1, double shift,
                                                               double *__restrict__ out, int nx, int ny, int nz,
                                                               long long S)
{
    const int k = blockIdx.x * kGatherThreads + threadIdx.x;
    if (k >= total) return;
    const Nbr n(idx[k], nx, ny, nz);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        if (i < i0 || i >= i1) continue;
        out[(size_t)(i - i0) * total + k] = double(a[(size_t)i * S + n.src(i)]) + weight(i) * shift;
    }
}

// the inverse: A_i(x - c_i) = in[(i - i0) * total + k] - w_i shift at the
// selected sites
template <typename T>
__global__ void __launch_bounds__(kGatherThreads) k_masked_set(T *__restrict__ a, const int *__restrict__ idx,
                                                               int total, int i0, int i1, double shift,
                                                               const double *__restrict__ in, int nx, int ny, int nz,
                                                               long long S)
{
    const int k = blockIdx.x * kGatherThreads + threadIdx.x;
    if (k >= total) return;
    const Nbr n(idx[k], nx, ny, nz);
#pragma unroll
    for (int i = 0; i < Q; i++) {
        if (i < i0 || i >= i1) continue;
        a[(size_t)i * S + n.src(i)] = T(in[(size_t)(i - i0) * total + k] - weight(i) * shift);
    }
}

inline int mask_blocks(long long N) { return (int)((N + kTile - 1) / kTile); }

inline unsigned gather_blocks(long long total) { return (unsigned)((total + kGatherThreads - 1) / kGatherThreads); }

}  // namespace

// scratch: counts [nb], offsets [nb + 1], site indices [N]
size_t masked_scratch_ints(long long N) { return 2 * (size_t)mask_blocks(N) + 1 + (size_t)N; }

// counts, offsets and site indices of the selected sites
int launch_mask_scan(lb_ctx *c, const unsigned char *mask_d, int *scratch)
{
    const int nb = mask_blocks(c->N);
    int *counts = scratch, *offsets = scratch + nb, *idx = scratch + 2 * nb + 1;
    const bool vec = ((unsigned long long)mask_d & 15) == 0;
    if (vec)
        k_mask_count<true><<<nb, kTileThreads, 0, c->stream>>>(mask_d, c->N, counts);
    else
        k_mask_count<false><<<nb, kTileThreads, 0, c->stream>>>(mask_d, c->N, counts);
    k_mask_scan<<<1, kMaskThreads, 0, c->stream>>>(counts, nb, offsets);
    if (vec)
        k_mask_index<true><<<nb, kTileThreads, 0, c->stream>>>(mask_d, c->N, offsets, idx);
    else
        k_mask_index<false><<<nb, kTileThreads, 0, c->stream>>>(mask_d, c->N, offsets, idx);
    return check_launch();
}

int masked_total_offset(long long N) { return 2 * mask_blocks(N); }   // index of offsets[nb] in the scratch

int launch_masked_moments(lb_ctx *c, long long total, const int *scratch, double *rho, double *u, double *phi)
{
    if (total <= 0) return LB_OK;
    const int *idx = scratch + 2 * mask_blocks(c->N) + 1;
    const int cur = c->buf.cur;
    const double hF[3] = {0.5 * c->force[0], 0.5 * c->force[1], 0.5 * c->force[2]};
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const unsigned grid = gather_blocks(total);
    return by_precision(c, [&](auto P) {
        using T = typename decltype(P)::T;
        constexpr bool SH = decltype(P)::SH;
        const T *fa = (const T *)c->buf.f[cur], *ga = (const T *)c->buf.g[cur];
        if (c->reduced)
            k_masked_moments<T, SH, true><<<grid, kGatherThreads, 0, c->stream>>>(
                fa, ga, idx, (int)total, c->p.rho0, hF[0], hF[1], hF[2], rho, u, phi, nx, ny, nz, c->S);
        else
            k_masked_moments<T, SH, false><<<grid, kGatherThreads, 0, c->stream>>>(
                fa, ga, idx, (int)total, c->p.rho0, hF[0], hF[1], hF[2], rho, u, phi, nx, ny, nz, c->S);
        return check_launch();
    });
}

int launch_masked_rows(lb_ctx *c, long long total, const int *scratch, int which, int i0, int i1, double *io,
                       int to_device_state)
{
    if (total <= 0) return LB_OK;
    const int *idx = scratch + 2 * mask_blocks(c->N) + 1;
    const int cur = c->buf.cur;
    const double shift = (which == 0 && c->p.precision == LB_FP32_SHIFTED) ? c->p.rho0 : 0.0;
    void *a = which == 0 ? c->buf.f[cur] : c->buf.g[cur];
    const int nx = c->p.nx, ny = c->p.ny, nz = c->p.nz;
    const unsigned grid = gather_blocks(total);
    const int tot = (int)total;
    return by_precision(c, [&](auto P) {
        using T = typename decltype(P)::T;
        if (to_device_state)
            k_masked_set<T><<<grid, kGatherThreads, 0, c->stream>>>((T *)a, idx, tot, i0, i1, shift, io, nx, ny, nz,
                                                                    c->S);
        else
            k_masked_get<T><<<grid, kGatherThreads, 0, c->stream>>>((const T *)a, idx, tot, i0, i1, shift, io, nx,
                                                                    ny, nz, c->S);
        return check_launch();
    });
}

}  // namespace lbk
