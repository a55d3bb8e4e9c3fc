// lb_batch.cu -- an ensemble of independent lattices (uneven extents and
// parameters) advanced by one persistent launch, captured in a CUDA graph.
//
// Every lattice is an ordinary context (its own buffers and parameters).  The
// work of one timestep of a lattice is a list of (lattice, block of sites)
// items.  A grid of CTAs that all fit on the GPU at once (a cooperative
// launch) is split into groups (plan_groups): by default, with no more
// lattices than CTAs, each lattice gets a group of its own, sized to its
// share of the work (otherwise every CTA is a group holding several whole
// lattices); the plan can also be k groups of whole lattices balanced by
// work, k = 1 being the whole grid.  A group's CTAs walk its
// slice of the work list twice per timestep -- the phi pass, then the
// collide/stream pass -- with a time-bounded barrier of that group alone
// after each, and loop over the timesteps inside the kernel.  Lattices never
// wait for one another, so no grid-wide barrier and its tail remain.  The
// per-site arithmetic is the default step's (lb_site.cuh), or, for an
// ensemble whose lattices all have tau_g = 1 and that was switched to the
// reduced form, the reduced form's two passes (lb_t1.cuh): the collide pass
// over the same (lattice, block) items, then the phi pass over (lattice, x
// block, warp group, z run) tiles.  The launch (with a reset of the barrier
// state) is captured once per (steps, parity) into a CUDA graph and
// replayed.  The block size and CTAs per SM -- the paper's TPB and its
// per-thread work (targetDP Sec. III.C) -- are the knobs the autotuner sets.
#include <cuda_runtime.h>

#include <algorithm>
#include <map>
#include <new>
#include <queue>
#include <utility>
#include <vector>

#include "d3q19.cuh"
#include "lb_internal.cuh"
#include "lb_site.cuh"
#include "lb_t1.cuh"

namespace lbk {

namespace {

// CTA size limit and CTAs per SM the register budget must allow (measured:
// 3 x 256 threads FP32 and 2 x 256 FP64 beat the unconstrained allocation
// by 11 % and 9 %; the FP32 reduced form gains another 6 % at 4 x 256,
// 64 registers, where the general form loses 3 % to spills)
#ifndef LBK_BATCH_MAXT32
#define LBK_BATCH_MAXT32 256
#endif
#ifndef LBK_BATCH_MINB32
#define LBK_BATCH_MINB32 3
#endif
#ifndef LBK_BATCH_MINB32_RED
#define LBK_BATCH_MINB32_RED 4
#endif
#ifndef LBK_BATCH_PHI_V
#define LBK_BATCH_PHI_V 2
#endif
#ifndef LBK_BATCH_MINB64
#define LBK_BATCH_MINB64 2
#endif
constexpr int kBatchMaxThreads = LBK_BATCH_MAXT32;     // FP32 CTA size limit
constexpr int kBatchMaxThreads64 = 256;   // FP64: more registers per thread

template <typename T>
struct LatDesc {
    int nx, ny, nz;
    int kzc;   // reduced form: z planes per phi-pass tile
    long long N, S;
    const T *f[2];
    const T *g[2];
    T *phi;
    Coll<T> p;
};

#ifndef LBK_BATCH_T1_KZC
#define LBK_BATCH_T1_KZC 8
#endif
constexpr int kBatchT1Kzc = LBK_BATCH_T1_KZC;   // z run of a reduced-form phi tile in the ensemble
constexpr int kBatchPhiV = LBK_BATCH_PHI_V;   // phi-pass work items per trip (general form)

struct GridBarrier {
    unsigned int count;
    unsigned int gen;
};

// CTAs [cta0, cta0 + m) advance the lattices whose collide items are
// work[wo, wo + wn) and whose reduced-form phi tiles are work_t1[to, to + tn)
struct Group {
    int cta0, m;
    int wo, wn;
    int to, tn;
};

__device__ __forceinline__ unsigned long long batch_ns()
{
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

// Barrier of nblocks co-resident CTAs (one group).  Time-bounded: a CTA that
// waits longer than timeout_ns (or sees that another CTA already gave up)
// sets the error flag and returns false instead of hanging.
__device__ bool grid_sync(GridBarrier *bar, unsigned int nblocks, long long timeout_ns, unsigned int *err,
                          int *s_fail)
{
    __syncthreads();
    if (threadIdx.x == 0) {
        volatile unsigned int *vgen = &bar->gen;
        const unsigned int gen = *vgen;
        __threadfence();
        int fail = 0;
        if (atomicAdd(&bar->count, 1u) == nblocks - 1) {
            atomicExch(&bar->count, 0u);
            __threadfence();
            atomicAdd(&bar->gen, 1u);
        } else {
            const unsigned long long t0 = batch_ns();
            while (*vgen == gen) {
                if (*(volatile unsigned int *)err || (long long)(batch_ns() - t0) > timeout_ns) {
                    atomicOr(err, 1u);
                    fail = 1;
                    break;
                }
                __nanosleep(32);
            }
        }
        __threadfence();
        *s_fail = fail;
    }
    __syncthreads();
    return !*s_fail;
}

template <typename T, bool SH, bool RED>
__global__ void __launch_bounds__(sizeof(T) == 8 ? kBatchMaxThreads64 : kBatchMaxThreads,
                                  sizeof(T) == 8 ? LBK_BATCH_MINB64 : (RED ? LBK_BATCH_MINB32_RED : LBK_BATCH_MINB32))
    k_batch(const LatDesc<T> *__restrict__ lats, const int2 *__restrict__ work, const int4 *__restrict__ work_t1,
            const Group *__restrict__ groups, const int *__restrict__ cta_group, int nsteps, int parity0,
            GridBarrier *bars, unsigned int *err, long long timeout_ns, int skip_cta)
{
    __shared__ int s_fail;
    const int gi = cta_group[blockIdx.x];
    if (gi < 0) return;   // a CTA the plan left without work
    const Group G = groups[gi];
    GridBarrier *bar = bars + gi;
    const int r = blockIdx.x - G.cta0, wend = G.wo + G.wn;
    if (threadIdx.x == 0) s_fail = 0;
    if constexpr (RED) {
        constexpr int KY = PhiTile<T>::KY;
        const int warps = blockDim.x >> 5, warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
        const int tend = G.to + G.tn;
        for (int t = 0; t < nsteps; t++) {
            const int a = (parity0 + t) & 1;
            for (int w = G.wo + r; w < wend; w += G.m) {
                const int2 it = work[w];
                const LatDesc<T> &L = lats[it.x];
                const long long s = (long long)it.y * blockDim.x + threadIdx.x;
                if (s < L.N)
                    t1_collide_site<T, SH, 7>(L.f[a], const_cast<T *>(L.g[a]), const_cast<T *>(L.f[1 - a]), L.p,
                                              L.nx, L.ny, L.nz, L.S, (int)s);
            }
            if ((int)blockIdx.x == skip_cta) return;   // test hook: this CTA never arrives
            if (!grid_sync(bar, G.m, timeout_ns, err, &s_fail)) return;
            for (int w = G.to + r; w < tend; w += G.m) {
                const int4 it = work_t1[w];   // (lattice, x block, warp group, z run)
                const LatDesc<T> &L = lats[it.x];
                t1_phi_tile<T, KY>(L.g[a], const_cast<T *>(L.g[1 - a]), L.nx, L.ny, L.nz, L.kzc, L.S, it.y,
                                   (it.z * warps + warp) * KY, it.w, lane);
            }
            if (!grid_sync(bar, G.m, timeout_ns, err, &s_fail)) return;
        }
    } else {
        for (int t = 0; t < nsteps; t++) {
            const int a = (parity0 + t) & 1;
            // kBatchPhiV work items per trip, their loads independent, so that
            // the phi pass keeps as many loads in flight as its own kernel
            // would at full occupancy (the collide pass sets the residency)
            for (int w0 = G.wo + r; w0 < wend; w0 += kBatchPhiV * G.m) {
#pragma unroll
                for (int u = 0; u < kBatchPhiV; u++) {
                    const int w = w0 + u * G.m;
                    if (w >= wend) break;
                    const int2 it = work[w];
                    const LatDesc<T> &L = lats[it.x];
                    const long long s = (long long)it.y * blockDim.x + threadIdx.x;
                    if (s < L.N) {
                        const Nbr n((int)s, L.nx, L.ny, L.nz);
                        L.phi[s] = phi_site(L.g[a], n, L.S);
                    }
                }
            }
            if ((int)blockIdx.x == skip_cta) return;   // test hook: this CTA never arrives
            if (!grid_sync(bar, G.m, timeout_ns, err, &s_fail)) return;
            for (int w = G.wo + r; w < wend; w += G.m) {
                const int2 it = work[w];
                const LatDesc<T> &L = lats[it.x];
                const long long s = (long long)it.y * blockDim.x + threadIdx.x;
                if (s < L.N) {
                    const Nbr n((int)s, L.nx, L.ny, L.nz);
                    collide_site<T, SH>(L.f[a], L.g[a], L.phi, const_cast<T *>(L.f[1 - a]),
                                        const_cast<T *>(L.g[1 - a]), L.p, n, s, L.S);
                }
            }
            if (!grid_sync(bar, G.m, timeout_ns, err, &s_fail)) return;
        }
    }
}

// Longest-processing-time rule: the lattices, largest first (stable), each
// to the bin with the least work so far (ties to the lower bin).
void lpt_bins(int n, const long long *items, int nbins, int *bin, std::vector<long long> &load)
{
    std::vector<int> order(n);
    for (int k = 0; k < n; k++) order[k] = k;
    std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return items[a] > items[b]; });
    using Load = std::pair<long long, int>;   // (work so far, bin)
    std::priority_queue<Load, std::vector<Load>, std::greater<Load>> q;
    for (int g = 0; g < nbins; g++) q.push(Load(0, g));
    load.assign(nbins, 0);
    for (int k : order) {
        const Load l = q.top();
        q.pop();
        bin[k] = l.second;
        load[l.second] = l.first + items[k];
        q.push(Load(load[l.second], l.second));
    }
}

// CTAs of the groups with work load[g]: one each, then each further CTA to
// the group whose per-CTA share ceil(load / CTAs) is largest (ties to the
// lower index) until the CTAs run out or every share is 1.
std::vector<long long> share_ctas(const std::vector<long long> &load, int ctas)
{
    const int ng = (int)load.size();
    std::vector<long long> mm(ng, 1);
    auto share = [&](int g) { return (load[g] + mm[g] - 1) / mm[g]; };
    auto lower = [&](int a, int b) {   // a ranks below b in the queue
        const long long sa = share(a), sb = share(b);
        return sa != sb ? sa < sb : a > b;
    };
    std::priority_queue<int, std::vector<int>, decltype(lower)> q(lower);
    for (int g = 0; g < ng; g++) q.push(g);
    for (int left = ctas - ng; left > 0; left--) {
        const int g = q.top();
        if (share(g) <= 1) break;
        q.pop();
        mm[g]++;
        q.push(g);
    }
    return mm;
}

// The CTA plan.  bins = 0: with n <= ctas lattice k is group k; with more
// lattices than CTAs every CTA is a group, filled by the LPT rule.  bins >= 1:
// min(bins, n, ctas) groups, filled with whole lattices by the LPT rule.
// CTAs go to the groups by share_ctas.
int plan_groups(int n, const long long *items, int ctas, int bins, int *group, int *cta0, int *m, int *ngroups)
{
    if (n < 1 || ctas < 1 || bins < 0 || !items || !group || !cta0 || !m || !ngroups) return LB_ERR_INVALID;
    for (int k = 0; k < n; k++)
        if (items[k] < 1) return LB_ERR_INVALID;
    std::vector<long long> load;
    int ng;
    if (bins == 0 && n <= ctas) {
        ng = n;
        load.assign(items, items + n);
        for (int k = 0; k < n; k++) group[k] = k;
    } else {
        ng = bins == 0 ? ctas : std::min(bins, std::min(n, ctas));
        lpt_bins(n, items, ng, group, load);
    }
    const std::vector<long long> mm = share_ctas(load, ctas);
    int c = 0;
    for (int g = 0; g < ng; g++) {
        cta0[g] = c;
        m[g] = (int)mm[g];
        c += m[g];
    }
    *ngroups = ng;
    return LB_OK;
}

}  // namespace
}  // namespace lbk

struct lb_batch {
    int n = 0;
    int precision = LB_FP64;
    std::vector<lb_ctx *> ctx;
    cudaStream_t user_stream = nullptr;
    cudaStream_t stream = nullptr;            // own stream: graphs cannot be captured on the legacy stream
    cudaEvent_t ev_in = nullptr, ev_out = nullptr;
    void *d_lats = nullptr;
    int2 *d_work = nullptr;
    int nwork = 0;
    int4 *d_work_t1 = nullptr;                 // reduced form: phi-pass tiles
    int nwork_t1 = 0;
    lbk::Group *d_groups = nullptr;            // the CTA plan
    int *d_cta_group = nullptr;                // group of every CTA (-1: idle)
    int ngroups = 0;
    int bins = 0;                              // lb_batch_set_plan: 0 = a group per lattice, k = k groups
    int reduced = 0;                           // all lattices in the tau_g = 1 reduced form
    lbk::GridBarrier *d_bar = nullptr;         // one per group
    int skip_cta = -1;                         // test hook: first CTA of the largest group
    unsigned int *d_err = nullptr;
    int threads = 256;                         // sites per work item = threads per CTA
    int ctas_per_sm = 0;                       // 0 = as many as fit
    int grid = 0;
    int parity = 0;                            // timesteps taken, mod 2
    long long timeout_ns = 1000000000LL;
    int debug_skip = 0;
    std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
};

namespace {

void drop_graphs(lb_batch *b)
{
    for (auto &kv : b->graphs) cudaGraphExecDestroy(kv.second);
    b->graphs.clear();
}

template <typename T, bool SH>
int batch_tables(lb_batch *b)
{
    // co-resident grid
    int dev = 0, sms = 0, per_sm = 0;
    int rc = lbk::cuda_status(cudaGetDevice(&dev));
    if (!rc) rc = lbk::cuda_status(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
    if (!rc)
        rc = lbk::cuda_status(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
            &per_sm, b->reduced ? lbk::k_batch<T, SH, true> : lbk::k_batch<T, SH, false>, b->threads, 0));
    if (rc) return rc;
    if (per_sm < 1) return LB_ERR_INVALID;
    const int use = b->ctas_per_sm > 0 && b->ctas_per_sm < per_sm ? b->ctas_per_sm : per_sm;
    b->grid = use * sms;

    // per lattice: descriptor, collide items, reduced-form phi tiles
    const int n = b->n;
    std::vector<lbk::LatDesc<T>> L(n);
    std::vector<std::vector<int4>> tiles(n);
    std::vector<long long> nb(n);
    for (int k = 0; k < n; k++) {
        lb_ctx *c = b->ctx[k];
        L[k].nx = c->p.nx;
        L[k].ny = c->p.ny;
        L[k].nz = c->p.nz;
        L[k].N = c->N;
        L[k].S = c->S;
        for (int l = 0; l < 2; l++) {
            L[k].f[l] = (const T *)c->buf.f[l];
            L[k].g[l] = (const T *)c->buf.g[l];
        }
        L[k].phi = (T *)c->phi;
        L[k].p = lbk::make_coll<T>(c->p);
        L[k].kzc = c->p.nz < lbk::kBatchT1Kzc ? c->p.nz : lbk::kBatchT1Kzc;
        nb[k] = (c->N + b->threads - 1) / b->threads;
        if (b->reduced) {
            const int rows = (b->threads / 32) * lbk::PhiTile<T>::KY;   // y rows of one warp group
            const int gx = (c->p.nx + lbk::kPhiOut - 1) / lbk::kPhiOut, gy = (c->p.ny + rows - 1) / rows;
            const int gz = (c->p.nz + L[k].kzc - 1) / L[k].kzc;
            for (int z = 0; z < gz; z++)
                for (int y = 0; y < gy; y++)
                    for (int x = 0; x < gx; x++) tiles[k].push_back(make_int4(k, x, y, z));
        }
    }

    // CTA groups, and the work lists ordered group by group
    std::vector<int> lat_group(n), cta0(std::min(n, b->grid)), m(std::min(n, b->grid));
    int ng = 0;
    rc = lbk::plan_groups(n, nb.data(), b->grid, b->bins, lat_group.data(), cta0.data(), m.data(), &ng);
    if (rc) return rc;
    std::vector<lbk::Group> groups(ng);
    std::vector<int> cta_group(b->grid, -1);
    std::vector<int2> work;
    std::vector<int4> work_t1;
    for (int g = 0; g < ng; g++) {
        lbk::Group &G = groups[g];
        G.cta0 = cta0[g];
        G.m = m[g];
        G.wo = (int)work.size();
        G.to = (int)work_t1.size();
        for (int k = 0; k < n; k++) {
            if (lat_group[k] != g) continue;
            for (long long j = 0; j < nb[k]; j++) work.push_back(make_int2(k, (int)j));
            work_t1.insert(work_t1.end(), tiles[k].begin(), tiles[k].end());
        }
        G.wn = (int)work.size() - G.wo;
        G.tn = (int)work_t1.size() - G.to;
        for (int i = 0; i < G.m; i++) cta_group[G.cta0 + i] = g;
    }

    cudaFree(b->d_lats);
    cudaFree(b->d_work);
    cudaFree(b->d_work_t1);
    cudaFree(b->d_groups);
    cudaFree(b->d_cta_group);
    cudaFree(b->d_bar);
    b->d_lats = nullptr;
    b->d_work = nullptr;
    b->d_work_t1 = nullptr;
    b->d_groups = nullptr;
    b->d_cta_group = nullptr;
    b->d_bar = nullptr;
    b->ngroups = 0;
    auto upload = [&](void **dst, const void *src, size_t bytes) {
        if (rc || !bytes) return;
        rc = lbk::cuda_status(cudaMalloc(dst, bytes));
        if (!rc) rc = lbk::cuda_status(cudaMemcpy(*dst, src, bytes, cudaMemcpyHostToDevice));
    };
    upload(&b->d_lats, L.data(), sizeof(lbk::LatDesc<T>) * n);
    upload((void **)&b->d_work, work.data(), sizeof(int2) * work.size());
    upload((void **)&b->d_work_t1, work_t1.data(), sizeof(int4) * work_t1.size());
    upload((void **)&b->d_groups, groups.data(), sizeof(lbk::Group) * groups.size());
    upload((void **)&b->d_cta_group, cta_group.data(), sizeof(int) * cta_group.size());
    if (!rc) rc = lbk::cuda_status(cudaMalloc(&b->d_bar, sizeof(lbk::GridBarrier) * ng));
    if (rc) return rc;
    b->nwork = (int)work.size();
    b->nwork_t1 = (int)work_t1.size();
    b->ngroups = ng;
    b->skip_cta = -1;
    for (int g = 0, best = 1; g < ng; g++)
        if (groups[g].m > best) {
            best = groups[g].m;
            b->skip_cta = groups[g].cta0;
        }
    return LB_OK;
}

int tables(lb_batch *b)
{
    drop_graphs(b);
    return b->precision == LB_FP64 ? batch_tables<double, false>(b) : batch_tables<float, true>(b);
}

template <typename T, bool SH>
int capture(lb_batch *b, int nsteps, int parity, cudaGraphExec_t *out)
{
    if (b->debug_skip && b->skip_cta < 0) return LB_ERR_INVALID;   // no group of two CTAs to test with
    cudaGraph_t graph = nullptr;
    int rc = lbk::cuda_status(cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal));
    if (rc) return rc;
    cudaMemsetAsync(b->d_bar, 0, sizeof(lbk::GridBarrier) * b->ngroups, b->stream);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)b->grid);
    cfg.blockDim = dim3((unsigned)b->threads);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = b->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const lbk::LatDesc<T> *lats = (const lbk::LatDesc<T> *)b->d_lats;
    const cudaError_t le =
        cudaLaunchKernelEx(&cfg, b->reduced ? lbk::k_batch<T, SH, true> : lbk::k_batch<T, SH, false>, lats,
                           (const int2 *)b->d_work, (const int4 *)b->d_work_t1, (const lbk::Group *)b->d_groups,
                           (const int *)b->d_cta_group, nsteps, parity, b->d_bar, b->d_err, b->timeout_ns,
                           b->debug_skip ? b->skip_cta : -1);
    const cudaError_t ce = cudaStreamEndCapture(b->stream, &graph);
    rc = lbk::cuda_status(le != cudaSuccess ? le : ce);
    if (!rc) rc = lbk::cuda_status(cudaGraphInstantiate(out, graph, 0));
    if (graph) cudaGraphDestroy(graph);
    return rc;
}

int batch_sync(lb_batch *b)
{
    unsigned int flag = 0;
    int rc = lbk::cuda_status(cudaMemcpyAsync(&flag, b->d_err, sizeof(flag), cudaMemcpyDeviceToHost, b->stream));
    if (!rc) rc = lbk::cuda_status(cudaStreamSynchronize(b->stream));
    if (!rc) rc = lbk::cuda_status(cudaStreamSynchronize(b->user_stream));
    if (rc) return rc;
    if (flag) {
        rc = lbk::cuda_status(cudaMemsetAsync(b->d_err, 0, sizeof(unsigned int), b->stream));
        if (!rc) rc = lbk::cuda_status(cudaStreamSynchronize(b->stream));
        return rc ? rc : LB_ERR_TIMEOUT;
    }
    return LB_OK;
}

bool index_ok(const lb_batch *b, int k) { return b && k >= 0 && k < b->n; }

}  // namespace

extern "C" {

void lb_batch_destroy(lb_batch *b)
{
    if (!b) return;
    if (b->stream) cudaStreamSynchronize(b->stream);
    drop_graphs(b);
    for (lb_ctx *c : b->ctx) {
        // a member adopted into the ensemble shares its error flag (freed
        // below); one created before a failure still owns its own
        if (c->batch_owned) lbk::release_from_batch(c);
        lb_destroy(c);
    }
    cudaFree(b->d_lats);
    cudaFree(b->d_work);
    cudaFree(b->d_work_t1);
    cudaFree(b->d_groups);
    cudaFree(b->d_cta_group);
    cudaFree(b->d_bar);
    cudaFree(b->d_err);
    if (b->ev_in) cudaEventDestroy(b->ev_in);
    if (b->ev_out) cudaEventDestroy(b->ev_out);
    if (b->stream) cudaStreamDestroy(b->stream);
    cudaGetLastError();
    delete b;
}

int lb_batch_create(int n, const lb_params *p, void *cuda_stream, lb_batch **out)
{
    if (!out) return LB_ERR_INVALID;
    *out = nullptr;
    if (n < 1 || !p) return LB_ERR_INVALID;
    if (p[0].precision != LB_FP64 && p[0].precision != LB_FP32_SHIFTED) return LB_ERR_INVALID;
    for (int k = 1; k < n; k++)
        if (p[k].precision != p[0].precision) return LB_ERR_INVALID;
    lb_batch *b = new (std::nothrow) lb_batch();
    if (!b) return LB_ERR_NOMEM;
    b->n = n;
    b->precision = p[0].precision;
    b->user_stream = (cudaStream_t)cuda_stream;
    int rc = LB_OK;
    for (int k = 0; k < n && !rc; k++) {
        lb_ctx *c = nullptr;
        rc = lb_create(&p[k], cuda_stream, &c);
        if (!rc) b->ctx.push_back(c);
    }
    if (!rc) rc = lbk::cuda_status(cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking));
    if (!rc) rc = lbk::cuda_status(cudaEventCreateWithFlags(&b->ev_in, cudaEventDisableTiming));
    if (!rc) rc = lbk::cuda_status(cudaEventCreateWithFlags(&b->ev_out, cudaEventDisableTiming));
    if (!rc) rc = lbk::cuda_status(cudaMalloc(&b->d_err, sizeof(unsigned int)));
    if (!rc) rc = lbk::cuda_status(cudaMemset(b->d_err, 0, sizeof(unsigned int)));
    if (!rc)
        for (lb_ctx *c : b->ctx) lbk::adopt_into_batch(c, b->d_err);
    if (!rc) rc = tables(b);
    if (rc) {
        lb_batch_destroy(b);
        return rc;
    }
    *out = b;
    return LB_OK;
}

int lb_batch_plan(int n, const long long *items, int ctas, int bins, int *group, int *cta0, int *m, int *ngroups)
{
    return lbk::plan_groups(n, items, ctas, bins, group, cta0, m, ngroups);
}

int lb_batch_set_plan(lb_batch *b, int bins)
{
    if (!b || bins < 0) return LB_ERR_INVALID;
    if (bins == b->bins) return LB_OK;
    int rc = batch_sync(b);
    if (rc) return rc;
    const int old = b->bins;
    b->bins = bins;
    rc = tables(b);
    if (rc) {
        b->bins = old;
        tables(b);
    }
    return rc;
}

int lb_batch_groups(const lb_batch *b, int *ngroups)
{
    if (!b || !ngroups) return LB_ERR_INVALID;
    *ngroups = b->ngroups;
    return LB_OK;
}

int lb_batch_size(const lb_batch *b, int *n, int *work_items, int *grid, int *threads)
{
    if (!b) return LB_ERR_INVALID;
    if (n) *n = b->n;
    if (work_items) *work_items = b->nwork;
    if (grid) *grid = b->grid;
    if (threads) *threads = b->threads;
    return LB_OK;
}

int lb_batch_set_launch(lb_batch *b, int threads, int ctas_per_sm)
{
    const int maxt = b && b->precision == LB_FP64 ? lbk::kBatchMaxThreads64 : lbk::kBatchMaxThreads;
    if (!b || threads < 32 || threads > maxt || threads % 32 != 0 || ctas_per_sm < 0) return LB_ERR_INVALID;
    const int old_t = b->threads, old_c = b->ctas_per_sm;
    b->threads = threads;
    b->ctas_per_sm = ctas_per_sm;
    const int rc = tables(b);
    if (rc) {
        b->threads = old_t;
        b->ctas_per_sm = old_c;
        tables(b);
    }
    return rc;
}

int lb_batch_set_wait_timeout(lb_batch *b, long long timeout_ns)
{
    if (!b || timeout_ns < 1000 || timeout_ns > 60000000000LL) return LB_ERR_INVALID;
    b->timeout_ns = timeout_ns;
    drop_graphs(b);
    return LB_OK;
}

int lb_batch_debug_skip_arrival(lb_batch *b, int enable)
{
    if (!b) return LB_ERR_INVALID;
    b->debug_skip = enable ? 1 : 0;
    drop_graphs(b);
    return LB_OK;
}

lb_ctx *lb_batch_lattice(lb_batch *b, int k) { return index_ok(b, k) ? b->ctx[k] : nullptr; }

int lb_batch_run(lb_batch *b, int nsteps)
{
    if (!b || nsteps < 0) return LB_ERR_INVALID;
    if (nsteps == 0) return LB_OK;
    const auto key = std::make_pair(nsteps, b->parity);
    auto it = b->graphs.find(key);
    if (it == b->graphs.end()) {
        cudaGraphExec_t exec = nullptr;
        const int rc = b->precision == LB_FP64 ? capture<double, false>(b, nsteps, b->parity, &exec)
                                               : capture<float, true>(b, nsteps, b->parity, &exec);
        if (rc) return rc;
        it = b->graphs.emplace(key, exec).first;
    }
    int rc = lbk::cuda_status(cudaEventRecord(b->ev_in, b->user_stream));
    if (!rc) rc = lbk::cuda_status(cudaStreamWaitEvent(b->stream, b->ev_in, 0));
    if (!rc) rc = lbk::cuda_status(cudaGraphLaunch(it->second, b->stream));
    if (!rc) rc = lbk::cuda_status(cudaEventRecord(b->ev_out, b->stream));
    if (!rc) rc = lbk::cuda_status(cudaStreamWaitEvent(b->user_stream, b->ev_out, 0));
    if (rc) return rc;
    b->parity ^= (nsteps & 1);
    for (lb_ctx *c : b->ctx) {
        c->buf.cur = b->parity;
        if (b->reduced) c->m_valid = 1;
    }
    return LB_OK;
}

int lb_batch_set_form(lb_batch *b, int reduced)
{
    if (!b || (reduced != 0 && reduced != 1)) return LB_ERR_INVALID;
    if (reduced == b->reduced) return LB_OK;
    if (reduced)
        for (lb_ctx *c : b->ctx)
            if (c->p.tau_g != 1.0) return LB_ERR_INVALID;
    int rc = batch_sync(b);
    for (lb_ctx *c : b->ctx) {
        if (!rc) rc = lbk::taug1_convert(c, reduced);
        if (!rc) c->reduced = reduced;
    }
    if (!rc) rc = lbk::cuda_status(cudaStreamSynchronize(b->user_stream));
    if (rc) return rc;
    b->reduced = reduced;
    return tables(b);
}

int lb_batch_sync(lb_batch *b)
{
    if (!b) return LB_ERR_INVALID;
    return batch_sync(b);
}

}  // extern "C"
