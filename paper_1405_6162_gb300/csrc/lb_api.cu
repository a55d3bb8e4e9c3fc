// lb_api.cu -- the extern "C" entry points of liblb (declared in lb.h).
//
// The context owns the device-side lattice (the paper's "target copy",
// targetDP Sec. III.A); every caller array is borrowed for the duration of
// the call (host) or until the work queued on the context's stream has run
// (device).
#include <cmath>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <new>

#include "d3q19.cuh"
#include "lb_internal.cuh"

namespace {

thread_local char g_last_error[256] = "";

std::mutex g_alloc_mu;
lb_alloc_fn g_alloc = nullptr;
lb_free_fn g_free = nullptr;
void *g_alloc_user = nullptr;

void *dev_alloc(lb_ctx *c, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (c->alloc) return c->alloc(bytes, (void *)c->stream, c->alloc_user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return p;
}

void dev_free(lb_ctx *c, void *p, size_t bytes)
{
    if (!p) return;
    if (bytes == 0) bytes = 256;
    if (c->free_fn)
        c->free_fn(p, bytes, (void *)c->stream, c->alloc_user);
    else
        cudaFree(p);
}

size_t dist_bytes(const lb_ctx *c) { return (size_t)lbk::Q * (size_t)c->S * c->esize; }
size_t io_bytes(const lb_ctx *c) { return 5 * (size_t)c->N * sizeof(double); }

void free_all(lb_ctx *c)
{
    for (int k = 0; k < 2; k++) {
        dev_free(c, c->buf.f[k], dist_bytes(c));
        dev_free(c, c->buf.g[k], dist_bytes(c));
        c->buf.f[k] = c->buf.g[k] = nullptr;
    }
    dev_free(c, c->phi, (size_t)c->N * c->esize);
    dev_free(c, c->io, io_bytes(c));
    dev_free(c, c->partial, (size_t)lbk::kReduceBlocks * 5 * sizeof(double));
    dev_free(c, c->dev_out, 8 * sizeof(double));
    dev_free(c, c->lag_counters, (size_t)(c->p.nz + 1) * sizeof(unsigned long long));
    if (!c->batch_owned) dev_free(c, c->err_flag, sizeof(unsigned int));
    dev_free(c, c->mask_buf, (size_t)c->N);
    dev_free(c, c->mask_scratch, lbk::masked_scratch_ints(c->N) * sizeof(int));
    c->mask_buf = nullptr;
    c->mask_scratch = nullptr;
    dev_free(c, c->adj, 6 * (size_t)c->N * sizeof(double));
    dev_free(c, c->adj_part, (size_t)lbk::adjoint_blocks(c->N) * sizeof(double));
    c->adj = nullptr;
    c->adj_part = nullptr;
    c->lag_counters = nullptr;
    c->err_flag = nullptr;
    c->phi = nullptr;
    c->io = nullptr;
    c->partial = nullptr;
    c->dev_out = nullptr;
}

bool finite_pos(double v) { return std::isfinite(v); }

int validate(const lb_params *p)
{
    if (!p) return LB_ERR_INVALID;
    if (p->nx < 1 || p->ny < 1 || p->nz < 1) return LB_ERR_INVALID;
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (N >= (1LL << 31)) return LB_ERR_INVALID;
    const double v[] = {p->tau, p->tau_g, p->rho0, p->gamma, p->A, p->B, p->kappa};
    for (double x : v)
        if (!finite_pos(x)) return LB_ERR_INVALID;
    if (!(p->tau > 0.5) || !(p->tau_g > 0.5) || !(p->rho0 > 0.0)) return LB_ERR_INVALID;
    if (p->precision != LB_FP64 && p->precision != LB_FP32_SHIFTED && p->precision != LB_FP64_DF)
        return LB_ERR_INVALID;
    return LB_OK;
}

int ensure_io(lb_ctx *c)
{
    if (c->io) return LB_OK;
    c->io = (double *)dev_alloc(c, io_bytes(c));
    return c->io ? LB_OK : LB_ERR_NOMEM;
}

// Synchronise the stream, then report (and clear) a device-side wait that
// gave up since the last check.
int sync(lb_ctx *c)
{
    unsigned int flag = 0;
    int rc = lbk::cuda_status(cudaMemcpyAsync(&flag, c->err_flag, sizeof(flag), cudaMemcpyDeviceToHost, c->stream));
    if (!rc) rc = lbk::cuda_status(cudaStreamSynchronize(c->stream));
    if (rc) return rc;
    if (flag) {
        rc = lbk::cuda_status(cudaMemsetAsync(c->err_flag, 0, sizeof(unsigned int), c->stream));
        if (!rc) rc = lbk::cuda_status(cudaStreamSynchronize(c->stream));
        return rc ? rc : LB_ERR_TIMEOUT;
    }
    return LB_OK;
}

int copy(lb_ctx *c, void *dst, const void *src, size_t bytes, cudaMemcpyKind kind)
{
    if (bytes == 0) return LB_OK;
    return lbk::cuda_status(cudaMemcpyAsync(dst, src, bytes, kind, c->stream));
}

}  // namespace

namespace lbk {

int cuda_status(cudaError_t e)
{
    if (e == cudaSuccess) return LB_OK;
    std::snprintf(g_last_error, sizeof(g_last_error), "%s: %s", cudaGetErrorName(e), cudaGetErrorString(e));
    return e == cudaErrorMemoryAllocation ? LB_ERR_NOMEM : LB_ERR_CUDA;
}

int check_launch() { return cuda_status(cudaGetLastError()); }

void adopt_into_batch(lb_ctx *c, unsigned int *shared_err)
{
    cudaStreamSynchronize(c->stream);
    dev_free(c, c->err_flag, sizeof(unsigned int));
    c->err_flag = shared_err;
    c->batch_owned = 1;
}

void release_from_batch(lb_ctx *c)
{
    c->err_flag = nullptr;
    c->batch_owned = 0;
}

}  // namespace lbk

extern "C" {

const char *lb_strerror(int code)
{
    switch (code) {
    case LB_OK: return "ok";
    case LB_ERR_INVALID: return "invalid argument";
    case LB_ERR_NOMEM: return "device allocation failed";
    case LB_ERR_CUDA: return "CUDA error";
    case LB_ERR_NONFINITE: return "non-finite value in the lattice state";
    case LB_ERR_TIMEOUT: return "bounded device-side wait timed out";
    default: return "unknown error code";
    }
}

const char *lb_last_error(void) { return g_last_error; }

int lb_set_allocator(lb_alloc_fn alloc, lb_free_fn free_fn, void *user)
{
    if ((alloc == nullptr) != (free_fn == nullptr)) return LB_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_alloc_mu);
    g_alloc = alloc;
    g_free = free_fn;
    g_alloc_user = alloc ? user : nullptr;
    return LB_OK;
}

int lb_create(const lb_params *p, void *cuda_stream, lb_ctx **out)
{
    if (!out) return LB_ERR_INVALID;
    *out = nullptr;
    int rc = validate(p);
    if (rc) return rc;
    lb_ctx *c = new (std::nothrow) lb_ctx();
    if (!c) return LB_ERR_NOMEM;
    c->p = *p;
    c->stream = (cudaStream_t)cuda_stream;
    c->N = (long long)p->nx * p->ny * p->nz;
    c->S = lbk::component_stride(c->N);
    c->esize = p->precision == LB_FP32_SHIFTED ? sizeof(float) : 8;   // double or two floats
    {
        std::lock_guard<std::mutex> lk(g_alloc_mu);
        c->alloc = g_alloc;
        c->free_fn = g_free;
        c->alloc_user = g_alloc_user;
    }
    rc = lbk::cuda_status(cudaGetDevice(&c->device));
    if (rc) {
        delete c;
        return rc;
    }
    for (int k = 0; k < 2; k++) {
        c->buf.f[k] = dev_alloc(c, dist_bytes(c));
        c->buf.g[k] = dev_alloc(c, dist_bytes(c));
    }
    c->phi = dev_alloc(c, (size_t)c->N * c->esize);
    c->partial = (double *)dev_alloc(c, (size_t)lbk::kReduceBlocks * 5 * sizeof(double));
    c->dev_out = (double *)dev_alloc(c, 8 * sizeof(double));
    c->lag_counters = (unsigned long long *)dev_alloc(c, (size_t)(p->nz + 1) * sizeof(unsigned long long));
    c->err_flag = (unsigned int *)dev_alloc(c, sizeof(unsigned int));
    bool ok = c->phi && c->partial && c->dev_out && c->lag_counters && c->err_flag;
    for (int k = 0; k < 2; k++) ok = ok && c->buf.f[k] && c->buf.g[k];
    if (!ok) {
        free_all(c);
        delete c;
        return LB_ERR_NOMEM;
    }
    rc = lbk::cuda_status(cudaMemsetAsync(c->lag_counters, 0, (size_t)(p->nz + 1) * sizeof(unsigned long long),
                                          c->stream));
    if (!rc) rc = lbk::cuda_status(cudaMemsetAsync(c->err_flag, 0, sizeof(unsigned int), c->stream));
    for (int k = 0; k < 2 && !rc; k++) {
        rc = lbk::cuda_status(cudaMemsetAsync(c->buf.f[k], 0, dist_bytes(c), c->stream));
        if (!rc) rc = lbk::cuda_status(cudaMemsetAsync(c->buf.g[k], 0, dist_bytes(c), c->stream));
    }
    if (rc) {
        lb_destroy(c);
        return rc;
    }
    *out = c;
    return LB_OK;
}

void lb_destroy(lb_ctx *c)
{
    if (!c || c->batch_owned) return;   // ensemble members are freed by lb_batch_destroy
    cudaStreamSynchronize(c->stream);
    cudaGetLastError();
    free_all(c);
    delete c;
}

// the adjoint scratch, allocated on first use; on failure nothing is kept
static int ensure_adj(lb_ctx *c)
{
    if (c->adj && c->adj_part) return LB_OK;
    const size_t adj_bytes = 6 * (size_t)c->N * sizeof(double);
    const size_t part_bytes = (size_t)lbk::adjoint_blocks(c->N) * sizeof(double);
    if (!c->adj) c->adj = (double *)dev_alloc(c, adj_bytes);
    if (!c->adj_part) c->adj_part = (double *)dev_alloc(c, part_bytes);
    if (c->adj && c->adj_part) return LB_OK;
    dev_free(c, c->adj, adj_bytes);
    dev_free(c, c->adj_part, part_bytes);
    c->adj = nullptr;
    c->adj_part = nullptr;
    return LB_ERR_NOMEM;
}

int lb_adjoint_step(lb_ctx *c, const double *f, const double *g, const double *af_in, const double *ag_in,
                    double *af_out, double *ag_out, double *dkappa)
{
    if (!c || c->p.precision != LB_FP64 || c->npts != 7 || lbk::uses_mrt(c) || !f || !g || !af_in || !ag_in ||
        !af_out || !ag_out || !dkappa)
        return LB_ERR_INVALID;
    if (af_out == af_in || ag_out == ag_in || af_out == ag_in || ag_out == af_in) return LB_ERR_INVALID;
    const int rc = ensure_adj(c);
    if (rc) return rc;
    return lbk::launch_adjoint_step(c, f, g, af_in, ag_in, af_out, ag_out, dkappa, c->adj, c->adj_part);
}

int lb_adjoint_seed(lb_ctx *c, const double *phi_bar, double *af, double *ag)
{
    if (!c || c->p.precision != LB_FP64 || !phi_bar || !af || !ag || af == ag) return LB_ERR_INVALID;
    return lbk::launch_adjoint_seed(c, phi_bar, af, ag);
}

int lb_adjoint_init(lb_ctx *c, const double *phi0, const double *u0, const double *af0, const double *ag0,
                    double *phi0_bar, double *dkappa)
{
    if (!c || c->p.precision != LB_FP64 || c->npts != 7 || lbk::uses_mrt(c) || !phi0 || !af0 || !ag0 ||
        !phi0_bar || !dkappa)
        return LB_ERR_INVALID;
    const int rc = ensure_adj(c);
    if (rc) return rc;
    return lbk::launch_adjoint_init(c, phi0, u0, af0, ag0, phi0_bar, dkappa, c->adj, c->adj_part);
}

int lb_sync(lb_ctx *c)
{
    if (!c) return LB_ERR_INVALID;
    return sync(c);
}

int lb_set_wait_timeout(lb_ctx *c, long long timeout_ns)
{
    if (!c || timeout_ns < 1000 || timeout_ns > 60000000000LL) return LB_ERR_INVALID;
    c->wait_timeout_ns = timeout_ns;
    return LB_OK;
}

int lb_debug_wait_skew(lb_ctx *c, unsigned long long skew)
{
    if (!c) return LB_ERR_INVALID;
    c->lag_target_skew = skew;
    return LB_OK;
}

int lb_get_info(const lb_ctx *c, int *nx, int *ny, int *nz, int *precision)
{
    if (!c) return LB_ERR_INVALID;
    if (nx) *nx = c->p.nx;
    if (ny) *ny = c->p.ny;
    if (nz) *nz = c->p.nz;
    if (precision) *precision = c->p.precision;
    return LB_OK;
}

int lb_init(lb_ctx *c, const double *phi0, const double *u0, int ptr_kind)
{
    if (!c || !phi0 || (ptr_kind != LB_HOST && ptr_kind != LB_DEVICE)) return LB_ERR_INVALID;
    const size_t nb = (size_t)c->N * sizeof(double);
    if (ptr_kind == LB_DEVICE) {
        int rc = lbk::launch_init(c, phi0, u0);
        if (!rc && c->reduced) rc = lbk::taug1_convert(c, 1);
        return rc;
    }
    int rc = ensure_io(c);
    if (rc) return rc;
    rc = copy(c, c->io, phi0, nb, cudaMemcpyHostToDevice);
    if (!rc && u0) rc = copy(c, c->io + c->N, u0, 3 * nb, cudaMemcpyHostToDevice);
    if (!rc) rc = lbk::launch_init(c, c->io, u0 ? c->io + c->N : nullptr);
    if (!rc && c->reduced) rc = lbk::taug1_convert(c, 1);
    if (!rc) rc = sync(c);
    return rc;
}

int lb_step(lb_ctx *c, int nsteps)
{
    if (!c || nsteps < 0 || c->batch_owned) return LB_ERR_INVALID;
    if (nsteps == 0) return LB_OK;
    if (c->reduced) return lbk::launch_step_taug1(c, nsteps);
    if (c->kernel == LB_KERNEL_AUTO && lbk::auto_uses_bulk(c)) return lbk::launch_step_bulk_auto(c, nsteps);
    if (c->kernel == LB_KERNEL_TWO_PASS || c->kernel == LB_KERNEL_AUTO) return lbk::launch_step_two_pass(c, nsteps);
    if (c->kernel == LB_KERNEL_STAGED) return lbk::launch_step_staged(c, nsteps);
    if (c->kernel == LB_KERNEL_SLAB) return lbk::launch_step_slab(c, nsteps);
    if (c->kernel == LB_KERNEL_LAG) return lbk::launch_step_lag(c, nsteps);
    if (c->kernel == LB_KERNEL_BULK) return lbk::launch_step_bulk(c, nsteps);
    return lbk::launch_step_fused(c, nsteps);
}

// kernels whose phi stencil is fixed to 7 points (staged in shared memory)
static bool seven_point_only(int kernel)
{
    return kernel == LB_KERNEL_FUSED || kernel == LB_KERNEL_STAGED || kernel == LB_KERNEL_SLAB ||
           kernel == LB_KERNEL_LAG || kernel == LB_KERNEL_BULK;
}

static bool any_force(const double *F) { return F[0] != 0.0 || F[1] != 0.0 || F[2] != 0.0; }

int lb_set_collision(lb_ctx *c, int model, double tau_bulk, double tau_ghost)
{
    if (!c || c->batch_owned) return LB_ERR_INVALID;
    if (model != LB_COLLISION_BGK && model != LB_COLLISION_MRT) return LB_ERR_INVALID;
    if (model == LB_COLLISION_MRT) {
        if (!(tau_bulk > 0.5) || !(tau_ghost > 0.5) || !std::isfinite(tau_bulk) || !std::isfinite(tau_ghost))
            return LB_ERR_INVALID;
        if (c->kernel != LB_KERNEL_AUTO && c->kernel != LB_KERNEL_TWO_PASS) return LB_ERR_INVALID;
        c->tau_bulk = tau_bulk;
        c->tau_ghost = tau_ghost;
    }
    c->collision = model;
    return LB_OK;
}

int lb_set_force(lb_ctx *c, double fx, double fy, double fz)
{
    if (!c || c->batch_owned) return LB_ERR_INVALID;
    if (!std::isfinite(fx) || !std::isfinite(fy) || !std::isfinite(fz)) return LB_ERR_INVALID;
    const double F[3] = {fx, fy, fz};
    if (any_force(F) && c->kernel != LB_KERNEL_AUTO && c->kernel != LB_KERNEL_TWO_PASS) return LB_ERR_INVALID;
    for (int a = 0; a < 3; a++) c->force[a] = F[a];
    return LB_OK;
}

int lb_set_stencil(lb_ctx *c, int points)
{
    if (!c || c->batch_owned) return LB_ERR_INVALID;
    if (points != 7 && points != 19 && points != 27) return LB_ERR_INVALID;
    if (points != 7 && seven_point_only(c->kernel)) return LB_ERR_INVALID;
    c->npts = points;
    return LB_OK;
}

int lb_set_kernel(lb_ctx *c, int kernel, int block_x, int block_y, int z_chunk)
{
    if (!c) return LB_ERR_INVALID;
    if (kernel < LB_KERNEL_AUTO || kernel > LB_KERNEL_BULK || c->batch_owned) return LB_ERR_INVALID;
    if (block_x < 0 || block_y < 0 || z_chunk < 0) return LB_ERR_INVALID;
    if (c->npts != 7 && seven_point_only(kernel)) return LB_ERR_INVALID;
    if (c->p.precision == LB_FP64_DF && kernel != LB_KERNEL_AUTO && kernel != LB_KERNEL_TWO_PASS &&
        kernel != LB_KERNEL_TAUG1)
        return LB_ERR_INVALID;
    if (lbk::uses_mrt(c) && kernel != LB_KERNEL_AUTO && kernel != LB_KERNEL_TWO_PASS) return LB_ERR_INVALID;
    if (kernel == LB_KERNEL_AUTO || kernel == LB_KERNEL_TWO_PASS) {
        int rc = lbk::two_pass_validate(block_x, block_y, z_chunk);
        if (rc) return rc;
    } else if (kernel == LB_KERNEL_STAGED) {
        int rc = lbk::staged_validate(c->p.precision, block_x, block_y, z_chunk);
        if (rc) return rc;
    } else if (kernel == LB_KERNEL_TAUG1) {
        int rc = lbk::taug1_validate(c->p, block_x, block_y, z_chunk);
        if (rc) return rc;
    } else if (kernel == LB_KERNEL_LAG) {
        int rc = lbk::lag_validate(block_x, block_y, z_chunk);
        if (rc) return rc;
    } else if (kernel == LB_KERNEL_SLAB) {
        int rc = lbk::slab_validate(c->p.precision, block_x, block_y, z_chunk);
        if (rc) return rc;
    } else if (kernel == LB_KERNEL_BULK) {
        int rc = lbk::bulk_validate(c->p, block_x, block_y, z_chunk);
        if (rc) return rc;
    } else if (kernel == LB_KERNEL_FUSED) {
        int rc = lbk::fused_validate(c->p.precision, block_x, block_y, z_chunk);
        if (rc) return rc;
    }
    const int want_reduced = kernel == LB_KERNEL_TAUG1;
    if (want_reduced != c->reduced) {
        const int rc = lbk::taug1_convert(c, want_reduced);
        if (rc) return rc;
        c->reduced = want_reduced;
    }
    c->kernel = kernel;
    c->block_x = block_x;
    c->block_y = block_y;
    c->z_chunk = z_chunk;
    return LB_OK;
}

int lb_moments(lb_ctx *c, double *rho, double *u, double *phi, int ptr_kind)
{
    if (!c || (ptr_kind != LB_HOST && ptr_kind != LB_DEVICE)) return LB_ERR_INVALID;
    if (!rho && !u && !phi) return LB_OK;
    if (ptr_kind == LB_DEVICE) {
        if (!c->reduced) return lbk::launch_moments(c, rho, u, phi);
        int rc = (rho || u) ? lbk::launch_moments(c, rho, u, nullptr) : LB_OK;
        if (!rc && phi) rc = lbk::taug1_phi_out(c, phi);
        return rc;
    }
    int rc = ensure_io(c);
    if (rc) return rc;
    const size_t N = (size_t)c->N, nb = N * sizeof(double);
    if (c->reduced) {
        rc = (rho || u) ? lbk::launch_moments(c, rho ? c->io : nullptr, u ? c->io + N : nullptr, nullptr) : LB_OK;
        if (!rc && phi) rc = lbk::taug1_phi_out(c, c->io + 4 * N);
    } else {
        rc = lbk::launch_moments(c, rho ? c->io : nullptr, u ? c->io + N : nullptr, phi ? c->io + 4 * N : nullptr);
    }
    if (!rc && rho) rc = copy(c, rho, c->io, nb, cudaMemcpyDeviceToHost);
    if (!rc && u) rc = copy(c, u, c->io + N, 3 * nb, cudaMemcpyDeviceToHost);
    if (!rc && phi) rc = copy(c, phi, c->io + 4 * N, nb, cudaMemcpyDeviceToHost);
    if (!rc) rc = sync(c);
    return rc;
}

int lb_reduce(lb_ctx *c, double out[5])
{
    if (!c || !out) return LB_ERR_INVALID;
    int rc = lbk::launch_reduce(c, c->dev_out);
    if (!rc) rc = copy(c, out, c->dev_out, 5 * sizeof(double), cudaMemcpyDeviceToHost);
    if (!rc) rc = sync(c);
    if (rc) return rc;
    for (int k = 0; k < 5; k++)
        if (!std::isfinite(out[k])) return LB_ERR_NONFINITE;
    return LB_OK;
}

int lb_get_state(lb_ctx *c, double *f, double *g, int ptr_kind)
{
    if (!c || (ptr_kind != LB_HOST && ptr_kind != LB_DEVICE)) return LB_ERR_INVALID;
    if (ptr_kind == LB_DEVICE) {
        if (!c->reduced) return lbk::launch_get_state(c, f, g);
        int rc = f ? lbk::launch_get_state(c, f, nullptr) : LB_OK;
        if (!rc && g) rc = lbk::taug1_g_rows(c, 0, lbk::Q, g);
        return rc;
    }
    int rc = ensure_io(c);
    if (rc) return rc;
    const size_t N = (size_t)c->N;
    double *dst[2] = {f, g};
    for (int which = 0; which < 2 && !rc; which++) {
        if (!dst[which]) continue;
        for (int i0 = 0; i0 < lbk::Q && !rc; i0 += 5) {
            const int i1 = i0 + 5 < lbk::Q ? i0 + 5 : lbk::Q;
            rc = (which == 1 && c->reduced) ? lbk::taug1_g_rows(c, i0, i1, c->io)
                                            : lbk::launch_rows(c, which, i0, i1, c->io, 0);
            if (!rc) rc = copy(c, dst[which] + (size_t)i0 * N, c->io, (size_t)(i1 - i0) * N * sizeof(double),
                               cudaMemcpyDeviceToHost);
            if (!rc) rc = sync(c);
        }
    }
    return rc;
}

int lb_set_state(lb_ctx *c, const double *f, const double *g, int ptr_kind)
{
    if (!c || (ptr_kind != LB_HOST && ptr_kind != LB_DEVICE)) return LB_ERR_INVALID;
    if (ptr_kind == LB_DEVICE) {
        int rc = lbk::launch_set_state(c, f, g);
        if (!rc && c->reduced && g) rc = lbk::taug1_convert(c, 1);
        return rc;
    }
    int rc = ensure_io(c);
    if (rc) return rc;
    const size_t N = (size_t)c->N;
    const double *src[2] = {f, g};
    for (int which = 0; which < 2 && !rc; which++) {
        if (!src[which]) continue;
        for (int i0 = 0; i0 < lbk::Q && !rc; i0 += 5) {
            const int i1 = i0 + 5 < lbk::Q ? i0 + 5 : lbk::Q;
            rc = copy(c, c->io, src[which] + (size_t)i0 * N, (size_t)(i1 - i0) * N * sizeof(double),
                      cudaMemcpyHostToDevice);
            if (!rc) rc = lbk::launch_rows(c, which, i0, i1, c->io, 1);
            if (!rc) rc = sync(c);
        }
    }
    if (!rc && c->reduced && g) rc = lbk::taug1_convert(c, 1);
    if (!rc) rc = sync(c);
    return rc;
}

// Device mask and the compaction offsets of the selected sites; *total
// receives their number (synchronises the stream).
static int masked_prepare(lb_ctx *c, const unsigned char *mask, int ptr_kind, const unsigned char **mask_d,
                          long long *total)
{
    // the compaction buffers (and, for a host mask, its device copy) are
    // allocated on first use; a failure keeps nothing allocated by this call
    const size_t scratch_bytes = lbk::masked_scratch_ints(c->N) * sizeof(int);
    const bool new_scratch = !c->mask_scratch, new_buf = ptr_kind == LB_HOST && !c->mask_buf;
    if (new_scratch) c->mask_scratch = (int *)dev_alloc(c, scratch_bytes);
    if (new_buf) c->mask_buf = (unsigned char *)dev_alloc(c, (size_t)c->N);
    if (!c->mask_scratch || (ptr_kind == LB_HOST && !c->mask_buf)) {
        if (new_scratch) {
            dev_free(c, c->mask_scratch, scratch_bytes);
            c->mask_scratch = nullptr;
        }
        if (new_buf) {
            dev_free(c, c->mask_buf, (size_t)c->N);
            c->mask_buf = nullptr;
        }
        return LB_ERR_NOMEM;
    }
    int rc = LB_OK;
    if (ptr_kind == LB_HOST) {
        rc = copy(c, c->mask_buf, mask, (size_t)c->N, cudaMemcpyHostToDevice);
        *mask_d = c->mask_buf;
    } else {
        *mask_d = mask;
    }
    if (!rc) rc = lbk::launch_mask_scan(c, *mask_d, c->mask_scratch);
    int tot = 0;
    if (!rc) rc = copy(c, &tot, c->mask_scratch + lbk::masked_total_offset(c->N), sizeof(int), cudaMemcpyDeviceToHost);
    if (!rc) rc = sync(c);
    *total = tot;
    return rc;
}

int lb_moments_masked(lb_ctx *c, const unsigned char *mask, double *rho, double *u, double *phi, long long *count,
                      int ptr_kind)
{
    if (!c || !mask || (ptr_kind != LB_HOST && ptr_kind != LB_DEVICE)) return LB_ERR_INVALID;
    const unsigned char *mask_d = nullptr;
    long long total = 0;
    int rc = masked_prepare(c, mask, ptr_kind, &mask_d, &total);
    if (rc) return rc;
    if (count) *count = total;
    if (total == 0 || (!rho && !u && !phi)) return LB_OK;
    if (ptr_kind == LB_DEVICE) return lbk::launch_masked_moments(c, total, c->mask_scratch, rho, u, phi);
    rc = ensure_io(c);
    if (rc) return rc;
    const size_t nb = (size_t)total * sizeof(double);
    // rho and u through the staging buffer (4 total values), then phi
    if (rho || u) {
        rc = lbk::launch_masked_moments(c, total, c->mask_scratch, c->io, c->io + total, nullptr);
        if (!rc && rho) rc = copy(c, rho, c->io, nb, cudaMemcpyDeviceToHost);
        if (!rc && u) rc = copy(c, u, c->io + total, 3 * nb, cudaMemcpyDeviceToHost);
        if (!rc) rc = sync(c);
    }
    if (!rc && phi) {
        rc = lbk::launch_masked_moments(c, total, c->mask_scratch, nullptr, nullptr, c->io);
        if (!rc) rc = copy(c, phi, c->io, nb, cudaMemcpyDeviceToHost);
        if (!rc) rc = sync(c);
    }
    return rc;
}

// rows of f (which = 0) or g (1) between the lattice and [19][total] arrays
static int masked_state(lb_ctx *c, const unsigned char *mask, double *f, double *g, const double *fin,
                        const double *gin, long long *count, int ptr_kind, int to_device_state)
{
    if (!c || !mask || (ptr_kind != LB_HOST && ptr_kind != LB_DEVICE) || c->reduced) return LB_ERR_INVALID;
    const unsigned char *mask_d = nullptr;
    long long total = 0;
    int rc = masked_prepare(c, mask, ptr_kind, &mask_d, &total);
    if (rc) return rc;
    if (count) *count = total;
    if (total == 0) return LB_OK;
    double *out[2] = {f, g};
    const double *in[2] = {fin, gin};
    if (ptr_kind == LB_DEVICE) {
        for (int which = 0; which < 2 && !rc; which++) {
            double *buf = to_device_state ? const_cast<double *>(in[which]) : out[which];
            if (buf) rc = lbk::launch_masked_rows(c, total, c->mask_scratch, which, 0, lbk::Q, buf, to_device_state);
        }
        return rc;
    }
    rc = ensure_io(c);
    if (rc) return rc;
    const size_t T = (size_t)total;
    for (int which = 0; which < 2 && !rc; which++) {
        if (to_device_state ? !in[which] : !out[which]) continue;
        for (int i0 = 0; i0 < lbk::Q && !rc; i0 += 4) {   // 4 rows of total values fit the 4N staging buffer
            const int i1 = i0 + 4 < lbk::Q ? i0 + 4 : lbk::Q;
            const size_t bytes = (size_t)(i1 - i0) * T * sizeof(double);
            if (to_device_state) {
                rc = copy(c, c->io, in[which] + (size_t)i0 * T, bytes, cudaMemcpyHostToDevice);
                if (!rc) rc = lbk::launch_masked_rows(c, total, c->mask_scratch, which, i0, i1, c->io, 1);
            } else {
                rc = lbk::launch_masked_rows(c, total, c->mask_scratch, which, i0, i1, c->io, 0);
                if (!rc) rc = copy(c, out[which] + (size_t)i0 * T, c->io, bytes, cudaMemcpyDeviceToHost);
            }
            if (!rc) rc = sync(c);
        }
    }
    return rc;
}

int lb_get_state_masked(lb_ctx *c, const unsigned char *mask, double *f, double *g, long long *count, int ptr_kind)
{
    return masked_state(c, mask, f, g, nullptr, nullptr, count, ptr_kind, 0);
}

int lb_set_state_masked(lb_ctx *c, const unsigned char *mask, const double *f, const double *g, int ptr_kind)
{
    return masked_state(c, mask, nullptr, nullptr, f, g, nullptr, ptr_kind, 1);
}

}  // extern "C"
