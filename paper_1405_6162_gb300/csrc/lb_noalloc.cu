// lb_noalloc.cu -- an FP64 timestep that allocates no device memory.
//
// Some callers cannot allocate device memory when they want to step a
// lattice: a host application whose device memory is entirely reserved by
// its own allocator (so a cudaMalloc from a library would fail or fragment
// it), or a latency-critical loop that must never enter cudaMalloc/cudaFree,
// which can block the whole device.  lb_step_fp64_noalloc serves them: the
// caller passes every input and output buffer, and the only scratch the step
// needs -- the order parameter phi of one lattice, written by the phi pass and
// read by the collision pass -- lives in a fixed array of this file, placed in
// device memory when the library is loaded and kept by every GPU that loads
// it until the process exits.
#include <cuda_runtime.h>

#include <cmath>
#include <mutex>

#include "d3q19.cuh"
#include "lb_internal.cuh"

namespace {

// Largest lattice (sites) the fixed scratch can serve: 64^3 sites of phi.
constexpr long long kNoAllocMaxSites = 262144;

// The scratch itself.  Every call uses the same array: each call writes the
// whole part it reads (phi of every site) before reading it, so nothing has
// to start at zero, and calls that overlap on the GPU race on it.
static __device__ __align__(256) double g_phi_scratch[kNoAllocMaxSites];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
double *g_scratch_ptr[kMaxDevices] = {};

// Device address of g_phi_scratch on the current device.  In host code the
// array's name is only a host-side stand-in, so its device address is looked
// up once per device (with that device current) and cached.
int scratch_address(double **out)
{
    int dev = 0;
    int rc = lbk::cuda_status(cudaGetDevice(&dev));
    if (rc) return rc;
    if (dev < 0 || dev >= kMaxDevices) return LB_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_scratch_ptr[dev]) {
        void *p = nullptr;
        rc = lbk::cuda_status(cudaGetSymbolAddress(&p, g_phi_scratch));
        if (rc) return rc;
        g_scratch_ptr[dev] = static_cast<double *>(p);
    }
    *out = g_scratch_ptr[dev];
    return LB_OK;
}

// [a, a + bytes) and [b, b + bytes) share a byte
bool overlap(const void *a, const void *b, size_t bytes)
{
    const char *x = static_cast<const char *>(a), *y = static_cast<const char *>(b);
    return x < y + bytes && y < x + bytes;
}

bool valid(const lb_params *p)
{
    if (!p || p->nx < 1 || p->ny < 1 || p->nz < 1) return false;
    const double v[] = {p->tau, p->tau_g, p->rho0, p->gamma, p->A, p->B, p->kappa};
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return p->tau > 0.5 && p->tau_g > 0.5 && p->rho0 > 0.0 && p->precision == LB_FP64;
}

}  // namespace

extern "C" int lb_step_fp64_noalloc(const lb_params *p, const double *fa, const double *ga, double *fb,
                                    double *gb, void *cuda_stream)
{
    if (!valid(p) || !fa || !ga || !fb || !gb) return LB_ERR_INVALID;
    const long long N = (long long)p->nx * p->ny * p->nz;
    if (N > kNoAllocMaxSites) return LB_ERR_INVALID;   // lattice larger than the fixed scratch
    // each output must share no byte with the other output or with an input
    // (the inputs are only read and may overlap each other)
    const size_t bytes = (size_t)lbk::Q * (size_t)N * sizeof(double);
    if (overlap(fb, gb, bytes) || overlap(fb, fa, bytes) || overlap(fb, ga, bytes) || overlap(gb, fa, bytes) ||
        overlap(gb, ga, bytes))
        return LB_ERR_INVALID;
    double *phi = nullptr;
    const int rc = scratch_address(&phi);
    if (rc) return rc;
    return lbk::launch_two_pass_fp64_raw(*p, fa, ga, phi, fb, gb, N, (cudaStream_t)cuda_stream);
}
