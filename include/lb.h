/*
 * lb.h -- C ABI of the GB300 (sm_103a) binary-fluid lattice Boltzmann library.
 *
 * One timestep of the symmetric binary fluid on a periodic D3Q19 lattice:
 * phi = sum_i g_i, 7-point finite differences of phi, the fused BGK collision
 * of the density distribution f (equilibrium carrying the free-energy
 * pressure tensor) and of the order-parameter distribution g (equilibrium
 * carrying Gamma*mu, mu = A phi + B phi^3 - kappa lap phi), then streaming.
 * This is the "binary collision" benchmark of targetDP (Gray & Stratford,
 * 2014), Sec. IV: an LB collision on a mixture of two fluids with inner
 * extents 19 (momenta) and 3 (dimensions), on a lattice whose order parameter
 * is advanced by finite differences (Sec. II.A).  The paper prints no
 * equations; the model is written out beside lb_step below.
 *
 * The library surface restates the paper's host API (Sec. III.B memory
 * management: targetMalloc / copyToTarget / copyFromTarget /
 * copyConstant<X>ToTarget; Sec. III.C execution: TARGET_LAUNCH / syncTarget)
 * as a stateful context: the library owns the device-side lattice (the
 * paper's "target copy", Sec. III.A) and the caller owns every host or device
 * array it passes in.
 *
 * Conventions (all entry points):
 *  - Return LB_OK (0) on success or a negative LB_ERR_* code; nothing aborts.
 *    lb_strerror() names a code, lb_last_error() gives the last CUDA error
 *    text seen by the calling thread.
 *  - Sites are ordered x fastest: s = x + nx*(y + ny*z), N = nx*ny*nz.
 *    Scalar fields are double[N]; vector fields are SoA double[3][N];
 *    distributions are SoA double[19][N] (value i of site s at i*N + s).
 *  - Every array crossing the ABI is FP64 whatever the storage precision.
 *  - ptr_kind says where a caller array lives: LB_HOST (pageable or pinned
 *    host memory) or LB_DEVICE (device memory of the context's GPU).
 *  - Work is ordered on the CUDA stream given at creation (NULL = the legacy
 *    default stream).  Calls that return host data synchronise that stream;
 *    calls on device pointers do not.
 *  - A context must not be used from two threads at once.
 *
 * Velocity order of the distributions at the ABI (i: c_i, weight w_i):
 *    0: ( 0, 0, 0) 1/3
 *    1: (+1, 0, 0)  2: (-1, 0, 0)  3: ( 0,+1, 0)  4: ( 0,-1, 0)
 *    5: ( 0, 0,+1)  6: ( 0, 0,-1)                               1/18
 *    7: (+1,+1, 0)  8: (-1,-1, 0)  9: (+1,-1, 0) 10: (-1,+1, 0)
 *   11: (+1, 0,+1) 12: (-1, 0,-1) 13: (+1, 0,-1) 14: (-1, 0,+1)
 *   15: ( 0,+1,+1) 16: ( 0,-1,-1) 17: ( 0,+1,-1) 18: ( 0,-1,+1)  1/36
 * Odd i and i+1 are opposite velocities.
 */
#ifndef LB_H
#define LB_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
    LB_OK = 0,
    LB_ERR_INVALID = -1,   /* bad argument, size or state                     */
    LB_ERR_NOMEM = -2,     /* device allocation failed                        */
    LB_ERR_CUDA = -3,      /* a CUDA call failed; see lb_last_error()         */
    LB_ERR_NONFINITE = -4, /* a reduction found NaN or Inf in the state       */
    LB_ERR_TIMEOUT = -5    /* a bounded device-side wait gave up              */
};

/* Storage/arithmetic precision of the distributions. */
enum {
    LB_FP64 = 0,          /* f, g stored and computed in double               */
    LB_FP32_SHIFTED = 1,  /* float storage and arithmetic of f_i - w_i rho0
                             and of g_i; FP64 only in lb_reduce's sums         */
    LB_FP64_DF = 2        /* double-float: each value stored and computed as
                             an unevaluated sum of two floats (~48 bits,
                             unit roundoff ~2^-48), on the FP32 units; the
                             default two-pass step and the tau_g = 1 reduced
                             form only (LB_KERNEL_AUTO / _TWO_PASS / _TAUG1),
                             not in ensembles or the adjoint                 */
};

enum { LB_HOST = 0, LB_DEVICE = 1 };

/* Step kernels selectable with lb_set_kernel(). */
enum {
    LB_KERNEL_AUTO = 0,     /* library default, the fastest measured on GB300:
                               LB_KERNEL_BULK (3 slots, clusters of 2, 16
                               planes) for FP32-shifted 7-point BGK steps on
                               rows of 256 sites with ny even, else
                               LB_KERNEL_TWO_PASS                            */
    LB_KERNEL_TWO_PASS = 1, /* phi pass + collide/stream pass (phi buffer)     */
    LB_KERNEL_FUSED = 2,    /* single pass, phi halo staged in shared memory   */
    LB_KERNEL_STAGED = 3,   /* single pass, planes staged by asynchronous
                               copies into a 3-buffer shared-memory pipeline   */
    LB_KERNEL_SLAB = 4,     /* single pass, per z-slab: phi of the slab into
                               shared memory, then a barrier-free collision    */
    LB_KERNEL_LAG = 5,      /* single pass, lagged pipeline: the CTA with
                               ticket c computes phi of site block c and
                               collides block c - D; bounded waits            */
    LB_KERNEL_TAUG1 = 6,    /* tau_g = 1 only: g kept as phi and (gmh, u),
                               whose equilibria it is exactly; 49 words/site  */
    LB_KERNEL_BULK = 7      /* single pass, one CTA per x-row marching z: the
                               19 pulled g rows of each plane copied into
                               shared memory by bulk asynchronous copies (g
                               read from HBM once), phi rows shared along y
                               in a thread-block cluster; FP64 or
                               FP32-shifted, nx * element size a multiple of
                               16 bytes, nx <= 256                            */
};

/* Collision of f, lb_set_collision(). */
enum {
    LB_COLLISION_BGK = 0,   /* single relaxation time tau (default)            */
    LB_COLLISION_MRT = 1    /* shear stress at 1/tau, bulk stress at
                               1/tau_bulk, the 9 ghost modes at 1/tau_ghost    */
};

typedef struct lb_ctx lb_ctx;

/* Physical and lattice parameters of one periodic lattice. */
typedef struct {
    int nx, ny, nz;   /* lattice extents, each >= 1                         */
    double tau;       /* BGK relaxation time of f, > 1/2                    */
    double tau_g;     /* relaxation time of g, > 1/2                        */
    double rho0;      /* reference density (initial rho; the FP32 shift)    */
    double gamma;     /* mobility parameter Gamma                           */
    double A, B;      /* bulk free-energy coefficients                      */
    double kappa;     /* interfacial (gradient) coefficient                 */
    int precision;    /* LB_FP64 or LB_FP32_SHIFTED                         */
} lb_params;

/* Optional device allocator (e.g. a framework's caching allocator).
 * alloc returns a device pointer of at least `bytes` (256-byte aligned) or
 * NULL; free releases it.  `stream` is the context's stream. */
typedef void *(*lb_alloc_fn)(size_t bytes, void *stream, void *user);
typedef void (*lb_free_fn)(void *ptr, size_t bytes, void *stream, void *user);

/* Install the allocator used by contexts created afterwards (process-wide;
 * both NULL restores cudaMalloc/cudaFree).  A context keeps the allocator it
 * was created with.  Returns LB_ERR_INVALID if exactly one of the two is NULL.
 * Paper: targetMalloc / targetFree, Sec. III.B. */
int lb_set_allocator(lb_alloc_fn alloc, lb_free_fn free_fn, void *user);

/* Create a context: validates *p, allocates the two double-buffered SoA
 * distribution arrays (2 x 2 x 19 x N values of 8 or 4 bytes) plus an N-site
 * phi buffer and reduction scratch on the current CUDA device.  The state is
 * undefined until lb_init or lb_set_state.  *out receives the context.
 * Errors: LB_ERR_INVALID (NULL pointer, extent < 1, N >= 2^31, tau or tau_g
 * <= 1/2, rho0 <= 0, unknown precision), LB_ERR_NOMEM, LB_ERR_CUDA.
 * Paper: targetMalloc, Sec. III.B. */
int lb_create(const lb_params *p, void *cuda_stream, lb_ctx **out);

/* Release every device buffer of c (NULL is a no-op).  Synchronises c's
 * stream first.  Paper: targetFree, Sec. III.B. */
void lb_destroy(lb_ctx *c);

/* Initial state: rho = rho0, u = u0 (u0 == NULL: fluid at rest), phi = phi0;
 * the stencils of phi0 (lb_set_stencil; 7 points by default) give mu and the
 * pressure tensor, and f, g are
 * set to their equilibria (computed in FP64, then stored in the context's
 * precision).  phi0 is double[N], u0 SoA double[3][N], both in ptr_kind
 * memory; they are read before the call returns (LB_HOST) or before later
 * work on the stream (LB_DEVICE).  Errors: LB_ERR_INVALID, LB_ERR_CUDA.
 * Paper: copyToTarget, Sec. III.B. */
int lb_init(lb_ctx *c, const double *phi0, const double *u0, int ptr_kind);

/* Advance nsteps (>= 0) timesteps, asynchronously on the context's stream.
 * One timestep, per site x (all arithmetic in the context's precision):
 *   phi = sum_i g_i;  d_a phi = (phi(x+e_a) - phi(x-e_a))/2;
 *   lap phi = sum of the 6 face neighbours - 6 phi(x);
 *   rho = sum_i f_i;  u = sum_i f_i c_i / rho;
 *   mu = A phi + B phi^3 - kappa lap phi;
 *   P_ab = [A/2 phi^2 + 3B/4 phi^4 - kappa phi lap phi - kappa/2 |grad phi|^2]
 *          delta_ab + kappa d_a phi d_b phi;
 *   feq_i = w_i [rho + 3 rho c_i.u + 9/2 (P + rho u u):(c_i c_i - I/3)];
 *   geq_i = w_i [phi + 3 phi c_i.u
 *               + 9/2 ((Gamma mu - phi/3) I + phi u u):(c_i c_i - I/3)];
 *   f*_i = f_i - (f_i - feq_i)/tau;  g*_i = g_i - (g_i - geq_i)/tau_g;
 *   f_i(x + c_i, t+1) = f*_i(x, t), likewise g (periodic wrap).
 * Errors: LB_ERR_INVALID (c NULL, nsteps < 0), LB_ERR_CUDA.
 * Paper: the binary-collision benchmark, Sec. IV; TARGET_LAUNCH, Sec. III.C. */
int lb_step(lb_ctx *c, int nsteps);

/* Moments of the current state: rho[N], u[3][N] (SoA, = sum f c / rho) and
 * phi[N], written in FP64 to ptr_kind memory; any output may be NULL.
 * LB_HOST synchronises the stream before returning.  Errors: LB_ERR_INVALID,
 * LB_ERR_CUDA.  Paper: copyFromTarget, Sec. III.B. */
int lb_moments(lb_ctx *c, double *rho, double *u, double *phi, int ptr_kind);

/* Lattice totals out[5] = {sum rho, sum rho u_x, sum rho u_y, sum rho u_z,
 * sum phi} (host array), accumulated in FP64 on the GPU in a fixed order
 * (bitwise reproducible).  Synchronises the stream.  Returns
 * LB_ERR_NONFINITE (with out filled) if any total is NaN or Inf.
 * Paper: reductions are named as future work in Sec. V. */
int lb_reduce(lb_ctx *c, double out[5]);

/* Copy the full state out / in as post-streaming distributions f(x, t),
 * g(x, t): double[19][N] each, in the ABI velocity order, ptr_kind memory.
 * lb_get_state with LB_HOST synchronises.  These are the checkpoint /
 * restart entry points.  Errors: LB_ERR_INVALID, LB_ERR_CUDA.
 * Paper: copyFromTarget / copyToTarget, Sec. III.B. */
int lb_get_state(lb_ctx *c, double *f, double *g, int ptr_kind);
int lb_set_state(lb_ctx *c, const double *f, const double *g, int ptr_kind);

/* Masked copy-out: the moments (as lb_moments) of the sites whose mask byte
 * is non-zero, compacted in site order: rho[count], u[3][count] (row stride
 * count), phi[count].  mask is unsigned char[N] in ptr_kind memory, as are
 * the outputs, which must hold at least count values per row (N always
 * suffices); any output may be NULL.  *count (host, may be NULL) receives
 * the number of selected sites.  Synchronises the stream (the count is read
 * back).  Works in every kernel form.  Errors: LB_ERR_INVALID, LB_ERR_NOMEM,
 * LB_ERR_CUDA.  Paper: copyFromTargetMasked, Sec. III.B (a stream compaction
 * on the GPU). */
int lb_moments_masked(lb_ctx *c, const unsigned char *mask, double *rho, double *u, double *phi,
                      long long *count, int ptr_kind);

/* Masked state I/O: the post-streaming f, g (as lb_get_state) of the
 * selected sites as double[19][count] each (row stride count), and the
 * inverse, which overwrites only the selected sites.  Refused
 * (LB_ERR_INVALID) in the tau_g = 1 reduced form.  Synchronise the stream.
 * Paper: copyFromTargetMasked / copyToTargetMasked, Sec. III.B. */
int lb_get_state_masked(lb_ctx *c, const unsigned char *mask, double *f, double *g, long long *count,
                        int ptr_kind);
int lb_set_state_masked(lb_ctx *c, const unsigned char *mask, const double *f, const double *g, int ptr_kind);

/* Select the step kernel (LB_KERNEL_*) and its launch shape: block_x x
 * block_y threads per CTA and z_chunk planes per CTA of the fused, staged
 * and slab kernels (0 = library default for any of the three).  For
 * LB_KERNEL_AUTO and LB_KERNEL_TWO_PASS block_x is the threads per CTA of
 * both passes (a multiple of 32 up to 256; 0 = 256), block_y the sites per
 * thread of the phi pass (1, 2 or 4; 0 = 1) and z_chunk must be 0.  For
 * LB_KERNEL_LAG block_x must be 0 or 256, block_y 0 or 1, and z_chunk is the
 * lag slack in site blocks beyond the stencil's reach (0 = default 128).
 * For LB_KERNEL_BULK block_x is the number of shared-memory plane slots of
 * g (3..8, or 2 in FP32: the lean form, no copies ahead, three CTAs per SM;
 * 0 = 3), block_y the CTAs per cluster along
 * y (1, 2, 4 or 8, dividing ny; 0 = 4) and z_chunk the planes each CTA
 * marches (0 = 32).
 * LB_KERNEL_TAUG1 requires tau_g == 1 (LB_ERR_INVALID otherwise) and
 * converts the stored state to its reduced form (selecting another kernel
 * converts back); its phi pass takes block_x y rows per warp (1, 2 or 4;
 * 4 not in LB_FP64_DF; 0 = 1 in FP32, 2 otherwise), block_y warps per CTA
 * (1..8; 0 = 4) and z_chunk planes per warp (0 = sized for about three
 * waves of CTAs; cut to nz).  In that form lb_set_state keeps g only through
 * phi = sum_i g_i (all the tau_g = 1 dynamics uses) and lb_get_state reports
 * g as the streamed equilibria of the previous step (after lb_init or
 * lb_set_state: the equilibrium at each site).  Ensemble members refuse
 * lb_set_kernel.  Validated against the
 * kernel's limits; LB_ERR_INVALID otherwise.  Paper: the tunable VVL and TPB
 * of TARGET_TLP / TARGET_LAUNCH, Sec. III.C. */
int lb_set_kernel(lb_ctx *c, int kernel, int block_x, int block_y, int z_chunk);

/* Points of the finite-difference stencils of phi (gradient and Laplacian)
 * used by later lb_init and lb_step calls: 7 (default) = nearest faces,
 * d_a phi = (phi(x + e_a) - phi(x - e_a))/2, lap phi = sum of the 6 face
 * neighbours - 6 phi(x); 19 or 27 = the isotropic lattice-weighted
 * differences d_a phi = 3 sum_c W_c c_a phi(x + c),
 * lap phi = 6 sum_c W_c (phi(x + c) - phi(x)) over the D3Q19 (W = 1/18
 * faces, 1/36 edges) or D3Q27 (2/27, 1/54, 1/216 corners) neighbourhood.
 * The stored state is unchanged.  19 and 27 run on LB_KERNEL_AUTO,
 * LB_KERNEL_TWO_PASS and LB_KERNEL_TAUG1; LB_ERR_INVALID for another
 * points value, for the other kernels (now or in a later lb_set_kernel), for
 * ensemble members, and lb_adjoint_* refuse contexts set to 19 or 27.
 * Paper: the "standard finite-difference" order-parameter update, Sec. II.A
 * (which names no stencil). */
int lb_set_stencil(lb_ctx *c, int points);

/* Collision of f used by later lb_step calls: LB_COLLISION_BGK (tau_bulk and
 * tau_ghost ignored) or LB_COLLISION_MRT, the multiple-relaxation-time
 * collision defined by projections onto the second-order Hermite space of
 * D3Q19: with N = sum (f - feq) c c split into bulk ((tr N/3) I) and
 * traceless shear parts, the shear part relaxes at 1/tau (shear viscosity
 * (tau - 1/2)/3), the bulk part at 1/tau_bulk (bulk viscosity
 * (2/9)(tau_bulk - 1/2)) and the 9 ghost directions (orthogonal to 1, c and
 * c c) at 1/tau_ghost; with all three equal it is BGK.  g keeps its BGK
 * collision (tau_g).  Requires tau_bulk, tau_ghost > 1/2, a kernel that is
 * LB_KERNEL_AUTO or LB_KERNEL_TWO_PASS (others, now or in a later
 * lb_set_kernel, give LB_ERR_INVALID), not an ensemble member; lb_adjoint_*
 * refuse MRT contexts.  Paper: the "binary collision" kernel's collision
 * operator, Sec. IV (BGK is its form; MRT is Ludwig's other). */
int lb_set_collision(lb_ctx *c, int model, double tau_bulk, double tau_ghost);

/* Uniform body force density F applied by Guo's scheme from the next
 * lb_step: u = (sum f c + F/2)/rho enters the equilibria and lb_moments'
 * velocity, the momentum of every site grows by F per step, and the
 * second-order force terms relax with (1 - w/2) of the shear and bulk rates
 * (with BGK, of 1/tau).  lb_reduce's momentum is sum f c (without F/2).
 * (0, 0, 0) switches it off.  Same kernel, ensemble and adjoint limits as
 * LB_COLLISION_MRT.  Paper: no counterpart (a NEXT extension of the
 * collision). */
int lb_set_force(lb_ctx *c, double fx, double fy, double fz);

/* Synchronise the context's stream; returns LB_ERR_TIMEOUT if a bounded
 * device-side wait (the lagged kernel's inter-CTA waits) gave up since the
 * last synchronising call -- the state is then invalid until lb_init or
 * lb_set_state -- else LB_OK or LB_ERR_CUDA.  Every call that synchronises
 * (host-pointer lb_moments / lb_get_state / lb_set_state / lb_init,
 * lb_reduce) reports such a timeout the same way.
 * Paper: syncTarget (cudaThreadSynchronize with error checking), Sec. III.C. */
int lb_sync(lb_ctx *c);

/* Upper bound, in nanoseconds (1e3 .. 6e10), of every device-side wait of
 * the context (default 1e9).  Paper: no counterpart (the paper's kernels
 * never wait on one another). */
int lb_set_wait_timeout(lb_ctx *c, long long timeout_ns);

/* Test hook: add `skew` to the lagged kernel's wait targets so that no wait
 * can be satisfied and every one runs into its time bound (the timeout path
 * without a GPU fault); with LB_KERNEL_BULK any non-zero skew makes every
 * CTA's copy producer stop after its first plane, so the consumers' waits
 * run into their bound.  0 restores normal operation.  Paper: no
 * counterpart. */
int lb_debug_wait_skew(lb_ctx *c, unsigned long long skew);

/* One FP64 timestep that allocates no device memory, for callers that
 * cannot allocate: a host application whose device memory is entirely
 * reserved by its own allocator, or a latency-critical loop that must never
 * enter cudaMalloc/cudaFree (which can block the whole device).  The paper
 * has no counterpart.
 *   p       lattice and model parameters; p->precision must be LB_FP64 and
 *           nx*ny*nz at most 262144 (64^3), else LB_ERR_INVALID.
 *   fa, ga  input: device double[19][N] (ABI velocity order, site s =
 *           x + nx*(y + ny*z)) holding the post-collision values of the
 *           previous timestep, i.e. the post-streaming state is
 *           f_i(x, t) = fa[i*N + site(x - c_i)] (likewise g).
 *   fb, gb  output, same layout and convention for time t+1; neither may
 *           share a byte with the other output or with an input
 *           (LB_ERR_INVALID); the inputs may overlap each other.
 *   cuda_stream  stream the work is queued on (NULL = legacy default);
 *           the call returns before the work runs.
 * The arithmetic is lb_step's two-pass kernel pair.  The order parameter
 * between the two passes lives in one fixed device array of 262144 doubles
 * (2 MiB) inside the library, held by every GPU that loads it until the
 * process exits and shared by all calls: calls that overlap on the GPU race
 * on it.  Each call writes every value of it that it reads, so nothing needs
 * clearing between calls.  The first call on a device looks up that array's
 * device address (set-up); make that first call before any stream capture.
 * Errors: LB_ERR_INVALID, LB_ERR_CUDA. */
int lb_step_fp64_noalloc(const lb_params *p, const double *fa, const double *ga, double *fb, double *gb,
                         void *cuda_stream);

/* ---- Reverse mode (adjoint) of the FP64 timestep ----
 * For gradients of a loss on the state at time T with respect to the
 * initial order parameter and kappa (back-propagation through time).
 * States and adjoints use the ABI convention: device double[19][N] arrays,
 * post-streaming, ABI velocity order.  Contexts must be LB_FP64.  The adjoint
 * scratch (6 N doubles) is allocated on first use.  Paper: no counterpart
 * (the method's own gradients are not in the paper).
 *
 * One reverse step: given F(t) = (f, g) and F_bar(t+1) = (af_in, ag_in),
 * writes F_bar(t) = (af_out, ag_out) (must not alias the inputs) and adds
 * this step's dJ/dkappa to *dkappa (a device double).  It transposes, in
 * order, the streaming, the collision (with the stress, mu and u = j/rho
 * recomputed from F(t)), the 7-point stencils and phi = sum g. */
int lb_adjoint_step(lb_ctx *c, const double *f, const double *g, const double *af_in, const double *ag_in,
                    double *af_out, double *ag_out, double *dkappa);

/* Start of the reverse sweep for a loss on phi_T = sum_i g_i(T) (the
 * order parameter read out at time T): given dJ/dphi_T (device double[N]),
 * writes F_bar(T) = (af, ag), device double[19][N] each: af = 0 and
 * ag[i*N + s] = phi_bar[s] for every i (the transpose of the sum over i).
 * Errors: LB_ERR_INVALID (NULL pointers, af == ag, not LB_FP64),
 * LB_ERR_CUDA. */
int lb_adjoint_seed(lb_ctx *c, const double *phi_bar, double *af, double *ag);

/* Reverse of lb_init: given F_bar(0) = (af0, ag0), writes dJ/dphi0 to
 * phi0_bar (device double[N]) and adds the initialisation's dJ/dkappa to
 * *dkappa.  phi0 and u0 (NULL = fluid at rest) are device arrays as in
 * lb_init. */
int lb_adjoint_init(lb_ctx *c, const double *phi0, const double *u0, const double *af0, const double *ag0,
                    double *phi0_bar, double *dkappa);

/* ---- Ensembles: many independent lattices in one persistent launch ----
 * An ensemble holds n lattices of any extents and parameters (one precision
 * for all).  lb_batch_run advances every lattice by nsteps timesteps with
 * one cooperative (co-resident) kernel launch that loops over the steps and
 * over a (lattice, block of sites) work list.  The grid is split into CTA
 * groups by lb_batch_plan: each group advances its own lattices with a
 * barrier of its CTAs alone between the phi pass and the collide/stream
 * pass, so lattices never wait for one another.  The launch is captured in
 * a CUDA graph (one per step count and parity) and replayed.  Per-site
 * arithmetic is exactly lb_step's.  Paper: the tunable thread-block size
 * TPB and per-thread work of TARGET_LAUNCH / TARGET_TLP, Sec. III.C. */
typedef struct lb_batch lb_batch;

/* Create an ensemble of n lattices with parameters p[0..n-1] (same
 * precision), work ordered after cuda_stream.  Errors as lb_create. */
int lb_batch_create(int n, const lb_params *p, void *cuda_stream, lb_batch **out);

/* Free the ensemble and all its lattices (NULL is a no-op). */
void lb_batch_destroy(lb_batch *b);

/* Lattice k of the ensemble as a context for lb_init, lb_moments,
 * lb_reduce, lb_get_state, lb_set_state and lb_sync (NULL if k is out of
 * range).  It belongs to the ensemble: lb_step on it returns LB_ERR_INVALID
 * and lb_destroy ignores it. */
lb_ctx *lb_batch_lattice(lb_batch *b, int k);

/* Advance every lattice by nsteps (>= 0), asynchronously after the work
 * queued on the ensemble's stream.  Errors: LB_ERR_INVALID, LB_ERR_CUDA;
 * a group barrier that timed out is reported by lb_batch_sync (or lb_sync
 * of any member) as LB_ERR_TIMEOUT, after which the states are invalid
 * until re-initialised. */
int lb_batch_run(lb_batch *b, int nsteps);

/* Synchronise; LB_ERR_TIMEOUT if a group barrier gave up since the last
 * check (the flag is then cleared). */
int lb_batch_sync(lb_batch *b);

/* Launch shape: threads per CTA (= sites per work item; multiple of 32, at
 * most 256) and CTAs per SM (0 = as many as fit; the grid is
 * always co-resident).  Paper: TPB and VVL tuning, Sec. III.C and IV. */
int lb_batch_set_launch(lb_batch *b, int threads, int ctas_per_sm);

/* Form of the ensemble's step: 0 = the general two-pass step (default), 1 =
 * the tau_g = 1 reduced form of LB_KERNEL_TAUG1 for every lattice (g kept as
 * phi and (gmh, u); the collide pass over the same site blocks, then the phi
 * pass over tiles of 30 x-columns, 32/threads-per-CTA warps of rows and 8
 * z planes).  Converts every member's stored state (lb_get_state /
 * lb_moments of a member report the same state before and after).
 * LB_ERR_INVALID unless every lattice has tau_g == 1.  Synchronises.
 * Paper: no counterpart (the tau_g = 1 form of the collision). */
int lb_batch_set_form(lb_batch *b, int reduced);

/* n lattices, work items per pass, CTAs in the grid, threads per CTA. */
int lb_batch_size(const lb_batch *b, int *n, int *work_items, int *grid, int *threads);

/* CTA plan of the ensemble (lb_batch_plan's bins): 0 = a group of CTAs per
 * lattice (default), 1 = one group of all CTAs walking the whole work list
 * with a grid-wide barrier between the passes, k >= 2 = k groups of whole
 * lattices balanced by work.  Same results for every plan.  Synchronises.
 * Paper: no counterpart. */
int lb_batch_set_plan(lb_batch *b, int bins);

/* Number of CTA groups of the ensemble's current plan. */
int lb_batch_groups(const lb_batch *b, int *ngroups);

/* The CTA plan of an ensemble (host only; needs no GPU): n lattices with
 * items[k] >= 1 work items per pass over ctas >= 1 co-resident CTAs.
 *  - The groups: bins = 0 and n <= ctas: lattice k is group k.  bins = 0
 *    and n > ctas: ctas groups.  bins >= 1: min(bins, n, ctas) groups.  In
 *    the last two cases the lattices, largest first (stable), each go to the
 *    group with the least work so far (ties to the lower group).
 *  - The CTAs: every group starts with one; each further CTA goes to the
 *    group with the largest per-CTA share ceil(work / CTAs) (ties to the
 *    lower index) until the CTAs run out or every share is 1 (the CTAs left
 *    over stay idle).
 * Outputs (host arrays): group[k] (n entries) and, per group g, its first
 * CTA cta0[g] and CTA count m[g] (min(n, ctas) entries; groups occupy
 * consecutive CTAs from 0); *ngroups.  LB_ERR_INVALID on a bad argument. */
int lb_batch_plan(int n, const long long *items, int ctas, int bins, int *group, int *cta0, int *m,
                  int *ngroups);

/* Bound (ns) of every group-barrier wait (default 1e9). */
int lb_batch_set_wait_timeout(lb_batch *b, long long timeout_ns);

/* Test hook: the first CTA of the largest group leaves before the group's
 * first barrier, so the group's other CTAs run into the time bound of their
 * wait (the timeout path without a GPU fault); lb_batch_run returns
 * LB_ERR_INVALID while the hook is on and no group has two CTAs.  0
 * restores normal operation.  Paper: no counterpart. */
int lb_batch_debug_skip_arrival(lb_batch *b, int enable);

/* Measurement helper: queue on cuda_stream one launch of `blocks` CTAs of
 * 256 threads that do nothing but independent FP64 fused multiply-adds
 * (16 chains of `iters` each per thread; iters a positive multiple of 4,
 * at most 2^30), for timing the FP64 pipe's peak with events around the
 * call; *flops_out (host) receives the launch's flop count (2 per FMA).  sink: device double[blocks], written only if a
 * chain's sum hits an impossible value (it keeps the work alive).  Errors:
 * LB_ERR_INVALID, LB_ERR_CUDA.  Paper: no counterpart (the FP64 roofline
 * of the timestep). */
int lb_probe_fp64_fma(int blocks, long long iters, double *sink, void *cuda_stream, double *flops_out);

/* Extents and precision of c (any output may be NULL). */
int lb_get_info(const lb_ctx *c, int *nx, int *ny, int *nz, int *precision);

/* Text of an LB_* code, and of the last CUDA error seen by this thread. */
const char *lb_strerror(int code);
const char *lb_last_error(void);

#ifdef __cplusplus
}
#endif

#endif /* LB_H */
