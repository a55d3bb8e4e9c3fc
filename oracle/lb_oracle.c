/*
 * lb_oracle.c -- plain, slow CPU oracle of the symmetric binary-fluid lattice
 * Boltzmann timestep on a periodic D3Q19 lattice.
 *
 * TEST INFRASTRUCTURE ONLY.  The test-suite, the package smoke check and the
 * benchmark's CPU-baseline leg are the only callers.  The CUDA library never
 * links, loads or calls this file and shares no code, table or header with it.
 *
 * The paper (Gray & Stratford, targetDP, 2014) benchmarks the "binary
 * collision" kernel of Ludwig: a lattice Boltzmann collision on a mixture of
 * two fluids (Sec. IV), with inner loops over the 19 discrete momenta and the
 * 3 spatial dimensions (Sec. IV), on a lattice whose order parameter is
 * advanced with "standard finite-difference techniques" (Sec. II.A).  The
 * paper prints no equations; this file follows the standard symmetric
 * free-energy model, read as:
 *
 *   free energy   F = A/2 phi^2 + B/4 phi^4 + kappa/2 |grad phi|^2
 *   chem. pot.    mu = A phi + B phi^3 - kappa lap phi
 *   pressure      P_ab = [A/2 phi^2 + 3B/4 phi^4 - kappa phi lap phi
 *                        - kappa/2 |grad phi|^2] delta_ab + kappa d_a phi d_b phi
 *   f equilibrium feq_i = w_i [rho + rho c.u/cs2 + S_ab Q_iab/(2 cs2^2)],
 *                 S = P + rho u u
 *   g equilibrium geq_i = w_i [phi + phi c.u/cs2 + G_ab Q_iab/(2 cs2^2)],
 *                 G = (Gamma mu - phi cs2) delta + phi u u
 *   BGK           f* = f - (f - feq)/tau,  g* = g - (g - geq)/tau_g
 *   streaming     f_i(x + c_i, t+1) = f*_i(x, t)
 *
 * with Q_iab = c_ia c_ib - cs2 delta_ab, cs2 = 1/3, u = sum_i f_i c_i / rho,
 * phi = sum_i g_i, and the 7-point stencils d_a phi = (phi(x+e_a) -
 * phi(x-e_a))/2, lap phi = sum of the 6 face neighbours - 6 phi(x).
 *
 * Distributions are stored SoA: value i of site s at f[i*N + s], with site
 * s = x + nx*(y + ny*z).  The velocity set is built by enumerating (cx,cy,cz)
 * in {-1,0,1}^3 in lexicographic order and keeping |c|^2 <= 2; callers map it
 * to any other ordering through orc_velocity_set().
 *
 * Compile as FP64 (default) or, with -DORC_COMPLEX, as a complex-step build in
 * which every field and parameter is "double complex" (every operation here is
 * analytic, so Im(L(p + ih))/h is dL/dp to rounding).
 */
#include <stdlib.h>
#include <string.h>

#ifdef ORC_COMPLEX
#include <complex.h>
typedef double complex real;
#else
typedef double real;
#endif

#define NV 19

/* layout of the parameter vector prm[] */
enum { P_TAU = 0, P_TAUG, P_RHO0, P_GAMMA, P_A, P_B, P_KAPPA, P_COUNT };

static int cv[NV][3];
static double wv[NV];
static int built = 0;

/* D3Q19: rest (w = 1/3), 6 faces (w = 1/18), 12 edges (w = 1/36). */
static void velocity_set(void)
{
    if (built) return;
    int n = 0;
    for (int a = -1; a <= 1; a++)
        for (int b = -1; b <= 1; b++)
            for (int c = -1; c <= 1; c++) {
                int c2 = a * a + b * b + c * c;
                if (c2 > 2) continue;
                cv[n][0] = a; cv[n][1] = b; cv[n][2] = c;
                wv[n] = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
                n++;
            }
    built = 1;
}

static long wrap(long a, long n) { return ((a % n) + n) % n; }

static long site(long x, long y, long z, int nx, int ny, int nz)
{
    return wrap(x, nx) + (long)nx * (wrap(y, ny) + (long)ny * wrap(z, nz));
}

int orc_nvel(void) { return NV; }

void orc_velocity_set(int *c, double *w)
{
    velocity_set();
    for (int i = 0; i < NV; i++) {
        for (int a = 0; a < 3; a++) c[3 * i + a] = cv[i][a];
        w[i] = wv[i];
    }
}

/* 7-point finite differences of phi on the periodic lattice. */
void orc_gradients(int nx, int ny, int nz, const real *phi, real *grad, real *lap)
{
    long N = (long)nx * ny * nz;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long s = site(x, y, z, nx, ny, nz);
                real xp = phi[site(x + 1, y, z, nx, ny, nz)];
                real xm = phi[site(x - 1, y, z, nx, ny, nz)];
                real yp = phi[site(x, y + 1, z, nx, ny, nz)];
                real ym = phi[site(x, y - 1, z, nx, ny, nz)];
                real zp = phi[site(x, y, z + 1, nx, ny, nz)];
                real zm = phi[site(x, y, z - 1, nx, ny, nz)];
                grad[0 * N + s] = (xp - xm) / 2.0;
                grad[1 * N + s] = (yp - ym) / 2.0;
                grad[2 * N + s] = (zp - zm) / 2.0;
                lap[s] = xp + xm + yp + ym + zp + zm - 6.0 * phi[s];
            }
}

/* Chemical potential and thermodynamic pressure tensor at one site. */
void orc_site_thermo(const real *prm, real phi, const real *d, real lap,
                     real *mu, real *P /* [3][3] */)
{
    real A = prm[P_A], B = prm[P_B], kappa = prm[P_KAPPA];
    *mu = A * phi + B * phi * phi * phi - kappa * lap;
    real dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    real pb = 0.5 * A * phi * phi + 0.75 * B * phi * phi * phi * phi
              - kappa * phi * lap - 0.5 * kappa * dd;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++)
            P[3 * a + b] = (a == b ? pb : 0.0) + kappa * d[a] * d[b];
}

/* Equilibria of f and g at one site, given rho, momentum j = rho u, phi and
 * its derivatives. */
void orc_site_equilibrium(const real *prm, real rho, const real *j, real phi,
                          const real *d, real lap, real *feq, real *geq)
{
    velocity_set();
    const double cs2 = 1.0 / 3.0;
    real u[3], mu, P[9], S[3][3], G[3][3];
    for (int a = 0; a < 3; a++) u[a] = j[a] / rho;
    orc_site_thermo(prm, phi, d, lap, &mu, P);
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            S[a][b] = P[3 * a + b] + rho * u[a] * u[b];
            G[a][b] = (a == b ? prm[P_GAMMA] * mu - phi * cs2 : 0.0) + phi * u[a] * u[b];
        }
    for (int i = 0; i < NV; i++) {
        real cu = 0.0, sq = 0.0, gq = 0.0;
        for (int a = 0; a < 3; a++) cu += cv[i][a] * u[a];
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double Q = cv[i][a] * cv[i][b] - (a == b ? cs2 : 0.0);
                sq += S[a][b] * Q;
                gq += G[a][b] * Q;
            }
        feq[i] = wv[i] * (rho + rho * cu / cs2 + sq / (2.0 * cs2 * cs2));
        geq[i] = wv[i] * (phi + phi * cu / cs2 + gq / (2.0 * cs2 * cs2));
    }
}

/* f = feq(rho0, rho0 u0, phi0), g = geq(...): the initial state.  u0 is SoA
 * [3][N] or NULL for a fluid at rest. */
void orc_init(int nx, int ny, int nz, const real *prm, const real *phi0,
              const real *u0, real *f, real *g)
{
    velocity_set();
    long N = (long)nx * ny * nz;
    real *grad = malloc(sizeof(real) * 3 * N);
    real *lap = malloc(sizeof(real) * N);
    orc_gradients(nx, ny, nz, phi0, grad, lap);
    real rho = prm[P_RHO0];
    for (long s = 0; s < N; s++) {
        real j[3], d[3], feq[NV], geq[NV];
        for (int a = 0; a < 3; a++) {
            j[a] = u0 ? rho * u0[a * N + s] : 0.0;
            d[a] = grad[a * N + s];
        }
        orc_site_equilibrium(prm, rho, j, phi0[s], d, lap[s], feq, geq);
        for (int i = 0; i < NV; i++) {
            f[i * N + s] = feq[i];
            g[i * N + s] = geq[i];
        }
    }
    free(grad);
    free(lap);
}

/* nsteps timesteps in place: phi = sum g; stencils; collide f and g; stream. */
void orc_step(int nx, int ny, int nz, const real *prm, real *f, real *g, int nsteps)
{
    velocity_set();
    long N = (long)nx * ny * nz;
    real *phi = malloc(sizeof(real) * N);
    real *grad = malloc(sizeof(real) * 3 * N);
    real *lap = malloc(sizeof(real) * N);
    real *fs = malloc(sizeof(real) * NV * N);
    real *gs = malloc(sizeof(real) * NV * N);
    for (int t = 0; t < nsteps; t++) {
        for (long s = 0; s < N; s++) {
            real acc = 0.0;
            for (int i = 0; i < NV; i++) acc += g[i * N + s];
            phi[s] = acc;
        }
        orc_gradients(nx, ny, nz, phi, grad, lap);
#pragma omp parallel for
        for (long s = 0; s < N; s++) {
            real rho = 0.0, j[3] = {0.0, 0.0, 0.0}, d[3], feq[NV], geq[NV];
            for (int i = 0; i < NV; i++) {
                rho += f[i * N + s];
                for (int a = 0; a < 3; a++) j[a] += f[i * N + s] * cv[i][a];
            }
            for (int a = 0; a < 3; a++) d[a] = grad[a * N + s];
            orc_site_equilibrium(prm, rho, j, phi[s], d, lap[s], feq, geq);
            for (int i = 0; i < NV; i++) {
                fs[i * N + s] = f[i * N + s] - (f[i * N + s] - feq[i]) / prm[P_TAU];
                gs[i * N + s] = g[i * N + s] - (g[i * N + s] - geq[i]) / prm[P_TAUG];
            }
        }
#pragma omp parallel for
        for (int z = 0; z < nz; z++)
            for (int y = 0; y < ny; y++)
                for (int x = 0; x < nx; x++) {
                    long s = site(x, y, z, nx, ny, nz);
                    for (int i = 0; i < NV; i++) {
                        long dst = site(x + cv[i][0], y + cv[i][1], z + cv[i][2], nx, ny, nz);
                        f[i * N + dst] = fs[i * N + s];
                        g[i * N + dst] = gs[i * N + s];
                    }
                }
    }
    free(phi); free(grad); free(lap); free(fs); free(gs);
}

/* rho = sum f, u = sum f c / rho (SoA [3][N]), phi = sum g. */
void orc_moments(int nx, int ny, int nz, const real *f, const real *g,
                 real *rho, real *u, real *phi)
{
    velocity_set();
    long N = (long)nx * ny * nz;
    for (long s = 0; s < N; s++) {
        real r = 0.0, j[3] = {0.0, 0.0, 0.0}, p = 0.0;
        for (int i = 0; i < NV; i++) {
            r += f[i * N + s];
            for (int a = 0; a < 3; a++) j[a] += f[i * N + s] * cv[i][a];
            p += g[i * N + s];
        }
        if (rho) rho[s] = r;
        if (u) for (int a = 0; a < 3; a++) u[a * N + s] = j[a] / r;
        if (phi) phi[s] = p;
    }
}

/* Lattice totals: out = {sum rho, sum rho u_x, sum rho u_y, sum rho u_z, sum phi}. */
void orc_reduce(int nx, int ny, int nz, const real *f, const real *g, real *out)
{
    velocity_set();
    long N = (long)nx * ny * nz;
    for (int k = 0; k < 5; k++) out[k] = 0.0;
    for (long s = 0; s < N; s++)
        for (int i = 0; i < NV; i++) {
            out[0] += f[i * N + s];
            for (int a = 0; a < 3; a++) out[1 + a] += f[i * N + s] * cv[i][a];
            out[4] += g[i * N + s];
        }
}
