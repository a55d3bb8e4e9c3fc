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
 * The *_n entry points also take the isotropic 19- and 27-point stencils
 * (the paper only says "standard finite-difference"; these are read as the
 * lattice-weighted differences over the D3Q19 / D3Q27 neighbourhoods):
 *   d_a phi = (1/cs2) sum_c W_c c_a phi(x + c),
 *   lap phi = (2/cs2) sum_c W_c (phi(x + c) - phi(x)),
 * with the D3Q19 weights above, or the D3Q27 weights 8/27 (rest), 2/27
 * (faces), 1/54 (edges), 1/216 (corners).  Both reproduce the 7-point
 * stencils on fields that vary along one axis only.
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
#ifdef _OPENMP
#include <omp.h>
#endif
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

/* Threads the parallel loops of this build use (1 without OpenMP). */
int orc_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

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

/* Isotropic 19- or 27-point differences (see the header); npts = 7 is
 * orc_gradients. */
void orc_gradients_n(int nx, int ny, int nz, int npts, const real *phi, real *grad, real *lap)
{
    if (npts == 7) {
        orc_gradients(nx, ny, nz, phi, grad, lap);
        return;
    }
    long N = (long)nx * ny * nz;
    const double cs2 = 1.0 / 3.0;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long s = site(x, y, z, nx, ny, nz);
                real d[3] = {0.0, 0.0, 0.0}, l = 0.0;
                for (int a = -1; a <= 1; a++)
                    for (int b = -1; b <= 1; b++)
                        for (int c = -1; c <= 1; c++) {
                            int c2 = a * a + b * b + c * c;
                            double W;
                            if (npts == 19) {
                                if (c2 > 2) continue;
                                W = (c2 == 0) ? 1.0 / 3.0 : (c2 == 1) ? 1.0 / 18.0 : 1.0 / 36.0;
                            } else {
                                W = (c2 == 0) ? 8.0 / 27.0 : (c2 == 1) ? 2.0 / 27.0 : (c2 == 2) ? 1.0 / 54.0 : 1.0 / 216.0;
                            }
                            real v = phi[site(x + a, y + b, z + c, nx, ny, nz)];
                            d[0] += W * a * v;
                            d[1] += W * b * v;
                            d[2] += W * c * v;
                            l += W * (v - phi[s]);
                        }
                for (int a = 0; a < 3; a++) grad[a * N + s] = d[a] / cs2;
                lap[s] = 2.0 * l / cs2;
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
void orc_init_n(int nx, int ny, int nz, int npts, const real *prm, const real *phi0,
                const real *u0, real *f, real *g)
{
    velocity_set();
    long N = (long)nx * ny * nz;
    real *grad = malloc(sizeof(real) * 3 * N);
    real *lap = malloc(sizeof(real) * N);
    orc_gradients_n(nx, ny, nz, npts, phi0, grad, lap);
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

void orc_init(int nx, int ny, int nz, const real *prm, const real *phi0,
              const real *u0, real *f, real *g)
{
    orc_init_n(nx, ny, nz, 7, prm, phi0, u0, f, g);
}

/* nsteps timesteps in place: phi = sum g; stencils (npts = 7, 19 or 27
 * points); collide f and g; stream. */
void orc_step_n(int nx, int ny, int nz, int npts, const real *prm, real *f, real *g, int nsteps)
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
        orc_gradients_n(nx, ny, nz, npts, phi, grad, lap);
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

void orc_step(int nx, int ny, int nz, const real *prm, real *f, real *g, int nsteps)
{
    orc_step_n(nx, ny, nz, 7, prm, f, g, nsteps);
}

/* Multiple-relaxation-time collision of f with a Guo body force.
 *
 * The collision is defined by projections, so that it does not depend on a
 * choice of moment basis.  With m0 = sum h, m1 = sum h c, m2 = sum h c c, the
 * second-order Hermite part of a vector h is
 *   H(h)_i = w_i [m0 + c_i.m1/cs2 + Q_i:(m2 - m0 cs2 I)/(2 cs2^2)]
 * and its ghost part is h - H(h) (the 9 directions of D3Q19 orthogonal to
 * 1, c and c c).  At each site, with body force F (force density):
 *   rho = sum f, j = sum f c, u = (j + F/2)/rho, feq = feq(rho, rho u, ...),
 *   N = sum (f - feq) c c, split into its bulk part (tr N/3) I and the
 *       traceless shear part; G = u F + F u split the same way;
 *   X = (1 - w_s) N_shear + (1 - w_b) N_bulk
 *     + (1 - w_s/2) G_shear + (1 - w_b/2) G_bulk,
 *   f*_i = feq_i + w_i [c_i.F/(2 cs2) + Q_i:X/(2 cs2^2)]
 *        + (1 - w_gh) ghost(f - feq)_i,
 * with w_s = 1/tau (shear), w_b = 1/tau_bulk, w_gh = 1/tau_ghost.  The
 * momentum after collision is j + F; with all three rates equal and F = 0
 * this is the BGK collision of orc_step.  g relaxes by BGK (tau_g) toward
 * geq evaluated with the same u.  mrt[] = {tau_bulk, tau_ghost, Fx, Fy, Fz}.
 */
void orc_step_mrt(int nx, int ny, int nz, int npts, const real *prm, const real *mrt, real *f, real *g,
                  int nsteps)
{
    velocity_set();
    const double cs2 = 1.0 / 3.0;
    long N = (long)nx * ny * nz;
    real *phi = malloc(sizeof(real) * N);
    real *grad = malloc(sizeof(real) * 3 * N);
    real *lap = malloc(sizeof(real) * N);
    real *fs = malloc(sizeof(real) * NV * N);
    real *gs = malloc(sizeof(real) * NV * N);
    const real ws = 1.0 / prm[P_TAU], wb = 1.0 / mrt[0], wgh = 1.0 / mrt[1];
    const real F[3] = {mrt[2], mrt[3], mrt[4]};
    for (int t = 0; t < nsteps; t++) {
        for (long s = 0; s < N; s++) {
            real acc = 0.0;
            for (int i = 0; i < NV; i++) acc += g[i * N + s];
            phi[s] = acc;
        }
        orc_gradients_n(nx, ny, nz, npts, phi, grad, lap);
#pragma omp parallel for
        for (long s = 0; s < N; s++) {
            real rho = 0.0, j[3] = {0.0, 0.0, 0.0}, u[3], ju[3], d[3], feq[NV], geq[NV], h[NV];
            for (int i = 0; i < NV; i++) {
                rho += f[i * N + s];
                for (int a = 0; a < 3; a++) j[a] += f[i * N + s] * cv[i][a];
            }
            for (int a = 0; a < 3; a++) {
                u[a] = (j[a] + 0.5 * F[a]) / rho;
                ju[a] = rho * u[a];
                d[a] = grad[a * N + s];
            }
            orc_site_equilibrium(prm, rho, ju, phi[s], d, lap[s], feq, geq);
            /* moments of h = f - feq */
            real m0 = 0.0, m1[3] = {0.0, 0.0, 0.0}, m2[3][3] = {{0.0}};
            for (int i = 0; i < NV; i++) {
                h[i] = f[i * N + s] - feq[i];
                m0 += h[i];
                for (int a = 0; a < 3; a++) {
                    m1[a] += h[i] * cv[i][a];
                    for (int b = 0; b < 3; b++) m2[a][b] += h[i] * cv[i][a] * cv[i][b];
                }
            }
            real trN = (m2[0][0] + m2[1][1] + m2[2][2]) / 3.0;
            real G[3][3], X[3][3], trG = 2.0 * (u[0] * F[0] + u[1] * F[1] + u[2] * F[2]) / 3.0;
            for (int a = 0; a < 3; a++)
                for (int b = 0; b < 3; b++) {
                    G[a][b] = u[a] * F[b] + F[a] * u[b];
                    real nb = (a == b) ? trN : 0.0, gb = (a == b) ? trG : 0.0;
                    X[a][b] = (1.0 - ws) * (m2[a][b] - nb) + (1.0 - wb) * nb
                              + (1.0 - 0.5 * ws) * (G[a][b] - gb) + (1.0 - 0.5 * wb) * gb;
                }
            for (int i = 0; i < NV; i++) {
                real hm1 = 0.0, cF = 0.0, qN = 0.0, qX = 0.0;
                for (int a = 0; a < 3; a++) {
                    hm1 += cv[i][a] * m1[a];
                    cF += cv[i][a] * F[a];
                    for (int b = 0; b < 3; b++) {
                        double Q = cv[i][a] * cv[i][b] - (a == b ? cs2 : 0.0);
                        qN += Q * (m2[a][b] - (a == b ? m0 * cs2 : 0.0));
                        qX += Q * X[a][b];
                    }
                }
                real herm = wv[i] * (m0 + hm1 / cs2 + qN / (2.0 * cs2 * cs2));
                real ghost = h[i] - herm;
                fs[i * N + s] = feq[i] + wv[i] * (cF / (2.0 * cs2) + qX / (2.0 * cs2 * cs2)) + (1.0 - wgh) * ghost;
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

#ifndef ORC_COMPLEX
/* ------------------------------------------------------------------------
 * Reverse mode (adjoint) of the timestep and of the initialisation, FP64.
 *
 * State F(t) = (f, g)(x, t) after streaming.  Adjoint F_bar(t) = dJ/dF(t).
 * One reverse step, given F(t) and F_bar(t+1):
 *   1. streaming transposed: fs_bar_i(x) = f_bar_i(x + c_i, t+1) (g alike);
 *   2. per site, the collision's vector-Jacobian product, which yields
 *      f_bar(x, t), the direct part of g_bar, and the adjoints of phi, of the
 *      gradient d_a phi and of lap phi at x, plus dJ/dkappa;
 *   3. the stencils transposed: phi_bar(x) gathers
 *      (d_bar_a(x - e_a) - d_bar_a(x + e_a))/2 and
 *      sum_a (l_bar(x - e_a) + l_bar(x + e_a)) - 6 l_bar(x);
 *   4. phi = sum g transposed: g_bar_i(x, t) += phi_bar(x).
 * The collision's forward quantities are recomputed from F(t).
 * ---------------------------------------------------------------------- */

/* Adjoint of the equilibrium map at one site.  Given weights fe_bar[i] on
 * feq_i and ge_bar[i] on geq_i, accumulate the adjoints of rho, j, phi, the
 * gradient d, lap, and kappa.  ``with_flow`` = 0 treats rho and j as
 * constants (the initial state, where they are inputs). */
static void equilibrium_vjp(const double *prm, double rho, const double *j, double phi,
                            const double *d, double lap, const double *fe_bar, const double *ge_bar,
                            int with_flow, double *rho_bar, double *j_bar, double *phi_bar,
                            double *d_bar, double *lap_bar, double *kappa_bar)
{
    const double cs2 = 1.0 / 3.0;
    double A = prm[P_A], B = prm[P_B], kappa = prm[P_KAPPA], gam = prm[P_GAMMA];
    double u[3];
    for (int a = 0; a < 3; a++) u[a] = j[a] / rho;
    /* feq_i = w_i [rho + c.j/cs2 + (c S c - cs2 tr S)/(2 cs2^2)]
     * geq_i = w_i [phi + phi c.u/cs2 + (c G c - cs2 tr G)/(2 cs2^2)] */
    double Sb[3][3] = {{0}}, Gb[3][3] = {{0}};
    double u_bar[3] = {0, 0, 0};
    for (int i = 0; i < NV; i++) {
        double cu = 0.0;
        for (int a = 0; a < 3; a++) cu += cv[i][a] * u[a];
        double wf = wv[i] * fe_bar[i], wg = wv[i] * ge_bar[i];
        *rho_bar += wf;
        for (int a = 0; a < 3; a++) {
            j_bar[a] += wf * cv[i][a] / cs2;
            u_bar[a] += wg * phi * cv[i][a] / cs2;
        }
        *phi_bar += wg * (1.0 + cu / cs2);
        for (int a = 0; a < 3; a++)
            for (int b = 0; b < 3; b++) {
                double Q = cv[i][a] * cv[i][b] - (a == b ? cs2 : 0.0);
                Sb[a][b] += wf * Q / (2.0 * cs2 * cs2);
                Gb[a][b] += wg * Q / (2.0 * cs2 * cs2);
            }
    }
    /* G = (Gamma mu - phi cs2) I + phi u u */
    double trG = Gb[0][0] + Gb[1][1] + Gb[2][2];
    double mu_bar = gam * trG;
    *phi_bar += -cs2 * trG;
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            *phi_bar += Gb[a][b] * u[a] * u[b];
            u_bar[a] += Gb[a][b] * phi * u[b];
            u_bar[b] += Gb[a][b] * phi * u[a];
        }
    /* S = pb I + kappa d d + rho u u, with rho u u = j j / rho */
    double pb_bar = Sb[0][0] + Sb[1][1] + Sb[2][2];
    for (int a = 0; a < 3; a++)
        for (int b = 0; b < 3; b++) {
            d_bar[a] += Sb[a][b] * kappa * d[b];
            d_bar[b] += Sb[a][b] * kappa * d[a];
            *kappa_bar += Sb[a][b] * d[a] * d[b];
            if (with_flow) {
                j_bar[a] += Sb[a][b] * j[b] / rho;
                j_bar[b] += Sb[a][b] * j[a] / rho;
                *rho_bar -= Sb[a][b] * j[a] * j[b] / (rho * rho);
            }
        }
    /* pb = A/2 phi^2 + 3B/4 phi^4 - kappa phi lap - kappa/2 |d|^2 */
    double dd = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
    *phi_bar += pb_bar * (A * phi + 3.0 * B * phi * phi * phi - kappa * lap);
    *lap_bar += -kappa * phi * pb_bar;
    for (int a = 0; a < 3; a++) d_bar[a] += -kappa * d[a] * pb_bar;
    *kappa_bar += pb_bar * (-phi * lap - 0.5 * dd);
    /* mu = A phi + B phi^3 - kappa lap */
    *phi_bar += mu_bar * (A + 3.0 * B * phi * phi);
    *lap_bar += -kappa * mu_bar;
    *kappa_bar += -lap * mu_bar;
    /* u = j / rho */
    if (with_flow) {
        for (int a = 0; a < 3; a++) {
            j_bar[a] += u_bar[a] / rho;
            *rho_bar -= u_bar[a] * j[a] / (rho * rho);
        }
    }
}

/* phi_bar(x) += transposed 7-point stencils of (d_bar, lap_bar). */
static void stencil_transpose(int nx, int ny, int nz, const double *d_bar, const double *lap_bar,
                              double *phi_bar)
{
    long N = (long)nx * ny * nz;
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long s = site(x, y, z, nx, ny, nz);
                long xp = site(x + 1, y, z, nx, ny, nz), xm = site(x - 1, y, z, nx, ny, nz);
                long yp = site(x, y + 1, z, nx, ny, nz), ym = site(x, y - 1, z, nx, ny, nz);
                long zp = site(x, y, z + 1, nx, ny, nz), zm = site(x, y, z - 1, nx, ny, nz);
                phi_bar[s] += (d_bar[0 * N + xm] - d_bar[0 * N + xp]) / 2.0
                            + (d_bar[1 * N + ym] - d_bar[1 * N + yp]) / 2.0
                            + (d_bar[2 * N + zm] - d_bar[2 * N + zp]) / 2.0
                            + lap_bar[xm] + lap_bar[xp] + lap_bar[ym] + lap_bar[yp]
                            + lap_bar[zm] + lap_bar[zp] - 6.0 * lap_bar[s];
            }
}

/* One reverse step: (f, g) = F(t); (af, ag) holds F_bar(t+1) on entry and
 * F_bar(t) on return; *dkappa accumulates dJ/dkappa of this step. */
void orc_step_adjoint(int nx, int ny, int nz, const double *prm, const double *f, const double *g,
                      double *af, double *ag, double *dkappa)
{
    velocity_set();
    long N = (long)nx * ny * nz;
    double *phi = malloc(sizeof(double) * N), *grad = malloc(sizeof(double) * 3 * N);
    double *lap = malloc(sizeof(double) * N);
    double *fs_bar = malloc(sizeof(double) * NV * N), *gs_bar = malloc(sizeof(double) * NV * N);
    double *phi_bar = calloc(N, sizeof(double)), *d_bar = calloc(3 * N, sizeof(double));
    double *lap_bar = calloc(N, sizeof(double));
    double omega = 1.0 / prm[P_TAU], omega_g = 1.0 / prm[P_TAUG];
    for (long s = 0; s < N; s++) {
        double acc = 0.0;
        for (int i = 0; i < NV; i++) acc += g[i * N + s];
        phi[s] = acc;
    }
    orc_gradients(nx, ny, nz, phi, grad, lap);
    /* 1. streaming transposed */
    for (int z = 0; z < nz; z++)
        for (int y = 0; y < ny; y++)
            for (int x = 0; x < nx; x++) {
                long s = site(x, y, z, nx, ny, nz);
                for (int i = 0; i < NV; i++) {
                    long dst = site(x + cv[i][0], y + cv[i][1], z + cv[i][2], nx, ny, nz);
                    fs_bar[i * N + s] = af[i * N + dst];
                    gs_bar[i * N + s] = ag[i * N + dst];
                }
            }
    /* 2. collision, transposed per site */
    double kap = 0.0;
    for (long s = 0; s < N; s++) {
        double rho = 0.0, j[3] = {0, 0, 0}, d[3], fe_bar[NV], ge_bar[NV];
        for (int i = 0; i < NV; i++) {
            rho += f[i * N + s];
            for (int a = 0; a < 3; a++) j[a] += f[i * N + s] * cv[i][a];
        }
        for (int a = 0; a < 3; a++) d[a] = grad[a * N + s];
        for (int i = 0; i < NV; i++) {
            fe_bar[i] = omega * fs_bar[i * N + s];
            ge_bar[i] = omega_g * gs_bar[i * N + s];
        }
        double rho_bar = 0.0, j_bar[3] = {0, 0, 0}, pb = 0.0, db[3] = {0, 0, 0}, lb = 0.0;
        equilibrium_vjp(prm, rho, j, phi[s], d, lap[s], fe_bar, ge_bar, 1, &rho_bar, j_bar, &pb, db, &lb,
                        &kap);
        phi_bar[s] += pb;
        for (int a = 0; a < 3; a++) d_bar[a * N + s] = db[a];
        lap_bar[s] = lb;
        for (int i = 0; i < NV; i++) {
            double jc = 0.0;
            for (int a = 0; a < 3; a++) jc += j_bar[a] * cv[i][a];
            af[i * N + s] = (1.0 - omega) * fs_bar[i * N + s] + rho_bar + jc;
            ag[i * N + s] = (1.0 - omega_g) * gs_bar[i * N + s];
        }
    }
    /* 3. stencils transposed; 4. phi = sum g transposed */
    stencil_transpose(nx, ny, nz, d_bar, lap_bar, phi_bar);
    for (long s = 0; s < N; s++)
        for (int i = 0; i < NV; i++) ag[i * N + s] += phi_bar[s];
    *dkappa += kap;
    free(phi); free(grad); free(lap); free(fs_bar); free(gs_bar);
    free(phi_bar); free(d_bar); free(lap_bar);
}

/* Reverse of the initialisation F(0) = equilibria(rho0, rho0 u0, phi0):
 * given F_bar(0) = (af, ag), phi0_bar receives dJ/dphi0 (overwritten) and
 * *dkappa accumulates the initialisation's part of dJ/dkappa. */
void orc_init_adjoint(int nx, int ny, int nz, const double *prm, const double *phi0, const double *u0,
                      const double *af, const double *ag, double *phi0_bar, double *dkappa)
{
    velocity_set();
    long N = (long)nx * ny * nz;
    double *grad = malloc(sizeof(double) * 3 * N), *lap = malloc(sizeof(double) * N);
    double *d_bar = calloc(3 * N, sizeof(double)), *lap_bar = calloc(N, sizeof(double));
    orc_gradients(nx, ny, nz, phi0, grad, lap);
    double rho = prm[P_RHO0], kap = 0.0;
    for (long s = 0; s < N; s++) {
        double j[3], d[3], fe_bar[NV], ge_bar[NV];
        for (int a = 0; a < 3; a++) {
            j[a] = u0 ? rho * u0[a * N + s] : 0.0;
            d[a] = grad[a * N + s];
        }
        for (int i = 0; i < NV; i++) {
            fe_bar[i] = af[i * N + s];
            ge_bar[i] = ag[i * N + s];
        }
        double rho_bar = 0.0, j_bar[3] = {0, 0, 0}, pb = 0.0, db[3] = {0, 0, 0}, lb = 0.0;
        equilibrium_vjp(prm, rho, j, phi0[s], d, lap[s], fe_bar, ge_bar, 0, &rho_bar, j_bar, &pb, db, &lb,
                        &kap);
        phi0_bar[s] = pb;
        for (int a = 0; a < 3; a++) d_bar[a * N + s] = db[a];
        lap_bar[s] = lb;
    }
    stencil_transpose(nx, ny, nz, d_bar, lap_bar, phi0_bar);
    *dkappa += kap;
    free(grad); free(lap); free(d_bar); free(lap_bar);
}
#endif /* ORC_COMPLEX */
