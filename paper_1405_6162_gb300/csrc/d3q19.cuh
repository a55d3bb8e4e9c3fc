// d3q19.cuh -- D3Q19 velocity set and the per-site binary-fluid collision.
//
// The collision is the "binary collision" of targetDP Sec. IV: BGK
// relaxation of the density distribution f toward an equilibrium whose
// second moment carries the free-energy pressure tensor, and of the
// order-parameter distribution g toward an equilibrium whose second moment is
// Gamma*mu (symmetric free energy, Sec. II.A "free energy based approach").
// Velocities come in opposite pairs (2k-1, 2k), so each equilibrium is
// evaluated once per pair as (even part) +/- (odd part).
#pragma once

#include <cuda_runtime.h>

#ifndef LBK_ST_CS
#define LBK_ST_CS 0   // 1: stores of post-collision values with the streaming (.cs) hint
#endif

namespace lbk {

constexpr int Q = 19;


// a * b + c; one fused operation for float and double (contracted), and the
// fused double-float form for df64 (df64.cuh)
template <typename T>
__device__ __forceinline__ T fmadd(T a, T b, T c)
{
    return a * b + c;
}

// a * b + (c + d); for df64 one fused form (df64.cuh) that renormalises once
template <typename T>
__device__ __forceinline__ T fmadd_sum(T a, T b, T c, T d)
{
    return fmadd(a, b, c + d);
}

// the relaxation of an opposite pair: fp = c fp + (s + a), fm = c fm + (s - a);
// for df64 one pass of paired FP32 instructions over both (df64.cuh)
template <typename T>
__device__ __forceinline__ void relax_pair(T c, T &fp, T &fm, T s, T a)
{
    fp = fmadd_sum(c, fp, s, a);
    fm = fmadd_sum(c, fm, s, -a);
}

template <typename T>
__device__ __forceinline__ void store(T *p, T v)
{
#if LBK_ST_CS
    __stcs(p, v);
#else
    *p = v;
#endif
}

// ABI velocity order: 0 rest; 1..6 faces; 7..18 edges; odd/even = opposite.
__host__ __device__ constexpr int cx(int i) {
    return (i == 1 || i == 7 || i == 9 || i == 11 || i == 13) ? 1
         : (i == 2 || i == 8 || i == 10 || i == 12 || i == 14) ? -1 : 0;
}
__host__ __device__ constexpr int cy(int i) {
    return (i == 3 || i == 7 || i == 10 || i == 15 || i == 17) ? 1
         : (i == 4 || i == 8 || i == 9 || i == 16 || i == 18) ? -1 : 0;
}
__host__ __device__ constexpr int cz(int i) {
    return (i == 5 || i == 11 || i == 14 || i == 15 || i == 18) ? 1
         : (i == 6 || i == 12 || i == 13 || i == 16 || i == 17) ? -1 : 0;
}
__host__ __device__ constexpr double weight(int i) {
    return i == 0 ? 1.0 / 3.0 : (i <= 6 ? 1.0 / 18.0 : 1.0 / 36.0);
}

// x / 2 (exact in binary floating point)
__device__ __forceinline__ float half(float x) { return 0.5f * x; }
__device__ __forceinline__ double half(double x) { return 0.5 * x; }

// Relaxation and free-energy parameters in the arithmetic type T.  The
// relaxation constants fold omega = 1/tau into the lattice weights so that
// the step evaluates f* = (1 - omega) f + omega feq with one multiply-add
// per direction (likewise g with omega_g); they are computed in double on
// the host and rounded once.
template <typename T>
struct Coll {
    T omega, omega_g;      // 1/tau, 1/tau_g
    T rho0;                // shift of the FP32 form
    T gamma, A, B, kappa;
    T hA, qB;              // A/2, 3B/4 (the bulk pressure's coefficients)
    T cf, f0, f1, f2, f1h, f2h, f1t, f2t;   // 1-omega; omega*w_k; omega*w_k*9/2; omega*w_k*3
    T cg, g0, g1, g2, g1h, g2h, g1t, g2t;   // the same with omega_g
};

// Equilibria of f and g at one site.  R is rho (SH = false) or rho - rho0
// (SH = true: the result is feq_i - w_i rho0).  j = sum f c = rho u.
// sink(i, feq_i, geq_i) is called once per direction, i a literal after
// inlining.
template <typename T, bool SH, typename Sink>
__device__ __forceinline__ void equilibria(const Coll<T>& p, T R, T jx, T jy, T jz,
                                           T phi, T dx, T dy, T dz, T lap, Sink&& sink)
{
    const T third = T(1.0 / 3.0);
    const T rho = SH ? p.rho0 + R : R;
    const T rinv = T(1) / rho;
    const T ux = jx * rinv, uy = jy * rinv, uz = jz * rinv;
    const T phi2 = phi * phi;
    const T mu = phi * (p.A + p.B * phi2) - p.kappa * lap;
    const T pb = phi2 * (T(0.5) * p.A + T(0.75) * p.B * phi2)
               - p.kappa * (phi * lap + T(0.5) * (dx * dx + dy * dy + dz * dz));
    // S = P + rho u u
    const T Sxx = pb + p.kappa * dx * dx + jx * ux;
    const T Syy = pb + p.kappa * dy * dy + jy * uy;
    const T Szz = pb + p.kappa * dz * dz + jz * uz;
    const T Sxy = p.kappa * dx * dy + jx * uy;
    const T Sxz = p.kappa * dx * dz + jx * uz;
    const T Syz = p.kappa * dy * dz + jy * uz;
    const T t3 = (Sxx + Syy + Szz) * third;
    // g: G = (Gamma mu - phi/3) I + phi u u;  G:Q_i = phi (c.u)^2 - phi u^2/3 + (Gamma mu - phi/3)(c^2 - 1)
    const T pu2 = phi * (ux * ux + uy * uy + uz * uz) * third;
    const T gm = p.gamma * mu - phi * third;

    const T w0 = T(1.0 / 3.0), w1 = T(1.0 / 18.0), w2 = T(1.0 / 36.0);
    const T h = T(4.5), three = T(3);

    sink(0, w0 * (R - h * t3), w0 * (phi - h * (pu2 + gm)));

    // faces: S:Q = S_aa - t3
    {
        T fs = w1 * (R + h * (Sxx - t3)), fa = w1 * three * jx;
        T gs = w1 * (phi + h * (phi * ux * ux - pu2)), ga = w1 * three * phi * ux;
        sink(1, fs + fa, gs + ga); sink(2, fs - fa, gs - ga);
    }
    {
        T fs = w1 * (R + h * (Syy - t3)), fa = w1 * three * jy;
        T gs = w1 * (phi + h * (phi * uy * uy - pu2)), ga = w1 * three * phi * uy;
        sink(3, fs + fa, gs + ga); sink(4, fs - fa, gs - ga);
    }
    {
        T fs = w1 * (R + h * (Szz - t3)), fa = w1 * three * jz;
        T gs = w1 * (phi + h * (phi * uz * uz - pu2)), ga = w1 * three * phi * uz;
        sink(5, fs + fa, gs + ga); sink(6, fs - fa, gs - ga);
    }
    // edges: S:Q = S_aa + S_bb +/- 2 S_ab - t3
#define LBK_EDGE(IP, IM, SAA, SBB, SAB, JA, JB, UA, UB, SGN)                          \
    {                                                                                 \
        const T cu = UA + SGN * UB;                                                   \
        T fs = w2 * (R + h * (SAA + SBB + SGN * T(2) * SAB - t3));                    \
        T fa = w2 * three * (JA + SGN * JB);                                          \
        T gs = w2 * (phi + h * (phi * cu * cu - pu2 + gm));                           \
        T ga = w2 * three * phi * cu;                                                 \
        sink(IP, fs + fa, gs + ga); sink(IM, fs - fa, gs - ga);                       \
    }
    LBK_EDGE(7, 8, Sxx, Syy, Sxy, jx, jy, ux, uy, T(1))
    LBK_EDGE(9, 10, Sxx, Syy, Sxy, jx, jy, ux, uy, T(-1))
    LBK_EDGE(11, 12, Sxx, Szz, Sxz, jx, jz, ux, uz, T(1))
    LBK_EDGE(13, 14, Sxx, Szz, Sxz, jx, jz, ux, uz, T(-1))
    LBK_EDGE(15, 16, Syy, Szz, Syz, jy, jz, uy, uz, T(1))
    LBK_EDGE(17, 18, Syy, Szz, Syz, jy, jz, uy, uz, T(-1))
#undef LBK_EDGE
}

// Density moments of a (possibly shifted) distribution: R = sum f, j = sum f c.
template <typename T>
__device__ __forceinline__ void density_moments(const T (&f)[Q], T& R, T& jx, T& jy, T& jz)
{
    R = ((f[0] + f[1]) + (f[2] + f[3])) + ((f[4] + f[5]) + (f[6] + f[7]))
      + ((f[8] + f[9]) + (f[10] + f[11])) + ((f[12] + f[13]) + (f[14] + f[15]))
      + ((f[16] + f[17]) + f[18]);
    jx = (f[1] - f[2]) + (f[7] - f[8]) + (f[9] - f[10]) + (f[11] - f[12]) + (f[13] - f[14]);
    jy = (f[3] - f[4]) + (f[7] - f[8]) - (f[9] - f[10]) + (f[15] - f[16]) + (f[17] - f[18]);
    jz = (f[5] - f[6]) + (f[11] - f[12]) - (f[13] - f[14]) + (f[15] - f[16]) - (f[17] - f[18]);
}

template <typename T>
__device__ __forceinline__ T sum19(const T (&g)[Q])
{
    return ((g[0] + g[1]) + (g[2] + g[3])) + ((g[4] + g[5]) + (g[6] + g[7]))
         + ((g[8] + g[9]) + (g[10] + g[11])) + ((g[12] + g[13]) + (g[14] + g[15]))
         + ((g[16] + g[17]) + g[18]);
}

// In-place BGK collision of f at one site given phi and its stencil values
// (also returns u and mu):
// f*_i = (1 - omega) f_i + omega feq_i with omega feq_i expanded per weight
// class (rest, face, edge) and per opposite pair, sharing every partial sum.
template <typename T, bool SH>
__device__ __forceinline__ void collide_f(const Coll<T>& p, T (&f)[Q], T phi, T dx, T dy, T dz, T lap,
                                          T& ux, T& uy, T& uz, T& mu)
{
    T R, jx, jy, jz;
    density_moments(f, R, jx, jy, jz);
    const T rho = SH ? p.rho0 + R : R;
    const T rinv = T(1) / rho;
    ux = jx * rinv;
    uy = jy * rinv;
    uz = jz * rinv;
    const T phi2 = phi * phi;
    mu = phi * (p.A + p.B * phi2) - p.kappa * lap;
    const T pb = phi2 * (p.hA + p.qB * phi2) - p.kappa * (phi * lap + half(dx * dx + dy * dy + dz * dz));
    // S = P + rho u u
    const T Sxx = pb + p.kappa * dx * dx + jx * ux;
    const T Syy = pb + p.kappa * dy * dy + jy * uy;
    const T Szz = pb + p.kappa * dz * dz + jz * uz;
    const T Sxy = p.kappa * dx * dy + jx * uy;
    const T Sxz = p.kappa * dx * dz + jx * uz;
    const T Syz = p.kappa * dy * dz + jy * uz;

    // ---- f: omega feq_i = omega w_i (R - 9/2 t3) + 9/2 omega w_i c_i c_i : S + 3 omega w_i c_i . j,
    // t3 = tr S / 3, so 9/2 t3 = 3/2 tr S (3/2 exact in binary)
    const T cf = p.cf;
    const T b = R - T(1.5) * (Sxx + Syy + Szz);
    f[0] = fmadd(cf, f[0], p.f0 * b);
    const T B1 = p.f1 * b, B2 = p.f2 * b;
#define LBK_FACE(IP, IM, SAA, JA)                                  \
    {                                                              \
        const T s_ = fmadd(p.f1h, SAA, B1), a_ = p.f1t * JA;       \
        relax_pair(cf, f[IP], f[IM], s_, a_);                      \
    }
    LBK_FACE(1, 2, Sxx, jx)
    LBK_FACE(3, 4, Syy, jy)
    LBK_FACE(5, 6, Szz, jz)
#undef LBK_FACE
    // edge pairs (a+b, -a-b) = (IP, IM) and (a-b, -a+b) = (KP, KM); 2 f2h = f1h
#define LBK_EDGES(IP, IM, KP, KM, SAA, SBB, SAB, JA, JB)             \
    {                                                                \
        const T e_ = fmadd(p.f2h, SAA + SBB, B2), o_ = p.f1h * SAB;  \
        const T sp = e_ + o_, sm = e_ - o_;                          \
        const T ap = p.f2t * (JA + JB), am = p.f2t * (JA - JB);      \
        relax_pair(cf, f[IP], f[IM], sp, ap);                        \
        relax_pair(cf, f[KP], f[KM], sm, am);                        \
    }
    LBK_EDGES(7, 8, 9, 10, Sxx, Syy, Sxy, jx, jy)
    LBK_EDGES(11, 12, 13, 14, Sxx, Szz, Sxz, jx, jz)
    LBK_EDGES(15, 16, 17, 18, Syy, Szz, Syz, jy, jz)
#undef LBK_EDGES
}

// In-place BGK collision of g at one site with velocity u and chemical
// potential mu.
template <typename T>
__device__ __forceinline__ void collide_g(const Coll<T>& p, T (&g)[Q], T phi, T ux, T uy, T uz, T mu)
{
    const T third = T(1.0 / 3.0), h = T(4.5);
    // ---- g: omega_g geq_i = omega_g w_i [phi + 3 phi c.u + 9/2 (phi (c.u)^2 - phi u^2/3 + (Gamma mu - phi/3)(c^2 - 1))]
    const T cg = p.cg;
    const T px = phi * ux, py = phi * uy, pz = phi * uz;
    const T gm = p.gamma * mu - phi * third;
    const T bg = phi - T(1.5) * (px * ux + py * uy + pz * uz);   // phi - 9/2 phi u^2 / 3
    g[0] = fmadd(cg, g[0], p.g0 * (bg - h * gm));
    const T G1 = p.g1 * bg, G2 = p.g2 * (bg + h * gm);
#define LBK_GFACE(IP, IM, PA, UA)                                   \
    {                                                               \
        const T s_ = fmadd(p.g1h, PA * UA, G1), a_ = p.g1t * PA;    \
        relax_pair(cg, g[IP], g[IM], s_, a_);                       \
    }
    LBK_GFACE(1, 2, px, ux)
    LBK_GFACE(3, 4, py, uy)
    LBK_GFACE(5, 6, pz, uz)
#undef LBK_GFACE
#define LBK_GEDGE(IP, IM, PC, CU)                                   \
    {                                                               \
        const T pc_ = PC, cu_ = CU;                                 \
        const T s_ = fmadd(p.g2h, pc_ * cu_, G2), a_ = p.g2t * pc_; \
        relax_pair(cg, g[IP], g[IM], s_, a_);                       \
    }
    LBK_GEDGE(7, 8, px + py, ux + uy)
    LBK_GEDGE(9, 10, px - py, ux - uy)
    LBK_GEDGE(11, 12, px + pz, ux + uz)
    LBK_GEDGE(13, 14, px - pz, ux - uz)
    LBK_GEDGE(15, 16, py + pz, uy + uz)
    LBK_GEDGE(17, 18, py - pz, uy - uz)
#undef LBK_GEDGE
    if constexpr (sizeof(T) == 4) {
        // In float the folded weights do not sum to omega_g (1/3 + 6/18 +
        // 12/36 rounds to 1 + 1.5e-8), which would bias sum g* -- phi -- by
        // that fraction every step.  The rest value takes up the difference
        // instead, g*_0 = phi - sum_{i>0} g*_i, so phi is conserved up to
        // unbiased rounding (carrying that sum's rounding errors as well was
        // measured to change nothing).
        T s = ((g[1] + g[2]) + (g[3] + g[4])) + ((g[5] + g[6]) + (g[7] + g[8]));
        s += ((g[9] + g[10]) + (g[11] + g[12])) + ((g[13] + g[14]) + (g[15] + g[16])) + (g[17] + g[18]);
        g[0] = phi - s;
    }
}

// In-place BGK collision of f (collide_f) and of g at one site.
template <typename T, bool SH>
__device__ __forceinline__ void collide(const Coll<T>& p, T (&f)[Q], T (&g)[Q],
                                        T phi, T dx, T dy, T dz, T lap)
{
    T ux, uy, uz, mu;
    collide_f<T, SH>(p, f, phi, dx, dy, dz, lap, ux, uy, uz, mu);
    collide_g<T>(p, g, phi, ux, uy, uz, mu);
}

// Rates and body force of the multiple-relaxation-time collision, with the
// combinations the kernel uses formed on the host (in double, rounded once).
template <typename T>
struct Mrt {
    T cs, cb;          // 1 - w_s, 1 - w_b          (w_s = 1/tau, w_b = 1/tau_bulk)
    T hs, hb;          // 1 - w_s/2, 1 - w_b/2      (Guo's factors)
    T og, cgh, kf;     // w_gh, 1 - w_gh, (2 - w_gh)/2   (w_gh = 1/tau_ghost)
    T Fx, Fy, Fz;      // body force density
    T hFx, hFy, hFz;   // F/2
};

// In-place multiple-relaxation-time collision of f with a Guo body force,
// then the BGK collision of g with the force-corrected velocity
// u = (j + F/2)/rho.  With N = sum (f - feq) c c (= Pi - R/3 I - S in the
// shifted form), G = u F + F u, each split into bulk (trace/3 I) and shear
// (traceless) parts,
//   X  = (1 - w_s) N_s + (1 - w_b) N_b + (1 - w_s/2) G_s + (1 - w_b/2) G_b,
// and the ghost part of f - feq relaxed at w_gh, the post-collision value is
//   f*_i = (1 - w_gh) f_i + w_i [R' + 3 c_i.J' + 9/2 Q_i:S'],
//   R' = w_gh R,  J' = w_gh rho u + (2 - w_gh)/2 F,
//   S' = w_gh S + X - (1 - w_gh) N,
// which is BGK when the three rates are equal and F = 0.
template <typename T, bool SH>
__device__ __forceinline__ void collide_mrt(const Coll<T>& p, const Mrt<T>& m, T (&f)[Q], T (&g)[Q],
                                            T phi, T dx, T dy, T dz, T lap)
{
    T R, jx, jy, jz;
    density_moments(f, R, jx, jy, jz);
    const T third = T(1.0 / 3.0), h = T(4.5);
    const T rho = SH ? p.rho0 + R : R;
    const T rinv = T(1) / rho;
    const T Jx = jx + m.hFx, Jy = jy + m.hFy, Jz = jz + m.hFz;   // rho u
    const T ux = Jx * rinv, uy = Jy * rinv, uz = Jz * rinv;
    const T phi2 = phi * phi;
    const T mu = phi * (p.A + p.B * phi2) - p.kappa * lap;
    const T pb = phi2 * (T(0.5) * p.A + T(0.75) * p.B * phi2)
               - p.kappa * (phi * lap + T(0.5) * (dx * dx + dy * dy + dz * dz));
    // S = P + rho u u
    const T Sxx = pb + p.kappa * dx * dx + Jx * ux;
    const T Syy = pb + p.kappa * dy * dy + Jy * uy;
    const T Szz = pb + p.kappa * dz * dz + Jz * uz;
    const T Sxy = p.kappa * dx * dy + Jx * uy;
    const T Sxz = p.kappa * dx * dz + Jx * uz;
    const T Syz = p.kappa * dy * dz + Jy * uz;
    // second moment of the stored values (sum f c c)
    const T e7 = f[7] + f[8], e9 = f[9] + f[10], e11 = f[11] + f[12], e13 = f[13] + f[14];
    const T e15 = f[15] + f[16], e17 = f[17] + f[18];
    const T Pxx = (f[1] + f[2]) + (e7 + e9) + (e11 + e13);
    const T Pyy = (f[3] + f[4]) + (e7 + e9) + (e15 + e17);
    const T Pzz = (f[5] + f[6]) + (e11 + e13) + (e15 + e17);
    const T Pxy = e7 - e9, Pxz = e11 - e13, Pyz = e15 - e17;
    // N = Pi - R/3 I - S, bulk part nb, shear part N - nb I
    const T R3 = R * third;
    const T Nxx = Pxx - R3 - Sxx, Nyy = Pyy - R3 - Syy, Nzz = Pzz - R3 - Szz;
    const T Nxy = Pxy - Sxy, Nxz = Pxz - Sxz, Nyz = Pyz - Syz;
    const T nb = (Nxx + Nyy + Nzz) * third;
    // G = u F + F u, bulk part gb
    const T Gxx = T(2) * ux * m.Fx, Gyy = T(2) * uy * m.Fy, Gzz = T(2) * uz * m.Fz;
    const T Gxy = ux * m.Fy + uy * m.Fx, Gxz = ux * m.Fz + uz * m.Fx, Gyz = uy * m.Fz + uz * m.Fy;
    const T gb = (Gxx + Gyy + Gzz) * third;
    // S' = w_gh S + X - (1 - w_gh) N; X's bulk terms act on the trace only
    const T xb = m.cb * nb + m.hb * gb - (m.cs * nb + m.hs * gb);   // bulk minus shear rate, times I
    const T a = m.cs - m.cgh;                                       // N's net shear coefficient
    const T Spxx = m.og * Sxx + a * Nxx + m.hs * Gxx + xb;
    const T Spyy = m.og * Syy + a * Nyy + m.hs * Gyy + xb;
    const T Spzz = m.og * Szz + a * Nzz + m.hs * Gzz + xb;
    const T Spxy = m.og * Sxy + a * Nxy + m.hs * Gxy;
    const T Spxz = m.og * Sxz + a * Nxz + m.hs * Gxz;
    const T Spyz = m.og * Syz + a * Nyz + m.hs * Gyz;
    const T t3 = (Spxx + Spyy + Spzz) * third;
    const T Rp = m.og * R;
    const T Jpx = m.og * Jx + m.kf * m.Fx, Jpy = m.og * Jy + m.kf * m.Fy, Jpz = m.og * Jz + m.kf * m.Fz;

    const T cf = m.cgh;
    const T w0 = T(1.0 / 3.0), w1 = T(1.0 / 18.0), w2 = T(1.0 / 36.0);
    const T b = Rp - h * t3;
    f[0] = fmadd(cf, f[0], w0 * b);
    const T B1 = w1 * b, B2 = w2 * b;
    const T f1h = w1 * h, f1t = w1 * T(3), f2h = w2 * h, f2t = w2 * T(3);
#define LBK_MFACE(IP, IM, SAA, JA)                                 \
    {                                                              \
        const T s_ = fmadd(f1h, SAA, B1), a_ = f1t * JA;           \
        f[IP] = fmadd(cf, f[IP], s_ + a_);                         \
        f[IM] = fmadd(cf, f[IM], s_ - a_);                         \
    }
    LBK_MFACE(1, 2, Spxx, Jpx)
    LBK_MFACE(3, 4, Spyy, Jpy)
    LBK_MFACE(5, 6, Spzz, Jpz)
#undef LBK_MFACE
#define LBK_MEDGES(IP, IM, KP, KM, SAA, SBB, SAB, JA, JB)            \
    {                                                                \
        const T e_ = fmadd(f2h, SAA + SBB, B2), o_ = f1h * SAB;      \
        const T sp = e_ + o_, sm = e_ - o_;                          \
        const T ap = f2t * (JA + JB), am = f2t * (JA - JB);          \
        f[IP] = fmadd(cf, f[IP], sp + ap);                           \
        f[IM] = fmadd(cf, f[IM], sp - ap);                           \
        f[KP] = fmadd(cf, f[KP], sm + am);                           \
        f[KM] = fmadd(cf, f[KM], sm - am);                           \
    }
    LBK_MEDGES(7, 8, 9, 10, Spxx, Spyy, Spxy, Jpx, Jpy)
    LBK_MEDGES(11, 12, 13, 14, Spxx, Spzz, Spxz, Jpx, Jpz)
    LBK_MEDGES(15, 16, 17, 18, Spyy, Spzz, Spyz, Jpy, Jpz)
#undef LBK_MEDGES
    collide_g<T>(p, g, phi, ux, uy, uz, mu);
}

}  // namespace lbk
