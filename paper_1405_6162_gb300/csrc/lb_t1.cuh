// lb_t1.cuh -- per-site and per-tile pieces of the tau_g = 1 reduced form,
// shared by the one-lattice kernels (lb_taug1.cu) and the ensemble kernel
// (lb_batch.cu).  The storage and the two passes are described in
// lb_taug1.cu.
#pragma once

#include "d3q19.cuh"
#include "df64.cuh"
#include "lb_site.cuh"

namespace lbk {

// a source site's moments expanded for geq: base by c^2 (0, 1, 2), 3 phi, 9/2 phi, u
template <typename T>
struct Eq {
    T b0, b1, b2, a3, a45, ux, uy, uz;
};

template <typename T>
__device__ __forceinline__ Eq<T> make_eq(T phi, T gmh, T ux, T uy, T uz)
{
    Eq<T> e;
    const T u2 = ux * ux + uy * uy + uz * uz;
    e.b1 = phi - T(1.5) * phi * u2;
    e.b0 = e.b1 - gmh;
    e.b2 = e.b1 + gmh;
    e.a3 = T(3) * phi;
    e.a45 = T(4.5) * phi;
    e.ux = ux;
    e.uy = uy;
    e.uz = uz;
    return e;
}

template <typename T>
__device__ __forceinline__ T gmh_of(T phi, T mu, T gamma)
{
    return T(4.5) * (gamma * mu - phi * T(1.0 / 3.0));
}

// c_i . u with the zero components left out; i a literal after inlining
template <typename T>
__device__ __forceinline__ T cdot(int i, T ux, T uy, T uz)
{
    T r = cx(i) > 0 ? ux : -ux;
    if (cx(i) == 0) r = cy(i) > 0 ? uy : -uy;
    else if (cy(i) != 0) r = cy(i) > 0 ? add_px(r, uy) : sub_px(r, uy);
    if (cx(i) == 0 && cy(i) == 0) r = cz(i) > 0 ? uz : -uz;
    else if (cz(i) != 0) r = cz(i) > 0 ? add_px(r, uz) : sub_px(r, uz);
    return r;
}

// geq_i from expanded moments; i a literal after inlining
template <typename T>
__device__ __forceinline__ T geq_eq(int i, const Eq<T> &e)
{
    const int c2 = cx(i) * cx(i) + cy(i) * cy(i) + cz(i) * cz(i);
    if (c2 == 0) {
        if constexpr (sizeof(T) == 4) {
            // the float weights sum to 1 + e1 and their (c^2 - 1) moment is e2
            // instead of 0 (e1, e2 from the rounded values); the rest term
            // removes the bias e1 P + e2 gmh they would give sum_i geq_i
            constexpr double w0f = double(float(1.0 / 3.0)), w1f = double(float(1.0 / 18.0)),
                             w2f = double(float(1.0 / 36.0));
            constexpr float e1 = float(w0f + 6.0 * w1f + 12.0 * w2f - 1.0);
            constexpr float e2 = float(12.0 * w2f - w0f);
            return T(weight(0)) * e.b0 - (e1 * e.b1 + e2 * (e.b1 - e.b0));
        }
        return T(weight(0)) * e.b0;
    }
    const T cu = cdot(i, e.ux, e.uy, e.uz);
    const T base = c2 == 1 ? e.b1 : e.b2;
    return T(weight(i)) * add_px(base, cu * add_px(e.a3, e.a45 * cu));
}

// The phi pass's form of the equilibria.  For an opposite pair (i, i + 1;
// i odd, c_{i+1} = -c_i) with cu = c_i . u,
//   geq_i = S + A,  geq_{i+1} = S - A,  S = w (b + 9/2 phi cu^2),  A = 3 w phi cu,
// w and b those of the pair's weight class, so that a pair costs one S and
// one A.  The class terms are formed once per source site.
static_assert(cx(2) == -cx(1) && cy(4) == -cy(3) && cz(6) == -cz(5) && cx(8) == -cx(7) && cy(8) == -cy(7) &&
                  cy(10) == -cy(9) && cz(12) == -cz(11) && cz(14) == -cz(13) && cy(16) == -cy(15) &&
                  cz(16) == -cz(15) && cy(18) == -cy(17) && cz(18) == -cz(17),
              "opposite directions are (i, i + 1), i odd");

template <typename T>
struct EqPair {
    T r0;                       // geq_0
    T wb[2], wq[2], wa[2];      // per class (faces, edges): w b, 9/2 w phi, 3 w phi
    T ux, uy, uz;
};

template <typename T>
__device__ __forceinline__ EqPair<T> pair_form(const Eq<T> &e)
{
    EqPair<T> p;
    p.r0 = geq_eq(0, e);
    const T w1 = T(weight(1)), w2 = T(weight(7));
    p.wb[0] = w1 * e.b1;
    p.wb[1] = w2 * e.b2;
    p.wq[0] = w1 * e.a45;
    p.wq[1] = w2 * e.a45;
    p.wa[0] = w1 * e.a3;
    p.wa[1] = w2 * e.a3;
    p.ux = e.ux;
    p.uy = e.uy;
    p.uz = e.uz;
    return p;
}

// the quad (gmh, u) of a site: one vector access
template <typename T>
struct Quad;
template <>
struct Quad<float> {
    static __device__ __forceinline__ void load(const float *__restrict__ q, long long s, float (&v)[4])
    {
        const float4 a = reinterpret_cast<const float4 *>(q)[s];
        v[0] = a.x, v[1] = a.y, v[2] = a.z, v[3] = a.w;
    }
    static __device__ __forceinline__ void store(float *__restrict__ q, long long s, float a, float b, float c,
                                                 float d)
    {
        reinterpret_cast<float4 *>(q)[s] = make_float4(a, b, c, d);
    }
};
template <>
struct Quad<double> {
    static __device__ __forceinline__ void load(const double *__restrict__ q, long long s, double (&v)[4])
    {
        const double2 a = reinterpret_cast<const double2 *>(q)[2 * s], b = reinterpret_cast<const double2 *>(q)[2 * s + 1];
        v[0] = a.x, v[1] = a.y, v[2] = b.x, v[3] = b.y;
    }
    static __device__ __forceinline__ void store(double *__restrict__ q, long long s, double a, double b, double c,
                                                 double d)
    {
        reinterpret_cast<double2 *>(q)[2 * s] = make_double2(a, b);
        reinterpret_cast<double2 *>(q)[2 * s + 1] = make_double2(c, d);
    }
};

template <>
struct Quad<df64> {
    static __device__ __forceinline__ void load(const df64 *__restrict__ q, long long s, df64 (&v)[4])
    {
        const float4 a = reinterpret_cast<const float4 *>(q)[2 * s], b = reinterpret_cast<const float4 *>(q)[2 * s + 1];
        v[0] = df64(a.x, a.y), v[1] = df64(a.z, a.w), v[2] = df64(b.x, b.y), v[3] = df64(b.z, b.w);
    }
    static __device__ __forceinline__ void store(df64 *__restrict__ q, long long s, df64 a, df64 b, df64 c, df64 d)
    {
        reinterpret_cast<float4 *>(q)[2 * s] = make_float4(a.hi, a.lo, b.hi, b.lo);
        reinterpret_cast<float4 *>(q)[2 * s + 1] = make_float4(c.hi, c.lo, d.hi, d.lo);
    }
};

// warp shuffles of one value (a double-float moves as its two floats)
template <typename T>
__device__ __forceinline__ T shfl_up1(T v)
{
    return __shfl_up_sync(0xffffffffu, v, 1);
}
template <typename T>
__device__ __forceinline__ T shfl_down1(T v)
{
    return __shfl_down_sync(0xffffffffu, v, 1);
}
template <>
__device__ __forceinline__ df64 shfl_up1(df64 v)
{
    return df64(__shfl_up_sync(0xffffffffu, v.hi, 1), __shfl_up_sync(0xffffffffu, v.lo, 1));
}
template <>
__device__ __forceinline__ df64 shfl_down1(df64 v)
{
    return df64(__shfl_down_sync(0xffffffffu, v.hi, 1), __shfl_down_sync(0xffffffffu, v.lo, 1));
}

// the quads start at component 1 (S is a multiple of 64 elements, so they are aligned)
template <typename T>
__device__ __forceinline__ const T *quads(const T *g, long long S) { return g + S; }
template <typename T>
__device__ __forceinline__ T *quads(T *g, long long S) { return g + S; }

// moments of site src stored in the reduced form
template <typename T>
__device__ __forceinline__ Eq<T> load_eq(const T *__restrict__ g, long long S, long long src)
{
    T v[4];
    Quad<T>::load(quads(g, S), src, v);
    return make_eq(g[src], v[0], v[1], v[2], v[3]);
}

// The collide pass at site s: pull f, the NP-point stencil of phi(t) from
// component 0 of level a, the general collision's f part; write f* and the
// quad (gmh, u) of (s, t) into level a.
template <typename T, bool SH, int NP>
__device__ __forceinline__ void t1_collide_site(const T *__restrict__ fa, T *__restrict__ ga, T *__restrict__ fb,
                                                const Coll<T> &p, int nx, int ny, int nz, long long S, int s)
{
    const Nbr n(s, nx, ny, nz);
    const T *phi = ga;
    T f[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = fa[(size_t)i * S + n.src(i)];
    const T ph = phi[s];
    T dx, dy, dz, lap;
    stencil_np<NP, T>(phi, n, ph, dx, dy, dz, lap);
    // the general collision's f part; g's result is its equilibrium, kept as moments
    T ux, uy, uz, mu;
    collide_f<T, SH>(p, f, ph, dx, dy, dz, lap, ux, uy, uz, mu);
#pragma unroll
    for (int i = 0; i < Q; i++) fb[(size_t)i * S + s] = f[i];
    Quad<T>::store(quads(ga, S), s, gmh_of(ph, mu, p.gamma), ux, uy, uz);
}

constexpr int kPhiOut = 30;    // output columns per warp

#ifndef LBK_T1_KY32
#define LBK_T1_KY32 1
#endif
#ifndef LBK_T1_KY64
#define LBK_T1_KY64 2
#endif
#ifndef LBK_T1_KYDF
#define LBK_T1_KYDF 2
#endif
template <typename T>
struct PhiTile {
    // y rows per lane (the default launch; lb_set_kernel picks 1, 2 or 4)
    static constexpr int KY = is_df64<T>::value ? LBK_T1_KYDF : sizeof(T) == 8 ? LBK_T1_KY64 : LBK_T1_KY32;
};

__device__ __forceinline__ int wrap_up(int v, int n)
{
    while (v >= n) v -= n;   // v < 2n + 32: a few iterations at most
    return v;
}

// raw moments (phi, gmh, u) of site o
template <typename T>
__device__ __forceinline__ void t1_load_site(const T *__restrict__ ga, const T *__restrict__ q0, int o, T (&d)[5])
{
    T v[4];
    Quad<T>::load(q0, o, v);
    d[0] = ga[o], d[1] = v[0], d[2] = v[1], d[3] = v[2], d[4] = v[3];
}

// The phi pass for the tile of one warp: x columns bx*30 - 1 .. bx*30 + 30
// (lane = column - bx*30 + 1), y rows y0 .. y0 + KY - 1, output planes
// bz*kzc .. bz*kzc + kzc - 1.  No block-level synchronisation.  Source plane
// j of the run (z0 + j - 1, j = 0 .. nzc + 1) is summed row by row; once a
// row's moments are expanded its registers take the same row of plane
// j + 1, so a plane of arithmetic covers each load's latency and one plane
// of raw moments is held.  Site offsets fit an int (N < 2^31).
template <typename T, int KY>
__device__ __forceinline__ void t1_phi_tile(const T *__restrict__ ga, T *__restrict__ gb, int nx, int ny, int nz,
                                            int kzc, long long S, int bx, int y0, int bz, int lane)
{
    if (y0 >= ny) return;   // uniform over the warp
    const int z0 = bz * kzc;
    const int nzc = min(kzc, nz - z0);   // output planes z0 .. z0 + nzc - 1
    const int xu = bx * kPhiOut + lane - 1;   // unwrapped column, -1 .. nx + 30
    const int x = wrap_up(xu + nx, nx);
    const bool out_x = lane >= 1 && lane <= kPhiOut && xu < nx;
    const int plane = nx * ny;
    int yoff[KY + 2];
#pragma unroll
    for (int k = 0; k < KY + 2; k++) yoff[k] = x + wrap_up(y0 - 1 + k + ny, ny) * nx;
    // partial sums of output plane oz live in slot oz mod 3
    T acc[3][KY], acc_r[3][KY], acc_l[3][KY];
#pragma unroll
    for (int q = 0; q < 3; q++)
#pragma unroll
        for (int a = 0; a < KY; a++) acc[q][a] = acc_r[q][a] = acc_l[q][a] = T(0);
    const T *q0 = quads(ga, S);
    T raw[KY + 2][5];
    // source plane 0 of the run
    int zl = wrap_up(z0 - 1 + nz, nz) * plane;   // offset of the next plane to load
#pragma unroll
    for (int r = 0; r < KY + 2; r++) t1_load_site(ga, q0, zl + yoff[r], raw[r]);
    zl += plane;
    if (zl == plane * nz) zl = 0;
    for (int j0 = 0; j0 < nzc + 2; j0 += 3) {
#pragma unroll
        for (int k = 0; k < 3; k++) {
            const int j = j0 + k;
            if (j >= nzc + 2) break;   // uniform over the warp
            const bool more = j + 1 < nzc + 2;   // uniform: plane j + 1 is part of the run
            // the partial sum that direction i of source row ry feeds: output
            // row ry + c_y, slot of output plane j - 1 + c_z, this column or
            // (through the shuffles) column x + c_x
            auto slot = [&](int i, int oy) -> T & {
                const int q = (k + 2 + cz(i)) % 3;
                return cx(i) == 0 ? acc[q][oy] : cx(i) > 0 ? acc_r[q][oy] : acc_l[q][oy];
            };
#pragma unroll
            for (int ry = -1; ry <= KY; ry++) {
                T (&c5)[5] = raw[ry + 1];
                const Eq<T> e = make_eq(c5[0], c5[1], c5[2], c5[3], c5[4]);
                if (more) t1_load_site(ga, q0, zl + yoff[ry + 1], c5);
                if constexpr (is_df64<T>::value) {
                    // double-float: the pair form (measured: 7.59 against 6.21
                    // GLUPS at 256^3; in float and double the compiler already
                    // shares c.u between opposite directions, and the pair
                    // form's longer-lived class terms cost occupancy there)
                    const EqPair<T> ep = pair_form(e);
                    if (ry >= 0 && ry < KY) {
                        T &a = slot(0, ry);
                        a = add_px(a, ep.r0);
                    }
#pragma unroll
                    for (int i = 1; i < Q; i += 2) {
                        const int op = ry + cy(i), om = ry - cy(i);   // output rows of i and i + 1
                        const bool hp = op >= 0 && op < KY, hm = om >= 0 && om < KY;
                        if (!hp && !hm) continue;
                        const int c = i <= 6 ? 0 : 1;
                        const T cu = cdot(i, ep.ux, ep.uy, ep.uz);
                        const T S = fmadd(ep.wq[c] * cu, cu, ep.wb[c]);
                        if (hp) {
                            T &a = slot(i, op);
                            a = fmadd(ep.wa[c], cu, add_px(a, S));    // + S + A
                        }
                        if (hm) {
                            T &a = slot(i + 1, om);
                            a = fmadd(-ep.wa[c], cu, add_px(a, S));   // + S - A
                        }
                    }
                } else {
#pragma unroll
                    for (int i = 0; i < Q; i++) {
                        const int oy = ry + cy(i);
                        if (oy < 0 || oy >= KY) continue;
                        T &a = slot(i, oy);
                        a += geq_eq(i, e);
                    }
                }
            }
            if (more) {
                zl += plane;
                if (zl == plane * nz) zl = 0;
            }
            // output plane j - 2 (slot (k + 1) mod 3) is complete
            const int qd = (k + 1) % 3;
            const int oz = j - 2;
#pragma unroll
            for (int a = 0; a < KY; a++) {
                const T from_left = shfl_up1(acc_r[qd][a]);
                const T from_right = shfl_down1(acc_l[qd][a]);
                if (out_x && oz >= 0 && y0 + a < ny)
                    gb[yoff[a + 1] + (z0 + oz) * plane] = add_px(acc[qd][a], add_px(from_left, from_right));
                acc[qd][a] = acc_r[qd][a] = acc_l[qd][a] = T(0);
            }
        }
    }
}


}  // namespace lbk
