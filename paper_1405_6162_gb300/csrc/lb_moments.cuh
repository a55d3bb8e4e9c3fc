// lb_moments.cuh -- the macroscopic moments of one site in FP64 for output:
// rho = sum f, u = (sum f c + F/2) / rho and phi = sum g of the pulled
// post-streaming distributions f_i(x) = A_i(x - c_i) (targetDP Sec. II.A:
// the moments of the distributions give the hydrodynamic fields).  Shared by
// the whole-lattice and the masked moments kernels so that both give the
// same bits.
//
// GB300 runs FP64 at 1/64 of its FP32 rate, and converting 38 stored values
// to double and summing them there made the output kernel FP64-bound.  So
// float and double-float storage are summed in double-float arithmetic
// (df64.cuh: every float is exact as a double-float; each addition errs by
// ~2^-48 of the larger operand, far below float storage's rounding and
// ~1e-14 over the 18 additions of a double-float sum) and only the sums
// leave for double; double storage is summed in double.
#pragma once

#include "d3q19.cuh"
#include "df64.cuh"
#include "lb_site.cuh"

namespace lbk {

template <typename T>
struct MomentSum {
    using type = double;
};
template <>
struct MomentSum<float> {
    using type = df64;
};
template <>
struct MomentSum<df64> {
    using type = df64;
};

__device__ __forceinline__ df64 moment_term(float v) { return df64(v, 0.0f); }
__device__ __forceinline__ double moment_term(double v) { return v; }
__device__ __forceinline__ df64 moment_term(df64 v) { return v; }

__device__ __forceinline__ double to_double(df64 v) { return double(v); }
__device__ __forceinline__ double to_double(double v) { return v; }

// rho and u at site n (SH: f stored shifted by w_i rho0); hF = F/2
template <typename T, bool SH>
__device__ __forceinline__ void site_rho_u(const T *__restrict__ fa, const Nbr &n, long long S, double rho0,
                                           double hFx, double hFy, double hFz, double &rho, double (&u)[3])
{
    using A = typename MomentSum<T>::type;
    A f[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) f[i] = moment_term(fa[(size_t)i * S + n.src(i)]);
    A R, jx, jy, jz;
    density_moments(f, R, jx, jy, jz);
    rho = SH ? rho0 + to_double(R) : to_double(R);
    const double rinv = 1.0 / rho;
    u[0] = (to_double(jx) + hFx) * rinv;
    u[1] = (to_double(jy) + hFy) * rinv;
    u[2] = (to_double(jz) + hFz) * rinv;
}

// phi at site n of the general form (all 19 g rows)
template <typename T>
__device__ __forceinline__ double site_phi(const T *__restrict__ ga, const Nbr &n, long long S)
{
    using A = typename MomentSum<T>::type;
    A g[Q];
#pragma unroll
    for (int i = 0; i < Q; i++) g[i] = moment_term(ga[(size_t)i * S + n.src(i)]);
    return to_double(sum19(g));
}

}  // namespace lbk
