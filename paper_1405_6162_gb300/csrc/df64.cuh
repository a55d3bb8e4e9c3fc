// df64.cuh -- double-float arithmetic: a value is the unevaluated sum hi + lo
// of two floats with |lo| <= ulp(hi)/2, about 48 significant bits, computed
// entirely on the FP32 pipe.
//
// GB300 executes FP64 at 1/64 of its FP32 rate; the FP64 step is bound by
// that pipe.  This type lets the same templated collision run at FP64-class
// accuracy (unit roundoff ~2^-48 instead of 2^-53) on the FP32 units.
//
// The building blocks are the error-free transformations of Knuth (TwoSum)
// and Dekker (Fast2Sum), and the fused-multiply-add form of TwoProduct
// (a*b = p + e exactly with e = fma(a, b, -p)); addition follows the
// accurate double-double addition (both component pairs summed exactly, two
// renormalisations, or the cheaper form with the low parts added to the
// error term), multiplication keeps the cross terms hi*lo.  Every
// float operation is written with the _rn intrinsics so that the compiler
// cannot contract a product and a sum into one FMA, which would break the
// error-free transformations.
#pragma once

#include <cuda_runtime.h>

namespace lbk {

struct __align__(8) df64 {
    float hi, lo;

    df64() = default;
    __host__ __device__ constexpr df64(float h, float l) : hi(h), lo(l) {}
    // round a double to the nearest double-float (hi = float(d), lo = the
    // float nearest to the remainder)
    __host__ __device__ constexpr explicit df64(double d)
        : hi(static_cast<float>(d)), lo(static_cast<float>(d - static_cast<double>(static_cast<float>(d)))) {}
    __host__ __device__ constexpr explicit df64(int i) : df64(static_cast<double>(i)) {}
    __host__ __device__ constexpr explicit operator double() const
    {
        return static_cast<double>(hi) + static_cast<double>(lo);
    }
};

template <typename T>
struct is_df64 {
    static constexpr bool value = false;
};
template <>
struct is_df64<df64> {
    static constexpr bool value = true;
};

namespace dfops {

// s + e = a + b exactly (Knuth)
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    const float bb = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb));
}

// s + e = a + b exactly when |a| >= |b| (Dekker)
__device__ __forceinline__ void fast_two_sum(float a, float b, float &s, float &e)
{
    s = __fadd_rn(a, b);
    e = __fsub_rn(b, __fsub_rn(s, a));
}

}  // namespace dfops

// Two floats in one 64-bit register (the first value in the low half) and
// the paired FP32 instructions of sm_100 and later (add/sub/mul/fma
// .rn.f32x2): one issue computes both halves, each rounded as its scalar
// instruction would be.  Plain asm with outputs only, so the compiler may
// merge or drop them like ordinary arithmetic.
namespace px2 {

__device__ __forceinline__ unsigned long long pack(float lo, float hi)
{
    unsigned long long r;
    asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
    return r;
}
__device__ __forceinline__ void unpack(unsigned long long v, float &lo, float &hi)
{
    asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}
__device__ __forceinline__ unsigned long long add(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("add.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long sub(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long mul(unsigned long long a, unsigned long long b)
{
    unsigned long long r;
    asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
    return r;
}
__device__ __forceinline__ unsigned long long fma(unsigned long long a, unsigned long long b, unsigned long long c)
{
    unsigned long long r;
    asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
    return r;
}
__device__ __forceinline__ void two_sum(unsigned long long a, unsigned long long b, unsigned long long &s,
                                        unsigned long long &e)
{
    s = add(a, b);
    const unsigned long long bb = sub(s, a);
    e = add(sub(a, sub(s, bb)), sub(b, bb));
}

}  // namespace px2

#ifndef LBK_DF64_ACCURATE_ADD
#define LBK_DF64_ACCURATE_ADD 0
#endif

__device__ __forceinline__ df64 operator+(df64 a, df64 b)
{
#if LBK_DF64_ACCURATE_ADD
    // both component pairs summed exactly: error ~2^-48 of the result
    float s1, s2, t1, t2;
    dfops::two_sum(a.hi, b.hi, s1, s2);
    dfops::two_sum(a.lo, b.lo, t1, t2);
    s2 = __fadd_rn(s2, t1);
    dfops::fast_two_sum(s1, s2, s1, s2);
    s2 = __fadd_rn(s2, t2);
    df64 r;
    dfops::fast_two_sum(s1, s2, r.hi, r.lo);
    return r;
#else
    // the high parts summed exactly, the low parts added to the error: error
    // ~2^-48 of the larger operand (the absolute accuracy double arithmetic
    // gives a sum of such operands)
    float s, e;
    dfops::two_sum(a.hi, b.hi, s, e);
    e = __fadd_rn(e, __fadd_rn(a.lo, b.lo));
    df64 r;
    dfops::fast_two_sum(s, e, r.hi, r.lo);
    return r;
#endif
}

__device__ __forceinline__ df64 operator-(df64 a) { return df64(-a.hi, -a.lo); }
__device__ __forceinline__ df64 operator-(df64 a, df64 b) { return a + (-b); }

// a + b bitwise as operator+ (the cheaper form), with the high parts' sum
// and the low parts' sum issued as one paired instruction.  Whether that
// pays depends on the kernel's register allocation (measured: the reduced
// form's phi pass gains, the two-pass collision loses), so the kernels
// choose it per call site.
__device__ __forceinline__ df64 add_px(df64 a, df64 b)
{
    float s, l;
    px2::unpack(px2::add(px2::pack(a.hi, a.lo), px2::pack(b.hi, b.lo)), s, l);
    const float bb = __fsub_rn(s, a.hi);
    float e = __fadd_rn(__fsub_rn(a.hi, __fsub_rn(s, bb)), __fsub_rn(b.hi, bb));
    e = __fadd_rn(e, l);
    df64 r;
    dfops::fast_two_sum(s, e, r.hi, r.lo);
    return r;
}
__device__ __forceinline__ df64 sub_px(df64 a, df64 b) { return add_px(a, -b); }
__device__ __forceinline__ float add_px(float a, float b) { return a + b; }
__device__ __forceinline__ float sub_px(float a, float b) { return a - b; }
__device__ __forceinline__ double add_px(double a, double b) { return a + b; }
__device__ __forceinline__ double sub_px(double a, double b) { return a - b; }

__device__ __forceinline__ df64 operator*(df64 a, df64 b)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    df64 r;
    dfops::fast_two_sum(p, e, r.hi, r.lo);
    return r;
}

// x / 2: both parts halved, exactly (barring underflow)
__device__ __forceinline__ df64 half(df64 a) { return df64(0.5f * a.hi, 0.5f * a.lo); }

// a / b: a float quotient refined twice by the residual a - q b
__device__ __forceinline__ df64 operator/(df64 a, df64 b)
{
    const float q1 = __fdiv_rn(a.hi, b.hi);
    const df64 r1 = a - b * df64(q1, 0.0f);
    const float q2 = __fdiv_rn(r1.hi, b.hi);
    const df64 r2 = r1 - b * df64(q2, 0.0f);
    const float q3 = __fdiv_rn(r2.hi, b.hi);
    float s, e;
    dfops::fast_two_sum(q1, q2, s, e);
    return df64(s, e) + df64(q3, 0.0f);
}

// a * b + c with the product's error terms folded into the addition
__device__ __forceinline__ df64 fmadd(df64 a, df64 b, df64 c)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s, t;
    dfops::two_sum(p, c.hi, s, t);
    t = __fadd_rn(t, __fadd_rn(e, c.lo));
    df64 r;
    dfops::fast_two_sum(s, t, r.hi, r.lo);
    return r;
}

// a * b + (c + d) renormalised once: the product's error terms, the two
// exact sums' errors (c.hi + d.hi, then the product) and the low parts are
// added to one error term (23 float operations instead of the 26 of
// fmadd(a, b, c + d), the same ~2^-48 bound relative to the largest term)
__device__ __forceinline__ df64 fmadd_sum(df64 a, df64 b, df64 c, df64 d)
{
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    float s1, t1, s, t2;
    dfops::two_sum(c.hi, d.hi, s1, t1);
    dfops::two_sum(p, s1, s, t2);
    const float t = __fadd_rn(__fadd_rn(t1, t2), __fadd_rn(e, __fadd_rn(c.lo, d.lo)));
    df64 r;
    dfops::fast_two_sum(s, t, r.hi, r.lo);
    return r;
}


// The relaxation of an opposite pair, fp = c fp + (s + a) and
// fm = c fm + (s - a), each fmadd_sum's float sequence, both values through
// one pass of paired FP32 instructions (bitwise the two fmadd_sum results;
// half the issue slots for this part of the collision).
__device__ __forceinline__ void relax_pair(df64 c, df64 &fp, df64 &fm, df64 s, df64 a)
{
    using namespace px2;
    const unsigned long long ch = pack(c.hi, c.hi), cl = pack(c.lo, c.lo);
    const unsigned long long bh = pack(fp.hi, fm.hi), bl = pack(fp.lo, fm.lo);
    const unsigned long long sh = pack(s.hi, s.hi), sl = pack(s.lo, s.lo);
    const unsigned long long ah = pack(a.hi, -a.hi), al = pack(a.lo, -a.lo);
    const unsigned long long p = mul(ch, bh);
    float p0, p1;
    unpack(p, p0, p1);
    unsigned long long e = fma(ch, bh, pack(-p0, -p1));
    e = fma(ch, bl, e);
    e = fma(cl, bh, e);
    unsigned long long s1, t1, sum, t2;
    two_sum(sh, ah, s1, t1);
    two_sum(p, s1, sum, t2);
    const unsigned long long t = add(add(t1, t2), add(e, add(sl, al)));
    // fast two-sum of (sum, t)
    const unsigned long long rh = add(sum, t);
    const unsigned long long rl = sub(t, sub(rh, sum));
    unpack(rh, fp.hi, fm.hi);
    unpack(rl, fp.lo, fm.lo);
}

__device__ __forceinline__ df64 &operator+=(df64 &a, df64 b) { return a = a + b; }
__device__ __forceinline__ df64 &operator-=(df64 &a, df64 b) { return a = a - b; }
__device__ __forceinline__ df64 &operator*=(df64 &a, df64 b) { return a = a * b; }

}  // namespace lbk
