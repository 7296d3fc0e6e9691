// Float-float ("double-single") arithmetic on the FP32 pipe.
//
// A value is the unevaluated sum hi + lo of two floats with |lo| <= ulp(hi)/2,
// about 48 significant bits. The building blocks are the error-free
// transformations of floating-point arithmetic:
//   * Knuth's TwoSum (The Art of Computer Programming, vol. 2, 4.2.2): a + b =
//     s + e exactly for any floats a, b, with s = fl(a + b);
//   * Dekker's FastTwoSum (Dekker 1971, "A floating-point technique for
//     extending the available precision"): the same with three operations when
//     |a| >= |b|;
//   * the FMA form of Dekker's TwoProduct: a b = p + e exactly, p = fl(a b),
//     e = fma(a, b, -p).
// Addition and multiplication of float-float values follow Dekker's
// double-length operations built from these; division and square root take
// one correction step of the float quotient or root against its float-float
// residual. Every operation that must round on its own uses an explicitly
// rounded intrinsic, so that the compiler cannot contract it into an FMA.
//
// These routines serve the refinement of the final iteration: residuals of
// the Kalman and RTS recursions evaluated to about 1e-14 relative from FP32
// inputs, at roughly a tenth of FP32 throughput (the FP64 pipe of this GPU
// runs at 1/64 of the FP32 rate).
#pragma once

#include "pes_math.cuh"

namespace pes {

struct ff {
    float hi, lo;
};

PES_DEV ff ff_make(float a) { return ff{a, 0.0f}; }

// TwoSum: s + e = a + b exactly.
PES_DEV ff two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float bv = __fsub_rn(s, a);
    const float av = __fsub_rn(s, bv);
    const float e = __fadd_rn(__fsub_rn(a, av), __fsub_rn(b, bv));
    return ff{s, e};
}

// FastTwoSum: s + e = a + b exactly when |a| >= |b| (or a = 0).
PES_DEV ff fast_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b);
    const float e = __fsub_rn(b, __fsub_rn(s, a));
    return ff{s, e};
}

// TwoProduct: p + e = a b exactly (barring underflow).
PES_DEV ff two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    const float e = __fmaf_rn(a, b, -p);
    return ff{p, e};
}

PES_DEV ff ff_neg(ff x) { return ff{-x.hi, -x.lo}; }

// x + y (Dekker's addition: the error is below about 2^-46 (|x| + |y|)).
PES_DEV ff ff_add(ff x, ff y)
{
    const ff s = two_sum(x.hi, y.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(x.lo, y.lo));
    return fast_two_sum(s.hi, e);
}

PES_DEV ff ff_sub(ff x, ff y) { return ff_add(x, ff_neg(y)); }

PES_DEV ff ff_add_f(ff x, float b)
{
    const ff s = two_sum(x.hi, b);
    return fast_two_sum(s.hi, __fadd_rn(s.lo, x.lo));
}

// a - b for floats, exactly.
PES_DEV ff ff_diff_f(float a, float b) { return two_sum(a, -b); }

// x y
PES_DEV ff ff_mul(ff x, ff y)
{
    const ff p = two_prod(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.lo, p.lo);
    e = __fmaf_rn(x.lo, y.hi, e);
    return fast_two_sum(p.hi, e);
}

// x b for a float b
PES_DEV ff ff_mul_f(ff x, float b)
{
    const ff p = two_prod(x.hi, b);
    return fast_two_sum(p.hi, __fmaf_rn(x.lo, b, p.lo));
}

// acc + x y, with the product's low part folded into the sum's
PES_DEV ff ff_fma(ff x, ff y, ff acc)
{
    const ff p = two_prod(x.hi, y.hi);
    float e = __fmaf_rn(x.hi, y.lo, p.lo);
    e = __fmaf_rn(x.lo, y.hi, e);
    const ff s = two_sum(acc.hi, p.hi);
    const float t = __fadd_rn(s.lo, __fadd_rn(acc.lo, e));
    return fast_two_sum(s.hi, t);
}

// acc + x b for a float b
PES_DEV ff ff_fma_f(ff x, float b, ff acc)
{
    const ff p = two_prod(x.hi, b);
    const float e = __fmaf_rn(x.lo, b, p.lo);
    const ff s = two_sum(acc.hi, p.hi);
    const float t = __fadd_rn(s.lo, __fadd_rn(acc.lo, e));
    return fast_two_sum(s.hi, t);
}

// acc + a b for floats a, b
PES_DEV ff ff_fma_ff(float a, float b, ff acc)
{
    const ff p = two_prod(a, b);
    const ff s = two_sum(acc.hi, p.hi);
    const float t = __fadd_rn(s.lo, __fadd_rn(acc.lo, p.lo));
    return fast_two_sum(s.hi, t);
}

// A dot-product accumulator in the manner of Ogita, Rump and Oishi's Dot2
// ("Accurate sum and dot product", 2005): TwoSum of the running sum with each
// product's high part, every rounding error (of the products and of the sums)
// collected in a plain float, one renormalisation at the end. The result is as
// accurate as if the dot product were formed in twice the working precision,
// with three fewer operations per term than a float-float fma.
struct ffacc {
    float s, c;
};

PES_DEV ffacc acc_of(ff x) { return ffacc{x.hi, x.lo}; }
PES_DEV ffacc acc_of_f(float x) { return ffacc{x, 0.0f}; }

// a += x b (x float-float, b float)
PES_DEV void acc_add(ffacc& a, ff x, float b)
{
    const ff p = two_prod(x.hi, b);
    const ff t = two_sum(a.s, p.hi);
    a.s = t.hi;
    a.c = __fadd_rn(a.c, __fadd_rn(t.lo, __fmaf_rn(x.lo, b, p.lo)));
}

// a += x b (floats)
PES_DEV void acc_add(ffacc& a, float x, float b)
{
    const ff p = two_prod(x, b);
    const ff t = two_sum(a.s, p.hi);
    a.s = t.hi;
    a.c = __fadd_rn(a.c, __fadd_rn(t.lo, p.lo));
}

// a += x y (float-float)
PES_DEV void acc_add(ffacc& a, ff x, ff y)
{
    const ff p = two_prod(x.hi, y.hi);
    const float e = __fmaf_rn(x.lo, y.hi, __fmaf_rn(x.hi, y.lo, p.lo));
    const ff t = two_sum(a.s, p.hi);
    a.s = t.hi;
    a.c = __fadd_rn(a.c, __fadd_rn(t.lo, e));
}

// a += x (float-float)
PES_DEV void acc_add(ffacc& a, ff x)
{
    const ff t = two_sum(a.s, x.hi);
    a.s = t.hi;
    a.c = __fadd_rn(a.c, __fadd_rn(t.lo, x.lo));
}

PES_DEV ff acc_done(ffacc a) { return two_sum(a.s, a.c); }

// 1 / y: the float reciprocal corrected once by its float-float residual.
PES_DEV ff ff_rcp(ff y)
{
    const float q = __frcp_rn(y.hi);
    // r = 1 - q y
    const ff qy = ff_mul_f(y, q);
    const ff r = ff_sub(ff{1.0f, 0.0f}, qy);
    return fast_two_sum(q, __fmul_rn(r.hi, q));
}

// x / y
PES_DEV ff ff_div(ff x, ff y)
{
    const float ry = __frcp_rn(y.hi);
    const float q1 = __fmul_rn(x.hi, ry);
    const ff r = ff_sub(x, ff_mul_f(y, q1));
    const float q2 = __fmul_rn(r.hi, ry);
    const ff q = fast_two_sum(q1, q2);
    // a second correction: the float reciprocal is correctly rounded, but the
    // first quotient can carry two rounding errors
    const ff r2 = ff_sub(x, ff_mul(y, q));
    return ff_add_f(q, __fmul_rn(r2.hi, ry));
}

// sqrt(x) for x > 0: the float root corrected once (Newton step on s^2 = x).
PES_DEV ff ff_sqrt(ff x)
{
    const float s = __fsqrt_rn(x.hi);
    const ff r = ff_sub(x, two_prod(s, s));
    return fast_two_sum(s, __fmul_rn(r.hi, __frcp_rn(2.0f * s)));
}

PES_DEV float ff_to_f(ff x) { return __fadd_rn(x.hi, x.lo); }

// Taylor coefficients as float-float pairs: (-1)^k / (2k+1)! (sine) and
// (-1)^k / (2k+2)! (one minus cosine), k = 0 .. 9.
__constant__ const float kSinC[10][2] = {
    {1.0f, 0.0f},
    {-0.1666666716337204f, 4.967053879312289e-09f},
    {0.008333333767950535f, -4.34617203337595e-10f},
    {-0.00019841270113829523f, 2.725596874933456e-12f},
    {2.7557318844628753e-06f, 3.793571224297229e-14f},
    {-2.5052107943679403e-08f, -4.4176230446483665e-16f},
    {1.6059044372074283e-10f, -5.352526511562726e-18f},
    {-7.647163609812713e-13f, -1.2200710471178288e-20f},
    {2.8114573589663704e-15f, -1.0462084739763658e-22f},
    {-8.220635078476521e-18f, -1.681478096855898e-25f}};
__constant__ const float kOmcC[10][2] = {
    {0.5f, 0.0f},
    {-0.0416666679084301f, 1.2417634698280722e-09f},
    {0.0013888889225199819f, -3.3631094437103215e-11f},
    {-2.4801587642286904e-05f, 3.40699609366682e-13f},
    {2.755731998149713e-07f, -7.575112209051195e-15f},
    {-2.0876755879584152e-09f, -1.1082839147459852e-16f},
    {1.147074536050896e-11f, 2.372207689231238e-19f},
    {-4.7794772561329454e-14f, -7.62544404448643e-22f},
    {1.5619206814541513e-16f, 1.5404471465941993e-24f},
    {-4.110317590937049e-19f, -3.237511732860265e-27f}};

// sin(a) and 1 - cos(a) for |a| <= pi/4 by their Taylor series (Horner in
// a^2, through a^19 and a^20: the first omitted terms are below 2^-60 of the
// sums there). For |a| < 1/16 six terms reach the same accuracy.
PES_DEV void ff_sin_omc_small(ff a, ff* sn, ff* omc)
{
    const ff a2 = ff_mul(a, a);
    const int top = fabsf(a.hi) < 0.0625f ? 5 : 9;
    ff ps = ff{kSinC[top][0], kSinC[top][1]};
    ff pc = ff{kOmcC[top][0], kOmcC[top][1]};
#pragma unroll 1
    for (int k = top - 1; k >= 0; --k) {
        ps = ff_fma(a2, ps, ff{kSinC[k][0], kSinC[k][1]});
        pc = ff_fma(a2, pc, ff{kOmcC[k][0], kOmcC[k][1]});
    }
    *sn = ff_mul(a, ps);
    *omc = ff_mul(a2, pc);
}

// sin(a), cos(a) and 1 - cos(a) for |a| < 2^11: reduction by the nearest
// multiple n of pi/2 (Cody and Waite's split of pi/2 into P1 + P2 + P3, whose
// first two parts have few enough bits that n P1 and n P2 are exact), then the
// series.
PES_DEV void ff_sincos(ff a, ff* sn, ff* cs, ff* omc)
{
    const float n = rintf(__fmul_rn(a.hi, 0.6366197466850281f));
    ff r = a;
    if (n != 0.0f) {
        const float P1 = 1.5703125f;                     // 8 significant bits
        const float P2 = 4.8375129699707031e-04f;        // 12 significant bits
        const float P3 = 7.549790126404332e-08f;         // pi/2 - P1 - P2, to float
        r = ff_add_f(r, -__fmul_rn(n, P1));
        r = ff_add_f(r, -__fmul_rn(n, P2));
        r = ff_sub(r, two_prod(n, P3));
    }
    ff s, o;
    ff_sin_omc_small(r, &s, &o);
    const ff c = ff_sub(ff_make(1.0f), o);
    const int q = ((int)n) & 3;
    if (q == 0) {
        *sn = s;
        *cs = c;
        *omc = o;
    } else if (q == 1) {   // sin(r + pi/2) = cos r, cos(r + pi/2) = -sin r
        *sn = c;
        *cs = ff_neg(s);
        *omc = ff_add_f(s, 1.0f);
    } else if (q == 2) {
        *sn = ff_neg(s);
        *cs = ff_neg(c);
        *omc = ff_add_f(c, 1.0f);
    } else {
        *sn = ff_neg(c);
        *cs = s;
        *omc = ff_sub(ff_make(1.0f), s);
    }
}

}  // namespace pes
