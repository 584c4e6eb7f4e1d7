// Float-float arithmetic: a value held as an unevaluated sum h + l of two
// floats with |l| <= ulp(h) / 2, carrying about 48 significant bits on the
// FP32 pipes.  It replaces FP64 where the kernels need more than float
// precision: GB300 issues FP64 at a small fraction of its FP32 rate.
//
// Error-free transformations: Knuth's TwoSum, Dekker's FastTwoSum, the
// FMA-based TwoProd (Dekker 1971; Ogita, Rump and Oishi 2005).  On the
// device the _rn intrinsics keep the compiler from contracting or
// reordering the compensated steps; the header also compiles as plain C++
// (built with -ffp-contract=off) so that the host can check the same code.
#pragma once

#include <math.h>

#if defined(__CUDACC__)
#define OSOG_HD __host__ __device__ __forceinline__
#else
#define OSOG_HD inline
#endif

namespace osog {

#if defined(__CUDA_ARCH__)
OSOG_HD float f_add(float a, float b) { return __fadd_rn(a, b); }
OSOG_HD float f_sub(float a, float b) { return __fsub_rn(a, b); }
OSOG_HD float f_mul(float a, float b) { return __fmul_rn(a, b); }
OSOG_HD float f_fma(float a, float b, float c) { return __fmaf_rn(a, b, c); }
OSOG_HD float f_rcp(float a) { return __frcp_rn(a); }
OSOG_HD float f_div(float a, float b) { return __fdiv_rn(a, b); }
OSOG_HD float f_sqrt(float a) { return __fsqrt_rn(a); }
#else
OSOG_HD float f_add(float a, float b) { return a + b; }
OSOG_HD float f_sub(float a, float b) { return a - b; }
OSOG_HD float f_mul(float a, float b) { return a * b; }
OSOG_HD float f_fma(float a, float b, float c) { return fmaf(a, b, c); }
OSOG_HD float f_rcp(float a) { return 1.0f / a; }
OSOG_HD float f_div(float a, float b) { return a / b; }
OSOG_HD float f_sqrt(float a) { return sqrtf(a); }
#endif

struct ff {
    float h, l;
};

OSOG_HD ff two_sum(float a, float b) {
    const float s = f_add(a, b);
    const float bb = f_sub(s, a);
    const float e = f_add(f_sub(a, f_sub(s, bb)), f_sub(b, bb));
    return {s, e};
}
OSOG_HD ff fast_two_sum(float a, float b) {  // |a| >= |b|
    const float s = f_add(a, b);
    return {s, f_sub(b, f_sub(s, a))};
}
OSOG_HD ff two_prod(float a, float b) {  // a b exactly
    const float p = f_mul(a, b);
    return {p, f_fma(a, b, -p)};
}
OSOG_HD ff ff_add(ff a, ff b) {
    const ff s = two_sum(a.h, b.h);
    const float e = f_add(s.l, f_add(a.l, b.l));
    return fast_two_sum(s.h, e);
}
OSOG_HD ff ff_add_f(ff a, float b) {
    const ff s = two_sum(a.h, b);
    return fast_two_sum(s.h, f_add(s.l, a.l));
}
OSOG_HD ff ff_mul(ff a, ff b) {
    const float p = f_mul(a.h, b.h);
    float e = f_fma(a.h, b.h, -p);
    e = f_fma(a.h, b.l, e);
    e = f_fma(a.l, b.h, e);
    return fast_two_sum(p, e);
}
OSOG_HD ff ff_neg(ff a) { return {-a.h, -a.l}; }

// 1 / a of a float a != 0: the correctly rounded reciprocal r leaves a
// residual 1 - a r that a fused multiply-add gives exactly, and
// 1/a = r (1 + e + e^2 + ...) with |e| <= 2^-24.
OSOG_HD ff ff_recip(float a) {
    const float r = f_rcp(a);
    const float e = f_fma(-a, r, 1.0f);
    return fast_two_sum(r, f_mul(r, e));
}
// 1 / d of a float-float d: one Newton step from the float reciprocal of
// d.h, with the residual 1 - d r taken to float-float accuracy.
OSOG_HD ff ff_recip_ff(ff d) {
    const float r = f_rcp(d.h);
    const float e = f_fma(-d.l, r, f_fma(-d.h, r, 1.0f));
    return fast_two_sum(r, f_mul(r, e));
}
// sqrt(d) of a float-float d > 0: the correctly rounded root s of d.h and
// one correction (d - s^2) / (2 s), the residual taken exactly by a fused
// multiply-add.
OSOG_HD ff ff_root(ff d) {
    const float s = f_sqrt(d.h);
    const float e = f_add(f_fma(-s, s, d.h), d.l);
    return fast_two_sum(s, f_div(f_mul(0.5f, e), s));
}

// ------------------------------------------------------- cos and sin
// 1 / n! to double precision (n <= 18, n! exact in double), evaluated by
// the compiler: the constants below are float-float splits of it.
OSOG_HD constexpr double inv_factorial(int n) {
    double f = 1.0;
    for (int i = 2; i <= n; ++i) f *= (double)i;
    return 1.0 / f;
}
template <int N, int SIGN>
struct InvFact {  // SIGN / N! as float-float
    static constexpr double v = SIGN * inv_factorial(N);
    static constexpr float h = (float)v;
    static constexpr float l = (float)(v - (double)h);
};

// pi / 2 as an unevaluated sum of three floats, from its double split
// 1.5707963267948966 + 6.123233995736766e-17 (pi / 2 to 34 digits is
// 1.570796326794896619231321691639751); each step below subtracts nearby
// values, exactly by Sterbenz's lemma.
constexpr double kHalfPiHi = 1.5707963267948966;
constexpr double kHalfPiLo = 6.123233995736766e-17;
constexpr float kHalfPi1 = (float)kHalfPiHi;
constexpr float kHalfPi2 = (float)((kHalfPiHi - (double)kHalfPi1) + kHalfPiLo);
constexpr float kHalfPi3 = (float)(((kHalfPiHi - (double)kHalfPi1) - (double)kHalfPi2) + kHalfPiLo);
constexpr float kMaxReducedAngle = 1048576.0f;  // 2^20 rad

// cos and sin of a float angle th (|th| <= 2^20) as float-float, to about
// 2^-46 absolute.  Cody-Waite reduction x = th - k pi/2 with the three-part
// constant above (every product k pi_i taken exactly by TwoProd), then the
// Taylor series of sin and cos on |x| <= pi/4 (+ rounding of k):
//   sin x = x (1 - u/3! + u^2/5! - ... + u^7/15!),
//   cos x = 1 - u/2! + u^2/4! - ... + u^8/16!,   u = x^2 <= 0.62,
// truncated where the next term is below 2^-54.  The highest terms (u^5 on
// for sin, u^6 on for cos), below 3e-9 in size, are summed in float; the rest
// by float-float Horner steps.  The quadrant k mod 4 then rotates the pair.
OSOG_HD void ff_sincos(float th, ff *c, ff *s) {
    const float k = rintf(f_mul(th, 0.636619772f));
    const ff p1 = two_prod(k, kHalfPi1), p2 = two_prod(k, kHalfPi2);
    ff x = two_sum(th, -p1.h);
    x = ff_add_f(x, -p1.l);
    x = ff_add_f(x, -p2.h);
    x = ff_add_f(x, -p2.l);
    x = ff_add_f(x, -f_mul(k, kHalfPi3));
    const ff u = ff_mul(x, x);
    // sin: float tail u^5 .. u^7, then u^4 .. u^0 in float-float
    float t = f_fma(u.h, (float)InvFact<15, -1>::v, (float)InvFact<13, 1>::v);
    t = f_fma(u.h, t, (float)InvFact<11, -1>::v);
    ff y = {t, 0.f};
    y = ff_add(ff_mul(y, u), ff{InvFact<9, 1>::h, InvFact<9, 1>::l});
    y = ff_add(ff_mul(y, u), ff{InvFact<7, -1>::h, InvFact<7, -1>::l});
    y = ff_add(ff_mul(y, u), ff{InvFact<5, 1>::h, InvFact<5, 1>::l});
    y = ff_add(ff_mul(y, u), ff{InvFact<3, -1>::h, InvFact<3, -1>::l});
    y = ff_add(ff_mul(y, u), ff{1.f, 0.f});
    const ff sn = ff_mul(x, y);
    // cos: float tail u^6 .. u^8, then u^5 .. u^0 in float-float
    t = f_fma(u.h, (float)InvFact<16, 1>::v, (float)InvFact<14, -1>::v);
    t = f_fma(u.h, t, (float)InvFact<12, 1>::v);
    y = {t, 0.f};
    y = ff_add(ff_mul(y, u), ff{InvFact<10, -1>::h, InvFact<10, -1>::l});
    y = ff_add(ff_mul(y, u), ff{InvFact<8, 1>::h, InvFact<8, 1>::l});
    y = ff_add(ff_mul(y, u), ff{InvFact<6, -1>::h, InvFact<6, -1>::l});
    y = ff_add(ff_mul(y, u), ff{InvFact<4, 1>::h, InvFact<4, 1>::l});
    y = ff_add(ff_mul(y, u), ff{InvFact<2, -1>::h, InvFact<2, -1>::l});
    const ff cs = ff_add(ff_mul(y, u), ff{1.f, 0.f});
    const int q = (int)k & 3;  // two's complement: -1 & 3 = 3
    *c = q == 0 ? cs : q == 1 ? ff_neg(sn) : q == 2 ? ff_neg(cs) : sn;
    *s = q == 0 ? sn : q == 1 ? cs : q == 2 ? ff_neg(sn) : ff_neg(cs);
}

// The row quadric of an ellipse with semi-axes a, b and direction (c, s):
// with D = b^2 c^2 + a^2 s^2 (alpha = D / (a^2 b^2), the coefficient of x^2
// in (u/a)^2 + (v/b)^2 along a row),
//   m = -c s (b^2 - a^2) / D,   1/alpha = a^2 b^2 / D,
//   kappa = a^2 b^2 / D^2,      sqrt(alpha) = sqrt(D) / (a b),
// all in float-float from one reciprocal of D.
struct Quadric {
    ff m, inv_alpha, kappa, sqrt_alpha;
};
OSOG_HD Quadric ellipse_quadric(float a, float b, ff c, ff s) {
    const ff a2 = two_prod(a, a), b2 = two_prod(b, b);
    const ff D = ff_add(ff_mul(b2, ff_mul(c, c)), ff_mul(a2, ff_mul(s, s)));
    const ff R = ff_recip_ff(D);
    const ff ab2 = ff_mul(a2, b2);
    Quadric q;
    q.m = ff_neg(ff_mul(ff_mul(ff_mul(c, s), ff_add(b2, ff_neg(a2))), R));
    q.inv_alpha = ff_mul(ab2, R);
    q.kappa = ff_mul(ab2, ff_mul(R, R));
    q.sqrt_alpha = ff_mul(ff_root(D), ff_recip_ff(two_prod(a, b)));
    return q;
}

}  // namespace osog
