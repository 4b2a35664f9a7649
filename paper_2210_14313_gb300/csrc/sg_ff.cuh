// Float-float ("FF") arithmetic for the fold: a value is an unevaluated sum
// hi + lo of two floats with |lo| <= ulp(hi)/2, about 44 significant bits.
// Everything runs on the FP32 pipes, which GB300 has at 72x the rate of its
// FP64 pipe.  The error-free transformations are Knuth's TwoSum and the
// FMA-based TwoProduct (Dekker 1971 / Ogita, Rump & Oishi 2005); the
// explicit __f*_rn intrinsics keep the compiler from contracting or
// reassociating them.
#pragma once
#include <cuda_runtime.h>

struct ff2 {
    float hi, lo;
};

__device__ __forceinline__ ff2 ff_make(float hi, float lo) { return ff2{hi, lo}; }

// Splits a double into hi + lo (exact up to the double's 53 bits minus 48).
__device__ __forceinline__ ff2 ff_from_double(double v) {
    const float hi = (float)v;
    return ff2{hi, (float)(v - (double)hi)};
}

__device__ __forceinline__ double ff_to_double(ff2 a) { return (double)a.hi + (double)a.lo; }

// s + e == a + b exactly, |a| >= |b| required.
__device__ __forceinline__ ff2 ff_fast_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    return ff2{s, __fsub_rn(b, __fsub_rn(s, a))};
}

// s + e == a + b exactly, any order.
__device__ __forceinline__ ff2 ff_two_sum(float a, float b) {
    const float s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    return ff2{s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z))};
}

__device__ __forceinline__ ff2 ff_add(ff2 a, ff2 b) {
    ff2 s = ff_two_sum(a.hi, b.hi);
    const float e = __fadd_rn(s.lo, __fadd_rn(a.lo, b.lo));
    return ff_fast_two_sum(s.hi, e);
}

__device__ __forceinline__ ff2 ff_add_f(ff2 a, float b) {
    ff2 s = ff_two_sum(a.hi, b);
    return ff_fast_two_sum(s.hi, __fadd_rn(s.lo, a.lo));
}

__device__ __forceinline__ ff2 ff_mul(ff2 a, ff2 b) {
    const float p = __fmul_rn(a.hi, b.hi);
    float e = __fmaf_rn(a.hi, b.hi, -p);
    e = __fmaf_rn(a.hi, b.lo, e);
    e = __fmaf_rn(a.lo, b.hi, e);
    return ff_fast_two_sum(p, e);
}

__device__ __forceinline__ ff2 ff_mul_f(ff2 a, float b) {
    const float p = __fmul_rn(a.hi, b);
    float e = __fmaf_rn(a.hi, b, -p);
    e = __fmaf_rn(a.lo, b, e);
    return ff_fast_two_sum(p, e);
}

// One float-float Horner step: a * x + c.
__device__ __forceinline__ ff2 ff_horner(ff2 a, ff2 x, ff2 c) { return ff_add(ff_mul(a, x), c); }

// expm1 of a float-float argument (|x| below ~87; below -87 the result is
// -1 to float-float precision).  Cody & Waite reduction x = k ln2 + r with
// ln 2 in three floats (k * ln2_hi exact), the Taylor series of expm1(r) on
// |r| <= ln2/2: terms r^j/j! for j >= 7 in float (their rounding stays
// below 2e-14 relative), j <= 6 in float-float; then
// expm1(x) = 2^k expm1(r) + (2^k - 1) with 2^k - 1 exact as a float pair.
// The low part x.lo enters as expm1(x) = E + (1 + E) expm1(x.lo).
__device__ __forceinline__ ff2 ff_expm1(ff2 x) {
    const float k = fminf(fmaxf(rintf(x.hi * 1.44269502e+00f), -126.f), 127.f);
    const float r_hi = __fmaf_rn(-k, 6.93145752e-01f, x.hi);  // exact
    ff2 t = ff2{__fmul_rn(-k, 1.42860677e-06f), 0.f};
    t.lo = __fmaf_rn(-k, 1.42860677e-06f, -t.hi);
    t.lo = __fmaf_rn(-k, 5.49792315e-14f, t.lo);
    ff2 r = ff_add(ff2{r_hi, 0.f}, t);
    // float tail: sum_{j>=7} r^(j-7)/j!, j = 7..11
    float q = __fmaf_rn(r.hi, 2.50521079e-08f, 2.75573200e-07f);
    q = __fmaf_rn(q, r.hi, 2.75573188e-06f);
    q = __fmaf_rn(q, r.hi, 2.48015876e-05f);
    q = __fmaf_rn(q, r.hi, 1.98412701e-04f);
    // float-float Horner for j = 6 .. 1
    ff2 h = ff_add(ff_mul_f(r, q), ff2{1.38888892e-03f, -3.36310944e-11f});  // 1/6!
    h = ff_horner(h, r, ff2{8.33333377e-03f, -4.34617203e-10f});            // 1/5!
    h = ff_horner(h, r, ff2{4.16666679e-02f, -1.24176347e-09f});            // 1/4!
    h = ff_horner(h, r, ff2{1.66666672e-01f, -4.96705388e-09f});            // 1/3!
    h = ff_horner(h, r, ff2{0.5f, 0.f});                                     // 1/2!
    h = ff_horner(h, r, ff2{1.0f, 0.f});
    ff2 p = ff_mul(h, r);  // expm1(r)
    const int ki = (int)k;
    const float scale = __int_as_float((ki + 127) << 23);
    ff2 e;
    if (ki == 0) {
        e = p;
    } else {
        ff2 ps = ff2{p.hi * scale, p.lo * scale};  // exact scaling by 2^k
        ff2 m1 = ki > 0 ? ff_fast_two_sum(scale, -1.0f) : ff_fast_two_sum(-1.0f, scale);  // 2^k - 1
        e = ff_add(ps, m1);
    }
    // contribution of x.lo: (1 + E) expm1(x.lo), expm1(x.lo) = x.lo + x.lo^2/2 to
    // well below float-float precision (|x.lo| <= 2^-25 |x.hi|; the square
    // term matters once |x| is large, where (1 + E) x.lo^2 / 2 is not small
    // against E)
    const float xl = __fmaf_rn(0.5f * x.lo, x.lo, x.lo);
    const float corr = __fmaf_rn(e.hi, xl, xl);
    return ff_add_f(e, corr);
}

// sin and cos of a float-float argument: x = k pi/2 + r with pi/2 in four
// floats (the first two with 12 significant bits, so k * part is exact for
// |k| < 2^11), Taylor series on |r| <= pi/4 with the terms up to r^9 (sin)
// and r^8 (cos) in float-float and the rest in float, quadrant by k mod 4.
// |x| >= 3000 goes through double sincos (exact to float-float precision).
__device__ __forceinline__ void ff_sincos(ff2 x, ff2 *s, ff2 *c) {
    if (fabsf(x.hi) >= 3000.f) {
        double ds, dc;
        sincos(ff_to_double(x), &ds, &dc);
        *s = ff_from_double(ds);
        *c = ff_from_double(dc);
        return;
    }
    const float k = rintf(x.hi * 6.36619747e-01f);
    ff2 r = ff2{__fmaf_rn(-k, 1.57080078e+00f, x.hi), 0.f};             // exact
    r = ff_add_f(r, __fmul_rn(-k, -4.45358455e-06f));                    // exact product
    ff2 t = ff2{__fmul_rn(-k, -8.70551575e-10f), 0.f};
    t.lo = __fmaf_rn(-k, -8.70551575e-10f, -t.hi);
    t.lo = __fmaf_rn(-k, 5.72118892e-18f, t.lo);
    r = ff_add(r, t);
    r = ff_add_f(r, x.lo);
    const ff2 z = ff_mul(r, r);
    // sin r = r (1 + z (-1/3! + z (1/5! + z (-1/7! + z (1/9! + z q)))))
    float qs = __fmaf_rn(z.hi, -7.64716361e-13f, 1.60590444e-10f);  // -1/15!, 1/13!
    qs = __fmaf_rn(qs, z.hi, -2.50521079e-08f);                     // -1/11!
    ff2 hs = ff_add(ff_mul_f(z, qs), ff2{2.75573188e-06f, 3.79357122e-14f});   // 1/9!
    hs = ff_horner(hs, z, ff2{-1.98412701e-04f, 2.72559688e-12f});            // -1/7!
    hs = ff_horner(hs, z, ff2{8.33333377e-03f, -4.34617203e-10f});            // 1/5!
    hs = ff_horner(hs, z, ff2{-1.66666672e-01f, 4.96705388e-09f});            // -1/3!
    hs = ff_horner(hs, z, ff2{1.0f, 0.f});
    const ff2 sn = ff_mul(hs, r);
    // cos r = 1 + z (-1/2! + z (1/4! + z (-1/6! + z (1/8! + z q))))
    float qc = __fmaf_rn(z.hi, -1.14707454e-11f, 2.08767559e-09f);  // -1/14!, 1/12!
    qc = __fmaf_rn(qc, z.hi, -2.75573200e-07f);                     // -1/10!
    ff2 hc = ff_add(ff_mul_f(z, qc), ff2{2.48015876e-05f, -3.40699609e-13f});  // 1/8!
    hc = ff_horner(hc, z, ff2{-1.38888892e-03f, 3.36310944e-11f});            // -1/6!
    hc = ff_horner(hc, z, ff2{4.16666679e-02f, -1.24176347e-09f});            // 1/4!
    hc = ff_horner(hc, z, ff2{-0.5f, 0.f});
    hc = ff_horner(hc, z, ff2{1.0f, 0.f});
    const int q = (int)k & 3;
    const ff2 a = (q & 1) ? hc : sn, b = (q & 1) ? sn : hc;
    *s = (q & 2) ? ff2{-a.hi, -a.lo} : a;
    *c = ((q + 1) & 2) ? ff2{-b.hi, -b.lo} : b;
}
