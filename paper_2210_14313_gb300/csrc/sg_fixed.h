// Double-precision sin, cos and expm1 of the FP64 fold, evaluated in 64-bit
// fixed-point integer arithmetic.
//
// GB300 issues FP64 at 1/72 of the FP32 rate (measured), while a 32 x 32 -> 64-bit
// integer multiply-add runs on the integer pipes at a much higher rate, so
// the polynomial parts of the per-point deviation (Section 3's G evaluation)
// are evaluated on integers: every intermediate is an unsigned magnitude
// with a fixed binary point, and only the conversion of the argument, the
// point's sum and weight, and the final scaling by the argument stay in
// FP64.  The polynomials are the minimax fits of gen_poly.py (Remez
// exchange), their coefficients rounded to 0.64 fixed point.  Each product
// drops the low words (at most 2 units of 2^-64 too small), so the fixed-point
// results carry absolute errors of a few units of 2^-63, far below the
// rounding of a double; the results are within about 1 ulp of the functions.
//
// Formats: "m.n" is an unsigned 64-bit integer v standing for v 2^-n.
// Host and device share the code (the host build is the test harness).
#pragma once

#if defined(__CUDACC__)
#define SG_FX __host__ __device__ __forceinline__
#else
#include <math.h>
#include <string.h>
#define SG_FX static inline
#endif

typedef unsigned long long sg_u64;

SG_FX sg_u64 sg_fx_bits(double x) {
#if defined(__CUDA_ARCH__)
    return (sg_u64)__double_as_longlong(x);
#else
    sg_u64 b;
    memcpy(&b, &x, sizeof(b));
    return b;
#endif
}

SG_FX double sg_fx_from_bits(sg_u64 b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof(x));
    return x;
#endif
}

// number of leading zero bits (64 for 0)
SG_FX int sg_fx_clz(sg_u64 v) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// floor(a b / 2^64) less 0, 1 or 2: the product of the low words and the low
// halves of the two cross products are left out
SG_FX sg_u64 sg_fx_mulhi(sg_u64 a, sg_u64 b) {
    const unsigned a1 = (unsigned)(a >> 32), a0 = (unsigned)a;
    const unsigned b1 = (unsigned)(b >> 32), b0 = (unsigned)b;
#if defined(__CUDA_ARCH__)
    return (sg_u64)a1 * b1 + __umulhi(a1, b0) + __umulhi(a0, b1);
#else
    return (sg_u64)a1 * b1 + (((sg_u64)a1 * b0) >> 32) + (((sg_u64)a0 * b1) >> 32);
#endif
}

// |x| 2^q truncated to an integer, for |x| 2^q < 2^64 (q <= 64)
SG_FX sg_u64 sg_fx_fix(double x, int q) {
    const sg_u64 b = sg_fx_bits(x) & 0x7fffffffffffffffull;
    const int e = (int)(b >> 52);
    const sg_u64 m = (b & 0xfffffffffffffull) | ((sg_u64)(e != 0) << 52);
    const int s = (e != 0 ? e : 1) - 1075 + q;  // |x| 2^q = m 2^s
    return s >= 0 ? m << s : (s > -64 ? m >> -s : 0ull);
}

// (-1)^neg v 2^-q as a double, rounded to nearest (ties away from zero); the
// result must be a normal number or zero (v = 0)
SG_FX double sg_fx_to_double(sg_u64 v, sg_u64 neg, int q) {
    const int n = sg_fx_clz(v) & 63;
    const sg_u64 m = v << n;                             // leading one at bit 63
    const sg_u64 sig = (m >> 11) + ((m >> 10) & 1ull);   // 53 bits, may round up to 2^53
    const sg_u64 b = ((sg_u64)(1085 - n - q) << 52) + sig;
    return sg_fx_from_bits((v ? b : 0ull) | (neg << 63));
}

// as sg_fx_to_double, for any q: results below the normal range are flushed
// to zero
SG_FX double sg_fx_to_double_f(sg_u64 v, sg_u64 neg, int q) {
    const int n = sg_fx_clz(v) & 63;
    const sg_u64 m = v << n;
    const sg_u64 sig = (m >> 11) + ((m >> 10) & 1ull);
    const int ef = 1085 - n - q;  // biased exponent less one
    const sg_u64 b = ((sg_u64)ef << 52) + sig;
    return sg_fx_from_bits((v != 0 && ef >= 0 ? b : 0ull) | (neg << 63));
}

// A double as |x| = m 2^(e - 1086) with m its significand shifted to bit 63
// (the leading one at bit 63 for normal numbers) and e its biased exponent
// (1 for subnormals); neg is its sign bit.
struct SgFxNorm {
    sg_u64 m, neg;
    int e;
};

SG_FX SgFxNorm sg_fx_norm(double x) {
    const sg_u64 b = sg_fx_bits(x);
    const int e = (int)((b >> 52) & 0x7ff);
    SgFxNorm r;
    r.m = ((b & 0xfffffffffffffull) | ((sg_u64)(e != 0) << 52)) << 11;
    r.e = e != 0 ? e : 1;
    r.neg = b >> 63;
    return r;
}

// sin r = r + r^3 S(r^2), S = sum s_k z^k, signs -, +, -, +, -, +
#define SG_FX_SIN0 3074457345618251973ull
#define SG_FX_SIN1 153722867280706050ull
#define SG_FX_SIN2 3660068266438490ull
#define SG_FX_SIN3 50834271173124ull
#define SG_FX_SIN4 462104732607ull
#define SG_FX_SIN5 2932336757ull
// cos r = 1 - r^2/2 + r^4 C(r^2), C = sum c_k z^k, signs +, -, +, -, +, -
#define SG_FX_COS0 768614336404563290ull
#define SG_FX_COS1 25620477880122949ull
#define SG_FX_COS2 457508533339211ull
#define SG_FX_COS3 5083427220231ull
#define SG_FX_COS4 38508871062ull
#define SG_FX_COS5 209528007ull
// expm1 x = x + x^2 P(x), P = sum p_k x^k, all positive
#define SG_FX_EXP0 9223372036854775824ull
#define SG_FX_EXP1 3074457345618260416ull
#define SG_FX_EXP2 768614336404561741ull
#define SG_FX_EXP3 153722867280698342ull
#define SG_FX_EXP4 25620477880287604ull
#define SG_FX_EXP5 3660068276833369ull
#define SG_FX_EXP6 457508531194926ull
#define SG_FX_EXP7 50834143488035ull
#define SG_FX_EXP8 5083443533633ull
#define SG_FX_EXP9 463178704675ull
#define SG_FX_EXP10 38508184979ull

// For a = |r| in 0.64, |r| <= 0.7854: the correction w = -z S(z) of
// sin r = r (1 - w) in 0.64 and cos r in 1.63.  With alternating signs every
// Horner partial sum has the sign of its leading coefficient, so the
// magnitudes obey |P_k| = |s_k| - z |P_{k+1}| (>= 0).
SG_FX void sg_fx_sincos_k(sg_u64 a, sg_u64 *w, sg_u64 *kc) {
    const sg_u64 z = sg_fx_mulhi(a, a);  // r^2, 0.64
    sg_u64 p = SG_FX_SIN5;
    p = SG_FX_SIN4 - sg_fx_mulhi(z, p);
    p = SG_FX_SIN3 - sg_fx_mulhi(z, p);
    p = SG_FX_SIN2 - sg_fx_mulhi(z, p);
    p = SG_FX_SIN1 - sg_fx_mulhi(z, p);
    p = SG_FX_SIN0 - sg_fx_mulhi(z, p);                 // -S(z)
    *w = sg_fx_mulhi(z, p);                             // -z S(z)
    sg_u64 c = SG_FX_COS5;
    c = SG_FX_COS4 - sg_fx_mulhi(z, c);
    c = SG_FX_COS3 - sg_fx_mulhi(z, c);
    c = SG_FX_COS2 - sg_fx_mulhi(z, c);
    c = SG_FX_COS1 - sg_fx_mulhi(z, c);
    c = SG_FX_COS0 - sg_fx_mulhi(z, c);                 // C(z)
    const sg_u64 h = (1ull << 63) - sg_fx_mulhi(z, c);  // 1/2 - z C(z), 0.64
    *kc = (1ull << 63) - (sg_fx_mulhi(z, h) >> 1);      // 1 - z (1/2 - z C(z))
}

// sin r and cos r for |r| <= 0.7854: sin r = r - r w, one rounding after
// the fixed-point part
SG_FX void sg_fx_sincos(double r, double *s, double *c) {
    sg_u64 w, kc;
    sg_fx_sincos_k(sg_fx_fix(r, 64), &w, &kc);
    *s = fma(-r, sg_fx_to_double(w, 0ull, 64), r);
    *c = sg_fx_to_double(kc, 0ull, 63);
}

// sin(phi) and cos(phi) of an item: magnitudes in 1.63 and sign masks
// (all ones when negative)
struct SgFxPhase {
    sg_u64 ms, mc, ns, nc;
};

SG_FX SgFxPhase sg_fx_phase(double s, double c) {
    SgFxPhase p;
    p.ms = sg_fx_fix(s, 63);
    p.mc = sg_fx_fix(c, 63);
    p.ns = (sg_u64)((long long)sg_fx_bits(s) >> 63);
    p.nc = (sg_u64)((long long)sg_fx_bits(c) >> 63);
    return p;
}

// For a = |H| in 0.64, |H| <= 0.7854, and H's sign mask nh: the magnitude of
// B = (sin H / H) (sin phi cos H + cos phi sin H) in 3.61, and its sign mask
SG_FX sg_u64 sg_fx_osc_b(sg_u64 a, sg_u64 nh, const SgFxPhase &ph, sg_u64 *nb) {
    sg_u64 w, kc;
    sg_fx_sincos_k(a, &w, &kc);
    const sg_u64 ks = (1ull << 63) - (w >> 1);                  // sin H / H, 1.63
    const sg_u64 t1 = sg_fx_mulhi(ph.ms, kc);                   // |sin phi| cos H, 2.62
    const sg_u64 t2 = sg_fx_mulhi(ph.mc, sg_fx_mulhi(a, ks));   // |cos phi| |sin H|, 2.62
    const sg_u64 n2 = ph.nc ^ nh;
    const sg_u64 u = ((t1 ^ ph.ns) - ph.ns) + ((t2 ^ n2) - n2);  // sin(phi + H), signed 2.62
    *nb = (sg_u64)((long long)u >> 63);
    return sg_fx_mulhi((u ^ *nb) - *nb, ks);
}

// sin(H) sin(phi + H) for |H| <= 0.7854, as H B.  The absolute error is a few
// units of |H| 2^-61: within 2 ulp of the result unless |sin(phi + H)| is
// small, where it stays far below the rounding error of the same expression
// evaluated in FP64.
SG_FX double sg_fx_osc_dev(double H, const SgFxPhase &ph) {
    sg_u64 nb;
    const sg_u64 b = sg_fx_osc_b(sg_fx_fix(H, 64), (sg_u64)((long long)sg_fx_bits(H) >> 63), ph, &nb);
    return H * sg_fx_to_double(b, nb & 1ull, 61);
}

// w sin(H) sin(phi + H) for |H| <= 0.7854: the product H B w formed from B
// and the normalised significands of H and w, rounded once; g is w as a
// normalised 64-bit significand (sg_fx_norm of a double, or a weight kept to
// 64 bits)
SG_FX double sg_fx_osc_dev_wn(double H, const SgFxNorm &g, const SgFxPhase &ph) {
    const SgFxNorm h = sg_fx_norm(H);
    sg_u64 nb;
    const sg_u64 b = sg_fx_osc_b(sg_fx_fix(H, 64), 0ull - h.neg, ph, &nb);
    const sg_u64 v = sg_fx_mulhi(sg_fx_mulhi(b, h.m), g.m);  // |H B w| 2^(2105 - eH - ew)
    return sg_fx_to_double_f(v, (nb ^ h.neg ^ g.neg) & 1ull, 2105 - h.e - g.e);
}

SG_FX double sg_fx_osc_dev_w(double H, double w, const SgFxPhase &ph) {
    return sg_fx_osc_dev_wn(H, sg_fx_norm(w), ph);
}

// P(x) of expm1(x) = x + x^2 P(x) in 0.64, for a = |x| in 0.64, |x| <= ln2/2
// (about 0.3466), and x's sign mask n.  All coefficients are positive, so
// the Horner sums P_k = p_k +- |x| P_{k+1} stay positive.
SG_FX sg_u64 sg_fx_expm1_p(sg_u64 a, sg_u64 n) {
    sg_u64 p = SG_FX_EXP10;
    p = SG_FX_EXP9 + ((sg_fx_mulhi(a, p) ^ n) - n);
    p = SG_FX_EXP8 + ((sg_fx_mulhi(a, p) ^ n) - n);
    p = SG_FX_EXP7 + ((sg_fx_mulhi(a, p) ^ n) - n);
    p = SG_FX_EXP6 + ((sg_fx_mulhi(a, p) ^ n) - n);
    p = SG_FX_EXP5 + ((sg_fx_mulhi(a, p) ^ n) - n);
    p = SG_FX_EXP4 + ((sg_fx_mulhi(a, p) ^ n) - n);
    p = SG_FX_EXP3 + ((sg_fx_mulhi(a, p) ^ n) - n);
    p = SG_FX_EXP2 + ((sg_fx_mulhi(a, p) ^ n) - n);
    p = SG_FX_EXP1 + ((sg_fx_mulhi(a, p) ^ n) - n);
    return SG_FX_EXP0 + ((sg_fx_mulhi(a, p) ^ n) - n);
}

// expm1(x) for |x| <= ln2/2 as x + x (x P(x)), one rounding after the
// fixed-point part
SG_FX double sg_fx_expm1(double x) {
    const sg_u64 a = sg_fx_fix(x, 64);
    const sg_u64 n = (sg_u64)((long long)sg_fx_bits(x) >> 63);
    return fma(x, sg_fx_to_double(sg_fx_mulhi(a, sg_fx_expm1_p(a, n)), n & 1ull, 64), x);
}

// w expm1(x) for |x| <= ln2/2: the product x (1 + x P(x)) w formed from the
// normalised significands of x and w, rounded once (g: w as a normalised
// 64-bit significand)
SG_FX double sg_fx_expm1_wn(double x, const SgFxNorm &g) {
    const SgFxNorm h = sg_fx_norm(x);
    const sg_u64 a = sg_fx_fix(x, 64), n = 0ull - h.neg;
    const sg_u64 t = sg_fx_mulhi(a, sg_fx_expm1_p(a, n)) >> 2;  // |x| P(x), 2.62
    const sg_u64 k = (1ull << 62) + ((t ^ n) - n);               // 1 + x P(x), 2.62
    const sg_u64 v = sg_fx_mulhi(sg_fx_mulhi(k, h.m), g.m);       // |x k w| 2^(2106 - ex - ew)
    return sg_fx_to_double_f(v, (h.neg ^ g.neg) & 1ull, 2106 - h.e - g.e);
}

SG_FX double sg_fx_expm1_w(double x, double w) { return sg_fx_expm1_wn(x, sg_fx_norm(w)); }

// A weight kept to 64 bits (SgFxNorm) split into two doubles hi + lo: hi its
// leading 53 bits, lo the remaining 11 (both exact; 0 below the normal range)
SG_FX void sg_fx_norm_split(const SgFxNorm &g, double *hi, double *lo) {
    const sg_u64 s = g.neg << 63;
    *hi = g.e >= 1 ? sg_fx_from_bits(s | ((sg_u64)g.e << 52) | ((g.m >> 11) & 0xfffffffffffffull)) : 0.0;
    const int el = g.e - 63;  // biased exponent of 2^(e - 1086), the unit of m's last bit
    const sg_u64 low = g.m & 0x7ffull;
    *lo = (low && el >= 1) ? sg_fx_from_bits(s | ((sg_u64)el << 52)) * (double)low : 0.0;
}
