// Exact summation of doubles in a 128-bit integer window, for the fold's
// deterministic reduction of chunk, group and item sums.
//
// The terms of one sum are scaled to a common unit 2^(E - 1075 - SG_XG), E
// the largest biased exponent among them: a term with exponent e becomes its
// 53-bit significand shifted by e - E + SG_XG (<= SG_XG) bits, truncated
// towards zero below the unit (at most 2^-(SG_XG + 52) of the largest term,
// the same for every order of summation).  Up to 2^22 terms then add
// exactly as two's complement 128-bit integers, so the sum does not depend
// on the order of the additions at all, and it is rounded to a double pair
// (s, c) only once at the end (s the nearest double to the sum, c the
// nearest double to the rest).  On GB300 a dependent FP64 addition costs on
// the order of 10^2 cycles; the integer additions cost a few.
#pragma once

#if defined(__CUDACC__) || defined(__CUDACC_RTC__)
#define SG_XS __host__ __device__ __forceinline__
#else
#include <math.h>
#include <string.h>
#define SG_XS static inline
#endif

#define SG_XG 52  // guard bits below the largest term's unit in the last place

struct SgX {
    unsigned long long lo, hi;  // two's complement, value = hi 2^64 + lo
};

SG_XS unsigned long long sg_xs_bits(double x) {
#if defined(__CUDA_ARCH__)
    return (unsigned long long)__double_as_longlong(x);
#else
    unsigned long long b;
    memcpy(&b, &x, sizeof(b));
    return b;
#endif
}

SG_XS double sg_xs_double(unsigned long long b) {
#if defined(__CUDA_ARCH__)
    return __longlong_as_double((long long)b);
#else
    double x;
    memcpy(&x, &b, sizeof(x));
    return x;
#endif
}

SG_XS int sg_xs_clz(unsigned long long v) {
#if defined(__CUDA_ARCH__)
    return __clzll((long long)v);
#else
    return v ? __builtin_clzll(v) : 64;
#endif
}

// a / b (a, b >= 0) to float precision without an FP64 division (on GB300
// a chain of dependent FP64 steps): the quotient of the significands in
// float, the exponents subtracted as integers.  Zeros, subnormals,
// infinities and NaNs take the double division.  The kernels' output
// records and the host's combine of sharded batches both form the
// condition number with it, so that the two agree bit for bit.
SG_XS double sg_ratio(double a, double b) {
    const unsigned long long ba = sg_xs_bits(a), bb = sg_xs_bits(b);
    const int ea = (int)((ba >> 52) & 0x7ff), eb = (int)((bb >> 52) & 0x7ff);
    if (ea == 0 || eb == 0 || ea == 0x7ff || eb == 0x7ff) return a / b;
    const unsigned int fa = 0x3f800000u | (unsigned int)((ba >> 29) & 0x7fffff);
    const unsigned int fb = 0x3f800000u | (unsigned int)((bb >> 29) & 0x7fffff);
#if defined(__CUDA_ARCH__)
    const float q = __fdiv_rn(__uint_as_float(fa), __uint_as_float(fb));
#else
    float ma, mb;
    memcpy(&ma, &fa, sizeof(ma));
    memcpy(&mb, &fb, sizeof(mb));
    const float q = ma / mb;
#endif
    return ldexp((double)q, ea - eb);
}

// biased exponent of |v| (1 for zero and subnormals)
SG_XS int sg_x_exp(double v) {
    const int e = (int)((sg_xs_bits(v) >> 52) & 0x7ff);
    return e ? e : 1;
}

// a += v in the unit of the largest exponent E (E >= the exponent of v)
SG_XS void sg_x_add(SgX &a, double v, int E) {
    const unsigned long long b = sg_xs_bits(v);
    const int e = (int)((b >> 52) & 0x7ff);
    const unsigned long long m = (b & 0xfffffffffffffull) | ((unsigned long long)(e != 0) << 52);
    const int s = (e ? e : 1) - E + SG_XG;  // |v| = m 2^s units
    unsigned long long lo, hi;
    if (s >= 64) {  // not reached for s <= SG_XG < 64; kept for completeness
        lo = 0;
        hi = m << (s - 64);
    } else if (s > 0) {
        lo = m << s;
        hi = m >> (64 - s);
    } else if (s > -64) {
        lo = m >> -s;
        hi = 0;
    } else {
        lo = 0;
        hi = 0;
    }
    if (b >> 63) {  // negate
        lo = ~lo + 1;
        hi = ~hi + (lo == 0);
    }
    a.lo += lo;
    a.hi += hi + (a.lo < lo);
}

// a >>= k, arithmetic (towards minus infinity), k >= 0: moves a sum to a
// coarser unit
SG_XS void sg_x_shr(SgX &a, int k) {
    if (k <= 0) return;
    const unsigned long long sgn = (unsigned long long)((long long)a.hi >> 63);
    if (k >= 128) {
        a.lo = sgn;
        a.hi = sgn;
    } else if (k >= 64) {
        a.lo = (unsigned long long)((long long)a.hi >> (k - 64));
        a.hi = sgn;
    } else {
        a.lo = (a.lo >> k) | (a.hi << (64 - k));
        a.hi = (unsigned long long)((long long)a.hi >> k);
    }
}

// A running sum whose unit follows the largest exponent seen so far: a new
// larger term first moves the sum to the coarser unit.  The result depends
// only on the order of the terms (fixed by the caller), not on timing.
SG_XS void sg_x_add_adaptive(SgX &a, int &E, double v) {
    const int e = sg_x_exp(v);
    if (e > E) {
        sg_x_shr(a, e - E);
        E = e;
    }
    sg_x_add(a, v, E);
}

SG_XS void sg_x_plus(SgX &a, const SgX &b) {
    a.lo += b.lo;
    a.hi += b.hi + (a.lo < b.lo);
}

// magnitude mag (128 bits) times 2^x as the nearest double (ties away from
// zero); 0 below the normal range
SG_XS double sg_x_mag_double(unsigned long long lo, unsigned long long hi, int x) {
    if (!(lo | hi)) return 0.0;
    const int p = hi ? 127 - sg_xs_clz(hi) : 63 - sg_xs_clz(lo);  // top bit
    unsigned long long sig;
    if (p <= 52) {
        sig = lo << (52 - p);
    } else {
        const int sh = p - 52;  // 1 .. 75
        unsigned long long t, rb;
        if (sh < 64) {
            t = (lo >> sh) | (sh ? hi << (64 - sh) : 0);
            rb = (lo >> (sh - 1)) & 1ull;
        } else {
            t = hi >> (sh - 64);
            rb = sh == 64 ? lo >> 63 : (hi >> (sh - 65)) & 1ull;
        }
        sig = t + rb;
    }
    const int ef = p + x + 1022;  // biased exponent less one
    if (ef < 0) return 0.0;
    return sg_xs_double(((unsigned long long)ef << 52) + sig);
}

// the sum a (unit 2^(E - 1075 - SG_XG)) as s + c: s the nearest double, c the
// nearest double to a - s
SG_XS void sg_x_pair(SgX a, int E, double *s, double *c) {
    const unsigned long long neg = a.hi >> 63;
    if (neg) {
        a.lo = ~a.lo + 1;
        a.hi = ~a.hi + (a.lo == 0);
    }
    const int x = E - 1075 - SG_XG;
    const double hs = sg_x_mag_double(a.lo, a.hi, x);
    // the rest a - |s|, exactly, in the same unit
    double hc = 0.0;
    if (hs != 0.0) {
        const unsigned long long b = sg_xs_bits(hs);
        const int e = (int)(b >> 52);
        const unsigned long long m = (b & 0xfffffffffffffull) | (1ull << 52);
        const int sh = e - 1075 - x;  // |s| = m 2^sh units, sh >= 0 when |s| > 2^53 units
        if (sh > 0) {
            unsigned long long slo, shi;
            if (sh >= 64) {
                slo = 0;
                shi = m << (sh - 64);
            } else {
                slo = m << sh;
                shi = m >> (64 - sh);
            }
            // r = a - s (signed)
            unsigned long long rlo = a.lo - slo;
            unsigned long long rhi = a.hi - shi - (a.lo < slo);
            const unsigned long long rneg = rhi >> 63;
            if (rneg) {
                rlo = ~rlo + 1;
                rhi = ~rhi + (rlo == 0);
            }
            hc = sg_x_mag_double(rlo, rhi, x);
            if (rneg) hc = -hc;
        }
    }
    *s = neg ? -hs : hs;
    *c = neg ? -hc : hc;
}
