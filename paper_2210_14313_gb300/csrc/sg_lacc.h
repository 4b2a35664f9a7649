// A long fixed-point accumulator for order-independent sums of doubles: the
// single-integral fold adds every chunk's sum into one per CTA, and the last
// CTA adds the CTAs' accumulators, all as integers.
//
// A value is sum_k D_k 2^(32k + SG_LA_E0), k = 0 .. SG_LA_DIGITS-1, held as
// SG_LA_DIGITS signed 64-bit limbs that each collect 32-bit digits: a double
// enters as its significand cut into 32-bit digits at fixed positions (at
// most three digits are non-zero), and each digit is added into its limb
// with one integer addition.  No carry moves between limbs while adding, so
// the limbs can be updated by independent atomic additions, and up to 2^31
// terms fit before a limb could overflow.  Integer addition is associative,
// so the sum is the same for every order and every split of the terms over
// threads, CTAs or launches; it is rounded once at the end.  The window
// covers 2^SG_LA_E0 = 2^-576 to 2^448: bits of a term below 2^-576 are cut
// off (towards zero, the same in every order), terms of magnitude 2^447 or
// more, infinities and NaNs set the overflow flag instead.
//
// This is the classical "long accumulator" of exact dot products
// (U. Kulisch, "Computer Arithmetic and Validity", de Gruyter 2008) with
// the carry-save digit layout that lets the parts update independently.
#pragma once

#include "sg_xsum.h"

#define SG_LA_DIGITS 32
#define SG_LA_E0 (-576)

// Digit k of v (signed: the digit of |v| with the sign of v); sets *ovf for
// terms outside the window.
SG_XS long long sg_la_digit(double v, int k, int *ovf) {
    const unsigned long long b = sg_xs_bits(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0x7ff) {
        *ovf = 1;
        return 0;
    }
    const unsigned long long m = (b & 0xfffffffffffffull) | ((unsigned long long)(e != 0) << 52);
    if (!m) return 0;
    // |v| = m 2^(s + SG_LA_E0)
    const int s = (e ? e : 1) - 1075 - SG_LA_E0;
    if (s + 53 > 32 * SG_LA_DIGITS - 1) {
        *ovf = 1;
        return 0;
    }
    const int lo = 32 * k - s;  // digit k holds bits lo .. lo + 31 of m
    unsigned long long dg;
    if (lo >= 53 || lo <= -32) dg = 0;
    else if (lo >= 0) dg = (m >> lo) & 0xffffffffull;
    else dg = (m << -lo) & 0xffffffffull;
    return (b >> 63) ? -(long long)dg : (long long)dg;
}

// Digit k of an exact 128-bit sum t whose unit is 2^(E - 1075 - SG_XG)
// (sg_xsum.h): the 32 bits of |t| that fall in limb k, with the sign of t
// (bits below the window are cut off towards zero, as sg_la_digit does for a
// double); *mag gets the digit of |t|.  Sets *ovf when |t| reaches 2^447 or
// when E marks an infinite or NaN term (E = 0x7ff).  A chunk's sum enters
// the accumulator this way without being rounded to doubles first.
SG_XS long long sg_la_x_digit(SgX t, int E, int k, int *ovf, long long *mag) {
    const unsigned long long neg = t.hi >> 63;
    if (neg) {
        t.lo = ~t.lo + 1;
        t.hi = ~t.hi + (t.lo == 0);
    }
    // bit i of |t| has weight 2^(u + i + SG_LA_E0) (u relative to the window)
    const int u = E - 1075 - SG_XG - SG_LA_E0;
    if (E >= 0x7ff) {
        *ovf = 1;
    } else if (t.hi | t.lo) {
        const int p = t.hi ? 127 - sg_xs_clz(t.hi) : 63 - sg_xs_clz(t.lo);  // top bit
        if (u + p > 32 * SG_LA_DIGITS - 2) *ovf = 1;
    }
    const int o = 32 * k - u;  // digit k holds bits o .. o + 31 of |t|
    unsigned long long dg;
    if (o >= 128 || o <= -32) dg = 0;
    else if (o >= 64) dg = t.hi >> (o - 64);
    else if (o > 0) dg = (t.lo >> o) | (t.hi << (64 - o));
    else if (o == 0) dg = t.lo;
    else dg = t.lo << -o;
    dg &= 0xffffffffull;
    *mag = (long long)dg;
    return neg ? -(long long)dg : (long long)dg;
}

// Index of the lowest digit that can be non-zero for v (its non-zero digits
// lie in k0 .. k0 + 2), or -1 when v has no bits inside the window; sets
// *ovf for terms above it, infinities and NaNs.
SG_XS int sg_la_first_digit(double v, int *ovf) {
    const unsigned long long b = sg_xs_bits(v);
    const int e = (int)((b >> 52) & 0x7ff);
    if (e == 0x7ff) {
        *ovf = 1;
        return -1;
    }
    if (!(b & 0x7fffffffffffffffull)) return -1;
    const int s = (e ? e : 1) - 1075 - SG_LA_E0;  // lowest bit of the significand
    if (s + 53 > 32 * SG_LA_DIGITS - 1) {
        *ovf = 1;
        return -1;
    }
    if (s + 53 <= 0) return -1;
    return (s < 0 ? 0 : s) >> 5;
}

// The value of the limbs as s + c (s the double nearest the sum of the top
// 128 bits of its magnitude, c the double nearest the rest of those bits);
// the bits below the top 128 are dropped (at most 2^-96 of |sum|).  The
// limbs are normalised in place on the way (each ends up holding one 32-bit
// digit of the magnitude), so that the kernels can run this on an array in
// shared memory without a register copy of it.
SG_XS void sg_la_round(long long *limb, double *s, double *c) {
    long long carry = 0;
#pragma unroll 1
    for (int k = 0; k < SG_LA_DIGITS; k++) {
        const long long t = limb[k] + carry;
        limb[k] = (long long)((unsigned long long)t & 0xffffffffull);
        carry = t >> 32;  // arithmetic: floor division by 2^32
    }
    const int neg = carry < 0;
    if (neg) {  // two's complement of the digit string
        unsigned long long cy = 1;
#pragma unroll 1
        for (int k = 0; k < SG_LA_DIGITS; k++) {
            const unsigned long long t = ((~(unsigned long long)limb[k]) & 0xffffffffull) + cy;
            limb[k] = (long long)(t & 0xffffffffull);
            cy = t >> 32;
        }
    }
    int h = SG_LA_DIGITS - 1;
    while (h >= 0 && limb[h] == 0) h--;
    if (h < 0) {
        *s = 0.0;
        *c = 0.0;
        return;
    }
    if (h < 3) h = 3;
    SgX a;
    a.hi = ((unsigned long long)limb[h] << 32) | (unsigned long long)limb[h - 1];
    a.lo = ((unsigned long long)limb[h - 2] << 32) | (unsigned long long)limb[h - 3];
    // unit of the window: 2^(32 (h - 3) + SG_LA_E0) = 2^(E - 1075 - SG_XG);
    // a magnitude with the top bit set moves one bit down (sg_x_pair reads
    // the window as two's complement)
    int E = 32 * (h - 3) + SG_LA_E0 + 1075 + SG_XG;
    if (a.hi >> 63) {
        a.lo = (a.lo >> 1) | (a.hi << 63);
        a.hi >>= 1;
        E += 1;
    }
    double hs, hc;
    sg_x_pair(a, E, &hs, &hc);
    *s = neg ? -hs : hs;
    *c = neg ? -hc : hc;
}

// The value of 32 limbs as s + c by the rounding the kernels use when the
// limbs are spread over a warp (one limb per lane): one carry step brings
// every limb below 2^53 (the top limb keeps its carries), so that
// limb_k * 2^(32k + SG_LA_E0) is an exact double; those 32 doubles are added
// exactly in a 128-bit window under the largest of them (terms more than
// 104 bits below it are cut towards zero) and rounded to s + c once.  The
// host combine of sharded batches calls this, so that it rounds exactly as
// the kernels do.
SG_XS void sg_la_round_w(const long long *L, double *s, double *c) {
    double t[SG_LA_DIGITS];
    int E = 1;
    for (int k = 0; k < SG_LA_DIGITS; k++) {
        long long v = k == SG_LA_DIGITS - 1 ? L[k] : (long long)((unsigned long long)L[k] & 0xffffffffull);
        if (k > 0) v += L[k - 1] >> 32;  // arithmetic shift: floor division by 2^32
        // v * 2^(32k + SG_LA_E0), exact: |v| < 2^53 and the power of two is a normal double
        t[k] = (double)v * sg_xs_double((unsigned long long)(32 * k + SG_LA_E0 + 1023) << 52);
        const int e = sg_x_exp(t[k]);
        E = e > E ? e : E;
    }
    SgX a = {0ull, 0ull};
    for (int k = 0; k < SG_LA_DIGITS; k++) sg_x_add(a, t[k], E);
    sg_x_pair(a, E, s, c);
}
