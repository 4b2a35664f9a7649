// Deterministic reduction of the fold's chunk slots on the device: per-lane
// compensated sums, the xor-butterfly lane combine, the two-level ticketing
// of complete_chunk and the assembly of an item's output record.  Shared by
// the built-in fold kernels and the fold kernel compiled at run time for a
// user integrand (so it compiles under nvcc and NVRTC alike).
#pragma once
#include "sg_internal.h"

#define SG_FULL_MASK 0xffffffffu

// Neumaier's compensated addition (Neumaier 1974): (s, c) += v.
__device__ __forceinline__ void neu_add(double &s, double &c, double v) {
    double t = s + v;
    if (fabs(s) >= fabs(v)) c += (s - t) + v;
    else c += (v - t) + s;
    s = t;
}

// Value of a finished item: mult * (base_rel + T), relative to the
// integral's scale exp(log f(c)).  Forward items write their output record
// as Q = mant * 2^exp2; adjoint sub-sums write their relative value.
__device__ inline void assemble_item(const SgItemDev *items, const SgItemVar *vars, const SgBaseDev *bases,
                              const int *item_integral, SgOutDev *out, double *vout, int *flags,
                              double guard_tol, double unit_roundoff, int item, double T, double AB) {
    const SgItemDev *I = items + item;
    const SgItemVar V = vars[item];
    const double rel = V.mult * (V.base_rel + T);
    const double absrel = fabs(V.mult) * (fabs(V.base_rel) + AB);
    const int g = item_integral[item];
    if (g < 0) {
        vout[I->out] = rel;
        return;
    }
    const SgBaseDev B = bases[g];
    // Q = exp(log_hi + log_lo) * rel = 2^e0 * scale_m * rel
    const double e0 = B.scale_e2;
    int e1 = 0;
    const double mant = frexp(B.scale_m * rel, &e1);
    SgOutDev o;
    o.mant = mant;
    o.exp2 = e0 + e1;
    o.value = ldexp(mant, (int)(e0 + e1));
    o.cond = absrel / fabs(rel);
    o.err_est = 0.05 * unit_roundoff * o.cond;
    o.sum = rel;
    o.abs_sum = absrel;
    out[I->out] = o;
    if (flags && guard_tol > 0.0) flags[item] = o.err_est > guard_tol ? 1 : 0;
}

// Combines the lanes' compensated pairs (s, c) and absolute sums with an
// xor butterfly: at level o, lane l merges with lane l ^ o.  TwoSum returns
// the exact rounding error of s_l + s_m, which does not depend on the order
// of its operands, so both partners compute bitwise the same pair and every
// lane ends with the same result; the tree is fixed, so the result does not
// depend on which warp runs it.  Five levels of dependent FP64 work instead
// of a 32-step lane-serial sum.
// (s, c) += (s2, c2) for compensated pairs; symmetric in its two operands.
__device__ __forceinline__ void pair_add(double &s, double &c, double s2, double c2) {
    const double t = __dadd_rn(s, s2);
    const double z = __dsub_rn(t, s);
    const double e = __dadd_rn(__dsub_rn(s, __dsub_rn(t, z)), __dsub_rn(s2, z));
    s = t;
    c = __dadd_rn(__dadd_rn(c, c2), e);
}

__device__ __forceinline__ void lane_combine(double &s, double &c, double &ab) {
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const double s2 = __shfl_xor_sync(SG_FULL_MASK, s, o);
        const double c2 = __shfl_xor_sync(SG_FULL_MASK, c, o);
        const double a2 = __shfl_xor_sync(SG_FULL_MASK, ab, o);
        pair_add(s, c, s2, c2);
        ab = __dadd_rn(ab, a2);
    }
}

// Lane l adds x[l], x[l+32], ... into four compensated accumulators (the
// t-th load of a batch into accumulator t mod 4, four independent chains),
// which are then merged and the lanes combined by lane_combine: a fixed
// summation order whichever warp runs it.  Each lane issues its loads eight
// at a time (missing ones read as zero, which leaves a compensated sum
// unchanged), so that the L2 latency is paid once per batch.
__device__ inline void reduce_slots(const double2 *slots, unsigned long long n, int lane, double &S,
                             double &C, double &AB) {
    double s[4] = {0.0, 0.0, 0.0, 0.0}, c[4] = {0.0, 0.0, 0.0, 0.0}, ab = 0.0;
    for (unsigned long long q0 = lane; q0 < n; q0 += 8 * 32) {
        double2 v[8];
#pragma unroll
        for (int t = 0; t < 8; t++) {
            const unsigned long long q = q0 + t * 32;
            v[t] = q < n ? __ldcg(slots + q) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int t = 0; t < 8; t++) {
            neu_add(s[t & 3], c[t & 3], v[t].x);
            ab += v[t].y;
        }
    }
    pair_add(s[0], c[0], s[1], c[1]);
    pair_add(s[2], c[2], s[3], c[3]);
    pair_add(s[0], c[0], s[2], c[2]);
    lane_combine(s[0], c[0], ab);
    S = s[0];
    C = c[0];
    AB = ab;
}

// Same over group records (s, c, abs).
__device__ inline void reduce_groups(const SgGroupSlot *g, unsigned long long n, int lane, double &S,
                              double &C, double &AB) {
    double s[4] = {0.0, 0.0, 0.0, 0.0}, c[4] = {0.0, 0.0, 0.0, 0.0}, ab = 0.0;
    for (unsigned long long q0 = lane; q0 < n; q0 += 8 * 32) {
        double2 v[8], w[8];
#pragma unroll
        for (int t = 0; t < 8; t++) {
            const unsigned long long q = q0 + t * 32;
            v[t] = q < n ? __ldcg((const double2 *)(g + q)) : make_double2(0.0, 0.0);
            w[t] = q < n ? __ldcg((const double2 *)(g + q) + 1) : make_double2(0.0, 0.0);
        }
#pragma unroll
        for (int t = 0; t < 8; t++) {
            pair_add(s[t & 3], c[t & 3], v[t].x, v[t].y);
            ab += w[t].x;
        }
    }
    pair_add(s[0], c[0], s[1], c[1]);
    pair_add(s[2], c[2], s[3], c[3]);
    pair_add(s[0], c[0], s[2], c[2]);
    lane_combine(s[0], c[0], ab);
    S = s[0];
    C = c[0];
    AB = ab;
}

// Called by the warp that wrote chunk c's slot.  Two-level ticketing: the
// last chunk of a group reduces the group, the last group reduces the item
// and calls finish(T, AB) on lane 0 with the item's compensated sum T and its
// sum of absolute values AB.
template <typename Finish>
__device__ inline void complete_chunk(const SgFoldArgs &A, int item, unsigned long long c, int lane,
                                      Finish finish) {
    const SgItemDev *I = A.items + item;
    const unsigned long long local = c - I->chunk0;
    const unsigned long long g = local / SG_GROUP;
    const unsigned long long gfirst = g * SG_GROUP;
    const unsigned long long gsize =
        I->nchunk - gfirst < (unsigned long long)SG_GROUP ? I->nchunk - gfirst : SG_GROUP;
    unsigned int ticket = 0;
    if (lane == 0) {
        __threadfence();
        ticket = atomicAdd(A.group_done + I->group0 + g, 1u);
    }
    ticket = __shfl_sync(SG_FULL_MASK, ticket, 0);
    if (ticket + 1ull != gsize) return;
    __threadfence();
    double S, C, AB;
    reduce_slots((const double2 *)(A.slots + I->chunk0 + gfirst), gsize, lane, S, C, AB);
    if (lane == 0) {
        SgGroupSlot gs;
        gs.s = S;
        gs.c = C;
        gs.abs = AB;
        gs.pad = 0.0;
        A.gslots[I->group0 + g] = gs;
        __threadfence();
        ticket = atomicAdd(A.item_done + item, 1u);
    }
    ticket = __shfl_sync(SG_FULL_MASK, ticket, 0);
    if (ticket + 1ull != I->ngroups) return;
    __threadfence();
    reduce_groups(A.gslots + I->group0, I->ngroups, lane, S, C, AB);
    if (lane == 0) finish(S + C, AB);
}

// complete_chunk with the built-in assembly of the output record.
__device__ inline void complete_chunk(const SgFoldArgs &A, int item, unsigned long long c, int lane) {
    complete_chunk(A, item, c, lane, [&](double T, double AB) {
        assemble_item(A.items, A.vars, A.bases, A.item_integral, A.out, A.vout, A.flags, A.guard_tol,
                      A.unit_roundoff, item, T, AB);
    });
}

