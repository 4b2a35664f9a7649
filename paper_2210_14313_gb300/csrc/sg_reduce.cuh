// Deterministic reduction of the fold's chunk slots on the device: exact
// sums in a 128-bit integer window (sg_xsum.h) across the lanes of a warp,
// the two-level ticketing of complete_chunk and the assembly of an item's
// output record.  Shared by
// the built-in fold kernels and the fold kernel compiled at run time for a
// user integrand (so it compiles under nvcc and NVRTC alike).
#pragma once
#include "sg_internal.h"
#include "sg_xsum.h"

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
// as Q = mant * 2^exp2; adjoint sub-sums write their relative value.  The
// item's values V, the integral's base B (g < 0: an adjoint sub-sum) and
// its output index come from the caller, which can load them early.
__device__ inline void assemble_values(const SgItemVar &V, const SgBaseDev &B, int g, long long out_idx,
                                       SgOutDev *out, double *vout, int *flags, double guard_tol,
                                       double unit_roundoff, int item, double T, double AB) {
    const double rel = V.mult * (V.base_rel + T);
    const double absrel = fabs(V.mult) * (fabs(V.base_rel) + AB);
    if (g < 0) {
        vout[out_idx] = rel;
        return;
    }
    // Q = exp(log_hi + log_lo) * rel = 2^e0 * scale_m * rel
    const double e0 = B.scale_e2;
    int e1 = 0;
    const double mant = frexp(B.scale_m * rel, &e1);
    SgOutDev o;
    o.mant = mant;
    o.exp2 = e0 + e1;
    o.value = ldexp(mant, (int)(e0 + e1));
    o.cond = sg_ratio(absrel, fabs(rel));  // three digits suffice for the error estimate
    o.err_est = 0.05 * unit_roundoff * o.cond;
    o.sum = rel;
    o.abs_sum = absrel;
    out[out_idx] = o;
    if (flags && guard_tol > 0.0) flags[item] = o.err_est > guard_tol ? 1 : 0;
}

__device__ inline void assemble_item(const SgItemDev *items, const SgItemVar *vars, const SgBaseDev *bases,
                              const int *item_integral, SgOutDev *out, double *vout, int *flags,
                              double guard_tol, double unit_roundoff, int item, double T, double AB) {
    const int g = item_integral[item];
    const SgBaseDev B = g >= 0 ? bases[g] : SgBaseDev{};
    assemble_values(vars[item], B, g, items[item].out, out, vout, flags, guard_tol, unit_roundoff, item, T, AB);
}

// Warp-wide exact sums (sg_xsum.h): the largest exponent among the lanes'
// terms fixes the unit; the lanes' 128-bit partial sums are added by an xor
// butterfly of integer additions, which gives every lane the same total in
// any order; the total is rounded once to a pair (s, c).
__device__ __forceinline__ int warp_max_exp(int e) { return (int)__reduce_max_sync(SG_FULL_MASK, (unsigned)e); }

__device__ __forceinline__ void warp_xadd(SgX &a) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        SgX b;
        b.lo = __shfl_xor_sync(SG_FULL_MASK, a.lo, o);
        b.hi = __shfl_xor_sync(SG_FULL_MASK, a.hi, o);
        sg_x_plus(a, b);
    }
}

__device__ __forceinline__ void warp_xsum(SgX a, int E, double &s, double &c) {
    warp_xadd(a);
    sg_x_pair(a, E, &s, &c);
}

// The exact sum of one double per lane, rounded to the nearest double.
__device__ __forceinline__ double warp_sum(double v) {
    const int E = warp_max_exp(sg_x_exp(v));
    SgX a = {0ull, 0ull};
    sg_x_add(a, v, E);
    double s, c;
    warp_xsum(a, E, s, c);
    return s;
}

// Sum of a group's chunk slots (sum + lo, abs): at most SG_GROUP = 64
// slots, two per lane, held in registers while the largest exponents are
// found.
__device__ inline void reduce_slots(const SgSlot *slots, unsigned long long n, int lane, double &S,
                             double &C, double &AB) {
    static_assert(SG_GROUP <= 64, "two slots per lane");
    const double2 z = make_double2(0.0, 0.0);
    const double2 v0 = (unsigned long long)lane < n ? __ldcg((const double2 *)(slots + lane)) : z;
    const double2 v1 = (unsigned long long)lane + 32 < n ? __ldcg((const double2 *)(slots + lane + 32)) : z;
    const double l0 = (unsigned long long)lane < n ? __ldcg(&slots[lane].lo) : 0.0;
    const double l1 = (unsigned long long)lane + 32 < n ? __ldcg(&slots[lane + 32].lo) : 0.0;
    const int Es = warp_max_exp(max(max(sg_x_exp(v0.x), sg_x_exp(v1.x)), max(sg_x_exp(l0), sg_x_exp(l1))));
    const int Ea = warp_max_exp(max(sg_x_exp(v0.y), sg_x_exp(v1.y)));
    SgX as = {0ull, 0ull}, aa = {0ull, 0ull};
    sg_x_add(as, v0.x, Es);
    sg_x_add(as, v1.x, Es);
    sg_x_add(as, l0, Es);
    sg_x_add(as, l1, Es);
    sg_x_add(aa, v0.y, Ea);
    sg_x_add(aa, v1.y, Ea);
    double ac;
    warp_xsum(as, Es, S, C);
    warp_xsum(aa, Ea, AB, ac);
}

// Ticket increment with acquire-release semantics at GPU scope: the calling
// thread's earlier writes become visible to whichever thread later reads the
// incremented count, and the caller sees the writes released by the earlier
// increments.
__device__ __forceinline__ unsigned ticket_add(unsigned *p) {
    unsigned v;
    asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(v) : "l"(p) : "memory");
    return v;
}

// Same over group records: s and c of every group in one sum, abs in another.
__device__ inline void reduce_groups(const SgGroupSlot *g, unsigned long long n, int lane, double &S,
                              double &C, double &AB) {
    int Es = 1, Ea = 1;
    for (unsigned long long q = lane; q < n; q += 32) {
        const double2 v = __ldcg((const double2 *)(g + q));
        const double a = __ldcg(&g[q].abs);
        Es = max(Es, max(sg_x_exp(v.x), sg_x_exp(v.y)));
        Ea = max(Ea, sg_x_exp(a));
    }
    Es = warp_max_exp(Es);
    Ea = warp_max_exp(Ea);
    SgX as = {0ull, 0ull}, aa = {0ull, 0ull};
    for (unsigned long long q = lane; q < n; q += 32) {
        const double2 v = __ldcg((const double2 *)(g + q));
        sg_x_add(as, v.x, Es);
        sg_x_add(as, v.y, Es);
        sg_x_add(aa, __ldcg(&g[q].abs), Ea);
    }
    double ac;
    warp_xsum(as, Es, S, C);
    warp_xsum(aa, Ea, AB, ac);
}

// Called by the warp that wrote chunk c's slot.  Two-level ticketing: the
// last chunk of a group reduces the group, the last group reduces the item
// and calls finish(T, AB) on lane 0 with the item's sum T (the double pair
// of the exact sum, added) and its sum of absolute values AB.
template <typename Finish>
__device__ inline void complete_chunk(const SgFoldArgs &A, int item, unsigned long long c, int lane,
                                      Finish finish) {
    const SgItemDev *I = A.items + item;
    const unsigned long long local = c - I->chunk0;
    const unsigned long long g = local / SG_GROUP;
    const unsigned long long gfirst = g * SG_GROUP;
    const unsigned long long gsize =
        I->nchunk - gfirst < (unsigned long long)SG_GROUP ? I->nchunk - gfirst : SG_GROUP;
    // lane 0 wrote the chunk's slot; its ticket releases it, and the last
    // ticket of the group acquires all of the group's slots (the warp barrier
    // passes the ordering on to the other lanes)
    unsigned int ticket = 0;
    if (lane == 0) ticket = ticket_add(A.group_done + I->group0 + g);
    ticket = __shfl_sync(SG_FULL_MASK, ticket, 0);
    if (ticket + 1ull != gsize) return;
    __syncwarp();
    double S, C, AB;
    reduce_slots(A.slots + I->chunk0 + gfirst, gsize, lane, S, C, AB);
    if (lane == 0) {
        SgGroupSlot gs;
        gs.s = S;
        gs.c = C;
        gs.abs = AB;
        gs.pad = 0.0;
        A.gslots[I->group0 + g] = gs;
        ticket = ticket_add(A.item_done + item);
    }
    ticket = __shfl_sync(SG_FULL_MASK, ticket, 0);
    if (ticket + 1ull != I->ngroups) return;
    __syncwarp();
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

