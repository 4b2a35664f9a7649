// Generated by _build.py: sources that NVRTC compiles for user integrands.
static const char sg_src_internal[] = R"SG_RAW(// Internal data layout shared by the host planner and the CUDA kernels of
// libsg.  Not part of the public ABI (see include/sg.h).
//
// Vocabulary (Section 2.1 and Algorithms 3.1-3.3 of the paper):
//  - excess k = l - 1 of a direction's level l; a direction with k = 0 sits
//    at the centre c = 1/2 with weight 1 ("inactive");
//  - a subgrid is a set of active directions i_1 < ... < i_r with excesses;
//  - its first r-1 active directions form the *prefix*, the last one is the
//    *tail* direction folded by the inner loop;
//  - a *pattern* fixes r and the 1-D rule block of every position (which
//    difference rule / full rule / telescoped tail rule), so all subgrids of
//    a pattern have the same number of points and differ only in which
//    directions are active (an r-subset of {0..d-1});
//  - a *chunk* is a contiguous range of lexicographic ranks of those
//    r-subsets: the unit of work stealing.
#pragma once
#ifndef __CUDACC_RTC__
#include <stdint.h>
#endif

#define SG_MAX_LEVEL 13       // 1-D rule levels 1..13 (4097 nodes, nested rules)
#define SG_MAX_L 12           // largest excess level q - d
#define SG_MAX_R SG_MAX_L     // active directions per subgrid
#define SG_MAX_D 8192         // largest dimension
#define SG_BINOM_K (SG_MAX_R + 2)

// Family of a user integrand compiled at run time (sg_integrand_create): its
// tables hold the node coordinates x instead of phi_i(x).
#define SG_FAM_USER 5

// Integrand deviation kinds evaluated per point (the "G" of the kernels).
#define SG_GK_EXPM1 0  // D = expm1(S)                 (exp-linear, gaussian(s), product peak)
#define SG_GK_OSC 1    // D = cos(phi + S) - cos(phi)   (oscillatory)

// Block kinds of a rule (node/weight lists on [0,1]).
#define SG_BLK_DELTA 0  // J^{k+1} - J^k on the union node set, k >= 1
#define SG_BLK_FULL 1   // J^{k+1}, k >= 1
#define SG_BLK_TAIL 2   // J^{M+1} - J^1, M >= 1 (telescoped last direction)

// One integral (or one adjoint sub-sum) as the kernels see it.
struct SgItemDev {
    int d;            // directions enumerated by the patterns (d or d-1)
    int skip;         // actual direction left out of the enumeration (-1: none)
    int gk;           // SG_GK_*
    int out;          // index of the output record
    long long tab;    // first table entry of the item (entries are (phi, w) pairs)
    long long pat0;   // first pattern of the item
    int npat;         // number of patterns
    int pad;
    unsigned long long chunk0;  // first chunk of the item
    unsigned long long nchunk;  // chunks of the item
    unsigned long long group0;  // first reduction group of the item (SG_GROUP chunks each)
    unsigned long long ngroups; // reduction groups of the item
};

// Role of an item, from which the per-call values below are derived once
// the integral's parameters and base quantities are on the device.
#define SG_ROLE_FORWARD 0        // the integral itself
#define SG_ROLE_FORWARD_SHIFT 1  // same sum with the phase advanced by pi/2 (oscillatory gradient)
#define SG_ROLE_ADJOINT 2        // direction `dir` pinned at node x, other directions summed
struct SgItemRole {
    int role;
    int integral;
    int dir;
    int pad;
    double x;
};

// Per-call, parameter-dependent values of an item.
struct SgItemVar {
    double base_rel;  // the sum's centre term (1, cos(phase), ...)
    double mult;      // item value = mult * (base_rel + T), relative to the integral's scale
    double sin_phi, cos_phi;    // oscillatory phase of the per-point deviation
};

// One pattern of one item, or a contiguous range of its subsets (the planner
// may give the end of the work queue smaller chunks, and then splits a
// pattern into two records).
struct SgPatDev {
    int item;         // index into the item array
    int r;            // active directions (prefix r-1, tail 1)
    int A;            // prefix node tuples = prod of prefix block sizes
    int tm;           // tail block nodes per direction
    long long toff;   // table offset of the tail block (relative to item.tab)
    long long poff[SG_MAX_R - 1];  // table offsets of the prefix blocks
    int pm[SG_MAX_R - 1];          // nodes per direction of the prefix blocks
    double coef;      // multiplier of the pattern's sum (1, or Eq. 2.6 coefficient)
    unsigned long long rank0;  // first subset rank of this record
    unsigned long long nsub;   // end rank (exclusive): subsets [rank0, nsub) of the C(d, r)
    unsigned long long spc;    // subsets per chunk (1 when a subset is split)
    int asplit;                // chunks per subset (prefix-tuple blocks); 1 = no split
    int ablk;                  // prefix tuples per block when split
    unsigned long long chunk0; // first global chunk of this pattern
};

// Chunks per reduction group: the warp that completes the last chunk of a
// group sums the group's slots; the warp that completes the last group of an
// item sums the group results.  Both sums run in a fixed order.
#define SG_GROUP 64

// Per-group partial result: compensated pair and absolute sum.
struct alignas(32) SgGroupSlot {
    double s, c, abs, pad;
};

// Per-chunk partial result (written once by the warp that ran the chunk).
struct alignas(16) SgSlot {
    double sum;
    double abs;
};

// Per-output record on the device (matches sg_dev_result's first fields).
struct SgOutDev {
    double mant, exp2, value, cond, err_est, sum, abs_sum;
};

// Base quantities of an integral: Q = scale * (base + T), scale = exp(log_hi + log_lo)
// = 2^scale_e2 * scale_m (split once by the setup kernel, so that assembling
// a finished item needs no exponential).
struct SgBaseDev {
    double log_hi, log_lo;   // log of f(c) (exponential kinds), 0 for oscillatory
    double base;             // 1 or cos(theta_c)
    double sin_th, cos_th;   // theta_c for the oscillatory kind
    double scale_e2;         // integer power of two of the scale
    double scale_m;          // the scale's remaining factor, in [2^-1/2, 2^1/2]
};

// Arguments of a fold kernel (the built-in ones and a compiled user integrand's).
struct SgFoldArgs {
    const SgItemDev *items;
    const SgItemVar *vars;           // per item, filled by the setup kernel
    int nitems;
    const SgPatDev *pats;
    const unsigned long long *pat_chunk0;  // per pattern, ascending
    long long npat;
    unsigned long long nchunks;
    const void *tab;                 // float2* or double2*
    const unsigned long long *binom; // [k][n] table
    SgSlot *slots;                   // per chunk
    SgGroupSlot *gslots;             // per reduction group
    unsigned int *group_done;        // per group chunk tickets (zeroed before launch)
    unsigned long long *work;        // work-stealing counter (zeroed before launch)
    unsigned int *item_done;         // per item group tickets (zeroed before launch)
    const SgBaseDev *bases;          // per integral, for the final assembly
    const int *item_integral;        // per item: integral index (-1: adjoint sub-sum)
    SgOutDev *out;                   // per output
    double *vout;                    // adjoint sub-sum values (per output index)
    int *flags;                      // guard flags per item (written when guard_tol > 0)
    const int *skip_unflagged;       // if non-NULL: only items with flags[item] != 0 are run
    double guard_tol;
    double unit_roundoff;            // 2^-24 or 2^-53
};
)SG_RAW";
static const char sg_src_fold_logic[] = R"SG_RAW(// Enumeration primitives of the fold, shared by the CUDA kernel and the
// host-side index checker used in the tests (host and device inline code).
#pragma once
#include "sg_internal.h"

#ifdef __CUDACC__
#define SG_HD __host__ __device__ __forceinline__
#else
#define SG_HD inline
#endif

// C(n, k) from the [k][n] table (0 outside the table's domain).
SG_HD unsigned long long sg_binom(const unsigned long long *B, int n, int k) {
    if (n < 0 || k < 0 || k > n || n > SG_MAX_D || k >= SG_BINOM_K) return 0ull;
#ifdef __CUDA_ARCH__
    return __ldg(B + (size_t)k * (SG_MAX_D + 1) + n);
#else
    return B[(size_t)k * (SG_MAX_D + 1) + n];
#endif
}

// Lexicographic unranking of an r-subset {i_0 < ... < i_{r-1}} of [0, d).
// Given the previous element p, the number of subsets whose next element is
// smaller than v is C(d-p-1, k) - C(d-v, k) with k the elements still to
// place; v is found by binary search (C(d-v, k) decreases in v).
SG_HD void sg_unrank_lex(unsigned long long rank, int d, int r, const unsigned long long *B,
                         int *idx) {
    int p = -1;
    for (int t = 0; t < r; t++) {
        const int k = r - t;
        const unsigned long long total = sg_binom(B, d - p - 1, k);
        const unsigned long long target = total - rank;
        int lo = p + 1, hi = d - k;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (sg_binom(B, d - mid, k) >= target) lo = mid;
            else hi = mid - 1;
        }
        rank -= total - sg_binom(B, d - lo, k);
        idx[t] = lo;
        p = lo;
    }
}

// The same unranking, searched 32 candidates at a time (one per lane of a
// warp): for position t the answer v is the largest value in [lo, hi] with
// C(d-v, k) >= target.  A round tests lo + j*step, j = 0..31, with
// step = ceil((hi-lo+1)/32); `mask` has bit j set where the test holds (bit
// 0 always does) and the answer lies in the window after the last set bit.
// Rounds repeat until step = 1; d <= 8192 needs at most three.
struct SgUnrankPos {
    int k, lo, hi, step;
    unsigned long long total, target;
};

SG_HD void sg_unrank_begin(SgUnrankPos *u, unsigned long long rank, int d, int r, int t, int p,
                           const unsigned long long *B) {
    u->k = r - t;
    u->total = sg_binom(B, d - p - 1, u->k);
    u->target = u->total - rank;
    u->lo = p + 1;
    u->hi = d - u->k;
    u->step = (u->hi - u->lo + 32) / 32;
}

// Candidate of lane j in the current round and whether its test holds.
SG_HD int sg_unrank_candidate(const SgUnrankPos *u, int j) { return u->lo + j * u->step; }
SG_HD bool sg_unrank_test(const SgUnrankPos *u, int v, int d, const unsigned long long *B) {
    return v <= u->hi && sg_binom(B, d - v, u->k) >= u->target;
}

// Narrows the window after a round; returns 1 when lo is the answer.
SG_HD int sg_unrank_narrow(SgUnrankPos *u, unsigned mask) {
#ifdef __CUDA_ARCH__
    const int j = 31 - __clz(mask);
#else
    int j = 31;
    while (!((mask >> j) & 1u)) j--;
#endif
    const int done = u->step == 1;
    u->lo += j * u->step;
    if (!done) {
        const int hi = u->lo + u->step - 1;
        if (hi < u->hi) u->hi = hi;
        u->step = (u->hi - u->lo + 32) / 32;
    }
    return done;
}

// Lexicographic successor of a subset whose last element is d-1: the
// largest position t < r-1 that can still grow is incremented and the
// following positions restart right after it.  Returns 0 when exhausted.
SG_HD int sg_next_prefix(int *idx, int d, int r) {
    int t = r - 2;
    while (t >= 0 && idx[t] >= d - r + t) t--;
    if (t < 0) return 0;
    idx[t]++;
    for (int u = t + 1; u < r; u++) idx[u] = idx[u - 1] + 1;
    return 1;
}

// Enumerated direction -> actual direction when direction `skip` is left out.
SG_HD int sg_actual_dir(int i, int skip) { return i + (skip >= 0 && i >= skip); }

// Tail entries of a run whose last active direction takes the enumerated
// values plast .. plast + run - 1: one or two contiguous table segments
// (two when the actual directions jump over `skip`).
struct SgTailSegs {
    long long base1, base2;
    int E1, E2;
};

SG_HD SgTailSegs sg_tail_segments(long long toff, int tm, int plast, int run, int skip) {
    SgTailSegs s;
    const int a0 = sg_actual_dir(plast, skip), a1 = sg_actual_dir(plast + run - 1, skip);
    s.base1 = toff + (long long)a0 * tm;
    if (skip > a0 && skip < a1) {
        s.E1 = (skip - a0) * tm;
        s.E2 = (a1 - skip) * tm;
        s.base2 = toff + (long long)(skip + 1) * tm;
    } else {
        s.E1 = (a1 - a0 + 1) * tm;
        s.E2 = 0;
        s.base2 = 0;
    }
    return s;
}

// Lane position in the flat point space of a run, f = a * E + e (prefix
// tuple a, tail entry e): lane l starts at f = l and advances by 32, so every
// warp instruction but the last of a run has all 32 lanes busy, whatever
// the tail length E.
struct SgFlatPos {
    int a, e, da, de, E;
    SG_HD SgFlatPos(int lane, int E_) : E(E_) {
        da = 32 / E;
        de = 32 - da * E;
        a = lane / E;
        e = lane - a * E;
    }
    SG_HD void step() {
        e += de;
        a += da;
        if (e >= E) {
            e -= E;
            a++;
        }
    }
};

// Lane layout of the float fold: lane l takes tail entries e0, e0 + estep,
// ... and for each of them prefix tuples a0, a0 + astep, ...  With a tail of
// E >= 32 entries the whole warp shares every tuple (estep = 32, astep = 1);
// a shorter tail splits the warp into 32 / E groups of E lanes, group g
// taking tuples g, g + 32/E, ...; lanes beyond the last whole group idle.
struct SgLaneGroups {
    int e0, estep, a0, astep;
    bool active;
    SG_HD SgLaneGroups(int lane, int E) {
        const int G = E >= 32 ? 1 : 32 / E, Eg = E >= 32 ? 32 : E;
        a0 = lane / Eg;
        e0 = lane - a0 * Eg;
        estep = Eg;
        astep = G;
        active = a0 < G;
    }
};

// Table entry of prefix position t for prefix node tuple q (mixed radix over
// the prefix block sizes, the last prefix position fastest).  Returns the
// entry offset relative to the item's table and leaves q / m in *q.
SG_HD long long sg_prefix_entry(const SgPatDev *P, int t, int dir_actual, int *q) {
    const int m = P->pm[t];
    const int jt = *q % m;
    *q /= m;
    return P->poff[t] + (long long)dir_actual * m + jt;
}

// Work of chunk c of pattern P: subsets [rank, rank + cnt) and prefix node
// tuples [a_lo, a_hi).  A subset with more points than the chunk target is
// split over several chunks by prefix-tuple blocks (then cnt = 1).
SG_HD void sg_chunk_span(const SgPatDev *P, unsigned long long c, unsigned long long *rank,
                         unsigned long long *cnt, int *a_lo, int *a_hi) {
    const unsigned long long local = c - P->chunk0;
    if (P->asplit <= 1) {
        *rank = P->rank0 + local * P->spc;
        *cnt = P->nsub - *rank < P->spc ? P->nsub - *rank : P->spc;
        *a_lo = 0;
        *a_hi = P->A;
    } else {
        const unsigned long long sub = local / (unsigned long long)P->asplit;
        *rank = P->rank0 + sub;
        *cnt = 1;
        const int blk = (int)(local - sub * (unsigned long long)P->asplit);
        *a_lo = blk * P->ablk;
        *a_hi = *a_lo + P->ablk < P->A ? *a_lo + P->ablk : P->A;
    }
}

#if defined(__CUDACC__)
// Lexicographic unranking of the chunk's first r-subset by the whole warp:
// each round tests 32 candidates of one position at once (sg_unrank_*), so
// a position costs one or two rounds of parallel table loads instead of a
// serial binary search.  Lane 0 writes the subset to idx.
__device__ __forceinline__ void unrank_warp(unsigned long long rank, int d, int r,
                                            const unsigned long long *B, int *idx, int lane) {
    int p = -1;
    for (int t = 0; t < r; t++) {
        SgUnrankPos u;
        sg_unrank_begin(&u, rank, d, r, t, p, B);
        for (;;) {
            const unsigned m = __ballot_sync(0xffffffffu, sg_unrank_test(&u, sg_unrank_candidate(&u, lane), d, B));
            if (sg_unrank_narrow(&u, m)) break;
        }
        rank -= u.total - sg_binom(B, d - u.lo, u.k);
        if (lane == 0) idx[t] = u.lo;
        p = u.lo;
    }
}
#endif
)SG_RAW";
static const char sg_src_reduce[] = R"SG_RAW(// Deterministic reduction of the fold's chunk slots on the device: per-lane
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

)SG_RAW";
static const char sg_src_user_kernel[] = R"SG_RAW(// Fold kernel for a user integrand.  Not compiled into the library: it is
// compiled at run time by NVRTC (sg_integrand_create), after the user's
// source, which defines for a state of SG_USER_K doubles
//
//   __device__ void sg_user_centre(double *s, const double *p, int d);
//       the state of the centre point c = (1/2, ..., 1/2);
//   __device__ void sg_user_move(double *s, int i, double x, const double *p, int d);
//       moves direction i of the point held in s from 1/2 to x;
//   __device__ double sg_user_value(const double *s, const double *p, int d);
//       f at the point held in s;
//   optionally, with SG_USER_DEVIATION defined,
//   __device__ double sg_user_deviation(const double *s, const double *sc, const double *p, int d);
//       f(x) - f(c) for the points held in s and sc, without cancellation.
//
// This is the paper's multilevel dimension iteration with a vector state
// (Section 3: the symbolic function f_{t-m} after the first directions are
// fixed is represented by the state): per run, the prefix directions of
// every prefix node tuple are moved once into a state kept in shared memory;
// each point of the run then moves one more direction (its last active one)
// and evaluates.  Enumeration, chunking and the deterministic reduction are
// the built-in folds' (sg_fold_logic.h, sg_reduce.cuh); the tables hold the
// node coordinates and weights (SG_FAM_USER).  Sum in FP64:
//   Q = f(c) + sum_p W_p (f(x_p) - f(c)).
#include "sg_fold_logic.h"
#include "sg_reduce.cuh"

#ifndef SG_USER_K
#error "SG_USER_K (state size) must be defined"
#endif
#define SG_USER_APAD 64  // prefix tuples per warp in shared memory

struct SgUserArgs {
    const double *params;  // the user's parameters (device)
    int d;                 // dimension
    int pad;
};

// per-point deviation f(x) - f(c)
__device__ __forceinline__ double sg_user_dev(const double *s, const double *sc, double fc, const double *p,
                                              int d) {
#ifdef SG_USER_DEVIATION
    return sg_user_deviation(s, sc, p, d);
#else
    return sg_user_value(s, p, d) - fc;
#endif
}

extern "C" __global__ void sg_user_fold(SgFoldArgs A, SgUserArgs U) {
    extern __shared__ double sg_user_smem[];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const int SW = SG_USER_K + 1;  // state + weight per prefix tuple
    double *sS = sg_user_smem + (size_t)warp * SG_USER_APAD * SW;
    int *sIdx = (int *)(sg_user_smem + (size_t)nw * SG_USER_APAD * SW) + warp * SG_MAX_R;
    const double *p = U.params;
    const int dU = U.d;
    double sc[SG_USER_K];
    sg_user_centre(sc, p, dU);
    const double fc = sg_user_value(sc, p, dU);
    bool waited = false;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(A.work, 1ull);
        c = __shfl_sync(SG_FULL_MASK, c, 0);
        if (c >= A.nchunks) break;
        long long lo = 0, hi = A.npat - 1;
        while (lo < hi) {
            const long long mid = (lo + hi + 1) >> 1;
            if (__ldg(A.pat_chunk0 + mid) <= c) lo = mid;
            else hi = mid - 1;
        }
        const SgPatDev *P = A.pats + lo;
        const int item = P->item;
        const SgItemDev *I = A.items + item;
        const int d = I->d, r = P->r, tm = P->tm;
        unsigned long long rank, cnt;
        int a_lo, a_hi;
        sg_chunk_span(P, c, &rank, &cnt, &a_lo, &a_hi);
        unrank_warp(rank, d, r, A.binom, sIdx, lane);
        if (!waited) {  // the tables come from the setup kernel (dependent launch)
            asm volatile("griddepcontrol.wait;" ::: "memory");
            waited = true;
        }
        __syncwarp();
        const double2 *__restrict__ tab = (const double2 *)A.tab + I->tab;
        double acc = 0.0;
        while (cnt > 0) {
            const int plast = sIdx[r - 1];
            const int run = (unsigned long long)(d - plast) < cnt ? d - plast : (int)cnt;
            const long long tbase = P->toff + (long long)plast * tm;  // no left-out direction here
            const int E = run * tm;
            for (int ab = a_lo; ab < a_hi; ab += SG_USER_APAD) {
                const int At = a_hi - ab < SG_USER_APAD ? a_hi - ab : SG_USER_APAD;
                for (int a = lane; a < At; a += 32) {
                    int q = ab + a;
                    double s[SG_USER_K];
                    for (int k = 0; k < SG_USER_K; k++) s[k] = sc[k];
                    double W = 1.0;
                    for (int t = r - 2; t >= 0; t--) {
                        const int dir = sIdx[t];
                        const double2 e = tab[sg_prefix_entry(P, t, dir, &q)];
                        sg_user_move(s, dir, e.x, p, dU);
                        W *= e.y;
                    }
                    for (int k = 0; k < SG_USER_K; k++) sS[a * SW + k] = s[k];
                    sS[a * SW + SG_USER_K] = W;
                }
                __syncwarp();
                const int da = E >= 32 ? 0 : 32 / E, de = 32 - da * E;
                int a = lane / E, e = lane - (lane / E) * E;
                while (a < At) {
                    double s[SG_USER_K];
                    for (int k = 0; k < SG_USER_K; k++) s[k] = sS[a * SW + k];
                    const double2 te = tab[tbase + e];
                    sg_user_move(s, plast + e / tm, te.x, p, dU);
                    acc = fma(sS[a * SW + SG_USER_K] * te.y, sg_user_dev(s, sc, fc, p, dU), acc);
                    e += de;
                    a += da;
                    if (e >= E) {
                        e -= E;
                        a++;
                    }
                }
                __syncwarp();
            }
            cnt -= run;
            if (cnt > 0) {
                __syncwarp();
                if (lane == 0) sg_next_prefix(sIdx, d, r);
                __syncwarp();
            }
        }
        for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(SG_FULL_MASK, acc, o);
        if (lane == 0) {
            SgSlot sl;
            sl.sum = acc * P->coef;
            sl.abs = fabs(acc * P->coef);
            A.slots[c] = sl;
        }
        complete_chunk(A, item, c, lane, [&](double T, double AB) {
            // Q = f(c) + T
            const double q = fc + T;
            int e2 = 0;
            const double mant = frexp(q, &e2);
            SgOutDev o;
            o.mant = mant;
            o.exp2 = (double)e2;
            o.value = q;
            o.cond = (fabs(fc) + AB) / fabs(q);
            o.err_est = 0.05 * A.unit_roundoff * o.cond;
            o.sum = q;
            o.abs_sum = fabs(fc) + AB;
            A.out[I->out] = o;
        });
    }
}
)SG_RAW";
