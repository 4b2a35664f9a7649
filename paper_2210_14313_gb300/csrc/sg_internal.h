// Internal data layout shared by the host planner and the CUDA kernels of
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
#define SG_BLK_NEW 3    // the nodes level k+1 adds to levels 1..k, k >= 1 (merged form;
                        // the point weights come from a per-pattern table)

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
    long long woff;            // merged form: first weight of the pattern (weights of prefix
                               // tuple a, tail node j at woff + a * tm + j); -1 otherwise
};

// Chunks per reduction group: the warp that completes the last chunk of a
// group sums the group's slots; the warp that completes the last group of an
// item sums the group results.  Both sums run in a fixed order.
#define SG_GROUP 64

// Per-group partial result: the group's exact sum as a pair of doubles
// (s the nearest double, c the rest) and its absolute sum.
struct alignas(32) SgGroupSlot {
    double s, c, abs, pad;
};

// A merged-form point weight for the FP64 fold, kept to 64 significant
// bits: |w| = m 2^(e - 1086) with m's leading one at bit 63, sign neg.
struct alignas(16) SgW64 {
    unsigned long long m;
    int e;
    int neg;
};

// Per-chunk partial result (written once by the warp that ran the chunk):
// the chunk's sum as sum + lo (lo is the rest of an exact sum that the FP64
// merged fold keeps below the double sum; 0 elsewhere) and its absolute sum.
struct alignas(32) SgSlot {
    double sum;
    double abs;
    double lo;
    double pad;
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
// Where chunk c starts: its pattern and the first r-subset of its span
// (enumerated directions), unranked once per plan on the device.
struct alignas(32) SgChunkStart {
    int pat;
    unsigned short idx[SG_MAX_R];
    int pad;
};

struct SgFoldArgs {
    const SgItemDev *items;
    const SgItemVar *vars;           // per item, filled by the setup kernel
    int nitems;
    const SgPatDev *pats;
    const unsigned long long *pat_chunk0;  // per pattern, ascending
    long long npat;
    const SgChunkStart *chunk_start; // per chunk (NULL: found by search and unranking)
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
    double unit_roundoff;            // effective unit roundoff: err_est = 0.05 * this * cond
    // Single-integral plans (one forward item, no guard): every chunk's sum
    // goes into a long accumulator in the CTA's shared memory (sg_lacc.h),
    // each CTA adds its accumulator into the launch's accumulator `lacc`
    // (2 SG_LA_DIGITS limbs: the sum, then the absolute sum) and the last
    // CTA to finish rounds it and assembles the result.  cta_done[0] counts
    // finished CTAs, cta_done[1] flags a term outside the accumulator's
    // window; that last CTA returns lacc, both counters and the work counter
    // to zero.
    int single;
    long long *lacc;
    unsigned int *cta_done;
    // merged form: point weights of every pattern (SgW64 for the FP64 fold,
    // float pairs hi + lo for the float and float-float folds)
    const void *wtab;
    // Batches and gradients (not single): when ilacc is set, every chunk adds
    // its sum and absolute sum into its item's long accumulator
    // (2 SG_LA_DIGITS limbs per item, zeroed before the launch) with integer
    // atomics and counts itself in item_done; the warp that completes an
    // item rounds and assembles it, unless no_assemble (a shard of a batch,
    // whose items the host combines).  Without ilacc: the per-chunk slots.
    long long *ilacc;
    int no_assemble;
    // chunks [chunk_lo, chunk_hi) of the plan's queue (chunk_hi 0: all)
    unsigned long long chunk_lo, chunk_hi;
};
