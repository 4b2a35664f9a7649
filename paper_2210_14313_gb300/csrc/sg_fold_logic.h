// Enumeration primitives of the fold, shared by the CUDA kernel and the
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

// Division by a block size without a divide instruction: for 0 <= q < 2^31
// and 1 <= m < 2^31, with l = ceil(log2 m) and M = floor(2^(31 + l) / m) + 1
// (< 2^32), q / m = floor(q M / 2^(31 + l)) (Granlund & Montgomery,
// "Division by invariant integers using multiplication", 1994, Thm. 4.2).
struct SgDivMagic {
    unsigned M;
    int sh;
};

SG_HD SgDivMagic sg_div_magic(int m) {
#ifdef __CUDA_ARCH__
    const int l = m > 1 ? 32 - __clz(m - 1) : 0;
#else
    int l = 0;
    while ((1ll << l) < (long long)m) l++;
#endif
    SgDivMagic g;
    g.M = (unsigned)((1ull << (31 + l)) / (unsigned long long)m + 1ull);
    g.sh = 31 + l;
    return g;
}

SG_HD int sg_div_magic_q(int q, SgDivMagic g) {
    return (int)(((unsigned long long)(unsigned)q * g.M) >> g.sh);
}

// One prefix position of the current run: the table row of its direction,
// its block size m and m's division magic.
struct SgPrefixPos {
    long long row;
    SgDivMagic dm;
    int m, pad;
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
