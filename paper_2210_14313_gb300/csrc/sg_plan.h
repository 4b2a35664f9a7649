// Host planner of libsg: turns integrals into items, table blocks,
// patterns and work-stealing chunks (pure host code, no CUDA calls).
#pragma once
#include <vector_types.h>

#include <vector>

#include "../../include/sg.h"
#include "sg_kernels.h"

typedef unsigned long long u64;

struct sg_rule_s {
    int kind = 0, max_level = 0, device = 0;
    // blocks [bk][k], k = 1..max_level-1
    std::vector<double> x[4][SG_MAX_LEVEL], w[4][SG_MAX_LEVEL];
    int off[4][SG_MAX_LEVEL] = {};
    double2 *d_xw = nullptr;  // device copy of all blocks (set by sg_rule_init)
};


struct BlockRef {
    int bk, k;
    bool operator<(const BlockRef &o) const { return bk != o.bk ? bk < o.bk : k < o.k; }
    bool operator==(const BlockRef &o) const { return bk == o.bk && k == o.k; }
};

struct PatSpec {
    int r;
    BlockRef pre[SG_MAX_R - 1];
    BlockRef tail;
    double coef;
    long long woff = -1;  // merged form: first weight in the plan's weight arrays
};

struct Req {
    sg_rule rule;
    int fam, d, L, form;
    long long param_off;
    int grad;
    int ppc = 0;  // points per chunk for this integral (0: the precision's tuning)
    bool operator==(const Req &o) const {
        return rule == o.rule && fam == o.fam && d == o.d && L == o.L && form == o.form &&
               param_off == o.param_off && grad == o.grad && ppc == o.ppc;
    }
};

struct Plan {
    unsigned long long id = 0;  // unique per built plan (never reused, unlike its address)
    bool narrow = false;        // a single FP64 integral: the fold build for 2 CTAs per SM
    std::vector<Req> reqs;
    int prec = 0;
    sg_tuning tune{};
    int device = 0;
    // host copies
    std::vector<SgIntegralDev> integrals;
    std::vector<SgBlockDev> blocks;
    std::vector<BlockRef> block_refs;  // rule block of each table block (host side)
    std::vector<long long> block_end;
    std::vector<SgItemDev> items;
    std::vector<SgItemRole> roles;
    std::vector<int> item_integral;
    std::vector<int> int_item_ptr, int_items;  // items of each integral (CSR)
    std::vector<SgPatDev> pats;
    std::vector<u64> pat_chunk0;
    long long nentries = 0;
    u64 nchunks = 0;
    u64 ngroups = 0;
    int nout = 0;
    long long nv = 0;
    std::vector<u64> points, evals;  // per integral (forward sum only)
    // merged-form point weights of every pattern that uses them, in the two
    // formats the folds read (64-bit significands; float pairs hi + lo)
    std::vector<SgW64> wt64;
    std::vector<float2> wtff;
    u64 total_evals = 0;             // every item, adjoint included
    int max_d = 0;
    // gradient (single integral)
    int vstride = 0;
    std::vector<int> delta_off, delta_m;
    // device copies (one allocation)
    void *dmem = nullptr;
    SgIntegralDev *d_integrals = nullptr;
    SgBlockDev *d_blocks = nullptr;
    long long *d_block_end = nullptr;
    SgItemDev *d_items = nullptr;
    SgItemRole *d_roles = nullptr;
    int *d_item_integral = nullptr;
    int *d_int_item_ptr = nullptr, *d_int_items = nullptr;
    SgPatDev *d_pats = nullptr;
    u64 *d_pat_chunk0 = nullptr;
    SgChunkStart *d_chunk_start = nullptr;  // per chunk, filled on the device at upload
    const SgW64 *d_wt64 = nullptr;
    const float2 *d_wtff = nullptr;
    int *d_delta_off = nullptr, *d_delta_m = nullptr;
    double2 *d_delta_xw = nullptr;  // the rule's block array (borrowed)
    int launch_ctas = 0;
};

// C(n, k) in 128 bits, saturating at 2^127.
unsigned __int128 binom128(long long n, int k);
// Pattern list of one Smolyak sum (see sg_plan.cpp).
void gen_patterns(int form, int d, int L, std::vector<PatSpec> &out);
// Nodes per direction of a rule block.
int tab_m(sg_rule rule, BlockRef b);
void drop_empty_patterns(sg_rule rule, std::vector<PatSpec> &specs);
// Merged-form point weights of the patterns `specs` (d directions, excess
// budget L) appended to the plan's weight arrays, times `factor`; sets each
// pattern's woff.  False when there would be more than 2^24 weights.
bool merged_weights(sg_rule rule, int d, int L, double factor, std::vector<PatSpec> &specs, Plan *P);
// n_d^q of Eq. 2.6 (false if beyond 64 bits).
bool count_points(int kind, int d, int L, u64 *out);
// Builds the host arrays of a plan; device fields stay empty.
// resident_warps: warps the persistent fold grid keeps on the device (sets the chunk size).
sg_status build_plan_host(const std::vector<Req> &reqs, int prec, const sg_tuning &tune,
                          long long resident_warps, Plan **out);
void plan_free_host(Plan *P);
