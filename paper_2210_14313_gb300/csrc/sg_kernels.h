// Launch wrappers of libsg's CUDA kernels (host-callable, no torch types).
#pragma once
#include <cuda_runtime.h>

#include "sg_internal.h"

// One 1-D rule block attached to an integral's table: m nodes per direction
// for d directions, entries (phi_i(x_j), w_j) at table[off + i*m + j].
struct SgBlockDev {
    long long off;        // absolute table entry offset
    int m;                // nodes per direction
    int integral;         // integral index (params, family)
    const double2 *xw;    // the rule block's (x_j, w_j) on the device
};

// Per integral data the setup kernel needs.
struct SgIntegralDev {
    int fam;              // sg_family
    int d;
    long long param_off;  // offset of the 2d parameters in the pool
    int flag_item;        // item whose guard flag gates the FP64 table build (-1: always)
    int pad;
};

#define SG_SETUP_INLINE 32  // block descriptors passed by value when a plan has this few

struct SgSetupArgs {
    const SgBlockDev *blocks;
    const long long *block_end;  // inclusive prefix sum of block entry counts
    int nblocks;
    int ninline;                 // > 0: blocks/ends below are valid copies (kernel parameters)
    SgBlockDev blk_inline[SG_SETUP_INLINE];
    long long end_inline[SG_SETUP_INLINE];
    long long nentries;
    const SgIntegralDev *integrals;
    int nintegrals;
    const double *params;
    float2 *tab32;                // may be NULL
    double2 *tab64;               // may be NULL
    float4 *tabff;                // float-float (value hi, lo, weight hi, lo); may be NULL
    SgBaseDev *bases;             // one per integral
    const int *flags;             // guard flags per item (NULL: build all)
    // per-item values, computed by each integral's warp right after its base
    // quantities (0: left to sg_launch_prep)
    int do_items;
    const int *int_item_ptr;      // items of integral g: int_items[ptr[g] .. ptr[g+1])
    const int *int_items;
    const SgItemRole *roles;
    const SgItemDev *items;
    const int *item_integral;
    SgItemVar *vars;
    SgOutDev *out;
    double *vout;
    double unit_roundoff;
};



// Fills the per-chunk start records of a plan (pattern and first subset).
cudaError_t sg_launch_chunk_starts(const SgItemDev *items, const SgPatDev *pats, const unsigned long long *pat_chunk0,
                                   long long npat, unsigned long long nchunks, const unsigned long long *binom,
                                   SgChunkStart *out, cudaStream_t s);

#define SG_APAD 128  // prefix states per warp held in shared memory

// Grid sizing of the persistent fold kernel.
struct SgLaunchCfg {
    int ctas;
    int warps_per_cta;
    int dependent;  // launch as a programmatic dependent of the preceding kernel
};

// Plans with more chunks than this launch the fold plainly: the dependent
// launch saves a few microseconds of setup overlap but, measured on GB300,
// costs about 0.14 us per chunk serialised over the whole grid (a 1.5e7-chunk
// FP64 batch took 5.0 s instead of 2.9 s).
#define SG_DEPENDENT_LAUNCH_MAX_CHUNKS 65536

// Binomial table C(n, k), n <= SG_MAX_D, k < SG_BINOM_K (saturating), layout [k][n].
void sg_fill_binomials(unsigned long long *host_table);

cudaError_t sg_launch_setup(const SgSetupArgs &a, cudaStream_t s);

struct SgPrepArgs {
    const SgItemRole *roles;
    const SgItemDev *items;
    int nitems;
    const SgIntegralDev *integrals;
    const double *params;
    const SgBaseDev *bases;
    const int *item_integral;
    SgItemVar *vars;
    // items without any chunk (nothing beyond the centre term) are finished here
    SgOutDev *out;
    double *vout;
    int *flags;
    double unit_roundoff;
};
// Fills the per-call item values (phases, multipliers) after the setup kernel.
cudaError_t sg_launch_prep(const SgPrepArgs &a, cudaStream_t s);
// prec: 0 = double tables, 1 = float tables, 2 = float-float tables.
cudaError_t sg_launch_fold(const SgFoldArgs &a, int prec, int gk, SgLaunchCfg cfg, cudaStream_t s);
// Resident CTAs per SM of the fold kernel for this precision / warps per CTA.
int sg_fold_occupancy(int prec, int gk, int warps_per_cta);

struct SgGradArgs {
    int fam, d, L;
    const double *params;        // 2d parameters (device)
    const double2 *delta_xw;     // DELTA blocks of the rule, concatenated for k = 1..L
    const int *delta_off;        // offsets of block k in delta_xw (k = 1..L), and m_k
    const int *delta_m;
    const double *v;             // adjoint sub-sums, [i][sum_k m_k]
    int vstride;
    const SgOutDev *q;           // forward value record (relative, see below)
    const SgOutDev *qh;          // phase-shifted forward value (oscillatory) or NULL
    const SgBaseDev *base;
    double *grad_rel;            // out: 2d values, dQ/dtheta / scale
};
cudaError_t sg_launch_grad(const SgGradArgs &a, cudaStream_t s);

// Ceiling microbenchmarks (see sg_ceiling in include/sg.h).  Returns the
// number of points (or flops) one launch performs.
double sg_launch_ceiling(int prec, int kind, int sms, double *d_out, cudaStream_t s);

// Evaluates the fold's elementary functions (kind 0: expm1 -> y[i]; kind 1:
// sincos -> y[2i], y[2i+1]) in precision prec (0 double, 1 float) on device
// arrays, for accuracy tests.
cudaError_t sg_launch_fn(int kind, int prec, const double *x, double *y, int n, cudaStream_t s);
