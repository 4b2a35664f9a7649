/*
 * sg.h - C ABI of libsg: Smolyak sparse-grid quadrature on one GB300 GPU,
 * evaluated by multilevel dimension iteration (MDI).
 *
 * What the library computes (Zhong & Feng, "An efficient and fast sparse grid
 * algorithm for high-dimensional numerical integration", Section 2.1):
 *
 *   Q_d^q f = sum_{q-d+1 <= |l| <= q} (-1)^{q-|l|} C(d-1, q-|l|)
 *             sum_{|l| fixed} (J^{l_1} x ... x J^{l_d}) f               (Eq. 2.6)
 *
 * on the unit cube [0,1]^d, with J^l the level-l 1-D rule (Eqs. 2.10, 2.11,
 * 2.13, mapped from [-1,1] to [0,1]).  q = d + L; L = q - d >= 0 is the
 * "excess level".  The GPU evaluates the equal coordinate-wise form (Eq. 2.9,
 * read as a sum of tensor products of difference rules J^l - J^{l-1}) with
 * the direction-by-direction folding of Algorithms 3.1-3.3: the grid is never
 * stored, and partial sums over the leading directions of a cluster of points
 * are reused for every point of the cluster.
 *
 * Integrands are the Genz-type families of the paper's Section 4 and 5
 * tests.  Parameters are always 2d doubles, params = [a_0..a_{d-1},
 * u_0..u_{d-1}]:
 *   SG_FAM_EXP_LINEAR    f = exp(sum a_i x_i)                       (a)
 *   SG_FAM_OSCILLATORY   f = cos(2 pi u_0 + sum a_i x_i)            (a, u_0)
 *   SG_FAM_PRODUCT_PEAK  f = prod 1 / (a_i^-2 + (x_i - u_i)^2)      (a, u)
 *   SG_FAM_GAUSSIAN      f = exp(-sum a_i^2 (x_i - u_i)^2)          (a, u)
 *   SG_FAM_GAUSSIAN_LIN  f = exp(-sum a_i (x_i - u_i)^2)            (a, u)
 * Unused entries are ignored (their gradient is 0).
 *
 * Conventions for every entry point:
 *  - Status codes are returned; nothing throws across the ABI.  On error the
 *    outputs are left untouched.
 *  - `stream` is a cudaStream_t (NULL = the legacy default stream) of the
 *    current device.  Host-result entry points synchronise that stream
 *    before returning; sg_integrate_async does not.
 *  - The library owns rule handles and its internal device scratch (cached
 *    per device and grown on demand, freed at process exit).  The caller
 *    owns every params / result buffer it passes.
 *  - Calls from different host threads must use different streams.
 *  - Results are Q = mant * 2^exp2 (the product-peak value underflows a
 *    double for d >~ 150); `value` holds ldexp(mant, exp2).
 */
#ifndef SG_H
#define SG_H

#include <stddef.h>
#include <stdint.h>

#if defined(__GNUC__)
#define SG_API __attribute__((visibility("default")))
#else
#define SG_API
#endif

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    SG_OK = 0,
    SG_EINVAL = 1,       /* NULL pointer, bad enum, d < 1, q < d, ... */
    SG_ERANGE = 2,       /* size beyond a documented limit */
    SG_ENOMEM = 3,       /* device or host allocation failed */
    SG_ECUDA = 4,        /* a CUDA runtime call failed */
    SG_ETIMEOUT = 5,     /* reserved: no kernel of this library waits on another */
    SG_EUNSUPPORTED = 6  /* combination not implemented (e.g. gradient of comb form) */
} sg_status;

/* 1-D rules; the numbering is the paper's r (Section 3.1). */
typedef enum {
    SG_RULE_TRAPEZOID = 1,        /* Eq. 2.10; level 1 = midpoint (reading of the paper) */
    SG_RULE_CLENSHAW_CURTIS = 2,  /* Eq. 2.11; n_1 = 1, n_l = 2^(l-1) + 1, nested */
    SG_RULE_GAUSS_PATTERSON = 3,  /* Eq. 2.12; n_l = 2^l - 1 (members up to 63 nodes), nested */
    SG_RULE_GAUSS_LEGENDRE = 4    /* Eq. 2.13; n_l = l, not nested */
} sg_rule_kind;

/* How the 1-D level l maps to a member of the rule family. */
typedef enum {
    SG_GROWTH_STANDARD = 0,  /* level l is the l-th member (the n_l of sg_rule_kind) */
    SG_GROWTH_SLOW = 1       /* Section 5.4's accuracy levels: level l is the smallest member
                                exact for polynomials of degree 2l - 1, so the trapezoid and
                                Clenshaw-Curtis rules have N = 1, 3, 5, 9, 9, 17, 17, 17, 17, 33
                                and Gauss-Patterson N = 1, 3, 3, 7, 7, 7, 15, ...; Gauss-Legendre
                                is unchanged.  Levels that repeat a member add nothing. */
} sg_growth;

typedef enum {
    SG_FAM_EXP_LINEAR = 0,
    SG_FAM_OSCILLATORY = 1,
    SG_FAM_PRODUCT_PEAK = 2,
    SG_FAM_GAUSSIAN = 3,
    SG_FAM_GAUSSIAN_LIN = 4
} sg_family;

typedef enum {
    SG_PREC_FP64 = 0,   /* every step in IEEE double */
    SG_PREC_MIXED = 1,  /* integrand evaluation and per-cluster folds in float;
                           cross-cluster and cross-chunk sums exact in a
                           128-bit integer window, rounded once to double */
    SG_PREC_FF = 2      /* float-float: tables, folds and the per-point deviation
                           as unevaluated pairs of floats (about 44 bits) on the
                           FP32 pipes; cross-chunk sums in double */
} sg_precision;

/* Which algebraic form of the same Smolyak sum the kernels enumerate.  All
 * three give Q_d^q f up to rounding. */
typedef enum {
    SG_FORM_AUTO = 0,        /* SG_FORM_MERGED (gradients: SG_FORM_TELESCOPED) */
    SG_FORM_DIFFERENCE = 1,  /* sum_{|k|<=L} of tensor products of difference rules (Eq. 2.9) */
    SG_FORM_TELESCOPED = 2,  /* difference rules in all but the last active direction;
                                the last direction folds J^{M+1} - J^1 at once (Alg. 3.1) */
    SG_FORM_COMBINATION = 3, /* Eq. 2.6 literally (binomial coefficients) */
    SG_FORM_MERGED = 4       /* every distinct point once, with its merged weight (Eq. 2.8):
                                the difference-form terms of all subgrids that share a point
                                added into one weight, computed on the host in double-double;
                                fewest evaluations, and no worse conditioned than the
                                difference form */
} sg_form;

typedef struct sg_rule_s *sg_rule;  /* opaque, library-owned */

typedef struct {
    double value;      /* ldexp(mant, exp2); 0 or inf when out of double range */
    double mant;       /* 0.5 <= |mant| < 1 (or 0) */
    int64_t exp2;
    double cond;       /* sum_p |W_p D_p| / |sum|: conditioning of the signed sum */
    double err_est;    /* estimated relative rounding error of the result: 0.05 u cond
                          (u = 2^-53 FP64, 2^-44 float-float), 0.5 2^-24 cond mixed */
    uint64_t points;   /* n_d^q: points of Eq. 2.6 with repetition (the metric's unit) */
    uint64_t evals;    /* integrand deviations the kernels evaluated */
    double seconds;    /* device time of the call (CUDA events) */
} sg_result;

/* Device-side result record written by sg_integrate_async (7 doubles). */
typedef struct {
    double mant;
    double exp2;       /* integer-valued */
    double value;
    double cond;
    double err_est;
    double sum;        /* base + T before scaling (diagnostic) */
    double abs_sum;    /* sum |W_p D_p| (diagnostic) */
} sg_dev_result;

/*
 * Builds the 1-D rule tables of Eqs. 2.10, 2.11, 2.12 or 2.13 on [0,1] for
 * levels 1..max_level (host and device copies on the current device).  The
 * handle may be used with any d and q with q - d + 1 <= max_level.
 * Limits: 1 <= max_level <= 13 (4097 nodes for the nested rules).
 * Errors: SG_EINVAL (bad kind, NULL out), SG_ERANGE (max_level), SG_ENOMEM,
 * SG_ECUDA.
 */
SG_API sg_status sg_rule_init(sg_rule_kind kind, int max_level, sg_rule *out);

/*
 * As sg_rule_init, for the rule of Eq. 2.12 too and with a choice of level
 * growth (sg_growth).  The paper's Tables 4.1-4.9 and 5.1-5.5 use
 * SG_RULE_GAUSS_PATTERSON with SG_GROWTH_SLOW, their accuracy level k being
 * q = d + k - 1.  Limits: 1 <= max_level <= 13, and every level up to
 * max_level must have a member (Gauss-Patterson with standard growth:
 * max_level <= 6).  Errors as sg_rule_init; SG_EINVAL for a bad growth.
 */
SG_API sg_status sg_rule_init_growth(sg_rule_kind kind, sg_growth growth, int max_level, sg_rule *out);

/* Frees a handle from sg_rule_init.  NULL is accepted. */
SG_API sg_status sg_rule_destroy(sg_rule rule);

/*
 * Copies the level-`level` rule on [0,1] (nodes ascending) into caller-owned
 * host arrays x, w of capacity *n; on return *n = node count.  With x or w
 * NULL only *n is set.  Errors: SG_EINVAL, SG_ERANGE (level, capacity).
 */
SG_API sg_status sg_rule_nodes(sg_rule rule, int level, double *x, double *w, int *n);

/*
 * n_d^q = sum over the multi-indices of Eq. 2.6 of prod_i n_{l_i}: the point
 * count with repetition, the unit of the points/s metric.  Also the number
 * of integrand deviations the kernels evaluate for `form` (evals may be
 * NULL; SG_FORM_AUTO is resolved as for SG_PREC_FP64).
 * Errors: SG_EINVAL, SG_ERANGE (count beyond 2^64).
 */
SG_API sg_status sg_count_points(sg_rule rule, int d, int q, sg_form form, uint64_t *points,
                          uint64_t *evals);

/*
 * One integral Q_d^q f.  params: 2d doubles, host memory (params_on_device
 * = 0) or device memory of the current device (1).  Blocking: the result is
 * valid on return.  Limits: 1 <= d <= 8192, 0 <= q - d <= max_level - 1,
 * q - d <= 12, and the subgrid count must fit in 64 bits.
 * Errors: SG_EINVAL, SG_ERANGE, SG_ENOMEM, SG_ECUDA.
 */
SG_API sg_status sg_integrate(sg_rule rule, sg_family fam, const double *params, int params_on_device,
                       int d, int q, sg_precision prec, sg_form form, void *stream,
                       sg_result *out);

/*
 * Asynchronous variant: params and the result live in device memory of the
 * current device; every step is enqueued on `stream` and nothing
 * synchronises.  The first call for a (rule, d, q, prec, form) builds and
 * uploads that plan (host work plus a synchronous copy): do it once before
 * timing or capturing.  Same limits and errors as sg_integrate.
 */
SG_API sg_status sg_integrate_async(sg_rule rule, sg_family fam, const double *d_params, int d, int q,
                             sg_precision prec, sg_form form, void *stream,
                             sg_dev_result *d_out);

/* One batch entry: rule, family, dimension, q, and the offset of its 2d
 * parameters in the shared parameter pool. */
typedef struct {
    sg_rule rule;
    sg_family fam;
    int d;
    int q;
    uint64_t param_offset;
} sg_item;

/*
 * A batch of n integrals of uneven d and level, run by one persistent
 * work-stealing launch (plus a table-setup launch), replayed from a CUDA graph
 * cached for this batch layout.  params_pool: host (params_on_device = 0) or
 * device memory; item k reads pool[param_offset .. param_offset + 2d).
 * With prec = SG_PREC_MIXED and guard_tol > 0, items whose estimated
 * rounding error exceeds guard_tol are recomputed in float-float
 * (SG_PREC_FF) by a second persistent launch in the same graph, and those whose
 * float-float estimate still exceeds it by a third one in FP64.  The mixed
 * estimate is 0.5 * 2^-24 * cond (an upper bound of the float fold's error
 * over the 4096-integral batch workload).  out: n host records.  Blocking.
 * Limits: 1 <= n <= 65536, per item as sg_integrate.
 */
SG_API sg_status sg_integrate_batch(const sg_item *items, int n, const double *params_pool,
                             int params_on_device, sg_precision prec, double guard_tol,
                             void *stream, sg_result *out);

/*
 * Value and gradient: dparams[j] = dQ / dparams[j] for all 2d parameters,
 * written to caller-owned host (dparams_on_device = 0) or device memory.
 * Computed by a hand-written adjoint kernel: for each direction i, the sum
 * over every point where direction i is active of W_p f(x_p) times the
 * partial derivative factor of direction i, with the other directions folded
 * as in the forward pass; the centre term of each direction comes from Q.
 * Supported with SG_FORM_DIFFERENCE / SG_FORM_TELESCOPED / AUTO; the
 * combination form gives SG_EUNSUPPORTED.  Blocking.
 */
SG_API sg_status sg_integrate_grad(sg_rule rule, sg_family fam, const double *params,
                            int params_on_device, int d, int q, sg_precision prec, void *stream,
                            sg_result *out, double *dparams, int dparams_on_device);

/*
 * General integrands (the paper's symbolic functions, Section 3, with a
 * vector state).  A user integrand is CUDA C++ source that defines, for a
 * state of `state_size` doubles (1..16):
 *   __device__ void sg_user_centre(double *s, const double *p, int d);
 *       the state of the centre point c = (1/2, ..., 1/2);
 *   __device__ void sg_user_move(double *s, int i, double x, const double *p, int d);
 *       moves direction i (0-based) of the point held in s from 1/2 to x
 *       (each direction is moved at most once, in increasing order);
 *   __device__ double sg_user_value(const double *s, const double *p, int d);
 *       f at the point held in s;
 * and optionally, after #define SG_USER_DEVIATION,
 *   __device__ double sg_user_deviation(const double *s, const double *sc,
 *                                       const double *p, int d);
 *       f(x) - f(c) for the points held in s and sc, free of cancellation
 *       (without it the kernel forms sg_user_value(s) - f(c)).
 * p points to the caller's parameter array.  sg_integrand_create compiles it
 * with NVRTC for the current device together with the library's fold kernel
 * (prefix directions moved once per prefix node tuple, one more move and one
 * evaluation per point).  Errors: SG_EINVAL (NULL, or the source does not
 * compile: *out is then a handle whose compiler log sg_integrand_log
 * returns, to be destroyed), SG_ERANGE (state_size), SG_EUNSUPPORTED (no
 * NVRTC library found), SG_ENOMEM, SG_ECUDA.
 */
typedef struct sg_integrand_s *sg_integrand;
SG_API sg_status sg_integrand_create(const char *source, int state_size, sg_integrand *out);
SG_API sg_status sg_integrand_destroy(sg_integrand f);

/* Copies the compiler log (NUL-terminated, truncated to cap) and its length. */
SG_API sg_status sg_integrand_log(sg_integrand f, char *buf, size_t cap, size_t *len);

/*
 * Q_d^q f for a user integrand f (FP64, telescoped form; host or device
 * params of nparams >= 0 doubles).  Blocking, like sg_integrate; the result
 * is Q = f(c) + sum_p W_p (f(x_p) - f(c)) with the same fields.  Errors as
 * sg_integrate; SG_EINVAL also for a handle that failed to compile or was
 * compiled for another device.
 */
SG_API sg_status sg_integrate_user(sg_rule rule, sg_integrand f, const double *params, int nparams,
                                   int params_on_device, int d, int q, void *stream, sg_result *out);

/* Static description of a status code. */
SG_API const char *sg_status_string(sg_status s);

/* Tuning knobs used by the launches (read by the autotuner; see
 * sg_autotune).  points_per_chunk: target integrand evaluations per
 * work-stealing chunk; ctas_per_sm: resident CTAs per SM of the persistent
 * grid; warps_per_cta: warps per CTA. */
typedef struct {
    int points_per_chunk;
    int ctas_per_sm;
    int warps_per_cta;
} sg_tuning;

/* Reads / sets the tuning used for precision `prec` (process-wide). */
SG_API sg_status sg_get_tuning(sg_precision prec, sg_tuning *t);
SG_API sg_status sg_set_tuning(sg_precision prec, const sg_tuning *t);

/*
 * Times the given batch (as sg_integrate_batch would run it, without the
 * guard) under each candidate of a built-in grid of (points_per_chunk,
 * ctas_per_sm, warps_per_cta), keeps the fastest for `prec` and returns it
 * in *best (and its median time in *best_ms).  Blocking; runs each candidate
 * `reps` times.  Errors as sg_integrate_batch.
 */
SG_API sg_status sg_autotune(const sg_item *items, int n, const double *params_pool,
                      int params_on_device, sg_precision prec, int reps, void *stream,
                      sg_tuning *best, double *best_ms);


/*
 * A batch split into shards (no counterpart in the paper; the paper runs on
 * one CPU).  The subgrids of a batch are independent, so its chunk queue can
 * be cut into nshards contiguous ranges, each run by its own call (on one
 * GPU or, one process per GPU, on several).  sg_integrate_batch_shard runs
 * shard `shard` of `nshards` of the same batch sg_integrate_batch would run
 * (no guard; same planning) and returns, per item k (input order), the item's
 * long accumulator over the shard's chunks in partials[k * SG_SHARD_LIMBS ..]
 * (caller-owned host memory, n * SG_SHARD_LIMBS int64: the exact sum of the
 * chunk sums as 32 carry-save limbs, then the absolute sum) and, in info[k]
 * (caller-owned host, may be NULL), the item's values the combine needs.
 * Every shard computes the same info.  sg_shard_combine adds the shards'
 * limbs (integer additions: exact, in any order) and rounds and assembles
 * each item as the kernels do, so the results are bitwise the same for every
 * nshards, including 1, and the same as sg_integrate_batch's for the same
 * items and precision.  The exchange between GPUs is the limbs: 512 bytes
 * per item per shard.  Blocking.  Errors: SG_EINVAL (NULL, shard out of
 * range), SG_ERANGE (nshards > 65536), and those of sg_integrate_batch.
 */
#define SG_SHARD_LIMBS 64
typedef struct {
    double mult, base_rel;      /* item value = mult (base_rel + T), relative to the scale */
    double scale_m, scale_e2;   /* scale = scale_m 2^scale_e2 */
    double unit_roundoff;       /* of the precision, for the error estimate */
    uint64_t points, evals;
} sg_shard_info;
SG_API sg_status sg_integrate_batch_shard(const sg_item *items, int n, const double *params_pool,
                                          int params_on_device, sg_precision prec, int shard, int nshards,
                                          void *stream, long long *partials, sg_shard_info *info);
SG_API sg_status sg_shard_combine(const long long *const *partials, int nshards, const sg_shard_info *info,
                                  int n, sg_result *out);

/*
 * Per-class tuning of the batch path (no counterpart in the paper; the
 * paper's step sizes m and s of Algorithm 3.3 have no analogue on the GPU).
 * A class is (family, rule, ceil(log2 d), q - d, precision).  For every class
 * present in the items, sg_autotune_classes times the class's items as a
 * batch (as sg_integrate_batch runs them, without the guard) under each
 * candidate chunk size (1024, 4096, 16384, 65536, 262144 points per chunk),
 * `reps` times after one warm-up, and keeps the fastest.  The table applies
 * to every later sg_integrate_batch call in this process (the items of a
 * class are planned with its chunk size; other items keep the precision's
 * tuning) and is written to `path` as JSON unless path is NULL; *nclasses
 * (may be NULL) receives the table's size.  sg_tuning_load replaces the
 * table by one read from such a file; sg_tuning_clear empties it.  Chunk
 * sizes change only the order in which terms are added: results agree to
 * rounding.  Blocking.  Errors: SG_EINVAL (NULL, bad file), and those of
 * sg_integrate_batch.
 */
SG_API sg_status sg_autotune_classes(const sg_item *items, int n, const double *params_pool,
                                     int params_on_device, sg_precision prec, int reps, void *stream,
                                     const char *path, int *nclasses);
SG_API sg_status sg_tuning_load(const char *path, int *nclasses);
SG_API sg_status sg_tuning_clear(void);

/*
 * Measurement hooks (no counterpart in the paper).  sg_profile_begin starts
 * recording CUDA events around every fold-kernel launch this library
 * enqueues on `stream` (not inside graph replays); sg_profile_end
 * synchronises the stream, returns the summed device time of those launches
 * in ms and their count, and stops recording.  Errors: SG_EINVAL, SG_ECUDA.
 */
SG_API sg_status sg_profile_begin(void *stream);
SG_API sg_status sg_profile_end(void *stream, double *fold_ms, int *launches);

/*
 * Throughput ceiling of the fold's per-point work on this GPU: the same
 * sequence as the fold's inner loop (argument add, weight product,
 * deviation, weighted accumulate; in `prec`) on register-resident data, on
 * a full grid of the device, without loads, enumeration or reduction.
 * kind 0: expm1 deviation, 1: oscillatory deviation (points/s), 2: plain
 * fused multiply-add chains (FLOP/s).  Blocking.  Errors: SG_EINVAL,
 * SG_ECUDA.
 */
SG_API sg_status sg_ceiling(sg_precision prec, int kind, void *stream, double *rate);

/*
 * Accuracy hook (no counterpart in the paper): evaluates the elementary
 * functions the fold uses per point, in the given precision, on n device
 * arguments d_x.  kind 0: y[i] = expm1(x[i]); kind 1: y[2i] = sin(x[i]),
 * y[2i+1] = cos(x[i]).  d_y is caller-owned device memory (n or 2n
 * doubles).  Asynchronous on `stream`.  Errors: SG_EINVAL, SG_ECUDA.
 */
SG_API sg_status sg_eval_functions(int kind, sg_precision prec, const double *d_x, double *d_y, int n,
                                   void *stream);

/*
 * One integral without any memory allocation (the paper has no counterpart;
 * this exists for callers that must not allocate).  Some callers cannot call
 * cudaMalloc or any allocator where they integrate: a host thread in a
 * latency-critical loop (cudaMalloc/cudaFree synchronise the device and
 * stall other streams), or a runtime that owns all device memory and forbids
 * libraries to allocate behind its back.  This entry point takes the rule
 * kind instead of a handle, device params (2d doubles) and a device result
 * record, like sg_integrate_async, and uses the telescoped form.  Its device
 * scratch is one fixed array of about 5.2 MB inside the library, held by
 * every GPU that loads the library until the process exits.
 * Rules: the four kinds with standard growth (Gauss-Patterson: q - d <= 5).
 * Limits: 1 <= d <= 1024, 0 <= q - d <= 6, at most 131072 table entries
 * (d times the summed node counts of the rule blocks) and 65536 work chunks;
 * larger problems return SG_ERANGE.  The first call on a device (with that
 * device current) resolves the array's address and uploads a table with a
 * synchronous copy: make it before any stream capture.  All calls share the
 * array and leave their data in it (work tickets are cleared at the start of
 * each call); calls that overlap on the GPU race on it and must be
 * serialised by the caller.  Errors: SG_EINVAL, SG_ERANGE, SG_ECUDA.
 */
SG_API sg_status sg_integrate_noalloc(sg_rule_kind kind, sg_family fam, const double *d_params, int d,
                                      int q, sg_precision prec, void *stream, sg_dev_result *d_out);

#ifdef __cplusplus
}
#endif

#endif /* SG_H */
