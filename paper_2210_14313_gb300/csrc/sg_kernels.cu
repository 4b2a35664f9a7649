// CUDA kernels of libsg (sm_103a).
//
// The hot path is sg_fold_kernel: a persistent, work-stealing kernel in
// which each warp takes a chunk of subgrids of one pattern (Section 2.1,
// Eq. 2.9 read as sums of tensor products of difference rules), unranks the
// first subgrid (lexicographic r-subset of the directions), and walks the
// chunk as *runs*: maximal sequences of subgrids that share their first r-1
// active directions (the prefix) and differ only in the last one.  This is
// the paper's multilevel dimension iteration (Algorithms 3.1-3.3): the
// prefix directions are folded once per run into per-node-tuple states
// (partial argument S_a and weight W_a, the "symbolic function" of Eq. 3.10
// held as numbers), staged in shared memory, and every point of the run
// then costs one table load, one add, one deviation evaluation and one FMA.
// No point of the grid is ever stored.
//
// Integrands are generalised-additive, f(x) = F(theta + sum_i phi_i(x_i)),
// with F = exp (exp-linear, gaussian, gaussian-lin, product peak via
// phi = log psi) or F = cos (oscillatory).  Per point the kernel evaluates
// the deviation from the centre value without cancellation:
//   exp:  D = expm1(S)                  (relative to f(c))
//   cos:  D = cos(phi + S) - cos(phi) = -2 sin(S/2) sin(phi + S/2)
// and accumulates W * D.  Since every non-centre subgrid's weights sum to
// zero, sum W f = sum W D, and the cancelling signed sum stays small.
//
// Reduction is deterministic: each chunk writes one (sum, abs) slot, the
// warps that complete a group of slots and then an item's last group
// (ticket counters) add them exactly in a 128-bit integer window
// (sg_xsum.h), so no order of additions can change a bit.
//
// In FP64 the deviation's polynomials run in 64-bit fixed point on the
// integer pipes (sg_fixed.h): GB300 issues FP64 at 1/72 of its FP32 rate.
#include <math.h>
#include <stdio.h>

#include <type_traits>

#include "sg_ff.cuh"
#include "sg_fixed.h"
#include "sg_fold_logic.h"
#include "sg_kernels.h"
#include "sg_lacc.h"
#include "sg_reduce.cuh"

#define FULL_MASK 0xffffffffu

// ---------------------------------------------------------------------------
// helpers
// ---------------------------------------------------------------------------


// Per-direction deviation phi_i(x) - phi_i(1/2) of each family, in FP64,
// written without cancellation.
__device__ __forceinline__ double phi_dev(int fam, double a, double u, double x) {
    switch (fam) {
    case 0:  // exp-linear: a (x - 1/2)
    case 1:  // oscillatory: a (x - 1/2)
        return a * (x - 0.5);
    case 2: {  // product peak: log(psi(x)/psi(1/2)), psi = 1/(a^-2 + (x-u)^2)
        double v = x - u;
        double eps = (0.5 - x) * (0.5 + x - 2.0 * u) / (1.0 / (a * a) + v * v);
        return log1p(eps);
    }
    case 3:  // gaussian: -a^2 [(x-u)^2 - (1/2-u)^2]
        return -a * a * (x - 0.5) * (x + 0.5 - 2.0 * u);
    case 4:  // gaussian-lin: -a [(x-u)^2 - (1/2-u)^2]
        return -a * (x - 0.5) * (x + 0.5 - 2.0 * u);
    }
    return 0.0;
}

// Table value of a direction's deviation: phi_dev, except that the
// oscillatory family stores half the phase deviation, so that the per-point
// deviation -2 sin(S/2) sin(phi + S/2) needs no halving of the folded S.
__device__ __forceinline__ double phi_table(int fam, double a, double u, double x) {
    const double v = phi_dev(fam, a, u, x);
    return fam == 1 ? 0.5 * v : v;
}

// phi_i(1/2): the direction's share of log f(c) (exponential families) or of
// the phase (oscillatory).
__device__ __forceinline__ double phi_centre(int fam, double a, double u) {
    switch (fam) {
    case 0:
    case 1:
        return 0.5 * a;
    case 2:
        return -log(1.0 / (a * a) + (0.5 - u) * (0.5 - u));
    case 3:
        return -a * a * (0.5 - u) * (0.5 - u);
    case 4:
        return -a * (0.5 - u) * (0.5 - u);
    }
    return 0.0;
}

// Float-float precision tag: table entries and prefix states are float4
// (value hi, lo, weight hi, lo).
struct FFTag {};

template <typename T> struct V2T;
template <> struct V2T<float> { typedef float2 type; };
template <> struct V2T<double> { typedef double2 type; };
template <> struct V2T<FFTag> { typedef float4 type; };

// expm1 in float for the fold's argument range (no special-case paths): Cody & Waite argument reduction x = k ln2 + r, |r| <= ln2/2,
// with ln 2 split so that k * ln2_hi is exact, the Taylor series of
// expm1(r) to degree 8 (truncation below 2.1e-10 relative), and
// expm1(x) = 2^k expm1(r) + (2^k - 1), which is r's series itself when
// k = 0.  k is clamped to [-126, 127]: below -87 the result is -1 to float
// precision; the fold's arguments stay far below the overflow end.
__device__ __forceinline__ float sg_expm1f(float x) {
    const float k = fminf(fmaxf(rintf(x * 1.44269504088896341f), -126.f), 127.f);
    float r = fmaf(-k, 6.93145752e-1f, x);
    r = fmaf(-k, 1.42860677e-6f, r);
    float h = fmaf(r, 2.48015873e-5f, 1.98412698e-4f);  // 1/8!, 1/7!
    h = fmaf(h, r, 1.38888889e-3f);                     // 1/6!
    h = fmaf(h, r, 8.33333333e-3f);                     // 1/5!
    h = fmaf(h, r, 4.16666667e-2f);                     // 1/4!
    h = fmaf(h, r, 1.66666667e-1f);                     // 1/3!
    h = fmaf(h, r, 0.5f);
    const float p = fmaf(r * r, h, r);
    const float scale = __int_as_float(((int)k + 127) << 23);
    return fmaf(scale, p, scale - 1.0f);
}

// sin and cos in double for the fold (|x| < 2^20; larger arguments, Inf and
// NaN take CUDA's sincos out of line).  Cody & Waite reduction
// x = k pi/2 + r with pi/2 in three parts, the first two of 33 significant
// bits so that k * part is exact for |k| < 2^20; k is rounded by adding
// 1.5 * 2^52 to x * 2/pi, whose low word then holds k mod 2^32 (the
// quadrant).  On |r| <= 0.7854 (pi/4 plus rounding) sin r and cos r come from
// the fixed-point polynomials of sg_fixed.h.  The quadrant swaps and sign
// flips are integer operations on the result words.  Arguments below pi/4
// skip the reduction (in the fold most lanes of a warp agree on this
// branch).
__device__ __noinline__ double2 sg_sincos_slow(double x) {
    double s, c;
    sincos(x, &s, &c);
    return make_double2(s, c);
}

__device__ __forceinline__ double sg_flip_sign(double v, unsigned m) {
    return __hiloint2double(__double2hiint(v) ^ (int)m, __double2loint(v));
}

__device__ __forceinline__ void sg_sincos_d(double x, double *sp, double *cp) {
    const int hx = __double2hiint(x) & 0x7fffffff;
    if (hx < 0x3fe921fb) {  // |x| < 0.7853975... (just below pi/4)
        sg_fx_sincos(x, sp, cp);
        return;
    }
    if (hx >= 0x41300000) {  // |x| >= 2^20, Inf, NaN
        const double2 v = sg_sincos_slow(x);
        *sp = v.x;
        *cp = v.y;
        return;
    }
    const double magic = 6755399441055744.0;  // 1.5 * 2^52
    const double t = fma(x, 6.36619772367581382433e-01, magic);
    const unsigned q = (unsigned)__double2loint(t);
    const double k = t - magic;
    double r = fma(-k, 1.57079632673412561417e+00, x);  // pi/2 head (33 bits)
    r = fma(-k, 6.07710050630396597660e-11, r);         // middle (33 bits)
    r = fma(-k, 2.02226624879595063540e-21, r);         // tail
    double sr, cr;
    sg_fx_sincos(r, &sr, &cr);
    // x = k pi/2 + r: (sin, cos) = (s, c), (c, -s), (-s, -c), (-c, s) for k mod 4
    const double a = (q & 1u) ? cr : sr, b = (q & 1u) ? sr : cr;
    *sp = sg_flip_sign(a, (q & 2u) << 30);
    *cp = sg_flip_sign(b, ((q + 1u) & 2u) << 30);
}

// expm1 in double for the fold:
//   |x| < ln2/2: the fixed-point polynomial of sg_fixed.h;
//   |x| < 700:   Cody & Waite reduction x = k ln2 + r with ln 2 in two parts
//                (head of 32 bits: k * head exact), k rounded by adding
//                1.5 * 2^52, expm1(r) as above, and
//                expm1(x) = 2^k expm1(r) + (2^k - 1) with 2^k from integer bits;
//   otherwise (overflow, -1, Inf, NaN): the library expm1 out of line.
__device__ __noinline__ double sg_expm1_slow(double x) { return expm1(x); }

__device__ __forceinline__ double sg_expm1_d(double x) {
    const int hx = __double2hiint(x) & 0x7fffffff;
    if (hx < 0x3fd62e42) return sg_fx_expm1(x);   // |x| < 0.34657...
    if (hx >= 0x4085e000) return sg_expm1_slow(x);  // |x| >= 700, Inf, NaN
    const double magic = 6755399441055744.0;  // 1.5 * 2^52
    const double t = fma(x, 1.4426950408889634, magic);
    const int k = __double2loint(t);
    const double kd = t - magic;
    double r = fma(-kd, 6.9314718060195446e-01, x);  // ln 2 head (32 bits)
    r = fma(-kd, -4.2009150726810846e-11, r);         // tail
    const double scale = __hiloint2double((k + 1023) << 20, 0);
    return fma(scale, sg_fx_expm1(r), scale - 1.0);
}

// Per-point deviation (the "G" evaluation).
template <typename T, int GK> __device__ __forceinline__ T gdev(T S, T sphi, T cphi);
template <> __device__ __forceinline__ float gdev<float, SG_GK_EXPM1>(float S, float, float) {
    return sg_expm1f(S);
}
// Oscillatory: H is half the folded phase deviation; returns
// sin(H) sin(phi + H), and the factor -2 of
// cos(phi + 2H) - cos(phi) = -2 sin(H) sin(phi + H) sits in the weights.
template <> __device__ __forceinline__ float gdev<float, SG_GK_OSC>(float H, float sphi, float cphi) {
    float sh, ch;
    sincosf(H, &sh, &ch);
    return sh * fmaf(sphi, ch, cphi * sh);
}

// The FP64 deviation times a tail weight w: w expm1(S), or for the
// oscillatory kind w sin(H) sin(phi + H) (factor -2 in the prefix weights),
// in fixed point (one rounding) on |S| < ln2/2 and |H| < pi/4, through the
// double functions above otherwise.
template <int GK>
__device__ __forceinline__ double gdevw_d(double S, double w, double sphi, double cphi, const SgFxPhase &ph) {
    const int hx = __double2hiint(S) & 0x7fffffff;
    if constexpr (GK == SG_GK_EXPM1) {
        double v = sg_fx_expm1_w(S, w);
        if (hx >= 0x3fd62e42) v = sg_expm1_d(S) * w;
        return v;
    } else {
        double v = sg_fx_osc_dev_w(S, w, ph);
        if (hx >= 0x3fe921fb) {
            double sh, ch;
            sg_sincos_d(S, &sh, &ch);
            v = sh * fma(sphi, ch, cphi * sh) * w;
        }
        return v;
    }
}

// The same with the weight kept to 64 bits (merged form): the fixed-point
// product takes the whole significand; the paths through the double
// functions add the weight's low part with one more multiply-add.
template <int GK>
__device__ __forceinline__ double gdevw_dn(double S, const SgFxNorm &g, double sphi, double cphi,
                                           const SgFxPhase &ph) {
    const int hx = __double2hiint(S) & 0x7fffffff;
    if constexpr (GK == SG_GK_EXPM1) {
        double v = sg_fx_expm1_wn(S, g);
        if (hx >= 0x3fd62e42) {
            double whi, wlo;
            sg_fx_norm_split(g, &whi, &wlo);
            const double e = sg_expm1_d(S);
            v = fma(e, whi, e * wlo);
        }
        return v;
    } else {
        double v = sg_fx_osc_dev_wn(S, g, ph);
        if (hx >= 0x3fe921fb) {
            double sh, ch, whi, wlo;
            sg_sincos_d(S, &sh, &ch);
            sg_fx_norm_split(g, &whi, &wlo);
            const double t = sh * fma(sphi, ch, cphi * sh);
            v = fma(t, whi, t * wlo);
        }
        return v;
    }
}

// Float-float deviation (see sg_ff.cuh): expm1, or for the oscillatory kind
// sin(H) sin(phi + H) = sin(H) (sin(phi) cos(H) + cos(phi) sin(H)).
template <int GK> __device__ __forceinline__ ff2 gdev_ff(ff2 S, ff2 sphi, ff2 cphi) {
    if constexpr (GK == SG_GK_EXPM1) {
        return ff_expm1(S);
    } else {
        ff2 sh, ch;
        ff_sincos(S, &sh, &ch);
        return ff_mul(sh, ff_add(ff_mul(sphi, ch), ff_mul(cphi, sh)));
    }
}

// Weight factor of the deviation kind (see gdev).
template <int GK> __device__ __forceinline__ double gdev_weight() { return GK == SG_GK_OSC ? -2.0 : 1.0; }

// ---------------------------------------------------------------------------
// the fold: one chunk of one pattern, processed by one warp
// ---------------------------------------------------------------------------

// Error-free sum of two floats (Knuth's TwoSum): s + e == a + b exactly.
__device__ __forceinline__ void two_sum(float a, float b, float &s, float &e) {
    s = __fadd_rn(a, b);
    const float z = __fsub_rn(s, a);
    e = __fadd_rn(__fsub_rn(a, __fsub_rn(s, z)), __fsub_rn(b, z));
}

// Per-lane accumulators of a fold: a double for the FP64 path; for the mixed
// path a float pair (running sum + TwoSum error term) fed with plain float
// partial sums of 8 points, so that no double-precision instruction sits in
// the inner loop (GB300 runs FP64 at 1/72 of the FP32 rate, measured).
struct FoldAcc {
    double acc = 0.0;
    float hs = 0.f, hc = 0.f, habs = 0.f;
    ff2 fa = {0.f, 0.f};  // float-float path
    // FP64 merged path: an exact running sum in a 128-bit window whose unit
    // follows the largest term (sg_xsum.h).  The merged weights are large
    // and of both signs, and rounding a double running sum after each of
    // their terms costs digits the difference forms, with many more and
    // smaller terms, do not lose.
    SgX xa = {0ull, 0ull};
    int xe = 1;
};

// Prefix state of one prefix node tuple: partial argument S and weight W.
template <typename T> struct PrefixState;
template <> struct PrefixState<float> { typedef float2 type; };
template <> struct PrefixState<double> { typedef double2 type; };
template <> struct PrefixState<FFTag> { typedef float4 type; };

// Table entry of tail entry e: segment 1 holds e < E1, segment 2 the rest.
template <typename V2>
__device__ __forceinline__ V2 tail_entry(const V2 *__restrict__ tab, long long base1, int E1, long long base2,
                                         int e) {
    return tab[e < E1 ? base1 + e : base2 + (e - E1)];
}

// Weights of a merged-form pattern (SgFoldArgs::wtab + SgPatDev::woff): the
// point of prefix tuple a and tail node j has weight wt[a * tm + j].
struct SgMergedW {
    const void *wt;
    int tm;
    SgDivMagic dm;  // division by tm
};

// Folds the points (prefix tuple a < At) x (tail entries e < E1 + E2) of one
// run.  Tail entries come from up to two contiguous table segments (two
// when the enumerated directions jump over a left-out direction).  With MW
// (merged form) the weight of a point is read from the pattern's weight
// table (prefix tuple ab + a, tail node e mod tm) instead of being the
// product of the prefix and tail weights.
template <typename T, int GK, bool MW>
__device__ __forceinline__ void fold_run(const typename V2T<T>::type *__restrict__ tab,
                                         long long base1, int E1, long long base2, int E2,
                                         const typename PrefixState<T>::type *sP, int At, T sphi,
                                         T cphi, int lane, FoldAcc &F, const SgMergedW &M, int ab) {
    typedef typename V2T<T>::type V2;
    const int E = E1 + E2;
    if constexpr (sizeof(T) == 4) {
        // float (FP32 pipe, charged per warp instruction): lanes take tail
        // entries, each lane's entry stays in registers while it walks the
        // prefix tuples; a tail shorter than 32 splits the warp into groups
        // that take different tuples (SgLaneGroups).  Plain float partial
        // sums of 8 points feed the TwoSum accumulator.
        const SgLaneGroups g(lane, E);
        if (!g.active) return;
        float hs = F.hs, hc = F.hc, habs = F.habs;
        for (int e = g.e0; e < E; e += g.estep) {
            const V2 te = tab[e < E1 ? base1 + e : base2 + (e - E1)];
            // merged weights as float pairs: one weight serves every subset of
            // its pattern, so its rounding error would add up coherently; the
            // low part costs one more FMA per point
            const float2 *wrow = nullptr;
            if constexpr (MW) wrow = (const float2 *)M.wt + (e - sg_div_magic_q(e, M.dm) * M.tm) + (size_t)ab * M.tm;
            int a = g.a0;
            for (; a + 7 * g.astep < At; a += 8 * g.astep) {
                float part = 0.f;
#pragma unroll
                for (int u = 0; u < 8; u++) {
                    const float2 p = sP[a + u * g.astep];
                    const float D = gdev<float, GK>(p.x + te.x, sphi, cphi);
                    if constexpr (MW) {
                        const float2 w = __ldg(wrow + (size_t)(a + u * g.astep) * M.tm);
                        part = fmaf(w.x, D, fmaf(w.y, D, part));
                        habs = fmaf(fabsf(w.x), fabsf(D), habs);
                    } else {
                        const float W = p.y * te.y;
                        part = fmaf(W, D, part);
                        habs = fmaf(fabsf(W), fabsf(D), habs);
                    }
                }
                float t, err;
                two_sum(hs, part, t, err);
                hs = t;
                hc += err;
            }
            float part = 0.f;
            for (; a < At; a += g.astep) {
                const float2 p = sP[a];
                const float D = gdev<float, GK>(p.x + te.x, sphi, cphi);
                if constexpr (MW) {
                    const float2 w = __ldg(wrow + (size_t)a * M.tm);
                    part = fmaf(w.x, D, fmaf(w.y, D, part));
                    habs = fmaf(fabsf(w.x), fabsf(D), habs);
                } else {
                    const float W = p.y * te.y;
                    part = fmaf(W, D, part);
                    habs = fmaf(fabsf(W), fabsf(D), habs);
                }
            }
            float t, err;
            two_sum(hs, part, t, err);
            hs = t;
            hc += err;
        }
        F.hs = hs;
        F.hc = hc;
        F.habs = habs;
    } else {
        // FP64: the flat layout (idle lanes at the end of a run cost the FP64
        // pipe nothing on GB300; the lane groups measured no faster)
        SgFlatPos f(lane, E);
        double acc = F.acc;
        const SgFxPhase ph = sg_fx_phase(sphi, cphi);
        for (; f.a < At; f.step()) {
            const double2 p = sP[f.a];
            const V2 te = tail_entry(tab, base1, E1, base2, f.e);
            if constexpr (MW) {
                // the weight to 64 bits: it serves every subset of its pattern,
                // so its rounding error would add up coherently over them
                const int j = f.e - sg_div_magic_q(f.e, M.dm) * M.tm;
                const ulonglong2 w = __ldg((const ulonglong2 *)M.wt + (size_t)(ab + f.a) * M.tm + j);
                SgFxNorm g;  // SgW64: m, then e and neg in the second word
                g.m = w.x;
                g.e = (int)(unsigned)w.y;
                g.neg = w.y >> 32;
                sg_x_add_adaptive(F.xa, F.xe, gdevw_dn<GK>(p.x + te.x, g, sphi, cphi, ph));
            } else {
                acc = fma(p.y, gdevw_d<GK>(p.x + te.x, te.y, sphi, cphi, ph), acc);
            }
        }
        F.acc = acc;
    }
}

// Float-float fold of one run (same lane layout as fold_run).
template <int GK, bool MW>
__device__ __forceinline__ void fold_run_ff(const float4 *__restrict__ tab, long long base1, int E1,
                                            long long base2, int E2, const float4 *sP, int At, ff2 sphi,
                                            ff2 cphi, int lane, FoldAcc &F, const SgMergedW &M, int ab) {
    SgFlatPos f(lane, E1 + E2);
    ff2 fa = F.fa;
    float habs = F.habs;
    for (; f.a < At; f.step()) {
        const float4 p = sP[f.a];
        const float4 te = tail_entry(tab, base1, E1, base2, f.e);
        const ff2 S = ff_add(ff2{p.x, p.y}, ff2{te.x, te.y});
        ff2 W;
        if constexpr (MW) {
            const int j = f.e - sg_div_magic_q(f.e, M.dm) * M.tm;
            const float2 w = __ldg((const float2 *)M.wt + (size_t)(ab + f.a) * M.tm + j);
            W = ff2{w.x, w.y};
        } else {
            W = ff_mul(ff2{p.z, p.w}, ff2{te.z, te.w});
        }
        const ff2 D = gdev_ff<GK>(S, sphi, cphi);
        fa = ff_add(fa, ff_mul(W, D));
        habs = fmaf(fabsf(W.hi), fabsf(D.hi), habs);
    }
    F.fa = fa;
    F.habs = habs;
}

template <typename T, int GK, bool MW>
__device__ void fold_chunk(const SgFoldArgs &A, const SgPatDev *__restrict__ P,
                           const SgItemDev *__restrict__ I, unsigned long long c,
                           typename PrefixState<T>::type *sP, SgPrefixPos *sPos, int *sIdx, int lane,
                           FoldAcc &F,
                           bool &waited) {
    typedef typename V2T<T>::type V2;
    const V2 *__restrict__ tab = (const V2 *)A.tab + I->tab;
    const int d = I->d, r = P->r, skip = I->skip, tm = P->tm;
    unsigned long long rank, cnt;
    int a_lo, a_hi;
    sg_chunk_span(P, c, &rank, &cnt, &a_lo, &a_hi);
    if (A.chunk_start) {
        if (lane < r) sIdx[lane] = __ldg(&A.chunk_start[c].idx[lane]);
    } else {
        unrank_warp(rank, d, r, A.binom, sIdx, lane);
    }
    // everything above reads only the plan; the tables and item values come
    // from the setup kernel, which may still be finishing (programmatic
    // dependent launch).  One wait per warp suffices: once it returns the
    // setup kernel has finished.
    if (!waited) {
        cudaGridDependencySynchronize();
        waited = true;
    }
    // the prefix positions' block sizes and their division magics (per chunk)
    if (lane < r - 1) {
        const int m = P->pm[lane];
        sPos[lane].m = m;
        sPos[lane].dm = sg_div_magic(m);
    }
    __syncwarp();
    const SgItemVar *V = A.vars + (I - A.items);
    typedef typename std::conditional<std::is_same<T, FFTag>::value, float, T>::type TS;
    const TS sphi = (TS)V->sin_phi, cphi = (TS)V->cos_phi;
    const ff2 ffsphi = ff_from_double(V->sin_phi), ffcphi = ff_from_double(V->cos_phi);
    SgMergedW M;
    if constexpr (MW) {
        M.tm = tm;
        M.dm = sg_div_magic(tm);
        M.wt = sizeof(T) == 8 ? (const void *)((const SgW64 *)A.wtab + P->woff)
                              : (const void *)((const float2 *)A.wtab + P->woff);
    }
    while (cnt > 0) {
        const int plast = sIdx[r - 1];
        const int run = (unsigned long long)(d - plast) < cnt ? d - plast : (int)cnt;
        const SgTailSegs seg = sg_tail_segments(P->toff, tm, plast, run, skip);
        // this run's table rows of the prefix directions
        if (lane < r - 1) sPos[lane].row = P->poff[lane] + (long long)sg_actual_dir(sIdx[lane], skip) * sPos[lane].m;
        __syncwarp();
        for (int ab = a_lo; ab < a_hi; ab += SG_APAD) {
            const int At = a_hi - ab < SG_APAD ? a_hi - ab : SG_APAD;
            // fold the prefix directions: one state per prefix node tuple (its
            // digits in the mixed radix of the block sizes, the last fastest)
            // FP64, d > 32: the table rows of every position are first
            // requested into L1 (prefetches carry no data, so they are all in
            // flight at once).  Large tables are read mostly once per SM, and
            // one latency per prefix instead of one per position took a
            // d = 100 integral from 45 to 38 us; small tables stay in L1 and
            // float folds are issue-bound, and there the extra pass costs
            // (d = 12: 25 -> 29 us; a float batch: +10%).
            if constexpr (std::is_same<T, double>::value) {
                if (d > 32) {
                    for (int a = lane; a < At; a += 32) {
                        int q = ab + a;
                        for (int t = r - 2; t >= 0; t--) {
                            const SgPrefixPos pp = sPos[t];
                            const int qn = sg_div_magic_q(q, pp.dm);
                            asm volatile("prefetch.global.L1 [%0];" ::"l"(tab + pp.row + (q - qn * pp.m)));
                            q = qn;
                        }
                    }
                }
            }
            for (int a = lane; a < At; a += 32) {
                int q = ab + a;
                if constexpr (std::is_same<T, FFTag>::value) {  // float-float
                    ff2 S = {0.f, 0.f}, W = {(float)gdev_weight<GK>(), 0.f};
                    for (int t = r - 2; t >= 0; t--) {
                        const SgPrefixPos pp = sPos[t];
                        const int qn = sg_div_magic_q(q, pp.dm);
                        const V2 e = tab[pp.row + (q - qn * pp.m)];
                        q = qn;
                        S = ff_add(S, ff2{e.x, e.y});
                        if constexpr (!MW) W = ff_mul(W, ff2{e.z, e.w});
                    }
                    sP[a] = make_float4(S.hi, S.lo, W.hi, W.lo);
                } else {
                    T S = 0, W = (T)gdev_weight<GK>();
                    for (int t = r - 2; t >= 0; t--) {
                        const SgPrefixPos pp = sPos[t];
                        const int qn = sg_div_magic_q(q, pp.dm);
                        const V2 e = tab[pp.row + (q - qn * pp.m)];
                        q = qn;
                        S += e.x;
                        if constexpr (!MW) W *= e.y;
                    }
                    sP[a].x = S;
                    sP[a].y = W;
                }
            }
            __syncwarp();
            if constexpr (std::is_same<T, FFTag>::value)
                fold_run_ff<GK, MW>(tab, seg.base1, seg.E1, seg.base2, seg.E2, sP, At, ffsphi, ffcphi, lane, F,
                                    M, ab);
            else
                fold_run<T, GK, MW>(tab, seg.base1, seg.E1, seg.base2, seg.E2, sP, At, sphi, cphi, lane, F, M,
                                    ab);
            __syncwarp();
        }
        cnt -= run;
        if (cnt > 0) {
            if (lane == 0) sg_next_prefix(sIdx, d, r);
            __syncwarp();
        }
    }
}

// The value of a long accumulator held one limb per lane, as s + c, by
// the warp: one carry step brings every limb below 2^53 so that
// limb * 2^(32 lane + SG_LA_E0) is an exact double, and those 32 doubles are
// added exactly in a 128-bit window (sg_xsum.h; terms more than 104 bits
// below the largest are cut towards zero, the same on every run).
__device__ __forceinline__ void la_warp_round(long long L, int lane, double &s, double &c) {
    const long long hi = L >> 32;  // arithmetic: floor division by 2^32
    const long long up = __shfl_up_sync(FULL_MASK, hi, 1);
    long long v = lane == 31 ? L : (long long)((unsigned long long)L & 0xffffffffull);
    if (lane > 0) v += up;
    const double t = (double)v * sg_xs_double((unsigned long long)(32 * lane + SG_LA_E0 + 1023) << 52);
    const int E = warp_max_exp(sg_x_exp(t));
    SgX a = {0ull, 0ull};
    sg_x_add(a, t, E);
    warp_xsum(a, E, s, c);
}

// End of a single-integral fold (SgFoldArgs::single): the CTA adds the
// non-zero limbs of its long accumulator into the launch's accumulator with
// integer atomics (the order of the additions cannot change the sum, so the
// result does not depend on which CTA ran which chunk); the last CTA to
// finish rounds it, assembles the output record and returns the launch's
// accumulator and counters to zero for the next launch.  Everything here is
// latency on the path of every call: the sum and the absolute sum are
// rounded by two warps side by side, and the values the assembly needs are
// loaded while they do.
__device__ __noinline__ void finish_single(const SgFoldArgs &A, long long *s_la, int *s_flag, double *s_r) {
    const int NL = 2 * SG_LA_DIGITS;
    __syncthreads();
    for (int k = threadIdx.x; k < NL; k += blockDim.x) {
        const long long v = s_la[k];
        if (v) atomicAdd((unsigned long long *)&A.lacc[k], (unsigned long long)v);
    }
    if (threadIdx.x == 0 && s_flag[0]) atomicOr(A.cta_done + 1, 1u);
    __threadfence();  // this CTA's additions before its count (one fence serves both)
    __syncthreads();
    // the values the assembly needs (from the setup kernel; one item, integral
    // 0), requested by every CTA's thread 0 together with its count, so that
    // the last CTA has them when its sums are rounded
    SgItemVar V;
    SgBaseDev B;
    long long oi = 0;
    const int g = 0;
    if (threadIdx.x == 0) {
        cudaGridDependencySynchronize();
        V = A.vars[0];
        B = A.bases[0];
        oi = A.items[0].out;
        s_flag[1] = atomicAdd(A.cta_done, 1u) == gridDim.x - 1;
    }
    __syncthreads();
    // two warps: warp 0 holds the sum's limbs, warp 1 the absolute sum's (a
    // one-warp CTA rounds both in turn)
    const bool two = blockDim.x >= 64;
    if (!s_flag[1] || (int)threadIdx.x >= (two ? NL : 32)) return;
    __threadfence();
    const int lane = threadIdx.x & 31;
    const long long L = __ldcg(A.lacc + threadIdx.x);
    A.lacc[threadIdx.x] = 0;
    long long La = 0;
    if (!two) {
        La = __ldcg(A.lacc + SG_LA_DIGITS + lane);
        A.lacc[SG_LA_DIGITS + lane] = 0;
    }
    bool ovf = false;
    if (threadIdx.x == 0) ovf = __ldcg(A.cta_done + 1) != 0u;
    double s, c;
    la_warp_round(L, lane, s, c);
    if (two) {
        if (threadIdx.x == 32) s_r[0] = s + c;
        asm volatile("bar.sync 1, 64;" ::: "memory");  // the two rounding warps
    } else {
        double as, ac;
        la_warp_round(La, lane, as, ac);
        if (threadIdx.x == 0) s_r[0] = as + ac;
    }
    if (threadIdx.x == 0) {
        const double T = ovf ? __longlong_as_double(0x7ff8000000000000ll) : s + c;
        assemble_values(V, B, g, oi, A.out, A.vout, A.flags, A.guard_tol, A.unit_roundoff, 0, T, s_r[0]);
        *A.work = 0ull;
        A.cta_done[0] = 0u;
        A.cta_done[1] = 0u;
    }
}

// A finished chunk of a batch item (SgFoldArgs::ilacc): lane k adds digit k
// of the chunk's sum (d1) and absolute sum (d2) into the item's long
// accumulator with integer atomics (a few lanes of each are non-zero), then
// the chunk counts itself; the warp that counts the item's last chunk
// rounds the accumulator and assembles the item.  Integer additions in any
// order give the same limbs, so the result does not depend on which warp
// ran which chunk, nor on how the chunks were split over launches (shards).
__device__ __noinline__ void complete_chunk_item(const SgFoldArgs &A, int item, long long d1, long long d2,
                                                 int ovf, int lane) {
    long long *L = A.ilacc + (size_t)item * 2 * SG_LA_DIGITS;
    // a term outside the window (or not finite) marks the absolute sum, which
    // is otherwise never negative; the item then assembles as NaN
    if (__any_sync(FULL_MASK, ovf) && lane == 0)
        atomicAdd((unsigned long long *)&L[2 * SG_LA_DIGITS - 1], (unsigned long long)(-(1ll << 40)));
    if (d1) atomicAdd((unsigned long long *)&L[lane], (unsigned long long)d1);
    if (d2) atomicAdd((unsigned long long *)&L[SG_LA_DIGITS + lane], (unsigned long long)d2);
    if (A.no_assemble) return;
    __threadfence();
    __syncwarp();
    unsigned int ticket = 0;
    if (lane == 0) ticket = ticket_add(A.item_done + item);
    ticket = __shfl_sync(FULL_MASK, ticket, 0);
    const SgItemDev *I = A.items + item;
    if (ticket + 1ull != I->nchunk) return;
    __syncwarp();
    const long long Ls = __ldcg(L + lane), La = __ldcg(L + SG_LA_DIGITS + lane);
    double s, c, as, ac;
    la_warp_round(Ls, lane, s, c);
    la_warp_round(La, lane, as, ac);
    if (lane == 0) {
        const double T = as + ac < 0.0 ? __longlong_as_double(0x7ff8000000000000ll) : s + c;
        assemble_item(A.items, A.vars, A.bases, A.item_integral, A.out, A.vout, A.flags, A.guard_tol,
                      A.unit_roundoff, item, T, as + ac);
    }
}

template <typename T>
__device__ __forceinline__ void fold_kernel_body(const SgFoldArgs &A) {
    typedef typename PrefixState<T>::type PS;
    extern __shared__ __align__(16) unsigned char smem[];
    __shared__ long long s_la[2 * SG_LA_DIGITS];
    __shared__ int s_flag[2];
    __shared__ double s_r[1];
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    PS *sP = (PS *)smem + (size_t)warp * SG_APAD;
    SgPrefixPos *sPos = (SgPrefixPos *)(smem + (size_t)nw * SG_APAD * sizeof(PS)) + warp * SG_MAX_R;
    int *sIdx = (int *)(smem + (size_t)nw * (SG_APAD * sizeof(PS) + SG_MAX_R * sizeof(SgPrefixPos))) + warp * SG_MAX_R;
    bool waited = false;
    if (A.single) {
        for (int k = threadIdx.x; k < 2 * SG_LA_DIGITS; k += blockDim.x) s_la[k] = 0;
        if (threadIdx.x == 0) s_flag[0] = 0;
        __syncthreads();
    }
    const unsigned long long c_end = A.chunk_hi ? A.chunk_hi : A.nchunks;
    // the first chunk of every warp is fixed (no atomic at the start, where all
    // warps would contend for the counter at once; consecutive chunks, often
    // alike in cost, go to different SMs); the later ones come from the counter
    bool first = true;
    for (;;) {
        unsigned long long c = 0;
        if (first) {
            c = A.chunk_lo + (unsigned long long)warp * gridDim.x + blockIdx.x;
        } else {
            if (lane == 0) c = A.chunk_lo + (unsigned long long)gridDim.x * nw + atomicAdd(A.work, 1ull);
            c = __shfl_sync(FULL_MASK, c, 0);
        }
        first = false;
        if (c >= c_end) break;
        // pattern of chunk c: last pattern with chunk0 <= c
        long long lo = 0, hi = A.npat - 1;
        if (A.chunk_start) {
            lo = __ldg(&A.chunk_start[c].pat);
        } else {
            while (lo < hi) {
                long long mid = (lo + hi + 1) >> 1;
                if (__ldg(A.pat_chunk0 + mid) <= c) lo = mid;
                else hi = mid - 1;
            }
        }
        const SgPatDev *P = A.pats + lo;
        const int item = P->item;
        if (A.skip_unflagged && !A.flags[item]) continue;
        const SgItemDev *I = A.items + item;
        FoldAcc F;
        if (P->woff >= 0 && A.wtab) {
            if (I->gk == SG_GK_OSC) fold_chunk<T, SG_GK_OSC, true>(A, P, I, c, sP, sPos, sIdx, lane, F, waited);
            else fold_chunk<T, SG_GK_EXPM1, true>(A, P, I, c, sP, sPos, sIdx, lane, F, waited);
        } else {
            if (I->gk == SG_GK_OSC) fold_chunk<T, SG_GK_OSC, false>(A, P, I, c, sP, sPos, sIdx, lane, F, waited);
            else fold_chunk<T, SG_GK_EXPM1, false>(A, P, I, c, sP, sPos, sIdx, lane, F, waited);
        }
        const double cf = P->coef;  // 1 for most patterns
        if ((A.single || A.ilacc) && cf == 1.0) {
            // the chunk's exact sum over the lanes (a 128-bit integer window,
            // sg_xsum.h) and its absolute sum enter the long accumulators
            // digit by digit: integer operations only, no rounding to doubles
            SgX xs = {0ull, 0ull}, xm = {0ull, 0ull};
            int Es, Em;
            if constexpr (std::is_same<T, double>::value) {
                if (P->woff >= 0 && A.wtab) {
                    Es = warp_max_exp(F.xe);
                    xs = F.xa;
                    sg_x_shr(xs, Es - F.xe);
                } else {
                    Es = warp_max_exp(sg_x_exp(F.acc));
                    sg_x_add(xs, F.acc, Es);
                }
                Em = Es;  // the FP64 fold skips |W D| per point: the chunk's |sum| stands in
            } else {
                const double v = std::is_same<T, float>::value ? (double)F.hs + (double)F.hc : ff_to_double(F.fa);
                Es = warp_max_exp(sg_x_exp(v));
                sg_x_add(xs, v, Es);
                Em = warp_max_exp(sg_x_exp((double)F.habs));
                sg_x_add(xm, (double)F.habs, Em);
            }
            warp_xadd(xs);
            int ovf = 0;
            long long m = 0;
            const long long d1 = sg_la_x_digit(xs, Es, lane, &ovf, &m);
            long long d2 = m;
            if constexpr (!std::is_same<T, double>::value) {
                warp_xadd(xm);
                sg_la_x_digit(xm, Em, lane, &ovf, &m);
                d2 = m;
            }
            if (A.single) {
                // lane k adds digit k into the CTA's long accumulator (no two
                // lanes share a limb)
                if (d1) atomicAdd((unsigned long long *)&s_la[lane], (unsigned long long)d1);
                if (d2) atomicAdd((unsigned long long *)&s_la[SG_LA_DIGITS + lane], (unsigned long long)d2);
                if (ovf) s_flag[0] = 1;
            } else {
                complete_chunk_item(A, item, d1, d2, ovf, lane);
            }
            continue;
        }
        // other coefficients (the combination form's binomials) and the
        // chunk-slot reduction: the chunk's sum over the lanes, exact before
        // one rounding
        double acc, aabs, acc_lo = 0.0;
        if constexpr (std::is_same<T, double>::value) {
            // the FP64 fold skips |W D| per point: the chunk's |sum| stands in
            if (P->woff >= 0 && A.wtab) {
                // merged: the lanes' exact sums, aligned and added exactly, kept as
                // a pair of doubles
                const int E = warp_max_exp(F.xe);
                sg_x_shr(F.xa, E - F.xe);
                warp_xsum(F.xa, E, acc, acc_lo);
            } else {
                acc = warp_sum(F.acc);
            }
            aabs = fabs(acc);
        } else {
            acc = warp_sum(std::is_same<T, float>::value ? (double)F.hs + (double)F.hc : ff_to_double(F.fa));
            aabs = warp_sum((double)F.habs);
        }
        const double vsum = cf == 1.0 ? acc : acc * cf, vabs = cf == 1.0 ? aabs : aabs * fabs(cf);
        const double vlo = cf == 1.0 ? acc_lo : acc_lo * cf;
        if (A.single || A.ilacc) {
            // lane k's digit of the chunk's sum (both parts) and absolute sum
            // (at most three lanes of each are non-zero)
            int ovf = 0;
            const long long d1 = sg_la_digit(vsum, lane, &ovf) + sg_la_digit(vlo, lane, &ovf);
            const long long d2 = sg_la_digit(vabs, lane, &ovf);
            if (A.single) {
                if (d1) atomicAdd((unsigned long long *)&s_la[lane], (unsigned long long)d1);
                if (d2) atomicAdd((unsigned long long *)&s_la[SG_LA_DIGITS + lane], (unsigned long long)d2);
                if (ovf) s_flag[0] = 1;
            } else {
                complete_chunk_item(A, item, d1, d2, ovf, lane);
            }
            continue;
        }
        if (lane == 0) {
            SgSlot sl;
            sl.sum = vsum;
            sl.abs = vabs;
            sl.lo = acc_lo;
            sl.pad = 0.0;
            A.slots[c] = sl;
        }
        complete_chunk(A, item, c, lane);
    }
    if (A.single) finish_single(A, s_la, s_flag, s_r);
}

// Float fold: register budget for 4 CTAs of 8 warps per SM.  Double fold,
// two builds: without a register budget (84 registers, 2 CTAs of 8 warps
// per SM) for single integrals, and with one for 3 CTAs per SM (80
// registers, a few bytes spilled) for batches, whose throughput gains 10 -
// 13% from the extra warps covering the dependent integer chains of the
// fixed-point deviation; on single integrals of d = 100 and 1000 the spill
// cost 25% (measured on GB300).
__global__ void __launch_bounds__(256, 4) sg_fold_kernel_f(SgFoldArgs A) { fold_kernel_body<float>(A); }
__global__ void sg_fold_kernel_d(SgFoldArgs A) { fold_kernel_body<double>(A); }
__global__ void __launch_bounds__(256, 3) sg_fold_kernel_d3(SgFoldArgs A) { fold_kernel_body<double>(A); }
__global__ void __launch_bounds__(256, 2) sg_fold_kernel_x(SgFoldArgs A) { fold_kernel_body<FFTag>(A); }

// ---------------------------------------------------------------------------
// setup: per-integral base quantities and the (phi, w) tables
// ---------------------------------------------------------------------------

// Per-call item values: the oscillatory phase of the per-point deviation and
// the centre term, from the integral's centre phase theta_c (or log f(c)).
__device__ __forceinline__ SgItemVar item_values(const SgItemRole &R, const SgIntegralDev &G,
                                                 const SgBaseDev &B, const double *params) {
    SgItemVar V;
    double sn = B.sin_th, cs = B.cos_th;
    if (R.role != SG_ROLE_FORWARD && G.fam == 1) {  // advance the phase by pi/2
        const double t = sn;
        sn = cs;
        cs = -t;
    }
    double shift = 0.0;
    if (R.role == SG_ROLE_ADJOINT) {
        const double *p = params + G.param_off;
        shift = phi_dev(G.fam, p[R.dir], p[G.d + R.dir], R.x);
    }
    if (G.fam == 1) {
        // phase theta + shift: rotate (sin, cos) by the shift
        double ss = 0.0, cc = 1.0;
        if (shift != 0.0) sincos(shift, &ss, &cc);
        V.sin_phi = sn * cc + cs * ss;
        V.cos_phi = cs * cc - sn * ss;
        V.base_rel = V.cos_phi;
        V.mult = 1.0;
    } else {
        V.sin_phi = 0.0;
        V.cos_phi = 1.0;
        V.base_rel = 1.0;
        V.mult = shift != 0.0 ? exp(shift) : 1.0;
    }
    return V;
}

// Blocks [0, nbase) compute one integral each: log f(c), or the oscillatory
// centre phase, as an exact sum in a 128-bit window (see below).  A
// whole block per integral spreads a long sum over the SM's four FP64
// units.  The remaining blocks fill table entries.
__global__ void __launch_bounds__(256) sg_setup_kernel(SgSetupArgs A, int nbase) {
    // let a fold launched as a programmatic dependent start its plan-only work
    cudaTriggerProgrammaticLaunchCompletion();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    if ((int)blockIdx.x < nbase) {
        __shared__ SgX sh_x[8];
        __shared__ int sh_e[8];
        __shared__ SgBaseDev sh_b;
        const int g = blockIdx.x;
        const SgIntegralDev G = A.integrals[g];
        const double *a = A.params + G.param_off, *u = a + G.d;
        // each thread's first item, loaded now so that the dependent loads
        // overlap the centre sum instead of following it
        const int ti0 = A.do_items ? A.int_item_ptr[g] : 0, ti1 = A.do_items ? A.int_item_ptr[g + 1] : 0;
        int it0 = -1;
        SgItemRole role0;
        unsigned long long nch0 = 1;
        if (ti0 + (int)threadIdx.x < ti1) {
            it0 = A.int_items[ti0 + threadIdx.x];
            role0 = A.roles[it0];
            nch0 = A.items[it0].nchunk;
        }
        // log f(c) (or the centre phase) as an exact sum in a 128-bit window
        // (sg_xsum.h): each thread keeps a running sum of its terms, whose
        // unit follows the largest term so far; the block then aligns the
        // threads' sums to the largest unit and adds them as integers.  The
        // result is the same on every call, and no FP64 operation sits in a
        // dependency chain (on GB300 each would cost ~10^2 cycles).
        // Up to 32 terms take one warp and no block barriers (every step
        // here is latency on the path of a single integral; longer sums are
        // faster spread over the block).
        const bool one_warp = G.d <= 32;
        if (one_warp && warp > 0 && !(A.do_items && ti1 - ti0 > 1)) return;
        SgX acc = {0ull, 0ull};
        int E = 1;
        if (G.fam != SG_FAM_USER && (!one_warp || warp == 0))  // a user integrand's parameters have no fixed layout
            for (int i = one_warp ? lane : (int)threadIdx.x; i < G.d; i += one_warp ? 32 : (int)blockDim.x)
                sg_x_add_adaptive(acc, E, phi_centre(G.fam, a[i], u[i]));
        int Eb = warp_max_exp(E);
        if (!one_warp) {
            if (lane == 0) sh_e[warp] = Eb;
            __syncthreads();
            Eb = sh_e[0];
            for (int w = 1; w < nw; w++) Eb = max(Eb, sh_e[w]);
        }
        sg_x_shr(acc, Eb - E);
        warp_xadd(acc);
        if (!one_warp) {
            if (lane == 0) sh_x[warp] = acc;
            __syncthreads();
        }
        if (threadIdx.x == 0) {
            SgX t = acc;
            if (!one_warp) {
                t = sh_x[0];
                for (int w = 1; w < nw; w++) sg_x_plus(t, sh_x[w]);
            }
            double s, c;
            sg_x_pair(t, Eb, &s, &c);
            SgBaseDev B;
            if (G.fam == 1) {
                B.log_hi = 0.0;
                B.log_lo = 0.0;
                sg_sincos_d(6.28318530717958647693 * u[0] + (s + c), &B.sin_th, &B.cos_th);
                B.base = B.cos_th;
            } else {
                B.log_hi = s;
                B.log_lo = c;
                B.base = 1.0;
                B.sin_th = 0.0;
                B.cos_th = 1.0;
            }
            // exp(log_hi + log_lo) = 2^e0 exp(r), r = log_hi - e0 ln 2 + log_lo with
            // ln 2 split in two (Cody & Waite): the result's scale without overflow
            // (1 for the oscillatory family, whose values are not scaled)
            if (B.log_hi == 0.0 && B.log_lo == 0.0) {
                B.scale_e2 = 0.0;
                B.scale_m = 1.0;
            } else {
                const double ln2_hi = 6.93147180369123816490e-01, ln2_lo = 1.90821492927058770002e-10;
                const double e0 = floor(B.log_hi * 1.44269504088896338700);
                const double rr = ((B.log_hi - e0 * ln2_hi) - e0 * ln2_lo) + B.log_lo;
                B.scale_e2 = e0;
                B.scale_m = 1.0 + sg_expm1_d(rr);
            }
            A.bases[g] = B;
            sh_b = B;
            if (A.do_items && ti1 - ti0 == 1) {
                // one item (a single forward integral): its values right away
                A.vars[it0] = item_values(role0, G, B, A.params);
                if (nch0 == 0)
                    assemble_item(A.items, A.vars, A.bases, A.item_integral, A.out, A.vout, nullptr, 0.0,
                                  A.unit_roundoff, it0, 0.0, 0.0);
            }
        }
        if (!A.do_items || ti1 - ti0 == 1) return;
        __syncthreads();
        const SgBaseDev B = sh_b;
        for (int t = ti0 + threadIdx.x; t < ti1; t += blockDim.x) {
            const bool first = t == ti0 + (int)threadIdx.x;
            const int it = first ? it0 : A.int_items[t];
            A.vars[it] = item_values(first ? role0 : A.roles[it], G, B, A.params);
            if ((first ? nch0 : A.items[it].nchunk) == 0)
                assemble_item(A.items, A.vars, A.bases, A.item_integral, A.out, A.vout, nullptr, 0.0,
                              A.unit_roundoff, it, 0.0, 0.0);
        }
        return;
    }
    const long long stride = (long long)(gridDim.x - nbase) * blockDim.x;
    for (long long e = (long long)(blockIdx.x - nbase) * blockDim.x + threadIdx.x; e < A.nentries;
         e += stride) {
        int lo = 0, hi = A.nblocks - 1;  // first block whose end > e
        SgBlockDev B;
        long long local;
        if (A.ninline) {  // descriptors in the kernel parameters: no dependent loads
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (A.end_inline[mid] > e) hi = mid;
                else lo = mid + 1;
            }
            B = A.blk_inline[lo];
            local = e - (lo ? A.end_inline[lo - 1] : 0);
        } else {
            while (lo < hi) {
                const int mid = (lo + hi) >> 1;
                if (__ldg(A.block_end + mid) > e) hi = mid;
                else lo = mid + 1;
            }
            B = A.blocks[lo];
            local = e - (lo ? __ldg(A.block_end + lo - 1) : 0);
        }
        const SgIntegralDev G = A.integrals[B.integral];
        if (A.flags && G.flag_item >= 0 && !A.flags[G.flag_item]) continue;
        const int i = (int)(local / B.m), j = (int)(local - (long long)i * B.m);
        const double2 xw = B.xw[j];
        const double *p = A.params + G.param_off;
        const double phi = G.fam == SG_FAM_USER ? xw.x : phi_table(G.fam, p[i], p[G.d + i], xw.x);
        if (A.tab64) A.tab64[B.off + local] = make_double2(phi, xw.y);
        if (A.tab32) A.tab32[B.off + local] = make_float2((float)phi, (float)xw.y);
        if (A.tabff) {
            const ff2 fp = ff_from_double(phi), fw = ff_from_double(xw.y);
            A.tabff[B.off + local] = make_float4(fp.hi, fp.lo, fw.hi, fw.lo);
        }
    }
}

// One thread per chunk: its pattern (last pattern whose first chunk is <= c)
// and the first subset of its span, unranked (lexicographic order).
__global__ void sg_chunk_start_kernel(const SgItemDev *items, const SgPatDev *pats,
                                      const unsigned long long *pat_chunk0, long long npat,
                                      unsigned long long nchunks, const unsigned long long *binom,
                                      SgChunkStart *out) {
    for (unsigned long long c = (unsigned long long)blockIdx.x * blockDim.x + threadIdx.x; c < nchunks;
         c += (unsigned long long)gridDim.x * blockDim.x) {
        long long lo = 0, hi = npat - 1;
        while (lo < hi) {
            const long long mid = (lo + hi + 1) >> 1;
            if (pat_chunk0[mid] <= c) lo = mid;
            else hi = mid - 1;
        }
        const SgPatDev *P = pats + lo;
        unsigned long long rank, cnt;
        int a_lo, a_hi, idx[SG_MAX_R];
        sg_chunk_span(P, c, &rank, &cnt, &a_lo, &a_hi);
        sg_unrank_lex(rank, items[P->item].d, P->r, binom, idx);
        SgChunkStart cs;
        cs.pat = (int)lo;
        for (int t = 0; t < SG_MAX_R; t++) cs.idx[t] = (unsigned short)(t < P->r ? idx[t] : 0);
        cs.pad = 0;
        out[c] = cs;
    }
}

cudaError_t sg_launch_chunk_starts(const SgItemDev *items, const SgPatDev *pats, const unsigned long long *pat_chunk0,
                                   long long npat, unsigned long long nchunks, const unsigned long long *binom,
                                   SgChunkStart *out, cudaStream_t s) {
    if (nchunks == 0) return cudaSuccess;
    const unsigned long long blocks = (nchunks + 255) / 256 < 4096 ? (nchunks + 255) / 256 : 4096;
    sg_chunk_start_kernel<<<(unsigned)blocks, 256, 0, s>>>(items, pats, pat_chunk0, npat, nchunks, binom, out);
    return cudaGetLastError();
}

__global__ void sg_prep_kernel(SgPrepArgs A) {
    const int it = blockIdx.x * blockDim.x + threadIdx.x;
    if (it >= A.nitems) return;
    const SgItemRole R = A.roles[it];
    A.vars[it] = item_values(R, A.integrals[R.integral], A.bases[R.integral], A.params);
    if (A.items[it].nchunk == 0)
        assemble_item(A.items, A.vars, A.bases, A.item_integral, A.out, A.vout, A.flags, 0.0,
                      A.unit_roundoff, it, 0.0, 0.0);
}

// ---------------------------------------------------------------------------
// adjoint assembly: one thread per parameter
// ---------------------------------------------------------------------------

// dQ/dtheta = sum_p W_p h(x_p), h = g(x_i) F_h(x_p) with F_h = f (exponential
// families) or cos(phase + pi/2) (oscillatory, d/da_i).  Splitting
// g(x_i) = g(c) + (g(x_i) - g(c)):
//   dQ/dtheta / scale = g(c) Q_h/scale
//        + sum_{k, j} dw_{k,j} (g(x_j) - g(c)) V_{i,k,j},
// where V_{i,k,j} is the Smolyak sum over the other directions (budget
// L - k) with direction i at node j of the level-(k+1) difference rule,
// computed by the fold kernel as adjoint sub-sums.
__device__ __forceinline__ void grad_factor(int fam, bool is_u, double a, double u, double x,
                                            double *g) {
    switch (fam) {
    case 0:
        *g = is_u ? 0.0 : x;
        return;
    case 1:
        *g = is_u ? 0.0 : x;
        return;
    case 2: {
        const double den = 1.0 / (a * a) + (x - u) * (x - u);
        *g = is_u ? 2.0 * (x - u) / den : 2.0 / (a * a * a) / den;
        return;
    }
    case 3:
        *g = is_u ? 2.0 * a * a * (x - u) : -2.0 * a * (x - u) * (x - u);
        return;
    case 4:
        *g = is_u ? 2.0 * a * (x - u) : -(x - u) * (x - u);
        return;
    }
    *g = 0.0;
}

__global__ void sg_grad_kernel(SgGradArgs A) {
    const int j = blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= 2 * A.d) return;
    const bool is_u = j >= A.d;
    const int i = is_u ? j - A.d : j;
    const double a = A.params[i], u = A.params[A.d + i];
    if (A.fam == 1 && is_u) {  // oscillatory: only u_0 matters, d/du_0 = 2 pi Q_h
        A.grad_rel[j] = (i == 0) ? 6.28318530717958647693 * A.qh->sum : 0.0;
        return;
    }
    if (A.fam == 0 && is_u) {
        A.grad_rel[j] = 0.0;
        return;
    }
    const double qrel = (A.fam == 1) ? A.qh->sum : A.q->sum;
    double gc;
    grad_factor(A.fam, is_u, a, u, 0.5, &gc);
    double s = 0.0, c = 0.0;
    neu_add(s, c, gc * qrel);
    const double *v = A.v + (size_t)i * A.vstride;
    int col = 0;
    for (int k = 1; k <= A.L; k++) {
        const double2 *xw = A.delta_xw + A.delta_off[k];
        for (int jn = 0; jn < A.delta_m[k]; jn++, col++) {
            double gx;
            grad_factor(A.fam, is_u, a, u, xw[jn].x, &gx);
            neu_add(s, c, xw[jn].y * (gx - gc) * v[col]);
        }
    }
    A.grad_rel[j] = s + c;
}

// ---------------------------------------------------------------------------
// launch wrappers
// ---------------------------------------------------------------------------

cudaError_t sg_launch_setup(const SgSetupArgs &a, cudaStream_t s) {
    const int threads = 256;
    const int nbase = a.nintegrals;  // one block per integral
    long long eblocks = (a.nentries + threads - 1) / threads;
    if (eblocks > 152 * 16) eblocks = 152 * 16;
    if (eblocks < 1) eblocks = 1;
    sg_setup_kernel<<<(unsigned)(nbase + eblocks), threads, 0, s>>>(a, nbase);
    return cudaGetLastError();
}

// prec: 0 FP64 (single-integral build), 1 float, 2 float-float, 3 FP64
// (batch build, 3 CTAs per SM)
static size_t fold_smem(int prec, int warps) {
    const size_t psz = prec == 1 ? sizeof(float2) : (prec == 2 ? sizeof(float4) : sizeof(double2));
    return (size_t)warps * (SG_APAD * psz + SG_MAX_R * (sizeof(SgPrefixPos) + sizeof(int)));
}

int sg_fold_occupancy(int prec, int gk, int warps_per_cta) {
    (void)gk;
    int n = 0;
    const size_t sm = fold_smem(prec, warps_per_cta);
    if (prec == 2)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sg_fold_kernel_x, 32 * warps_per_cta, sm);
    else if (prec == 1)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sg_fold_kernel_f, 32 * warps_per_cta, sm);
    else if (prec == 3)
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sg_fold_kernel_d3, 32 * warps_per_cta, sm);
    else
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&n, sg_fold_kernel_d, 32 * warps_per_cta, sm);
    return n;
}

cudaError_t sg_launch_fold(const SgFoldArgs &a, int prec, int gk, SgLaunchCfg cfg, cudaStream_t s) {
    (void)gk;
    const size_t sm = fold_smem(prec, cfg.warps_per_cta);
    // programmatic dependent launch: the fold may begin while the preceding
    // kernel in the stream finishes; it waits (cudaGridDependencySynchronize)
    // before it reads that kernel's output
    cudaLaunchConfig_t lc = {};
    lc.gridDim = dim3(cfg.ctas);
    lc.blockDim = dim3(32 * cfg.warps_per_cta);
    lc.dynamicSmemBytes = sm;
    lc.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    lc.attrs = attr;
    lc.numAttrs = cfg.dependent ? 1 : 0;
    if (prec == 2) return cudaLaunchKernelEx(&lc, sg_fold_kernel_x, a);
    if (prec == 1) return cudaLaunchKernelEx(&lc, sg_fold_kernel_f, a);
    if (prec == 3) return cudaLaunchKernelEx(&lc, sg_fold_kernel_d3, a);
    return cudaLaunchKernelEx(&lc, sg_fold_kernel_d, a);
}

cudaError_t sg_launch_prep(const SgPrepArgs &a, cudaStream_t s) {
    const int threads = 128;
    sg_prep_kernel<<<(a.nitems + threads - 1) / threads, threads, 0, s>>>(a);
    return cudaGetLastError();
}

cudaError_t sg_launch_grad(const SgGradArgs &a, cudaStream_t s) {
    const int threads = 128;
    const int blocks = (2 * a.d + threads - 1) / threads;
    sg_grad_kernel<<<blocks, threads, 0, s>>>(a);
    return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// ceiling microbenchmarks
// ---------------------------------------------------------------------------

// The fold's inner loop on register-resident data: 8 tail entries per
// thread, an argument drifting per sweep so nothing can be hoisted.
template <typename T, int GK>
__global__ void __launch_bounds__(256) sg_ceiling_kernel(int sweeps, double *out) {
    T dl[8], wl[8];
#pragma unroll
    for (int k = 0; k < 8; k++) {
        dl[k] = (T)((k - 3.5) * 0.05 + threadIdx.x * 1e-5);
        wl[k] = (T)((k & 1) ? -0.25 : 0.3);
    }
    T S = (T)(blockIdx.x * 1e-6), W = (T)0.7;
    const T sphi = (T)0.3, cphi = (T)0.95;
    const SgFxPhase ph = sg_fx_phase(0.3, 0.95);
    double acc = 0.0, aabs = 0.0;
    float hs = 0.f, hc = 0.f, habs = 0.f;
    for (int it = 0; it < sweeps; it++) {
        if constexpr (sizeof(T) == 4) {
#pragma unroll
            for (int k = 0; k < 8; k++) {
                const float s = S + dl[k], w = W * wl[k];
                const float D = gdev<float, GK>(s, sphi, cphi);
                float t, e;
                two_sum(hs, __fmul_rn(w, D), t, e);
                hs = t;
                hc += e;
                habs = fmaf(fabsf(w), fabsf(D), habs);
            }
        } else {
            // as the FP64 fold: one sum, the weighted deviation, one FMA
#pragma unroll
            for (int k = 0; k < 8; k++) acc = fma(W, gdevw_d<GK>(S + dl[k], wl[k], sphi, cphi, ph), acc);
        }
        S += (T)1e-7;
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = acc + 1e-30 * aabs + (double)hs + (double)hc + 1e-30 * habs;
}

// Eight independent fused multiply-add chains per thread.
template <typename T>
__global__ void __launch_bounds__(256) sg_fma_kernel(int sweeps, double *out) {
    T x[8];
    const T a = (T)0.999999, b = (T)1e-7;
#pragma unroll
    for (int k = 0; k < 8; k++) x[k] = (T)(threadIdx.x + k);
    for (int it = 0; it < sweeps; it++) {
#pragma unroll
        for (int k = 0; k < 8; k++) x[k] = x[k] * a + b;
    }
    T s = 0;
#pragma unroll
    for (int k = 0; k < 8; k++) s += x[k];
    out[blockIdx.x * blockDim.x + threadIdx.x] = (double)s;
}

// The float-float inner loop on register-resident data.
template <int GK>
__global__ void __launch_bounds__(256) sg_ceiling_ff_kernel(int sweeps, double *out) {
    ff2 dl[4], wl[4];
#pragma unroll
    for (int k = 0; k < 4; k++) {
        dl[k] = ff2{(float)((k - 1.5) * 0.05 + threadIdx.x * 1e-5), 1e-12f};
        wl[k] = ff2{(k & 1) ? -0.25f : 0.3f, 1e-10f};
    }
    ff2 S = {(float)(blockIdx.x * 1e-6), 0.f}, W = {0.7f, 0.f};
    const ff2 sphi = {0.3f, 0.f}, cphi = {0.95f, 0.f};
    ff2 fa = {0.f, 0.f};
    float habs = 0.f;
    for (int it = 0; it < sweeps; it++) {
#pragma unroll
        for (int k = 0; k < 4; k++) {
            const ff2 s = ff_add(S, dl[k]), w = ff_mul(W, wl[k]);
            const ff2 D = gdev_ff<GK>(s, sphi, cphi);
            fa = ff_add(fa, ff_mul(w, D));
            habs = fmaf(fabsf(w.hi), fabsf(D.hi), habs);
        }
        S = ff_add_f(S, 1e-7f);
    }
    out[blockIdx.x * blockDim.x + threadIdx.x] = ff_to_double(fa) + 1e-30 * habs;
}

double sg_launch_ceiling(int prec, int kind, int sms, double *d_out, cudaStream_t s) {
    if (prec == 2 && kind != 2) {
        const int threads = 256, blocks = sms * 8;
        const int sweeps = 1 << 9;
        if (kind == 1) sg_ceiling_ff_kernel<SG_GK_OSC><<<blocks, threads, 0, s>>>(sweeps, d_out);
        else sg_ceiling_ff_kernel<SG_GK_EXPM1><<<blocks, threads, 0, s>>>(sweeps, d_out);
        return 4.0 * threads * (double)blocks * sweeps;
    }
    if (prec == 2) prec = 1;
    const int threads = 256, blocks = sms * 8;
    int sweeps;
    double per = 8.0 * threads * (double)blocks;
    if (kind == 2) {
        sweeps = prec ? 1 << 16 : 1 << 11;
        if (prec) sg_fma_kernel<float><<<blocks, threads, 0, s>>>(sweeps, d_out);
        else sg_fma_kernel<double><<<blocks, threads, 0, s>>>(sweeps, d_out);
        per *= 2.0;  // two flops per fused multiply-add
    } else {
        sweeps = prec ? 1 << 11 : 1 << 7;
        if (prec) {
            if (kind == 1) sg_ceiling_kernel<float, SG_GK_OSC><<<blocks, threads, 0, s>>>(sweeps, d_out);
            else sg_ceiling_kernel<float, SG_GK_EXPM1><<<blocks, threads, 0, s>>>(sweeps, d_out);
        } else {
            if (kind == 1) sg_ceiling_kernel<double, SG_GK_OSC><<<blocks, threads, 0, s>>>(sweeps, d_out);
            else sg_ceiling_kernel<double, SG_GK_EXPM1><<<blocks, threads, 0, s>>>(sweeps, d_out);
        }
    }
    return per * sweeps;
}

// ---------------------------------------------------------------------------
// function check: the fold's elementary functions on given arguments
// ---------------------------------------------------------------------------

__global__ void sg_fn_kernel(int kind, int prec, const double *x, double *y, int n) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    if (prec == 2) {
        const ff2 a = ff_from_double(x[i]);
        if (kind == 0) {
            y[i] = ff_to_double(ff_expm1(a));
        } else {
            ff2 s, c;
            ff_sincos(a, &s, &c);
            y[2 * i] = ff_to_double(s);
            y[2 * i + 1] = ff_to_double(c);
        }
        return;
    }
    if (kind == 0) {
        y[i] = prec ? (double)sg_expm1f((float)x[i]) : sg_expm1_d(x[i]);
    } else {
        if (prec) {
            float s, c;
            sincosf((float)x[i], &s, &c);
            y[2 * i] = s;
            y[2 * i + 1] = c;
        } else {
            double s, c;
            sg_sincos_d(x[i], &s, &c);
            y[2 * i] = s;
            y[2 * i + 1] = c;
        }
    }
}

cudaError_t sg_launch_fn(int kind, int prec, const double *x, double *y, int n, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    sg_fn_kernel<<<(n + 255) / 256, 256, 0, s>>>(kind, prec, x, y, n);
    return cudaGetLastError();
}
