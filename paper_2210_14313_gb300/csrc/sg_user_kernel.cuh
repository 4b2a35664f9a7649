// Fold kernel for a user integrand.  Not compiled into the library: it is
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
    if (A.nchunks == 0) {  // q = d: the rule is the centre point alone
        if (blockIdx.x == 0 && threadIdx.x == 0) {
            asm volatile("griddepcontrol.wait;" ::: "memory");
            int e2 = 0;
            SgOutDev o;
            o.mant = frexp(fc, &e2);
            o.exp2 = (double)e2;
            o.value = fc;
            o.cond = 1.0;
            o.err_est = 0.05 * A.unit_roundoff;
            o.sum = fc;
            o.abs_sum = fabs(fc);
            A.out[A.items[0].out] = o;
        }
        return;
    }
    bool waited = false;
    for (;;) {
        unsigned long long c = 0;
        if (lane == 0) c = atomicAdd(A.work, 1ull);
        c = __shfl_sync(SG_FULL_MASK, c, 0);
        if (c >= A.nchunks) break;
        long long lo = 0, hi = A.npat - 1;
        if (A.chunk_start) {
            lo = __ldg(&A.chunk_start[c].pat);
        } else {
            while (lo < hi) {
                const long long mid = (lo + hi + 1) >> 1;
                if (__ldg(A.pat_chunk0 + mid) <= c) lo = mid;
                else hi = mid - 1;
            }
        }
        const SgPatDev *P = A.pats + lo;
        const int item = P->item;
        const SgItemDev *I = A.items + item;
        const int d = I->d, r = P->r, tm = P->tm;
        unsigned long long rank, cnt;
        int a_lo, a_hi;
        sg_chunk_span(P, c, &rank, &cnt, &a_lo, &a_hi);
        if (A.chunk_start) {
            if (lane < r) sIdx[lane] = __ldg(&A.chunk_start[c].idx[lane]);
        } else {
            unrank_warp(rank, d, r, A.binom, sIdx, lane);
        }
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
        acc = warp_sum(acc);
        if (lane == 0) {
            SgSlot sl;
            sl.sum = acc * P->coef;
            sl.abs = fabs(acc * P->coef);
            sl.lo = 0.0;
            sl.pad = 0.0;
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
