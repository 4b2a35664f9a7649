/*
 * Plain CPU oracle for Smolyak sparse-grid quadrature (test infrastructure).
 *
 * This file is test infrastructure only: the tests, the smoke check and the
 * CPU-baseline leg of the benchmark load it; the library never does.  It
 * shares no code with the CUDA path.
 *
 * What it computes (all in IEEE double, round to nearest):
 *
 *   Q_d^q f = sum_{q-d+1 <= |l| <= q} (-1)^{q-|l|} C(d-1, q-|l|)
 *             sum_{l in N_{d,|l|}} (J^{l_1} x ... x J^{l_d}) f        (Eq. 2.6)
 *
 * on the unit cube [0,1]^d, with q = d + L.  The same value is reached by the
 * coordinate-wise reformulation (Eq. 2.9), read as the sum over all level
 * multi-indices with |l| <= q of tensor products of difference rules
 * Delta_l = J^l - J^{l-1}, Delta_1 = J^1 (Section 2.1).  The default path
 * (or_integrate with form 0) enumerates that difference form: every tensor
 * point of every subgrid is visited, the full d-vector x_p is built, and f is
 * evaluated from scratch in O(d) work per point, with no reuse between
 * points.  Form 1 enumerates Eq. 2.6 literally.
 *
 * Cancellation: the signed weights make sum_p W_p f(x_p) lose digits, so the
 * difference form adds W_p * (f(x_p) - f(c)) with c = (1/2, ..., 1/2): every
 * subgrid except the centre one has weights summing to zero, so this is the
 * same sum.  f(x_p) - f(c) is evaluated in a form without cancellation
 * (expm1, a sine product, log1p), and the sum is a Neumaier compensated sum.
 *
 * 1-D rules on [0,1] (the paper's rules on [-1,1] mapped by x -> (x+1)/2,
 * w -> w/2):
 *   trapezoid        Eq. 2.10; level 1 read as the single midpoint, weight 1
 *   Clenshaw-Curtis  Eq. 2.11; n_1 = 1, n_l = 2^(l-1) + 1, explicit weights
 *   Gauss-Patterson  Eq. 2.12; n_l = 2^l - 1, nested; nodes and weights from
 *                    the table sg_gp_table.h (Patterson extensions computed
 *                    at 300 digits by gen_gp_table.py)
 *   Gauss-Legendre   Eq. 2.13; n_l = l, zeros of P_l by Newton's method
 * Growth: by default level l is the rule's l-th member.  With the flag
 * OR_SLOW in `kind`, level l is the smallest member exact for polynomials of
 * degree 2l - 1 (the paper's accuracy-level convention of Section 5.4:
 * trapezoid and Clenshaw-Curtis N = 1, 3, 5, 9, 9, 17, 17, 17, 17, 33, ...;
 * Gauss-Patterson N = 1, 3, 3, 7, 7, 7, 15, ...); Gauss-Legendre has n_l = l
 * either way.  Two consecutive levels on the same member have a zero
 * difference rule.
 *
 * Parameters: params[0..d) = a, params[d..2d) = u, for every family:
 *   0 exp-linear   f = exp(sum a_i x_i)
 *   1 oscillatory  f = cos(2 pi u_0 + sum a_i x_i)
 *   2 product peak f = prod 1/(a_i^-2 + (x_i - u_i)^2)
 *   3 gaussian     f = exp(-sum a_i^2 (x_i - u_i)^2)
 *   4 gaussian-lin f = exp(-sum a_i (x_i - u_i)^2)
 * and, for the library's compiled user integrands (test families):
 *  10 corner peak  f = (1 + sum a_i x_i)^-(d+1)
 *  11 norm         f = exp(-sqrt(sum a_i (x_i - u_i)^2))
 *  12 two sums     f = (sum a_i x_i) exp(-sum u_i x_i^2)
 *  13 polynomial   f = (sum a_i x_i)^3 + (sum u_i x_i)^2
 *
 * Results are returned as (mant, exp2) with Q = mant * 2^exp2, because the
 * product-peak value underflows a double at large d.
 *
 * Determinism: work is split into units (first active dimension, its level,
 * its node); each unit is summed in a fixed order into its own compensated
 * slot, and the slots are merged in unit order, so the result does not depend
 * on the number of threads.
 */
#include <math.h>
#include <pthread.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <unistd.h>

#include "sg_gp_table.h"

#define OR_MAX_LEVEL 13 /* largest member of a nested rule: 4097 nodes */
#define OR_MAX_ACC 32   /* largest accuracy level (levels 1 .. L + 1) */
#define OR_SLOW 16      /* flag in `kind`: the paper's delayed growth */

enum { R_TRAP = 1, R_CC = 2, R_GP = 3, R_GL = 4 };
enum { F_EXPLIN = 0, F_OSC = 1, F_PEAK = 2, F_GAUSS = 3, F_GAUSSLIN = 4 };
/* Integrands outside the generalised-additive model, for the library's user
 * integrands (sg_integrand_create): evaluated at every point from the full
 * d-vector, f(x) - f(c) formed directly. */
enum { F_UCORNER = 10, F_UNORM = 11, F_UPROD2 = 12, F_UPOLY = 13 };
enum { FORM_DIFF = 0, FORM_COMB = 1 };

/* ------------------------------------------------------------------------ */
/* 1-D rules                                                                 */
/* ------------------------------------------------------------------------ */

/* Node count of member r of a rule family (0 if out of range). */
static int member_nodes(int rule, int r) {
    if (r < 1) return 0;
    if (rule == R_GL) return r <= OR_MAX_LEVEL ? r : 0;
    if (rule == R_GP) return r <= OR_GP_LEVELS ? (1 << r) - 1 : 0;
    if (rule != R_CC && rule != R_TRAP) return 0;
    if (r > OR_MAX_LEVEL) return 0;
    return r == 1 ? 1 : (1 << (r - 1)) + 1;
}

/* Degree of polynomial exactness that selects member r under the delayed
 * growth: Clenshaw-Curtis with n (odd) nodes integrates degree n exactly (the
 * trapezoid rule follows the same sequence, Section 5.4); Gauss-Patterson
 * with 2^r - 1 nodes is exact to degree 3 * 2^(r-1) - 1 (degree 1 for r = 1). */
static int member_degree(int rule, int r) {
    if (rule == R_GP) return r == 1 ? 1 : 3 * (1 << (r - 1)) - 1;
    return member_nodes(R_CC, r);
}

/* Member of the rule family that serves accuracy level `level`. */
static int level_member(int kind, int level) {
    int rule = kind & 15;
    if (level < 1) return 0;
    if (!(kind & OR_SLOW) || rule == R_GL) return level;
    for (int r = 1; r <= OR_MAX_LEVEL; r++) {
        if (member_nodes(rule, r) == 0) return 0;
        if (member_degree(rule, r) >= 2 * level - 1) return r;
    }
    return 0;
}

static int level_nodes(int kind, int level) {
    return member_nodes(kind & 15, level_member(kind, level));
}

/* Legendre P_n and P_{n-1} at x by the three-term recurrence. */
static void legendre(int n, double x, double *pn, double *pn1) {
    double p0 = 1.0, p1 = x;
    if (n == 0) { *pn = 1.0; *pn1 = 0.0; return; }
    for (int k = 1; k < n; k++) {
        double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
        p0 = p1;
        p1 = p2;
    }
    *pn = p1;
    *pn1 = p0;
}

/* Eq. 2.13: nodes are the zeros of P_n on [-1,1], weights
 * 2 / ((1 - x^2) P_n'(x)^2).  Newton from the asymptotic guess
 * cos(pi (i - 1/4) / (n + 1/2)); the upper half is mirrored so the rule is
 * exactly symmetric and the middle node of an odd rule is exactly 0. */
static void gl_rule(int n, double *x, double *w) {
    for (int i = 1; i <= (n + 1) / 2; i++) {
        double z = cos(M_PI * (i - 0.25) / (n + 0.5));
        double dp = 0.0;
        for (int it = 0; it < 100; it++) {
            double pn, pn1;
            legendre(n, z, &pn, &pn1);
            dp = n * (z * pn - pn1) / (z * z - 1.0);
            double dz = pn / dp;
            z -= dz;
            if (fabs(dz) < 1e-17) break;
        }
        double pn, pn1;
        legendre(n, z, &pn, &pn1);
        dp = n * (z * pn - pn1) / (z * z - 1.0);
        double wi = 2.0 / ((1.0 - z * z) * dp * dp);
        if (2 * i - 1 == n) z = 0.0;
        /* zero i is near +1; store ascending on [-1,1] */
        x[n - i] = z;
        w[n - i] = wi;
        x[i - 1] = -z;
        w[i - 1] = wi;
    }
}

/* Eq. 2.11 on [-1,1]: x_j = -cos(pi (j-1)/(n-1)), end weights 1/(n(n-2)),
 * interior weights (2/(n-1)) (1 + 2 sum'_{k=1}^{(n-1)/2} cos(2 pi (j-1) k/(n-1)) / (1-4k^2))
 * with the last term of the sum halved. */
static void cc_rule(int n, double *x, double *w) {
    if (n == 1) { x[0] = 0.0; w[0] = 2.0; return; }
    int N = n - 1;
    for (int j = 0; j < n; j++) {
        x[j] = -cos(M_PI * (double)j / (double)N);
        if (2 * j == N) x[j] = 0.0;
        if (j == 0 || j == N) {
            w[j] = 1.0 / ((double)n * (double)(n - 2));
        } else {
            double s = 0.0;
            int K = N / 2;
            for (int k = 1; k <= K; k++) {
                double t = cos(2.0 * M_PI * (double)j * (double)k / (double)N) / (1.0 - 4.0 * k * k);
                if (k == K) t *= 0.5;
                s += t;
            }
            w[j] = 2.0 / (double)N * (1.0 + 2.0 * s);
        }
    }
    x[0] = -1.0;
    x[N] = 1.0;
}

/* Eq. 2.10 with the midpoint reading of level 1: equispaced nodes, spacing
 * h = 2/(n-1), weights h with both ends halved. */
static void trap_rule(int n, double *x, double *w) {
    if (n == 1) { x[0] = 0.0; w[0] = 2.0; return; }
    int N = n - 1;
    for (int j = 0; j < n; j++) {
        x[j] = -1.0 + 2.0 * (double)j / (double)N;
        w[j] = 2.0 / (double)N;
    }
    w[0] *= 0.5;
    w[N] *= 0.5;
}

/* Level-l rule on [0,1], nodes ascending.  Returns the node count. */
int or_rule(int kind, int level, double *x, double *w) {
    int n = level_nodes(kind, level);
    int rule = kind & 15;
    if (n <= 0 || (kind & ~(15 | OR_SLOW))) return -1;
    if (!x || !w) return n;
    if (rule == R_GP) {  /* tabulated on [0,1] already */
        int r = level_member(kind, level);
        memcpy(x, or_gp_x[r], sizeof(double) * n);
        memcpy(w, or_gp_w[r], sizeof(double) * n);
        return n;
    }
    if (rule == R_GL) gl_rule(n, x, w);
    else if (rule == R_CC) cc_rule(n, x, w);
    else if (rule == R_TRAP) trap_rule(n, x, w);
    else return -1;
    for (int j = 0; j < n; j++) {
        x[j] = 0.5 * (x[j] + 1.0);
        w[j] = 0.5 * w[j];
    }
    if (n % 2 == 1) x[n / 2] = 0.5;
    return n;
}

/* Difference rule Delta_l = J^l - J^{l-1} on the union of both node sets
 * (Delta_1 = J^1).  Nested rules (trapezoid, CC): node j of level l-1 is node
 * 2j of level l, matched by index.  Gauss-Legendre: consecutive levels share
 * no node, so the union is the concatenation.  Returns the node count. */
int or_delta_rule(int kind, int level, double *x, double *w) {
    int n = level_nodes(kind, level);
    int rule = kind & 15;
    if (n <= 0 || (kind & ~(15 | OR_SLOW))) return -1;
    if (level == 1) return or_rule(kind, 1, x, w);
    /* same member as the level below: the difference rule is zero */
    if (level_member(kind, level) == level_member(kind, level - 1)) return 0;
    int n0 = level_nodes(kind, level - 1);
    int nested = (rule != R_GL);
    int total = nested ? n : n + n0;
    if (!x || !w) return total;
    double x0[(1 << (OR_MAX_LEVEL - 1)) + 1], w0[(1 << (OR_MAX_LEVEL - 1)) + 1];
    or_rule(kind, level, x, w);
    or_rule(kind, level - 1, x0, w0);
    if (nested) {
        /* node j of the coarser member is node 2j (trapezoid, CC: shared
         * ends) or 2j + 1 (Gauss-Patterson: a new node in every gap) */
        if (n0 == 1) {
            w[n / 2] -= w0[0];
        } else {
            for (int j = 0; j < n0; j++) w[2 * j + (rule == R_GP)] -= w0[j];
        }
    } else {
        for (int j = 0; j < n0; j++) {
            x[n + j] = x0[j];
            w[n + j] = -w0[j];
        }
    }
    return total;
}

/* ------------------------------------------------------------------------ */
/* Compensated sum (Neumaier 1974)                                           */
/* ------------------------------------------------------------------------ */

typedef struct { double s, c, abs; } csum;

static void cs_add(csum *a, double v) {
    double t = a->s + v;
    if (fabs(a->s) >= fabs(v)) a->c += (a->s - t) + v;
    else a->c += (v - t) + a->s;
    a->s = t;
    a->abs += fabs(v);
}

static double cs_value(const csum *a) { return a->s + a->c; }

/* ------------------------------------------------------------------------ */
/* Integrand families                                                        */
/* ------------------------------------------------------------------------ */

typedef struct {
    int fam, d;
    const double *a, *u;
    double logscale, logscale_lo; /* log f(c) = logscale + logscale_lo (exponential
                                   * families), 0 for oscillatory */
    double theta_c;  /* phase at the centre, reduced to [-pi, pi] */
    double base;     /* f(c) / scale: 1, or cos(theta_c) */
} family;

static double general_value(int fam, const double *a, const double *u, int d, const double *x) {
    double s = 0.0, t = 0.0;
    switch (fam) {
    case F_UCORNER:
        for (int i = 0; i < d; i++) s += a[i] * x[i];
        return pow(1.0 + s, -(double)(d + 1));
    case F_UNORM:
        for (int i = 0; i < d; i++) s += a[i] * (x[i] - u[i]) * (x[i] - u[i]);
        return exp(-sqrt(s));
    case F_UPROD2:
        for (int i = 0; i < d; i++) {
            s += a[i] * x[i];
            t += u[i] * x[i] * x[i];
        }
        return s * exp(-t);
    case F_UPOLY:
        for (int i = 0; i < d; i++) {
            s += a[i] * x[i];
            t += u[i] * x[i];
        }
        return s * s * s + t * t;
    }
    return 0.0;
}

static int is_general(int fam) { return fam >= F_UCORNER && fam <= F_UPOLY; }

static void family_init(family *F, int fam, const double *params, int d) {
    F->fam = fam;
    F->d = d;
    F->a = params;
    F->u = params + d;
    /* log f(c) as a compensated sum: at d = 200 the product peak has
     * |log f(c)| ~ 1500, where one ulp of a plain double sum is already a
     * relative error of 2e-13 in f(c). */
    csum s = {0, 0, 0};
    F->theta_c = 0.0;
    F->base = 1.0;
    switch (fam) {
    case F_EXPLIN:
        for (int i = 0; i < d; i++) cs_add(&s, 0.5 * F->a[i]);
        break;
    case F_GAUSS:
        for (int i = 0; i < d; i++) cs_add(&s, -F->a[i] * F->a[i] * (0.5 - F->u[i]) * (0.5 - F->u[i]));
        break;
    case F_GAUSSLIN:
        for (int i = 0; i < d; i++) cs_add(&s, -F->a[i] * (0.5 - F->u[i]) * (0.5 - F->u[i]));
        break;
    case F_PEAK:
        for (int i = 0; i < d; i++) {
            double ai = F->a[i], v = 0.5 - F->u[i];
            cs_add(&s, -log(1.0 / (ai * ai) + v * v));
        }
        break;
    case F_OSC: {
        double t = 2.0 * M_PI * F->u[0];
        for (int i = 0; i < d; i++) t += 0.5 * F->a[i];
        F->theta_c = remainder(t, 2.0 * M_PI);
        F->base = cos(F->theta_c);
        break;
    }
    }
    F->logscale = s.s;
    F->logscale_lo = s.c;
    if (is_general(fam)) {  /* scale 1, base f(c) */
        double c[d > 0 ? d : 1];
        for (int i = 0; i < d; i++) c[i] = 0.5;
        F->base = general_value(fam, F->a, F->u, d, c);
    }
}

/* (f(x) - f(c)) / scale, evaluated from the full d-vector x. */
static double family_dev(const family *F, const double *x) {
    const double *a = F->a, *u = F->u;
    int d = F->d;
    double s = 0.0;
    if (is_general(F->fam)) return general_value(F->fam, a, u, d, x) - F->base;
    switch (F->fam) {
    case F_EXPLIN:
        for (int i = 0; i < d; i++) s += a[i] * (x[i] - 0.5);
        return expm1(s);
    case F_GAUSS:
        /* a^2 [(x-u)^2 - (1/2-u)^2] = a^2 (x - 1/2)(x + 1/2 - 2u) */
        for (int i = 0; i < d; i++) s -= a[i] * a[i] * (x[i] - 0.5) * (x[i] + 0.5 - 2.0 * u[i]);
        return expm1(s);
    case F_GAUSSLIN:
        for (int i = 0; i < d; i++) s -= a[i] * (x[i] - 0.5) * (x[i] + 0.5 - 2.0 * u[i]);
        return expm1(s);
    case F_PEAK:
        /* psi(x)/psi(c) = 1 + eps, eps = (1/2 - x)(1/2 + x - 2u) / (a^-2 + (x-u)^2) */
        for (int i = 0; i < d; i++) {
            double ai = a[i], v = x[i] - u[i];
            double eps = (0.5 - x[i]) * (0.5 + x[i] - 2.0 * u[i]) / (1.0 / (ai * ai) + v * v);
            s += log1p(eps);
        }
        return expm1(s);
    case F_OSC:
        /* cos(t + D) - cos(t) = -2 sin(D/2) sin(t + D/2) */
        for (int i = 0; i < d; i++) s += a[i] * (x[i] - 0.5);
        return -2.0 * sin(0.5 * s) * sin(F->theta_c + 0.5 * s);
    }
    return 0.0;
}

/* f(x) / scale, evaluated directly (no deviation); used by the literal Eq. 2.6 form. */
static double family_val(const family *F, const double *x) {
    const double *a = F->a, *u = F->u;
    int d = F->d;
    double s = 0.0;
    if (is_general(F->fam)) return general_value(F->fam, a, u, d, x);
    switch (F->fam) {
    case F_EXPLIN:
        for (int i = 0; i < d; i++) s += a[i] * x[i];
        return exp(s - F->logscale);
    case F_GAUSS:
        for (int i = 0; i < d; i++) s -= a[i] * a[i] * (x[i] - u[i]) * (x[i] - u[i]);
        return exp(s - F->logscale);
    case F_GAUSSLIN:
        for (int i = 0; i < d; i++) s -= a[i] * (x[i] - u[i]) * (x[i] - u[i]);
        return exp(s - F->logscale);
    case F_PEAK:
        for (int i = 0; i < d; i++) {
            double v = x[i] - u[i];
            s -= log(1.0 / (a[i] * a[i]) + v * v);
        }
        return exp(s - F->logscale);
    case F_OSC:
        s = 2.0 * M_PI * u[0];
        for (int i = 0; i < d; i++) s += a[i] * x[i];
        return cos(s);
    }
    return 0.0;
}

/* ------------------------------------------------------------------------ */
/* Enumeration of the sparse grid                                            */
/* ------------------------------------------------------------------------ */

/* Rules attached to the excess k = l - 1 of an active dimension (k >= 1):
 * the difference rule Delta_{k+1} (form 0) or the full rule J^{k+1} (form 1).
 * An inactive dimension (k = 0) sits at the centre 1/2 with weight 1, which
 * is both Delta_1 and J^1. */
typedef struct {
    int kind, d, L, form;
    int n[OR_MAX_ACC + 1];
    double *x[OR_MAX_ACC + 1], *w[OR_MAX_ACC + 1];
    int K_lo;                     /* lowest |k| that belongs to the rule */
    double coef[OR_MAX_ACC + 1]; /* multiplier per |k| */
} grid;

static double binom(int n, int k) {
    if (k < 0 || k > n) return 0.0;
    double r = 1.0;
    for (int i = 1; i <= k; i++) r = r * (double)(n - k + i) / (double)i;
    return floor(r + 0.5);
}

static int grid_init(grid *G, int kind, int d, int L, int form) {
    memset(G, 0, sizeof(*G));
    if (d < 1 || L < 0 || L + 1 > OR_MAX_ACC) return -1;
    for (int l = 1; l <= L + 1; l++)
        if (or_rule(kind, l, 0, 0) <= 0) return -1;
    G->kind = kind; G->d = d; G->L = L; G->form = form;
    for (int k = 1; k <= L; k++) {
        int n = (form == FORM_DIFF) ? or_delta_rule(kind, k + 1, 0, 0) : or_rule(kind, k + 1, 0, 0);
        G->n[k] = n;
        G->x[k] = (double *)malloc(sizeof(double) * n);
        G->w[k] = (double *)malloc(sizeof(double) * n);
        if (form == FORM_DIFF) or_delta_rule(kind, k + 1, G->x[k], G->w[k]);
        else or_rule(kind, k + 1, G->x[k], G->w[k]);
    }
    if (form == FORM_DIFF) {
        G->K_lo = 0;
        for (int K = 0; K <= L; K++) G->coef[K] = 1.0;
    } else {
        /* Eq. 2.6: q - d + 1 <= |l| <= q  <=>  L - d + 1 <= |k| <= L,
         * coefficient (-1)^(q-|l|) C(d-1, q-|l|) with q - |l| = L - |k|. */
        G->K_lo = L - d + 1 > 0 ? L - d + 1 : 0;
        for (int K = 0; K <= L; K++)
            G->coef[K] = ((L - K) % 2 ? -1.0 : 1.0) * binom(d - 1, L - K);
    }
    return 0;
}

static void grid_free(grid *G) {
    for (int k = 1; k <= G->L; k++) { free(G->x[k]); free(G->w[k]); }
}

typedef struct visitor visitor;
struct visitor {
    void (*visit)(visitor *V, const double *x, double W);
};

/* Visits every tensor point whose active dimensions after the ones already
 * placed lie in [next, d): the current point x first (the subgrid in which no
 * further dimension is active), then each extension by one more active
 * dimension i, excess k <= rem, node j.  K is the current |k|. */
static void walk(const grid *G, double *x, int next, int rem, int K, double W, visitor *V) {
    if (K >= G->K_lo) V->visit(V, x, W * G->coef[K]);
    if (rem == 0) return;
    for (int i = next; i < G->d; i++) {
        for (int k = 1; k <= rem; k++)
            for (int j = 0; j < G->n[k]; j++) {
                x[i] = G->x[k][j];
                walk(G, x, i + 1, rem - k, K + k, W * G->w[k][j], V);
            }
        x[i] = 0.5;
    }
}

/* A unit is the set of points whose first active dimension is i with
 * excess k and node j.  Unit index -> (i, k, j), in (i, k, j) order. */
static int unit_count(const grid *G) {
    int per = 0;
    for (int k = 1; k <= G->L; k++) per += G->n[k];
    return G->d * per;
}

static void unit_walk(const grid *G, double *x, int unit, visitor *V) {
    int per = 0;
    for (int k = 1; k <= G->L; k++) per += G->n[k];
    int i = unit / per, r = unit % per, k = 1;
    while (r >= G->n[k]) { r -= G->n[k]; k++; }
    x[i] = G->x[k][r];
    walk(G, x, i + 1, G->L - k, k, G->w[k][r], V);
    x[i] = 0.5;
}

/* ------------------------------------------------------------------------ */
/* Integration                                                               */
/* ------------------------------------------------------------------------ */

typedef struct {
    visitor base;
    const family *F;
    int form;
    csum acc;
} int_visitor;

static void int_visit(visitor *V, const double *x, double W) {
    int_visitor *I = (int_visitor *)V;
    if (I->form == FORM_DIFF) cs_add(&I->acc, W * family_dev(I->F, x));
    else cs_add(&I->acc, W * family_val(I->F, x));
}

typedef struct {
    const grid *G;
    const family *F;
    csum *slots;
    int nunits;
    int next; /* shared unit counter */
} int_job;

static void *int_worker(void *arg) {
    int_job *J = (int_job *)arg;
    double *x = (double *)malloc(sizeof(double) * J->G->d);
    for (int i = 0; i < J->G->d; i++) x[i] = 0.5;
    for (;;) {
        int u = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (u >= J->nunits) break;
        int_visitor V = {{int_visit}, J->F, J->G->form, {0, 0, 0}};
        unit_walk(J->G, x, u, &V.base);
        J->slots[u] = V.acc;
    }
    free(x);
    return 0;
}

static int resolve_threads(int nthreads) {
    if (nthreads > 0) return nthreads;
    long n = sysconf(_SC_NPROCESSORS_ONLN);
    return n > 0 ? (int)n : 1;
}

/* Splits the log-scale s_hi + s_lo into 2^e0 * exp(r), |r| < ln 2, with ln 2
 * in two parts (Cody & Waite) so that r keeps its accuracy for large |s|. */
static void split_log(double s_hi, double s_lo, double *e0, double *r) {
    const double ln2_hi = 6.93147180369123816490e-01, ln2_lo = 1.90821492927058770002e-10;
    double e = floor(s_hi / M_LN2);
    *e0 = e;
    *r = ((s_hi - e * ln2_hi) - e * ln2_lo) + s_lo;
}

/*
 * Smolyak value Q_d^{d+L} f on [0,1]^d.  form 0: difference form (Eq. 2.9
 * read as sums of difference rules), form 1: combination form (Eq. 2.6).
 * out[0] = mant, out[1] = exp2 (Q = mant * 2^exp2), out[2] = Q as a double
 * (may under/overflow), out[3] = sum |terms| / |sum| (conditioning of the
 * final sum, scale removed), out[4] = number of points visited.
 * Returns 0, or -1 on invalid arguments.
 */
int or_integrate(int kind, int fam, const double *params, int d, int L, int form,
                 int nthreads, double *out) {
    if (!params || !out || ((fam < 0 || fam > 4) && !is_general(fam))) return -1;
    if (form != FORM_DIFF && form != FORM_COMB) return -1;
    grid G;
    if (grid_init(&G, kind, d, L, form)) return -1;
    family F;
    family_init(&F, fam, params, d);

    int nunits = unit_count(&G);
    csum *slots = (csum *)calloc(nunits > 0 ? nunits : 1, sizeof(csum));
    int_job J = {&G, &F, slots, nunits, 0};
    int nt = resolve_threads(nthreads);
    if (nt > nunits) nt = nunits > 0 ? nunits : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nt);
    for (int t = 0; t < nt; t++) pthread_create(&th[t], 0, int_worker, &J);
    for (int t = 0; t < nt; t++) pthread_join(th[t], 0);
    free(th);

    csum tot = {0, 0, 0};
    if (form == FORM_DIFF) {
        cs_add(&tot, F.base);
    } else {
        /* centre point, |k| = 0 */
        double *x = (double *)malloc(sizeof(double) * d);
        for (int i = 0; i < d; i++) x[i] = 0.5;
        if (G.K_lo == 0) cs_add(&tot, G.coef[0] * family_val(&F, x));
        free(x);
    }
    for (int u = 0; u < nunits; u++) {
        cs_add(&tot, slots[u].s);
        cs_add(&tot, slots[u].c);
        tot.abs += slots[u].abs - fabs(slots[u].s) - fabs(slots[u].c);
    }
    double T = cs_value(&tot);
    double e0, r;
    split_log(F.logscale, F.logscale_lo, &e0, &r);
    int e1;
    double mant = frexp(exp(r) * T, &e1);
    out[0] = mant;
    out[1] = e0 + e1;
    out[2] = ldexp(mant, (int)(e0 + e1));
    out[3] = tot.abs / fabs(T);
    free(slots);
    grid_free(&G);
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Point listing (tiny grids)                                                */
/* ------------------------------------------------------------------------ */

typedef struct {
    visitor base;
    int d;
    long count, cap;
    double *X, *W;
} pt_visitor;

static void pt_visit(visitor *V, const double *x, double W) {
    pt_visitor *P = (pt_visitor *)V;
    if (P->count < P->cap) {
        memcpy(P->X + (size_t)P->count * P->d, x, sizeof(double) * P->d);
        P->W[P->count] = W;
    }
    P->count++;
}

/*
 * Every tensor point of every subgrid, with its weight (including the
 * combination coefficient in form 1), in enumeration order; repeated points
 * are listed once per subgrid, as in the count n_d^q.  X is row-major
 * [cap][d].  Returns the number of points (which may exceed cap: then only
 * the first cap are written), or -1 on invalid arguments.
 */
long or_points(int kind, int d, int L, int form, double *X, double *W, long cap) {
    grid G;
    if (form != FORM_DIFF && form != FORM_COMB) return -1;
    if (grid_init(&G, kind, d, L, form)) return -1;
    pt_visitor P = {{pt_visit}, d, 0, (X && W) ? cap : 0, X, W};
    double *x = (double *)malloc(sizeof(double) * d);
    for (int i = 0; i < d; i++) x[i] = 0.5;
    walk(&G, x, 0, L, 0, 1.0, &P.base);
    free(x);
    grid_free(&G);
    return P.count;
}

/* n_d^q = sum over the multi-indices of Eq. 2.6 of prod_i n_{l_i} (the point
 * count with repetition), summed dimension by dimension as a polynomial in
 * the excess.  Exact below 2^64. */
uint64_t or_count_points(int kind, int d, int L) {
    if (d < 1 || L < 0 || L + 1 > OR_MAX_ACC) return 0;
    for (int l = 1; l <= L + 1; l++)
        if (or_rule(kind, l, 0, 0) <= 0) return 0;
    unsigned __int128 c[OR_MAX_ACC + 1] = {0}, nc[OR_MAX_ACC + 1];
    c[0] = 1;
    for (int i = 0; i < d; i++) {
        for (int K = 0; K <= L; K++) nc[K] = 0;
        for (int K = 0; K <= L; K++)
            for (int k = 0; k + K <= L; k++)
                nc[K + k] += c[K] * (unsigned __int128)level_nodes(kind, k + 1);
        for (int K = 0; K <= L; K++) c[K] = nc[K];
    }
    unsigned __int128 tot = 0;
    int lo = L - d + 1 > 0 ? L - d + 1 : 0;
    for (int K = lo; K <= L; K++) tot += c[K];
    return (uint64_t)tot;
}

/* Distinct points of the sparse grid of a nested rule (trapezoid,
 * Clenshaw-Curtis, Gauss-Patterson).  In one dimension the points new at
 * level l are n_l - n_{l-1} (n_0 = 0); a point of the grid belongs to exactly
 * one multi-index l with |l| <= q at which each of its coordinates is new, so
 * the count is sum_{|l| <= q} prod_i (n_{l_i} - n_{l_i - 1}).  0 for
 * Gauss-Legendre (not nested) or invalid arguments.  Exact below 2^64. */
uint64_t or_count_distinct(int kind, int d, int L) {
    if ((kind & 15) == R_GL) return 0;
    if (d < 1 || L < 0 || L + 1 > OR_MAX_ACC) return 0;
    for (int l = 1; l <= L + 1; l++)
        if (or_rule(kind, l, 0, 0) <= 0) return 0;
    unsigned __int128 c[OR_MAX_ACC + 1] = {0}, nc[OR_MAX_ACC + 1];
    c[0] = 1;
    for (int i = 0; i < d; i++) {
        for (int K = 0; K <= L; K++) nc[K] = 0;
        for (int K = 0; K <= L; K++)
            for (int k = 0; k + K <= L; k++)
                nc[K + k] += c[K] * (unsigned __int128)(level_nodes(kind, k + 1) - level_nodes(kind, k));
        for (int K = 0; K <= L; K++) c[K] = nc[K];
    }
    unsigned __int128 tot = 0;
    for (int K = 0; K <= L; K++) tot += c[K];
    return (uint64_t)tot;
}

/* ------------------------------------------------------------------------ */
/* Gradient with respect to the parameters                                   */
/* ------------------------------------------------------------------------ */

/* For every family, d f / d theta = h(x) with h depending on x through f (or
 * the phase) and the single coordinate x_i that theta belongs to.  The
 * quadrature of h uses the same deviation idea as the value:
 * Q(h) = h(c) + sum_{p not centre} W_p (h(x_p) - h(c)).
 * gdev returns (h(x) - h(c)) / scale and gc returns h(c) / scale. */
static double grad_pre(const family *F, const double *x) {
    if (F->fam != F_OSC) return family_dev(F, x);
    double s = 0.0;
    for (int t = 0; t < F->d; t++) s += F->a[t] * (x[t] - 0.5);
    return s;
}

/* pre = grad_pre(F, x): the deviation D for the exponential families, the
 * phase offset sum a_t (x_t - 1/2) for the oscillatory one. */
static void grad_terms(const family *F, const double *x, double pre, int idx, double *hdev,
                       double *hc) {
    int d = F->d;
    int is_u = idx >= d, i = is_u ? idx - d : idx;
    double ai = F->a[i], ui = F->u[i], xi = x[i];
    if (F->fam == F_OSC) {
        double s = pre;
        /* sin(t + D) - sin(t) = 2 cos(t + D/2) sin(D/2) */
        double dsin = 2.0 * cos(F->theta_c + 0.5 * s) * sin(0.5 * s);
        double sc = sin(F->theta_c);
        if (!is_u) {            /* d/da_i cos(theta) = -x_i sin(theta) */
            *hc = -0.5 * sc;
            *hdev = -xi * dsin - (xi - 0.5) * sc;
        } else if (i == 0) {    /* d/du_0 = -2 pi sin(theta) */
            *hc = -2.0 * M_PI * sc;
            *hdev = -2.0 * M_PI * dsin;
        } else {
            *hc = 0.0;
            *hdev = 0.0;
        }
        return;
    }
    /* exponential families: d f / d theta = g(x_i) f, f/scale = 1 + D */
    double D = pre;
    double g, g0;
    switch (F->fam) {
    case F_EXPLIN:
        g = is_u ? 0.0 : xi;
        g0 = is_u ? 0.0 : 0.5;
        break;
    case F_GAUSS:
        g = is_u ? 2.0 * ai * ai * (xi - ui) : -2.0 * ai * (xi - ui) * (xi - ui);
        g0 = is_u ? 2.0 * ai * ai * (0.5 - ui) : -2.0 * ai * (0.5 - ui) * (0.5 - ui);
        break;
    case F_GAUSSLIN:
        g = is_u ? 2.0 * ai * (xi - ui) : -(xi - ui) * (xi - ui);
        g0 = is_u ? 2.0 * ai * (0.5 - ui) : -(0.5 - ui) * (0.5 - ui);
        break;
    case F_PEAK: {
        double den = 1.0 / (ai * ai) + (xi - ui) * (xi - ui);
        double den0 = 1.0 / (ai * ai) + (0.5 - ui) * (0.5 - ui);
        g = is_u ? 2.0 * (xi - ui) / den : 2.0 / (ai * ai * ai) / den;
        g0 = is_u ? 2.0 * (0.5 - ui) / den0 : 2.0 / (ai * ai * ai) / den0;
        break;
    }
    default:
        g = g0 = 0.0;
    }
    *hc = g0;
    *hdev = g * D + (g - g0);
}

typedef struct {
    visitor base;
    const family *F;
    const int *idx;
    int nidx;
    csum *acc; /* nidx sums */
} grad_visitor;

static void grad_visit(visitor *V, const double *x, double W) {
    grad_visitor *G = (grad_visitor *)V;
    double pre = grad_pre(G->F, x);
    for (int t = 0; t < G->nidx; t++) {
        double hdev, hc;
        grad_terms(G->F, x, pre, G->idx[t], &hdev, &hc);
        cs_add(&G->acc[t], W * hdev);
    }
}

typedef struct {
    const grid *G;
    const family *F;
    const int *idx;
    int nidx;
    csum *slots; /* [nunits][nidx] */
    int nunits;
    int next;
} grad_job;

static void *grad_worker(void *arg) {
    grad_job *J = (grad_job *)arg;
    double *x = (double *)malloc(sizeof(double) * J->G->d);
    for (int i = 0; i < J->G->d; i++) x[i] = 0.5;
    for (;;) {
        int u = __atomic_fetch_add(&J->next, 1, __ATOMIC_RELAXED);
        if (u >= J->nunits) break;
        grad_visitor V = {{grad_visit}, J->F, J->idx, J->nidx, J->slots + (size_t)u * J->nidx};
        unit_walk(J->G, x, u, &V.base);
    }
    free(x);
    return 0;
}

/*
 * Gradient of the difference-form Smolyak value with respect to the
 * parameters listed in idx (0 <= idx < 2d: a_i for idx < d, u_{idx-d}
 * otherwise).  Writes out_value[0..1] = (mant, exp2) of Q as or_integrate
 * does, and grad[t] such that dQ/dtheta_{idx[t]} = grad[t] * 2^exp2 (the
 * same exponent as Q).  Returns 0, or -1 on invalid arguments.
 */
int or_gradient(int kind, int fam, const double *params, int d, int L, const int *idx,
                int nidx, int nthreads, double *out_value, double *grad) {
    if (!params || !idx || nidx < 1 || !out_value || !grad || fam < 0 || fam > 4) return -1;
    for (int t = 0; t < nidx; t++)
        if (idx[t] < 0 || idx[t] >= 2 * d) return -1;
    double qv[5];
    if (or_integrate(kind, fam, params, d, L, FORM_DIFF, nthreads, qv)) return -1;
    grid G;
    if (grid_init(&G, kind, d, L, FORM_DIFF)) return -1;
    family F;
    family_init(&F, fam, params, d);
    int nunits = unit_count(&G);
    csum *slots = (csum *)calloc((size_t)(nunits > 0 ? nunits : 1) * nidx, sizeof(csum));
    grad_job J = {&G, &F, idx, nidx, slots, nunits, 0};
    int nt = resolve_threads(nthreads);
    if (nt > nunits) nt = nunits > 0 ? nunits : 1;
    pthread_t *th = (pthread_t *)malloc(sizeof(pthread_t) * nt);
    for (int t = 0; t < nt; t++) pthread_create(&th[t], 0, grad_worker, &J);
    for (int t = 0; t < nt; t++) pthread_join(th[t], 0);
    free(th);

    double e0, r;
    split_log(F.logscale, F.logscale_lo, &e0, &r);
    int e1 = (int)(qv[1] - e0); /* Q = frexp(exp(r) T) * 2^(e0 + e1) */
    double *x = (double *)malloc(sizeof(double) * d);
    for (int i = 0; i < d; i++) x[i] = 0.5;
    for (int t = 0; t < nidx; t++) {
        double hdev, hc;
        grad_terms(&F, x, grad_pre(&F, x), idx[t], &hdev, &hc);
        csum tot = {0, 0, 0};
        cs_add(&tot, hc);
        for (int u = 0; u < nunits; u++) {
            cs_add(&tot, slots[(size_t)u * nidx + t].s);
            cs_add(&tot, slots[(size_t)u * nidx + t].c);
        }
        grad[t] = ldexp(exp(r) * cs_value(&tot), -e1);
    }
    out_value[0] = qv[0];
    out_value[1] = qv[1];
    free(x);
    free(slots);
    grid_free(&G);
    return 0;
}
