// Host construction of the 1-D rules on [0,1] and the rule blocks the
// kernels fold (library side; independent of the test oracle).
//
// Rules (paper Section 2.2, mapped from [-1,1] by x -> (x+1)/2, w -> w/2):
//  - trapezoid (Eq. 2.10): n_1 = 1 (midpoint, weight 1), n_l = 2^(l-1) + 1
//    equispaced nodes, end weights halved;
//  - Clenshaw-Curtis (Eq. 2.11): n_1 = 1, n_l = 2^(l-1) + 1 nodes at the
//    Chebyshev extrema; weights from the cosine series of the interpolatory
//    rule (Trefethen, "Spectral Methods in MATLAB", 2000, clencurt), with the
//    cosine arguments reduced exactly in integers;
//  - Gauss-Legendre (Eq. 2.13): n_l = l; nodes are the eigenvalues of the
//    Jacobi matrix of the Legendre recurrence (Golub & Welsch 1969), found by
//    Sturm-sequence bisection and polished by Newton's method, weights
//    2 (1 - x^2) / (n P_{n-1}(x))^2;
//  - Gauss-Patterson (Eq. 2.12): members of 1, 3, 7, 15, 31, 63 nodes, each
//    adding to the previous one the zeros of the polynomial G orthogonal,
//    against the product Q of the existing node factors, to all polynomials
//    of lower degree (Patterson 1968).  The new zeros are found by Newton's
//    method on the orthogonality conditions themselves, with Q and G kept in
//    product form and the integrals done by a Gauss-Legendre rule that is
//    exact for them, all in double-double arithmetic (Dekker 1971); the
//    weights are the integrals of the Lagrange basis polynomials.  Double
//    precision alone loses the 63-node member to cancellation.
// Growth: level l is member l by default; with SG_KIND_SLOW in `kind` it is
// the smallest member exact for degree 2l - 1 (Section 5.4's accuracy
// levels; the trapezoid rule follows Clenshaw-Curtis).  Equal members at
// consecutive levels make an empty difference block.
// Nested rules are generated from the finest level by index, so a node of
// level l-1 is bit-identical to its copy in level l.
#include "sg_rules.h"

#include <math.h>
#include <string.h>

#include <algorithm>
#include <cmath>
#include <vector>

static const double kPi = 3.14159265358979323846;

// Nodes of member r of a rule family (0 if out of range).
static int member_nodes(int rule, int r) {
    if (r < 1 || r > SG_MAX_LEVEL) return 0;
    if (rule == 4) return r;
    if (rule == 3) return r <= SG_GP_MEMBERS ? (1 << r) - 1 : 0;
    if (rule != 1 && rule != 2) return 0;
    return r == 1 ? 1 : (1 << (r - 1)) + 1;
}

// Polynomial degree member r integrates exactly, as used by the slow growth
// (Clenshaw-Curtis with n odd nodes: n; Gauss-Patterson: 3 * 2^(r-1) - 1).
static int member_degree(int rule, int r) {
    if (rule == 3) return r == 1 ? 1 : 3 * (1 << (r - 1)) - 1;
    return member_nodes(2, r);
}

int sg_level_member(int kind, int level) {
    const int rule = kind & 15;
    if (level < 1 || level > SG_MAX_LEVEL || (kind & ~(15 | SG_KIND_SLOW))) return 0;
    if (!(kind & SG_KIND_SLOW) || rule == 4) return member_nodes(rule, level) ? level : 0;
    for (int r = 1; member_nodes(rule, r); r++)
        if (member_degree(rule, r) >= 2 * level - 1) return r;
    return 0;
}

int sg_level_nodes(int kind, int level) { return member_nodes(kind & 15, sg_level_member(kind, level)); }

// ---- Gauss-Legendre ------------------------------------------------------

// Number of eigenvalues of the n x n Jacobi matrix (zero diagonal,
// off-diagonal b_k = k / sqrt(4k^2 - 1)) below x (Sturm count).
static int sturm_count(int n, double x) {
    int cnt = 0;
    double q = -x;
    if (q < 0) cnt++;
    for (int k = 1; k < n; k++) {
        double b2 = (double)k * k / (4.0 * k * k - 1.0);
        if (q == 0.0) q = 1e-300;
        q = -x - b2 / q;
        if (q < 0) cnt++;
    }
    return cnt;
}

// P_n(x) and P_{n-1}(x).
static void legendre_pair(int n, double x, double *pn, double *pm) {
    double a = 1.0, b = x;
    if (n == 0) { *pn = 1.0; *pm = 0.0; return; }
    for (int k = 2; k <= n; k++) {
        double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
        a = b;
        b = c;
    }
    *pn = b;
    *pm = a;
}

static void gauss_legendre(int n, double *x, double *w) {
    // k-th smallest eigenvalue by bisection on [-1, 1]
    for (int k = 0; k < (n + 1) / 2; k++) {
        double lo = -1.0, hi = 1.0;
        for (int it = 0; it < 200 && hi - lo > 1e-300; it++) {
            double mid = 0.5 * (lo + hi);
            if (mid == lo || mid == hi) break;
            if (sturm_count(n, mid) > k) hi = mid;
            else lo = mid;
        }
        double z = 0.5 * (lo + hi);
        for (int it = 0; it < 3; it++) {  // Newton polish on P_n
            double pn, pm;
            legendre_pair(n, z, &pn, &pm);
            double dp = n * (pm - z * pn) / (1.0 - z * z);
            double step = pn / dp;
            if (!(fabs(step) < 1e-3)) break;
            z -= step;
        }
        if (2 * k + 1 == n) z = 0.0;
        double pn, pm;
        legendre_pair(n, z, &pn, &pm);
        double wk = 2.0 * (1.0 - z * z) / ((n * pm) * (n * pm));
        x[k] = z;
        w[k] = wk;
        x[n - 1 - k] = -z;
        w[n - 1 - k] = wk;
    }
}

// ---- Gauss-Patterson -----------------------------------------------------

namespace {

// Double-double numbers hi + lo (|lo| <= ulp(hi)/2): Knuth's TwoSum and the
// FMA TwoProduct give the exact rounding errors (host code is compiled
// without floating-point contraction; std::fma is exact on every host).
struct dd {
    double hi, lo;
};
dd dd_two_sum(double a, double b) {
    const double s = a + b, z = s - a;
    return dd{s, (a - (s - z)) + (b - z)};
}
dd dd_fast(double a, double b) {
    const double s = a + b;
    return dd{s, b - (s - a)};
}
dd operator+(dd a, dd b) {
    dd s = dd_two_sum(a.hi, b.hi), t = dd_two_sum(a.lo, b.lo);
    s = dd_fast(s.hi, s.lo + t.hi);
    return dd_fast(s.hi, s.lo + t.lo);
}
dd operator-(dd a) { return dd{-a.hi, -a.lo}; }
dd operator-(dd a, dd b) { return a + (-b); }
dd operator*(dd a, dd b) {
    const double p = a.hi * b.hi;
    const double e = std::fma(a.hi, b.hi, -p) + (a.hi * b.lo + a.lo * b.hi);
    return dd_fast(p, e);
}
dd operator/(dd a, dd b) {
    const double q1 = a.hi / b.hi;
    dd r = a - b * dd{q1, 0.0};
    const double q2 = r.hi / b.hi;
    r = r - b * dd{q2, 0.0};
    const double q3 = r.hi / b.hi;
    return dd_fast(q1, q2) + dd{q3, 0.0};
}
dd ddv(double v) { return dd{v, 0.0}; }

// Gauss-Legendre rule of M points on [-1, 1] in double-double: the double
// nodes refined by Newton's method on P_M evaluated by its recurrence.
void gl_dd(int M, std::vector<dd> &t, std::vector<dd> &om) {
    std::vector<double> x0(M), w0(M);
    gauss_legendre(M, x0.data(), w0.data());
    t.assign(M, ddv(0.0));
    om.assign(M, ddv(0.0));
    for (int m = 0; m < M; m++) {
        dd x = ddv(x0[m]), pn, pm, dp;
        for (int it = 0; it < 3; it++) {
            pm = ddv(1.0);
            pn = x;
            for (int k = 1; k < M; k++) {
                const dd nx = (ddv(2.0 * k + 1.0) * x * pn - ddv((double)k) * pm) / ddv(k + 1.0);
                pm = pn;
                pn = nx;
            }
            dp = ddv((double)M) * (x * pn - pm) / (x * x - ddv(1.0));
            if (it < 2) x = x - pn / dp;
        }
        t[m] = x;
        om[m] = ddv(2.0) / ((ddv(1.0) - x * x) * dp * dp);
    }
}

// The n + 1 nodes that extend the rule with nodes `old` (n of them).
std::vector<dd> gp_extend(const std::vector<dd> &old) {
    const int n = (int)old.size(), M = 2 * n + 2;  // M-point GL is exact to degree 4n + 3 >= 3n + 1
    std::vector<dd> t, om;
    gl_dd(M, t, om);
    std::vector<dd> Q(M), P((size_t)M * (n + 1));
    for (int m = 0; m < M; m++) {
        dd q = ddv(1.0);
        for (int j = 0; j < n; j++) q = q * (ddv(2.0) * (t[m] - old[j]));
        Q[m] = om[m] * q;
        dd a = ddv(1.0), b = t[m];
        P[(size_t)m * (n + 1)] = a;
        if (n >= 1) P[(size_t)m * (n + 1) + 1] = b;
        for (int k = 1; k < n; k++) {
            const dd c = (ddv(2.0 * k + 1.0) * t[m] * b - ddv((double)k) * a) / ddv(k + 1.0);
            a = b;
            b = c;
            P[(size_t)m * (n + 1) + k + 1] = c;
        }
    }
    // start: one new node in each gap of the sorted old nodes (and the end
    // gaps), at the midpoint in the angle variable
    std::vector<double> edge(n + 2);
    edge[0] = -1.0;
    for (int j = 0; j < n; j++) edge[j + 1] = old[j].hi;
    edge[n + 1] = 1.0;
    std::vector<dd> y(n + 1);
    for (int i = 0; i <= n; i++) y[i] = ddv(cos(0.5 * (acos(edge[i]) + acos(edge[i + 1]))));
    const int N1 = n + 1;
    std::vector<dd> D((size_t)M * N1), pre(N1 + 1), suf(N1 + 1), J((size_t)N1 * N1), F(N1);
    for (int it = 0; it < 40; it++) {
        std::fill(J.begin(), J.end(), ddv(0.0));
        std::fill(F.begin(), F.end(), ddv(0.0));
        for (int m = 0; m < M; m++) {
            for (int i = 0; i < N1; i++) D[(size_t)m * N1 + i] = ddv(2.0) * (t[m] - y[i]);
            pre[0] = ddv(1.0);
            for (int i = 0; i < N1; i++) pre[i + 1] = pre[i] * D[(size_t)m * N1 + i];
            suf[N1] = ddv(1.0);
            for (int i = N1 - 1; i >= 0; i--) suf[i] = suf[i + 1] * D[(size_t)m * N1 + i];
            for (int k = 0; k < N1; k++) {
                const dd qp = Q[m] * P[(size_t)m * (n + 1) + k];
                F[k] = F[k] + qp * pre[N1];
                for (int i = 0; i < N1; i++) J[(size_t)k * N1 + i] = J[(size_t)k * N1 + i] - ddv(2.0) * qp * (pre[i] * suf[i + 1]);
            }
        }
        // J s = F by Gaussian elimination with partial pivoting
        std::vector<int> piv(N1);
        for (int i = 0; i < N1; i++) piv[i] = i;
        for (int c = 0; c < N1; c++) {
            int best = c;
            for (int r = c + 1; r < N1; r++)
                if (fabs(J[(size_t)r * N1 + c].hi) > fabs(J[(size_t)best * N1 + c].hi)) best = r;
            if (best != c) {
                for (int q = 0; q < N1; q++) std::swap(J[(size_t)c * N1 + q], J[(size_t)best * N1 + q]);
                std::swap(F[c], F[best]);
            }
            for (int r = c + 1; r < N1; r++) {
                const dd f = J[(size_t)r * N1 + c] / J[(size_t)c * N1 + c];
                for (int q = c; q < N1; q++) J[(size_t)r * N1 + q] = J[(size_t)r * N1 + q] - f * J[(size_t)c * N1 + q];
                F[r] = F[r] - f * F[c];
            }
        }
        double big = 0.0;
        for (int c = N1 - 1; c >= 0; c--) {
            dd v = F[c];
            for (int q = c + 1; q < N1; q++) v = v - J[(size_t)c * N1 + q] * F[q];
            F[c] = v / J[(size_t)c * N1 + c];
            big = std::max(big, fabs(F[c].hi));
        }
        for (int i = 0; i < N1; i++) y[i] = y[i] - F[i];
        if (big < 1e-30) break;
    }
    return y;
}

struct GpTable {
    std::vector<double> x[SG_GP_MEMBERS + 1], w[SG_GP_MEMBERS + 1];  // on [0,1], ascending
    GpTable() {
        std::vector<dd> nodes(1, ddv(0.0));
        for (int r = 1; r <= SG_GP_MEMBERS; r++) {
            if (r > 1) {
                std::vector<dd> ext = gp_extend(nodes);
                nodes.insert(nodes.end(), ext.begin(), ext.end());
                std::sort(nodes.begin(), nodes.end(), [](const dd &a, const dd &b) {
                    return a.hi < b.hi || (a.hi == b.hi && a.lo < b.lo);
                });
            }
            const int N = (int)nodes.size(), Mw = N / 2 + 1;  // exact to degree 2 Mw - 1 >= N - 1
            std::vector<dd> t, om;
            gl_dd(Mw, t, om);
            x[r].resize(N);
            w[r].resize(N);
            for (int j = 0; j < N; j++) {
                dd wj = ddv(0.0);
                for (int m = 0; m < Mw; m++) {
                    dd l = ddv(1.0);
                    for (int k = 0; k < N; k++)
                        if (k != j) l = l * ((t[m] - nodes[k]) / (nodes[j] - nodes[k]));
                    wj = wj + om[m] * l;
                }
                const dd xj = (nodes[j] + ddv(1.0)) * ddv(0.5);
                x[r][j] = xj.hi + xj.lo;
                w[r][j] = 0.5 * (wj.hi + wj.lo);
            }
            // exact mirror symmetry (the lower half decides), middle node 1/2
            for (int j = 0; j < N / 2; j++) {
                x[r][N - 1 - j] = 1.0 - x[r][j];
                const double ws = 0.5 * (w[r][j] + w[r][N - 1 - j]);
                w[r][j] = w[r][N - 1 - j] = ws;
            }
            x[r][N / 2] = 0.5;
        }
    }
};

const GpTable &gp_table() {
    static const GpTable table;  // built once, thread-safe initialisation
    return table;
}

}  // namespace

// ---- Clenshaw-Curtis and trapezoid ---------------------------------------

// CC weights on [-1,1] for N+1 nodes x_j = cos(pi j / N) (N even):
// w_j = (c_j / N) (1 - sum_{k=1}^{N/2} b_k cos(2 pi j k / N) / (4k^2 - 1)),
// c_0 = c_N = 1, c_j = 2 otherwise, b_{N/2} = 1, b_k = 2 otherwise.
static void cc_weights(int N, double *w) {
    for (int j = 0; j <= N; j++) {
        double s = 0.0;
        for (int k = 1; k <= N / 2; k++) {
            double b = (2 * k == N) ? 1.0 : 2.0;
            long long m = ((long long)j * k) % N;  // exact reduction of j k / N
            s += b * cos(2.0 * kPi * (double)m / (double)N) / (4.0 * k * k - 1.0);
        }
        double c = (j == 0 || j == N) ? 1.0 : 2.0;
        w[j] = c / N * (1.0 - s);
    }
}

int sg_rule_level(int kind, int level, double *x, double *w) {
    int n = sg_level_nodes(kind, level);
    if (n == 0) return 0;
    if (n == 1) {
        x[0] = 0.5;
        w[0] = 1.0;
        return 1;
    }
    kind &= 15;
    if (kind == 3) {
        const GpTable &T = gp_table();
        int r = 1;  // member of n = 2^r - 1 nodes, whatever the growth
        while ((1 << r) - 1 < n) r++;
        for (int j = 0; j < n; j++) {
            x[j] = T.x[r][j];
            w[j] = T.w[r][j];
        }
        return n;
    }
    if (kind == 4) {
        gauss_legendre(n, x, w);
        for (int j = 0; j < n; j++) {
            x[j] = 0.5 + 0.5 * x[j];
            w[j] = 0.5 * w[j];
        }
        if (n % 2) x[n / 2] = 0.5;
        return n;
    }
    int N = n - 1;
    if (kind == 2) {
        cc_weights(N, w);
        // ascending on [0,1]: y_j = sin^2(pi j / (2N)); mirror the upper half
        for (int j = 0; j <= N / 2; j++) {
            double s = sin(kPi * (double)j / (2.0 * N));
            x[j] = s * s;
        }
        for (int j = N / 2 + 1; j <= N; j++) x[j] = 1.0 - x[N - j];
        x[N / 2] = 0.5;
        x[0] = 0.0;
        x[N] = 1.0;
        for (int j = 0; j <= N; j++) w[j] *= 0.5;
        // weights are symmetric: w_j (for cos(pi j/N) on [-1,1]) maps to y_{N-j}
        for (int j = 0; j < N / 2; j++) {
            double t = w[j];
            w[j] = w[N - j];
            w[N - j] = t;
        }
        return n;
    }
    for (int j = 0; j <= N; j++) {  // trapezoid
        x[j] = (double)j / (double)N;
        w[j] = 1.0 / (double)N;
    }
    w[0] *= 0.5;
    w[N] *= 0.5;
    return n;
}

// ---- blocks --------------------------------------------------------------

int sg_block(int kind, int bk, int k, double *x, double *w) {
    if (k < 1 || k + 1 > SG_MAX_LEVEL) return 0;
    static thread_local double xa[(1 << (SG_MAX_LEVEL - 1)) + 1], wa[(1 << (SG_MAX_LEVEL - 1)) + 1];
    static thread_local double xb[(1 << (SG_MAX_LEVEL - 1)) + 1], wb[(1 << (SG_MAX_LEVEL - 1)) + 1];
    int n = sg_rule_level(kind, k + 1, xa, wa);
    if (n == 0) return 0;
    if (bk == SG_BLK_FULL) {
        memcpy(x, xa, sizeof(double) * n);
        memcpy(w, wa, sizeof(double) * n);
        return n;
    }
    if (bk == SG_BLK_TAIL) {
        // J^{k+1} - J^1: subtract weight 1 at the centre
        memcpy(x, xa, sizeof(double) * n);
        memcpy(w, wa, sizeof(double) * n);
        for (int j = 0; j < n; j++)
            if (x[j] == 0.5) { w[j] -= 1.0; return n; }
        x[n] = 0.5;
        w[n] = -1.0;
        return n + 1;
    }
    if (bk == SG_BLK_NEW) {
        // the nodes of level k+1 that no level <= k has (nested rules repeat
        // their coarser nodes bit for bit; Gauss-Legendre levels share only
        // the centre); the weights of a merged-form point come from a
        // per-pattern table, so the block carries weight 1
        if (sg_level_member(kind, k + 1) == sg_level_member(kind, k)) return 0;
        std::vector<double> old;
        for (int l = 1; l <= k; l++) {
            const int m = sg_rule_level(kind, l, xb, wb);
            old.insert(old.end(), xb, xb + m);
        }
        std::sort(old.begin(), old.end());
        int c = 0;
        for (int j = 0; j < n; j++)
            if (!std::binary_search(old.begin(), old.end(), xa[j])) {
                x[c] = xa[j];
                w[c] = 1.0;
                c++;
            }
        return c;
    }
    // difference rule; zero (empty block) when both levels use the same member
    if (sg_level_member(kind, k + 1) == sg_level_member(kind, k)) return 0;
    int n0 = sg_rule_level(kind, k, xb, wb);
    memcpy(x, xa, sizeof(double) * n);
    memcpy(w, wa, sizeof(double) * n);
    if ((kind & 15) == 4) {  // not nested: concatenate with negated weights
        for (int j = 0; j < n0; j++) {
            x[n + j] = xb[j];
            w[n + j] = -wb[j];
        }
        return n + n0;
    }
    if (n0 == 1) {
        w[n / 2] -= wb[0];
    } else {
        // node j of the coarser member is node 2j of the finer one (trapezoid,
        // Clenshaw-Curtis: shared ends) or node 2j + 1 (Gauss-Patterson: one new
        // node in every gap)
        const int shift = (kind & 15) == 3 ? 1 : 0;
        for (int j = 0; j < n0; j++) w[2 * j + shift] -= wb[j];
    }
    return n;
}

int sg_block_size(int kind, int bk, int k) {
    int n = sg_level_nodes(kind, k + 1);
    if (n == 0 || k < 1) return 0;
    if (bk == SG_BLK_NEW) {
        static thread_local double x[2 * 4097 + 2], w[2 * 4097 + 2];
        return sg_block(kind, bk, k, x, w);
    }
    if (bk == SG_BLK_FULL) return n;
    if (bk == SG_BLK_TAIL) return (n % 2) ? n : n + 1;
    if (sg_level_member(kind, k + 1) == sg_level_member(kind, k)) return 0;
    return (kind & 15) == 4 ? n + sg_level_nodes(kind, k) : n;
}
