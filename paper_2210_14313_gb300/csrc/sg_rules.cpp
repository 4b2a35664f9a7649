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
//    2 (1 - x^2) / (n P_{n-1}(x))^2.
// Nested rules are generated from the finest level by index, so a node of
// level l-1 is bit-identical to its copy in level l.
#include "sg_rules.h"

#include <math.h>
#include <string.h>

static const double kPi = 3.14159265358979323846;

int sg_level_nodes(int kind, int level) {
    if (level < 1 || level > SG_MAX_LEVEL) return 0;
    if (kind == 4) return level;
    if (kind != 1 && kind != 2) return 0;
    return level == 1 ? 1 : (1 << (level - 1)) + 1;
}

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
    // difference rule
    int n0 = sg_rule_level(kind, k, xb, wb);
    memcpy(x, xa, sizeof(double) * n);
    memcpy(w, wa, sizeof(double) * n);
    if (kind == 4) {  // not nested: concatenate with negated weights
        for (int j = 0; j < n0; j++) {
            x[n + j] = xb[j];
            w[n + j] = -wb[j];
        }
        return n + n0;
    }
    if (n0 == 1) {
        w[n / 2] -= wb[0];
    } else {
        for (int j = 0; j < n0; j++) w[2 * j] -= wb[j];  // node j of level k is node 2j of level k+1
    }
    return n;
}

int sg_block_size(int kind, int bk, int k) {
    int n = sg_level_nodes(kind, k + 1);
    if (n == 0 || k < 1) return 0;
    if (bk == SG_BLK_FULL) return n;
    if (bk == SG_BLK_TAIL) return (n % 2) ? n : n + 1;
    return kind == 4 ? n + sg_level_nodes(kind, k) : n;
}
