"""CUDA sources of user integrands (sg_integrand_create) matching the oracle's
test families 10-13 (parameters: a = p[0..d), u = p[d..2d)), shared by the
CPU compile check and the GPU tests."""

CORNER = r"""
// f = (1 + sum a_i x_i)^-(d+1); state: (1 + sum a_i / 2, sum a_i (x_i - 1/2))
__device__ void sg_user_centre(double *s, const double *p, int d) {
    double t = 1.0;
    for (int i = 0; i < d; i++) t += 0.5 * p[i];
    s[0] = t;
    s[1] = 0.0;
}
__device__ void sg_user_move(double *s, int i, double x, const double *p, int d) { s[1] += p[i] * (x - 0.5); }
__device__ double sg_user_value(const double *s, const double *p, int d) {
    return pow(s[0] + s[1], -(double)(d + 1));
}
"""

CORNER_DEV = CORNER + r"""
#define SG_USER_DEVIATION
// (c + t)^-(d+1) - c^-(d+1) = c^-(d+1) expm1(-(d+1) log1p(t / c))
__device__ double sg_user_deviation(const double *s, const double *sc, const double *p, int d) {
    return pow(s[0], -(double)(d + 1)) * expm1(-(double)(d + 1) * log1p(s[1] / s[0]));
}
"""

NORM = r"""
// f = exp(-sqrt(sum a_i (x_i - u_i)^2)); state: the sum
__device__ void sg_user_centre(double *s, const double *p, int d) {
    double t = 0.0;
    for (int i = 0; i < d; i++) t += p[i] * (0.5 - p[d + i]) * (0.5 - p[d + i]);
    s[0] = t;
}
__device__ void sg_user_move(double *s, int i, double x, const double *p, int d) {
    const double u = p[d + i];
    s[0] += p[i] * ((x - u) * (x - u) - (0.5 - u) * (0.5 - u));
}
__device__ double sg_user_value(const double *s, const double *p, int d) { return exp(-sqrt(fmax(s[0], 0.0))); }
"""

TWO_SUMS = r"""
// f = (sum a_i x_i) exp(-sum u_i x_i^2); state: both sums
__device__ void sg_user_centre(double *s, const double *p, int d) {
    double t0 = 0.0, t1 = 0.0;
    for (int i = 0; i < d; i++) {
        t0 += 0.5 * p[i];
        t1 += 0.25 * p[d + i];
    }
    s[0] = t0;
    s[1] = t1;
}
__device__ void sg_user_move(double *s, int i, double x, const double *p, int d) {
    s[0] += p[i] * (x - 0.5);
    s[1] += p[d + i] * (x * x - 0.25);
}
__device__ double sg_user_value(const double *s, const double *p, int d) { return s[0] * exp(-s[1]); }
"""

POLY = r"""
// f = (sum a_i x_i)^3 + (sum u_i x_i)^2; state: both sums
__device__ void sg_user_centre(double *s, const double *p, int d) {
    double t0 = 0.0, t1 = 0.0;
    for (int i = 0; i < d; i++) {
        t0 += 0.5 * p[i];
        t1 += 0.5 * p[d + i];
    }
    s[0] = t0;
    s[1] = t1;
}
__device__ void sg_user_move(double *s, int i, double x, const double *p, int d) {
    s[0] += p[i] * (x - 0.5);
    s[1] += p[d + i] * (x - 0.5);
}
__device__ double sg_user_value(const double *s, const double *p, int d) {
    return s[0] * s[0] * s[0] + s[1] * s[1];
}
"""

# exp-linear through the user interface (checks it against the built-in family)
EXPLIN = r"""
#define SG_USER_DEVIATION
// f = exp(sum a_i x_i); state: (sum a_i / 2, sum a_i (x_i - 1/2))
__device__ void sg_user_centre(double *s, const double *p, int d) {
    double c = 0.0;
    for (int i = 0; i < d; i++) c += 0.5 * p[i];
    s[0] = c;
    s[1] = 0.0;
}
__device__ void sg_user_move(double *s, int i, double x, const double *p, int d) { s[1] += p[i] * (x - 0.5); }
__device__ double sg_user_value(const double *s, const double *p, int d) { return exp(s[0] + s[1]); }
__device__ double sg_user_deviation(const double *s, const double *sc, const double *p, int d) {
    return exp(s[0]) * expm1(s[1]);
}
"""

BROKEN = r"""
__device__ void sg_user_centre(double *s, const double *p, int d) { s[0] = undefined_name; }
"""

# (source, state size, oracle family)
CASES = {"corner": (CORNER, 2, 10), "corner_dev": (CORNER_DEV, 2, 10), "norm": (NORM, 1, 11),
         "two_sums": (TWO_SUMS, 2, 12), "poly": (POLY, 2, 13)}
