"""Coefficients of the FP64 fold's sin, cos and expm1 polynomials
(sg_fixed.h): weighted minimax fits by the Remez exchange algorithm
(Remez 1934; as in Cheney, Introduction to Approximation Theory, ch. 3),
computed in 60-digit arithmetic with mpmath and rounded to 0.64 fixed point.

    sin r  = r + r^3 S(r^2),          S of degree 5,  |r| <= 0.7854
    cos r  = 1 - r^2/2 + r^4 C(r^2),  C of degree 5,  |r| <= 0.7854
    expm1 x = x + x^2 P(x),           P of degree 10, |x| <= ln2/2

Each fit minimises the relative error of the function itself (the weight is
the factor that turns the polynomial's error into it).  Run as a script to
print the coefficient magnitudes with their signs and each polynomial's
largest relative error on a dense grid, evaluated exactly.
"""
import mpmath as mp

mp.mp.dps = 60


def remez(f, w, a, b, n, iters=40):
    """Degree-n polynomial p minimising max |w (f - p)| on [a, b]."""
    m = n + 2
    # Chebyshev extrema, nudged off the interval's interior zeros of w
    xs = [(a + b) / 2 - (b - a) / 2 * mp.cos(mp.pi * i / (m - 1)) + (b - a) * mp.mpf("1e-3") * (0 < i < m - 1)
          for i in range(m)]
    c = None
    for _ in range(iters):
        A = mp.matrix(m, m)
        rhs = mp.matrix(m, 1)
        for i, x in enumerate(xs):
            for j in range(n + 1):
                A[i, j] = x ** j
            A[i, n + 1] = (-1) ** i / w(x)
            rhs[i] = f(x)
        sol = mp.lu_solve(A, rhs)
        c = [sol[j] for j in range(n + 1)]
        lev = abs(sol[n + 1])
        N = 3000
        grid = [a + (b - a) * mp.mpf(k) / N for k in range(N + 1)]
        ev = [w(x) * (f(x) - mp.polyval(c[::-1], x)) for x in grid]
        ext = [0] + [k for k in range(1, N) if (ev[k] - ev[k - 1]) * (ev[k + 1] - ev[k]) <= 0] + [N]
        alt = []
        for k in ext:
            if alt and mp.sign(alt[-1][1]) == mp.sign(ev[k]):
                if abs(ev[k]) > abs(alt[-1][1]):
                    alt[-1] = (grid[k], ev[k])
            else:
                alt.append((grid[k], ev[k]))
        while len(alt) > m:
            alt.pop(0 if abs(alt[0][1]) < abs(alt[-1][1]) else -1)
        if len(alt) < m:
            break
        xs = [x for x, _ in alt]
        mx = max(abs(e) for _, e in alt)
        if (mx - lev) / mx < mp.mpf(10) ** -6:
            break
    return c


def _sin_t(z):
    r = mp.sqrt(z)
    return mp.mpf(-1) / 6 if z == 0 else (mp.sin(r) - r) / r ** 3


def _sin_w(z):
    r = mp.sqrt(z)
    return mp.mpf(10) ** -40 if z == 0 else r ** 3 / mp.sin(r)


def _cos_t(z):
    return mp.mpf(1) / 24 if z == 0 else (mp.cos(mp.sqrt(z)) - 1 + z / 2) / z ** 2


def _cos_w(z):
    return mp.mpf(10) ** -40 if z == 0 else z ** 2 / mp.cos(mp.sqrt(z))


def _expm1_t(x):
    return mp.mpf(1) / 2 if x == 0 else (mp.expm1(x) - x) / x ** 2


def _expm1_w(x):
    return mp.mpf(10) ** -40 if x == 0 else x ** 2 / abs(mp.expm1(x))


RHO = mp.mpf("0.7854")  # pi/4 and the reduction's rounding
H = mp.log(2) / 2 + mp.mpf("1e-6")
FITS = {
    # name: (target, weight, interval, degree)
    "sin": (_sin_t, _sin_w, (mp.mpf(0), RHO ** 2), 5),
    "cos": (_cos_t, _cos_w, (mp.mpf(0), RHO ** 2), 5),
    "expm1": (_expm1_t, _expm1_w, (-H, H), 10),
}


def fixed_coefficients(name):
    """The fit's coefficient magnitudes in unsigned 0.64 fixed point
    (round(|c| 2^64)) and their signs, lowest degree first: the integer
    evaluation (sg_fixed.h) works on magnitudes."""
    f, w, (a, b), n = FITS[name]
    c = remez(f, w, a, b, n)
    return [int(mp.nint(abs(x) * mp.mpf(2) ** 64)) for x in c], [1 if x > 0 else -1 for x in c]


def fixed_error(name, N=4000):
    """Largest relative error of the polynomial with the fixed-point
    coefficients, evaluated exactly, on a grid of N + 1 points."""
    f, w, (a, b), _ = FITS[name]
    mags, signs = fixed_coefficients(name)
    cm = [sg * mp.mpf(m) / mp.mpf(2) ** 64 for m, sg in zip(mags, signs)]
    return max(abs(w(x) * (f(x) - mp.polyval(cm[::-1], x)))
               for x in (a + (b - a) * mp.mpf(k) / N for k in range(N + 1)))


if __name__ == "__main__":
    for name in FITS:
        mags, signs = fixed_coefficients(name)
        print("%s: largest relative error %.3g; 0.64 magnitudes, lowest degree first:"
              % (name, float(fixed_error(name))))
        for m, sg in zip(mags, signs):
            print("    %s%dull" % ("+" if sg > 0 else "-", m))
