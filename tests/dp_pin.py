"""Independent high-precision Smolyak value for separable integrands.

Every test family is a product of one-dimensional factors,
f(x) = prod_i g_i(x_i) (the oscillatory one as the real part of a complex
product).  For such f the Smolyak sum over all multi-indices with |k| <= L of
tensor products of difference rules factorises: with
P_i(z) = sum_k (Delta_{k+1} g_i) z^k, the value is the sum of the
coefficients of z^0..z^L of prod_i P_i(z).  This takes O(d L^2) work and
never visits a point, so it checks the oracle's point enumeration, its
per-point evaluation and its summation by a different algorithm.  It is
evaluated in mpmath at 40 digits from the oracle's 1-D rules (the rules are
pinned separately against numpy and moment equations).

Delta_{k+1} g = J^{k+1} g - J^k g is formed from the two full rules, not from
the oracle's merged difference-rule nodes.
"""
import mpmath as mp
import numpy as np

import oracle

mp.mp.dps = 40


def _factor(fam, a, u, i, d, deriv=None):
    """g_i as an mpmath function of x (complex for the oscillatory family).
    deriv: None, 'a' or 'u' -> d g_i / d a_i or d g_i / d u_i."""
    ai, ui = a[i], u[i]
    if fam == 0:
        if deriv == 'a':
            return lambda x: x * mp.exp(ai * x)
        if deriv == 'u':
            return lambda x: mp.mpf(0)
        return lambda x: mp.exp(ai * x)
    if fam == 1:
        if deriv == 'a':
            return lambda x: 1j * x * mp.expj(ai * x)
        if deriv == 'u':
            return lambda x: mp.mpf(0)
        return lambda x: mp.expj(ai * x)
    if fam == 2:
        if deriv == 'a':
            return lambda x: 2 / ai**3 / (1 / ai**2 + (x - ui)**2)**2
        if deriv == 'u':
            return lambda x: 2 * (x - ui) / (1 / ai**2 + (x - ui)**2)**2
        return lambda x: 1 / (1 / ai**2 + (x - ui)**2)
    if fam == 3:
        if deriv == 'a':
            return lambda x: -2 * ai * (x - ui)**2 * mp.exp(-ai**2 * (x - ui)**2)
        if deriv == 'u':
            return lambda x: 2 * ai**2 * (x - ui) * mp.exp(-ai**2 * (x - ui)**2)
        return lambda x: mp.exp(-ai**2 * (x - ui)**2)
    if fam == 4:
        if deriv == 'a':
            return lambda x: -(x - ui)**2 * mp.exp(-ai * (x - ui)**2)
        if deriv == 'u':
            return lambda x: 2 * ai * (x - ui) * mp.exp(-ai * (x - ui)**2)
        return lambda x: mp.exp(-ai * (x - ui)**2)
    raise ValueError(fam)


class _Rules:
    def __init__(self, kind, L):
        self.r = []
        for lev in range(1, L + 2):
            x, w = oracle.rule(kind, lev)
            self.r.append(([mp.mpf(float(v)) for v in x], [mp.mpf(float(v)) for v in w]))

    def apply(self, lev, g):
        x, w = self.r[lev - 1]
        return mp.fsum(wi * g(xi) for xi, wi in zip(x, w))

    def poly(self, g, L):
        J = [self.apply(lev, g) for lev in range(1, L + 2)]
        return [J[0]] + [J[k] - J[k - 1] for k in range(1, L + 1)]


def _mul(p, q, L):
    r = [mp.mpc(0)] * (L + 1)
    for s, ps in enumerate(p):
        if ps == 0:
            continue
        for k in range(L + 1 - s):
            r[s + k] += ps * q[k]
    return r


def _params(params, d):
    a = [mp.mpf(float(v)) for v in params[:d]]
    u = [mp.mpf(float(v)) for v in params[d:2 * d]]
    return a, u


def smolyak_value(kind, fam, params, d, L):
    """Exact (40-digit) Smolyak value of the rule built from the oracle's
    1-D rules, as an mpmath number."""
    a, u = _params(params, d)
    R = _Rules(kind, L)
    acc = [mp.mpc(1)] + [mp.mpc(0)] * L
    for i in range(d):
        acc = _mul(acc, R.poly(_factor(fam, a, u, i, d), L), L)
    tot = mp.fsum(acc)
    if fam == 1:
        return mp.re(mp.expj(2 * mp.pi * u[0]) * tot)
    return mp.re(tot)


def smolyak_gradient(kind, fam, params, d, L, idx):
    """Exact derivatives of the Smolyak value w.r.t. params[idx[t]]."""
    a, u = _params(params, d)
    R = _Rules(kind, L)
    P = [R.poly(_factor(fam, a, u, i, d), L) for i in range(d)]
    pre = [[mp.mpc(1)] + [mp.mpc(0)] * L]
    for i in range(d):
        pre.append(_mul(pre[-1], P[i], L))
    suf = [[mp.mpc(1)] + [mp.mpc(0)] * L]
    for i in reversed(range(d)):
        suf.append(_mul(suf[-1], P[i], L))
    suf = suf[::-1]  # suf[i] = prod_{t >= i}
    phase = mp.expj(2 * mp.pi * u[0]) if fam == 1 else mp.mpf(1)
    out = []
    for j in idx:
        is_u = j >= d
        i = j - d if is_u else j
        if fam == 1 and is_u:
            if i == 0:
                tot = mp.fsum(_mul(pre[i], suf[i], L))
                out.append(mp.re(2j * mp.pi * phase * tot))
            else:
                out.append(mp.mpf(0))
            continue
        dP = R.poly(_factor(fam, a, u, i, d, 'u' if is_u else 'a'), L)
        rest = _mul(pre[i], suf[i + 1], L)
        tot = mp.fsum(_mul(rest, dP, L))
        out.append(mp.re(phase * tot))
    return out


def rel_err(mant, exp2, ref):
    v = mp.ldexp(mp.mpf(float(mant)), int(exp2))
    return float(abs(v - ref) / abs(ref))


def sample_idx(d, n=20, seed=7):
    """n parameter indices spread over a and u (fixed, reproducible)."""
    rng = np.random.default_rng(seed)
    k = min(n, 2 * d)
    return sorted(rng.choice(2 * d, size=k, replace=False).tolist())


def smolyak_value_f64(kind, fam, params, d, L):
    """The same separable DP in numpy float64 (fast; for many items at the
    mixed-precision tolerance).  Returns (rel, logscale): the value is
    exp(logscale) * rel for the exponential families, rel for oscillatory."""
    params = np.asarray(params, dtype=np.float64)
    a, u = params[:d], params[d:2 * d]
    rules = [oracle.rule(kind, lev) for lev in range(1, L + 2)]
    P = np.zeros((d, L + 1), dtype=complex)
    logscale = 0.0
    for lev, (x, w) in enumerate(rules):
        X = x[None, :]
        if fam == 0:
            g = np.exp(a[:, None] * (X - 0.5))
        elif fam == 1:
            g = np.exp(1j * a[:, None] * (X - 0.5))
        elif fam == 2:
            g = (1 / a[:, None] ** 2 + (0.5 - u[:, None]) ** 2) / (1 / a[:, None] ** 2 + (X - u[:, None]) ** 2)
        elif fam == 3:
            g = np.exp(-a[:, None] ** 2 * (X - 0.5) * (X + 0.5 - 2 * u[:, None]))
        else:
            g = np.exp(-a[:, None] * (X - 0.5) * (X + 0.5 - 2 * u[:, None]))
        P[:, lev] = g @ w
    D = np.concatenate([P[:, :1], P[:, 1:] - P[:, :-1]], axis=1)
    acc = np.zeros(L + 1, dtype=complex)
    acc[0] = 1
    for i in range(d):
        new = np.zeros(L + 1, dtype=complex)
        for k in range(L + 1):
            new[k:] += D[i, k] * acc[:L + 1 - k]
        acc = new
    tot = acc.sum()
    if fam == 1:
        th = 2 * np.pi * u[0] + 0.5 * a.sum()
        return float((np.exp(1j * th) * tot).real), 0.0
    if fam == 0:
        logscale = 0.5 * a.sum()
    elif fam == 2:
        logscale = -np.sum(np.log(1 / a ** 2 + (0.5 - u) ** 2))
    elif fam == 3:
        logscale = -np.sum(a ** 2 * (0.5 - u) ** 2)
    else:
        logscale = -np.sum(a * (0.5 - u) ** 2)
    return float(tot.real), float(logscale)
