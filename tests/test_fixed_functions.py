"""The fixed-point sin, cos and expm1 of the FP64 fold (sg_fixed.h), built
for the host, against mpmath: within about one ulp on the arguments the fold
hands them (|r| <= 0.7854 for sin and cos, |x| <= ln2/2 for expm1)."""
import numpy as np
import pytest

import index_check

mp = pytest.importorskip("mpmath")
U = 2.0 ** -53


def _args(lo, hi, n, seed):
    rng = np.random.default_rng(seed)
    tiny = 10.0 ** -np.arange(1, 30)
    return np.concatenate([rng.uniform(lo, hi, n), tiny, -tiny, [0.0, lo, hi, 1e-310, -1e-310]])


def test_expm1_relative_error():
    mp.mp.dps = 40
    x = _args(-0.3465, 0.3465, 4000, 1)
    y = index_check.fixed(0, x)
    worst = max(abs((mp.mpf(b) - mp.expm1(mp.mpf(a))) / mp.expm1(mp.mpf(a))) for a, b in zip(x, y) if a != 0)
    assert worst <= 1.5 * U, float(worst / U)
    assert y[x == 0].tolist() == [0.0] * int((x == 0).sum())


def test_sin_cos_errors():
    mp.mp.dps = 40
    x = _args(-0.7854, 0.7854, 4000, 2)
    y = index_check.fixed(1, x)
    s, c = y[0::2], y[1::2]
    ws = max(abs((mp.mpf(b) - mp.sin(mp.mpf(a))) / mp.sin(mp.mpf(a))) for a, b in zip(x, s) if a != 0)
    wc = max(abs(mp.mpf(b) - mp.cos(mp.mpf(a))) for a, b in zip(x, c))
    assert ws <= 1.5 * U, float(ws / U)
    assert wc <= 1.0 * U, float(wc / U)


@pytest.mark.parametrize("phi", [0.3, 2.0, -1.2, 4.0, np.pi / 2, 3.0, 1e-3, -2.5e-4])
def test_oscillatory_deviation(phi):
    # sin(H) sin(phi + H) with the phase constants rounded to doubles, as the
    # fold holds them; relative to the FP64 rounding scale
    # |sin H| (|sin phi cos H| + |cos phi sin H|) the error is below 2.5 ulp for
    # phases away from 0 mod pi, and always below |H| 2^-58 in absolute terms
    mp.mp.dps = 40
    x = _args(-0.7854, 0.7854, 1500, 3)
    y = index_check.fixed(2, x, phi)
    sp, cp = mp.mpf(float(np.sin(phi))), mp.mpf(float(np.cos(phi)))
    rel = absw = 0
    for a, b in zip(x, y):
        X = mp.mpf(a)
        ref = mp.sin(X) * (sp * mp.cos(X) + cp * mp.sin(X))
        scale = abs(mp.sin(X)) * (abs(sp * mp.cos(X)) + abs(cp * mp.sin(X)))
        if scale < 1e-290:  # subnormal results: IEEE's own precision limit
            assert abs(b) < 1e-290
            continue
        rel = max(rel, abs(mp.mpf(b) - ref) / scale)
        absw = max(absw, abs(mp.mpf(b) - ref) / abs(X))
    if abs(np.sin(phi)) > 0.1:
        assert rel <= 2.5 * U, float(rel / U)
    assert absw <= 2.0 ** -52, float(absw)


def _weights(n, seed):
    rng = np.random.default_rng(seed)
    w = rng.uniform(-1.0, 1.0, n) * 10.0 ** rng.uniform(-6, 0, n)
    w[:4] = [0.0, 1.0, -1.0, 2.0 ** -1000]
    return w


def test_weighted_expm1():
    # w expm1(x), rounded once from fixed point
    mp.mp.dps = 40
    x = _args(-0.3465, 0.3465, 3000, 4)
    w = _weights(len(x), 5)
    y = index_check.fixed(4, x, w=w)
    worst = 0
    for a, b, c in zip(x, w, y):
        ref = mp.expm1(mp.mpf(a)) * mp.mpf(b)
        if abs(ref) < 1e-290:
            assert abs(c) < 1e-290
            continue
        worst = max(worst, abs((mp.mpf(c) - ref) / ref))
    assert worst <= 1.0 * U, float(worst / U)


@pytest.mark.parametrize("phi", [0.3, 2.0, -1.2, 4.0, 3.0, 1e-3])
def test_weighted_oscillatory_deviation(phi):
    mp.mp.dps = 40
    x = _args(-0.7854, 0.7854, 1500, 6)
    w = _weights(len(x), 7)
    y = index_check.fixed(3, x, phi, w=w)
    sp, cp = mp.mpf(float(np.sin(phi))), mp.mpf(float(np.cos(phi)))
    rel = absw = 0
    for a, b, c in zip(x, w, y):
        X, Wt = mp.mpf(a), mp.mpf(b)
        ref = Wt * mp.sin(X) * (sp * mp.cos(X) + cp * mp.sin(X))
        scale = abs(Wt * mp.sin(X)) * (abs(sp * mp.cos(X)) + abs(cp * mp.sin(X)))
        if scale < 1e-290:
            assert abs(c) < 1e-290
            continue
        rel = max(rel, abs(mp.mpf(c) - ref) / scale)
        absw = max(absw, abs(mp.mpf(c) - ref) / abs(X * Wt))
    if abs(np.sin(phi)) > 0.1:
        assert rel <= 2.0 * U, float(rel / U)
    assert absw <= 2.0 ** -52, float(absw)


def test_fixed_point_to_double_rounds_to_nearest():
    # v 2^-q for 64-bit v: the nearest double (ties away from zero), signed,
    # and zero below the normal range
    from fractions import Fraction
    rng = np.random.default_rng(9)
    v = rng.integers(1, 2 ** 63, 3000, dtype=np.uint64) >> rng.integers(0, 63, 3000).astype(np.uint64)
    v[:4] = [1, 2 ** 53 - 1, 2 ** 53 + 1, 2 ** 63 + 1025]
    neg = rng.integers(0, 2, 3000).astype(np.uint64)
    q = rng.integers(0, 1100, 3000).astype(np.int32)
    y = index_check.fx_to_double(v, neg, q)
    for vi, ni, qi, yi in zip(v.tolist(), neg.tolist(), q.tolist(), y.tolist()):
        ex = Fraction(int(vi), 2 ** int(qi)) * (-1 if ni else 1)
        if abs(ex) < Fraction(2) ** -1022:
            assert yi == 0.0 or abs(Fraction(yi) - ex) <= Fraction(2) ** -1074
            continue
        f = float(ex)  # nearest, ties to even
        err = abs(Fraction(yi) - ex)
        assert err <= abs(Fraction(f) - ex) or err == abs(Fraction(f) - ex), (vi, ni, qi)
        assert abs(Fraction(yi) - ex) <= abs(ex) * Fraction(2) ** -53
