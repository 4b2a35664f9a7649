"""The reduction's exact summations, built for the host: the 128-bit window
of sg_xsum.h and the long accumulator of sg_lacc.h, against exact rational
sums, independent of the order of the terms and of how they are split."""
from fractions import Fraction

import numpy as np
import pytest

import index_check


def _exact(v):
    return sum((Fraction(float(x)) for x in v), Fraction(0))


def _cases():
    rng = np.random.default_rng(11)
    yield rng.standard_normal(64)
    yield rng.standard_normal(2048) * 10.0 ** rng.uniform(-12, 0, 2048)   # 40 binades
    v = rng.standard_normal(1000)
    yield np.concatenate([v, -v[::-1]])                                   # exact cancellation
    yield np.array([1.0, 2.0 ** -53, 2.0 ** -53, -1.0])                    # rounding-tie residue
    yield np.array([1e10, -1e10, 3.0, 1e-3])                               # cancellation, in the window
    yield np.array([0.0, -0.0, 0.0])
    yield rng.uniform(0, 1, 5000) * 1e-200


@pytest.mark.parametrize("k", range(7))
def test_window_sum_is_exact(k):
    v = list(_cases())[k]
    s, c = index_check.xsum(v)
    ex = _exact(v)
    # s is the double nearest the exact sum, s + c carries the rest
    assert s == float(ex)
    rest = ex - Fraction(s)
    assert c == float(rest)
    # any order gives the same pair
    rng = np.random.default_rng(k)
    assert index_check.xsum(rng.permutation(v)) == (s, c)


def test_terms_below_the_window_truncate_symmetrically():
    # the window ends 2^-104 below the largest term: what cancels above it
    # leaves only what lies inside it
    assert index_check.xsum(np.array([1e300, -1e300, 3.0, 1e-3])) == (0.0, 0.0)
    # a term 2^-120 below the largest falls under the unit 2^-(56 + 52) of it
    v = np.array([1.0, 2.0 ** -120, -(2.0 ** -120)])
    assert index_check.xsum(v) == (1.0, 0.0)
    v = np.array([1.0, 2.0 ** -120])
    assert index_check.xsum(v) == (1.0, 0.0)


@pytest.mark.parametrize("k", [0, 1, 2, 3, 6])
@pytest.mark.parametrize("nthreads", [1, 7, 256])
def test_adaptive_units_match_the_exact_sum(k, nthreads):
    # the setup kernel's running sums: units follow each thread's largest term;
    # growing units truncate at most 2^-104 of the largest term per step
    v = list(_cases())[k]
    s, c = index_check.xsum_adaptive(v, nthreads)
    ex = _exact(v)
    big = max(abs(float(x)) for x in v) if len(v) else 0.0
    err = abs(Fraction(s) + Fraction(c) - ex)
    assert err <= Fraction(len(v)) * Fraction(big) * Fraction(2) ** -103
    assert index_check.xsum_adaptive(v, nthreads) == (s, c)


def _lacc_cases():
    rng = np.random.default_rng(5)
    for v in list(_cases())[:6]:  # the seventh lies wholly below the window (2^-576)
        yield v
    yield rng.standard_normal(3000) * 10.0 ** rng.uniform(-150, 130, 3000)   # 280 binades
    yield np.array([2.0 ** 446, -(2.0 ** 446), 2.0 ** -570, 1.0])             # both window ends
    yield -rng.uniform(0, 1, 777)                                             # negative sum


@pytest.mark.parametrize("k", range(9))
@pytest.mark.parametrize("nparts", [1, 3, 152])
def test_long_accumulator_is_exact_and_split_invariant(k, nparts):
    v = list(_lacc_cases())[k]
    s, c, ovf = index_check.lacc(v, nparts)
    assert ovf == 0
    ex = _exact(v)
    # the top 128 bits of the sum are kept: s is the nearest double to the
    # exact sum (none of these cases sits near a tie), s + c within 2^-96
    assert s == float(ex)
    assert abs(Fraction(s) + Fraction(c) - ex) <= abs(ex) * Fraction(2) ** -96
    rng = np.random.default_rng(k)
    assert index_check.lacc(rng.permutation(v), 7) == (s, c, 0)


def test_long_accumulator_window_ends():
    # below 2^-576 a term is cut towards zero; from 2^447 on it overflows
    assert index_check.lacc(np.array([1.0, 2.0 ** -600]))[:2] == (1.0, 0.0)
    assert index_check.lacc(np.array([2.0 ** -570, 2.0 ** -600]))[:2] == (2.0 ** -570, 0.0)
    assert index_check.lacc(np.array([1.0, 2.0 ** 447]))[2] == 1
    assert index_check.lacc(np.array([1.0, float("inf")]))[2] == 1
    assert index_check.lacc(np.array([1.0, float("nan")]))[2] == 1
    assert index_check.lacc(np.array([0.0, -0.0])) == (0.0, 0.0, 0)


@pytest.mark.parametrize("k", range(6))
@pytest.mark.parametrize("nparts", [1, 4, 37])
def test_long_accumulator_fed_exact_window_sums(k, nparts):
    # each part's terms lie within 40 binades, so its 128-bit window sum is
    # exact and enters the limbs digit by digit without rounding: the total
    # is the exact sum, the same as with the terms fed one by one
    v = list(_cases())[k]
    s, c, ovf, amag = index_check.lacc_x(v, nparts)
    assert ovf == 0
    ex = _exact(v)
    assert s == float(ex)
    assert abs(Fraction(s) + Fraction(c) - ex) <= abs(ex) * Fraction(2) ** -96
    assert (s, c) == index_check.lacc(v, nparts)[:2]
    parts = [_exact(v[len(v) * p // nparts:len(v) * (p + 1) // nparts]) for p in range(nparts)]
    # (rounded once: ties away from zero, so within half an ulp)
    mag = sum(abs(x) for x in parts)
    assert abs(Fraction(amag) - mag) <= mag * Fraction(2) ** -53


def test_exact_window_digits_at_every_offset():
    # one term per part, its unit stepping through every offset of the
    # 32-bit digit grid (and across the ends of the 128-bit window sum)
    rng = np.random.default_rng(9)
    for e in range(-500, 420, 7):  # terms keep all their bits above 2^-576
        v = rng.standard_normal(3) * 2.0 ** e
        s, c, ovf, _ = index_check.lacc_x(v, 3)
        assert ovf == 0
        # exact: the sum of three terms has at most 55 bits (a tie between two
        # doubles rounds away from zero)
        assert Fraction(s) + Fraction(c) == _exact(v)
        assert abs(Fraction(s) - _exact(v)) <= abs(_exact(v)) * Fraction(2) ** -53
        assert index_check.lacc_x(-v, 3)[:2] == (-s, -c)


def test_exact_window_digits_window_ends():
    # below 2^-576 a part's sum is cut towards zero; from 2^447 on, and for
    # infinite or NaN terms, the overflow flag is set
    assert index_check.lacc_x(np.array([1.0, 2.0 ** -600]), 2)[:2] == (1.0, 0.0)
    assert index_check.lacc_x(np.array([2.0 ** -570, 2.0 ** -600]), 2)[:2] == (2.0 ** -570, 0.0)
    assert index_check.lacc_x(np.array([1.0, 2.0 ** 447]), 2)[2] == 1
    assert index_check.lacc_x(np.array([2.0 ** 446, 2.0 ** 446]), 1)[2] == 1   # the part's sum is 2^447
    assert index_check.lacc_x(np.array([2.0 ** 446, 2.0 ** 445]), 1)[2] == 0
    assert index_check.lacc_x(np.array([1.0, float("inf")]), 1)[2] == 1
    assert index_check.lacc_x(np.array([1.0, float("nan")]), 2)[2] == 1
    assert index_check.lacc_x(np.array([0.0, -0.0]), 1)[:3] == (0.0, 0.0, 0)


def test_ratio_to_float_precision():
    # the condition number's quotient: within float rounding of the exact
    # quotient for normal operands over the whole exponent range, the double
    # division for zeros, subnormals, infinities and NaNs
    rng = np.random.default_rng(4)
    a = rng.uniform(0.5, 1, 20000) * 2.0 ** rng.integers(-500, 500, 20000)  # quotients stay normal
    b = rng.uniform(0.5, 1, 20000) * 2.0 ** rng.integers(-500, 500, 20000)
    q = index_check.ratio(a, b)
    exact = [Fraction(x) / Fraction(y) for x, y in zip(a[:2000], b[:2000])]
    for qi, e in zip(q[:2000], exact):
        assert abs(Fraction(qi) - e) <= e * Fraction(2) ** -22
    ref = a / b
    ok = np.isfinite(ref) & (ref > 0)
    assert np.all(np.abs(q[ok] - ref[ok]) <= 2.0 ** -22 * ref[ok])
    special = index_check.ratio(np.array([0.0, 1.0, 5e-324, 1.0, np.inf, 1.0, 3.0]),
                                np.array([1.0, 0.0, 1.0, 5e-324, 1.0, np.nan, 3.0]))
    assert special[0] == 0.0 and special[1] == np.inf and special[2] == 5e-324
    assert special[3] == 1.0 / 5e-324 and special[4] == np.inf and np.isnan(special[5])
    assert special[6] == 1.0
