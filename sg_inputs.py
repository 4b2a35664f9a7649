"""Seeded synthetic inputs for the sparse-grid quadrature workloads.

This module holds no quadrature arithmetic: it only draws integrand parameters
and batch metadata.  Both the CPU oracle tests and the GPU path take their
inputs from here, so the two sides always integrate the same functions.

Random numbers come from SplitMix64 (G. L. Steele, D. Lea, C. H. Flood,
"Fast splittable pseudorandom number generators", OOPSLA 2014), turned into
doubles in [0, 1) from the top 53 bits.

Parameter layout, shared by every family: ``params = [a_0..a_{d-1}, u_0..u_{d-1}]``
(2d doubles).  Which entries a family reads:

* exp-linear   f = exp(sum a_i x_i)                       -> a (u unused)
* oscillatory  f = cos(2 pi u_0 + sum a_i x_i)            -> a, u_0
* product peak f = prod 1 / (a_i^-2 + (x_i - u_i)^2)      -> a, u
* gaussian     f = exp(-sum a_i^2 (x_i - u_i)^2)          -> a, u
* gaussian-lin f = exp(-sum a_i (x_i - u_i)^2)            -> a, u

These are the Genz-type test families of the paper's Section 4 and 5 tests,
on the unit cube [0,1]^d.  Draw order for one integrand: a_0..a_{d-1}, then
u_0..u_{d-1} (only u_0 for the oscillatory family), then a is rescaled.
"""
from __future__ import annotations

import numpy as np

MASK64 = (1 << 64) - 1

# Family and rule codes; they match the values of the C enums in include/sg.h.
FAM_EXP_LINEAR = 0
FAM_OSCILLATORY = 1
FAM_PRODUCT_PEAK = 2
FAM_GAUSSIAN = 3
FAM_GAUSSIAN_LIN = 4
FAMILY_NAMES = {0: "exp_linear", 1: "oscillatory", 2: "product_peak",
                3: "gaussian", 4: "gaussian_lin"}

RULE_TRAPEZOID = 1
RULE_CLENSHAW_CURTIS = 2
RULE_GAUSS_LEGENDRE = 4
RULE_NAMES = {1: "trapezoid", 2: "clenshaw_curtis", 4: "gauss_legendre"}


class SplitMix64:
    """SplitMix64 stream (Steele, Lea & Flood 2014)."""

    def __init__(self, seed: int):
        self.state = seed & MASK64

    def next_u64(self) -> int:
        self.state = (self.state + 0x9E3779B97F4A7C15) & MASK64
        z = self.state
        z = ((z ^ (z >> 30)) * 0xBF58476D1CE4E5B9) & MASK64
        z = ((z ^ (z >> 27)) * 0x94D049BB133111EB) & MASK64
        return z ^ (z >> 31)

    def uniform(self) -> float:
        """Double in [0, 1) from the top 53 bits."""
        return (self.next_u64() >> 11) * (1.0 / 9007199254740992.0)

    def uniforms(self, n: int) -> np.ndarray:
        return np.array([self.uniform() for _ in range(n)], dtype=np.float64)

    def randint(self, lo: int, hi: int) -> int:
        """Integer uniform on {lo, ..., hi} (inclusive)."""
        return lo + min(int(self.uniform() * (hi - lo + 1)), hi - lo)


def family_params(fam: int, d: int, seed: int, *, sum_a: float | None = None,
                  a_lo: float = 0.0, a_hi: float = 1.0, a_scale: float = 1.0) -> np.ndarray:
    """Draw the 2d parameters of one integrand.

    a_i ~ U(a_lo, a_hi), multiplied by ``a_scale``; if ``sum_a`` is given, a is
    then rescaled so that sum a_i = sum_a.  u_i ~ U(0, 1).
    """
    g = SplitMix64(seed)
    a = a_lo + (a_hi - a_lo) * g.uniforms(d)
    u = np.zeros(d)
    if fam == FAM_OSCILLATORY:
        u[0] = g.uniform()
    elif fam != FAM_EXP_LINEAR:
        u[:] = g.uniforms(d)
    a = a * a_scale
    if sum_a is not None:
        a = a * (sum_a / a.sum())
    return np.concatenate([a, u])


# --- the five workloads -----------------------------------------------------

SEED_CFG1 = 0x5EED0001
SEED_CFG2 = 0x5EED0002
SEED_CFG3 = 0x5EED0003
SEED_CFG4 = 0x5EED0004
SEED_CFG5 = 0x5EED0005


def _config(name, rule, fam, d, L, seed, **draw_kw):
    return dict(name=name, rule=rule, fam=fam, d=d, L=L, seed=seed, draw_kw=draw_kw,
                params=family_params(fam, d, seed, **draw_kw))


def cfg1():
    """d=4, Clenshaw-Curtis, q=d+5, exp-linear with c_i ~ U(0,1)."""
    return _config("cfg1_d4_cc_L5_explinear", RULE_CLENSHAW_CURTIS, FAM_EXP_LINEAR, 4, 5, SEED_CFG1)


def cfg2():
    """d=12, Gauss-Legendre (level i has i nodes), q=d+6, oscillatory,
    a_i ~ U(0,1) rescaled to sum 4.5, u_0 ~ U(0,1)."""
    return _config("cfg2_d12_gl_L6_oscillatory", RULE_GAUSS_LEGENDRE, FAM_OSCILLATORY, 12, 6, SEED_CFG2,
                   sum_a=4.5)


def cfg3(fam: int = FAM_PRODUCT_PEAK):
    """d=100, Clenshaw-Curtis, q=d+3, product peak or gaussian,
    a_i ~ U(0,1) rescaled to sum 7, u_i ~ U(0,1)."""
    return _config("cfg3_d100_cc_L3_" + FAMILY_NAMES[fam], RULE_CLENSHAW_CURTIS, fam, 100, 3, SEED_CFG3 + fam,
                   sum_a=7.0)


def cfg5():
    """d=1000, Clenshaw-Curtis, q=d+2, gaussian-lin with a_i ~ U(0.5,1.5)/d."""
    d = 1000
    return _config("cfg5_d1000_cc_L2_gaussian_lin", RULE_CLENSHAW_CURTIS, FAM_GAUSSIAN_LIN, d, 2, SEED_CFG5,
                   a_lo=0.5, a_hi=1.5, a_scale=1.0 / d)


def redraw(c, j: int) -> np.ndarray:
    """Parameters of draw j of a workload: the same distribution, seed
    c["seed"] + 2^16 j (draw 0 is the workload's own parameters)."""
    return family_params(c["fam"], c["d"], c["seed"] + 0x10000 * j, **c["draw_kw"])


def item_params(fam: int, d: int, seed: int) -> np.ndarray:
    """Parameters of one batch item, drawn as in the single-integral workloads."""
    if fam == FAM_EXP_LINEAR:
        return family_params(fam, d, seed)
    if fam == FAM_OSCILLATORY:
        return family_params(fam, d, seed, sum_a=4.5)
    return family_params(fam, d, seed, sum_a=7.0)


def batch(n: int = 4096, seed: int = SEED_CFG4, d_lo: int = 5, d_hi: int = 200,
          L_lo: int = 2, L_hi: int = 5):
    """Batch of ``n`` integrands: d ~ U{d_lo..d_hi}, q-d ~ U{L_lo..L_hi},
    rule uniform over {CC, GL}, family uniform over {exp-linear, oscillatory,
    product peak, gaussian}.  Metadata and parameters come from separate
    SplitMix64 streams.  Returns a list of dicts (rule, fam, d, L, params)."""
    meta = SplitMix64(seed)
    items = []
    for k in range(n):
        d = meta.randint(d_lo, d_hi)
        L = meta.randint(L_lo, L_hi)
        rule = RULE_CLENSHAW_CURTIS if meta.uniform() < 0.5 else RULE_GAUSS_LEGENDRE
        fam = meta.randint(0, 3)
        pseed = (seed * 0x100000001B3 + (k + 1) * 0x9E3779B97F4A7C15) & MASK64
        items.append(dict(rule=rule, fam=fam, d=d, L=L, params=item_params(fam, d, pseed)))
    return items
