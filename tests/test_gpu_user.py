"""User integrands compiled at run time (sg_integrand_create / sg_integrate_user)
against the oracle's test families 10-13, the exact integral of a polynomial,
and the built-in exp-linear family through the same interface."""
import math

import numpy as np
import pytest

import oracle
import sg_inputs as si
import user_integrands as ui

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2210_14313_gb300 as sg  # noqa: E402


@pytest.fixture(scope="module")
def integrands():
    out = {name: sg.Integrand(src, k) for name, (src, k, _) in ui.CASES.items()}
    out["explin"] = sg.Integrand(ui.EXPLIN, 2)
    return out


@pytest.fixture(scope="module")
def rules():
    return {"cc": sg.Rule(sg.RULE_CLENSHAW_CURTIS, max_level=8),
            "gl": sg.Rule(sg.RULE_GAUSS_LEGENDRE, max_level=8),
            "gp": sg.Rule(sg.RULE_GAUSS_PATTERSON, max_level=13, growth=sg.GROWTH_SLOW)}


KINDS = {"cc": 2, "gl": 4, "gp": 3 | oracle.SLOW}


def _params(fam, d, seed):
    rng = np.random.default_rng(seed)
    a = rng.uniform(0.2, 1.0, d)
    u = rng.uniform(0.0, 1.0, d)
    if fam == 10:
        a = a * (2.0 / a.sum())
    return np.concatenate([a, u])


@pytest.mark.parametrize("name", list(ui.CASES))
@pytest.mark.parametrize("rule,d,L", [("cc", 6, 4), ("gl", 12, 3), ("gp", 5, 7), ("cc", 40, 2)])
def test_user_integrands_match_oracle(integrands, rules, name, rule, d, L):
    fam = ui.CASES[name][2]
    p = _params(fam, d, 100 + d + L)
    r = sg.integrate_user(rules[rule], integrands[name], p, d, d + L)
    o = oracle.integrate(KINDS[rule], fam, p, d, L)
    # f(x) - f(c) is formed per point; its rounding is amplified by the
    # conditioning of the signed sum (the oracle's, which sums every point)
    tol = max(1e-12, 8 * 2.0 ** -53 * o.cond)
    assert abs(r.value - o.value) <= tol * abs(o.value), (name, rule, d, L, r.value, o.value, o.cond)
    assert r.points == oracle.count_points(KINDS[rule], d, L)


def test_user_polynomial_is_exact(integrands, rules):
    for rule, d, L in [("cc", 30, 1), ("gl", 10, 3), ("gp", 8, 2)]:
        p = _params(13, d, 7 + d)
        a, u = p[:d], p[d:]
        m = a.sum() / 2
        exact = m ** 3 + m * (a * a).sum() / 4 + (u.sum() / 2) ** 2 + (u * u).sum() / 12
        r = sg.integrate_user(rules[rule], integrands["poly"], p, d, d + L)
        assert abs(r.value - exact) <= 1e-12 * abs(exact), (rule, d, L)


def test_user_path_reproduces_a_built_in_family(integrands, rules):
    # exp(sum a_i x_i) through the user interface (with its own deviation) and
    # through the built-in exp-linear fold
    for rule, d, L in [("cc", 20, 3), ("gl", 12, 4)]:
        p = np.concatenate([si.item_params(si.FAM_EXP_LINEAR, d, 3 + d)[:d], np.zeros(d)])
        r = sg.integrate_user(rules[rule], integrands["explin"], p, d, d + L)
        b = sg.integrate(rules[rule], si.FAM_EXP_LINEAR, p, d, d + L, prec=sg.PREC_FP64)
        assert abs(r.value - b.value) <= 1e-13 * abs(b.value)


def test_user_params_on_device(integrands, rules):
    d, L = 8, 3
    p = _params(12, d, 5)
    host = sg.integrate_user(rules["cc"], integrands["two_sums"], p, d, d + L)
    dev = sg.integrate_user(rules["cc"], integrands["two_sums"], torch.tensor(p, device="cuda"), d, d + L)
    assert host.value == dev.value


def test_compile_error_is_reported():
    with pytest.raises(sg.SgError) as e:
        sg.Integrand(ui.BROKEN, 1)
    assert "undefined_name" in e.value.log


def test_user_centre_only_rule(integrands, rules):
    # q = d: the Smolyak rule is the centre point with weight 1
    d = 7
    p = _params(12, d, 3)
    r = sg.integrate_user(rules["cc"], integrands["two_sums"], p, d, d)
    a, u = p[:d], p[d:]
    assert r.value == pytest.approx(0.5 * a.sum() * math.exp(-0.25 * u.sum()), rel=1e-15)
    assert r.points == 1
