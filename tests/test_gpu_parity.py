"""GPU parity: the CUDA path (through the C ABI) against the CPU oracle.

Bars: FP64 relative error <= 1e-12; the mixed path (float evaluation and
folds, double combination) <= 1e-6 where its own error estimate says the
integrand is conditioned well enough (see test_mixed_guard for the rest).
"""
import math

import numpy as np
import pytest

import oracle
import sg_inputs as si
import dp_pin

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2210_14313_gb300 as sg  # noqa: E402

FP64_TOL = 1e-12
MIXED_TOL = 1e-6
FF_TOL = 1e-9


@pytest.fixture(scope="module")
def rules():
    r = {k: sg.Rule(k, max_level=10) for k in (1, 2, 4)}
    r[3] = sg.Rule(3, max_level=6)
    return r


def rel_err(r, o):
    """Relative error of a GPU Result against an oracle Result (mant, exp2)."""
    return abs(r.mant * 2.0 ** (r.exp2 - o.exp2) - o.mant) / abs(o.mant)


_ORACLE = {}


def oracle_value(c):
    key = (c["rule"], c["fam"], c["d"], c["L"], tuple(np.asarray(c["params"]).tolist()))
    if key not in _ORACLE:
        _ORACLE[key] = oracle.integrate(c["rule"], c["fam"], c["params"], c["d"], c["L"])
    return _ORACLE[key]


CONFIGS = [si.cfg1(), si.cfg2(), si.cfg3(si.FAM_PRODUCT_PEAK), si.cfg3(si.FAM_GAUSSIAN), si.cfg5()]


@pytest.mark.parametrize("form", [sg.FORM_TELESCOPED, sg.FORM_DIFFERENCE])
@pytest.mark.parametrize("c", CONFIGS, ids=lambda c: c["name"])
def test_fp64_configs(rules, c, form):
    r = sg.integrate(rules[c["rule"]], c["fam"], c["params"], c["d"], c["d"] + c["L"],
                     prec=sg.PREC_FP64, form=form)
    assert r.points == oracle.count_points(c["rule"], c["d"], c["L"])
    assert rel_err(r, oracle_value(c)) <= FP64_TOL


@pytest.mark.parametrize("prec", [sg.PREC_FP64, sg.PREC_FF])
@pytest.mark.parametrize("c", CONFIGS + [dict(name="gp_L4", rule=3, fam=1, d=9, L=4, params=si.item_params(1, 9, 31)),
                                         dict(name="trap_L5", rule=1, fam=2, d=6, L=5,
                                              params=si.item_params(2, 6, 32))],
                         ids=lambda c: c["name"])
def test_merged_form(rules, c, prec):
    # every distinct point once with its merged weight (Eq. 2.8): FP64 at the
    # FP64 bar, float-float at its own, the evaluations the distinct points
    r = sg.integrate(rules[c["rule"]], c["fam"], c["params"], c["d"], c["d"] + c["L"], prec=prec,
                     form=sg.FORM_MERGED)
    assert r.points == oracle.count_points(c["rule"], c["d"], c["L"])
    assert rel_err(r, oracle_value(c)) <= (FP64_TOL if prec == sg.PREC_FP64 else FF_TOL)
    if c["rule"] != 4:
        assert r.evals == oracle.count_distinct(c["rule"], c["d"], c["L"]) - 1


@pytest.mark.parametrize("c", [si.cfg3(si.FAM_PRODUCT_PEAK), si.cfg3(si.FAM_GAUSSIAN), si.cfg5(), si.cfg1()],
                         ids=lambda c: c["name"])
def test_mixed_merged_form(rules, c):
    r = sg.integrate(rules[c["rule"]], c["fam"], c["params"], c["d"], c["d"] + c["L"], prec=sg.PREC_MIXED,
                     form=sg.FORM_MERGED)
    err = rel_err(r, oracle_value(c))
    assert err <= MIXED_TOL, (err, r)
    assert err <= r.err_est


@pytest.mark.parametrize("c", [si.cfg1(), si.cfg2()], ids=lambda c: c["name"])
def test_fp64_combination_form(rules, c):
    # Eq. 2.6 literally; its binomial coefficients amplify rounding by the
    # conditioning of the combination, so the bar is scaled by it
    r = sg.integrate(rules[c["rule"]], c["fam"], c["params"], c["d"], c["d"] + c["L"],
                     prec=sg.PREC_FP64, form=sg.FORM_COMBINATION)
    assert rel_err(r, oracle_value(c)) <= max(FP64_TOL, 1e-15 * r.cond)


@pytest.mark.parametrize("c", [si.cfg3(si.FAM_PRODUCT_PEAK), si.cfg3(si.FAM_GAUSSIAN), si.cfg5(),
                               si.cfg1()], ids=lambda c: c["name"])
def test_mixed_configs(rules, c):
    r = sg.integrate(rules[c["rule"]], c["fam"], c["params"], c["d"], c["d"] + c["L"],
                     prec=sg.PREC_MIXED)
    err = rel_err(r, oracle_value(c))
    assert err <= MIXED_TOL, (err, r)
    assert err <= r.err_est  # the estimate bounds the error


# Gauss-Legendre integrals in FP64 under SG_FORM_AUTO (the merged form),
# every family, from low to high d, against the oracle at the FP64 bar.
AUTO_GL = [(d, L) for d, L in [(2, 8), (3, 7), (5, 6), (8, 5), (11, 6), (12, 6), (13, 6), (14, 5),
                               (14, 4), (20, 3), (33, 2), (46, 2), (200, 1), (7, 0)]]


@pytest.mark.parametrize("fam", [0, 1, 2, 3, 4])
@pytest.mark.parametrize("dL", AUTO_GL, ids=lambda t: "d%d_L%d" % t)
def test_fp64_auto_form_gauss_legendre(rules, dL, fam):
    d, L = dL
    c = dict(rule=4, fam=fam, d=d, L=L, params=si.item_params(fam, d, 500 + 7 * d + L))
    r = sg.integrate(rules[4], fam, c["params"], d, d + L, prec=sg.PREC_FP64)
    assert rel_err(r, oracle_value(c)) <= FP64_TOL
    pts, ev = sg.count_points(rules[4], d, d + L)
    assert r.points == pts == oracle.count_points(4, d, L)
    assert r.evals == ev
    # the merged form evaluates each distinct point once: no more than the
    # n_d^q of Eq. 2.6 once d > L (for d <= L it also visits the points of the
    # subgrids Eq. 2.6 leaves out, whose merged weights are zero)
    assert ev <= pts or d <= L


@pytest.mark.parametrize("c", CONFIGS, ids=lambda c: c["name"])
def test_float_float_configs(rules, c):
    # float-float evaluation on the FP32 pipes: far below the mixed bar on
    # every configuration, including the Gauss-Legendre one where float misses
    r = sg.integrate(rules[c["rule"]], c["fam"], c["params"], c["d"], c["d"] + c["L"], prec=sg.PREC_FF)
    err = rel_err(r, oracle_value(c))
    assert err <= FF_TOL, (err, r)
    assert err <= max(50 * r.err_est, 1e-14)


EDGE = [dict(name="d1_L6", rule=2, fam=3, d=1, L=6, params=si.item_params(3, 1, 5)),
        dict(name="L0", rule=4, fam=1, d=7, L=0, params=si.item_params(1, 7, 6)),
        dict(name="L1", rule=2, fam=2, d=33, L=1, params=si.item_params(2, 33, 9)),
        dict(name="d_lt_L", rule=4, fam=2, d=2, L=6, params=si.item_params(2, 2, 7)),
        dict(name="trapezoid", rule=1, fam=0, d=5, L=4, params=si.item_params(0, 5, 8)),
        dict(name="gl_deep", rule=4, fam=3, d=6, L=8, params=si.item_params(3, 6, 10)),
        dict(name="peak_d200_underflow", rule=2, fam=2, d=200, L=2,
             params=si.item_params(2, 200, 1234))]
EDGE += [dict(name="ragged%d" % k, **it) for k, it in enumerate(si.batch(n=10, seed=3, d_hi=40, L_hi=4))]


@pytest.mark.parametrize("c", EDGE, ids=lambda c: c["name"])
def test_fp64_edge_and_ragged(rules, c):
    r = sg.integrate(rules[c["rule"]], c["fam"], c["params"], c["d"], c["d"] + c["L"],
                     prec=sg.PREC_FP64)
    assert rel_err(r, oracle_value(c)) <= FP64_TOL


def test_fp64_is_bitwise_deterministic(rules):
    c = si.cfg2()
    a = sg.integrate(rules[4], c["fam"], c["params"], c["d"], c["d"] + c["L"], prec=sg.PREC_FP64)
    b = sg.integrate(rules[4], c["fam"], c["params"], c["d"], c["d"] + c["L"], prec=sg.PREC_FP64)
    assert a.mant == b.mant and a.exp2 == b.exp2
    c = si.cfg3(si.FAM_GAUSSIAN)
    a = sg.integrate(rules[2], c["fam"], c["params"], c["d"], c["d"] + c["L"], prec=sg.PREC_MIXED)
    b = sg.integrate(rules[2], c["fam"], c["params"], c["d"], c["d"] + c["L"], prec=sg.PREC_MIXED)
    assert a.mant == b.mant and a.exp2 == b.exp2


def test_tuning_changes_only_rounding(rules):
    c = si.cfg2()
    saved = sg.get_tuning(sg.PREC_FP64)
    try:
        vals = []
        for t in [(64, 1, 1), (512, 4, 4), (1 << 20, 16, 8)]:
            sg.set_tuning(sg.PREC_FP64, *t)
            r = sg.integrate(rules[4], c["fam"], c["params"], c["d"], c["d"] + c["L"])
            assert rel_err(r, oracle_value(c)) <= FP64_TOL
            vals.append(r.mant)
    finally:
        sg.set_tuning(sg.PREC_FP64, *saved)


def test_async_matches_blocking(rules):
    c = si.cfg2()
    q = c["d"] + c["L"]
    dp = torch.tensor(c["params"], dtype=torch.float64, device="cuda")
    out = torch.zeros(sg.DEV_RESULT_DOUBLES, dtype=torch.float64, device="cuda")
    sg.integrate_async(rules[4], c["fam"], dp, c["d"], q, out)
    torch.cuda.synchronize()
    r = sg.integrate(rules[4], c["fam"], c["params"], c["d"], q)
    assert out[0].item() == r.mant and int(out[1].item()) == r.exp2


def test_invalid_arguments_return_status(rules):
    lib = sg.load()
    import ctypes
    res = sg.sg_result()
    p = np.zeros(8)
    ptr = ctypes.c_void_p(p.ctypes.data)
    s = sg._stream_handle()
    assert lib.sg_integrate(rules[2].handle, 0, ptr, 0, 4, 3, 0, 0, s, ctypes.byref(res)) == 1   # q < d
    assert lib.sg_integrate(rules[2].handle, 9, ptr, 0, 4, 5, 0, 0, s, ctypes.byref(res)) == 1   # family
    assert lib.sg_integrate(rules[2].handle, 0, ptr, 0, 4, 4 + 10, 0, 0, s, ctypes.byref(res)) == 2  # level
    assert lib.sg_integrate(rules[2].handle, 0, ptr, 0, 9000, 9001, 0, 0, s, ctypes.byref(res)) == 2  # d
    with pytest.raises(sg.SgError):
        sg.integrate(rules[2], 0, p, 4, 3)


# ---------------------------------------------------------------------------
# batch
# ---------------------------------------------------------------------------

def _batch(items, rules):
    specs, pool, off = [], [], 0
    for it in items:
        specs.append((rules[it["rule"]], it["fam"], it["d"], it["d"] + it["L"], off))
        pool.append(np.asarray(it["params"]))
        off += 2 * it["d"]
    return specs, np.concatenate(pool)


def test_batch_fp64_matches_oracle(rules):
    items = si.batch(n=48, seed=11, d_hi=40, L_hi=4)
    specs, pool = _batch(items, rules)
    res = sg.integrate_batch(specs, pool, prec=sg.PREC_FP64)
    for it, r in zip(items, res):
        assert rel_err(r, oracle_value(it)) <= FP64_TOL
    # a second replay of the cached graph gives the same bits
    res2 = sg.integrate_batch(specs, pool, prec=sg.PREC_FP64)
    assert all(a.mant == b.mant for a, b in zip(res, res2))


def test_batch_matches_single_calls(rules):
    items = si.batch(n=16, seed=12, d_hi=60, L_hi=4)
    specs, pool = _batch(items, rules)
    res = sg.integrate_batch(specs, pool, prec=sg.PREC_FP64)
    for it, r in zip(items, res):
        s = sg.integrate(rules[it["rule"]], it["fam"], it["params"], it["d"], it["d"] + it["L"])
        assert abs(r.mant * 2.0 ** (r.exp2 - s.exp2) - s.mant) <= 1e-13 * abs(s.mant)


def test_mixed_guard(rules):
    # without the guard, badly conditioned items miss 1e-6 in float; with
    # it every item is within 1e-6 of the oracle
    items = si.batch(n=48, seed=13, d_hi=40, L_hi=4)
    specs, pool = _batch(items, rules)
    res = sg.integrate_batch(specs, pool, prec=sg.PREC_MIXED, guard_tol=MIXED_TOL / 4)
    for it, r in zip(items, res):
        assert rel_err(r, oracle_value(it)) <= MIXED_TOL
    raw = sg.integrate_batch(specs, pool, prec=sg.PREC_MIXED, guard_tol=0.0)
    for it, r in zip(items, raw):
        err = rel_err(r, oracle_value(it))
        if r.err_est <= MIXED_TOL / 4:
            assert err <= MIXED_TOL


def _dp_err(it, r):
    rel, ls = dp_pin.smolyak_value_f64(it["rule"], it["fam"], it["params"], it["d"], it["L"])
    if it["fam"] == si.FAM_OSCILLATORY:
        return abs(r.value - rel) / abs(rel)
    return abs(r.mant * math.exp(r.exp2 * math.log(2.0) - ls) - rel) / abs(rel)


def test_batch_full_size_guarded(rules):
    """The full 4096-item workload (d ~ U{5..200}, q - d ~ U{2..5}, four
    families, two rules) in one persistent launch per precision tier: float
    evaluation, the items whose error estimate exceeds 1e-6 / 4 recomputed in
    float-float and what that still leaves above it in FP64.  Every item must
    be within 1e-6 of the separable pin (a float64 evaluation of the same
    Smolyak sum by a different algorithm, whose own error is far below that),
    and the small ones within 1e-6 of the oracle."""
    items = si.batch()
    specs, pool = _batch(items, rules)
    res = sg.integrate_batch(specs, pool, prec=sg.PREC_MIXED, guard_tol=MIXED_TOL / 4)
    worst, checked = 0.0, 0
    for it, r in zip(items, res):
        err = _dp_err(it, r)
        worst = max(worst, err)
        assert err <= MIXED_TOL, (it["rule"], it["fam"], it["d"], it["L"], err, r.err_est)
        if r.points <= 2e5 and checked < 64:
            assert rel_err(r, oracle_value(it)) <= MIXED_TOL
            checked += 1
    assert checked >= 16
    print("full batch, guarded: %.3f s, worst error %.2e" % (res[0].seconds, worst))


def test_batch_full_size_float_estimate_bounds_the_error(rules):
    """The same batch in float evaluation alone: the items badly enough
    conditioned miss 1e-6 (the guard exists for them), but every item's error
    stays below its own estimate, which is what the guard decides on."""
    items = si.batch()
    specs, pool = _batch(items, rules)
    res = sg.integrate_batch(specs, pool, prec=sg.PREC_MIXED)
    above = 0
    for it, r in zip(items, res):
        err = _dp_err(it, r)
        assert err <= r.err_est, (it["rule"], it["fam"], it["d"], it["L"], err, r.err_est)
        above += err > MIXED_TOL
    print("full batch, float only: %.3f s, %d of %d items above 1e-6" % (res[0].seconds, above, len(items)))


# ---------------------------------------------------------------------------
# gradient
# ---------------------------------------------------------------------------

@pytest.mark.parametrize("fam", [0, 1, 2, 3, 4])
def test_grad_small_all_families(rules, fam):
    kind, d, L = (4, 7, 3) if fam % 2 else (2, 9, 3)
    p = si.item_params(fam, d, 77 + fam)
    r, g = sg.integrate_grad(rules[kind], fam, p, d, d + L)
    o, go = oracle.gradient(kind, fam, p, d, L, list(range(2 * d)))
    go = np.ldexp(go, o.exp2)
    assert rel_err(r, o) <= FP64_TOL
    assert np.abs(g - go).max() <= FP64_TOL * np.abs(go).max()


def test_grad_cfg5_matches_oracle_subset_and_fd(rules):
    c = si.cfg5()
    q = c["d"] + c["L"]
    r, g = sg.integrate_grad(rules[2], c["fam"], c["params"], c["d"], q)
    idx = dp_pin.sample_idx(c["d"])
    o, go = oracle.gradient(c["rule"], c["fam"], c["params"], c["d"], c["L"], idx)
    go = np.ldexp(go, o.exp2)
    assert np.abs(g[idx] - go).max() <= FP64_TOL * np.abs(go).max()
    # central differences of the GPU value itself
    p = np.asarray(c["params"])
    for j in idx[:6]:
        h = 1e-5 * max(abs(p[j]), 1e-3)
        pp, pm = p.copy(), p.copy()
        pp[j] += h
        pm[j] -= h
        fd = (sg.integrate(rules[2], c["fam"], pp, c["d"], q).value -
              sg.integrate(rules[2], c["fam"], pm, c["d"], q).value) / (2 * h)
        assert abs(fd - g[j]) <= 1e-6 * np.abs(g).max()
    # mixed-precision adjoint
    rm, gm = sg.integrate_grad(rules[2], c["fam"], c["params"], c["d"], q, prec=sg.PREC_MIXED)
    assert np.abs(gm - g).max() <= MIXED_TOL * np.abs(g).max()


def test_autograd_function(rules):
    c = si.cfg5()
    q = c["d"] + c["L"]
    p = torch.tensor(c["params"], dtype=torch.float64, device="cuda", requires_grad=True)
    val = sg.sg_quad(p, rules[2], c["fam"], c["d"], q)
    (3.0 * val).backward()
    _, g = sg.integrate_grad(rules[2], c["fam"], c["params"], c["d"], q)
    assert torch.allclose(p.grad.cpu(), torch.tensor(3.0 * g), rtol=0, atol=1e-15 * np.abs(g).max())


@pytest.mark.parametrize("prec", [sg.PREC_FP64, sg.PREC_MIXED])
def test_batch_shards_combine_bitwise(rules, prec):
    # the chunk queue cut into 1, 2 or 3 contiguous shards, each run by its own
    # call; the combined limbs give the same bits for every shard count, and
    # the same bits as the unsharded batch call
    items = si.batch(n=32, seed=23, d_hi=50, L_hi=4)
    specs, pool = _batch(items, rules)
    whole = sg.integrate_batch(specs, pool, prec=prec)
    bits = None
    for K in (1, 2, 3):
        parts, info = [], None
        for k in range(K):
            p, info = sg.integrate_batch_shard(specs, pool, k, K, prec=prec)
            parts.append(p)
        res = sg.shard_combine(parts, info)
        b = [(r.mant, r.exp2, r.cond) for r in res]
        assert bits is None or b == bits
        bits = b
    assert bits == [(r.mant, r.exp2, r.cond) for r in whole]
    if prec == sg.PREC_FP64:
        for it, r in zip(items, res):
            assert rel_err(r, oracle_value(it)) <= FP64_TOL


def test_autotune_classes_table_is_applied_and_changes_only_rounding(rules, tmp_path):
    # per-class chunk sizes: the table is written, read back and applied to
    # later batches, whose results agree with the untuned ones to rounding
    items = si.batch(n=40, seed=22, d_hi=60, L_hi=4)
    specs, pool = _batch(items, rules)
    sg.tuning_clear()
    try:
        base = sg.integrate_batch(specs, pool, prec=sg.PREC_FP64)
        path = str(tmp_path / "classes.json")
        n = sg.autotune_classes(specs, pool, prec=sg.PREC_FP64, reps=1, path=path)
        assert n > 0
        text = open(path).read()
        assert text.count("points_per_chunk") == n
        sg.tuning_clear()
        assert sg.tuning_load(path) == n
        tuned = sg.integrate_batch(specs, pool, prec=sg.PREC_FP64)
        for it, a, b in zip(items, base, tuned):
            assert abs(b.mant * 2.0 ** (b.exp2 - a.exp2) - a.mant) <= 1e-14 * abs(a.mant)
            assert rel_err(b, oracle_value(it)) <= FP64_TOL
    finally:
        sg.tuning_clear()


def test_autotune_picks_a_grid_point_and_keeps_results(rules):
    items = si.batch(n=12, seed=21, d_hi=40, L_hi=3)
    specs, pool = _batch(items, rules)
    saved = sg.get_tuning(sg.PREC_MIXED)
    try:
        best, ms = sg.autotune(specs, pool, prec=sg.PREC_MIXED, reps=1)
        assert best[0] in (2048, 8192, 32768, 131072) and best[1] in (4, 8, 16) and best[2] in (4, 8)
        assert ms > 0
        assert sg.get_tuning(sg.PREC_MIXED) == best
        res = sg.integrate_batch(specs, pool, prec=sg.PREC_MIXED)
        for it, r in zip(items, res):
            assert rel_err(r, oracle_value(it)) <= max(MIXED_TOL, r.err_est)
    finally:
        sg.set_tuning(sg.PREC_MIXED, *saved)
