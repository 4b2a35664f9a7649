"""CPU tests of the library side: the C ABI loads and exports every function
include/sg.h declares, and the planner + the fold kernel's enumeration
primitives (replayed on the host by tests/index_check) stay inside their
table blocks, visit every (prefix tuple, tail entry) pair once and give the
oracle's value."""
import math
import os
import re

import numpy as np
import pytest

import oracle
import sg_inputs as si
import index_check

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _header_functions():
    src = open(os.path.join(ROOT, "include", "sg.h")).read()
    return sorted(set(re.findall(r"SG_API\s+[\w\s\*]+?\b(sg_\w+)\s*\(", src)))


def test_library_exports_every_declared_function():
    import paper_2210_14313_gb300 as sg
    lib = sg.load()
    declared = _header_functions()
    assert len(declared) >= 12
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(sg.ABI_SYMBOLS) == declared


def test_status_strings():
    import paper_2210_14313_gb300 as sg
    lib = sg.load()
    for code in range(7):
        assert lib.sg_status_string(code)
    assert b"unknown" in lib.sg_status_string(99)


def test_invalid_arguments_rejected_without_gpu():
    # NULL handles / out pointers are rejected before any CUDA call
    import ctypes
    import paper_2210_14313_gb300 as sg
    lib = sg.load()
    assert lib.sg_rule_init(5, 4, ctypes.byref(ctypes.c_void_p())) == 1       # bad rule kind
    assert lib.sg_rule_init_growth(2, 7, 4, ctypes.byref(ctypes.c_void_p())) == 1  # bad growth
    assert lib.sg_rule_init_growth(3, 0, 7, ctypes.byref(ctypes.c_void_p())) == 2  # no 127-node member
    assert lib.sg_rule_init(2, 0, ctypes.byref(ctypes.c_void_p())) == 2       # level out of range
    assert lib.sg_rule_init(2, 4, None) == 1
    assert lib.sg_integrate(None, 0, None, 0, 4, 9, 0, 0, None, None) == 1
    r = sg.sg_result()
    assert lib.sg_integrate(None, 0, ctypes.c_void_p(1), 0, 4, 9, 0, 0, None, ctypes.byref(r)) == 1
    t = sg.sg_tuning(10, 8, 8)
    assert lib.sg_set_tuning(1, ctypes.byref(t)) == 2
    assert lib.sg_get_tuning(7, ctypes.byref(t)) == 1


def _oracle_rel(c, r):
    o = oracle.integrate(c["rule"], c["fam"], c["params"], c["d"], c["L"])
    if c["fam"] == si.FAM_OSCILLATORY:
        return abs(r["rel"] - o.value) / abs(o.value)
    q = r["rel"] * math.exp(r["logscale"] - o.exp2 * math.log(2.0))
    return abs(q - o.mant) / abs(o.mant)


CASES = [si.cfg1(), si.cfg2(), si.cfg3(si.FAM_PRODUCT_PEAK), si.cfg3(si.FAM_GAUSSIAN)]
CASES += [dict(name="ragged%d" % k, **it) for k, it in enumerate(si.batch(n=8, seed=3, d_hi=30, L_hi=4))]
CASES += [dict(name="d1", rule=2, fam=3, d=1, L=6, params=si.item_params(3, 1, 5)),
          dict(name="L0", rule=4, fam=1, d=7, L=0, params=si.item_params(1, 7, 6)),
          dict(name="d_lt_L", rule=4, fam=2, d=2, L=6, params=si.item_params(2, 2, 7)),
          dict(name="trap", rule=1, fam=0, d=5, L=4, params=si.item_params(0, 5, 8)),
          # Gauss-Patterson (Eq. 2.12) and the Section 5.4 accuracy levels (flag 16)
          dict(name="gp", rule=3, fam=1, d=5, L=4, params=si.item_params(1, 5, 9)),
          dict(name="gp_slow_test3", rule=3 | 16, fam=4, d=6, L=9, params=np.array([2.0] * 6 + [0.5] * 6)),
          dict(name="gp_slow_peak", rule=3 | 16, fam=2, d=4, L=8, params=si.item_params(2, 4, 10)),
          dict(name="cc_slow", rule=2 | 16, fam=3, d=6, L=6, params=si.item_params(3, 6, 11)),
          dict(name="trap_slow", rule=1 | 16, fam=0, d=4, L=5, params=si.item_params(0, 4, 12))]


@pytest.mark.parametrize("form", [1, 2, 3, 4])
@pytest.mark.parametrize("case", CASES, ids=lambda c: c["name"])
def test_fold_enumeration_matches_oracle(case, form):
    r = index_check.run(case["rule"], case["fam"], case["params"], case["d"], case["L"], form=form)
    assert r["violations"] == 0
    assert r["badpairs"] == 0
    assert r["evals"] == r["plan_evals"]
    tol = 1e-12 if form != 3 else 1e-11
    assert _oracle_rel(case, r) < tol


@pytest.mark.parametrize("d,r", [(1, 1), (5, 5), (12, 6), (33, 1), (100, 3), (1000, 2), (1025, 4),
                                 (8192, 1), (8192, 3), (8192, 12)])
def test_warp_unranking_matches_binary_search(d, r):
    # the kernel searches 32 candidates per round; up to three rounds for d <= 8192
    assert index_check.unrank_mismatches(d, r) == 0


@pytest.mark.parametrize("ppc,ctas,warps", [(64, 1, 1), (100, 3, 2), (1 << 20, 8, 8)])
def test_chunking_does_not_change_the_sum(ppc, ctas, warps):
    c = si.cfg2()
    r = index_check.run(c["rule"], c["fam"], c["params"], c["d"], c["L"], form=2, ppc=ppc,
                        ctas_per_sm=ctas, warps=warps)
    assert r["violations"] == 0 and r["badpairs"] == 0
    assert _oracle_rel(c, r) < 1e-12


@pytest.mark.parametrize("cfg,prec_ctas", [("cfg2", (2, 8)), ("cfg3", (2, 8)), ("cfg5", (2, 8)), ("cfg1", (2, 8))])
def test_single_integral_chunks_are_one_wave_with_few_runs(cfg, prec_ctas):
    # single integrals: the run-aware planner cuts the chunks by lane slots to
    # no more than the resident warps (152 SMs x CTAs x warps), every pair
    # still visited once; on d = 12 no chunk gathers the dozen short runs that
    # points-only chunks did (at most a handful)
    c = {"cfg1": si.cfg1, "cfg2": si.cfg2, "cfg5": si.cfg5}.get(cfg, lambda: si.cfg3(si.FAM_GAUSSIAN))()
    ctas, warps = prec_ctas
    r = index_check.run(c["rule"], c["fam"], c["params"], c["d"], c["L"], form=4, ppc=2048,
                        ctas_per_sm=ctas, warps=warps)
    assert r["violations"] == 0 and r["badpairs"] == 0
    assert r["evals"] == r["plan_evals"]
    assert r["chunks"] <= 152 * ctas * warps
    if cfg == "cfg2":
        assert r["max_runs"] <= 6
    # (the replay adds each lane's terms in plain double, not exactly as the
    # kernels do: merged weights of both signs cost it a few digits)
    assert _oracle_rel(c, r) < 1e-11


@pytest.mark.parametrize("case", [c for c in CASES if c["d"] >= 2 and c["rule"] & 16 == 0][:8],
                         ids=lambda c: c["name"])
def test_gradient_plan_enumeration(case):
    # gradient plans (the forward item plus the adjoint sub-sums, which leave
    # one direction out): with the run-aware chunks of single integrals every
    # table access stays in its block and every pair is visited once
    r = index_check.run(case["rule"], case["fam"], case["params"], case["d"], case["L"], form=2, grad=1)
    assert r["violations"] == 0
    assert r["badpairs"] == 0
    assert r["evals"] == r["plan_evals"]
    assert len(r["v"]) > 0 and np.all(np.isfinite(r["v"]))
    assert _oracle_rel(case, r) < 1e-12
    # the same sub-sums from point-sized chunks (one CTA of one warp per SM:
    # chunk targets above the tuned maximum, so no run-aware chunking)
    u = index_check.run(case["rule"], case["fam"], case["params"], case["d"], case["L"], form=2, grad=1,
                        ppc=64, ctas_per_sm=1, warps=1)
    assert u["violations"] == 0 and u["badpairs"] == 0
    scale = max(1e-300, float(np.max(np.abs(r["v"]))))
    assert np.max(np.abs(u["v"] - r["v"])) <= 1e-13 * scale


def test_merged_form_evaluates_each_distinct_point_once():
    # nested rules: the merged form's evaluations are the sparse grid's
    # distinct points less the centre (the oracle counts them by merging)
    for c in CASES:
        if c["rule"] & 15 == 4:
            continue
        r = index_check.run(c["rule"], c["fam"], c["params"], c["d"], c["L"], form=4)
        assert r["evals"] == oracle.count_distinct(c["rule"], c["d"], c["L"]) - 1


def test_n_d_q_matches_oracle_count():
    # the combination form evaluates exactly the points of Eq. 2.6's tensor
    # grids, except the all-centre point when that subgrid belongs to the rule
    # (d > L), whose deviation is zero by construction
    for c in CASES:
        r = index_check.run(c["rule"], c["fam"], c["params"], c["d"], c["L"], form=3)
        centre = 1 if c["d"] > c["L"] else 0
        assert r["evals"] == oracle.count_points(c["rule"], c["d"], c["L"]) - centre


@pytest.mark.parametrize("member", range(1, 7))
def test_library_gauss_patterson_matches_oracle_table(member):
    # two independent constructions: the library's double-double Newton
    # iteration and the oracle's 300-digit table (gen_gp_table.py)
    x, w = index_check.rule(3, member)
    xo, wo = oracle.rule(oracle.GP, member)
    assert x.size == xo.size == 2 ** member - 1
    assert np.all(np.abs(x - xo) <= np.spacing(np.maximum(xo, 1e-300)))
    assert np.all(np.abs(w - wo) <= 4e-16 * wo)


@pytest.mark.parametrize("kind", [1, 2, 3, 4])
def test_library_growth_matches_oracle(kind):
    for growth in (0, 16):
        top = 13 if (growth or kind != 3) else 6
        for level in range(1, top + 1):
            n = index_check.rule(kind | growth, level)[0].size
            assert n == oracle.rule(kind | growth, level)[0].size, (kind, growth, level)
        for k in range(1, top):
            xb, wb = index_check.block(kind | growth, 0, k)
            xo, wo = oracle.delta_rule(kind | growth, k + 1)
            assert xb.size == xo.size, (kind, growth, k)
            if xb.size:
                order, order_o = np.argsort(xb, kind="stable"), np.argsort(xo, kind="stable")
                assert np.allclose(xb[order], xo[order_o], rtol=0, atol=4e-16)
                assert np.allclose(wb[order], wo[order_o], rtol=0, atol=1e-14 * np.abs(wo).max())


def _nvrtc():
    import ctypes
    for name in ("libnvrtc.so", "/usr/local/cuda/lib64/libnvrtc.so"):
        try:
            return ctypes.CDLL(name)
        except OSError:
            pass
    pytest.skip("NVRTC not available")


def _nvrtc_compile(lib, source, k):
    # the program sg_integrand_create builds: user source + the library's fold
    # kernel, with its headers given to NVRTC by name
    import ctypes
    csrc = os.path.join(os.path.dirname(os.path.dirname(os.path.abspath(__file__))),
                        "paper_2210_14313_gb300", "csrc")
    from paper_2210_14313_gb300 import _build
    names = [n for _, n in _build.EMBEDDED]
    hdrs = [open(os.path.join(csrc, n)).read().encode() for n in names]
    prog = ctypes.c_void_p()
    src = (source + '\n#include "sg_user_kernel.cuh"\n').encode()
    nh = len(names)
    assert lib.nvrtcCreateProgram(ctypes.byref(prog), src, b"sg_user.cu", nh, (ctypes.c_char_p * nh)(*hdrs),
                                  (ctypes.c_char_p * nh)(*[n.encode() for n in names])) == 0
    opts = [b"--gpu-architecture=sm_103", ("-DSG_USER_K=%d" % k).encode(), b"-std=c++17", b"-default-device"]
    rc = lib.nvrtcCompileProgram(prog, len(opts), (ctypes.c_char_p * len(opts))(*opts))
    n = ctypes.c_size_t()
    lib.nvrtcGetProgramLogSize(prog, ctypes.byref(n))
    buf = ctypes.create_string_buffer(n.value + 1)
    lib.nvrtcGetProgramLog(prog, buf)
    lib.nvrtcDestroyProgram(ctypes.byref(prog))
    return rc, buf.value.decode(errors="replace")


def test_user_integrand_programs_compile():
    import user_integrands as ui
    lib = _nvrtc()
    for name, (src, k, _) in ui.CASES.items():
        rc, log = _nvrtc_compile(lib, src, k)
        assert rc == 0, (name, log)
    rc, log = _nvrtc_compile(lib, ui.EXPLIN, 2)
    assert rc == 0, log
    rc, log = _nvrtc_compile(lib, ui.BROKEN, 1)
    assert rc != 0 and "undefined_name" in log


def test_divide_free_block_digits():
    # the prefix digits' q / m by a multiplier (Granlund-Montgomery) for every
    # block size up to 5000 nodes
    assert index_check.divmagic_mismatches(5000) == 0


# ---------------------------------------------------------------------------
# merged form (Eq. 2.8): every distinct point once with its merged weight
# ---------------------------------------------------------------------------

MERGED_CASES = [(2, 3, 4), (2, 5, 3), (4, 4, 4), (4, 3, 6), (3, 3, 3), (1, 4, 3), (2 | 16, 3, 5), (3 | 16, 2, 6),
                (2, 1, 5), (4, 2, 1)]


@pytest.mark.parametrize("kind,d,L", MERGED_CASES)
def test_merged_weights_are_the_oracles_merged_point_weights(kind, d, L):
    # the oracle's difference-form points with their product weights, added
    # point by point, are the sparse grid's point weights (Eq. 2.8); the
    # planner's merged weights (a different algorithm: generating series of
    # the per-node difference weights, in double-double) must match them
    import oracle
    import index_check
    Xo, Wo = oracle.points(kind, d, L, oracle.FORM_DIFF)
    merged, mass = {}, {}
    # the two sides build their nodes by different formulas: points are
    # matched to 1e-12 (the nodes of these rules are at least 1e-4 apart)
    for x, w in zip(map(tuple, np.round(Xo, 12)), Wo):
        merged[x] = merged.get(x, 0.0) + w
        mass[x] = mass.get(x, 0.0) + abs(w)
    X, W = index_check.merged_points(kind, d, L)
    centre = tuple([0.5] * d)
    keys = [tuple(x) for x in np.round(X, 12)]
    assert len(set(keys)) == len(keys)                     # each point once
    assert set(keys) == set(merged) - {centre}             # every non-centre point
    for k, w in zip(keys, W):
        assert abs(w - merged[k]) <= 1e-13 * max(mass[k], 1.0), (k, w, merged[k])
    # with the centre's weight the weights sum to the volume of the cube
    assert abs(W.sum() + merged.get(centre, 0.0) - 1.0) <= 1e-12 * max(mass.values())


def test_class_tuning_table_loads_without_gpu(tmp_path):
    # the per-class chunk-size table of the batch path is host data: its file
    # round trip and its errors need no GPU
    import ctypes
    import paper_2210_14313_gb300 as sg
    lib = sg.load()
    p = tmp_path / "classes.json"
    p.write_text('{"classes": [\n'
                 '  {"family": 1, "rule": 4, "dbucket": 7, "L": 5, "prec": 1, "points_per_chunk": 16384},\n'
                 '  {"family": 0, "rule": 2, "dbucket": 8, "L": 5, "prec": 0, "points_per_chunk": 4096}\n]}\n')
    n = ctypes.c_int(0)
    assert lib.sg_tuning_load(str(p).encode(), ctypes.byref(n)) == 0 and n.value == 2
    bad = tmp_path / "bad.json"
    bad.write_text('{"classes": [{"family": 1, "rule": 4, "dbucket": 7, "L": 5, "prec": 7, '
                   '"points_per_chunk": 16384}]}\n')
    assert lib.sg_tuning_load(str(bad).encode(), ctypes.byref(n)) == 1          # bad precision
    assert lib.sg_tuning_load(str(tmp_path / "none.json").encode(), ctypes.byref(n)) == 1
    assert lib.sg_tuning_clear() == 0


@pytest.mark.parametrize("seed", range(12))
def test_run_aware_chunks_random_shapes(seed):
    # random single-integral shapes and warp counts (from one warp on one SM
    # up to 8 x 8 per SM): the budget search and the cut runs keep every
    # table access in its block, visit every pair once, stay within the
    # resident warps and give the oracle's value
    rng = np.random.default_rng(1000 + seed)
    kind = int(rng.choice([1, 2, 4]))
    fam = int(rng.integers(0, 5))
    d = int(rng.integers(2, 41))
    L = int(rng.integers(1, 6 if d < 20 else 4))
    ctas, warps = int(rng.integers(1, 9)), int(rng.integers(1, 9))
    case = dict(name="rnd%d" % seed, rule=kind, fam=fam, d=d, L=L, params=si.item_params(fam, d, 77 + seed))
    for form in (2, 4):
        r = index_check.run(kind, fam, case["params"], d, L, form=form, ppc=1 << 20, ctas_per_sm=ctas, warps=warps)
        assert r["violations"] == 0 and r["badpairs"] == 0
        assert r["evals"] == r["plan_evals"]
        assert r["chunks"] <= 152 * ctas * warps  # (fewer patterns than warps here)
        assert _oracle_rel(case, r) < 1e-11
