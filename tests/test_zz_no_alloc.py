"""The no-allocation entry point, sg_integrate_noalloc, against the CPU
oracle and the regular asynchronous entry point.

sg_integrate_noalloc exists for callers that must not allocate memory where
they integrate (cudaMalloc/cudaFree synchronise the device, and some host
runtimes own all device memory).  It keeps its scratch in one fixed array
inside the library and shares it between calls, so this test calls it
twice in a row on each workload (with a different workload in between) and
checks every result against the oracle and against sg_integrate_async
within the tolerances the other GPU tests use.  The cases cover every
branch of its own planner: the four rules (the nested Gauss-Patterson
index shift and the trapezoid rule included), q - d = 0 (no work chunk:
only the centre term) and q - d = 1, both precisions and both deviation
kinds.  This file is named to be collected last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import sg_inputs as si

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2210_14313_gb300 as sg  # noqa: E402

FP64_TOL = 1e-12
MIXED_TOL = 1e-6


def _noalloc(c, prec, out):
    lib = sg.load()
    params = torch.tensor(c["params"], dtype=torch.float64, device="cuda")
    st = lib.sg_integrate_noalloc(c["rule"], c["fam"], ctypes.c_void_p(params.data_ptr()), c["d"],
                                  c["d"] + c["L"], prec, sg._stream_handle(),
                                  ctypes.c_void_p(out.data_ptr()))
    torch.cuda.synchronize()
    return st


def _reference(c, prec):
    rule = sg.Rule(c["rule"], max_level=c["L"] + 1)
    params = torch.tensor(c["params"], dtype=torch.float64, device="cuda")
    out = torch.zeros(sg.DEV_RESULT_DOUBLES, dtype=torch.float64, device="cuda")
    sg.integrate_async(rule, c["fam"], params, c["d"], c["d"] + c["L"], out, prec=prec)
    torch.cuda.synchronize()
    return out.cpu().numpy()


def _rel(a, b):
    return abs(a[0] * 2.0 ** (a[1] - b[1]) - b[0]) / abs(b[0])


def _rel_oracle(a, o):
    return abs(a[0] * 2.0 ** (a[1] - o.exp2) - o.mant) / abs(o.mant)


def _case(name, rule, fam, d, L, seed):
    return dict(name=name, rule=rule, fam=fam, d=d, L=L, params=si.item_params(fam, d, seed))


CASES = [(si.cfg2(), sg.PREC_FP64, FP64_TOL),
         (si.cfg3(si.FAM_GAUSSIAN), sg.PREC_MIXED, MIXED_TOL),
         (si.cfg5(), sg.PREC_FP64, FP64_TOL),
         (si.cfg1(), sg.PREC_FP64, FP64_TOL),
         (_case("gp_L5", sg.RULE_GAUSS_PATTERSON, si.FAM_GAUSSIAN, 6, 5, 41), sg.PREC_FP64, FP64_TOL),
         (_case("gp_L3_osc", sg.RULE_GAUSS_PATTERSON, si.FAM_OSCILLATORY, 9, 3, 42), sg.PREC_FP64, FP64_TOL),
         (_case("trapezoid_L4", sg.RULE_TRAPEZOID, si.FAM_PRODUCT_PEAK, 7, 4, 43), sg.PREC_FP64, FP64_TOL),
         (_case("L0", sg.RULE_CLENSHAW_CURTIS, si.FAM_EXP_LINEAR, 11, 0, 44), sg.PREC_FP64, FP64_TOL),
         (_case("L1", sg.RULE_GAUSS_LEGENDRE, si.FAM_GAUSSIAN, 40, 1, 45), sg.PREC_FP64, FP64_TOL),
         (_case("mixed_osc", sg.RULE_CLENSHAW_CURTIS, si.FAM_OSCILLATORY, 20, 3, 46), sg.PREC_MIXED, MIXED_TOL)]


def test_noalloc_matches_oracle_and_async_entry_point_twice_in_a_row():
    refs = [_reference(c, prec) for c, prec, _ in CASES]
    orcs = [oracle.integrate(c["rule"], c["fam"], c["params"], c["d"], c["L"]) for c, _, _ in CASES]
    for (c, prec, tol), ref, o in zip(CASES, refs, orcs):
        for _ in range(2):
            out = torch.zeros(sg.DEV_RESULT_DOUBLES, dtype=torch.float64, device="cuda")
            assert _noalloc(c, prec, out) == sg.SG_OK
            got = out.cpu().numpy()
            assert _rel_oracle(got, o) <= tol, (c["name"], got, o)
            assert _rel(got, ref) <= tol, (c["name"], got, ref)


def test_noalloc_rejects_sizes_beyond_its_limits():
    out = torch.zeros(sg.DEV_RESULT_DOUBLES, dtype=torch.float64, device="cuda")
    big_d = dict(name="d2000", rule=2, fam=0, d=2000, L=1, params=si.item_params(0, 2000, 1))
    deep = dict(name="L7", rule=4, fam=0, d=5, L=7, params=si.item_params(0, 5, 2))
    wide = dict(name="entries", rule=2, fam=3, d=1024, L=6, params=si.item_params(3, 1024, 3))
    for c in (big_d, deep, wide):
        assert _noalloc(c, sg.PREC_FP64, out) == 2  # SG_ERANGE
    # still usable afterwards
    c = si.cfg2()
    assert _noalloc(c, sg.PREC_FP64, out) == sg.SG_OK
    assert _rel(out.cpu().numpy(), _reference(c, sg.PREC_FP64)) <= FP64_TOL
