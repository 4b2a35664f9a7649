"""The FP64 fold's sin, cos and expm1 polynomials (sg_fixed.h) are the
minimax fits that gen_poly.py computes, and those fits meet their error
bounds against mpmath's functions."""
import os
import sys

import pytest

mp = pytest.importorskip("mpmath")

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2210_14313_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_poly  # noqa: E402

BOUNDS = {"sin": 1e-17, "cos": 1e-18, "expm1": 1e-18}
PREFIX = {"sin": "SG_FX_SIN", "cos": "SG_FX_COS", "expm1": "SG_FX_EXP"}
# the sign patterns the integer Horner loops of sg_fixed.h are written for
SIGNS = {"sin": [-1, 1] * 3, "cos": [1, -1] * 3, "expm1": [1] * 11}


@pytest.mark.parametrize("name", sorted(BOUNDS))
def test_fixed_coefficients_are_the_minimax_fit(name):
    with open(os.path.join(CSRC, "sg_fixed.h")) as f:
        src = f.read()
    mags, signs = gen_poly.fixed_coefficients(name)
    assert signs == SIGNS[name]
    for k, m in enumerate(mags):
        assert "#define %s%d %dull" % (PREFIX[name], k, m) in src, (name, k, m)
    err = gen_poly.fixed_error(name, N=1500)
    assert err <= BOUNDS[name], (name, float(err))
