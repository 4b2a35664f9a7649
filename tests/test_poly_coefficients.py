"""The fold's double sin, cos and expm1 polynomials (sg_kernels.cu) are the
minimax fits that gen_poly.py computes, and those fits meet their error
bounds against mpmath's functions."""
import os
import sys

import pytest

mp = pytest.importorskip("mpmath")

CSRC = os.path.join(os.path.dirname(__file__), "..", "paper_2210_14313_gb300", "csrc")
sys.path.insert(0, CSRC)
import gen_poly  # noqa: E402

BOUNDS = {"sin": 2e-17, "cos": 2e-18, "expm1": 2e-18, "expm1_small": 2e-17}


@pytest.mark.parametrize("name", sorted(BOUNDS))
def test_kernel_coefficients_are_the_minimax_fit(name):
    with open(os.path.join(CSRC, "sg_kernels.cu")) as f:
        src = f.read()
    coef = gen_poly.coefficients(name)
    missing = [c for c in coef if repr(c) not in src and c != 0.5]
    assert not missing, (name, missing)
    err = gen_poly.rounded_error(name, coef, N=1500)
    assert err <= BOUNDS[name], (name, float(err))
