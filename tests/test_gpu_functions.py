"""Accuracy of the elementary functions the fold evaluates per point (the
library's own float expm1, double expm1 and double sincos; CUDA's sincosf
for the oscillatory deviation in float) on the GPU against numpy's double-precision libm, through the
sg_eval_functions hook of the C ABI."""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

torch = pytest.importorskip("torch")
if not torch.cuda.is_available():
    pytest.skip("no CUDA device", allow_module_level=True)

import paper_2210_14313_gb300 as sg  # noqa: E402

U32 = 2.0 ** -24
U64 = 2.0 ** -53


def _eval(kind, prec, x):
    xd = torch.tensor(x, dtype=torch.float64, device="cuda")
    yd = torch.zeros(len(x) * (2 if kind == 1 else 1), dtype=torch.float64, device="cuda")
    st = sg.load().sg_eval_functions(kind, prec, ctypes.c_void_p(xd.data_ptr()),
                                     ctypes.c_void_p(yd.data_ptr()), len(x), sg._stream_handle())
    assert st == 0
    torch.cuda.synchronize()
    return yd.cpu().numpy()


def _args(lo, hi, n=200001):
    rng = np.random.default_rng(1)
    x = np.concatenate([np.linspace(lo, hi, n), rng.uniform(lo, hi, n),
                        np.geomspace(1e-12, 1.0, 2001), -np.geomspace(1e-12, 1.0, 2001),
                        [0.0, 0.34657359, -0.34657359, 0.5 * np.pi, np.pi, -np.pi]])
    return x


def test_float_expm1_within_three_ulp():
    x = _args(-40.0, 40.0).astype(np.float32).astype(np.float64)
    y = _eval(0, sg.PREC_MIXED, x)
    ref = np.expm1(x)
    rel = np.abs(y - ref) / np.maximum(np.abs(ref), 1e-300)
    assert rel.max() <= 3 * U32, (rel.max(), x[rel.argmax()])


def test_float_sincos_accuracy():
    x = _args(-60.0, 60.0).astype(np.float32).astype(np.float64)
    y = _eval(1, sg.PREC_MIXED, x)
    s, c = y[0::2], y[1::2]
    rs, rc = np.sin(x), np.cos(x)
    assert np.abs(s - rs).max() <= 4 * U32
    assert np.abs(c - rc).max() <= 4 * U32
    big = np.abs(rs) > 1e-3
    assert (np.abs(s - rs)[big] / np.abs(rs[big])).max() <= 4 * U32
    small = np.abs(x) < 0.5
    assert (np.abs(s - rs)[small & (x != 0)] / np.abs(rs[small & (x != 0)])).max() <= 2 * U32


def test_double_sincos_accuracy():
    # the fold's own double sincos (Cody-Waite reduction, Taylor series) and,
    # from |x| = 2^20 on, the library sincos it defers to
    x = np.concatenate([_args(-60.0, 60.0), np.arange(-40, 41) * (0.5 * np.pi),
                        [1048575.75, 1048576.0, -1048576.5, 3.0e7, -1.0e10, 123456789.125]])
    y = _eval(1, sg.PREC_FP64, x)
    s, c = y[0::2], y[1::2]
    rs, rc = np.sin(x), np.cos(x)
    assert np.abs(s - rs).max() <= 4 * U64
    assert np.abs(c - rc).max() <= 4 * U64
    small = (np.abs(x) < 0.5) & (x != 0)
    assert (np.abs(s - rs)[small] / np.abs(rs[small])).max() <= 2 * U64


def test_double_expm1_accuracy():
    # the fold's own double expm1: short series below 2^-5, long series below
    # ln2/2, reduction above, the library expm1 from |x| = 700 on
    x = np.concatenate([_args(-40.0, 40.0), _args(-0.4, 0.4, n=50001), _args(-0.04, 0.04, n=50001),
                        [2.0 ** -5, -2.0 ** -5, 0.3465733528137207, -0.3465733528137207, 699.0, -699.0,
                         700.0, -745.0, 709.5]])
    y = _eval(0, sg.PREC_FP64, x)
    ref = np.expm1(x)
    ok = np.isfinite(ref) & (ref != 0)
    rel = np.abs(y[ok] - ref[ok]) / np.abs(ref[ok])
    assert rel.max() <= 3 * U64, (rel.max(), x[ok][rel.argmax()])
    assert y[x == 0.0].tolist() == [0.0] * int((x == 0.0).sum())


def test_float_float_expm1():
    x = np.concatenate([_args(-40.0, 40.0, n=50001), [1e-30, -1e-30, 5e-8, -5e-8]])
    y = _eval(0, sg.PREC_FF, x)
    ref = np.expm1(x)
    rel = np.abs(y - ref) / np.maximum(np.abs(ref), 1e-300)
    # a float pair holds the argument to about 2^-50 |x|, and the float
    # correction (1 + E) x.lo adds up to 2^-48 |x| relative: the bound is
    # 1e-13 for the arithmetic plus 2^-46 |x|
    bound = 1e-13 + 2.0 ** -46 * np.abs(x)
    assert np.all(rel <= bound), (rel.max(), x[np.argmax(rel / bound)])


def test_float_float_sincos():
    x = _args(-60.0, 60.0, n=50001)
    y = _eval(1, sg.PREC_FF, x)
    s, c = y[0::2], y[1::2]
    assert np.abs(s - np.sin(x)).max() <= 2e-13
    assert np.abs(c - np.cos(x)).max() <= 2e-13
    small = (np.abs(x) < 0.5) & (x != 0)
    assert (np.abs(s - np.sin(x))[small] / np.abs(np.sin(x[small]))).max() <= 1e-13
