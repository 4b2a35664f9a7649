"""Python access to the plain CPU oracle (test infrastructure only).

The oracle is a slow, direct C implementation of Smolyak quadrature; see
``sg_oracle.c`` for what it computes and which equations of the paper each
function follows.  Only the tests, the smoke check and the benchmark's CPU
baseline use it; the library never imports it.
"""
from __future__ import annotations

import ctypes
import os
import subprocess

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sg_oracle.c")
_DEPS = [_SRC, os.path.join(_HERE, "sg_gp_table.h")]
_LIB = os.path.join(_HERE, "liboracle.so")
_lib = None

FORM_DIFF = 0
FORM_COMB = 1
GP = 3     # Gauss-Patterson (rule kinds 1, 2, 4 as in the library)
SLOW = 16  # flag OR'ed into a rule kind: the paper's delayed growth (Section 5.4)


def build(force: bool = False) -> str:
    """Compile sg_oracle.c into liboracle.so next to it (gcc, IEEE double,
    no FMA contraction so that x86 and Arm hosts round identically)."""
    if force or not os.path.exists(_LIB) or any(os.path.getmtime(_LIB) < os.path.getmtime(p) for p in _DEPS):
        tmp = _LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fPIC",
                               "-shared", "-pthread", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    if _lib is None:
        build()
        lib = ctypes.CDLL(_LIB)
        dp = ctypes.POINTER(ctypes.c_double)
        ip = ctypes.POINTER(ctypes.c_int)
        lib.or_rule.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        lib.or_rule.restype = ctypes.c_int
        lib.or_delta_rule.argtypes = [ctypes.c_int, ctypes.c_int, dp, dp]
        lib.or_delta_rule.restype = ctypes.c_int
        lib.or_integrate.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int,
                                     ctypes.c_int, ctypes.c_int, dp]
        lib.or_integrate.restype = ctypes.c_int
        lib.or_points.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp,
                                  ctypes.c_long]
        lib.or_points.restype = ctypes.c_long
        lib.or_count_points.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.or_count_points.restype = ctypes.c_uint64
        lib.or_count_distinct.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int]
        lib.or_count_distinct.restype = ctypes.c_uint64
        lib.or_gradient.argtypes = [ctypes.c_int, ctypes.c_int, dp, ctypes.c_int, ctypes.c_int, ip,
                                    ctypes.c_int, ctypes.c_int, dp, dp]
        lib.or_gradient.restype = ctypes.c_int
        _lib = lib
    return _lib


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def rule(kind: int, level: int):
    """Level-``level`` 1-D rule on [0,1]: (nodes, weights)."""
    lib = _load()
    n = lib.or_rule(kind, level, None, None)
    if n < 0:
        raise ValueError("invalid rule/level")
    x = np.zeros(n)
    w = np.zeros(n)
    lib.or_rule(kind, level, _dp(x), _dp(w))
    return x, w


def delta_rule(kind: int, level: int):
    """Difference rule J^l - J^{l-1} on the union node set: (nodes, weights)."""
    lib = _load()
    n = lib.or_delta_rule(kind, level, None, None)
    if n < 0:
        raise ValueError("invalid rule/level")
    x = np.zeros(n)
    w = np.zeros(n)
    lib.or_delta_rule(kind, level, _dp(x), _dp(w))
    return x, w


class Result:
    """Oracle value Q = mant * 2**exp2, with the conditioning of its final sum."""

    def __init__(self, out):
        self.mant = float(out[0])
        self.exp2 = int(out[1])
        self.value = float(out[2])
        self.cond = float(out[3])

    def __repr__(self):
        return "Result(mant=%r, exp2=%d, value=%r, cond=%.3g)" % (
            self.mant, self.exp2, self.value, self.cond)


def integrate(kind: int, fam: int, params, d: int, L: int, form: int = FORM_DIFF,
              nthreads: int = 0) -> Result:
    """Smolyak value Q_d^{d+L} f on [0,1]^d (difference or combination form)."""
    lib = _load()
    p = np.ascontiguousarray(params, dtype=np.float64)
    if p.size != 2 * d:
        raise ValueError("params must hold 2d doubles")
    out = np.zeros(5)
    if lib.or_integrate(kind, fam, _dp(p), d, L, form, nthreads, _dp(out)) != 0:
        raise ValueError("invalid arguments")
    return Result(out)


def gradient(kind: int, fam: int, params, d: int, L: int, idx, nthreads: int = 0):
    """(Result, grad) with dQ/dparams[idx[t]] = grad[t] * 2**Result.exp2."""
    lib = _load()
    p = np.ascontiguousarray(params, dtype=np.float64)
    ix = np.ascontiguousarray(idx, dtype=np.int32)
    out = np.zeros(5)
    g = np.zeros(ix.size)
    rc = lib.or_gradient(kind, fam, _dp(p), d, L, ix.ctypes.data_as(ctypes.POINTER(ctypes.c_int)),
                         ix.size, nthreads, _dp(out), _dp(g))
    if rc != 0:
        raise ValueError("invalid arguments")
    out[2] = np.ldexp(out[0], int(out[1]))
    return Result(out), g


def points(kind: int, d: int, L: int, form: int = FORM_DIFF):
    """All tensor points (with repetition) and their weights: (X[n,d], W[n])."""
    lib = _load()
    n = lib.or_points(kind, d, L, form, None, None, 0)
    if n < 0:
        raise ValueError("invalid arguments")
    X = np.zeros((n, d))
    W = np.zeros(n)
    lib.or_points(kind, d, L, form, _dp(X), _dp(W), n)
    return X, W


def count_points(kind: int, d: int, L: int) -> int:
    """n_d^q: point count of Eq. 2.6's tensor grids, with repetition."""
    return int(_load().or_count_points(kind, d, L))


def count_distinct(kind: int, d: int, L: int) -> int:
    """Distinct points of the sparse grid of a nested rule (0 for Gauss-Legendre)."""
    return int(_load().or_count_distinct(kind, d, L))
