"""ctypes access to the host-side index checker of the fold kernel (tests only)."""
import ctypes
import os
import subprocess

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
CSRC = os.path.join(ROOT, "paper_2210_14313_gb300", "csrc")
LIB = os.path.join(HERE, "libsgcheck.so")
SRCS = [os.path.join(HERE, "sg_index_check.cpp"), os.path.join(CSRC, "sg_plan.cpp"),
        os.path.join(CSRC, "sg_rules.cpp")]
_lib = None


def build():
    deps = SRCS + [os.path.join(CSRC, h) for h in os.listdir(CSRC) if h.endswith(".h")]
    if not os.path.exists(LIB) or any(os.path.getmtime(p) > os.path.getmtime(LIB) for p in deps):
        tmp = LIB + ".tmp%d" % os.getpid()
        subprocess.check_call(["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-ffp-contract=off",
                               "-I/usr/local/cuda/include", "-o", tmp, *SRCS])
        os.replace(tmp, LIB)
    return LIB


def _load():
    global _lib
    if _lib is None:
        build()
        _lib = ctypes.CDLL(LIB)
        _lib.chk_run.restype = ctypes.c_int
    return _lib


def run(kind, fam, params, d, L, form=2, grad=0, ppc=2048, ctas_per_sm=8, warps=8):
    p = np.ascontiguousarray(params, dtype=np.float64)
    out = np.zeros(10)
    nv = ctypes.c_longlong(0)
    cap = 2 * d * 64 if grad else 1
    v = np.zeros(max(cap, 1))
    dp = ctypes.POINTER(ctypes.c_double)
    rc = _load().chk_run(kind, fam, p.ctypes.data_as(dp), d, L, form, grad, ppc, ctas_per_sm, warps,
                         out.ctypes.data_as(dp), v.ctypes.data_as(dp) if grad else None,
                         ctypes.byref(nv))
    if rc != 0:
        raise RuntimeError("chk_run failed with %d" % rc)
    return dict(rel=out[0], logscale=out[1], violations=int(out[2]), badpairs=int(out[3]),
                evals=int(out[4]), chunks=int(out[5]), plan_evals=int(out[6]), rel_shift=out[7], lane_slots=int(out[8]),
                max_runs=int(out[9]),
                v=v[:nv.value])


def unrank_mismatches(d, r, n=2000):
    """Mismatches between the kernel's 32-wide unranking rounds and the serial search."""
    lib = _load()
    lib.chk_unrank.restype = ctypes.c_longlong
    lib.chk_unrank.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_longlong]
    return lib.chk_unrank(d, r, n)


def rule(kind, level):
    """The library's level-``level`` rule on [0,1] (kind may carry the slow-growth flag 16)."""
    lib = _load()
    x = np.zeros(2 * 4097 + 2)
    w = np.zeros(2 * 4097 + 2)
    dp = ctypes.POINTER(ctypes.c_double)
    n = lib.chk_rule(kind, level, x.ctypes.data_as(dp), w.ctypes.data_as(dp))
    return x[:n].copy(), w[:n].copy()


def block(kind, bk, k):
    """The library's rule block (0 difference, 1 full, 2 telescoped tail) at excess k."""
    lib = _load()
    x = np.zeros(2 * 4097 + 2)
    w = np.zeros(2 * 4097 + 2)
    dp = ctypes.POINTER(ctypes.c_double)
    n = lib.chk_block(kind, bk, k, x.ctypes.data_as(dp), w.ctypes.data_as(dp))
    return x[:n].copy(), w[:n].copy()


def fixed(kind, x, phi=0.0, w=None):
    """The FP64 fold's fixed-point functions built for the host (sg_fixed.h):
    kind 0 expm1, kind 1 (sin, cos) pairs, kind 2 sin(x) sin(phi + x),
    kind 3 w sin(x) sin(phi + x), kind 4 w expm1(x)."""
    lib = _load()
    dp = ctypes.POINTER(ctypes.c_double)
    lib.chk_fixed.argtypes = [ctypes.c_int, dp, dp, dp, ctypes.c_longlong, ctypes.c_double]
    x = np.ascontiguousarray(x, dtype=np.float64)
    wv = np.ascontiguousarray(np.ones_like(x) if w is None else w, dtype=np.float64)
    y = np.zeros(len(x) * (2 if kind == 1 else 1))
    lib.chk_fixed(kind, x.ctypes.data_as(dp), wv.ctypes.data_as(dp), y.ctypes.data_as(dp), len(x), phi)
    return y


def xsum(v):
    """(s, c) of the reduction's exact 128-bit window sum of v (sg_xsum.h)."""
    lib = _load()
    dp = ctypes.POINTER(ctypes.c_double)
    lib.chk_xsum.argtypes = [dp, ctypes.c_longlong, dp]
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(2)
    lib.chk_xsum(v.ctypes.data_as(dp), len(v), out.ctypes.data_as(dp))
    return out[0], out[1]


def divmagic_mismatches(mmax):
    """Mismatches of the kernels' divide-free q / m for m <= mmax."""
    lib = _load()
    lib.chk_divmagic.restype = ctypes.c_longlong
    lib.chk_divmagic.argtypes = [ctypes.c_int]
    return lib.chk_divmagic(mmax)


def xsum_adaptive(v, nthreads):
    """(s, c) of the setup kernel's adaptive-unit window sums over nthreads."""
    lib = _load()
    dp = ctypes.POINTER(ctypes.c_double)
    lib.chk_xsum_adaptive.argtypes = [dp, ctypes.c_longlong, ctypes.c_int, dp]
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(2)
    lib.chk_xsum_adaptive(v.ctypes.data_as(dp), len(v), nthreads, out.ctypes.data_as(dp))
    return out[0], out[1]


def fx_to_double(v, neg, q):
    """sg_fx_to_double_f of (v, neg, q) triples (sg_fixed.h), built for the host."""
    lib = _load()
    lib.chk_fx_to_double.argtypes = [ctypes.c_void_p, ctypes.c_void_p, ctypes.c_void_p, ctypes.c_longlong,
                                     ctypes.c_void_p]
    v = np.ascontiguousarray(v, dtype=np.uint64)
    neg = np.ascontiguousarray(neg, dtype=np.uint64)
    q = np.ascontiguousarray(q, dtype=np.int32)
    y = np.zeros(len(v))
    lib.chk_fx_to_double(v.ctypes.data, neg.ctypes.data, q.ctypes.data, len(v), y.ctypes.data)
    return y


def lacc(v, nparts=1):
    """(s, c, overflow) of the single-integral fold's long accumulator
    (sg_lacc.h) over v, split into nparts parts whose limbs are added."""
    lib = _load()
    dp = ctypes.POINTER(ctypes.c_double)
    lib.chk_lacc.argtypes = [dp, ctypes.c_longlong, ctypes.c_int, dp]
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(4)
    lib.chk_lacc(v.ctypes.data_as(dp), len(v), nparts, out.ctypes.data_as(dp))
    if out[3]:
        raise AssertionError("%d non-zero digits outside the three added per term" % out[3])
    return out[0], out[1], int(out[2])


def lacc_x(v, nparts=1):
    """(s, c, overflow, |sum| of the parts) of the long accumulator fed with
    the exact 128-bit window sums of nparts parts of v (sg_la_x_digit)."""
    lib = _load()
    dp = ctypes.POINTER(ctypes.c_double)
    lib.chk_lacc_x.argtypes = [dp, ctypes.c_longlong, ctypes.c_int, dp]
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(4)
    lib.chk_lacc_x(v.ctypes.data_as(dp), len(v), nparts, out.ctypes.data_as(dp))
    return out[0], out[1], int(out[2]), out[3]


def ratio(a, b):
    """sg_ratio(a, b) elementwise (the library's float-precision quotient)."""
    lib = _load()
    dp = ctypes.POINTER(ctypes.c_double)
    lib.chk_ratio.argtypes = [dp, dp, ctypes.c_longlong, dp]
    a = np.ascontiguousarray(a, dtype=np.float64)
    b = np.ascontiguousarray(b, dtype=np.float64)
    out = np.zeros(len(a))
    lib.chk_ratio(a.ctypes.data_as(dp), b.ctypes.data_as(dp), len(a), out.ctypes.data_as(dp))
    return out


def merged_points(kind, d, L):
    """Every point of the merged form (distinct points of the sparse grid
    except the centre) with the planner's merged weight: (X[n, d], W[n])."""
    lib = _load()
    dp = ctypes.POINTER(ctypes.c_double)
    lib.chk_merged_points.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_longlong]
    lib.chk_merged_points.restype = ctypes.c_longlong
    n = lib.chk_merged_points(kind, d, L, None, None, 0)
    if n < 0:
        raise RuntimeError("merged weights failed")
    X = np.zeros((n, d))
    W = np.zeros(n)
    lib.chk_merged_points(kind, d, L, X.ctypes.data_as(dp), W.ctypes.data_as(dp), n)
    return X, W


def lacc_limbs(v):
    """The 32 carry-save limbs of the long accumulator over v (as the kernels add chunk sums)."""
    lib = _load()
    dp = ctypes.POINTER(ctypes.c_double)
    lib.chk_lacc_limbs.argtypes = [dp, ctypes.c_longlong, ctypes.c_void_p]
    v = np.ascontiguousarray(v, dtype=np.float64)
    out = np.zeros(32, dtype=np.int64)
    lib.chk_lacc_limbs(v.ctypes.data_as(dp), len(v), out.ctypes.data)
    return out
