"""Python binding of libsg: Smolyak sparse-grid quadrature on a GB300 GPU,
evaluated by multilevel dimension iteration.

Argument marshalling only: every step of the computation runs in the CUDA
kernels of ``libsg.so`` (built in-tree by ``_build.build()``).  There is no
CPU fallback: if the library cannot be loaded, every call raises.

PyTorch is used for device memory and streams: tensors passed here must be
float64, contiguous and on the current CUDA device; calls run on
``torch.cuda.current_stream()``.
"""
from __future__ import annotations

import ctypes
import os

import numpy as np

from ._build import LIB as _LIB_PATH, build as _build_lib

# enums of include/sg.h
RULE_TRAPEZOID, RULE_CLENSHAW_CURTIS, RULE_GAUSS_PATTERSON, RULE_GAUSS_LEGENDRE = 1, 2, 3, 4
GROWTH_STANDARD, GROWTH_SLOW = 0, 1
FAM_EXP_LINEAR, FAM_OSCILLATORY, FAM_PRODUCT_PEAK, FAM_GAUSSIAN, FAM_GAUSSIAN_LIN = 0, 1, 2, 3, 4
PREC_FP64, PREC_MIXED, PREC_FF = 0, 1, 2
FORM_AUTO, FORM_DIFFERENCE, FORM_TELESCOPED, FORM_COMBINATION, FORM_MERGED = 0, 1, 2, 3, 4

SG_OK = 0
STATUS_NAMES = {0: "SG_OK", 1: "SG_EINVAL", 2: "SG_ERANGE", 3: "SG_ENOMEM", 4: "SG_ECUDA",
                5: "SG_ETIMEOUT", 6: "SG_EUNSUPPORTED"}

# every function include/sg.h declares
ABI_SYMBOLS = ["sg_rule_init", "sg_rule_init_growth", "sg_rule_destroy", "sg_rule_nodes", "sg_count_points",
               "sg_integrate", "sg_integrate_async", "sg_integrate_batch", "sg_integrate_grad",
               "sg_status_string", "sg_get_tuning", "sg_set_tuning", "sg_autotune",
               "sg_profile_begin", "sg_profile_end", "sg_ceiling", "sg_integrate_noalloc",
               "sg_eval_functions", "sg_integrand_create", "sg_integrand_destroy", "sg_integrand_log",
               "sg_integrate_user", "sg_autotune_classes", "sg_tuning_load", "sg_tuning_clear", "sg_integrate_batch_shard", "sg_shard_combine"]


class SgError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__("%s failed: %s (%s)" % (where, STATUS_NAMES.get(status, status),
                                                 _status_text(status)))


class sg_result(ctypes.Structure):
    _fields_ = [("value", ctypes.c_double), ("mant", ctypes.c_double), ("exp2", ctypes.c_int64),
                ("cond", ctypes.c_double), ("err_est", ctypes.c_double),
                ("points", ctypes.c_uint64), ("evals", ctypes.c_uint64),
                ("seconds", ctypes.c_double)]


class sg_item(ctypes.Structure):
    _fields_ = [("rule", ctypes.c_void_p), ("fam", ctypes.c_int), ("d", ctypes.c_int),
                ("q", ctypes.c_int), ("param_offset", ctypes.c_uint64)]


class sg_tuning(ctypes.Structure):
    _fields_ = [("points_per_chunk", ctypes.c_int), ("ctas_per_sm", ctypes.c_int),
                ("warps_per_cta", ctypes.c_int)]


DEV_RESULT_DOUBLES = 7  # sg_dev_result: mant, exp2, value, cond, err_est, sum, abs_sum

_lib = None


def load(build_if_missing: bool = True):
    """Loads libsg.so (building it first if needed).  Raises if unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    if build_if_missing:
        _build_lib()
    if not os.path.exists(_LIB_PATH):
        raise ImportError("libsg.so is not built (%s); run paper_2210_14313_gb300._build.build()"
                          % _LIB_PATH)
    lib = ctypes.CDLL(_LIB_PATH)
    vp, dp, ip = ctypes.c_void_p, ctypes.POINTER(ctypes.c_double), ctypes.c_int
    lib.sg_rule_init.argtypes = [ip, ip, ctypes.POINTER(vp)]
    lib.sg_rule_init_growth.argtypes = [ip, ip, ip, ctypes.POINTER(vp)]
    lib.sg_rule_destroy.argtypes = [vp]
    lib.sg_rule_nodes.argtypes = [vp, ip, dp, dp, ctypes.POINTER(ctypes.c_int)]
    lib.sg_count_points.argtypes = [vp, ip, ip, ip, ctypes.POINTER(ctypes.c_uint64),
                                    ctypes.POINTER(ctypes.c_uint64)]
    lib.sg_integrate.argtypes = [vp, ip, vp, ip, ip, ip, ip, ip, vp, ctypes.POINTER(sg_result)]
    lib.sg_integrate_async.argtypes = [vp, ip, vp, ip, ip, ip, ip, vp, vp]
    lib.sg_integrate_batch.argtypes = [ctypes.POINTER(sg_item), ip, vp, ip, ip, ctypes.c_double, vp,
                                       ctypes.POINTER(sg_result)]
    lib.sg_integrate_grad.argtypes = [vp, ip, vp, ip, ip, ip, ip, vp, ctypes.POINTER(sg_result), vp, ip]
    lib.sg_status_string.argtypes = [ip]
    lib.sg_status_string.restype = ctypes.c_char_p
    lib.sg_get_tuning.argtypes = [ip, ctypes.POINTER(sg_tuning)]
    lib.sg_set_tuning.argtypes = [ip, ctypes.POINTER(sg_tuning)]
    lib.sg_autotune.argtypes = [ctypes.POINTER(sg_item), ip, vp, ip, ip, ip, vp,
                                ctypes.POINTER(sg_tuning), ctypes.POINTER(ctypes.c_double)]
    lib.sg_autotune_classes.argtypes = [ctypes.POINTER(sg_item), ip, vp, ip, ip, ip, vp, ctypes.c_char_p,
                                        ctypes.POINTER(ctypes.c_int)]
    lib.sg_tuning_load.argtypes = [ctypes.c_char_p, ctypes.POINTER(ctypes.c_int)]
    lib.sg_tuning_clear.argtypes = []
    lib.sg_integrate_batch_shard.argtypes = [ctypes.POINTER(sg_item), ip, vp, ip, ip, ip, ip, vp, vp, vp]
    lib.sg_shard_combine.argtypes = [ctypes.POINTER(ctypes.c_void_p), ip, vp, ip, ctypes.POINTER(sg_result)]
    lib.sg_profile_begin.argtypes = [vp]
    lib.sg_profile_end.argtypes = [vp, ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_int)]
    lib.sg_ceiling.argtypes = [ip, ip, vp, ctypes.POINTER(ctypes.c_double)]
    lib.sg_integrate_noalloc.argtypes = [ip, ip, vp, ip, ip, ip, vp, vp]
    lib.sg_eval_functions.argtypes = [ip, ip, vp, vp, ip, vp]
    lib.sg_integrand_create.argtypes = [ctypes.c_char_p, ip, ctypes.POINTER(vp)]
    lib.sg_integrand_destroy.argtypes = [vp]
    lib.sg_integrand_log.argtypes = [vp, ctypes.c_char_p, ctypes.c_size_t, ctypes.POINTER(ctypes.c_size_t)]
    lib.sg_integrate_user.argtypes = [vp, vp, vp, ip, ip, ip, ip, vp, ctypes.POINTER(sg_result)]
    for name in ABI_SYMBOLS:
        if name != "sg_status_string":
            getattr(lib, name).restype = ctypes.c_int
    _lib = lib
    return lib


def _status_text(status: int) -> str:
    try:
        return load().sg_status_string(status).decode()
    except Exception:  # noqa: BLE001 - only used inside error messages
        return "?"


def _check(status: int, where: str):
    if status != SG_OK:
        raise SgError(status, where)


def _stream_handle(stream=None):
    import torch
    if stream is not None:
        return ctypes.c_void_p(stream.cuda_stream)
    raw = getattr(torch._C, "_cuda_getCurrentRawStream", None)
    if raw is not None:  # the current stream's handle without building a Stream object
        return ctypes.c_void_p(raw(torch.cuda.current_device()))
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


def _require_cuda():
    import torch
    if not torch.cuda.is_available():
        raise RuntimeError("libsg needs a CUDA device; none is available")


class Rule:
    """A 1-D rule family (trapezoid / Clenshaw-Curtis / Gauss-Patterson /
    Gauss-Legendre) with device tables for levels 1..max_level; ``growth``
    GROWTH_SLOW selects the paper's accuracy levels (Section 5.4)."""

    def __init__(self, kind: int, max_level: int = 8, growth: int = GROWTH_STANDARD):
        _require_cuda()
        lib = load()
        h = ctypes.c_void_p()
        _check(lib.sg_rule_init_growth(kind, growth, max_level, ctypes.byref(h)), "sg_rule_init_growth")
        self.handle = h
        self.kind = kind
        self.growth = growth
        self.max_level = max_level

    def nodes(self, level: int):
        lib = load()
        n = ctypes.c_int(0)
        _check(lib.sg_rule_nodes(self.handle, level, None, None, ctypes.byref(n)), "sg_rule_nodes")
        x = np.zeros(n.value)
        w = np.zeros(n.value)
        _check(lib.sg_rule_nodes(self.handle, level, x.ctypes.data_as(ctypes.POINTER(ctypes.c_double)),
                                 w.ctypes.data_as(ctypes.POINTER(ctypes.c_double)), ctypes.byref(n)),
               "sg_rule_nodes")
        return x, w

    def close(self):
        if getattr(self, "handle", None):
            load().sg_rule_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:  # noqa: BLE001 - interpreter shutdown
            pass


class Result:
    """Q = mant * 2**exp2 with diagnostics (see sg_result in include/sg.h)."""

    def __init__(self, r: sg_result):
        self.value = r.value
        self.mant = r.mant
        self.exp2 = r.exp2
        self.cond = r.cond
        self.err_est = r.err_est
        self.points = r.points
        self.evals = r.evals
        self.seconds = r.seconds

    def __repr__(self):
        return ("Result(value=%r, mant=%r, exp2=%d, cond=%.3g, err_est=%.2g, points=%d, evals=%d, "
                "seconds=%.3g)" % (self.value, self.mant, self.exp2, self.cond, self.err_est,
                                   self.points, self.evals, self.seconds))


def _params_arg(params, d):
    """(pointer, on_device, keepalive) for a params array of 2d doubles."""
    if (type(params) is np.ndarray and params.dtype == np.float64 and params.flags.c_contiguous
            and params.size == 2 * d):
        return ctypes.c_void_p(params.ctypes.data), 0, params
    try:
        import torch
        if isinstance(params, torch.Tensor):
            if params.dtype != torch.float64 or not params.is_contiguous() or params.numel() != 2 * d:
                raise ValueError("params must be a contiguous float64 tensor of 2d elements")
            if params.is_cuda:
                return ctypes.c_void_p(params.data_ptr()), 1, params
            params = params.numpy()
    except ImportError:
        pass
    a = np.ascontiguousarray(params, dtype=np.float64)
    if a.size != 2 * d:
        raise ValueError("params must hold 2d doubles")
    return ctypes.c_void_p(a.ctypes.data), 0, a


def count_points(rule: Rule, d: int, q: int, form: int = FORM_AUTO):
    """(n_d^q, evaluations the kernels make) for this rule, d, q and form."""
    p, e = ctypes.c_uint64(), ctypes.c_uint64()
    _check(load().sg_count_points(rule.handle, d, q, form, ctypes.byref(p), ctypes.byref(e)),
           "sg_count_points")
    return p.value, e.value


def integrate(rule: Rule, fam: int, params, d: int, q: int, prec: int = PREC_FP64,
              form: int = FORM_AUTO, stream=None) -> Result:
    """One integral (blocking).  params: numpy array or float64 tensor of 2d entries."""
    ptr, on_dev, keep = _params_arg(params, d)
    r = sg_result()
    _check(load().sg_integrate(rule.handle, fam, ptr, on_dev, d, q, prec, form,
                               _stream_handle(stream), ctypes.byref(r)), "sg_integrate")
    del keep
    return Result(r)


def integrate_async(rule: Rule, fam: int, d_params, d: int, q: int, d_out, prec: int = PREC_FP64,
                    form: int = FORM_AUTO, stream=None):
    """Enqueues one integral; d_params (2d) and d_out (7 doubles) are CUDA
    float64 tensors.  Nothing synchronises."""
    _check(load().sg_integrate_async(rule.handle, fam, ctypes.c_void_p(d_params.data_ptr()), d, q,
                                     prec, form, _stream_handle(stream),
                                     ctypes.c_void_p(d_out.data_ptr())), "sg_integrate_async")


def _items(specs):
    """specs: list of (rule, fam, d, q, param_offset)."""
    arr = (sg_item * len(specs))()
    for k, (rule, fam, d, q, off) in enumerate(specs):
        arr[k].rule = rule.handle
        arr[k].fam = fam
        arr[k].d = d
        arr[k].q = q
        arr[k].param_offset = off
    return arr


def integrate_batch(specs, pool, prec: int = PREC_MIXED, guard_tol: float = 0.0, stream=None):
    """Batch of integrals in one persistent launch (CUDA graph).  specs: list of
    (rule, fam, d, q, param_offset); pool: parameters (numpy or CUDA tensor)."""
    arr = _items(specs)
    try:
        import torch
        on_dev = isinstance(pool, torch.Tensor) and pool.is_cuda
    except ImportError:
        on_dev = False
    if on_dev:
        ptr, keep = ctypes.c_void_p(pool.data_ptr()), pool
    else:
        keep = np.ascontiguousarray(pool, dtype=np.float64)
        ptr = ctypes.c_void_p(keep.ctypes.data)
    res = (sg_result * len(specs))()
    _check(load().sg_integrate_batch(arr, len(specs), ptr, 1 if on_dev else 0, prec, guard_tol,
                                     _stream_handle(stream), res), "sg_integrate_batch")
    del keep
    return [Result(r) for r in res]


class Integrand:
    """A user integrand compiled at run time (sg_integrand_create): CUDA C++
    source defining sg_user_centre / sg_user_move / sg_user_value (and
    optionally sg_user_deviation) over a state of ``state_size`` doubles."""

    def __init__(self, source: str, state_size: int):
        _require_cuda()
        lib = load()
        h = ctypes.c_void_p()
        st = lib.sg_integrand_create(source.encode(), state_size, ctypes.byref(h))
        if st != 0:
            log = _integrand_log(h) if h.value else ""
            if h.value:
                lib.sg_integrand_destroy(h)
            err = SgError(st, "sg_integrand_create")
            err.log = log
            raise err
        self.handle = h
        self.state_size = state_size

    def log(self) -> str:
        return _integrand_log(self.handle)

    def close(self):
        if getattr(self, "handle", None):
            load().sg_integrand_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _integrand_log(h) -> str:
    lib = load()
    n = ctypes.c_size_t(0)
    lib.sg_integrand_log(h, None, 0, ctypes.byref(n))
    buf = ctypes.create_string_buffer(n.value + 1)
    lib.sg_integrand_log(h, buf, n.value + 1, None)
    return buf.value.decode(errors="replace")


def integrate_user(rule: Rule, f: Integrand, params, d: int, q: int, stream=None) -> Result:
    """Q_d^q of a user integrand (FP64); params: host or CUDA array of doubles."""
    lib = load()
    if params is None:
        params = np.zeros(0)
    if isinstance(params, np.ndarray) or not hasattr(params, "data_ptr"):
        p = np.ascontiguousarray(params, dtype=np.float64)
        ptr, n, on_dev = p.ctypes.data_as(ctypes.c_void_p), p.size, 0
    else:
        import torch
        if params.dtype != torch.float64 or not params.is_contiguous():
            raise ValueError("params must be a contiguous float64 tensor")
        ptr, n, on_dev = ctypes.c_void_p(params.data_ptr()), params.numel(), 1
    r = sg_result()
    _check(lib.sg_integrate_user(rule.handle, f.handle, ptr, n, on_dev, d, q, _stream_handle(stream),
                                 ctypes.byref(r)), "sg_integrate_user")
    return Result(r)


def integrate_grad(rule: Rule, fam: int, params, d: int, q: int, prec: int = PREC_FP64, stream=None):
    """(Result, dQ/dparams as a numpy array of 2d entries) via the adjoint kernel."""
    ptr, on_dev, keep = _params_arg(params, d)
    g = np.zeros(2 * d)
    r = sg_result()
    _check(load().sg_integrate_grad(rule.handle, fam, ptr, on_dev, d, q, prec, _stream_handle(stream),
                                    ctypes.byref(r), ctypes.c_void_p(g.ctypes.data), 0),
           "sg_integrate_grad")
    del keep
    return Result(r), g


def get_tuning(prec: int):
    t = sg_tuning()
    _check(load().sg_get_tuning(prec, ctypes.byref(t)), "sg_get_tuning")
    return (t.points_per_chunk, t.ctas_per_sm, t.warps_per_cta)


def set_tuning(prec: int, points_per_chunk: int, ctas_per_sm: int, warps_per_cta: int):
    t = sg_tuning(points_per_chunk, ctas_per_sm, warps_per_cta)
    _check(load().sg_set_tuning(prec, ctypes.byref(t)), "sg_set_tuning")


def autotune(specs, pool, prec: int = PREC_MIXED, reps: int = 3, stream=None):
    """Times the batch under a grid of tunings, keeps the fastest; returns
    ((points_per_chunk, ctas_per_sm, warps_per_cta), median ms)."""
    arr = _items(specs)
    keep = np.ascontiguousarray(pool, dtype=np.float64)
    t = sg_tuning()
    ms = ctypes.c_double()
    _check(load().sg_autotune(arr, len(specs), ctypes.c_void_p(keep.ctypes.data), 0, prec, reps,
                              _stream_handle(stream), ctypes.byref(t), ctypes.byref(ms)),
           "sg_autotune")
    return (t.points_per_chunk, t.ctas_per_sm, t.warps_per_cta), ms.value


SHARD_LIMBS = 64


class sg_shard_info(ctypes.Structure):
    _fields_ = [("mult", ctypes.c_double), ("base_rel", ctypes.c_double), ("scale_m", ctypes.c_double),
                ("scale_e2", ctypes.c_double), ("unit_roundoff", ctypes.c_double), ("points", ctypes.c_uint64),
                ("evals", ctypes.c_uint64)]


def integrate_batch_shard(specs, pool, shard: int, nshards: int, prec: int = PREC_FP64, stream=None):
    """Shard `shard` of `nshards` of a batch (sg_integrate_batch_shard):
    (partials as an int64 array [n, SHARD_LIMBS], info array)."""
    arr = _items(specs)
    try:
        import torch
        on_dev = isinstance(pool, torch.Tensor) and pool.is_cuda
    except ImportError:
        on_dev = False
    if on_dev:
        ptr, keep = ctypes.c_void_p(pool.data_ptr()), pool
    else:
        keep = np.ascontiguousarray(pool, dtype=np.float64)
        ptr = ctypes.c_void_p(keep.ctypes.data)
    parts = np.zeros((len(specs), SHARD_LIMBS), dtype=np.int64)
    info = (sg_shard_info * len(specs))()
    _check(load().sg_integrate_batch_shard(arr, len(specs), ptr, 1 if on_dev else 0, prec, shard, nshards,
                                           _stream_handle(stream), ctypes.c_void_p(parts.ctypes.data),
                                           ctypes.cast(info, ctypes.c_void_p)), "sg_integrate_batch_shard")
    del keep
    return parts, info


def shard_combine(parts_list, info):
    """Adds the shards' limbs exactly and assembles every item (sg_shard_combine)."""
    parts_list = [np.ascontiguousarray(p, dtype=np.int64) for p in parts_list]
    n = parts_list[0].shape[0]
    ptrs = (ctypes.c_void_p * len(parts_list))(*[p.ctypes.data for p in parts_list])
    res = (sg_result * n)()
    _check(load().sg_shard_combine(ptrs, len(parts_list), ctypes.cast(info, ctypes.c_void_p), n, res),
           "sg_shard_combine")
    return [Result(r) for r in res]


def autotune_classes(specs, pool, prec: int = PREC_MIXED, reps: int = 1, path=None, stream=None) -> int:
    """Per-class chunk sizes for the batch path (sg_autotune_classes); returns
    the number of classes in the table, which later batches use."""
    arr = _items(specs)
    try:
        import torch
        on_dev = isinstance(pool, torch.Tensor) and pool.is_cuda
    except ImportError:
        on_dev = False
    if on_dev:
        ptr, keep = ctypes.c_void_p(pool.data_ptr()), pool
    else:
        keep = np.ascontiguousarray(pool, dtype=np.float64)
        ptr = ctypes.c_void_p(keep.ctypes.data)
    n = ctypes.c_int(0)
    _check(load().sg_autotune_classes(arr, len(specs), ptr, 1 if on_dev else 0, prec, reps,
                                      _stream_handle(stream), path.encode() if path else None,
                                      ctypes.byref(n)), "sg_autotune_classes")
    del keep
    return n.value


def tuning_load(path) -> int:
    """Loads a per-class table written by autotune_classes; returns its size."""
    n = ctypes.c_int(0)
    _check(load().sg_tuning_load(path.encode(), ctypes.byref(n)), "sg_tuning_load")
    return n.value


def tuning_clear():
    _check(load().sg_tuning_clear(), "sg_tuning_clear")


def profile_begin(stream=None):
    """Start timing every fold-kernel launch on the stream (CUDA events)."""
    _check(load().sg_profile_begin(_stream_handle(stream)), "sg_profile_begin")


def profile_end(stream=None):
    """(summed fold-kernel ms, launches) since profile_begin; synchronises."""
    ms, n = ctypes.c_double(), ctypes.c_int()
    _check(load().sg_profile_end(_stream_handle(stream), ctypes.byref(ms), ctypes.byref(n)),
           "sg_profile_end")
    return ms.value, n.value


def ceiling(prec: int, kind: int, stream=None) -> float:
    """Per-point throughput ceiling (points/s; kind 2: FMA FLOP/s) of this GPU."""
    r = ctypes.c_double()
    _check(load().sg_ceiling(prec, kind, _stream_handle(stream), ctypes.byref(r)), "sg_ceiling")
    return r.value


from .autograd import SgQuad, sg_quad  # noqa: E402,F401
