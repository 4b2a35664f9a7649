"""torch.autograd.Function around the forward and adjoint kernels.

``sg_quad(params, rule, fam, d, q)`` returns Q_d^q f as a 0-d float64 CUDA
tensor; its backward runs the library's adjoint kernel (sg_integrate_grad),
which gives dQ/dparams for all 2d parameters [a, u] at once.
"""
from __future__ import annotations

import ctypes

import torch

from . import (PREC_FP64, FORM_AUTO, sg_result, _check, _stream_handle, load)


class SgQuad(torch.autograd.Function):
    @staticmethod
    def forward(ctx, params, rule, fam, d, q, prec=PREC_FP64):
        if not (params.is_cuda and params.dtype == torch.float64 and params.numel() == 2 * d):
            raise ValueError("params must be a CUDA float64 tensor of 2d elements")
        p = params.contiguous()
        r = sg_result()
        _check(load().sg_integrate(rule.handle, fam, ctypes.c_void_p(p.data_ptr()), 1, d, q, prec,
                                   FORM_AUTO, _stream_handle(), ctypes.byref(r)), "sg_integrate")
        ctx.save_for_backward(p)
        ctx.cfg = (rule, fam, d, q, prec)
        return torch.tensor(r.value, dtype=torch.float64, device=params.device)

    @staticmethod
    def backward(ctx, grad_out):
        (p,) = ctx.saved_tensors
        rule, fam, d, q, prec = ctx.cfg
        g = torch.empty(2 * d, dtype=torch.float64, device=p.device)
        r = sg_result()
        _check(load().sg_integrate_grad(rule.handle, fam, ctypes.c_void_p(p.data_ptr()), 1, d, q, prec,
                                        _stream_handle(), ctypes.byref(r),
                                        ctypes.c_void_p(g.data_ptr()), 1), "sg_integrate_grad")
        return g * grad_out, None, None, None, None, None


def sg_quad(params, rule, fam, d, q, prec=PREC_FP64):
    return SgQuad.apply(params, rule, fam, d, q, prec)
