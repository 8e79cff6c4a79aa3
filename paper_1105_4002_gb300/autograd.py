"""phi(x; b) as a torch.autograd.Function.

forward:  phi = 1/2 ||A x - b||^2 + alpha TV_tau(x)  (tvr_phi_and_grad / _f64), saving r = A x - b;
backward: the VJP kernel (tvr_phi_vjp / _f64) gives
          grad_x = w (A^T r + alpha grad TV_tau(x)),  grad_b = -w r,
          w the upstream gradient of phi.
float32 tensors use the hot-path kernels; float64 tensors use the FP64 variants
(for gradcheck).  Only argument marshalling happens here.
"""
from __future__ import annotations

import ctypes

import torch

from . import System
from ._capi import check, lib


def _p(t):
    return ctypes.c_void_p(t.data_ptr()) if t is not None else None


class PhiFunction(torch.autograd.Function):
    @staticmethod
    def forward(ctx, x, b, system: System, alpha: float, tau: float):
        if x.dtype != b.dtype or x.dtype not in (torch.float32, torch.float64):
            raise TypeError("x and b must both be float32 or both float64")
        if not (x.is_cuda and b.is_cuda):
            raise ValueError("x and b must be CUDA tensors")
        x = x.detach().contiguous()
        b = b.detach().contiguous()
        if x.numel() != system.N or b.numel() != system.m:
            raise ValueError("x must have N entries and b m entries")
        stream = ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
        resid = torch.empty(system.m, dtype=x.dtype, device=x.device)
        phi = torch.empty(4, dtype=torch.float64, device=x.device)
        if x.dtype == torch.float32:
            st = lib().tvr_phi_and_grad(system.handle, _p(x), _p(b), float(alpha), float(tau),
                                        _p(phi), None, None, _p(resid), stream)
            check(st, "tvr_phi_and_grad")
        else:
            grad = torch.empty_like(x)
            st = lib().tvr_phi_and_grad_f64(system.handle, _p(x), _p(b), float(alpha), float(tau),
                                            _p(phi), None, _p(grad), _p(resid), stream)
            check(st, "tvr_phi_and_grad_f64")
        ctx.save_for_backward(x, resid)
        ctx.system, ctx.alpha, ctx.tau = system, float(alpha), float(tau)
        return phi[0].to(x.dtype)

    @staticmethod
    def backward(ctx, grad_out):
        x, resid = ctx.saved_tensors
        w = grad_out.detach().to(torch.float64).reshape(1).contiguous()
        gx = torch.empty_like(x)
        gb = torch.empty_like(resid) if ctx.needs_input_grad[1] else None
        stream = ctypes.c_void_p(torch.cuda.current_stream(x.device).cuda_stream)
        fn = lib().tvr_phi_vjp if x.dtype == torch.float32 else lib().tvr_phi_vjp_f64
        check(fn(ctx.system.handle, _p(x), _p(resid), ctx.alpha, ctx.tau, _p(w), _p(gx), _p(gb),
                 stream), "tvr_phi_vjp")
        return (gx if ctx.needs_input_grad[0] else None), gb, None, None, None


def phi(x, b, system: System, alpha: float, tau: float):
    """Differentiable phi(x; b) (0-dim tensor of x's dtype)."""
    return PhiFunction.apply(x, b, system, alpha, tau)
