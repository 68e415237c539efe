"""torch.autograd.Function wrappers of the library's calls (argument marshalling only).

Each Function's forward and backward call the C ABI; no arithmetic runs in Python.  Complex
gradients follow the paper's convention (Sec. 2.2.2), which is also torch's for a real loss:
the gradient of a complex tensor holds dL/d(re) + i dL/d(im).

* CgDcSolve  x = S_lambda^{-1} rhs by CG (Eq. 6, Sec. 2.3.2).  Its derivative is written
             through the same self-adjoint operator: grad_rhs = S^{-1} g (a second CG solve)
             and grad_lambda = -Re<S^{-1} g, x> (cg_dc_solve_backward).
* Denoiser   D_W(x) = x + CNN(x), the MoDL residual CNN (denoiser_forward / _backward).
* UnrolledStep  one MoDL block x_next = S_lambda^{-1}(A^H y + lambda D_W(x_t)) (unrolled_step /
             unrolled_step_backward_ex), or one VarNet stage (Eq. 5, Sec. 2.3.1) with kind
             DENOISER_VARNET, where lambda_t is part of the stage parameters.

Activations: by default each Denoiser and UnrolledStep application keeps its own workspace
(the MoDL denoiser's activations and output, or a VarNet stage's K x and Phi'(K x)) until its
backward, which then reuses them; with
store=False the backward recomputes them from the block input instead (the checkpointing of
Sec. 2.2.4).  The results are the same either way.

A^H y is data: UnrolledStep returns no gradient for it.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from .denoiser import ModlDenoiser
from .sense import SensePlan


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _c64(t: torch.Tensor, name: str, shape) -> torch.Tensor:
    if t.dtype != torch.complex64 or tuple(t.shape) != tuple(shape) or t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA complex64 tensor of shape {tuple(shape)}")
    return t.contiguous()


def _lam(lam: torch.Tensor, B: int) -> torch.Tensor:
    if lam.dtype != torch.float64 or lam.numel() not in (1, B) or lam.device.type != "cuda":
        raise ValueError("lambda must be a CUDA float64 tensor of 1 or B values")
    return lam.contiguous()


class CgDcSolve(torch.autograd.Function):
    """x = (A^H A + lambda I)^{-1} rhs by `iters` CG iterations from zero, per slice."""

    @staticmethod
    def forward(ctx, plan: SensePlan, rhs: torch.Tensor, lam: torch.Tensor, iters: int):
        shape = plan.img_shape()
        rhs = _c64(rhs, "rhs", shape)
        lam = _lam(lam, shape[0])
        x = plan.cg_solve(rhs, lam, iters)
        ctx.plan, ctx.iters = plan, iters
        ctx.save_for_backward(x, lam)
        return x

    @staticmethod
    def backward(ctx, grad_x):
        x, lam = ctx.saved_tensors
        g = _c64(grad_x, "grad_x", x.shape)
        gl = torch.empty(lam.numel(), dtype=torch.float64, device=x.device)
        v, gl = ctx.plan.cg_solve_backward(g, x, None, lam, ctx.iters, grad_lam=gl)
        return None, v, (gl if ctx.needs_input_grad[2] else None), None


class Denoiser(torch.autograd.Function):
    """D_W(x) = x + CNN(x) for x complex64 [B, H, W] and weights float32 (MoDL layout)."""

    @staticmethod
    def forward(ctx, weights: torch.Tensor, x: torch.Tensor, store: bool = True):
        B, H, W = x.shape
        x = _c64(x, "x", (B, H, W))
        dn = ModlDenoiser(B, H, W, device=x.device)
        out = dn.forward(weights.contiguous(), x)
        ctx.dn, ctx.store = (dn if store else None), store
        ctx.save_for_backward(weights, x)
        return out

    @staticmethod
    def backward(ctx, grad_out):
        weights, x = ctx.saved_tensors
        B, H, W = x.shape
        dn = ctx.dn if ctx.store else ModlDenoiser(B, H, W, device=x.device)
        gw = torch.zeros_like(weights)
        gx = dn.backward(weights.contiguous(), x, _c64(grad_out, "grad_out", x.shape), gw,
                         recompute=not ctx.store)
        ctx.dn = None
        return gw, gx, None


class UnrolledStep(torch.autograd.Function):
    """One unrolled block on `plan`: MoDL (kind DENOISER_MODL; weights float32 [113154],
    lam float64 [1]) or a VarNet stage (kind DENOISER_VARNET; weights = the stage's float32
    parameter vector, lambda_t inside it; pass lam=None)."""

    @staticmethod
    def forward(ctx, plan: SensePlan, kind: int, weights: torch.Tensor, lam, AHy: torch.Tensor,
                x_t: torch.Tensor, cg_iters: int = 10, store: bool = True):
        L = _lib.lib()
        shape = plan.img_shape()
        B, H, W = shape
        AHy = _c64(AHy, "AHy", shape)
        x_t = _c64(x_t, "x_t", shape)
        weights = weights.contiguous()
        if kind == _lib.DENOISER_MODL:
            lam = _lam(lam, 1)
            nb = L.denoiser_workspace_bytes(kind, B, H, W)
        elif kind == _lib.DENOISER_VARNET:
            lam = torch.zeros(1, dtype=torch.float64, device=x_t.device)  # unused by the call
            nb = L.varnet_workspace_bytes(B, H, W)
        else:
            raise ValueError("kind must be DENOISER_MODL or DENOISER_VARNET")
        if nb == 0:
            raise ValueError("unsupported shape")
        ws = torch.zeros(int(nb), dtype=torch.uint8, device=x_t.device)
        x_next = torch.empty_like(x_t)
        plan._sync_stream()
        _lib.check("unrolled_step", L.unrolled_step(
            plan._h, kind, _p(weights), _p(lam), _p(AHy), _p(x_t), _p(x_next), int(cg_iters),
            _p(ws), ws.numel()))
        ctx.plan, ctx.kind, ctx.iters = plan, kind, int(cg_iters)
        ctx.store = bool(store)
        ctx.ws = ws
        ctx.save_for_backward(weights, lam, AHy, x_t, x_next)
        return x_next

    @staticmethod
    def backward(ctx, grad_next):
        weights, lam, AHy, x_t, x_next = ctx.saved_tensors
        L = _lib.lib()
        g = _c64(grad_next, "grad_next", x_t.shape)
        grad_t = torch.empty_like(x_t)
        gw = torch.zeros_like(weights)
        gl = torch.zeros(1, dtype=torch.float64, device=x_t.device)
        ctx.plan._sync_stream()
        _lib.check("unrolled_step_backward_ex", L.unrolled_step_backward_ex(
            ctx.plan._h, ctx.kind, _p(weights), _p(lam), _p(AHy), _p(x_t), _p(x_next), _p(g),
            _p(grad_t), _p(gw), _p(gl), ctx.iters, _p(ctx.ws), ctx.ws.numel(),
            0 if ctx.store else 1))
        ctx.ws = None
        glam = gl if (ctx.kind == _lib.DENOISER_MODL and ctx.needs_input_grad[3]) else None
        return None, None, gw, glam, None, grad_t, None, None
