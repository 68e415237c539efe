"""Torch-facing wrapper of the MoDL denoiser entry points (marshalling only).

D_W(x) = x + CNN(x) of the MoDL update (Sec. 2.3.2, Eq. 6); the kernels live
in libsense.so (tcgen05 tensor-core convolutions for the 64-channel layers).
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


class ModlDenoiser:
    """Holds a zero-filled workspace for B x H x W complex images."""

    kind = _lib.DENOISER_MODL

    def __init__(self, B: int, H: int, W: int, device="cuda"):
        self.B, self.H, self.W = B, H, W
        self._lib = _lib.lib()
        nb = self._lib.denoiser_workspace_bytes(self.kind, B, H, W)
        if nb == 0:
            raise ValueError("unsupported denoiser shape")
        self.ws = torch.zeros(int(nb), dtype=torch.uint8, device=device)
        self.nparams = self._lib.denoiser_param_count(self.kind)

    def _chk(self, t, name, dtype, shape):
        if t.dtype != dtype or tuple(t.shape) != tuple(shape) or not t.is_contiguous() or t.device.type != "cuda":
            raise ValueError(f"{name} must be a contiguous CUDA {dtype} tensor of shape {tuple(shape)}")

    def forward(self, weights: torch.Tensor, x: torch.Tensor, out: torch.Tensor | None = None):
        self._chk(weights, "weights", torch.float32, (self.nparams,))
        self._chk(x, "x", torch.complex64, (self.B, self.H, self.W))
        o = out if out is not None else torch.empty_like(x)
        _lib.check("denoiser_forward", self._lib.denoiser_forward(
            self.kind, _p(weights), _p(x), _p(o), _p(self.ws), self.ws.numel(),
            self.B, self.H, self.W, _stream()))
        return o

    def backward(self, weights, x, grad_out, grad_weights, recompute=True, grad_x=None):
        """grad_x for x; adds dL/dW into grad_weights (float32, same layout as weights)."""
        self._chk(weights, "weights", torch.float32, (self.nparams,))
        self._chk(grad_weights, "grad_weights", torch.float32, (self.nparams,))
        self._chk(x, "x", torch.complex64, (self.B, self.H, self.W))
        self._chk(grad_out, "grad_out", torch.complex64, (self.B, self.H, self.W))
        gx = grad_x if grad_x is not None else torch.empty_like(x)
        _lib.check("denoiser_backward", self._lib.denoiser_backward(
            self.kind, _p(weights), _p(x), _p(grad_out), _p(gx), _p(grad_weights), _p(self.ws),
            self.ws.numel(), self.B, self.H, self.W, 1 if recompute else 0, _stream()))
        return gx

    def activations(self):
        """Views of the four BF16 [B, H, W, 64] activations and two gradient buffers in the workspace."""
        a = (C.c_size_t * 4)()
        g = (C.c_size_t * 2)()
        _lib.check("denoiser_workspace_offsets", self._lib.denoiser_workspace_offsets(
            self.kind, self.B, self.H, self.W, a, g))
        n = self.B * self.H * self.W * 64 * 2

        def view(off):
            return self.ws[off:off + n].view(torch.bfloat16).view(self.B, self.H, self.W, 64)
        return [view(a[i]) for i in range(4)], [view(g[i]) for i in range(2)]

    def status(self) -> int:
        v = C.c_int()
        _lib.check("denoiser_get_status", self._lib.denoiser_get_status(
            _p(self.ws), self.B, self.H, self.W, _stream(), C.byref(v)))
        return v.value
