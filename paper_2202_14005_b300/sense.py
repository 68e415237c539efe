"""Torch-facing wrappers of the libsense C ABI (argument marshalling only).

Every computation runs in the library's CUDA kernels; torch provides device
memory (tensors, the workspace) and the current stream.  Names follow the C
ABI and the paper's notation (A = P F C, Eq. 4; S_lambda = A^H A + lambda I,
Eq. 6).
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib


def _ptr(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def _stream():
    return C.c_void_p(torch.cuda.current_stream().cuda_stream)


def _req(t: torch.Tensor, name: str, dtype, shape):
    if t.device.type != "cuda":
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != dtype:
        raise ValueError(f"{name} must be {dtype}, got {t.dtype}")
    if tuple(t.shape) != tuple(shape):
        raise ValueError(f"{name} must have shape {tuple(shape)}, got {tuple(t.shape)}")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")


class SensePlan:
    """A plan for B slices, C coils, H x W images with fixed maps and mask.

    maps: complex64 [B, C, H, W], or [B, S, C, H, W] for S sets of maps
    (soft-SENSE, Sec. 2.3.3: images are then [B, S, H, W]);
    mask: float32 [W] (line mask) or [H, W].
    The plan keeps references to both tensors and owns a torch workspace.
    """

    def __init__(self, maps: torch.Tensor, mask: torch.Tensor):
        if maps.dim() == 5:
            B, NS, Cc, H, W = maps.shape
        else:
            B, Cc, H, W = maps.shape
            NS = 0
        _req(maps, "maps", torch.complex64, tuple(maps.shape))
        lines = 1 if mask.dim() == 1 else 0
        _req(mask, "mask", torch.float32, (W,) if lines else (H, W))
        self.B, self.C, self.H, self.W, self.S = B, Cc, H, W, NS
        self.maps, self.mask, self.lines = maps, mask, lines
        self._lib = _lib.lib()
        h = C.c_void_p()
        _lib.check("sense_plan_create", self._lib.sense_plan_create_sets(
            C.byref(h), B, max(NS, 1), Cc, H, W, _ptr(maps), _ptr(mask), lines, _stream()))
        self._h = h
        nb = C.c_size_t()
        _lib.check("sense_plan_workspace_bytes", self._lib.sense_plan_workspace_bytes(h, C.byref(nb)))
        self.workspace = torch.empty(int(nb.value), dtype=torch.uint8, device=maps.device)
        _lib.check("sense_plan_set_workspace",
                   self._lib.sense_plan_set_workspace(h, _ptr(self.workspace), nb.value))

    @classmethod
    def toeplitz(cls, maps: torch.Tensor, psf: torch.Tensor) -> "SensePlan":
        """Non-Cartesian plan (Sec. 2.3.3): A^H A applied as the convolution with the PSF on the
        2H x 2W grid (psf: complex64 [2H, 2W], e.g. from toeplitz_psf).  Normal operator and CG only."""
        B, Cc, H, W = maps.shape
        _req(maps, "maps", torch.complex64, (B, Cc, H, W))
        _req(psf, "psf", torch.complex64, (2 * H, 2 * W))
        self = cls.__new__(cls)
        self.B, self.C, self.H, self.W, self.S = B, Cc, H, W, 0
        self.maps, self.mask, self.lines, self.psf = maps, None, 0, psf
        self._lib = _lib.lib()
        h = C.c_void_p()
        _lib.check("sense_plan_create_toeplitz", self._lib.sense_plan_create_toeplitz(
            C.byref(h), B, Cc, H, W, _ptr(maps), _ptr(psf), _stream()))
        self._h = h
        nb = C.c_size_t()
        _lib.check("sense_plan_workspace_bytes", self._lib.sense_plan_workspace_bytes(h, C.byref(nb)))
        self.workspace = torch.empty(int(nb.value), dtype=torch.uint8, device=maps.device)
        _lib.check("sense_plan_set_workspace",
                   self._lib.sense_plan_set_workspace(h, _ptr(self.workspace), nb.value))
        return self

    # -- helpers
    def _sync_stream(self):
        _lib.check("sense_plan_set_stream", self._lib.sense_plan_set_stream(self._h, _stream()))

    def close(self):
        if getattr(self, "_h", None) is not None and self._h.value:
            self._lib.sense_plan_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def img_shape(self):
        return (self.B, self.S, self.H, self.W) if self.S else (self.B, self.H, self.W)

    # -- operators
    def forward(self, x: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """y = P F C x (Eq. 4)."""
        _req(x, "x", torch.complex64, self.img_shape())
        y = out if out is not None else torch.empty((self.B, self.C, self.H, self.W),
                                                    dtype=torch.complex64, device=x.device)
        self._sync_stream()
        _lib.check("sense_forward", self._lib.sense_forward(self._h, _ptr(x), _ptr(y)))
        return y

    def adjoint(self, y: torch.Tensor, out: torch.Tensor | None = None) -> torch.Tensor:
        """x = A^H y."""
        _req(y, "y", torch.complex64, (self.B, self.C, self.H, self.W))
        x = out if out is not None else torch.empty(self.img_shape(), dtype=torch.complex64,
                                                    device=y.device)
        self._sync_stream()
        _lib.check("sense_adjoint", self._lib.sense_adjoint(self._h, _ptr(y), _ptr(x)))
        return x

    def normal(self, x: torch.Tensor, lam: float = 0.0, out: torch.Tensor | None = None):
        """(A^H A + lambda I) x."""
        _req(x, "x", torch.complex64, self.img_shape())
        o = out if out is not None else torch.empty_like(x)
        self._sync_stream()
        _lib.check("sense_normal", self._lib.sense_normal(self._h, _ptr(x), _ptr(o), float(lam)))
        return o

    def cg_solve(self, rhs, lam: torch.Tensor, iters: int, x0=None, out=None, rr_hist=None):
        """x = S_lambda^{-1} rhs by `iters` CG iterations (lam: float64 [1] or [B] on device)."""
        _req(rhs, "rhs", torch.complex64, self.img_shape())
        if x0 is not None:
            _req(x0, "x0", torch.complex64, self.img_shape())
        if lam.dtype != torch.float64 or lam.device.type != "cuda" or lam.numel() not in (1, self.B):
            raise ValueError("lam must be a CUDA float64 tensor with 1 or B entries")
        lam = lam.contiguous()
        x = out if out is not None else torch.empty_like(rhs)
        if rr_hist is not None:
            _req(rr_hist, "rr_hist", torch.float64, (iters + 1, self.B))
        self._sync_stream()
        _lib.check("cg_dc_solve", self._lib.cg_dc_solve(
            self._h, _ptr(rhs), _ptr(x0), _ptr(x), _ptr(lam), lam.numel(), int(iters),
            _ptr(rr_hist)))
        return x

    def cg_solve_backward(self, grad_x, x, z, lam: torch.Tensor, iters: int,
                          grad_rhs=None, grad_lam=None):
        """(v = S^{-1} grad_x, Re<v, z - x>) for the block x = S^{-1}(b + lambda z)."""
        _req(grad_x, "grad_x", torch.complex64, self.img_shape())
        _req(x, "x", torch.complex64, self.img_shape())
        if z is not None:
            _req(z, "z", torch.complex64, self.img_shape())
        lam = lam.contiguous()
        v = grad_rhs if grad_rhs is not None else torch.empty_like(grad_x)
        gl = grad_lam if grad_lam is not None else torch.empty(lam.numel(), dtype=torch.float64,
                                                               device=grad_x.device)
        self._sync_stream()
        _lib.check("cg_dc_solve_backward", self._lib.cg_dc_solve_backward(
            self._h, _ptr(grad_x), _ptr(x), _ptr(z), _ptr(lam), lam.numel(), int(iters),
            _ptr(v), _ptr(gl)))
        return v, gl

    def normalize_max(self, x: torch.Tensor, other: torch.Tensor | None = None, scale: torch.Tensor | None = None):
        """x_b /= max |x_b| per slice (in place), other_b likewise (Sec. 2.3.1 data scaling)."""
        _req(x, "x", torch.complex64, self.img_shape())
        if other is not None:
            _req(other, "other", torch.complex64, self.img_shape())
        self._sync_stream()
        _lib.check("sense_normalize_max", self._lib.sense_normalize_max(self._h, _ptr(x), _ptr(other), _ptr(scale)))

    def status(self) -> int:
        v = C.c_int()
        _lib.check("sense_get_status", self._lib.sense_get_status(self._h, C.byref(v)))
        return v.value


def toeplitz_psf(traj: torch.Tensor, H: int, W: int) -> torch.Tensor:
    """PSF of a non-Cartesian trajectory (float32 [M, 2] = (ky, kx) in grid units, on the GPU)
    on the 2H x 2W embedding grid, complex64 [2H, 2W] (Sec. 2.3.3)."""
    if traj.device.type != "cuda" or traj.dtype != torch.float32 or traj.dim() != 2 or traj.shape[1] != 2:
        raise ValueError("traj must be a CUDA float32 [M, 2] tensor")
    traj = traj.contiguous()
    psf = torch.empty((2 * H, 2 * W), dtype=torch.complex64, device=traj.device)
    _lib.check("sense_toeplitz_psf", _lib.lib().sense_toeplitz_psf(_ptr(traj), traj.shape[0], H, W, _ptr(psf),
                                                                  _stream()))
    return psf


def _nudft_args(traj, maps):
    if traj.device.type != "cuda" or traj.dtype != torch.float32 or traj.dim() != 2 or traj.shape[1] != 2:
        raise ValueError("traj must be a CUDA float32 [M, 2] tensor")
    _req(maps, "maps", torch.complex64, tuple(maps.shape))
    if maps.dim() != 4:
        raise ValueError("maps must be complex64 [B, C, H, W]")
    return traj.contiguous()


def nudft_forward(traj: torch.Tensor, maps: torch.Tensor, x: torch.Tensor) -> torch.Tensor:
    """Non-Cartesian samples y [B, C, M] of images x [B, H, W] (direct non-uniform DFT, Sec. 2.3.3)."""
    traj = _nudft_args(traj, maps)
    B, Cc, H, W = maps.shape
    _req(x, "x", torch.complex64, (B, H, W))
    y = torch.empty((B, Cc, traj.shape[0]), dtype=torch.complex64, device=x.device)
    _lib.check("sense_nudft_forward", _lib.lib().sense_nudft_forward(
        _ptr(traj), traj.shape[0], B, Cc, H, W, _ptr(maps), _ptr(x), _ptr(y), _stream()))
    return y


def nudft_adjoint(traj: torch.Tensor, maps: torch.Tensor, y: torch.Tensor) -> torch.Tensor:
    """A^H y [B, H, W] of non-Cartesian samples y [B, C, M] (direct non-uniform DFT, Sec. 2.3.3)."""
    traj = _nudft_args(traj, maps)
    B, Cc, H, W = maps.shape
    _req(y, "y", torch.complex64, (B, Cc, traj.shape[0]))
    x = torch.empty((B, H, W), dtype=torch.complex64, device=y.device)
    _lib.check("sense_nudft_adjoint", _lib.lib().sense_nudft_adjoint(
        _ptr(traj), traj.shape[0], B, Cc, H, W, _ptr(maps), _ptr(y), _ptr(x), _stream()))
    return x
