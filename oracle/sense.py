"""SENSE operator A = P F C, adjoint and normal operator (oracle; test infrastructure only).

Eq. 4 ("inverse_problem", Sec. 2.3): A = P F C multiplies the image by the coil
sensitivity maps (C), Fourier transforms each coil image (F) and projects onto
the sampling pattern (P).  The MoDL update (Eq. 6) applies (A^H A + lambda I)
and its inverse; the VarNet update (Eq. 5) applies A^H A x - A^H y.

Layouts: image x [B, H, W]; maps S [B, C, H, W]; mask M either [H, W] or a
line mask [W] (constant along H, i.e. phase-encode lines along the last axis);
k-space y [B, C, H, W] on the full Cartesian grid (zero where M = 0).
P is the 0/1 mask multiply, so P^H P = P.

Soft-SENSE (several sets of maps, Sec. 2.3.3 "Extensions to the SENSE model"):
the image has one component per map set, x [B, NS, H, W], maps [B, NS, C, H, W];
coil image c is sum_s S_{s,c} x_s, so A x = {M F sum_s S_{s,c} x_s}_c and
(A^H y)_s = sum_c conj(S_{s,c}) F^{-1}(M y_c).  NS = 1 is plain SENSE.
"""
from __future__ import annotations

import numpy as np

from .fft import fftc, ifftc


def mask2d(mask: np.ndarray, H: int, W: int) -> np.ndarray:
    m = np.asarray(mask, dtype=np.float64)
    if m.ndim == 1:
        if m.shape[0] != W:
            raise ValueError("line mask must have W entries")
        return np.broadcast_to(m[None, :], (H, W))
    if m.shape != (H, W):
        raise ValueError("mask must be [H, W] or [W]")
    return m


def _lam(lam, B):
    lam = np.asarray(lam, dtype=np.float64).reshape(-1)
    if lam.size == 1:
        return np.full(B, lam[0])
    if lam.size != B:
        raise ValueError("lambda must have 1 or B entries")
    return lam


def forward(x: np.ndarray, maps: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """y = P F C x  (Eq. 4): y_c = M * F(S_c * x)."""
    x = np.asarray(x, dtype=np.complex128)
    S = np.asarray(maps, dtype=np.complex128)
    M = mask2d(mask, x.shape[-2], x.shape[-1])
    return M * fftc(S * x[:, None])


def adjoint(y: np.ndarray, maps: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """x = A^H y = C^H F^H P^H y = sum_c conj(S_c) * F^{-1}(M * y_c)."""
    y = np.asarray(y, dtype=np.complex128)
    S = np.asarray(maps, dtype=np.complex128)
    M = mask2d(mask, y.shape[-2], y.shape[-1])
    return np.sum(np.conj(S) * ifftc(M * y), axis=1)


def normal(x: np.ndarray, maps: np.ndarray, mask: np.ndarray, lam=0.0) -> np.ndarray:
    """(A^H A + lambda I) x, the operator S_lambda of the MoDL update (Eq. 6)."""
    x = np.asarray(x, dtype=np.complex128)
    out = adjoint(forward(x, maps, mask), maps, mask)
    return out + _lam(lam, x.shape[0])[:, None, None] * x


def dot(a: np.ndarray, b: np.ndarray) -> np.ndarray:
    """Per-slice inner product <a, b> = sum conj(a) * b over all but the first axis."""
    a = np.asarray(a, dtype=np.complex128)
    b = np.asarray(b, dtype=np.complex128)
    return np.sum(np.conj(a) * b, axis=tuple(range(1, a.ndim)))


# ------------------------------------------------------------ soft-SENSE
def forward_sets(x: np.ndarray, maps: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """y_c = M * F(sum_s S_{s,c} * x_s)  (x [B, NS, H, W], maps [B, NS, C, H, W])."""
    x = np.asarray(x, dtype=np.complex128)
    S = np.asarray(maps, dtype=np.complex128)
    M = mask2d(mask, x.shape[-2], x.shape[-1])
    return M * fftc(np.sum(S * x[:, :, None], axis=1))


def adjoint_sets(y: np.ndarray, maps: np.ndarray, mask: np.ndarray) -> np.ndarray:
    """(A^H y)_s = sum_c conj(S_{s,c}) * F^{-1}(M * y_c)  -> [B, NS, H, W]."""
    y = np.asarray(y, dtype=np.complex128)
    S = np.asarray(maps, dtype=np.complex128)
    M = mask2d(mask, y.shape[-2], y.shape[-1])
    return np.sum(np.conj(S) * ifftc(M * y)[:, None], axis=2)


def normal_sets(x: np.ndarray, maps: np.ndarray, mask: np.ndarray, lam=0.0) -> np.ndarray:
    """(A^H A + lambda I) x for the soft-SENSE operator."""
    x = np.asarray(x, dtype=np.complex128)
    out = adjoint_sets(forward_sets(x, maps, mask), maps, mask)
    return out + _lam(lam, x.shape[0])[:, None, None, None] * x
