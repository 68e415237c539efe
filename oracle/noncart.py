"""Non-Cartesian SENSE through the Toeplitz embedding of F^H P^H P F (oracle; test
infrastructure only).

Sec. 2.3.3 ("Extensions to the SENSE model"): for non-Cartesian sampling the
adjoint reconstruction A^H y and the point spread function (PSF) of the sampling
pattern are precomputed, and the joint forward-backward transform F^H P^H P F is
applied as a convolution with the PSF (the Toeplitz trick).

Definitions (written out; no gridding):
* trajectory k_m = (ky_m, kx_m), m < M, in grid units (the Cartesian grid is the
  integer lattice, k in [-H/2, H/2) x [-W/2, W/2));
* image coordinates n' = (n_y - H/2, n_x - W/2) for indices 0 <= n < (H, W), so
  that at integer k the transform is the centred unitary DFT of the Cartesian
  operator;
* forward (non-uniform DFT, unitary scaling):
      y_c(m) = (H W)^{-1/2} sum_n S_c(n) x(n) exp(-2 pi i (ky_m n'_y / H + kx_m n'_x / W));
* adjoint: x(n) = (H W)^{-1/2} sum_c conj(S_c(n)) sum_m y_c(m) exp(+2 pi i (...)).
  No density compensation (the paper names none).
* F^H P^H P F is then the convolution out(n) = sum_n' PSF(n - n') u(n') with
      PSF(d) = (H W)^{-1} sum_m exp(+2 pi i (ky_m d_y / H + kx_m d_x / W)),
  |d_y| < H, |d_x| < W; the Toeplitz embedding evaluates it as a circular
  convolution on the 2H x 2W grid (PSF placed at d mod (2H, 2W), zero at
  d_y = H or d_x = W), pad u to 2H x 2W, crop the result.
"""
from __future__ import annotations

import numpy as np

from .sense import _lam


def _phase(traj: np.ndarray, H: int, W: int) -> np.ndarray:
    """E[m, n] = exp(-2 pi i (ky_m n'_y / H + kx_m n'_x / W)), n flattened row-major."""
    t = np.asarray(traj, dtype=np.float64).reshape(-1, 2)
    ny = np.arange(H) - H // 2
    nx = np.arange(W) - W // 2
    ph = (t[:, 0, None, None] * ny[None, :, None] / H + t[:, 1, None, None] * nx[None, None, :] / W)
    return np.exp(-2j * np.pi * ph).reshape(t.shape[0], H * W)


def nudft_forward(x: np.ndarray, maps: np.ndarray, traj: np.ndarray) -> np.ndarray:
    """y [B, C, M] = (H W)^{-1/2} E (S_c x) per coil (direct sum)."""
    x = np.asarray(x, dtype=np.complex128)
    S = np.asarray(maps, dtype=np.complex128)
    B, C, H, W = S.shape
    E = _phase(traj, H, W)
    u = (S * x[:, None]).reshape(B, C, H * W)
    return np.einsum("mn,bcn->bcm", E, u) / np.sqrt(H * W)


def nudft_adjoint(y: np.ndarray, maps: np.ndarray, traj: np.ndarray) -> np.ndarray:
    """x [B, H, W] = (H W)^{-1/2} sum_c conj(S_c) E^H y_c (direct sum)."""
    y = np.asarray(y, dtype=np.complex128)
    S = np.asarray(maps, dtype=np.complex128)
    B, C, H, W = S.shape
    E = _phase(traj, H, W)
    u = np.einsum("mn,bcm->bcn", np.conj(E), y).reshape(B, C, H, W) / np.sqrt(H * W)
    return np.sum(np.conj(S) * u, axis=1)


def toeplitz_psf(traj: np.ndarray, H: int, W: int) -> np.ndarray:
    """The PSF on the 2H x 2W embedding grid (direct sum), complex128 [2H, 2W]."""
    t = np.asarray(traj, dtype=np.float64).reshape(-1, 2)
    dy = np.arange(2 * H)
    dy = np.where(dy < H, dy, dy - 2 * H)   # circular offsets -H .. H-1
    dx = np.arange(2 * W)
    dx = np.where(dx < W, dx, dx - 2 * W)
    ey = np.exp(2j * np.pi * t[:, 0, None] * dy[None, :] / H)   # [M, 2H]
    ex = np.exp(2j * np.pi * t[:, 1, None] * dx[None, :] / W)   # [M, 2W]
    psf = ey.T @ ex / (H * W)                                    # sum over samples
    psf[H, :] = 0.0     # offset -H does not occur between two pixels of an H-row image
    psf[:, W] = 0.0
    return psf


def toeplitz_normal(x: np.ndarray, maps: np.ndarray, psf: np.ndarray, lam=0.0) -> np.ndarray:
    """(A^H A + lambda I) x with F^H P^H P F applied as the PSF convolution:
    per coil pad S_c x to 2H x 2W, circular convolution with psf, crop, conj(S_c) combine."""
    x = np.asarray(x, dtype=np.complex128)
    S = np.asarray(maps, dtype=np.complex128)
    B, C, H, W = S.shape
    u = np.zeros((B, C, 2 * H, 2 * W), dtype=np.complex128)
    u[:, :, :H, :W] = S * x[:, None]
    v = np.fft.ifft2(np.fft.fft2(u) * np.fft.fft2(psf)[None, None])[:, :, :H, :W]
    return np.sum(np.conj(S) * v, axis=1) + _lam(lam, B)[:, None, None] * x
