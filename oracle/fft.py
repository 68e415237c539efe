"""Centred unitary discrete Fourier transform (oracle; test infrastructure only).

The paper's SENSE operator A = P F C (Eq. 4, Sec. 2.3 "Applications") applies
"the Fourier transform" F without fixing normalisation or centring.  Reading
taken here: the unitary DFT with the k-space origin at index c = floor(L/2),

    F_L[k, n] = L^{-1/2} exp(-2 pi i (k - c)(n - c) / L),

applied along both image axes.  Unitarity makes A^H A = I for a fully sampled
mask with sum_c |S_c|^2 = 1.  With c = floor(L/2) this equals
fftshift(fft(ifftshift(x), norm="ortho")) for both even and odd L.
"""
from __future__ import annotations

import numpy as np


def dft_matrix(L: int) -> np.ndarray:
    """Explicit centred unitary DFT matrix F_L (the definition above)."""
    c = L // 2
    k = np.arange(L)[:, None] - c
    n = np.arange(L)[None, :] - c
    return np.exp(-2j * np.pi * k * n / L) / np.sqrt(L)


def fftc(x: np.ndarray, axes=(-2, -1)) -> np.ndarray:
    """Centred unitary forward DFT over ``axes`` (library FFT as the step)."""
    x = np.asarray(x, dtype=np.complex128)
    return np.fft.fftshift(
        np.fft.fftn(np.fft.ifftshift(x, axes=axes), axes=axes, norm="ortho"), axes=axes)


def ifftc(x: np.ndarray, axes=(-2, -1)) -> np.ndarray:
    """Inverse of :func:`fftc` (= its adjoint, since F is unitary)."""
    x = np.asarray(x, dtype=np.complex128)
    return np.fft.fftshift(
        np.fft.ifftn(np.fft.ifftshift(x, axes=axes), axes=axes, norm="ortho"), axes=axes)
