"""Pins of the non-Cartesian (Toeplitz) oracle, Sec. 2.3.3: the PSF convolution
equals the direct non-uniform DFT pair, on-grid samples reduce to the centred
unitary DFT, and the operator is Hermitian positive semi-definite."""
import numpy as np
import pytest

import synth
from oracle import fft as offt
from oracle import noncart as onc
from oracle import sense as osense


def _case(H=8, W=10, C=3, B=2, spokes=5, samples=12, seed=3):
    rng = np.random.default_rng(seed)
    maps = np.stack([synth.coil_maps(C, H, W, rng) for _ in range(B)])
    traj = synth.radial_trajectory(spokes, samples, min(H, W))
    return maps, traj


def test_toeplitz_equals_direct_nudft_pair():
    maps, traj = _case()
    x = synth.randn_complex((2, 8, 10), 1)
    direct = onc.nudft_adjoint(onc.nudft_forward(x, maps, traj), maps, traj) + 0.2 * x
    psf = onc.toeplitz_psf(traj, 8, 10)
    np.testing.assert_allclose(onc.toeplitz_normal(x, maps, psf, 0.2), direct, atol=1e-11)


def test_nudft_adjoint_identity():
    maps, traj = _case(H=6, W=8, C=2, spokes=4, samples=10)
    x = synth.randn_complex((2, 6, 8), 2)
    y = synth.randn_complex((2, 2, traj.size // 2), 3)
    lhs = np.vdot(onc.nudft_forward(x, maps, traj), y)
    rhs = np.vdot(x, onc.nudft_adjoint(y, maps, traj))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_on_grid_samples_are_the_cartesian_operator():
    """With the full integer grid as trajectory the non-uniform DFT is the centred unitary DFT,
    and the Toeplitz normal operator equals the Cartesian one with a full mask (the identity)."""
    H, W = 6, 8
    ky, kx = np.meshgrid(np.arange(H) - H // 2, np.arange(W) - W // 2, indexing="ij")
    traj = np.stack([ky.ravel(), kx.ravel()], axis=1).astype(np.float64)
    rng = np.random.default_rng(4)
    maps = synth.coil_maps(2, H, W, rng)[None]
    x = synth.randn_complex((1, H, W), 5)
    y = onc.nudft_forward(x, maps, traj).reshape(1, 2, H, W)
    np.testing.assert_allclose(y, osense.forward(x, maps, np.ones(W, dtype=np.float32)), atol=1e-12)
    psf = onc.toeplitz_psf(traj, H, W)
    np.testing.assert_allclose(onc.toeplitz_normal(x, maps, psf, 0.0), x, atol=1e-12)


def test_psf_closed_forms():
    maps, traj = _case()
    H, W = 8, 10
    psf = onc.toeplitz_psf(traj, H, W)
    M = traj.size // 2
    assert abs(psf[0, 0] - M / (H * W)) < 1e-12                 # all phases 1 at d = 0
    d = (3, 4)
    assert abs(psf[d] - np.conj(psf[2 * H - 3, 2 * W - 4])) < 1e-12  # PSF(-d) = conj PSF(d)
    assert np.all(psf[H, :] == 0) and np.all(psf[:, W] == 0)


def test_toeplitz_operator_hermitian_psd():
    maps, traj = _case(H=4, W=6, C=2, B=1)
    psf = onc.toeplitz_psf(traj, 4, 6)
    n = 24
    A = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros((1, 4, 6), dtype=np.complex128)
        e.flat[j] = 1
        A[:, j] = onc.toeplitz_normal(e, maps, psf, 0.0).reshape(-1)
    assert np.abs(A - A.conj().T).max() < 1e-12
    assert np.linalg.eigvalsh(A).min() >= -1e-12
