"""Pins for the oracle's centred DFT and SENSE operators (CPU only).

Each check compares the oracle against something other than itself: a
brute-force double sum, a closed form (pure tone, delta), an identity the
mathematics fixes (Parseval, adjoint, full-mask identity), or an explicitly
built operator matrix.
"""
import cmath
import math

import numpy as np
import pytest

from oracle import fft as offt
from oracle import sense as osense
import synth


def brute_dft2c(x):
    """X[k1,k2] = (H W)^{-1/2} sum_{n1,n2} x[n1,n2] exp(-2 pi i ((k1-c1)(n1-c1)/H + (k2-c2)(n2-c2)/W))."""
    H, W = x.shape
    c1, c2 = H // 2, W // 2
    X = np.zeros((H, W), dtype=np.complex128)
    for k1 in range(H):
        for k2 in range(W):
            s = 0j
            for n1 in range(H):
                for n2 in range(W):
                    ph = ((k1 - c1) * (n1 - c1)) / H + ((k2 - c2) * (n2 - c2)) / W
                    s += x[n1, n2] * cmath.exp(-2j * math.pi * ph)
            X[k1, k2] = s / math.sqrt(H * W)
    return X


@pytest.mark.parametrize("shape", [(4, 6), (8, 8), (6, 10), (5, 7)])
def test_fftc_matches_brute_force_dft(shape):
    x = synth.randn_complex(shape, 11)
    np.testing.assert_allclose(offt.fftc(x), brute_dft2c(x), rtol=0, atol=1e-12)
    # inverse undoes forward, and the forward keeps the norm (unitary)
    np.testing.assert_allclose(offt.ifftc(offt.fftc(x)), x, atol=1e-13)
    assert abs(np.linalg.norm(offt.fftc(x)) - np.linalg.norm(x)) < 1e-12 * np.linalg.norm(x)


@pytest.mark.parametrize("L", [8, 9, 232, 368])
def test_pure_tone_and_delta(L):
    c = L // 2
    n = np.arange(L)
    # delta at the centre index -> constant L^{-1/2}
    d = np.zeros(L, dtype=np.complex128)
    d[c] = 1
    np.testing.assert_allclose(offt.fftc(d, axes=(-1,)), np.full(L, L ** -0.5), atol=1e-13)
    # a positive-frequency tone lands on index c + f with height sqrt(L)
    f = 3
    tone = np.exp(2j * np.pi * f * (n - c) / L)
    X = offt.fftc(tone, axes=(-1,))
    ref = np.zeros(L, dtype=np.complex128)
    ref[c + f] = math.sqrt(L)
    np.testing.assert_allclose(X, ref, atol=1e-11)


def _problem(H=8, W=8, C=3, B=2, seed=5, line=True, R=2.5):
    rng = np.random.default_rng(seed)
    maps = np.stack([synth.coil_maps(C, H, W, rng) for _ in range(B)])
    if line:
        mask = synth.line_mask(W, R, 2, "uniform", rng)
    else:
        mask = (rng.uniform(size=(H, W)) < 0.4).astype(np.float32)
    return maps, mask


@pytest.mark.parametrize("line", [True, False])
def test_adjoint_identity(line):
    maps, mask = _problem(H=6, W=10, C=4, line=line)
    B, C, H, W = maps.shape
    x = synth.randn_complex((B, H, W), 1)
    y = synth.randn_complex((B, C, H, W), 2)
    lhs = np.vdot(osense.forward(x, maps, mask), y)
    rhs = np.vdot(x, osense.adjoint(y, maps, mask))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_full_mask_is_identity():
    maps, _ = _problem(H=8, W=12, C=5)
    B, C, H, W = maps.shape
    x = synth.randn_complex((B, H, W), 3)
    lam = 0.37
    out = osense.normal(x, maps, np.ones(W, dtype=np.float32), lam)
    np.testing.assert_allclose(out, (1 + lam) * x, atol=1e-12)


def test_single_coil_single_line_is_tone_projection():
    H, W, f = 6, 8, 2
    maps = np.ones((1, 1, H, W), dtype=np.complex128)
    mask = np.zeros(W, dtype=np.float32)
    mask[W // 2 + f] = 1.0
    x = synth.randn_complex((1, H, W), 4)
    out = osense.normal(x, maps, mask, 0.0)[0]
    # closed form: each row is projected onto exp(2 pi i f (n - c)/W) / sqrt(W)
    c = W // 2
    e = np.exp(2j * np.pi * f * (np.arange(W) - c) / W) / math.sqrt(W)
    ref = np.stack([e * np.vdot(e, x[0, h]) for h in range(H)])
    np.testing.assert_allclose(out, ref, atol=1e-12)


def _normal_matrix(maps, mask, lam):
    B, C, H, W = maps.shape
    n = H * W
    M = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros((1, H, W), dtype=np.complex128)
        e.flat[j] = 1
        M[:, j] = osense.normal(e, maps[:1], mask, lam).reshape(-1)
    return M


@pytest.mark.parametrize("line", [True, False])
def test_normal_matrix_hermitian_pd_bounds(line):
    maps, mask = _problem(H=8, W=8, C=3, B=1, line=line)
    lam = 0.05
    M = _normal_matrix(maps, mask, lam)
    assert np.abs(M - M.conj().T).max() < 1e-13
    ev = np.linalg.eigvalsh(M)
    assert ev.min() >= lam - 1e-12 and ev.max() <= 1 + lam + 1e-12


def test_line_mask_reduces_to_rowwise_1d():
    """With a mask constant along H, F^H M F acts on each row with the 1-D
    operator F_W^H diag(m) F_W (F_H cancels against its inverse)."""
    maps, mask = _problem(H=6, W=10, C=3, B=1)
    x = synth.randn_complex((1, 6, 10), 9)
    FW = offt.dft_matrix(10)
    K1 = FW.conj().T @ np.diag(mask.astype(np.float64)) @ FW
    S = maps[0]
    ref = np.zeros((6, 10), dtype=np.complex128)
    for c in range(S.shape[0]):
        u = S[c] * x[0]
        ref += np.conj(S[c]) * (u @ K1.T)
    np.testing.assert_allclose(osense.normal(x, maps, mask, 0.0)[0], ref, atol=1e-12)


def test_forward_matches_matrix_form():
    maps, mask = _problem(H=5, W=6, C=2, B=1)
    x = synth.randn_complex((1, 5, 6), 10)
    FH, FW = offt.dft_matrix(5), offt.dft_matrix(6)
    y = osense.forward(x, maps, mask)
    for c in range(2):
        ref = (FH @ (maps[0, c] * x[0]) @ FW.T) * mask[None, :]
        np.testing.assert_allclose(y[0, c], ref, atol=1e-12)


# ------------------------------------------------------------ soft-SENSE (Sec. 2.3.3)
def _sets_problem(H=6, W=10, C=3, B=2, NS=2, seed=21, line=True):
    rng = np.random.default_rng(seed)
    maps = np.stack([np.stack([synth.coil_maps(C, H, W, rng) * (0.6 if s else 1.0) for s in range(NS)])
                     for _ in range(B)])  # [B, NS, C, H, W]
    mask = synth.line_mask(W, 2.5, 2, "uniform", rng) if line else \
        (rng.uniform(size=(H, W)) < 0.4).astype(np.float32)
    return maps, mask


def test_soft_sense_one_set_is_sense():
    maps, mask = _sets_problem(NS=1)
    x = synth.randn_complex((2, 6, 10), 31)
    y = synth.randn_complex((2, 3, 6, 10), 32)
    np.testing.assert_allclose(osense.forward_sets(x[:, None], maps, mask), osense.forward(x, maps[:, 0], mask),
                               atol=1e-14)
    np.testing.assert_allclose(osense.adjoint_sets(y, maps, mask)[:, 0], osense.adjoint(y, maps[:, 0], mask),
                               atol=1e-14)


@pytest.mark.parametrize("line", [True, False])
def test_soft_sense_adjoint_identity(line):
    maps, mask = _sets_problem(line=line)
    x = synth.randn_complex((2, 2, 6, 10), 33)
    y = synth.randn_complex((2, 3, 6, 10), 34)
    lhs = np.vdot(osense.forward_sets(x, maps, mask), y)
    rhs = np.vdot(x, osense.adjoint_sets(y, maps, mask))
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_soft_sense_full_mask_is_pointwise_gram():
    """Full sampling: F^H F = I, so (A^H A x)_s' = sum_s (sum_c conj(S_{s',c}) S_{s,c}) x_s pixel by pixel."""
    maps, _ = _sets_problem(H=8, W=12, C=4)
    x = synth.randn_complex((2, 2, 8, 12), 35)
    lam = 0.2
    G = np.einsum("bpchw,bschw->bpshw", np.conj(maps), maps)
    ref = np.einsum("bpshw,bshw->bphw", G, x) + lam * x
    np.testing.assert_allclose(osense.normal_sets(x, maps, np.ones(12, dtype=np.float32), lam), ref, atol=1e-12)


def test_soft_sense_normal_hermitian_psd_and_cg_matches_solve():
    from oracle import cg as ocg
    maps, mask = _sets_problem(H=4, W=6, C=3, B=1)
    n = 2 * 4 * 6
    lam = 0.05
    M = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros((1, 2, 4, 6), dtype=np.complex128)
        e.flat[j] = 1
        M[:, j] = osense.normal_sets(e, maps, mask, lam).reshape(-1)
    assert np.abs(M - M.conj().T).max() < 1e-13
    assert np.linalg.eigvalsh(M).min() >= lam - 1e-12
    b = synth.randn_complex((1, 2, 4, 6), 36)
    x, _ = ocg.cg_solve_sets(maps, mask, lam, b, None, n)
    np.testing.assert_allclose(x.reshape(-1), np.linalg.solve(M, b.reshape(-1)), atol=1e-9)
