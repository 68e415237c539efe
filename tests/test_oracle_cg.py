"""Pins for the oracle's CG solve and its reverse-mode derivative (CPU only)."""
import numpy as np
import pytest

from oracle import cg as ocg
from oracle import sense as osense
import synth


def _problem(H=8, W=8, C=3, B=2, seed=7):
    rng = np.random.default_rng(seed)
    maps = np.stack([synth.coil_maps(C, H, W, rng) for _ in range(B)])
    mask = synth.line_mask(W, 3, 2, "uniform", rng)
    return maps, mask


def test_cg_matches_dense_direct_solve():
    maps, mask = _problem(B=2)
    B, C, H, W = maps.shape
    lam = 0.05
    b = synth.randn_complex((B, H, W), 1)
    x, rr = ocg.cg_solve(maps, mask, lam, b, None, 64)
    for s in range(B):
        n = H * W
        M = np.zeros((n, n), dtype=np.complex128)
        for j in range(n):
            e = np.zeros((1, H, W), dtype=np.complex128)
            e.flat[j] = 1
            M[:, j] = osense.normal(e, maps[s:s + 1], mask, lam).reshape(-1)
        ref = np.linalg.solve(M, b[s].reshape(-1)).reshape(H, W)
        assert np.linalg.norm(x[s] - ref) <= 1e-10 * np.linalg.norm(ref)
    assert rr.shape == (65, B)


def test_cg_full_mask_one_iteration():
    maps, _ = _problem(B=1)
    B, C, H, W = maps.shape
    lam = 0.2
    b = synth.randn_complex((B, H, W), 2)
    x, rr = ocg.cg_solve(maps, np.ones(W, np.float32), lam, b, None, 1)
    np.testing.assert_allclose(x, b / (1 + lam), atol=1e-13)
    assert rr[1, 0] < 1e-25 * rr[0, 0]
    # further iterations on a converged slice are frozen (no breakdown)
    x3, _ = ocg.cg_solve(maps, np.ones(W, np.float32), lam, b, None, 3)
    np.testing.assert_allclose(x3, b / (1 + lam), atol=1e-13)


def test_cg_x0_independent_at_convergence_and_per_slice_lambda():
    maps, mask = _problem(B=2)
    B, C, H, W = maps.shape
    b = synth.randn_complex((B, H, W), 3)
    lam = np.array([0.05, 0.3])
    xa, _ = ocg.cg_solve(maps, mask, lam, b, None, 80)
    xb, _ = ocg.cg_solve(maps, mask, lam, b, synth.randn_complex((B, H, W), 4), 80)
    np.testing.assert_allclose(xa, xb, atol=1e-10)
    r = osense.normal(xa, maps, mask, lam) - b
    assert np.linalg.norm(r) < 1e-10 * np.linalg.norm(b)


def test_cg_breakdown_detected():
    maps, mask = _problem(B=1)
    b = synth.randn_complex((1, 8, 8), 5)
    with pytest.raises(ocg.CGBreakdown):
        ocg.cg_solve(maps, mask, -2.0, b, None, 3)


def test_cg_backward_matches_finite_differences():
    """Implicit derivative of x = S^{-1}(b + lambda z) vs central differences
    of L = sum |x - t|^2 with converged CG (Sec. 2.3.2 derivative identities)."""
    maps, mask = _problem(B=2, H=8, W=8)
    B, C, H, W = maps.shape
    it = 120
    b = synth.randn_complex((B, H, W), 6)
    z = synth.randn_complex((B, H, W), 7)
    t = synth.randn_complex((B, H, W), 8)
    lam = 0.07

    def loss(bb, zz, ll):
        x, _ = ocg.cg_solve(maps, mask, ll, bb + ll * zz, None, it)
        return float(np.sum(np.abs(x - t) ** 2)), x

    L0, x = loss(b, z, lam)
    g = 2 * (x - t)
    v, glam = ocg.cg_solve_backward(maps, mask, lam, g, x, z, it)
    eps = 1e-6
    # lambda
    fd = (loss(b, z, lam + eps)[0] - loss(b, z, lam - eps)[0]) / (2 * eps)
    assert abs(fd - glam.sum()) <= 1e-6 * abs(fd)
    # rhs b: real and imaginary parts of a few entries (grad = v)
    for idx in [(0, 1, 2), (1, 5, 3), (0, 7, 7)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            bp, bm = b.copy(), b.copy()
            bp[idx] += unit * eps
            bm[idx] -= unit * eps
            fd = (loss(bp, z, lam)[0] - loss(bm, z, lam)[0]) / (2 * eps)
            assert abs(fd - part(v[idx])) <= 1e-6 * max(1.0, abs(fd))
        # z enters as lambda * z: grad_z = lambda v
        zp, zm = z.copy(), z.copy()
        zp[idx] += eps
        zm[idx] -= eps
        fd = (loss(b, zp, lam)[0] - loss(b, zm, lam)[0]) / (2 * eps)
        assert abs(fd - lam * np.real(v[idx])) <= 1e-6 * max(1.0, abs(fd))


def test_truncated_cg_gradient_differs_from_implicit():
    """At 10 iterations the implicit formula is not the derivative of the
    truncated solver (why the FD gate runs on converged CG)."""
    maps, mask = _problem(B=1, H=8, W=8)
    b = synth.randn_complex((1, 8, 8), 9)
    lam = 0.02
    x10, _ = ocg.cg_solve(maps, mask, lam, b, None, 3)
    xinf, _ = ocg.cg_solve(maps, mask, lam, b, None, 200)
    assert np.linalg.norm(x10 - xinf) > 1e-4 * np.linalg.norm(xinf)
