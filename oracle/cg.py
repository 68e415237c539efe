"""Conjugate gradient for S_lambda = A^H A + lambda I and its derivative (oracle).

Test infrastructure only.

Sec. 2.3.2 (MoDL): the inversion nlop S^{-1}: (y, lambda) -> S_lambda^{-1} y is
applied with the conjugate gradient algorithm, and its derivatives are written
through S itself:

    D_y S^{-1}      : dy      -> S_lambda^{-1} dy
    D_lambda S^{-1} : dlambda -> -S_lambda^{-1} (D_lambda S at x) dlambda,
                      with D_lambda S at x = x  (S_lambda x = A^H A x + lambda x).

Readings where the paper is silent:
* CG runs exactly ``iters`` iterations (no tolerance), independently per slice
  (Hestenes-Stiefel form).  A slice whose residual norm is exactly zero is
  frozen; Re<p, S p> <= 0 on an active slice is a breakdown (error).
* The data-consistency block of MoDL is x = S^{-1}(b + lambda z), with
  b = A^H y and z = D_W(x^t) (Eq. 6).  Its reverse-mode derivative for a real
  loss with incoming gradient g (complex convention of Sec. 2.2.2) is
      v = S^{-1} g            (S Hermitian, so S^{-H} = S^{-1})
      grad_b = v,  grad_z = lambda v,
      grad_lambda = sum_b Re<v_b, z_b - x_b>,
  which is D_y S^{-1} applied to the rhs term lambda z plus D_lambda S^{-1}.
"""
from __future__ import annotations

import numpy as np

from .sense import normal, normal_sets, dot, _lam


class CGBreakdown(RuntimeError):
    pass


def cg(apply_S, b: np.ndarray, x0, iters: int):
    """Run ``iters`` CG iterations on every slice of b [B, ...].

    apply_S(p) must apply the Hermitian positive-definite operator slice-wise.
    Returns (x, rr) with rr [iters + 1, B] the squared residual norms
    ||r_i||^2 (rr[0] for the initial residual).
    """
    b = np.asarray(b, dtype=np.complex128)
    B = b.shape[0]
    x = np.zeros_like(b) if x0 is None else np.array(x0, dtype=np.complex128)
    r = b - apply_S(x) if x0 is not None else b.copy()
    p = r.copy()
    rr = np.real(dot(r, r))
    hist = [rr.copy()]
    shape = (B,) + (1,) * (b.ndim - 1)
    for _ in range(iters):
        active = rr > 0
        q = apply_S(p)
        pq = np.real(dot(p, q))
        if np.any(active & (pq <= 0)):
            raise CGBreakdown("Re<p, S p> <= 0 on an active slice")
        alpha = np.where(active, rr / np.where(active, pq, 1.0), 0.0)
        x = x + alpha.reshape(shape) * p
        r = r - alpha.reshape(shape) * q
        rr_new = np.real(dot(r, r))
        beta = np.where(active, rr_new / np.where(active, rr, 1.0), 0.0)
        p = np.where(active.reshape(shape), r + beta.reshape(shape) * p, p)
        rr = np.where(active, rr_new, rr)
        hist.append(rr.copy())
    return x, np.stack(hist)


def cg_solve(maps, mask, lam, rhs, x0, iters: int):
    """x = (A^H A + lambda I)^{-1} rhs by ``iters`` CG iterations from x0 (None -> 0)."""
    lam_b = _lam(lam, np.asarray(rhs).shape[0])
    return cg(lambda p: normal(p, maps, mask, lam_b), rhs, x0, iters)


def cg_solve_sets(maps, mask, lam, rhs, x0, iters: int):
    """Soft-SENSE data consistency (Sec. 2.3.3): x [B, NS, H, W] = (A^H A + lambda I)^{-1} rhs."""
    lam_b = _lam(lam, np.asarray(rhs).shape[0])
    return cg(lambda p: normal_sets(p, maps, mask, lam_b), rhs, x0, iters)


def cg_solve_backward(maps, mask, lam, grad_x, x, z, iters: int):
    """Reverse mode of the MoDL data-consistency block x = S^{-1}(b + lambda z).

    Returns (v, grad_lambda_per_slice): v = S^{-1} grad_x (= grad wrt the rhs
    b), and Re<v_b, z_b - x_b> per slice (sum them for a shared lambda).
    z may be None, in which case the rhs did not depend on lambda and the
    lambda gradient is -Re<v_b, x_b> (the pure D_lambda S^{-1} term).
    """
    v, _ = cg_solve(maps, mask, lam, grad_x, None, iters)
    x = np.asarray(x, dtype=np.complex128)
    zz = np.zeros_like(x) if z is None else np.asarray(z, dtype=np.complex128)
    return v, np.real(dot(v, zz - x))
