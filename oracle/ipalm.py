"""iPALM training update of the VarNet parameters with the filter constraints (oracle).

Test infrastructure only.

Sec. 2.3.1 trains the VarNet with iPALM, the inertial proximal alternating linearised
minimisation of Pock and Sabach (SIAM J. Imaging Sci. 2016), and Sec. 2.2 lists iPALM among
the training algorithms of the library.  The paper states neither the constraints nor the
inertial parameters; the readings taken here (all of them also listed with the design notes):

* blocks: per stage t the filters k^t_i, the RBF weights w^t_ij and the step size lambda^t;
  every block is updated from one gradient evaluation per minibatch (the stochastic form;
  the blocks share one forward and reverse pass);
* constraints (the variational-network convention): each complex filter has zero mean over
  its taps and Euclidean norm at most 1; lambda^t >= 0; the RBF weights are free;
* inertia alpha_k = beta_k = (k - 1) / (k + 2) at update k = 1, 2, ...; one step size
  tau per block kind.

Update k (x^0 = x^{-1} = the initial parameters, so z^0 = x^0):
    z^k     = x^k + alpha_k (x^k - x^{k-1})        (inertial point; alpha = beta)
    g       = gradient of the minibatch loss at z^k
    x^{k+1} = P(z^k - tau g)                         (the proximal map of the constraint
                                                      indicator is the projection P)

P on a filter: the constraint set is the intersection of the zero-mean subspace and the unit
ball centred at 0, which lies in that subspace, so P(v) = P_ball(P_mean(v)): subtract the mean,
then scale by min(1, 1 / ||.||).
"""
from __future__ import annotations

import numpy as np


def inertia(k: int) -> float:
    """alpha_k = (k - 1) / (k + 2) for update k >= 1 (so 0 for the first update)."""
    if k < 1:
        raise ValueError("updates are numbered from 1")
    return (k - 1) / (k + 2)


def project_filter(k: np.ndarray) -> np.ndarray:
    """Projection of complex filters [..., kh, kw] onto {zero mean over taps} and {||k|| <= 1}."""
    k = np.asarray(k, dtype=np.complex128)
    k = k - k.mean(axis=(-2, -1), keepdims=True)
    n = np.sqrt(np.sum(np.abs(k) ** 2, axis=(-2, -1), keepdims=True))
    return k * np.minimum(1.0, 1.0 / np.maximum(n, 1e-300))


def project(filt, rbf, lam):
    """P of every block: filters projected, RBF weights free, lambda clamped at 0."""
    return project_filter(filt), np.asarray(rbf, dtype=np.float64), np.maximum(np.asarray(lam, dtype=np.float64), 0.0)


def step(z, grad, tau):
    """x^{k+1} = P(z - tau g) for z and grad given as (filters, rbf, lambda) triples and
    tau = (tau_filters, tau_rbf, tau_lambda)."""
    return project(*(np.asarray(zi) - ti * np.asarray(gi) for zi, gi, ti in zip(z, grad, tau)))


def extrapolate(x, x_prev, alpha):
    """z = x + alpha (x - x_prev), blockwise."""
    return tuple(np.asarray(a) + alpha * (np.asarray(a) - np.asarray(b)) for a, b in zip(x, x_prev))


def run(x0, grad_fn, tau, iters: int):
    """iters iPALM updates from x0 with the gradient oracle grad_fn(z) -> grads; returns the
    final iterate and the list of inertial points z^k at which gradients were taken."""
    x_prev = x0
    x = x0
    zs = []
    for k in range(1, iters + 1):
        z = extrapolate(x, x_prev, inertia(k))
        zs.append(z)
        x_prev, x = x, step(z, grad_fn(z), tau)
    return x, zs
