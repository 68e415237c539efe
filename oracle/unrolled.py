"""MoDL and VarNet unrolled blocks, forward and reverse mode (oracle).

Test infrastructure only.

MoDL (Eq. 6 "update_modl", Sec. 2.3.2): x^0 = A^H y and
    x^{t+1} = (A^H A + lambda I)^{-1} (A^H y + lambda D_W(x^t)),  t = 0..T-1,
with one shared denoiser D_W and a learnable real lambda.

VarNet (Eq. 5 "update_vn", Sec. 2.3.1): x^0 = A^H y and
    x^{t+1} = x^t - sum_i (K_i^t)^T Phi_i^t'(K_i^t x^t) - lambda^t (A^H A x^t - A^H y).

Loss: L = mean over all image elements of |x_hat - x_gt|^2 (the paper trains
with an MSE loss; mean rather than sum is the reading taken).  Gradients follow
Sec. 2.2.2: for a real loss the complex gradient holds dL/d(re) + i dL/d(im).

Reverse mode recomputes each block's forward activations from the stored block
input (the checkpointing idea of Sec. 2.2.4), which is what the GPU path does.
"""
from __future__ import annotations

import numpy as np

from . import cg as _cg
from . import nn as _nn
from .sense import normal, dot


# ------------------------------------------------------------------- loss
def mse_loss(x, gt):
    d = np.asarray(x, dtype=np.complex128) - np.asarray(gt, dtype=np.complex128)
    return float(np.mean(np.abs(d) ** 2))


def mse_loss_grad(x, gt):
    d = np.asarray(x, dtype=np.complex128) - np.asarray(gt, dtype=np.complex128)
    return 2.0 * d / d.size


# ------------------------------------------------------------------- MoDL
def modl_block(x_t, AHy, maps, mask, ws, bs, lam, iters, act_round=None):
    """One MoDL block; returns (x_{t+1}, z = D_W(x_t))."""
    z, _ = _nn.modl_cnn_forward(x_t, ws, bs, act_round)
    rhs = np.asarray(AHy, dtype=np.complex128) + lam * z
    x, _ = _cg.cg_solve(maps, mask, lam, rhs, None, iters)
    return x, z


def modl_forward(AHy, maps, mask, ws, bs, lam, T, iters, act_round=None):
    """Returns (x^T, [x^0 .. x^T])."""
    xs = [np.asarray(AHy, dtype=np.complex128)]
    for _ in range(T):
        x, _ = modl_block(xs[-1], AHy, maps, mask, ws, bs, lam, iters, act_round)
        xs.append(x)
    return xs[-1], xs


def modl_block_backward(g_next, x_t, x_next, AHy, maps, mask, ws, bs, lam, iters, act_round=None,
                        grad_round=None):
    """Reverse mode of one MoDL block.

    Returns (g_t, grad_ws, grad_bs, grad_lambda).  The denoiser activations
    are recomputed from x_t.
    """
    z, cache = _nn.modl_cnn_forward(x_t, ws, bs, act_round)
    v, glam_b = _cg.cg_solve_backward(maps, mask, lam, g_next, x_next, z, iters)
    g_z = lam * v
    g_t, gws, gbs = _nn.modl_cnn_backward(x_t, ws, bs, g_z, cache, grad_round=grad_round)
    return g_t, gws, gbs, float(np.sum(glam_b))


def modl_train_grads(AHy, maps, mask, gt, ws, bs, lam, T, iters, act_round=None, grad_round=None):
    """Loss and gradients of one MoDL training step (x^0 = A^H y is constant)."""
    xT, xs = modl_forward(AHy, maps, mask, ws, bs, lam, T, iters, act_round)
    loss = mse_loss(xT, gt)
    g = mse_loss_grad(xT, gt)
    gws = [np.zeros_like(w) for w in ws]
    gbs = [np.zeros_like(b) for b in bs]
    glam = 0.0
    for t in range(T - 1, -1, -1):
        g, dws, dbs, dl = modl_block_backward(g, xs[t], xs[t + 1], AHy, maps, mask,
                                              ws, bs, lam, iters, act_round, grad_round)
        for i in range(len(ws)):
            gws[i] += dws[i]
            gbs[i] += dbs[i]
        glam += dl
    return loss, gws, gbs, glam, xT


# ----------------------------------------------------------------- VarNet
def varnet_stage(x_t, AHy, maps, mask, filt, wts, lam_t, rnd=None):
    """One VarNet gradient stage (Eq. 5).  rnd: optional rounding of the
    convolution operands (see nn.varnet_regulariser)."""
    reg, _ = _nn.varnet_regulariser(x_t, filt, wts, rnd)
    dc = normal(x_t, maps, mask, 0.0) - AHy
    return np.asarray(x_t, dtype=np.complex128) - reg - lam_t * dc


def varnet_forward(AHy, maps, mask, filt, wts, lam, rnd=None):
    xs = [np.asarray(AHy, dtype=np.complex128)]
    for t in range(len(lam)):
        xs.append(varnet_stage(xs[-1], AHy, maps, mask, filt[t], wts[t], lam[t], rnd))
    return xs[-1], xs


def varnet_stage_backward(g_next, x_t, AHy, maps, mask, filt, wts, lam_t, rnd=None):
    """Reverse mode of one stage: returns (g_t, grad_filt complex, grad_wts, grad_lam).

    With u = K x (real), the stage is x - K^T Phi'(u) - lam (N x - b), N = A^H A.
    rnd: optional rounding of the operands an implementation stores in reduced
    precision (the filters, Phi'(z), Phi''(z) K g, and x and g where they enter
    the filter gradient); K x and K g themselves are exact.  Identity by default.
    """
    rnd = rnd or _nn._ident
    wr = rnd(_nn.varnet_filters_real(filt))
    xr = _nn.c2r(x_t)
    gr = _nn.c2r(g_next)
    z = _nn.conv2d(xr, wr)
    phi = rnd(_nn.rbf(z, wts))
    dphi = _nn.rbf_grad_z(z, wts)
    Kg = _nn.conv2d(gr, wr)                       # K g  (real, [B, Nk, H, W])
    v = rnd(dphi * Kg)
    # d/dx of -K^T Phi'(K x): -K^T diag(Phi''(Kx)) K  (symmetric)
    reg_back = _nn.conv2d_transpose(v, wr)
    Ng = normal(g_next, maps, mask, 0.0)
    g_t = np.asarray(g_next, dtype=np.complex128) - _nn.r2c(reg_back) - lam_t * Ng
    # RBF weights: -sum_pix (K g)_i * phi_j(z_i)
    basis = _nn.rbf_basis(z)
    g_wts = -np.einsum("bkhw,bkhwj->kj", Kg, basis, optimize=True)
    # filters, two paths: through K^T (input g, output-grad phi) and through K
    _, gw1, _ = _nn.conv2d_backward(rnd(gr), wr, phi)     # <K g, phi>
    _, gw2, _ = _nn.conv2d_backward(rnd(xr), wr, v)       # <K x, dphi*Kg>
    gwr = -(gw1 + gw2)                                    # [Nk, 2, k, k]
    g_filt = gwr[:, 0] - 1j * gwr[:, 1]                   # w0 = Re k, w1 = -Im k
    dc = normal(x_t, maps, mask, 0.0) - AHy
    g_lam = -float(np.sum(np.real(dot(g_next, dc))))
    return g_t, g_filt, g_wts, g_lam


def varnet_train_grads(AHy, maps, mask, gt, filt, wts, lam, rnd=None):
    xT, xs = varnet_forward(AHy, maps, mask, filt, wts, lam, rnd)
    loss = mse_loss(xT, gt)
    g = mse_loss_grad(xT, gt)
    T = len(lam)
    g_filt = np.zeros_like(np.asarray(filt, dtype=np.complex128))
    g_wts = np.zeros_like(np.asarray(wts, dtype=np.float64))
    g_lam = np.zeros(T)
    for t in range(T - 1, -1, -1):
        g, gf, gw, gl = varnet_stage_backward(g, xs[t], AHy, maps, mask, filt[t], wts[t], lam[t], rnd)
        g_filt[t], g_wts[t], g_lam[t] = gf, gw, gl
    return loss, g_filt, g_wts, g_lam, xT
