"""Direct-sum convolutions and activations of the two learned regularisers (oracle).

Test infrastructure only.

* MoDL (Sec. 2.3.2, Eq. 6): residual denoiser D_W(x) = x + CNN(x), the CNN a
  stack of 3x3 convolutions with ReLU between them; complex images enter as
  two real channels (real, imaginary).  The workload here uses 2->64->64->64->64->2
  channels with biases and no batch normalisation.
* VarNet (Sec. 2.3.1, Eq. 5): regulariser gradient sum_i K_i^T Phi_i'(K_i x)
  with N_k complex 11x11 filters; the imaginary part of K_i x is discarded;
  Phi_i' is a weighted sum of N_w = 31 Gaussian radial basis functions.

Readings where the paper is silent: convolutions are cross-correlations with
zero "same" padding (deep-learning convention); the RBF centres are
mu_j = -1 + 2 j / (N_w - 1) on [-1, 1] and the common width is their spacing,
sigma = 2 / (N_w - 1).

Layouts: activations [B, Ch, H, W] float64; weights [Cout, Cin, k, k].
"""
from __future__ import annotations

import numpy as np


# ----------------------------------------------------------------- convolution
def conv2d(x: np.ndarray, w: np.ndarray, b=None) -> np.ndarray:
    """out[b,o,y,x] = bias[o] + sum_{c,dy,dx} w[o,c,dy,dx] * x[b,c,y+dy-p,x+dx-p] (zero padded)."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    B, Ci, H, W = x.shape
    Co, Ci2, kh, kw = w.shape
    assert Ci == Ci2
    ph, pw = kh // 2, kw // 2
    xp = np.pad(x, ((0, 0), (0, 0), (ph, ph), (pw, pw)))
    out = np.zeros((B, Co, H, W))
    for dy in range(kh):
        for dx in range(kw):
            out += np.einsum("oc,bchw->bohw", w[:, :, dy, dx], xp[:, :, dy:dy + H, dx:dx + W],
                             optimize=True)
    if b is not None:
        out += np.asarray(b, dtype=np.float64)[None, :, None, None]
    return out


def conv2d_backward(x: np.ndarray, w: np.ndarray, gout: np.ndarray):
    """Gradients of conv2d: (grad_x, grad_w, grad_b) for an incoming gradient gout."""
    x = np.asarray(x, dtype=np.float64)
    w = np.asarray(w, dtype=np.float64)
    g = np.asarray(gout, dtype=np.float64)
    B, Ci, H, W = x.shape
    Co, _, kh, kw = w.shape
    ph, pw = kh // 2, kw // 2
    xp = np.pad(x, ((0, 0), (0, 0), (ph, ph), (pw, pw)))
    gxp = np.zeros_like(xp)
    gw = np.zeros_like(w)
    for dy in range(kh):
        for dx in range(kw):
            gxp[:, :, dy:dy + H, dx:dx + W] += np.einsum("oc,bohw->bchw", w[:, :, dy, dx], g,
                                                         optimize=True)
            gw[:, :, dy, dx] = np.einsum("bohw,bchw->oc", g, xp[:, :, dy:dy + H, dx:dx + W],
                                         optimize=True)
    gx = gxp[:, :, ph:ph + H, pw:pw + W]
    gb = g.sum(axis=(0, 2, 3))
    return gx, gw, gb


def conv2d_transpose(u: np.ndarray, w: np.ndarray) -> np.ndarray:
    """Adjoint of the bias-free conv2d with respect to its input: K^T u."""
    B, Co, H, W = u.shape
    gx, _, _ = conv2d_backward(np.zeros((B, w.shape[1], H, W)), w, u)
    return gx


def relu(a):
    return np.maximum(a, 0.0)


def bf16_round(a):
    """Round to the nearest bfloat16 (ties to even), returned as float64.

    Storage precision of activations and gradients in the GPU path; values are
    first rounded to float32, then to 8 significand bits.
    """
    f = np.ascontiguousarray(np.asarray(a, dtype=np.float32))
    u = f.view(np.uint32).astype(np.uint64)
    lsb = (u >> 16) & 1
    r = ((u + 0x7FFF + lsb) >> 16) << 16
    return r.astype(np.uint32).view(np.float32).astype(np.float64).reshape(f.shape)


# ------------------------------------------------------------ complex <-> 2ch
def c2r(x: np.ndarray) -> np.ndarray:
    """Complex [B, H, W] -> real two-channel [B, 2, H, W] (real, imaginary)."""
    x = np.asarray(x, dtype=np.complex128)
    return np.stack([x.real, x.imag], axis=1)


def r2c(a: np.ndarray) -> np.ndarray:
    return a[:, 0] + 1j * a[:, 1]


# ------------------------------------------------------------- MoDL denoiser
def modl_cnn_forward(x: np.ndarray, ws, bs, act_round=None):
    """D_W(x) = x + CNN(x) for complex x [B, H, W]; returns (D(x), cache).

    act_round, if given, is applied to the network input and to every hidden
    activation after its ReLU (used to mirror storage precision in tests).
    """
    rnd = (lambda a: a) if act_round is None else act_round
    a = rnd(c2r(x))
    acts = [a]
    pre = []
    L = len(ws)
    for l in range(L):
        h = conv2d(a, ws[l], bs[l])
        pre.append(h)
        if l < L - 1:
            a = rnd(relu(h))
            acts.append(a)
        else:
            a = h
    out = np.asarray(x, dtype=np.complex128) + r2c(a)
    return out, {"acts": acts, "pre": pre}


def modl_cnn_backward(x: np.ndarray, ws, bs, grad_out: np.ndarray, cache=None, act_round=None,
                      grad_round=None):
    """Reverse mode of D_W: returns (grad_x complex, [grad_w], [grad_b]).

    grad_round, if given, is applied to the gradient with respect to each
    hidden pre-activation (after the ReLU mask), mirroring a storage precision.
    """
    if cache is None:
        _, cache = modl_cnn_forward(x, ws, bs, act_round)
    acts, pre = cache["acts"], cache["pre"]
    L = len(ws)
    g = c2r(grad_out)
    gws, gbs = [None] * L, [None] * L
    for l in range(L - 1, -1, -1):
        if l < L - 1:
            g = g * (pre[l] > 0)
            if grad_round is not None:
                g = grad_round(g)
        gx, gw, gb = conv2d_backward(acts[l], ws[l], g)
        gws[l], gbs[l] = gw, gb
        g = gx
    grad_x = np.asarray(grad_out, dtype=np.complex128) + r2c(g)
    return grad_x, gws, gbs


def modl_param_count(chans=(2, 64, 64, 64, 64, 2), k=3) -> int:
    return sum(ci * co * k * k + co for ci, co in zip(chans[:-1], chans[1:]))


# ------------------------------------------------------- VarNet regulariser
def rbf_centres(Nw: int = 31):
    mu = -1.0 + 2.0 * np.arange(Nw) / (Nw - 1)
    return mu, 2.0 / (Nw - 1)


def rbf(z: np.ndarray, wts: np.ndarray, Nw: int = 31):
    """Phi_i'(z) = sum_j w_ij exp(-(z - mu_j)^2 / (2 sigma^2)) for z [B, Nk, H, W], wts [Nk, Nw]."""
    mu, s = rbf_centres(Nw)
    e = np.exp(-(z[..., None] - mu) ** 2 / (2 * s * s))
    return np.einsum("bkhwj,kj->bkhw", e, wts, optimize=True)


def rbf_grad_z(z, wts, Nw: int = 31):
    """d Phi_i'(z) / dz = sum_j w_ij * (-(z - mu_j) / sigma^2) * exp(...)."""
    mu, s = rbf_centres(Nw)
    d = z[..., None] - mu
    e = np.exp(-d ** 2 / (2 * s * s))
    return np.einsum("bkhwj,kj->bkhw", -d / (s * s) * e, wts, optimize=True)


def rbf_basis(z, Nw: int = 31):
    mu, s = rbf_centres(Nw)
    return np.exp(-(z[..., None] - mu) ** 2 / (2 * s * s))


def varnet_filters_real(filt: np.ndarray) -> np.ndarray:
    """Complex filters k_i [Nk, k, k] as real conv weights [Nk, 2, k, k]:
    Re(k_i * x) = Re(k_i) * x_re - Im(k_i) * x_im (imaginary part discarded, Eq. 5)."""
    filt = np.asarray(filt, dtype=np.complex128)
    return np.stack([filt.real, -filt.imag], axis=1)


def _ident(a):
    return a


def varnet_regulariser(x: np.ndarray, filt: np.ndarray, wts: np.ndarray, rnd=None):
    """sum_i K_i^T Phi_i'(K_i x) as a complex image [B, H, W]; returns (value, z).

    rnd (default: none) models an implementation that stores the filters and
    Phi'(z) rounded; K x itself is taken as exact."""
    rnd = rnd or _ident
    wr = rnd(varnet_filters_real(filt))
    z = conv2d(c2r(x), wr)
    u = rnd(rbf(z, wts))
    return r2c(conv2d_transpose(u, wr)), z


def varnet_param_count(T=10, Nk=24, k=11, Nw=31) -> int:
    return T * (Nk * k * k * 2 + Nk * Nw + 1)
