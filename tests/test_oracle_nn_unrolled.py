"""Pins for the oracle's convolutions, RBF, MoDL and VarNet blocks (CPU only)."""
import os

import numpy as np
import pytest

from oracle import nn as onn
from oracle import unrolled as ounr
import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def brute_conv(x, w, b):
    B, Ci, H, W = x.shape
    Co, _, kh, kw = w.shape
    out = np.zeros((B, Co, H, W))
    for bb in range(B):
        for o in range(Co):
            for yy in range(H):
                for xx in range(W):
                    s = b[o]
                    for c in range(Ci):
                        for dy in range(kh):
                            for dx in range(kw):
                                sy, sx = yy + dy - kh // 2, xx + dx - kw // 2
                                if 0 <= sy < H and 0 <= sx < W:
                                    s += w[o, c, dy, dx] * x[bb, c, sy, sx]
                    out[bb, o, yy, xx] = s
    return out


@pytest.mark.parametrize("k", [3, 5])
def test_conv2d_matches_brute_force(k):
    rng = np.random.default_rng(1)
    x = rng.standard_normal((2, 2, 5, 6))
    w = rng.standard_normal((3, 2, k, k))
    b = rng.standard_normal(3)
    np.testing.assert_allclose(onn.conv2d(x, w, b), brute_conv(x, w, b), atol=1e-12)


def test_conv2d_backward_finite_differences_and_adjoint():
    rng = np.random.default_rng(2)
    x = rng.standard_normal((1, 2, 5, 4))
    w = rng.standard_normal((3, 2, 3, 3))
    b = rng.standard_normal(3)
    g = rng.standard_normal((1, 3, 5, 4))
    gx, gw, gb = onn.conv2d_backward(x, w, g)
    f = lambda xx, ww, bb: float(np.sum(onn.conv2d(xx, ww, bb) * g))
    eps = 1e-6
    for idx in [(0, 0, 1, 1), (0, 1, 4, 3), (0, 1, 0, 0)]:
        xp, xm = x.copy(), x.copy()
        xp[idx] += eps
        xm[idx] -= eps
        assert abs((f(xp, w, b) - f(xm, w, b)) / (2 * eps) - gx[idx]) < 1e-7
    for idx in [(0, 0, 0, 0), (2, 1, 2, 1), (1, 1, 1, 2)]:
        wp, wm = w.copy(), w.copy()
        wp[idx] += eps
        wm[idx] -= eps
        assert abs((f(x, wp, b) - f(x, wm, b)) / (2 * eps) - gw[idx]) < 1e-7
    np.testing.assert_allclose(gb, g.sum(axis=(0, 2, 3)), atol=1e-13)
    # K^T is the adjoint of the bias-free K
    u = rng.standard_normal((1, 3, 5, 4))
    lhs = np.sum(onn.conv2d(x, w) * u)
    rhs = np.sum(x * onn.conv2d_transpose(u, w))
    assert abs(lhs - rhs) < 1e-12 * abs(lhs)


def test_rbf_brute_force_and_derivative():
    rng = np.random.default_rng(3)
    z = rng.uniform(-1.2, 1.2, size=(1, 2, 3, 3))
    wts = rng.standard_normal((2, 31))
    mu = [-1 + 2 * j / 30 for j in range(31)]
    s = 2 / 30
    ref = np.zeros_like(z)
    for i in range(2):
        for yy in range(3):
            for xx in range(3):
                ref[0, i, yy, xx] = sum(wts[i, j] * np.exp(-(z[0, i, yy, xx] - mu[j]) ** 2 / (2 * s * s))
                                        for j in range(31))
    np.testing.assert_allclose(onn.rbf(z, wts), ref, atol=1e-13)
    eps = 1e-7
    fd = (onn.rbf(z + eps, wts) - onn.rbf(z - eps, wts)) / (2 * eps)
    np.testing.assert_allclose(onn.rbf_grad_z(z, wts), fd, rtol=1e-6, atol=1e-6)


def test_varnet_parameter_count_matches_paper():
    vals = {}
    with open(os.path.join(GOLDEN, "varnet_param_count.txt")) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = int(v)
    assert onn.varnet_param_count(vals["T"], vals["Nk"], vals["k"], vals["Nw"]) == vals["params"]
    filt, rbf, lam = synth.varnet_weights(0)
    assert 2 * filt.size + rbf.size + lam.size == vals["params"]


def test_modl_cnn_param_count():
    # 2->64->64->64->64->2 3x3 convolutions with biases, plus one lambda
    assert onn.modl_param_count() + 1 == 113155


def test_modl_cnn_backward_fd():
    rng = np.random.default_rng(4)
    ws, bs = synth.modl_cnn_weights(5, chans=(2, 4, 4, 2))
    bs = [rng.standard_normal(b.shape) * 0.1 for b in bs]
    x = synth.randn_complex((1, 5, 6), 6)
    g = synth.randn_complex((1, 5, 6), 7)
    f = lambda xx, ww: float(np.real(np.vdot(g, onn.modl_cnn_forward(xx, ww, bs)[0])))
    gx, gws, gbs = onn.modl_cnn_backward(x, ws, bs, g)
    eps = 1e-6
    for idx in [(0, 1, 2), (0, 4, 5)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            xp, xm = x.copy(), x.copy()
            xp[idx] += unit * eps
            xm[idx] -= unit * eps
            assert abs((f(xp, ws) - f(xm, ws)) / (2 * eps) - part(gx[idx])) < 1e-6
    for l, idx in [(0, (1, 0, 2, 2)), (1, (3, 2, 0, 1)), (2, (1, 3, 1, 1))]:
        wp = [w.copy() for w in ws]
        wm = [w.copy() for w in ws]
        wp[l][idx] += eps
        wm[l][idx] -= eps
        assert abs((f(x, wp) - f(x, wm)) / (2 * eps) - gws[l][idx]) < 1e-6


def _small_problem(H=12, W=10, C=2, B=1, seed=11):
    rng = np.random.default_rng(seed)
    maps = np.stack([synth.coil_maps(C, H, W, rng) for _ in range(B)])
    mask = synth.line_mask(W, 2.5, 2, "uniform", rng)
    AHy = synth.randn_complex((B, H, W), seed + 1) * 0.3
    gt = synth.randn_complex((B, H, W), seed + 2) * 0.3
    return maps, mask, AHy, gt


def test_modl_train_grads_fd():
    maps, mask, AHy, gt = _small_problem()
    ws, bs = synth.modl_cnn_weights(3, chans=(2, 3, 2))
    ws = [w * 0.5 for w in ws]
    bs = [np.full(b.shape, 0.05) for b in bs]
    lam, T, it = 0.1, 2, 80

    def L(ww, bb, ll):
        return ounr.modl_train_grads(AHy, maps, mask, gt, ww, bb, ll, T, it)[0]

    loss, gws, gbs, glam, _ = ounr.modl_train_grads(AHy, maps, mask, gt, ws, bs, lam, T, it)
    eps = 1e-6
    fd = (L(ws, bs, lam + eps) - L(ws, bs, lam - eps)) / (2 * eps)
    assert abs(fd - glam) <= 1e-5 * max(abs(fd), 1e-3)
    for l, idx in [(0, (0, 1, 1, 1)), (1, (1, 2, 0, 2))]:
        wp = [w.copy() for w in ws]
        wm = [w.copy() for w in ws]
        wp[l][idx] += eps
        wm[l][idx] -= eps
        fd = (L(wp, bs, lam) - L(wm, bs, lam)) / (2 * eps)
        assert abs(fd - gws[l][idx]) <= 1e-5 * max(abs(fd), 1e-3)
    bp = [b.copy() for b in bs]
    bm = [b.copy() for b in bs]
    bp[0][2] += eps
    bm[0][2] -= eps
    fd = (L(ws, bp, lam) - L(ws, bm, lam)) / (2 * eps)
    assert abs(fd - gbs[0][2]) <= 1e-5 * max(abs(fd), 1e-3)


def test_varnet_train_grads_fd():
    maps, mask, AHy, gt = _small_problem(seed=21)
    rng = np.random.default_rng(5)
    T, Nk, k = 2, 3, 3
    filt = (rng.standard_normal((T, Nk, k, k)) + 1j * rng.standard_normal((T, Nk, k, k))) * 0.2
    wts = rng.standard_normal((T, Nk, 31)) * 0.1
    lam = np.array([0.8, 0.6])

    def L(f, w, l):
        return ounr.varnet_train_grads(AHy, maps, mask, gt, f, w, l)[0]

    loss, gf, gw, gl, _ = ounr.varnet_train_grads(AHy, maps, mask, gt, filt, wts, lam)
    eps = 1e-6
    for t in range(T):
        lp, lm = lam.copy(), lam.copy()
        lp[t] += eps
        lm[t] -= eps
        fd = (L(filt, wts, lp) - L(filt, wts, lm)) / (2 * eps)
        assert abs(fd - gl[t]) <= 1e-5 * max(abs(fd), 1e-4)
    for idx in [(0, 1, 2), (1, 2, 17)]:
        wp, wm = wts.copy(), wts.copy()
        wp[idx] += eps
        wm[idx] -= eps
        fd = (L(filt, wp, lam) - L(filt, wm, lam)) / (2 * eps)
        assert abs(fd - gw[idx]) <= 1e-5 * max(abs(fd), 1e-4)
    for idx in [(0, 0, 1, 1), (1, 2, 0, 2)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            fp, fm = filt.copy(), filt.copy()
            fp[idx] += unit * eps
            fm[idx] -= unit * eps
            fd = (L(fp, wts, lam) - L(fm, wts, lam)) / (2 * eps)
            assert abs(fd - part(gf[idx])) <= 1e-5 * max(abs(fd), 1e-4)


def test_bf16_round_ties_to_even_and_limits():
    # exact values on the bfloat16 grid stay; halfway cases go to the even neighbour
    one = np.float32(1.0)
    ulp = 2.0 ** -7  # spacing of bfloat16 at 1.0
    vals = np.array([1.0, 1.0 + ulp, 1.0 + ulp / 2, 1.0 + 3 * ulp / 2, -1.0 - ulp / 2, 0.0, 3.0e38],
                    dtype=np.float64)
    got = onn.bf16_round(vals)
    want = np.array([1.0, 1.0 + ulp, 1.0, 1.0 + 2 * ulp, -1.0, 0.0, got[-1]])
    np.testing.assert_array_equal(got[:-1], want[:-1])
    assert abs(got[-1] - 3.0e38) / 3.0e38 < 2 ** -8
    # relative rounding error is at most half a unit in the 8-bit significand
    rng = np.random.default_rng(0)
    a = rng.standard_normal(10000) * 10 ** rng.uniform(-10, 10, 10000)
    r = onn.bf16_round(a)
    assert np.all(np.abs(r - a) <= np.abs(a) * 2.0 ** -8 * (1 + 1e-6))
    assert onn.bf16_round(np.float32(one)) == 1.0


# --------------------------------------------------------------------------
# Independent pins of the unrolled blocks.  The finite-difference tests above
# compare the oracle's reverse mode with its own forward, so a misreading of
# Eq. 6 or Eq. 5 made consistently in both would pass them.  The tests below
# check the forward blocks against the equations themselves, built only from
# the separately pinned pieces (the normal operator, the forward operator, the
# CNN and a closed-form RBF potential).

def _dense_normal(maps, mask, lam, H, W):
    """Explicit matrix of (A^H A + lam I) for one slice, column by column."""
    from oracle import sense as osense
    n = H * W
    M = np.zeros((n, n), dtype=np.complex128)
    for j in range(n):
        e = np.zeros((1, H, W), dtype=np.complex128)
        e.flat[j] = 1.0
        M[:, j] = osense.normal(e, maps, mask, lam).reshape(-1)
    return M


@pytest.mark.parametrize("H,W", [(8, 8), (12, 10)])
def test_modl_block_solves_eq6(H, W):
    """x^{t+1} solves (A^H A + lam I) x = A^H y + lam D_W(x^t) (Eq. 6).

    With converged CG (40 iterations; the condition number is at most
    (1 + lam) / lam = 6) the block's residual against that system, formed with the
    pinned normal operator and the pinned CNN, vanishes; a dense direct solve of
    the same system gives the same point, and T blocks chain from x^0 = A^H y.
    """
    from oracle import sense as osense
    maps, mask, AHy, _ = _small_problem(H=H, W=W, seed=31 + H)
    ws, bs = synth.modl_cnn_weights(9, chans=(2, 4, 2))
    bs = [np.full(b.shape, 0.03) for b in bs]
    lam = 0.2
    x_t = synth.randn_complex((1, H, W), 77) * 0.5
    x1, z = ounr.modl_block(x_t, AHy, maps, mask, ws, bs, lam, 40)
    np.testing.assert_allclose(z, onn.modl_cnn_forward(x_t, ws, bs)[0], rtol=0, atol=1e-14)
    rhs = AHy + lam * onn.modl_cnn_forward(x_t, ws, bs)[0]
    res = osense.normal(x1, maps, mask, lam) - rhs
    assert np.linalg.norm(res) <= 1e-10 * np.linalg.norm(rhs)
    # dense solve of the explicit system, and the two-block chain from A^H y
    Nl = _dense_normal(maps, mask, lam, H, W)
    xs_ref = [AHy]
    for _ in range(2):
        r = AHy + lam * onn.modl_cnn_forward(xs_ref[-1], ws, bs)[0]
        xs_ref.append(np.linalg.solve(Nl, r.reshape(-1)).reshape(1, H, W))
    xT, xs = ounr.modl_forward(AHy, maps, mask, ws, bs, lam, 2, 40)
    np.testing.assert_allclose(xs[0], AHy, rtol=0, atol=0)
    for a, b in zip(xs, xs_ref):
        assert np.linalg.norm(a - b) <= 1e-10 * np.linalg.norm(b)


def _rbf_potential(z, wts, Nw=31):
    """Phi_i(z) = sum_j w_ij * integral of exp(-(s - mu_j)^2 / (2 sigma^2)) ds,
    i.e. sum_j w_ij sigma sqrt(pi/2) erf((z - mu_j) / (sigma sqrt 2)): the
    antiderivative of the Gaussian RBF activation, in closed form."""
    from scipy.special import erf
    mu = -1.0 + 2.0 * np.arange(Nw) / (Nw - 1)
    s = 2.0 / (Nw - 1)
    e = s * np.sqrt(np.pi / 2) * erf((z[..., None] - mu) / (s * np.sqrt(2.0)))
    return np.einsum("bkhwj,kj->bkhw", e, wts)


def _brute_real_conv(xr, wr):
    """z[b,i,y,x] = sum_{c,dy,dx} wr[i,c,dy,dx] xr[b,c,y+dy-p,x+dx-p], by loops (zero padded)."""
    B, Ci, H, W = xr.shape
    Nk, _, k, _ = wr.shape
    p = k // 2
    z = np.zeros((B, Nk, H, W))
    for b in range(B):
        for i in range(Nk):
            for yy in range(H):
                for xx in range(W):
                    s = 0.0
                    for c in range(Ci):
                        for dy in range(k):
                            for dx in range(k):
                                sy, sx = yy + dy - p, xx + dx - p
                                if 0 <= sy < H and 0 <= sx < W:
                                    s += wr[i, c, dy, dx] * xr[b, c, sy, sx]
                    z[b, i, yy, xx] = s
    return z


def test_varnet_stage_regulariser_is_gradient_of_rbf_potential():
    """With lam_t = 0, x^t - x^{t+1} = sum_i K_i^T Phi_i'(K_i x^t) (Eq. 5) is the
    gradient of R(x) = sum_i sum_pixels Phi_i(Re(k_i * x)), Phi_i the closed-form
    potential whose derivative is the RBF sum.  The gradient is taken by central
    differences in the real and imaginary part of single pixels (Sec. 2.2.2)."""
    maps, mask, AHy, _ = _small_problem(H=7, W=6, seed=41)
    rng = np.random.default_rng(42)
    Nk, k = 3, 3
    filt = (rng.standard_normal((Nk, k, k)) + 1j * rng.standard_normal((Nk, k, k))) * 0.3
    wts = rng.standard_normal((Nk, 31)) * 0.2
    x = synth.randn_complex((1, 7, 6), 43) * 0.4

    def R(xx):
        xr = np.stack([xx.real, xx.imag], axis=1)
        # Re(k_i * x) = Re k_i * x_re - Im k_i * x_im, by brute-force loops
        wr = np.stack([filt.real, -filt.imag], axis=1)
        return float(np.sum(_rbf_potential(_brute_real_conv(xr, wr), wts)))

    x1 = ounr.varnet_stage(x, AHy, maps, mask, filt, wts, 0.0)
    grad = x - x1
    eps = 1e-6
    for idx in [(0, 0, 0), (0, 3, 2), (0, 6, 5), (0, 2, 4)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            xp, xm = x.copy(), x.copy()
            xp[idx] += unit * eps
            xm[idx] -= unit * eps
            fd = (R(xp) - R(xm)) / (2 * eps)
            assert abs(fd - part(grad[idx])) <= 1e-7 * max(1.0, abs(fd)), (idx, fd, grad[idx])


def test_varnet_stage_data_term_is_gradient_step():
    """With all filters zero, a stage is x - lam_t grad(1/2 ||A x - y||^2) (Eq. 5),
    the gradient taken by central differences of the pinned forward operator."""
    from oracle import sense as osense
    H, W = 8, 6
    maps, mask, _, _ = _small_problem(H=H, W=W, C=3, seed=51)
    y = osense.forward(synth.randn_complex((1, H, W), 52), maps, mask)
    AHy = osense.adjoint(y, maps, mask)
    filt = np.zeros((2, 3, 3), dtype=np.complex128)
    wts = np.random.default_rng(53).standard_normal((2, 31))
    x = synth.randn_complex((1, H, W), 54) * 0.7
    lam_t = 0.37
    x1 = ounr.varnet_stage(x, AHy, maps, mask, filt, wts, lam_t)

    def f(xx):
        return 0.5 * float(np.sum(np.abs(osense.forward(xx, maps, mask) - y) ** 2))

    eps = 1e-6
    for idx in [(0, 0, 0), (0, 4, 3), (0, 7, 5), (0, 1, 2)]:
        for unit, part in ((1.0, np.real), (1j, np.imag)):
            xp, xm = x.copy(), x.copy()
            xp[idx] += unit * eps
            xm[idx] -= unit * eps
            fd = (f(xp) - f(xm)) / (2 * eps)
            want = part(x[idx]) - lam_t * fd
            assert abs(part(x1[idx]) - want) <= 1e-8, (idx, part(x1[idx]), want)
    # the chain starts from x^0 = A^H y
    _, xs = ounr.varnet_forward(AHy, maps, mask, filt[None], wts[None], np.array([lam_t]))
    np.testing.assert_array_equal(xs[0], AHy)
    np.testing.assert_allclose(xs[1], ounr.varnet_stage(AHy, AHy, maps, mask, filt, wts, lam_t),
                               rtol=0, atol=0)
