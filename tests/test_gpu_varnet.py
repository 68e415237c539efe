"""GPU parity of the VarNet gradient stage (Eq. 5, Sec. 2.3.1) and its reverse
mode against the oracle.

Precision protocol: the filters are BF16 (the tests draw BF16-exact filters,
so the oracle sees the same values); K x and K g are computed from a two-term
BF16 split of the image (hi + lo) and are as accurate as FP32 accumulation;
Phi'(K x), Phi''(K x) K g, and x and g as operands of the filter gradient
are stored in BF16; the RBF sums run in FP32 over the 13 centres nearest z.
* Mirrored oracle (those stored operands rounded with bf16_round, FP64
  otherwise).  What remains is FP32 arithmetic: K x accumulates 726 products
  of zero-mean filters whose |products| exceed |z| 10-30x (z to ~1e-6, checked
  per layer below); Gaussian terms change by (|z - mu| / sigma^2) dz, so BF16
  storage of Phi'(z) occasionally rounds the other way; K^T and the filter
  gradient sum 2,904 such products again.  Observed (B300): 6e-5 to 5e-4
  relative L2 on the regulariser, stage gradient and parameter gradients.
  Bounds: 2e-3 on those and on whole stage outputs; 1e-4 on the lambda
  gradient, an FP64 dot with the FP32 residual A^H A x - A^H y.
* Exact oracle (no rounding): the BF16 storage of Phi' and Phi'' K g adds
  relative 2^-9 per element: observed 1e-3 to 3e-3; bound 2e-2.
* A chain of three stages (initial, monotone RBF weights), forward, MSE loss
  and the reverse pass through all stages: every stage passes the differences
  above on through its Jacobian, and the stage-0 gradients sit at the end of
  three reverse stages.  Observed 2e-5 to 1e-3; bounds 1e-2 on the stage
  outputs, the loss and the gradients.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import nn as onn
from oracle import sense as osense
from oracle import unrolled as ounr
from oracle.nn import bf16_round

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128 if np.iscomplexobj(a) or np.iscomplexobj(b) else np.float64)
    b = np.asarray(b, dtype=a.dtype)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def problem(B, Cc, H, W, seed):
    rng = np.random.default_rng(seed)
    maps = np.stack([synth.coil_maps(Cc, H, W, rng) for _ in range(B)]).astype(np.complex64)
    mask = synth.line_mask(W, 4.0, max(4, W // 16), "uniform", rng)
    gt = np.stack([synth.phantom(H, W, rng, 6) for _ in range(B)]).astype(np.complex64)
    noise = synth.complex_noise((B, Cc, H, W), 1e-3, rng)
    y = (osense.forward(gt, maps, mask) + mask * noise).astype(np.complex64)
    AHy = osense.adjoint(y, maps, mask).astype(np.complex64)
    return maps, mask, y, gt, AHy


def params(T, seed, lam=0.7, perturb=True):
    """Stage parameters, as float32 and as the float64 values the oracle sees
    (filters complex [T, 24, 11, 11]).  perturb: add noise to the initial RBF
    weights (a non-monotone Phi', so Phi'' changes sign)."""
    from paper_2202_14005_b300.varnet import pack_params, unpack_params
    filt, rbfw, _ = synth.varnet_weights(seed, T)
    filt = bf16_round(filt.real) + 1j * bf16_round(filt.imag)  # the kernels use BF16 filters
    rng = np.random.default_rng(seed + 100)
    if perturb:
        rbfw = rbfw + 0.05 * rng.standard_normal(rbfw.shape)
    vec = pack_params(filt, rbfw, np.full(T, lam))
    f, r, l = unpack_params(vec)
    return vec, f, r, l


def trainer(maps, mask, vec, AHy):
    from paper_2202_14005_b300.varnet import VarNetTrainer
    tr = VarNetTrainer(dev(maps), dev(mask), dev(vec))
    tr.xs[0].copy_(dev(AHy))
    return tr


SHAPES = [(2, 4, 24, 200), (1, 3, 12, 64), (1, 2, 16, 300)]


@pytest.mark.parametrize("shape", SHAPES)
def test_stage_forward(shape):
    B, Cc, H, W = shape
    maps, mask, y, gt, AHy = problem(B, Cc, H, W, seed=H + W)
    vec, f, r, lam = params(1, seed=W)
    x = (AHy + 0.05 * synth.randn_complex(AHy.shape, 3)).astype(np.complex64)
    tr = trainer(maps, mask, vec, AHy)
    out = torch.empty_like(tr.xs[0])
    tr.stage(0, dev(x), out)
    torch.cuda.synchronize()
    out = out.cpu().numpy()
    dc = osense.normal(x, maps, mask, 0.0) - AHy
    reg_gpu = x.astype(np.complex128) - out - lam[0] * dc
    reg_m, _ = onn.varnet_regulariser(x, f[0], r[0], bf16_round)
    reg_e, _ = onn.varnet_regulariser(x, f[0], r[0])
    print(f"varnet regulariser: mirrored {rel(reg_gpu, reg_m):.2e} exact {rel(reg_gpu, reg_e):.2e}")
    assert rel(reg_gpu, reg_m) <= 2e-3, rel(reg_gpu, reg_m)
    assert rel(reg_gpu, reg_e) <= 2e-2, rel(reg_gpu, reg_e)
    ref = ounr.varnet_stage(x, AHy, maps, mask, f[0], r[0], lam[0], bf16_round)
    assert rel(out, ref) <= 2e-3, rel(out, ref)
    assert tr.plan.status() == 0


def _backward(tr, x, g, nx=None):
    gt_ = torch.empty_like(tr.xs[0])
    tr.stage_backward(0, dev(x), dev(g), gt_, nx)
    torch.cuda.synchronize()
    return gt_


def _check_backward(tr, gt_, x, g, AHy, maps, mask, f, r, lam, tol_m, tol_e):
    from paper_2202_14005_b300.varnet import unpack_params
    gf, gr, gl = unpack_params(tr.gp[0].cpu().numpy())
    mir = ounr.varnet_stage_backward(g, x, AHy, maps, mask, f[0], r[0], lam[0], bf16_round)
    ex = ounr.varnet_stage_backward(g, x, AHy, maps, mask, f[0], r[0], lam[0])
    got = (gt_.cpu().numpy(), gf[0], gr[0])
    for name, a, m, e in zip(("grad_x", "grad_filters", "grad_rbf"), got, mir[:3], ex[:3]):
        print(f"varnet {name}: mirrored {rel(a, m):.2e} exact {rel(a, e):.2e}")
        assert rel(a, m) <= tol_m, f"{name} vs mirrored oracle: {rel(a, m):.3e}"
        assert rel(a, e) <= tol_e, f"{name} vs exact oracle: {rel(a, e):.3e}"
    assert abs(gl[0] - mir[3]) <= 1e-4 * abs(mir[3]), (gl[0], mir[3])
    # the reverse-mode regulariser term alone
    Ng = osense.normal(g, maps, mask, 0.0)
    back_gpu = g.astype(np.complex128) - got[0] - lam[0] * Ng
    back_m = g.astype(np.complex128) - mir[0] - lam[0] * Ng
    assert rel(back_gpu, back_m) <= tol_m, rel(back_gpu, back_m)


@pytest.mark.parametrize("shape", SHAPES)
def test_layer_outputs_from_workspace(shape):
    """Each layer of the reverse-mode recomputation against the oracle, fed the
    GPU's own inputs: z = K x and K g (FP32 accumulation of the three-term
    image split; observed 1e-6, bound 1e-4), u = Phi'(z) and v = Phi''(z) K g
    from the GPU's z and K g (FP32 sums of 13 Gaussians, then one BF16
    rounding: observed 1.7e-3, bound 4e-3 = 2^-8)."""
    B, Cc, H, W = shape
    maps, mask, y, gt, AHy = problem(B, Cc, H, W, seed=H + W + 1)
    vec, f, r, lam = params(1, seed=W + 1)
    x = (AHy + 0.05 * synth.randn_complex(AHy.shape, 5)).astype(np.complex64)
    g = (0.1 * synth.randn_complex(AHy.shape, 6)).astype(np.complex64)
    tr = trainer(maps, mask, vec, AHy)
    _backward(tr, x, g)
    u, v, z, kg = [t.float().cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2) for t in tr.activations()]
    wr = onn.varnet_filters_real(f[0])
    rz = onn.conv2d(onn.c2r(x), wr)
    rkg = onn.conv2d(onn.c2r(g), wr)
    print(f"varnet layers: z {rel(z, rz):.2e} Kg {rel(kg, rkg):.2e}")
    assert rel(z, rz) <= 1e-4
    assert rel(kg, rkg) <= 1e-4
    ru = onn.rbf(z, r[0])
    rv = onn.rbf_grad_z(z, r[0]) * kg
    print(f"varnet layers: u {rel(u[:, :24], ru):.2e} v {rel(v[:, :24], rv):.2e}")
    assert rel(u[:, :24], ru) <= 4e-3
    assert rel(v[:, :24], rv) <= 4e-3
    assert not u[:, 24:].any() and not v[:, 24:].any()


@pytest.mark.parametrize("shape", SHAPES)
def test_stage_backward(shape):
    B, Cc, H, W = shape
    maps, mask, y, gt, AHy = problem(B, Cc, H, W, seed=H + W + 1)
    vec, f, r, lam = params(1, seed=W + 1)
    x = (AHy + 0.05 * synth.randn_complex(AHy.shape, 5)).astype(np.complex64)
    g = (0.1 * synth.randn_complex(AHy.shape, 6)).astype(np.complex64)
    tr = trainer(maps, mask, vec, AHy)
    gt_ = _backward(tr, x, g)
    _check_backward(tr, gt_, x, g, AHy, maps, mask, f, r, lam, 2e-3, 2e-2)
    assert tr.plan.status() == 0


def test_stage_full_size_slice():
    """One slice of the knee workload (15 coils, 320 x 368: two full 128-pixel
    tiles and a 112-pixel tail), forward and reverse mode."""
    cfg = synth.CONFIGS[4]
    maps, mask, y, gt, AHy = problem(1, cfg.C, cfg.H, cfg.W, seed=41)
    vec, f, r, lam = params(1, seed=42, lam=1.0)
    x = AHy
    g = (1e-3 * synth.randn_complex(AHy.shape, 7)).astype(np.complex64)
    tr = trainer(maps, mask, vec, AHy)
    out = torch.empty_like(tr.xs[0])
    tr.stage(0, dev(x), out)
    gt_ = _backward(tr, x, g)
    out = out.cpu().numpy()
    ref = ounr.varnet_stage(x, AHy, maps, mask, f[0], r[0], lam[0], bf16_round)
    assert rel(out, ref) <= 2e-3, rel(out, ref)
    dc = osense.normal(x, maps, mask, 0.0) - AHy
    reg_gpu = x.astype(np.complex128) - out - lam[0] * dc
    reg_m, _ = onn.varnet_regulariser(x, f[0], r[0], bf16_round)
    reg_e, _ = onn.varnet_regulariser(x, f[0], r[0])
    print(f"varnet regulariser: mirrored {rel(reg_gpu, reg_m):.2e} exact {rel(reg_gpu, reg_e):.2e}")
    assert rel(reg_gpu, reg_m) <= 2e-3, rel(reg_gpu, reg_m)
    assert rel(reg_gpu, reg_e) <= 2e-2, rel(reg_gpu, reg_e)
    _check_backward(tr, gt_, x, g, AHy, maps, mask, f, r, lam, 2e-3, 2e-2)
    assert tr.plan.status() == 0


def test_backward_deterministic_accumulating_and_aliasing():
    maps, mask, y, gt, AHy = problem(2, 3, 16, 136, seed=8)
    vec, f, r, lam = params(1, seed=9)
    x = AHy
    g = (0.1 * synth.randn_complex(AHy.shape, 10)).astype(np.complex64)
    tr = trainer(maps, mask, vec, AHy)
    g1 = _backward(tr, x, g).clone()
    p1 = tr.gp.clone()
    g2 = _backward(tr, x, g)
    assert torch.equal(g1, g2)
    assert torch.equal(tr.gp, 2 * p1)  # gradients accumulate
    # A^H A x_t handed over by the forward pass gives the same bits as recomputing it
    nx = torch.empty_like(tr.xs[0])
    tr.stage(0, dev(x), torch.empty_like(tr.xs[0]), nx)
    tr.gp.zero_()
    g3 = _backward(tr, x, g, nx)
    assert torch.equal(g1, g3) and torch.equal(tr.gp, p1)
    # grad_t may overwrite x_t
    xa = dev(x)
    tr.gp.zero_()
    tr.stage_backward(0, xa, dev(g), xa)
    torch.cuda.synchronize()
    assert torch.equal(xa, g1) and torch.equal(tr.gp, p1)


def test_chain_training_gradients():
    """Three stages, MSE loss, full reverse mode against the mirrored oracle."""
    maps, mask, y, gt, AHy = problem(2, 4, 20, 136, seed=12)
    T = 3
    vec, f, r, lam = params(T, seed=13, lam=0.5, perturb=False)
    from paper_2202_14005_b300.varnet import VarNetTrainer, unpack_params
    tr = VarNetTrainer(dev(maps), dev(mask), dev(vec))
    loss = tr.gradients(dev(y), dev(gt))
    torch.cuda.synchronize()
    rloss, rgf, rgw, rgl, rxT = ounr.varnet_train_grads(AHy.astype(np.complex128), maps, mask, gt, f, r, lam,
                                                        bf16_round)
    _, rxs = ounr.varnet_forward(AHy.astype(np.complex128), maps, mask, f, r, lam, bf16_round)
    for t in range(T + 1):
        assert rel(tr.xs[t].cpu().numpy(), rxs[t]) <= 1e-2, f"x^{t}"
    assert abs(loss.item() - rloss) <= 1e-2 * rloss
    gf, gr, gl = unpack_params(tr.gp.cpu().numpy())
    for t in range(T):
        print(f"varnet chain stage {t}: x {rel(tr.xs[t + 1].cpu().numpy(), rxs[t + 1]):.2e} filters "
              f"{rel(gf[t], rgf[t]):.2e} rbf {rel(gr[t], rgw[t]):.2e} lambda {abs(gl[t] / rgl[t] - 1):.2e}")
    for t in range(T):
        assert rel(gf[t], rgf[t]) <= 1e-2, f"grad filters stage {t}"
        assert rel(gr[t], rgw[t]) <= 1e-2, f"grad rbf stage {t}"
        assert abs(gl[t] - rgl[t]) <= 1e-2 * abs(rgl[t]), f"grad lambda stage {t}"
    assert tr.plan.status() == 0


def test_stored_stage_state_matches_recompute():
    """The reverse pass reusing each stage's stored z = K x and u (one workspace per stage) against
    recomputing them in the reverse pass: the forward is identical, z = K x is bitwise the same, and
    u = Phi'(z) evaluated by the reverse kernel's epilogue can differ in the last bit from the
    forward kernel's (the compiler contracts the RBF arithmetic of the two kernels differently), so
    the gradients agree to rounding."""
    maps, mask, y, gt, AHy = problem(2, 4, 20, 136, seed=21)
    vec, *_ = params(3, seed=22, lam=0.5, perturb=True)
    from paper_2202_14005_b300.varnet import VarNetTrainer
    res = []
    for store in (True, False):
        tr = VarNetTrainer(dev(maps), dev(mask), dev(vec), store_activations=store)
        loss = tr.gradients(dev(y), dev(gt))
        torch.cuda.synchronize()
        assert len(tr.wss) == (3 if store else 1)
        res.append((loss.item(), tr.gp.cpu().numpy().copy(), tr.xs[-1].cpu().numpy()))
        assert tr.plan.status() == 0
    (l0, g0, x0), (l1, g1, x1) = res
    assert l0 == l1 and np.array_equal(x0, x1)
    assert rel(g0, g1) <= 1e-5


def test_deferred_parameter_gradients_bitwise_equal():
    """Reverse pass with each stage's parameter gradients left on the library's side streams
    (overlapping the next stages, one join at the end) against joining every stage: the same
    kernels in the same order per gradient, so the gradients are bitwise equal."""
    maps, mask, y, gt, AHy = problem(2, 4, 20, 136, seed=31)
    vec, *_ = params(4, seed=32, lam=0.5, perturb=True)
    from paper_2202_14005_b300.varnet import VarNetTrainer
    res = []
    for defer in (True, False):
        tr = VarNetTrainer(dev(maps), dev(mask), dev(vec))
        tr.defer_join = defer
        loss = tr.gradients(dev(y), dev(gt))
        torch.cuda.synchronize()
        res.append((loss.item(), tr.gp.cpu().numpy().copy()))
        assert tr.plan.status() == 0
    (l0, g0), (l1, g1) = res
    assert l0 == l1
    assert np.array_equal(g0, g1)
    assert np.count_nonzero(g0) > 0


def test_train_step_updates_and_clears_gradients():
    maps, mask, y, gt, AHy = problem(1, 3, 16, 64, seed=2)
    vec, *_ = params(2, seed=3)
    from paper_2202_14005_b300.varnet import VarNetTrainer
    tr = VarNetTrainer(dev(maps), dev(mask), dev(vec), lr=1e-3)
    p0 = tr.params.clone()
    losses = [tr.train_step(dev(y), dev(gt)).item() for _ in range(3)]
    torch.cuda.synchronize()
    assert not torch.equal(p0, tr.params)
    assert torch.count_nonzero(tr.gp).item() == 0
    assert all(np.isfinite(losses))


def test_host_argument_errors():
    from paper_2202_14005_b300 import _lib
    from paper_2202_14005_b300.sense import SensePlan
    L = _lib.lib()
    p = lambda t: C.c_void_p(t.data_ptr())
    maps, mask, y, gt, AHy = problem(1, 2, 8, 64, seed=1)
    vec, *_ = params(1, seed=1)
    tr = trainer(maps, mask, vec, AHy)
    x = tr.xs[0]
    out = torch.empty_like(x)
    pv = dev(vec)
    h = tr.plan._h
    ws = tr.ws
    EWORKSPACE, EINVAL_PTR, EUNSUPPORTED = -6, -2, -4
    assert L.varnet_stage(h, p(pv), p(x), p(x), p(out), None, p(ws), 16) == EWORKSPACE
    assert L.varnet_stage(h, p(pv), p(x), p(x), p(x), None, p(ws), ws.numel()) == EINVAL_PTR
    assert L.varnet_stage(h, p(pv), p(x), p(x), p(out), p(out), p(ws), ws.numel()) == EINVAL_PTR
    assert L.varnet_stage_backward(h, p(pv), p(x), p(x), None, p(out), p(out), p(pv), p(ws), ws.numel()) == \
        EINVAL_PTR
    mis = C.c_void_p(out.data_ptr() + 8)
    assert L.varnet_stage(h, p(pv), p(x), p(x), mis, None, p(ws), ws.numel()) == EINVAL_PTR
    # rows wider than the filter-gradient kernel covers
    W = 520
    maps2 = dev(synth.coil_maps(2, 8, W, np.random.default_rng(0))[None].astype(np.complex64))
    mask2 = dev(np.ones(W, dtype=np.float32))
    plan2 = SensePlan(maps2, mask2)
    x2 = torch.zeros((1, 8, W), dtype=torch.complex64, device="cuda")
    o2 = torch.empty_like(x2)
    nb = L.varnet_workspace_bytes(1, 8, W)
    ws2 = torch.zeros(int(nb), dtype=torch.uint8, device="cuda")
    assert L.varnet_stage(plan2._h, p(pv), p(x2), p(x2), p(o2), None, p(ws2), nb) == EUNSUPPORTED
    torch.cuda.synchronize()


def test_denoiser_and_unrolled_step_kind_varnet():
    """The VarNet kind of the generic calls: denoiser_forward/backward give the
    regulariser R(x) = sum_i K_i^T Phi_i'(K_i x) and its reverse mode (checked
    against the oracle stage with lambda = 0, whose regulariser terms carry the
    opposite sign); unrolled_step(_backward) equal varnet_stage(_backward) bit
    for bit."""
    from paper_2202_14005_b300 import _lib
    from paper_2202_14005_b300.varnet import unpack_params
    L = _lib.lib()
    p = lambda t: C.c_void_p(t.data_ptr())
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    VN = 1
    B, Cc, H, W = 2, 3, 16, 200
    maps, mask, y, gt, AHy = problem(B, Cc, H, W, seed=77)
    vec, f, r, lam = params(1, seed=78)
    x = (AHy + 0.05 * synth.randn_complex(AHy.shape, 9)).astype(np.complex64)
    g = (0.1 * synth.randn_complex(AHy.shape, 10)).astype(np.complex64)
    assert L.denoiser_param_count(VN) == vec.shape[1]
    nb = L.denoiser_workspace_bytes(VN, B, H, W)
    ws = torch.zeros(int(nb), dtype=torch.uint8, device="cuda")
    pv = dev(vec[0])
    xd, gd = dev(x), dev(g)
    out = torch.empty_like(xd)
    _lib.check("denoiser_forward", L.denoiser_forward(VN, p(pv), p(xd), p(out), p(ws), nb, B, H, W, st))
    gx = torch.empty_like(xd)
    gw = torch.zeros_like(pv)
    _lib.check("denoiser_backward", L.denoiser_backward(VN, p(pv), p(xd), p(gd), p(gx), p(gw), p(ws), nb,
                                                         B, H, W, 1, st))
    torch.cuda.synchronize()
    reg_m, _ = onn.varnet_regulariser(x, f[0], r[0], bf16_round)
    assert rel(out.cpu().numpy(), reg_m) <= 2e-3
    g_t, g_f, g_w, _ = ounr.varnet_stage_backward(g, x, AHy, maps, mask, f[0], r[0], 0.0, bf16_round)
    assert rel(gx.cpu().numpy(), g.astype(np.complex128) - g_t) <= 2e-3
    gf, gr, gl = unpack_params(gw.cpu().numpy())
    assert rel(gf[0], -g_f) <= 2e-3 and rel(gr[0], -g_w) <= 2e-3
    assert gl[0] == 0.0  # lambda_t is not a parameter of the regulariser
    # unrolled_step with the VarNet kind is the VarNet stage
    tr = trainer(maps, mask, vec, AHy)
    a1, a2 = torch.empty_like(xd), torch.empty_like(xd)
    tr.stage(0, xd, a1)
    lam_unused = torch.zeros(1, dtype=torch.float64, device="cuda")
    _lib.check("unrolled_step", L.unrolled_step(tr.plan._h, VN, p(tr.params[0]), p(lam_unused), p(tr.xs[0]),
                                                p(xd), p(a2), 0, p(tr.ws), tr.ws.numel()))
    b1 = _backward(tr, x, g)
    p1 = tr.gp.clone()
    tr.gp.zero_()
    b2 = torch.empty_like(xd)
    _lib.check("unrolled_step_backward", L.unrolled_step_backward(
        tr.plan._h, VN, p(tr.params[0]), p(lam_unused), p(tr.xs[0]), p(xd), p(a2), p(gd), p(b2), p(tr.gp[0]),
        p(lam_unused), 0, p(tr.ws), tr.ws.numel()))
    torch.cuda.synchronize()
    assert torch.equal(a1, a2) and torch.equal(b1, b2) and torch.equal(p1, tr.gp)
    assert lam_unused.item() == 0.0


def test_normalize_max_scales_each_slice():
    """sense_normalize_max: max |x_b| = 1 per slice afterwards, the second
    tensor scaled by the same factor, an all-zero slice untouched."""
    from paper_2202_14005_b300.varnet import VarNetTrainer
    maps, mask, y, gt, AHy = problem(3, 2, 16, 64, seed=4)
    vec, *_ = params(1, seed=5)
    tr = VarNetTrainer(dev(maps), dev(mask), dev(vec), normalize=True)
    yd = dev(y)
    yd[2].zero_()
    gtd = dev(gt)
    tr.forward(yd, gtd)
    torch.cuda.synchronize()
    a = AHy.astype(np.complex128)
    a[2] = 0
    m = np.abs(a).reshape(3, -1).max(axis=1)
    sc = tr.scale.cpu().numpy()
    assert np.allclose(sc[:2], 1 / m[:2], rtol=1e-5) and sc[2] == 1.0
    x0 = tr.xs[0].cpu().numpy()
    assert np.allclose(np.abs(x0[:2]).reshape(2, -1).max(axis=1), 1.0, rtol=1e-5)
    assert not x0[2].any()
    assert rel(tr.gtn.cpu().numpy()[:2], gt[:2] * sc[:2, None, None]) <= 1e-6
