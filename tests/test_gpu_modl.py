"""GPU parity of the MoDL unrolled blocks, the loss and one training step's
gradients against the oracle (Eq. 6; derivatives of S^{-1}, Sec. 2.3.2).

The oracle mirrors the GPU's storage precision (BF16 activations and layer
gradients, BF16 weights in the 64-channel layers); the CG path is FP32 with
FP64 scalars.  The rounding points match, but a rounding decision can still
differ where the GPU's FP32 value and the oracle's FP64 value fall on two
sides of a BF16 boundary (a jump of 2^-8 relative on that element); from the
second unrolled block on, such flips in the denoiser input add up to a few
1e-3, and in the reverse pass they also flip ReLU masks.  Tolerances:
* one block's reverse mode with both sides given identical inputs (x^t,
  x^{t+1}, dL/dx^{t+1}) and the oracle's reverse pass using the denoiser
  activations the GPU recomputed (so both take the same ReLU masks): the
  per-layer bound, 1e-2 relative;
* block outputs and the loss of the two-block chain: 1e-2;
* gradients of the whole two-block chain (two BF16 reverse chains in series,
  each input differing by the flips above): 5e-2 relative L2;
* the same kind of chain taken block by block, each block's reverse mode
  given the GPU's own intermediates (x^t, x^{t+1} and the incoming gradient
  the GPU produced for that block) and the oracle using the activations the
  GPU stored for that block: 1e-2 for every block and for the chain's sums;
* the forward against the exact oracle (FP32 master weights, FP64 arithmetic,
  no rounding hooks): 2e-2, the accumulated BF16 storage error of K blocks.
"""
import numpy as np
import pytest
import torch

import synth
from oracle import cg as ocg
from oracle import nn as onn
from oracle import sense as osense
from oracle import unrolled as ounr
from oracle.nn import bf16_round

from test_gpu_denoiser import make_weights, oracle_weights, unflat, rel

pytestmark = pytest.mark.gpu


def problem(B=2, C=4, H=24, W=232, seed=3):
    rng = np.random.default_rng(seed)
    maps = np.stack([synth.coil_maps(C, H, W, rng) for _ in range(B)]).astype(np.complex64)
    mask = synth.line_mask(W, 6.0, 24, "gaussian", rng)
    gt = np.stack([synth.phantom(H, W, rng, 6) for _ in range(B)]).astype(np.complex64)
    noise = synth.complex_noise((B, C, H, W), 1e-3, rng)
    y = (osense.forward(gt, maps, mask) + mask * noise).astype(np.complex64)
    return maps, mask, y, gt


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def test_modl_forward_blocks_and_training_gradients():
    from paper_2202_14005_b300.modl import ModlTrainer
    maps, mask, y, gt = problem()
    ws, bs, flat = make_weights(21)
    K, iters, lam = 2, 10, 0.05
    tr = ModlTrainer(dev(maps), dev(mask), dev(flat), lam, K, iters)
    loss = tr.gradients(dev(y), dev(gt))
    torch.cuda.synchronize()
    AHy = osense.adjoint(y, maps, mask).astype(np.complex64)
    wo = oracle_weights(ws)
    rloss, rgws, rgbs, rglam, rxT = ounr.modl_train_grads(
        AHy.astype(np.complex128), maps, mask, gt, wo, bs, lam, K, iters,
        act_round=bf16_round, grad_round=bf16_round)
    # forward: every block output
    _, rxs = ounr.modl_forward(AHy.astype(np.complex128), maps, mask, wo, bs, lam, K, iters,
                               act_round=bf16_round)
    for t in range(K + 1):
        assert rel(tr.xs[t].cpu().numpy(), rxs[t]) <= 1e-2, f"x^{t}"
    assert abs(loss.item() - rloss) <= 1e-2 * rloss
    gws, gbs = unflat(tr.gw.cpu().numpy().astype(np.float64))
    for l in range(5):
        assert rel(gws[l], rgws[l]) <= 5e-2, f"grad w{l + 1}"
        assert rel(gbs[l], rgbs[l]) <= 5e-2, f"grad b{l + 1}"
    assert abs(tr.gl.item() - rglam) <= 5e-2 * abs(rglam)
    assert tr.plan.status() == 0 and tr.denoiser_status() == 0


def test_modl_stored_activations_match_recompute():
    """The reverse pass reusing each block's stored activations and output (one denoiser workspace
    per block) gives bitwise the same loss and gradients as recomputing them from the block input."""
    from paper_2202_14005_b300.modl import ModlTrainer
    maps, mask, y, gt = problem(B=2, C=4, H=24, W=232, seed=13)
    ws, bs, flat = make_weights(17)
    res = []
    for store in (True, False):
        tr = ModlTrainer(dev(maps), dev(mask), dev(flat), 0.05, 3, 6, store_activations=store)
        loss = tr.gradients(dev(y), dev(gt))
        torch.cuda.synchronize()
        assert len(tr.dns) == (3 if store else 1)
        res.append((loss.item(), tr.gw.cpu().numpy().copy(), tr.gl.item(), tr.xs[-1].cpu().numpy()))
        assert tr.plan.status() == 0 and tr.denoiser_status() == 0
    (l0, g0, gl0, x0), (l1, g1, gl1, x1) = res
    assert l0 == l1 and gl0 == gl1
    assert np.array_equal(g0, g1) and np.array_equal(x0, x1)


def test_modl_block_reverse_mode_parity():
    """unrolled_step_backward against the oracle block derivative on identical inputs."""
    import ctypes as C
    from paper_2202_14005_b300 import _lib
    from paper_2202_14005_b300.modl import ModlTrainer
    maps, mask, y, gt = problem(B=2, C=5, H=20, W=232, seed=9)
    ws, bs, flat = make_weights(31)
    lam, iters = 0.05, 10
    tr = ModlTrainer(dev(maps), dev(mask), dev(flat), lam, 1, iters)
    tr.forward(dev(y))  # x^0 = A^H y, x^1
    torch.cuda.synchronize()
    x0 = tr.xs[0].cpu().numpy()
    x1 = tr.xs[1].cpu().numpy()
    g1 = (synth.randn_complex(x0.shape, 44) * 1e-3).astype(np.complex64)
    gd = dev(g1)
    gt0 = torch.empty_like(gd)
    L = _lib.lib()
    p = lambda t: C.c_void_p(t.data_ptr())
    _lib.check("unrolled_step_backward", L.unrolled_step_backward(
        tr.plan._h, _lib.DENOISER_MODL, p(tr.weights), p(tr.lam), p(tr.xs[0]), p(tr.xs[0]),
        p(tr.xs[1]), p(gd), p(gt0), p(tr.gw), p(tr.gl), iters, p(tr.dn.ws), tr.dn.ws.numel()))
    torch.cuda.synchronize()
    wo = oracle_weights(ws)
    # the GPU's recomputed activations of D(x^0) (left in the denoiser workspace)
    acts, _ = tr.dn.activations()
    A = [a.float().cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2) for a in acts]
    xr = bf16_round(onn.c2r(x0))
    z = x0.astype(np.complex128) + onn.r2c(onn.conv2d(A[3], wo[4], bs[4]))
    v, glam_b = ocg.cg_solve_backward(maps, mask, lam, g1, x1, z, iters)
    cache = {"acts": [xr] + A, "pre": A + [None]}  # ReLU masks: pre > 0 <=> stored activation > 0
    rg, rws, rbs = onn.modl_cnn_backward(x0, wo, bs, lam * v, cache=cache, grad_round=bf16_round)
    rgl = float(glam_b.sum())
    assert rel(gt0.cpu().numpy(), rg) <= 1e-2
    gws, gbs = unflat(tr.gw.cpu().numpy().astype(np.float64))
    for l in range(5):
        assert rel(gws[l], rws[l]) <= 1e-2, f"grad w{l + 1}"
        assert rel(gbs[l], rbs[l]) <= 1e-2, f"grad b{l + 1}"
    assert abs(tr.gl.item() - rgl) <= 1e-2 * abs(rgl)
    assert tr.plan.status() == 0 and tr.denoiser_status() == 0


def test_modl_train_step_updates_and_clears_gradients():
    from paper_2202_14005_b300.modl import ModlTrainer
    maps, mask, y, gt = problem(B=1, C=3, H=16, W=64, seed=5)
    ws, bs, flat = make_weights(22)
    tr = ModlTrainer(dev(maps), dev(mask), dev(flat), 0.05, 2, 5, lr=1e-3, lam_lr=1e-3)
    w0 = tr.weights.clone()
    l0 = tr.lam.clone()
    losses = [tr.train_step(dev(y), dev(gt)).item() for _ in range(3)]
    torch.cuda.synchronize()
    assert not torch.equal(w0, tr.weights) and not torch.equal(l0, tr.lam)
    assert torch.count_nonzero(tr.gw).item() == 0 and tr.gl.item() == 0.0
    assert all(np.isfinite(losses))
    assert tr.lam.item() >= 1e-6


def _block_reverse(tr, t, g_in, recompute=0):
    """unrolled_step_backward_ex of block t alone, into fresh gradient buffers."""
    import ctypes as C
    from paper_2202_14005_b300 import _lib
    p = lambda a: C.c_void_p(a.data_ptr())
    g_out = torch.empty_like(g_in)
    gw = torch.zeros_like(tr.weights)
    gl = torch.zeros(1, dtype=torch.float64, device="cuda")
    ws = tr._ws(t)
    _lib.check("unrolled_step_backward_ex", _lib.lib().unrolled_step_backward_ex(
        tr.plan._h, _lib.DENOISER_MODL, p(tr.weights), p(tr.lam), p(tr.xs[0]), p(tr.xs[t]),
        p(tr.xs[t + 1]), p(g_in), p(g_out), p(gw), p(gl), tr.iters, p(ws), ws.numel(), recompute))
    return g_out, gw, gl


def _oracle_block_reverse(dn, x_t, x_next, g_next, wo, bs, lam, solve):
    """The oracle's block derivative given the GPU's stored activations of D(x^t)
    (ReLU masks and layer inputs as the GPU took them); solve(g) applies S^{-1}."""
    acts, _ = dn.activations()
    A = [a.float().cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2) for a in acts]
    xr = bf16_round(onn.c2r(x_t))
    z = x_t.astype(np.complex128) + onn.r2c(onn.conv2d(A[3], wo[4], bs[4]))
    v = solve(g_next)
    glam = float(np.sum(np.real(np.conj(v) * (z - x_next))))
    cache = {"acts": [xr] + A, "pre": A + [None]}
    rg, rws, rbs = onn.modl_cnn_backward(x_t, wo, bs, lam * v, cache=cache, grad_round=bf16_round)
    return rg, rws, rbs, glam


def _check_block(tag, g_out, gw, gl, ref, tol=1e-2):
    rg, rws, rbs, rgl = ref
    errs = {"grad_x": rel(g_out.cpu().numpy(), rg)}
    gws, gbs = unflat(gw.cpu().numpy().astype(np.float64))
    for l in range(5):
        errs[f"w{l + 1}"] = rel(gws[l], rws[l])
        errs[f"b{l + 1}"] = rel(gbs[l], rbs[l])
    if gl is not None:
        errs["lambda"] = abs(gl.item() - rgl) / abs(rgl)
    print(tag, {k: f"{v:.2e}" for k, v in errs.items()})
    for k, v in errs.items():
        assert v <= tol, f"{tag} {k}: {v:.3e}"


def test_denoiser_reverse_mode_at_workload_shape():
    """denoiser_backward on the 4 x 256 x 232 workload (about 14 row segments per CTA in the
    64-channel weight-gradient kernel, the halo ring wrapping across tiles) against the
    oracle fed the GPU's recomputed activations: every layer's weight, bias and input
    gradient within 1e-2."""
    from paper_2202_14005_b300.denoiser import ModlDenoiser
    from test_gpu_denoiser import make_x
    cfg = synth.CONFIGS[3]
    B, H, W = cfg.B, cfg.H, cfg.W
    ws, bs, flat = make_weights(41)
    x = make_x(B, H, W, 43)
    g = (synth.randn_complex((B, H, W), 44) * 0.1).astype(np.complex64)
    dn = ModlDenoiser(B, H, W)
    wt = dev(flat)
    gw = torch.zeros_like(wt)
    gx = dn.backward(wt, dev(x), dev(g), gw, recompute=True)
    torch.cuda.synchronize()
    wo = oracle_weights(ws)
    acts, _ = dn.activations()
    A = [a.float().cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2) for a in acts]
    cache = {"acts": [bf16_round(onn.c2r(x))] + A, "pre": A + [None]}
    rg, rws, rbs = onn.modl_cnn_backward(x, wo, bs, g, cache=cache, grad_round=bf16_round)
    _check_block("denoiser 4x256x232", gx, gw, None, (rg, rws, rbs, None))
    assert dn.status() == 0


def test_unrolled_step_reverse_mode_at_workload_shape():
    """One MoDL block of the training workload (4 slices, 12 coils, 256 x 232, 10 CG
    iterations) in reverse mode from its stored activations, against the oracle block
    derivative on identical inputs (1e-2)."""
    from paper_2202_14005_b300.modl import ModlTrainer
    cfg = synth.CONFIGS[3]
    d = synth.make_slices(cfg)
    maps, mask = d["maps"].astype(np.complex64), d["mask"]
    y = (osense.forward(d["x_gt"], maps, mask) + mask * d["noise"]).astype(np.complex64)
    ws, bs, flat = make_weights(47)
    lam, iters = cfg.lam, cfg.cg_iters
    tr = ModlTrainer(dev(maps), dev(mask), dev(flat), lam, 1, iters)
    tr.forward(dev(y))
    torch.cuda.synchronize()
    x0, x1 = tr.xs[0].cpu().numpy(), tr.xs[1].cpu().numpy()
    g1 = (synth.randn_complex(x0.shape, 48) * 1e-3).astype(np.complex64)
    g0, gw, gl = _block_reverse(tr, 0, dev(g1), recompute=0)
    torch.cuda.synchronize()
    ref = _oracle_block_reverse(tr.dns[0], x0, x1, g1, oracle_weights(ws), bs, lam,
                                lambda g: ocg.cg_solve(maps, mask, lam, g, None, iters)[0])
    _check_block("block 4x12x256x232", g0, gw, gl, ref)
    assert tr.plan.status() == 0 and tr.denoiser_status() == 0


def test_modl_chain_gradients_block_by_block():
    """A three-block chain in reverse mode, one block at a time on the GPU's own
    intermediates: each block's gradients, and their sums over the chain, within 1e-2 of
    the oracle's block derivatives; the sums agree with the trainer's whole-chain
    gradients up to FP32 accumulation order."""
    from paper_2202_14005_b300.modl import ModlTrainer
    maps, mask, y, gt = problem(B=2, C=4, H=32, W=232, seed=23)
    ws, bs, flat = make_weights(25)
    K, iters, lam = 3, 10, 0.05
    wo = oracle_weights(ws)
    tr = ModlTrainer(dev(maps), dev(mask), dev(flat), lam, K, iters)
    tr.gradients(dev(y), dev(gt))              # whole chain, for the sums
    torch.cuda.synchronize()
    gw_chain, gl_chain = tr.gw.clone(), tr.gl.clone()
    import ctypes as C
    from paper_2202_14005_b300 import _lib
    tr.forward(dev(y))                          # the same forward again (bitwise)
    g = torch.empty_like(tr.xs[K])              # the loss gradient, as the whole-chain pass formed it
    loss = torch.zeros(1, dtype=torch.float64, device="cuda")
    p = lambda a: C.c_void_p(a.data_ptr())
    _lib.check("sense_mse_loss", _lib.lib().sense_mse_loss(tr.plan._h, p(tr.xs[K]), p(dev(gt)),
                                                           p(loss), p(g)))
    gw_sum = torch.zeros_like(tr.weights)
    gl_sum = 0.0
    rw_sum = [np.zeros_like(w) for w in wo]
    rb_sum = [np.zeros_like(b) for b in bs]
    rl_sum = 0.0
    solve = lambda gg: ocg.cg_solve(maps, mask, lam, gg, None, iters)[0]
    for t in range(K - 1, -1, -1):
        g_out, gw, gl = _block_reverse(tr, t, g, recompute=0)
        torch.cuda.synchronize()
        ref = _oracle_block_reverse(tr.dns[t], tr.xs[t].cpu().numpy(), tr.xs[t + 1].cpu().numpy(),
                                    g.cpu().numpy(), wo, bs, lam, solve)
        _check_block(f"block {t}", g_out, gw, gl, ref)
        gw_sum += gw
        gl_sum += gl.item()
        for l in range(5):
            rw_sum[l] += ref[1][l]
            rb_sum[l] += ref[2][l]
        rl_sum += ref[3]
        g = g_out
    gws, gbs = unflat(gw_sum.cpu().numpy().astype(np.float64))
    for l in range(5):
        assert rel(gws[l], rw_sum[l]) <= 1e-2, f"chain w{l + 1}"
        assert rel(gbs[l], rb_sum[l]) <= 1e-2, f"chain b{l + 1}"
    assert abs(gl_sum - rl_sum) <= 1e-2 * abs(rl_sum)
    # the whole-chain call adds the same block contributions (in another FP32 order)
    assert rel(gw_chain.cpu().numpy(), gw_sum.cpu().numpy()) <= 1e-5
    assert abs(gl_chain.item() - gl_sum) <= 1e-9 * abs(gl_sum)
    assert tr.plan.status() == 0 and tr.denoiser_status() == 0


def test_modl_forward_against_exact_oracle():
    """The GPU forward (BF16 weights and activations, FP32 CG) against the exact FP64
    oracle with the FP32 master weights and no rounding hooks: every block output within
    2e-2."""
    from paper_2202_14005_b300.modl import ModlTrainer
    maps, mask, y, gt = problem(B=2, C=6, H=48, W=232, seed=29)
    ws, bs, flat = make_weights(27)
    K, iters, lam = 3, 10, 0.05
    tr = ModlTrainer(dev(maps), dev(mask), dev(flat), lam, K, iters)
    tr.forward(dev(y))
    torch.cuda.synchronize()
    AHy = osense.adjoint(y, maps, mask)
    _, rxs = ounr.modl_forward(AHy, maps, mask, ws, bs, lam, K, iters)
    errs = [rel(tr.xs[t].cpu().numpy(), rxs[t]) for t in range(K + 1)]
    print("MoDL forward vs exact oracle, per block:", [f"{e:.2e}" for e in errs])
    for t, e in enumerate(errs):
        assert e <= 2e-2, f"x^{t}: {e:.3e}"
    assert tr.plan.status() == 0


def test_modl_block_on_toeplitz_plan():
    """unrolled_step and its reverse mode on a non-Cartesian (Toeplitz) plan, against the
    oracle block with the Toeplitz normal operator inside its CG (Sec. 2.3.3, Eq. 6)."""
    from oracle import noncart as onc
    from paper_2202_14005_b300.modl import ModlTrainer
    from paper_2202_14005_b300.sense import SensePlan, toeplitz_psf
    B, Cc, N = 2, 3, 40
    rng = np.random.default_rng(61)
    maps = np.stack([synth.coil_maps(Cc, N, N, rng) for _ in range(B)]).astype(np.complex64)
    traj = synth.radial_trajectory(24, 80, N).reshape(-1, 2).astype(np.float32)
    psf = toeplitz_psf(dev(traj), N, N)
    torch.cuda.synchronize()
    rpsf = psf.cpu().numpy().astype(np.complex128)
    plan = SensePlan.toeplitz(dev(maps), psf)
    ws, bs, flat = make_weights(63)
    # Without density compensation this trajectory's normal operator has its largest eigenvalue
    # near 35 (1 for a Cartesian mask), so lambda = 2 gives S_lambda the condition number
    # (35 + 2) / 2 < 21 of the Cartesian workloads, for which the tolerances are set.
    lam, iters = 2.0, 10
    tr = ModlTrainer(dev(maps), None, dev(flat), lam, 1, iters, plan=plan)
    gt = np.stack([synth.phantom(N, N, rng, 6) for _ in range(B)]).astype(np.complex64)
    AHy = onc.toeplitz_normal(gt, maps, rpsf, 0.0).astype(np.complex64)
    tr.forward_from_adjoint(dev(AHy))
    torch.cuda.synchronize()
    x0, x1 = tr.xs[0].cpu().numpy(), tr.xs[1].cpu().numpy()
    wo = oracle_weights(ws)
    # forward: the block output from the GPU's own denoiser output D(x^0)
    acts, _ = tr.dns[0].activations()
    A3 = acts[3].float().cpu().numpy().astype(np.float64).transpose(0, 3, 1, 2)
    z = x0.astype(np.complex128) + onn.r2c(onn.conv2d(A3, wo[4], bs[4]))
    Sl = lambda p_: onc.toeplitz_normal(p_, maps, rpsf, lam)
    rx1, _ = ocg.cg(Sl, AHy.astype(np.complex128) + lam * z, None, iters)
    assert rel(x1, rx1) <= 1e-4
    g1 = (synth.randn_complex(x0.shape, 64) * 1e-3).astype(np.complex64)
    g0, gw, gl = _block_reverse(tr, 0, dev(g1), recompute=0)
    torch.cuda.synchronize()
    ref = _oracle_block_reverse(tr.dns[0], x0, x1, g1, wo, bs, lam,
                                lambda g: ocg.cg(Sl, g, None, iters)[0])
    _check_block("toeplitz block", g0, gw, gl, ref)
    assert tr.plan.status() == 0 and tr.denoiser_status() == 0
