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
  each input differing by the flips above): 5e-2 relative L2.
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
