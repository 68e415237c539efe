"""The torch.autograd.Function wrappers (paper_2202_14005_b300.autograd) on the GPU.

A torch loss is back-propagated through each Function with .backward(); the gradients must
equal, bit for bit, those of the library's reverse-mode calls made directly with the same
incoming gradient (the wrappers add no arithmetic), and agree with the oracle:
* CgDcSolve: grad_rhs and grad_lambda against the oracle's CG derivative (1e-4, the CG
  tolerance);
* UnrolledStep (MoDL): one block against oracle.unrolled.modl_block_backward with the GPU's
  storage rounding (BF16 activations and layer gradients), at the block tolerance 1e-2;
* UnrolledStep (VarNet): one stage against the oracle stage derivative with the GPU's
  rounding points (2e-3, the VarNet tolerance).
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import cg as ocg
from oracle import sense as osense
from oracle import unrolled as ounr
from oracle.nn import bf16_round

from test_gpu_denoiser import make_weights, oracle_weights, unflat, rel

pytestmark = pytest.mark.gpu


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def problem(B=2, Cc=4, H=32, W=232, seed=91):
    rng = np.random.default_rng(seed)
    maps = np.stack([synth.coil_maps(Cc, H, W, rng) for _ in range(B)]).astype(np.complex64)
    mask = synth.line_mask(W, 6.0, 24, "gaussian", rng)
    gt = np.stack([synth.phantom(H, W, rng, 6) for _ in range(B)]).astype(np.complex64)
    noise = synth.complex_noise((B, Cc, H, W), 1e-3, rng)
    y = (osense.forward(gt, maps, mask) + mask * noise).astype(np.complex64)
    AHy = osense.adjoint(y, maps, mask).astype(np.complex64)
    return maps, mask, AHy, gt


def test_cg_dc_solve_function():
    from paper_2202_14005_b300.autograd import CgDcSolve
    from paper_2202_14005_b300.sense import SensePlan
    maps, mask, AHy, gt = problem()
    plan = SensePlan(dev(maps), dev(mask))
    lam = torch.tensor([0.05], dtype=torch.float64, device="cuda", requires_grad=True)
    rhs = dev(AHy).requires_grad_(True)
    x = CgDcSolve.apply(plan, rhs, lam, 10)
    seen = []
    x.register_hook(lambda g: seen.append(g.detach().clone()))
    loss = (x - dev(gt)).abs().pow(2).mean()
    loss.backward()
    torch.cuda.synchronize()
    g = seen[0]
    v_ref, gl_ref = plan.cg_solve_backward(g, x.detach(), None, lam.detach(), 10)
    torch.cuda.synchronize()
    assert torch.equal(rhs.grad, v_ref) and torch.equal(lam.grad, gl_ref)
    gn = g.cpu().numpy()
    v, glb = ocg.cg_solve_backward(maps, mask, 0.05, gn, x.detach().cpu().numpy(), None, 10)
    assert rel(rhs.grad.cpu().numpy(), v) <= 1e-4
    assert abs(lam.grad.item() - glb.sum()) <= 1e-4 * abs(glb.sum())
    assert plan.status() == 0


@pytest.mark.parametrize("store", [True, False])
def test_modl_block_function_matches_direct_call_and_oracle(store):
    from paper_2202_14005_b300 import _lib
    from paper_2202_14005_b300.autograd import UnrolledStep
    from paper_2202_14005_b300.denoiser import ModlDenoiser
    from paper_2202_14005_b300.sense import SensePlan
    maps, mask, AHy, gt = problem(seed=93)
    ws, bs, flat = make_weights(95)
    lam0, iters = 0.05, 10
    plan = SensePlan(dev(maps), dev(mask))
    weights = dev(flat).requires_grad_(True)
    lam = torch.tensor([lam0], dtype=torch.float64, device="cuda", requires_grad=True)
    x0 = dev(AHy)
    x_t = (x0 * 1.0).requires_grad_(True)  # the block input, a leaf so its gradient is kept
    x1 = UnrolledStep.apply(plan, _lib.DENOISER_MODL, weights, lam, x0, x_t, iters, store)
    seen = []
    x1.register_hook(lambda g: seen.append(g.detach().clone()))
    loss = (x1 - dev(gt)).abs().pow(2).mean()
    loss.backward()
    torch.cuda.synchronize()
    g1 = seen[0]
    # the same reverse mode called directly
    B, H, W = x0.shape
    dn = ModlDenoiser(B, H, W)
    L = _lib.lib()
    xn = torch.empty_like(x0)
    _lib.check("unrolled_step", L.unrolled_step(plan._h, _lib.DENOISER_MODL, _p(weights), _p(lam),
                                                _p(x0), _p(x0), _p(xn), iters, _p(dn.ws), dn.ws.numel()))
    gt0 = torch.empty_like(x0)
    gw = torch.zeros_like(weights)
    gl = torch.zeros(1, dtype=torch.float64, device="cuda")
    _lib.check("unrolled_step_backward_ex", L.unrolled_step_backward_ex(
        plan._h, _lib.DENOISER_MODL, _p(weights), _p(lam), _p(x0), _p(x0), _p(xn), _p(g1), _p(gt0),
        _p(gw), _p(gl), iters, _p(dn.ws), dn.ws.numel(), 0))
    torch.cuda.synchronize()
    assert torch.equal(xn, x1.detach())
    assert torch.equal(x_t.grad, gt0) and torch.equal(weights.grad, gw) and torch.equal(lam.grad, gl)
    # the oracle's block derivative with the GPU's storage rounding
    rg, rws, rbs, rgl = ounr.modl_block_backward(
        g1.cpu().numpy(), AHy, x1.detach().cpu().numpy(), AHy, maps, mask, oracle_weights(ws), bs,
        lam0, iters, act_round=bf16_round, grad_round=bf16_round)
    assert rel(x_t.grad.cpu().numpy(), rg) <= 1e-2
    gws, gbs = unflat(weights.grad.cpu().numpy().astype(np.float64))
    for l in range(5):
        assert rel(gws[l], rws[l]) <= 1e-2, f"grad w{l + 1}"
        assert rel(gbs[l], rbs[l]) <= 1e-2, f"grad b{l + 1}"
    assert abs(lam.grad.item() - rgl) <= 1e-2 * abs(rgl)
    assert plan.status() == 0 and dn.status() == 0


def test_denoiser_function_matches_direct_call():
    from paper_2202_14005_b300.autograd import Denoiser
    from paper_2202_14005_b300.denoiser import ModlDenoiser
    from test_gpu_denoiser import make_x
    B, H, W = 2, 24, 232
    ws, bs, flat = make_weights(97)
    x = dev(make_x(B, H, W, 98)).requires_grad_(True)
    weights = dev(flat).requires_grad_(True)
    out = Denoiser.apply(weights, x)
    tgt = dev(synth.randn_complex((B, H, W), 99).astype(np.complex64))
    seen = []
    out.register_hook(lambda g: seen.append(g.detach().clone()))
    (out - tgt).abs().pow(2).sum().backward()
    torch.cuda.synchronize()
    dn = ModlDenoiser(B, H, W)
    gw = torch.zeros_like(weights)
    gx = dn.backward(weights.detach(), x.detach(), seen[0], gw, recompute=True)
    torch.cuda.synchronize()
    assert torch.equal(gx, x.grad) and torch.equal(gw, weights.grad)


def test_varnet_stage_function_matches_direct_call_and_oracle():
    from paper_2202_14005_b300 import _lib
    from paper_2202_14005_b300.autograd import UnrolledStep
    from paper_2202_14005_b300.sense import SensePlan
    from paper_2202_14005_b300.varnet import pack_params
    B, Cc, H, W = 1, 4, 40, 64
    rng = np.random.default_rng(101)
    maps = np.stack([synth.coil_maps(Cc, H, W, rng) for _ in range(B)]).astype(np.complex64)
    mask = synth.line_mask(W, 4.0, 8, "uniform", rng)
    gt = np.stack([synth.phantom(H, W, rng, 6) for _ in range(B)]).astype(np.complex64)
    AHy = osense.adjoint(osense.forward(gt, maps, mask), maps, mask).astype(np.complex64)
    filt, rbf, lamv = synth.varnet_weights(103, T=1)
    rbf = rbf + 0.05 * np.random.default_rng(104).standard_normal(rbf.shape)
    prm = pack_params(filt, rbf, lamv)[0]
    plan = SensePlan(dev(maps), dev(mask))
    params = dev(prm).requires_grad_(True)
    x_t = dev(AHy).requires_grad_(True)
    x1 = UnrolledStep.apply(plan, _lib.DENOISER_VARNET, params, None, dev(AHy), x_t, 0, True)
    seen = []
    x1.register_hook(lambda g: seen.append(g.detach().clone()))
    (x1 - dev(gt)).abs().pow(2).mean().backward()
    torch.cuda.synchronize()
    g1 = seen[0]
    # oracle stage derivative with the GPU's rounding points (BF16 filters, Phi', Phi'' K g)
    f64 = prm.astype(np.float64)
    from paper_2202_14005_b300.varnet import unpack_params
    rf, rw, rl = unpack_params(f64)
    rg, gf, gwts, glam = ounr.varnet_stage_backward(g1.cpu().numpy(), AHy, AHy, maps, mask, rf[0], rw[0],
                                                    rl[0], rnd=bf16_round)
    assert rel(x_t.grad.cpu().numpy(), rg) <= 2e-3
    ref = pack_params(gf[None], gwts[None], np.array([glam])).astype(np.float64)[0]
    got = params.grad.cpu().numpy().astype(np.float64)
    nf = got.size - 24 * 31 - 1
    assert rel(got[:nf], ref[:nf]) <= 2e-3
    assert rel(got[nf:-1], ref[nf:-1]) <= 2e-3
    assert abs(got[-1] - ref[-1]) <= 1e-4 * abs(ref[-1])
    assert plan.status() == 0
