"""GPU parity of the iPALM update of the VarNet parameters (ipalm_update_varnet) against the
oracle (oracle.ipalm), and a short iPALM training run of the VarNet.

The update is elementwise apart from the per-filter mean and norm (FP32 block sums): 1e-6
relative L2 per block, and the constraints hold to FP32 rounding."""
import ctypes as C

import numpy as np
import pytest
import torch

import synth
from oracle import ipalm as oip

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_ipalm_update_matches_oracle():
    from paper_2202_14005_b300 import _lib
    from paper_2202_14005_b300.varnet import pack_params, unpack_params
    T = 3
    rng = np.random.default_rng(5)
    filt = (rng.standard_normal((T, 24, 11, 11)) + 1j * rng.standard_normal((T, 24, 11, 11))) * 0.2 + 0.01
    filt[0, :4] *= 0.001          # some filters end inside the unit ball, some on its boundary
    rbf = rng.standard_normal((T, 24, 31))
    lam = np.array([0.3, -0.2, 1.0])
    z = pack_params(filt, rbf, lam)
    g = pack_params(rng.standard_normal(filt.shape) + 1j * rng.standard_normal(filt.shape),
                    rng.standard_normal(rbf.shape), rng.standard_normal(T))
    xk = pack_params(filt * 0.9, rbf * 0.9, lam * 0.9)
    tau, alpha = (0.05, 0.1, 0.2), 0.4
    zd, gd, xd = (torch.from_numpy(a.copy()).cuda() for a in (z, g, xk))
    L = _lib.lib()
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    _lib.check("ipalm_update_varnet", L.ipalm_update_varnet(_p(zd), _p(gd), _p(xd), T, *tau, alpha, st))
    torch.cuda.synchronize()
    # oracle: x^{k+1} = P(z - tau g) blockwise, z^{k+1} = x^{k+1} + alpha (x^{k+1} - x^k)
    zb = unpack_params(z.astype(np.float64))
    gb = unpack_params(g.astype(np.float64))
    x1 = oip.step(zb, gb, tau)
    z1 = oip.extrapolate(x1, unpack_params(xk.astype(np.float64)), alpha)
    gx = unpack_params(xd.cpu().numpy().astype(np.float64))
    gz = unpack_params(zd.cpu().numpy().astype(np.float64))
    for got, want in ((gx, x1), (gz, z1)):
        for a, b in zip(got, want):
            assert rel(a, b) <= 1e-6
    assert torch.count_nonzero(gd).item() == 0
    f = gx[0]
    assert np.abs(f.mean(axis=(-2, -1))).max() <= 1e-6
    assert np.sqrt((np.abs(f) ** 2).sum(axis=(-2, -1))).max() <= 1 + 1e-6
    assert gx[2].min() >= 0.0
    # argument checks run before any launch
    assert L.ipalm_update_varnet(_p(zd), _p(gd), _p(xd), T, *tau, 1.0, st) == -7
    assert L.ipalm_update_varnet(_p(zd), _p(zd), _p(xd), T, *tau, 0.5, st) == -2


def test_varnet_trains_with_ipalm():
    from paper_2202_14005_b300.varnet import VarNetTrainer, pack_params, unpack_params
    B, Cc, H, W = 1, 4, 48, 64
    rng = np.random.default_rng(9)
    maps = torch.from_numpy(np.stack([synth.coil_maps(Cc, H, W, rng)]).astype(np.complex64)).cuda()
    mask = torch.from_numpy(synth.line_mask(W, 4.0, 8, "uniform", rng)).cuda()
    gt = torch.from_numpy(np.stack([synth.phantom(H, W, rng, 6)]).astype(np.complex64)).cuda()
    filt, rbf, lam = synth.varnet_weights(11, T=3)
    prm = torch.from_numpy(pack_params(filt, rbf, lam)).cuda()
    tr = VarNetTrainer(maps, mask, prm, normalize=True, optimizer="ipalm", ipalm_tau=(1e-3, 1e-3, 1e-2))
    y = tr.plan.forward(gt)
    losses = [tr.train_step(y, gt).item() for _ in range(20)]
    torch.cuda.synchronize()
    assert all(np.isfinite(losses)) and losses[-1] < losses[0]
    f, _, l = unpack_params(tr.iterate().cpu().numpy())
    assert np.abs(f.mean(axis=(-2, -1))).max() <= 1e-6
    assert np.sqrt((np.abs(f) ** 2).sum(axis=(-2, -1))).max() <= 1 + 1e-6
    assert l.min() >= 0.0
    assert torch.count_nonzero(tr.gp).item() == 0
    assert tr.plan.status() == 0
