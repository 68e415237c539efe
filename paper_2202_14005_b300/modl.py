"""MoDL training and inference on the libsense C ABI (call sequencing only).

One training step (Eq. 6, Sec. 2.3.2): x^0 = A^H y; K unrolled blocks
x^{t+1} = S_lambda^{-1}(A^H y + lambda D_W(x^t)) with shared weights; loss
mean |x^K - x_gt|^2; reverse mode block by block; Adam on the weights and lambda.
Every arithmetic step runs in the library's kernels.

Each block keeps its denoiser activations and output in a workspace of its own (about 0.6 GB
for the 4-slice 256 x 232 workload), and its reverse pass reuses them.  With
store_activations=False one workspace serves all blocks and each reverse pass recomputes the
activations from the block input instead (the checkpointing of Sec. 2.2.4); the results are the
same.
"""
from __future__ import annotations

import ctypes as C

import torch

from . import _lib
from .denoiser import ModlDenoiser
from .sense import SensePlan


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


class ModlTrainer:
    def __init__(self, maps: torch.Tensor, mask: torch.Tensor, weights: torch.Tensor, lam: float,
                 K: int, cg_iters: int, lr: float = 1e-4, lam_lr: float = 1e-4, plan: SensePlan | None = None,
                 store_activations: bool = True):
        # plan: an existing plan (e.g. a non-Cartesian Toeplitz plan, Sec. 2.3.3) instead of maps/mask
        self.plan = plan if plan is not None else SensePlan(maps, mask)
        B, H, W = self.plan.img_shape()
        self.B, self.H, self.W = B, H, W
        self.K, self.iters = K, cg_iters
        self.store = store_activations
        self.dns = [ModlDenoiser(B, H, W, device=maps.device) for _ in range(K if store_activations else 1)]
        self.dn = self.dns[0]
        self.weights = weights
        self.lam = torch.tensor([lam], dtype=torch.float64, device=maps.device)
        dev = maps.device
        self.gw = torch.zeros_like(weights)
        self.gl = torch.zeros(1, dtype=torch.float64, device=dev)
        self.m_w, self.v_w = torch.zeros_like(weights), torch.zeros_like(weights)
        self.m_l, self.v_l = torch.zeros_like(self.lam), torch.zeros_like(self.lam)
        self.xs = [torch.empty((B, H, W), dtype=torch.complex64, device=dev) for _ in range(K + 1)]
        self.g = [torch.empty((B, H, W), dtype=torch.complex64, device=dev) for _ in range(2)]
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        self.lr, self.lam_lr = lr, lam_lr
        self.t = 0
        self._lib = _lib.lib()

    def use_plan(self, plan: SensePlan) -> None:
        """Run later calls on another plan of the same image shape (another batch of slices:
        other maps, same mask), keeping the weights, optimizer state and workspaces."""
        if tuple(plan.img_shape()) != (self.B, self.H, self.W):
            raise ValueError("plan image shape differs from the trainer's")
        self.plan = plan

    def _step_args(self):
        return (self.plan._h, _lib.DENOISER_MODL, _p(self.weights), _p(self.lam))

    def forward(self, y: torch.Tensor) -> torch.Tensor:
        """x^K for k-space y [B, C, H, W] (also keeps every x^t)."""
        self.plan._sync_stream()
        self.plan.adjoint(y, out=self.xs[0])
        return self.forward_from_adjoint(None)

    def forward_from_adjoint(self, AHy: torch.Tensor | None) -> torch.Tensor:
        """x^K from a given x^0 = A^H y (the non-Cartesian case precomputes it, Sec. 2.3.3);
        None: x^0 already in self.xs[0]."""
        self.plan._sync_stream()
        if AHy is not None:
            self.xs[0].copy_(AHy)
        h, kind, w, lam = self._step_args()
        for t in range(self.K):
            ws = self._ws(t)
            _lib.check("unrolled_step", self._lib.unrolled_step(
                h, kind, w, lam, _p(self.xs[0]), _p(self.xs[t]), _p(self.xs[t + 1]), self.iters,
                _p(ws), ws.numel()))
        return self.xs[self.K]

    def _ws(self, t: int) -> torch.Tensor:
        return self.dns[t if self.store else 0].ws

    def denoiser_status(self) -> int:
        """OR of the device status words of the denoiser workspaces (0 = no error)."""
        st = 0
        for d in self.dns:
            st |= d.status()
        return st

    def gradients(self, y: torch.Tensor, gt: torch.Tensor):
        """Forward, loss and reverse mode; gradients accumulate into self.gw / self.gl."""
        self.forward(y)
        return self._reverse(gt)

    def gradients_from_adjoint(self, AHy: torch.Tensor, gt: torch.Tensor):
        """As gradients, from a given x^0 = A^H y (non-Cartesian data, Sec. 2.3.3)."""
        self.forward_from_adjoint(AHy)
        return self._reverse(gt)

    def train_step_from_adjoint(self, AHy: torch.Tensor, gt: torch.Tensor):
        loss = self.gradients_from_adjoint(AHy, gt)
        self._update()
        return loss

    def _reverse(self, gt: torch.Tensor):
        _lib.check("sense_mse_loss", self._lib.sense_mse_loss(
            self.plan._h, _p(self.xs[self.K]), _p(gt), _p(self.loss), _p(self.g[0])))
        h, kind, w, lam = self._step_args()
        cur = 0
        for t in range(self.K - 1, -1, -1):
            ws = self._ws(t)
            _lib.check("unrolled_step_backward_ex", self._lib.unrolled_step_backward_ex(
                h, kind, w, lam, _p(self.xs[0]), _p(self.xs[t]), _p(self.xs[t + 1]), _p(self.g[cur]),
                _p(self.g[cur ^ 1]), _p(self.gw), _p(self.gl), self.iters, _p(ws), ws.numel(),
                0 if self.store else 1))
            cur ^= 1
        return self.loss

    def train_step(self, y: torch.Tensor, gt: torch.Tensor):
        loss = self.gradients(y, gt)
        self._update()
        return loss

    def _update(self):
        self.t += 1
        st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        _lib.check("adam_update_f32", self._lib.adam_update_f32(
            _p(self.weights), _p(self.gw), _p(self.m_w), _p(self.v_w), self.weights.numel(),
            self.lr, 0.9, 0.999, 1e-8, self.t, st))
        _lib.check("adam_update_f64", self._lib.adam_update_f64(
            _p(self.lam), _p(self.gl), _p(self.m_l), _p(self.v_l), 1, self.lam_lr, 0.9, 0.999, 1e-8,
            self.t, 1e-6, st))
