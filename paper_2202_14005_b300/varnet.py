"""Variational Network training and inference on the libsense C ABI (call
sequencing only).

One training step (Eq. 5, Sec. 2.3.1): x^0 = A^H y (optionally scaled to max|x^0| = 1 per
slice, the paper's VarNet data scaling, with the target scaled alike); T gradient stages
x^{t+1} = x^t - sum_i K_i^T Phi_i'(K_i x^t) - lambda_t (A^H A x^t - A^H y),
each with its own filters, RBF weights and step size; loss mean |x^T - x_gt|^2;
reverse mode stage by stage from the stored stage inputs; Adam on all
parameters.  Every arithmetic step runs in the library's kernels.

Parameter vector of one stage (float32, 6,553 values): real-form filters
w[24][2][11][11] (w[i][0] = Re k_i, w[i][1] = -Im k_i), RBF weights r[24][31],
lambda_t.
"""
from __future__ import annotations

import ctypes as C

import numpy as np
import torch

from . import _lib
from .sense import SensePlan

NK, NW, KS = 24, 31, 11
N_FILT = NK * 2 * KS * KS
N_PARAM = N_FILT + NK * NW + 1


def _p(t):
    return None if t is None else C.c_void_p(t.data_ptr())


def pack_params(filt, rbf_w, lam) -> np.ndarray:
    """Stage parameters [T, 6553] float32 from complex filters [T, 24, 11, 11],
    RBF weights [T, 24, 31] and step sizes [T] (layout conversion only)."""
    filt = np.asarray(filt, dtype=np.complex128)
    T = filt.shape[0]
    wr = np.stack([filt.real, -filt.imag], axis=2).reshape(T, -1)
    return np.concatenate([wr, np.asarray(rbf_w, dtype=np.float64).reshape(T, -1),
                           np.asarray(lam, dtype=np.float64).reshape(T, 1)], axis=1).astype(np.float32)


def unpack_params(vec):
    """Inverse of pack_params: (complex filters, RBF weights, lambda) per stage."""
    v = np.asarray(vec, dtype=np.float64).reshape(-1, N_PARAM)
    wr = v[:, :N_FILT].reshape(-1, NK, 2, KS, KS)
    return wr[:, :, 0] - 1j * wr[:, :, 1], v[:, N_FILT:N_FILT + NK * NW].reshape(-1, NK, NW), v[:, -1]


class VarNetTrainer:
    """VarNet training on the library.  Each stage keeps z = K x^t and u = Phi'(z) in a workspace
    of its own (about 0.2 GB per stage for 4 slices of 320 x 368), and its reverse pass reuses them
    so that only K g is computed; with store_activations=False one workspace serves all stages and
    the reverse pass recomputes K x^t (the checkpointing of Sec. 2.2.4).  Results are the same.

    With a workspace per stage the reverse pass also keeps one gradient buffer per stage and lets
    each stage's parameter gradients run on the library's side streams beside the next stages
    (defer_join, joined once at the end of the pass); the gradients are bitwise the same."""

    def __init__(self, maps: torch.Tensor, mask: torch.Tensor, params: torch.Tensor, lr: float = 1e-4,
                 normalize: bool = False, store_activations: bool = True, plan: SensePlan | None = None,
                 optimizer: str = "adam", ipalm_tau=(1e-2, 1e-2, 1e-2)):
        # plan: an existing plan of the maps and mask instead of a new one
        self.plan = plan if plan is not None else SensePlan(maps, mask)
        B, H, W = self.plan.img_shape()
        self.B, self.H, self.W = B, H, W
        if params.dim() != 2 or params.shape[1] != N_PARAM or params.dtype != torch.float32:
            raise ValueError(f"params must be float32 [T, {N_PARAM}]")
        if not params.is_contiguous() or params.device != maps.device:
            raise ValueError("params must be contiguous and on the maps' device")
        self._lib = _lib.lib()
        if self._lib.varnet_param_count() != N_PARAM:
            raise RuntimeError("libsense VarNet parameter layout mismatch")
        self.T = params.shape[0]
        self.params = params
        dev = maps.device
        nb = self._lib.varnet_workspace_bytes(B, H, W)
        self.store = store_activations
        self.wss = [torch.zeros(int(nb), dtype=torch.uint8, device=dev)
                    for _ in range(self.T if store_activations else 1)]
        self.ws = self.wss[0]
        self.gp = torch.zeros_like(params)
        self.m, self.v = torch.zeros_like(params), torch.zeros_like(params)
        self.xs = [torch.empty((B, H, W), dtype=torch.complex64, device=dev) for _ in range(self.T + 1)]
        # A^H A x^t of every stage, written by the forward pass for the reverse pass
        self.nx = [torch.empty((B, H, W), dtype=torch.complex64, device=dev) for _ in range(self.T)]
        # gradient w.r.t. x^t for t = T .. 0; one buffer per stage when the joins are deferred
        self.defer_join = store_activations
        self.g = [torch.empty((B, H, W), dtype=torch.complex64, device=dev)
                  for _ in range(self.T + 1 if store_activations else 2)]
        self.loss = torch.zeros(1, dtype=torch.float64, device=dev)
        # data scaling max|x^0| = 1 per slice (Sec. 2.3.1); gtn holds the equally scaled target
        self.normalize = normalize
        self.scale = torch.ones(B, dtype=torch.float32, device=dev)
        self.gtn = torch.empty((B, H, W), dtype=torch.complex64, device=dev)
        self.lr = lr
        self.t = 0
        # optimizer "adam", or "ipalm" (Sec. 2.3.1): params then hold the inertial point z^k and
        # self.x the iterate x^k; the filter constraints are applied by every update
        if optimizer not in ("adam", "ipalm"):
            raise ValueError("optimizer must be 'adam' or 'ipalm'")
        self.optimizer = optimizer
        self.ipalm_tau = tuple(float(v) for v in ipalm_tau)
        self.x = params.clone() if optimizer == "ipalm" else None

    def _ws(self, t: int) -> torch.Tensor:
        return self.wss[t if self.store else 0]

    def use_plan(self, plan: SensePlan) -> None:
        """Run later calls on another plan of the same image shape (another batch of slices),
        keeping the parameters, optimizer state and workspaces."""
        if tuple(plan.img_shape()) != (self.B, self.H, self.W):
            raise ValueError("plan image shape differs from the trainer's")
        self.plan = plan

    def stage(self, t: int, x_t: torch.Tensor, x_next: torch.Tensor, nx_out: torch.Tensor | None = None):
        ws = self._ws(t)
        _lib.check("varnet_stage", self._lib.varnet_stage(
            self.plan._h, _p(self.params[t]), _p(self.xs[0]), _p(x_t), _p(x_next), _p(nx_out), _p(ws),
            ws.numel()))

    def stage_backward(self, t: int, x_t, grad_next, grad_t, nx_t: torch.Tensor | None = None,
                       reuse: bool = False, defer: bool = False):
        """Reverse pass of stage t; reuse: take z and u from the stage's workspace as stage(t) left
        them for the same x_t and parameters (else K x_t is recomputed); defer: leave the stage's
        parameter gradients running on the side streams (join() before reading self.gp or reusing
        the stage's workspace and buffers)."""
        ws = self._ws(t)
        flags = (0 if reuse else 1) | (2 if defer else 0)
        _lib.check("varnet_stage_backward_ex", self._lib.varnet_stage_backward_ex(
            self.plan._h, _p(self.params[t]), _p(self.xs[0]), _p(x_t), _p(nx_t), _p(grad_next), _p(grad_t),
            _p(self.gp[t]), _p(ws), ws.numel(), flags))

    def join(self):
        """The plan's stream waits for the library's side streams (deferred parameter gradients)."""
        _lib.check("sense_streams_join", self._lib.sense_streams_join(
            C.c_void_p(torch.cuda.current_stream().cuda_stream)))

    def activations(self, t: int = 0):
        """Views of the workspace activations of the last call on stage t's workspace:
        u, v (bfloat16 [B, H, W, 32]) and z = K x, K g (float32 [B, H, W, 24])."""
        ws = self._ws(t)
        off = (C.c_size_t * 4)()
        _lib.check("varnet_workspace_offsets", self._lib.varnet_workspace_offsets(self.B, self.H, self.W, off))
        n = self.B * self.H * self.W
        u = ws[off[0]:off[0] + n * 64].view(torch.bfloat16).view(self.B, self.H, self.W, 32)
        v = ws[off[1]:off[1] + n * 64].view(torch.bfloat16).view(self.B, self.H, self.W, 32)
        z = ws[off[2]:off[2] + n * 96].view(torch.float32).view(self.B, self.H, self.W, NK)
        kg = ws[off[3]:off[3] + n * 96].view(torch.float32).view(self.B, self.H, self.W, NK)
        return u, v, z, kg

    def forward(self, y: torch.Tensor, gt: torch.Tensor | None = None) -> torch.Tensor:
        """x^T for k-space y [B, C, H, W] (also keeps every x^t).  With normalize, x^0 = A^H y is
        scaled to max|x^0| = 1 per slice (self.scale) and gt, if given, is scaled alike into self.gtn."""
        self.plan._sync_stream()
        self.plan.adjoint(y, out=self.xs[0])
        if gt is not None:
            self.gtn.copy_(gt)
        if self.normalize:
            _lib.check("sense_normalize_max", self._lib.sense_normalize_max(
                self.plan._h, _p(self.xs[0]), _p(self.gtn) if gt is not None else None, _p(self.scale)))
        for t in range(self.T):
            self.stage(t, self.xs[t], self.xs[t + 1], self.nx[t])
        return self.xs[self.T]

    def gradients(self, y: torch.Tensor, gt: torch.Tensor):
        """Forward, loss and reverse mode; gradients accumulate into self.gp."""
        self.forward(y, gt)
        _lib.check("sense_mse_loss", self._lib.sense_mse_loss(
            self.plan._h, _p(self.xs[self.T]), _p(self.gtn), _p(self.loss), _p(self.g[0])))
        if self.defer_join:
            # g[T - t] holds the gradient w.r.t. x^t: every stage reads and writes its own buffers
            for t in range(self.T - 1, -1, -1):
                self.stage_backward(t, self.xs[t], self.g[self.T - 1 - t], self.g[self.T - t], self.nx[t],
                                    reuse=True, defer=True)
            self.join()
        else:
            cur = 0
            for t in range(self.T - 1, -1, -1):
                self.stage_backward(t, self.xs[t], self.g[cur], self.g[cur ^ 1], self.nx[t], reuse=self.store)
                cur ^= 1
        return self.loss

    def train_step(self, y: torch.Tensor, gt: torch.Tensor):
        loss = self.gradients(y, gt)
        self.t += 1
        st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
        if self.optimizer == "ipalm":
            # update k = self.t: gradient taken at z^k; next inertia alpha_{k+1} = k / (k + 3)
            tf, tr_, tl = self.ipalm_tau
            _lib.check("ipalm_update_varnet", self._lib.ipalm_update_varnet(
                _p(self.params), _p(self.gp), _p(self.x), self.T, tf, tr_, tl, self.t / (self.t + 3.0), st))
            return loss
        _lib.check("adam_update_f32", self._lib.adam_update_f32(
            _p(self.params), _p(self.gp), _p(self.m), _p(self.v), self.params.numel(), self.lr, 0.9,
            0.999, 1e-8, self.t, st))
        return loss

    def iterate(self) -> torch.Tensor:
        """The current parameters: x^k under iPALM (params holds the inertial point), else params."""
        return self.x if self.optimizer == "ipalm" else self.params
