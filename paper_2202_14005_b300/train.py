"""Training of the unrolled networks on operator-simulated data, and their held-out evaluation
against plain CG-SENSE on the same slices.

    python -m paper_2202_14005_b300.train --network modl [--steps N] [--train-slices N] ...

Data (Sec. 3 trains MoDL on 12-coil brain data at R = 6 and the VarNet on 15-coil knee data at
R = 4; those data sets are not available here, so seeded synthetic slices of the same shapes
stand in for them):
* ground truth: seeded random-ellipse phantoms with smooth phase (and texture for the MoDL
  workload), coil maps normalised to sum |S_c|^2 = 1, the workload's line mask;
* k-space: y = A x_gt, applied by the library's forward operator (Eq. 4), plus complex Gaussian
  noise (sigma 1e-3) at the sampled locations;
* training slices come from the "train" seed split and the evaluation slices from the
  workload's own seeds, so the two sets never share a slice.

Radial data (network modl_radial, Sec. 2.3.3): golden-angle radial samples simulated by the
library's non-uniform DFT with noise at the samples; x^0 = A^H y by the non-uniform adjoint; the
normal operator through the Toeplitz embedding of the trajectory's PSF; CG-SENSE with 30
iterations.

Training (every arithmetic step of the network in the library's kernels): MoDL (Eq. 6) with K
blocks sharing one residual CNN and a learnable lambda, or the VarNet (Eq. 5) with T stages,
Adam on all parameters, a constant learning rate with a tenfold decay over the last quarter of
the steps.  Evaluation: NRMSE = ||x - x_gt|| / ||x_gt|| per held-out slice, averaged, for the
trained network and for plain CG-SENSE ((A^H A + lambda I) x = A^H y by CG from x0 = A^H y) at
the workload's lambda and iteration count, and the best CG-SENSE over a small grid of lambda and
iteration counts chosen on the evaluation slices themselves (which favours CG-SENSE).
"""
from __future__ import annotations

import argparse
import json
import multiprocessing as mp
import os
import time

import numpy as np

CG_LAMBDAS = (0.005, 0.01, 0.02, 0.05, 0.1, 0.2)
CG_ITERS = (10, 30)


# ------------------------------------------------------------------ data (host side)
def _gen(args):
    import synth
    cfg_index, split, idx = args
    d = synth.make_slices(synth.CONFIGS[cfg_index], idx, split=split)
    return (d["x_gt"].astype(np.complex64), d["maps"].astype(np.complex64),
            d["noise"].astype(np.complex64), d["mask"])


def generate(cfg_index: int, split: str, n_slices: int, batch: int, workers: int = 0):
    """Host arrays of n_slices slices in batches of `batch` (a spawn pool: safe after CUDA
    initialisation)."""
    chunks = [(cfg_index, split, list(range(i, min(i + batch, n_slices))))
              for i in range(0, n_slices, batch)]
    workers = workers or min(len(chunks), os.cpu_count() or 1)
    if workers <= 1:
        return [_gen(c) for c in chunks]
    with mp.get_context("spawn").Pool(workers) as pool:
        return pool.map(_gen, chunks)


class Batch:
    """One batch on the device: maps, ground truth, its plan and simulated k-space."""

    def __init__(self, host, device="cuda"):
        import torch
        from .sense import SensePlan
        x_gt, maps, noise, mask = host
        self.gt = torch.from_numpy(x_gt).to(device)
        self.maps = torch.from_numpy(maps).to(device)
        self.mask = torch.from_numpy(mask).to(device)
        self.plan = SensePlan(self.maps, self.mask)
        y = self.plan.forward(self.gt)                       # A x_gt (Eq. 4) by the library
        self.y = y + self.mask * torch.from_numpy(noise).to(device)  # noise where sampled
        self.B = x_gt.shape[0]


class RadialBatch:
    """One batch of radially sampled slices (Sec. 2.3.3): non-Cartesian samples simulated by the
    library's non-uniform DFT, noise at the samples, x^0 = A^H y by the non-uniform adjoint and a
    Toeplitz plan (the trajectory's PSF) for the normal operator."""

    def __init__(self, host, traj, psf, noise_seed: int, sigma: float = 1e-3, device="cuda",
                 normalize: bool = False):
        import torch
        import synth
        from .sense import SensePlan, nudft_adjoint, nudft_forward
        x_gt, maps, _, _ = host
        self.gt = torch.from_numpy(x_gt).to(device)
        self.maps = torch.from_numpy(maps).to(device)
        self.mask = None  # no Cartesian mask: the plan holds the trajectory's PSF
        self.plan = SensePlan.toeplitz(self.maps, psf)
        self.B = x_gt.shape[0]
        M = traj.shape[0]
        noise = synth.complex_noise((self.B, maps.shape[1], M), sigma, np.random.default_rng([11, noise_seed]))
        y = nudft_forward(traj, self.maps, self.gt) + torch.from_numpy(noise.astype(np.complex64)).to(device)
        self.AHy = nudft_adjoint(traj, self.maps, y)
        if normalize:
            # the data scaling of Sec. 2.3.1 (max |x^0| = 1 per slice), target scaled alike: without
            # density compensation x^0 is far larger than x_gt (NRMSE is unchanged by the scaling)
            self.plan.normalize_max(self.AHy, self.gt)


def nrmse_per_slice(x, gt) -> np.ndarray:
    a = x.detach().cpu().numpy().astype(np.complex128)
    b = gt.detach().cpu().numpy().astype(np.complex128)
    return np.linalg.norm((a - b).reshape(a.shape[0], -1), axis=1) / \
        np.linalg.norm(b.reshape(b.shape[0], -1), axis=1)


def cg_sense(batches, lam: float, iters: int) -> np.ndarray:
    """Per-slice NRMSE of plain CG-SENSE from x0 = A^H y."""
    import torch
    out = []
    for b in batches:
        AHy = b.AHy if hasattr(b, "AHy") else b.plan.adjoint(b.y)
        lt = torch.tensor([lam], dtype=torch.float64, device=AHy.device)
        x = b.plan.cg_solve(AHy, lt, iters, x0=AHy)
        out.append(nrmse_per_slice(x, b.gt))
    return np.concatenate(out)


def cg_sense_report(batches, lam: float, iters: int) -> dict:
    at_cfg = float(cg_sense(batches, lam, iters).mean())
    best = (float("inf"), None, None)
    for it in CG_ITERS:
        for lm in CG_LAMBDAS:
            v = float(cg_sense(batches, lm, it).mean())
            if v < best[0]:
                best = (v, lm, it)
    return {"nrmse_cg_sense": at_cfg, "cg_sense_lambda": lam, "cg_sense_iters": iters,
            "nrmse_cg_sense_best": best[0], "cg_sense_best_lambda": best[1],
            "cg_sense_best_iters": best[2]}


# ------------------------------------------------------------------ MoDL
def modl_initial_weights(seed: int, last_scale: float = 0.1):
    """He-normal weights (zero biases) in the library's layout; the last layer is scaled by
    last_scale so that D_W starts close to the identity."""
    import synth
    ws, bs = synth.modl_cnn_weights(seed)
    ws[-1] = ws[-1] * last_scale
    return np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(ws, bs)]).astype(np.float32)


def _schedule(step: int, steps: int, lr: float) -> float:
    return lr if step < int(0.75 * steps) else 0.1 * lr


def _modl_step(tr, b):
    if hasattr(b, "AHy"):
        return tr.train_step_from_adjoint(b.AHy, b.gt)
    return tr.train_step(b.y, b.gt)


def _modl_infer(tr, b):
    if hasattr(b, "AHy"):
        return tr.forward_from_adjoint(b.AHy)
    return tr.forward(b.y)


def train_modl(train, evals, *, K=5, iters=10, lam0=0.05, steps=2000, lr=5e-4, lam_lr=1e-3,
               seed=3, log_every=100, store_activations=True, pre_steps=0) -> dict:
    """pre_steps > 0: the two-step schedule of Sec. 3 (MoDL): the weights and lambda are first
    trained for pre_steps steps with one unrolled block (K = 1), then `steps` steps with K."""
    import torch
    from .modl import ModlTrainer
    w = torch.from_numpy(modl_initial_weights(seed)).cuda()
    b0 = train[0]
    pre_curve = []
    if pre_steps > 0:
        rng0 = np.random.default_rng(seed + 1)
        t1 = ModlTrainer(b0.maps, b0.mask, w, lam0, 1, iters, lr=lr, lam_lr=lam_lr, plan=b0.plan,
                         store_activations=store_activations)
        for step in range(pre_steps):
            b = train[rng0.integers(len(train))]
            t1.use_plan(b.plan)
            t1.lr = _schedule(step, pre_steps, lr)
            t1.lam_lr = _schedule(step, pre_steps, lam_lr)
            loss = _modl_step(t1, b)
            if step % log_every == 0 or step == pre_steps - 1:
                pre_curve.append([step, float(loss.item())])
        lam0 = float(t1.lam.item())
        del t1
    tr = ModlTrainer(b0.maps, b0.mask, w, lam0, K, iters, lr=lr, lam_lr=lam_lr, plan=b0.plan,
                     store_activations=store_activations)

    def evaluate():
        out = []
        for b in evals:
            tr.use_plan(b.plan)
            out.append(nrmse_per_slice(_modl_infer(tr, b), b.gt))
        return float(np.concatenate(out).mean())

    nrmse0 = evaluate()
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(train))
    curve = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(steps):
        if step and step % len(train) == 0:
            order = rng.permutation(len(train))
        b = train[order[step % len(train)]]
        tr.use_plan(b.plan)
        tr.lr = _schedule(step, steps, lr)
        tr.lam_lr = _schedule(step, steps, lam_lr)
        loss = _modl_step(tr, b)
        if step % log_every == 0 or step == steps - 1:
            curve.append([step, float(loss.item())])
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    status = tr.denoiser_status() | tr.plan.status()
    return {"network": "modl", "K": K, "cg_iters": iters, "steps": steps, "lr": lr,
            "pre_steps_k1": pre_steps, "pre_loss_curve": pre_curve,
            "train_batches": len(train), "train_slices": sum(b.B for b in train),
            "eval_slices": sum(b.B for b in evals), "loss_curve": curve,
            "nrmse_untrained": nrmse0, "nrmse_learned": evaluate(),
            "lambda_learned": float(tr.lam.item()), "train_seconds": round(t_train, 2),
            "train_slices_per_s": round(steps * b0.B / t_train, 1), "device_status": status,
            "weights": tr.weights}


# ------------------------------------------------------------------ VarNet
def train_varnet(train, evals, *, steps=2000, lr=5e-4, seed=4, log_every=100, T=10,
                 optimizer="adam", ipalm_tau=(1e-2, 1e-2, 1e-2)) -> dict:
    import torch
    import synth
    from .varnet import VarNetTrainer, pack_params
    filt, rbf, lam = synth.varnet_weights(seed, T)
    prm = torch.from_numpy(pack_params(filt, rbf, lam)).cuda()
    b0 = train[0]
    tr = VarNetTrainer(b0.maps, b0.mask, prm, lr=lr, normalize=True, plan=b0.plan, optimizer=optimizer,
                       ipalm_tau=ipalm_tau)

    def evaluate():
        out = []
        for b in evals:
            tr.use_plan(b.plan)
            x = tr.forward(b.y, b.gt)   # x^T and the target, both scaled to max|x^0| = 1
            out.append(nrmse_per_slice(x, tr.gtn))
        return float(np.concatenate(out).mean())

    nrmse0 = evaluate()
    rng = np.random.default_rng(seed)
    order = rng.permutation(len(train))
    curve = []
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for step in range(steps):
        if step and step % len(train) == 0:
            order = rng.permutation(len(train))
        b = train[order[step % len(train)]]
        tr.use_plan(b.plan)
        tr.lr = _schedule(step, steps, lr)
        loss = tr.train_step(b.y, b.gt)
        if step % log_every == 0 or step == steps - 1:
            curve.append([step, float(loss.item())])
    torch.cuda.synchronize()
    t_train = time.perf_counter() - t0
    if optimizer == "ipalm":
        tr.params.copy_(tr.x)  # evaluate the iterate x^k, not the inertial point
    return {"network": "varnet", "T": T, "steps": steps, "lr": lr, "optimizer": optimizer,
            "ipalm_tau": list(ipalm_tau) if optimizer == "ipalm" else None,
            "train_batches": len(train), "train_slices": sum(b.B for b in train),
            "eval_slices": sum(b.B for b in evals), "loss_curve": curve,
            "nrmse_untrained": nrmse0, "nrmse_learned": evaluate(),
            "train_seconds": round(t_train, 2),
            "train_slices_per_s": round(steps * b0.B / t_train, 1), "device_status": tr.plan.status()}


# ------------------------------------------------------------------ driver
def run(network: str, steps: int, train_slices: int, eval_slices: int, lr: float,
        seed: int, log_every: int = 100, workers: int = 0, pre_steps: int = 0,
        optimizer: str = "adam", ipalm_tau=(1e-2, 1e-2, 1e-2)) -> dict:
    """Generate the data, train, and evaluate against CG-SENSE on the same held-out slices."""
    import synth
    cfg_index = {"modl": 3, "varnet": 4, "modl_radial": 5}[network]
    cfg = synth.CONFIGS[cfg_index]
    bsz = 4  # slices per training batch (the radial workload's inference batch is larger)
    t0 = time.perf_counter()
    host_train = generate(cfg_index, "train", train_slices, bsz, workers)
    host_eval = generate(cfg_index, "eval", eval_slices, bsz, workers)
    t_gen = time.perf_counter() - t0
    if network == "modl_radial":
        import torch
        from .sense import toeplitz_psf
        traj = torch.from_numpy(synth.radial_trajectory(cfg.extra["spokes"], cfg.extra["samples"], cfg.H)
                                .reshape(-1, 2).astype(np.float32)).cuda()
        psf = toeplitz_psf(traj, cfg.H, cfg.W)
        train = [RadialBatch(h, traj, psf, 1000 + i) for i, h in enumerate(host_train)]
        evals = [RadialBatch(h, traj, psf, i) for i, h in enumerate(host_eval)]
        res = train_modl(train, evals, K=cfg.extra["K"], iters=cfg.cg_iters, lam0=cfg.lam, steps=steps,
                         lr=lr, seed=seed, log_every=log_every, pre_steps=pre_steps)
        res.pop("weights")
        res["network"] = "modl_radial"
        res.update(cg_sense_report(evals, cfg.lam, 30))
    elif network == "modl":
        train = [Batch(h) for h in host_train]
        evals = [Batch(h) for h in host_eval]
        res = train_modl(train, evals, K=cfg.extra["K"], iters=cfg.cg_iters, lam0=cfg.lam, steps=steps,
                         lr=lr, seed=seed, log_every=log_every, pre_steps=pre_steps)
        res.pop("weights")
        res.update(cg_sense_report(evals, cfg.lam, cfg.cg_iters))
    else:
        train = [Batch(h) for h in host_train]
        evals = [Batch(h) for h in host_eval]
        res = train_varnet(train, evals, steps=steps, lr=lr, seed=seed, log_every=log_every,
                           T=cfg.extra["T"], optimizer=optimizer, ipalm_tau=ipalm_tau)
        res.update(cg_sense_report(evals, 0.05, 10))
    res["workload"] = cfg.name
    res["data_seconds"] = round(t_gen, 2)
    return res


def main(argv=None):
    ap = argparse.ArgumentParser(description=__doc__.split("\n\n")[0])
    ap.add_argument("--network", choices=["modl", "varnet", "modl_radial"], default="modl")
    ap.add_argument("--steps", type=int, default=2000)
    ap.add_argument("--train-slices", type=int, default=256)
    ap.add_argument("--eval-slices", type=int, default=16)
    ap.add_argument("--lr", type=float, default=5e-4)
    ap.add_argument("--seed", type=int, default=3)
    ap.add_argument("--log-every", type=int, default=100)
    ap.add_argument("--pre-steps", type=int, default=0,
                    help="MoDL: steps with one unrolled block before the K-block training (two-step)")
    ap.add_argument("--optimizer", choices=["adam", "ipalm"], default="adam", help="VarNet optimizer")
    ap.add_argument("--ipalm-tau", type=float, nargs=3, default=(1e-2, 1e-2, 1e-2),
                    metavar=("FILTERS", "RBF", "LAMBDA"), help="iPALM step sizes per block")
    ap.add_argument("--out", default=None, help="write the result as JSON to this file")
    a = ap.parse_args(argv)
    res = run(a.network, a.steps, a.train_slices, a.eval_slices, a.lr, a.seed, a.log_every,
              pre_steps=a.pre_steps, optimizer=a.optimizer, ipalm_tau=tuple(a.ipalm_tau))
    line = json.dumps(res)
    print(line, flush=True)
    if a.out:
        with open(a.out, "w") as f:
            f.write(line + "\n")


if __name__ == "__main__":
    main()
