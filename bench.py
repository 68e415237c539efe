"""Benchmark of the SENSE / CG data-consistency hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]

One step = one batched CG-SENSE reconstruction of the 256x232, 12-coil,
16-slice workload (R = 6 variable-density line mask, lambda = 0.05): x0 = A^H y
(sense_adjoint) followed by 10 CG iterations of (A^H A + lambda I) from x0
(cg_dc_solve), all in libsense kernels.  Inputs are seeded synthetic phantoms,
coil maps and k-space simulated with the library's own forward operator.

Printed (rank 0, one JSON line): slices/s with inputs resident in HBM (value),
the same through host buffers (e2e), the live roofline of the fused
normal-operator kernel (CUDA events around every launch inside the timed
region), the standalone normal-operator bandwidth, clocks sampled during the
timed region, and the FP64 CPU oracle timed on the host cores.
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import subprocess
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "unrolled-recon slices/s (fwd+bwd) & normal-op HBM GB/s vs plain CG-SENSE @NRMSE"
WORKLOAD = "cg_sense_b16_c12_256x232_R6_10it"
# DRAM bytes per launch of the fused CG normal-operator kernel from the committed
# ncu capture (profiles/normal_lines_cg_256x232_b16.md); None until captured for
# the current kernel version.
NCU_TRAFFIC_PER_LAUNCH = None


def peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return 6400.0, "fallback"


# ------------------------------------------------------------------ clocks
class ClockSampler:
    FIELDS = ("clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [p.strip() for p in ln.split(",")]
            if len(parts) < 8:
                continue
            try:
                sm.append(float(parts[0]))
                smax.append(float(parts[1]))
            except ValueError:
                continue
            for n, v in zip(names, parts[4:8]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# ------------------------------------------------------------- workload
def make_inputs(cfg, slice_offset=0):
    import numpy as np
    import synth
    d = synth.make_slices(cfg, range(slice_offset, slice_offset + cfg.B))
    return {"maps": d["maps"].astype(np.complex64), "mask": d["mask"],
            "x_gt": d["x_gt"].astype(np.complex64), "noise": d["noise"].astype(np.complex64)}


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import synth
    from paper_2202_14005_b300.sense import SensePlan

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    cfg = synth.CONFIGS[2]
    inp = make_inputs(cfg, slice_offset=rank * cfg.B)
    maps = torch.from_numpy(inp["maps"]).to(dev)
    mask = torch.from_numpy(inp["mask"]).to(dev)
    plan = SensePlan(maps, mask)
    # k-space simulated by the forward operator: y = A x_gt + M * noise
    y = plan.forward(torch.from_numpy(inp["x_gt"]).to(dev))
    y += torch.from_numpy(inp["noise"]).to(dev) * mask
    lam = torch.tensor([cfg.lam], dtype=torch.float64, device=dev)
    rhs = torch.empty((cfg.B, cfg.H, cfg.W), dtype=torch.complex64, device=dev)
    x = torch.empty_like(rhs)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2

    def step():
        plan.adjoint(y, out=rhs)
        plan.cg_solve(rhs, lam, cfg.cg_iters, x0=rhs, out=x)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    assert plan.status() == 0
    plan.profile_read()

    # ---- timed region (device-resident inputs)
    dist = torch.distributed if world > 1 else None
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    clk = ClockSampler(local_rank)
    clk.start()
    plan.profile(True)
    evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
           for _ in range(args.steps)]
    for i in range(args.steps):
        flush.zero_()  # evict L2 between timed steps (not inside the step's events)
        evs[i][0].record()
        step()
        evs[i][1].record()
    torch.cuda.synchronize()
    clocks = clk.stop()
    normal_ms, normal_n, launches = plan.profile_read()
    plan.profile(False)
    step_ms = [a.elapsed_time(b) for a, b in evs]
    t_ms = sum(step_ms)
    if dist:
        t = torch.tensor([t_ms], device=dev, dtype=torch.float64)
        dist.all_reduce(t, op=dist.ReduceOp.MAX)
        t_ms = float(t.item())
        dist.barrier()
    assert plan.status() == 0

    N = cfg.H * cfg.W
    B, C = cfg.B, cfg.C
    # algorithmic bytes of the timed fused-kernel launches: NM_RESID (x0, rhs, maps,
    # write r) once per step, NM_CG (r, maps, write p, q; plus p_old after iteration 0)
    per_step = 8 * N * B * ((C + 3) + (C + 3) + (cfg.cg_iters - 1) * (C + 4))
    alg_bytes = per_step * args.steps
    achieved = alg_bytes / (normal_ms * 1e-3) / 1e9 if normal_ms > 0 else None
    hbm, src = peaks()

    # ---- standalone normal operator (one launch per flush, CUDA events)
    xin = rhs.clone()
    xout = torch.empty_like(xin)
    nrep = 20
    tn = []
    for _ in range(3):
        plan.normal(xin, cfg.lam, out=xout)
    for _ in range(nrep):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan.normal(xin, cfg.lam, out=xout)
        e1.record()
        torch.cuda.synchronize()
        tn.append(e0.elapsed_time(e1))
    tn_med = statistics.median(tn)
    nbytes = 8 * N * B * (C + 2)
    normal_gbs = nbytes / (tn_med * 1e-3) / 1e9

    # ---- end to end through host buffers: H2D of the step's inputs (k-space and
    # coil maps) from pinned memory, the step, D2H of the reconstruction
    y_h = y.cpu().pin_memory()
    maps_h = maps.cpu().pin_memory()
    x_h = torch.empty(x.shape, dtype=x.dtype).pin_memory()
    e2e = []
    for i in range(max(args.steps // 2, 2) + 1):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        y.copy_(y_h, non_blocking=True)
        maps.copy_(maps_h, non_blocking=True)
        step()
        x_h.copy_(x, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        if i > 0:
            e2e.append(e0.elapsed_time(e1))
    e2e_ms = statistics.mean(e2e)
    h2d = y.numel() * 8 + maps.numel() * 8
    d2h = x.numel() * 8

    # reconstruction quality of this step against the phantoms (NRMSE)
    xr = x.cpu().numpy()
    gt = inp["x_gt"]
    nrmse = float(np.linalg.norm(xr - gt) / np.linalg.norm(gt))

    if rank != 0:
        return None
    value = B * world * args.steps / (t_ms * 1e-3)
    res = {
        "metric": METRIC, "value": round(value, 2), "unit": "slices/s", "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(t_ms / args.steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c64",
        "data": "synthetic (seeded ellipse phantoms, Gaussian coil maps, k-space from the forward operator)",
        "config": {"workload": WORKLOAD, "slices_per_gpu": B, "coils": C, "H": cfg.H, "W": cfg.W,
                   "R": cfg.R, "cg_iters": cfg.cg_iters, "lambda": cfg.lam,
                   "parallelism": f"replicas x{world}", "l2": "flushed (512 MB write) between timed steps"},
        "roofline": {"kernel": "k_normal_lines (CG mode, fused A^H A + lambda I)", "bound": "hbm",
                     "achieved": round(achieved, 1) if achieved else None, "peak": hbm,
                     "peak_source": src, "unit": "GB/s",
                     "frac": round(achieved / hbm, 4) if achieved else None,
                     "traffic": NCU_TRAFFIC_PER_LAUNCH,
                     "launches_timed": normal_n, "avg_launch_us": round(1e3 * normal_ms / max(normal_n, 1), 3),
                     "alg_bytes_per_launch": int(alg_bytes / max(normal_n, 1))},
        "normal_op": {"GB/s": round(normal_gbs, 1), "frac": round(normal_gbs / hbm, 4),
                      "median_us": round(tn_med * 1e3, 2), "alg_bytes": nbytes},
        "e2e": {"value": round(B * world / (e2e_ms * 1e-3), 2), "unit": "slices/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "ms_per_step": round(e2e_ms, 3)},
        "gpu_launches": launches,
        "clocks": clocks,
        "nrmse": {"cg_sense": round(nrmse, 5)},
    }
    return res


# ------------------------------------------------------------ CPU oracle
def _oracle_slice(args):
    """One slice of the workload on the FP64 oracle: A^H y, then 10 CG iterations."""
    os.environ["OMP_NUM_THREADS"] = "1"
    import numpy as np
    import synth
    from oracle import cg as ocg
    from oracle import sense as osense
    cfg_i, s = args
    cfg = synth.CONFIGS[cfg_i]
    d = synth.make_slices(cfg, [s])
    maps = d["maps"].astype(np.complex64)
    mask = d["mask"]
    y = (osense.forward(d["x_gt"], maps, mask) + mask * d["noise"]).astype(np.complex64)
    t0 = time.perf_counter()
    rhs = osense.adjoint(y, maps, mask)
    ocg.cg_solve(maps, mask, cfg.lam, rhs, rhs, cfg.cg_iters)
    return time.perf_counter() - t0


def cpu_baseline(steps=1, slices=None):
    """The oracle as it stands on the host cores: a process pool over slices."""
    import synth
    cfg = synth.CONFIGS[2]
    cores = os.cpu_count() or 1
    n = slices if slices is not None else min(cfg.B, cores)
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=min(n, cores)) as pool:
        pool.map(_oracle_slice, [(2, 0)])  # warm the workers' imports
        walls = []
        for _ in range(steps):
            t0 = time.perf_counter()
            pool.map(_oracle_slice, [(2, s) for s in range(n)])
            walls.append(time.perf_counter() - t0)
    wall = sum(walls)
    return {"value": round(n * steps / wall, 4), "unit": "slices/s", "cores": min(n, cores),
            "kind": "oracle",
            "sample": f"{n} of 16 slices x {steps} step(s) of the workload (A^H y + 10 CG iterations, "
                      f"FP64 NumPy, one process per slice, spawn pool); wall {wall:.1f} s"}


def run_reference(args, rank, world):
    if rank != 0:
        return None
    vals = []
    import synth
    cores = os.cpu_count() or 1
    n = min(synth.CONFIGS[2].B, cores)
    ctx = mp.get_context("spawn")
    with ctx.Pool(processes=n) as pool:
        pool.map(_oracle_slice, [(2, 0)])
        for i in range(args.warmup + args.steps):
            t0 = time.perf_counter()
            pool.map(_oracle_slice, [(2, s) for s in range(n)])
            if i >= args.warmup:
                vals.append(time.perf_counter() - t0)
    wall = sum(vals)
    value = n * len(vals) / wall
    return {"impl": "reference", "metric": METRIC, "value": round(value, 4), "unit": "slices/s",
            "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": round(1e3 * wall / len(vals), 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOAD, "slices_per_step": n},
            "cpu_baseline": {"value": round(value, 4), "unit": "slices/s", "cores": n,
                             "kind": "oracle",
                             "sample": f"{n} of 16 slices per step (FP64 NumPy oracle, spawn pool)"},
            "e2e": {"value": round(value, 4), "unit": "slices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    args = ap.parse_args()
    args.warmup = max(args.warmup, 3) if args.impl == "ours" else args.warmup

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return

    # the oracle's process pool is spawned before the first GPU call
    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(steps=1)

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res = run_ours(args, rank, world, local_rank)
    if res is not None:
        res["cpu_baseline"] = base
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
