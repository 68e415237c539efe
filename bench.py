"""Benchmark of the unrolled-reconstruction hot path on B300.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload modl_train|cg_sense|varnet_train|noncart_modl_infer]

Default step (modl_train): one MoDL training step on 4 slices of 256x232 with
12 coils (R = 6 variable-density line mask): x^0 = A^H y, five unrolled blocks
x^{t+1} = (A^H A + lambda I)^{-1}(A^H y + lambda D_W(x^t)) with 10 CG iterations
each, the MSE loss against the phantoms, the reverse pass through every block
(second CG solve per block, denoiser backward from the activations the forward kept) and
Adam on the 113,155 parameters — every step in libsense kernels (tensor-core
convolutions, fused normal operator, CG vector kernels).

Also measured: plain CG-SENSE on the 16-slice batch (slices/s, NRMSE) and the
standalone normal operator (GB/s).  After the timed region (untimed), MoDL is
trained on operator-simulated slices and evaluated on 16 held-out slices against
plain CG-SENSE on the same slices (nrmse_learned, nrmse_cg_sense).  Inputs are seeded synthetic phantoms, coil
maps and k-space simulated with the library's own forward operator.

Printed (rank 0, one JSON line): slices/s with inputs resident in HBM (value),
the same through host buffers (e2e: for the training workloads each step's inputs
are copied from pinned host memory on a second stream while the previous step runs),
the roofline of the dominant kernel (CUDA events around its launches inside the timed
region), a per-kernel breakdown, clocks sampled during the timed region, and the FP64
CPU oracle timed on the host cores.  The default run also measures the VarNet training
and radial MoDL inference workloads after the headline step (secondary_workloads).
"""
from __future__ import annotations

import argparse
import json
import math
import multiprocessing as mp
import os
import statistics
import sys
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "unrolled-recon slices/s (fwd+bwd) & normal-op HBM GB/s vs plain CG-SENSE @NRMSE"
# Training of the learned reconstruction reported beside the timed step (network, Adam steps,
# learning rate): operator-simulated training slices, evaluated on 16 held-out slices against
# plain CG-SENSE on the same slices (paper_2202_14005_b300.train).
LEARNED = {"modl_train": dict(network="modl", steps=3000, lr=1e-3),
           "varnet_train": dict(network="varnet", steps=3000, lr=5e-4, optimizer="ipalm",
                                ipalm_tau=(1e-2, 1e-2, 1e-1))}

WORKLOADS = {"modl_train": "modl_train_b4_c12_256x232_R6_K5_cg10", "cg_sense": "cg_sense_b16_c12_256x232_R6_10it",
             "varnet_train": "varnet_train_b4_c15_320x368_R4_T10",
             "noncart_modl_infer": "modl_infer_radial_b32_c12_256x256_96x512_K10_cg10"}
# DRAM bytes (read + write) per launch from the committed ncu captures under profiles/, per workload
# (None where no capture of the current kernel version exists for that workload):
# normal_lines a 16-slice residual-mode launch and cg_lines one 16-slice solve (cg_sense); cg_lines
# one 10-iteration solve, conv64_tc a forward launch and wgrad64 one launch of the 4-slice MoDL step;
# vn_* one launch each of the 4-slice 320x368 VarNet step.
# steps of the pipelined end-to-end loop (at least): the first step's input copy overlaps nothing,
# and a training or inference loop runs many steps
E2E_PIPELINED_STEPS = 30
# the HBM denominator the project statement quotes for the operator's roofline fraction
NOMINAL_HBM_GBS = 8000.0
NCU_TRAFFIC = {
    "cg_sense": {"normal_lines": 102.8e6, "cg_lines": 1.527e9},
    "modl_train": {"cg_lines": 26.7e6, "conv64_tc": 30.52e6, "wgrad64": 61.3e6},
    "varnet_train": {"vn_K": 31.18e6, "vn_KT": 41.5e6, "vn_wgrad": 70.9e6},
    # one Toeplitz application: its three passes (rows 567 MB, columns 754 MB, inverse rows 633 MB)
    "noncart_modl_infer": {"toeplitz": 1.955e9},
}
# what the reverse pass reuses from the forward pass of each training workload
REVERSE_PASS = {
    "modl_train": "each block's denoiser activations kept from the forward pass (no recompute)",
    "varnet_train": "each stage's K x and Phi'(K x) kept from the forward pass (K g alone recomputed)",
}
# kernel groups the library times with CUDA events when profiling is on
PROFILE_GROUPS = ("normal_lines", "conv64_tc", "wgrad64", "cg_vec", "fft_generic", "dn_2to64", "dn_64to2",
                  "dn_wgrad_small", "dn_reduce", "dn_pack", "unrolled_misc", "vn_K", "vn_Kbwd", "vn_KT",
                  "vn_wgrad", "vn_rbfgrad", "vn_misc", "toeplitz", "adjoint_lines", "cg_lines")


# ------------------------------------------------------------------ clocks
class _Nvml:
    """Read-only NVML queries through ctypes on the driver's libnvidia-ml (no Python binding
    needed): SM clock, its maximum and the clock-event reason bits of one device."""
    SM = 1  # NVML_CLOCK_SM
    REASONS = (("sw_power_cap", 0x4), ("hw_slowdown", 0x8), ("sw_thermal_slowdown", 0x20),
               ("hw_thermal_slowdown", 0x40))

    def __init__(self, pci: str | None, index: int):
        import ctypes as C
        self.C = C
        self.lib = C.CDLL("libnvidia-ml.so.1")
        if self.lib.nvmlInit_v2() != 0:
            raise RuntimeError("nvmlInit failed")
        self.h = C.c_void_p()
        rc = (self.lib.nvmlDeviceGetHandleByPciBusId_v2(pci.encode(), C.byref(self.h)) if pci
              else self.lib.nvmlDeviceGetHandleByIndex_v2(C.c_uint(index), C.byref(self.h)))
        if rc != 0:
            raise RuntimeError(f"no NVML device handle ({rc})")

    def _uint(self, fn, *args):
        v = self.C.c_uint()
        if fn(self.h, *args, self.C.byref(v)) != 0:
            raise RuntimeError("NVML query failed")
        return v.value

    def sm_mhz(self):
        return self._uint(self.lib.nvmlDeviceGetClockInfo, self.C.c_int(self.SM))

    def sm_max_mhz(self):
        return self._uint(self.lib.nvmlDeviceGetMaxClockInfo, self.C.c_int(self.SM))

    def reasons(self):
        v = self.C.c_ulonglong()
        if self.lib.nvmlDeviceGetCurrentClocksEventReasons(self.h, self.C.byref(v)) != 0:
            raise RuntimeError("NVML query failed")
        return [name for name, bit in self.REASONS if v.value & bit]

    def close(self):
        self.lib.nvmlShutdown()


class ClockSampler:
    """SM clock and clock-event reasons of one GPU, polled through NVML (read-only queries)
    every 5 ms from a background thread while the timed region runs."""

    def __init__(self, index: int):
        self.index = index  # CUDA device index; matched to the NVML device by PCI address
        self.pci = None
        try:
            import torch
            pr = torch.cuda.get_device_properties(index)
            self.pci = f"{pr.pci_domain_id:08x}:{pr.pci_bus_id:02x}:{pr.pci_device_id:02x}.0"
        except Exception:
            pass
        self.sm, self.reasons, self.smax = [], set(), None
        self.stop_evt = threading.Event()
        self.err = None

    def _poll(self):
        try:
            nv = _Nvml(self.pci, self.index)
            self.smax = nv.sm_max_mhz()
            while not self.stop_evt.is_set():
                self.sm.append(nv.sm_mhz())
                self.reasons.update(nv.reasons())
                time.sleep(0.005)
            nv.close()
        except Exception as e:  # NVML unavailable: no samples
            self.err = str(e)

    def start(self):
        self.stop_evt.clear()
        self.t = threading.Thread(target=self._poll, daemon=True)
        self.t.start()
        time.sleep(0.02)

    def stop(self):
        self.stop_evt.set()
        self.t.join(timeout=5)
        if not self.sm:
            return {"sm_mhz": None, "sm_max_mhz": self.smax, "reasons": [f"no samples: {self.err}"],
                    "samples": 0}
        return {"sm_mhz": statistics.median(self.sm), "sm_max_mhz": self.smax,
                "reasons": sorted(self.reasons), "samples": len(self.sm), "source": "nvml"}


# ------------------------------------------------------------- replicas
# Slices are independent (one CG per slice, per-slice scalars), so N GPUs run N replicas on
# disjoint slice ranges; the only exchange is the max of the timed region over ranks.
def replica_slice_offset(rank, slices_per_rank):
    """First seeded slice of this rank: rank r takes slices r*B .. r*B + B - 1."""
    return rank * slices_per_rank


def max_over_ranks(t_ms, dist, device):
    """The job's time is the slowest rank's (all-reduce MAX of one double)."""
    if not dist:
        return t_ms
    import torch
    t = torch.tensor([t_ms], device=device, dtype=torch.float64)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def whole_job_value(slices_per_rank, world, steps, t_ms):
    """Aggregate slices/s over all ranks for `steps` steps that took t_ms (max over ranks)."""
    return slices_per_rank * world * steps / (t_ms * 1e-3)


# ------------------------------------------------------------- workload
def make_inputs(cfg, slice_offset=0):
    import numpy as np
    import synth
    d = synth.make_slices(cfg, range(slice_offset, slice_offset + cfg.B))
    return {"maps": d["maps"].astype(np.complex64), "mask": d["mask"],
            "x_gt": d["x_gt"].astype(np.complex64), "noise": d["noise"].astype(np.complex64)}


def fp32_peak_tflops(sm_mhz):
    """FP32 FMA peak: 148 SMs x 128 lanes x 2 flop x clock (B300)."""
    return 148 * 128 * 2 * (sm_mhz or 2032.0) * 1e6 / 1e12


def measure_fp32_peak(dev, reps=5):
    """FP32 FMA peak of this GPU, measured: the library's register-only FMA probe (8 blocks of
    256 threads per SM, 8 independent chains per thread) timed with CUDA events; best of reps.
    Returns (TFLOP/s, median SM MHz sampled while it ran)."""
    import torch
    from paper_2202_14005_b300 import _lib
    import ctypes as C
    blocks, iters = 148 * 8, 20000
    flops = 2.0 * 8 * 256 * iters * blocks
    sink = torch.zeros(blocks, dtype=torch.float32, device=dev)
    st = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    L = _lib.lib()
    _lib.check("sense_fma_probe", L.sense_fma_probe(blocks, 100, C.c_void_p(sink.data_ptr()), st))
    clk = ClockSampler(dev.index or 0)
    clk.start()
    best = float("inf")
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        _lib.check("sense_fma_probe", L.sense_fma_probe(blocks, iters, C.c_void_p(sink.data_ptr()), st))
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    c = clk.stop()
    return flops / (best * 1e-3) / 1e12, c.get("sm_mhz")


def kernel_report(name, ms, n, alg, peaks_d, clocks, workload, alu_flops=None):
    """Achieved vs peak for one kernel group; alg = (kind, amount per launch).  alu_flops: FP32
    FLOPs per launch of the kernel's arithmetic, reported against the measured FP32 peak."""
    if n == 0 or ms <= 0:
        return None
    kind, per = alg
    t = ms * 1e-3 / n
    if kind == "hbm":
        ach = per / t / 1e9
        peak, unit = peaks_d["hbm_gbs"], "GB/s"
    elif kind == "tensor":
        ach = per / t / 1e12
        peak, unit = peaks_d["bf16_tflops_sustained"], "TFLOP/s"
    else:  # alu (FP32 FMA)
        ach = per / t / 1e12
        peak, unit = fp32_peak_tflops(clocks.get("sm_max_mhz")), "TFLOP/s"
    rep = {"kernel": name, "bound": kind, "achieved": round(ach, 2), "peak": round(peak, 1),
           "unit": unit, "frac": round(ach / peak, 4), "traffic": NCU_TRAFFIC.get(workload, {}).get(name),
           "launches": n, "avg_launch_us": round(1e3 * ms / n, 3), "alg_per_launch": per}
    if kind == "hbm":  # also against the 8 TB/s denominator the project statement quotes
        rep["frac_of_8tbs"] = round(ach / NOMINAL_HBM_GBS, 4)
    if alu_flops and peaks_d.get("fp32_tflops"):
        a = alu_flops / t / 1e12
        rep["alu"] = {"achieved": round(a, 2), "peak": round(peaks_d["fp32_tflops"], 1), "unit": "TFLOP/s",
                      "frac": round(a / peaks_d["fp32_tflops"], 4), "flop_per_launch": alu_flops,
                      "peak_source": "measured FP32 FMA probe"}
    return rep


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            d = json.load(f)
        return {"hbm_gbs": float(d["hbm_gbs"]), "bf16_tflops": float(d["bf16_tflops"]),
                "bf16_tflops_sustained": float(d["bf16_tflops_sustained"]), "source": "measured"}
    except Exception:
        return {"hbm_gbs": 6400.0, "bf16_tflops": 1800.0, "bf16_tflops_sustained": 1400.0,
                "source": "fallback"}


# --profile-step: the workload whose step is run once inside a CUDA profiler range (cudaProfilerStart
# / Stop) after its warm-up, for `ncu --profile-from-start off`; the process then exits
PROFILE_STEP = None


def timed_steps(step, steps, flush, dist, name=None):
    import torch
    from paper_2202_14005_b300 import _lib
    if PROFILE_STEP is not None and name == PROFILE_STEP:
        torch.cuda.synchronize()
        flush.zero_()
        torch.cuda.synchronize()
        torch.cuda.profiler.start()
        step()
        torch.cuda.synchronize()
        torch.cuda.profiler.stop()
        print(json.dumps({"profile_step": name, "status": "one step run inside the profiler range"}), flush=True)
        sys.exit(0)
    def run(profiled):
        # profiled: the library records a CUDA-event pair around every kernel group on the stream
        # it launches on (per-kernel durations for the roofline); those records add to the step's
        # own timeline, so the step time is taken from a pass without them
        if dist:
            dist.barrier()
        torch.cuda.synchronize()
        _lib.kernel_launches(reset=True)
        for k in PROFILE_GROUPS:
            _lib.profile_read(k)
        _lib.profile_enable(profiled)
        evs = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        for i in range(steps):
            flush.zero_()  # evict L2 between timed steps (outside the step's events)
            evs[i][0].record()
            step()
            evs[i][1].record()
        torch.cuda.synchronize()
        _lib.profile_enable(False)
        prof = {k: _lib.profile_read(k) for k in PROFILE_GROUPS}
        launches = _lib.kernel_launches(reset=True)
        return sum(a.elapsed_time(b) for a, b in evs), prof, launches

    run(True)                                   # the library creates its events on first use
    t_prof, prof, _ = run(True)                 # per-kernel durations, every event already created
    t_ms, _, launches = run(False)              # the step time
    return t_ms, prof, launches, t_prof


def run_ours(args, rank, world, local_rank):
    import numpy as np
    import torch
    import synth
    from paper_2202_14005_b300.sense import SensePlan
    from paper_2202_14005_b300.modl import ModlTrainer

    torch.cuda.set_device(local_rank)
    dev = torch.device("cuda", local_rank)
    dist = torch.distributed if world > 1 else None
    pk = load_peaks()
    pk["fp32_tflops"], pk["fp32_probe_sm_mhz"] = measure_fp32_peak(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)  # 512 MB > L2
    clk = ClockSampler(local_rank)
    res = {}

    # ---------------- plain CG-SENSE on the 16-slice batch (secondary, or main)
    c2 = synth.CONFIGS[2]
    inp2 = make_inputs(c2, slice_offset=replica_slice_offset(rank, c2.B))
    maps2 = torch.from_numpy(inp2["maps"]).to(dev)
    mask2 = torch.from_numpy(inp2["mask"]).to(dev)
    plan2 = SensePlan(maps2, mask2)
    y2 = plan2.forward(torch.from_numpy(inp2["x_gt"]).to(dev))
    y2 += torch.from_numpy(inp2["noise"]).to(dev) * mask2
    lam2 = torch.tensor([c2.lam], dtype=torch.float64, device=dev)
    rhs2 = torch.empty((c2.B, c2.H, c2.W), dtype=torch.complex64, device=dev)
    x2 = torch.empty_like(rhs2)

    def step_cg():
        plan2.adjoint(y2, out=rhs2)
        plan2.cg_solve(rhs2, lam2, c2.cg_iters, x0=rhs2, out=x2)

    for _ in range(args.warmup):
        step_cg()
    torch.cuda.synchronize()
    steps_cg = args.steps if args.workload == "cg_sense" else max(5, args.steps // 2)
    if args.workload == "cg_sense":
        clk.start()
    t_cg, prof_cg, launches_cg, t_cg_prof = timed_steps(step_cg, steps_cg, flush, dist, "cg_sense")
    if args.workload == "cg_sense":
        clocks = clk.stop()
    assert plan2.status() == 0
    gt2 = inp2["x_gt"]
    nrmse_cg = float(np.linalg.norm(x2.cpu().numpy() - gt2) / np.linalg.norm(gt2))
    N = c2.H * c2.W
    # standalone normal operator, one launch per L2 flush
    xin, xout = rhs2.clone(), torch.empty_like(rhs2)
    for _ in range(3):
        plan2.normal(xin, c2.lam, out=xout)
    tn = []
    for _ in range(20):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan2.normal(xin, c2.lam, out=xout)
        e1.record()
        torch.cuda.synchronize()
        tn.append(e0.elapsed_time(e1))
    tn_med = statistics.median(tn)
    nbytes = 8 * N * c2.B * (c2.C + 2)
    res["normal_op"] = {"workload": "256x232, 12 coils, 16 slices, lambda I", "GB/s": round(nbytes / (tn_med * 1e-3) / 1e9, 1),
                        "frac": round(nbytes / (tn_med * 1e-3) / 1e9 / pk["hbm_gbs"], 4),
                        "frac_of_8tbs": round(nbytes / (tn_med * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 4),
                        "median_us": round(tn_med * 1e3, 2), "alg_bytes": nbytes,
                        "alu": {"flop": 154.0 * N * c2.B * c2.C,
                                "TFLOP/s": round(154.0 * N * c2.B * c2.C / (tn_med * 1e-3) / 1e12, 2),
                                "frac": round(154.0 * N * c2.B * c2.C / (tn_med * 1e-3) / 1e12 / pk["fp32_tflops"], 4),
                                "peak_tflops": round(pk["fp32_tflops"], 1)}}
    # soft-SENSE normal operator (two map sets, Sec. 2.3.3) on the same batch: fused line kernel
    maps_s = torch.stack([maps2, 0.6 * torch.roll(maps2, 1, dims=1)], dim=1).contiguous()
    plan_s = SensePlan(maps_s, mask2)
    xs_in = torch.stack([rhs2, 0.5 * rhs2], dim=1).contiguous()
    xs_out = torch.empty_like(xs_in)
    for _ in range(3):
        plan_s.normal(xs_in, c2.lam, out=xs_out)
    ts = []
    for _ in range(20):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan_s.normal(xs_in, c2.lam, out=xs_out)
        e1.record()
        torch.cuda.synchronize()
        ts.append(e0.elapsed_time(e1))
    ts_med = statistics.median(ts)
    sbytes = 8 * N * c2.B * (2 * c2.C + 4)
    res["soft_sense_normal_op"] = {"workload": "256x232, 12 coils x 2 map sets, 16 slices, lambda I",
                                   "GB/s": round(sbytes / (ts_med * 1e-3) / 1e9, 1),
                                   "frac": round(sbytes / (ts_med * 1e-3) / 1e9 / pk["hbm_gbs"], 4),
                                   "frac_of_8tbs": round(sbytes / (ts_med * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 4),
                                   "median_us": round(ts_med * 1e3, 2), "alg_bytes": sbytes}
    del plan_s, maps_s
    # general 2-D mask (variable-density random sampling of the whole k-space plane, same
    # acceleration and fully sampled centre as the line mask): generic row / column transforms
    rng2 = np.random.default_rng(7)
    H2, W2 = c2.H, c2.W
    ky = (np.arange(H2) - H2 / 2) / (H2 / 2)
    kx = (np.arange(W2) - W2 / 2) / (W2 / 2)
    dens = np.exp(-(ky[:, None] ** 2 + kx[None, :] ** 2) / 0.18)
    dens *= (H2 * W2 / c2.R) / dens.sum()
    m2d = (rng2.uniform(size=(H2, W2)) < np.minimum(dens, 1.0)).astype(np.float32)
    m2d[H2 // 2 - 12:H2 // 2 + 12, W2 // 2 - 12:W2 // 2 + 12] = 1.0
    plan_2d = SensePlan(maps2, torch.from_numpy(m2d).to(dev))
    for _ in range(3):
        plan_2d.normal(xin, c2.lam, out=xout)
    t2d = []
    for _ in range(10):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        plan_2d.normal(xin, c2.lam, out=xout)
        e1.record()
        torch.cuda.synchronize()
        t2d.append(e0.elapsed_time(e1))
    t2d_med = statistics.median(t2d)
    b2d = 8 * N * c2.B * (c2.C + 2)
    res["normal_op_2d_mask"] = {"workload": f"256x232, 12 coils, 16 slices, 2-D mask ({m2d.mean():.3f} sampled), lambda I",
                                "GB/s": round(b2d / (t2d_med * 1e-3) / 1e9, 1),
                                "frac": round(b2d / (t2d_med * 1e-3) / 1e9 / pk["hbm_gbs"], 4),
                                "frac_of_8tbs": round(b2d / (t2d_med * 1e-3) / 1e9 / NOMINAL_HBM_GBS, 4),
                                "median_us": round(t2d_med * 1e3, 2), "alg_bytes": b2d,
                                "path": "generic row/column transforms (coil images through HBM)"}
    del plan_2d
    res["cg_sense"] = {"workload": WORKLOADS["cg_sense"], "slices_per_s": round(c2.B * world * steps_cg / (t_cg * 1e-3), 1),
                       "ms_per_step": round(t_cg / steps_cg, 4), "nrmse": round(nrmse_cg, 5)}

    cg_bytes = None  # algorithmic bytes of one whole-solve CG launch (line-mask workloads)
    pipe = None      # (device buffer sets, host inputs, step(k), result read back) for the pipelined e2e
    if args.workload == "cg_sense":
        cfg, B, t_ms, prof, launches, steps, t_prof = c2, c2.B, t_cg, prof_cg, launches_cg, steps_cg, t_cg_prof
        # initial residual (normal operator, maps + x + rhs + out) and the one-launch CG solve:
        # per iteration the normal operator (maps, r, p_old, p, q) and the update (p, q, x, r; x, r)
        # algorithmic bytes per unit (one slice): normal operator 8 N (C + 2) (read x and the
        # maps, write out), one CG iteration 8 N (C + 8) (the operator plus six vector passes)
        normal_bytes = 8 * N * c2.B * (c2.C + 2)
        cg_bytes = 8 * N * c2.B * (c2.C + 8) * c2.cg_iters
        # e2e through host buffers: k-space and maps in, reconstruction out
        y_h, maps_h = y2.cpu().pin_memory(), maps2.cpu().pin_memory()
        out_h = torch.empty(x2.shape, dtype=x2.dtype).pin_memory()
        ins = [(y2, y_h), (maps2, maps_h)]
        outs = [(out_h, x2)]
        step_fn = step_cg
        value_slices = B
    elif args.workload == "noncart_modl_infer":
        # Sec. 2.3.3: radial sampling, A^H A through the Toeplitz embedding (PSF on the 2x grid,
        # computed on the GPU from the trajectory); the radial samples are simulated with the
        # non-uniform DFT plus noise at the samples, and x^0 = A^H y (their non-uniform adjoint) is
        # precomputed, as in the paper; MoDL inference with K = 10 blocks of the config-3 CNN and
        # 10 CG iterations each (timed); plain 30-iteration CG-SENSE measured beside it.
        from paper_2202_14005_b300.sense import nudft_adjoint, nudft_forward, toeplitz_psf
        c5 = synth.CONFIGS[5]
        cfg = c5
        inp5 = make_inputs(c5, slice_offset=replica_slice_offset(rank, c5.B))
        maps5 = torch.from_numpy(inp5["maps"]).to(dev)
        traj = synth.radial_trajectory(c5.extra["spokes"], c5.extra["samples"], c5.H).reshape(-1, 2)
        traj_d = torch.from_numpy(traj.astype(np.float32)).to(dev)
        psf = toeplitz_psf(traj_d, c5.H, c5.W)
        plan5 = SensePlan.toeplitz(maps5, psf)
        gt5 = torch.from_numpy(inp5["x_gt"]).to(dev)
        y5 = nudft_forward(traj_d, maps5, gt5)
        noise5 = synth.complex_noise(tuple(y5.shape), 1e-3, np.random.default_rng([11, 5000 + rank]))
        y5 += torch.from_numpy(noise5.astype(np.complex64)).to(dev)
        AHy5 = nudft_adjoint(traj_d, maps5, y5)
        ws, bs = synth.modl_cnn_weights(5000 + rank)
        flat = np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(ws, bs)]).astype(np.float32)
        tr = ModlTrainer(maps5, None, torch.from_numpy(flat).to(dev), c5.lam, c5.extra["K"], c5.cg_iters,
                         plan=plan5, store_activations=False)  # inference: no reverse pass

        def step_nc():
            tr.forward_from_adjoint(AHy5)

        for _ in range(args.warmup):
            step_nc()
        torch.cuda.synchronize()
        assert plan5.status() == 0 and tr.denoiser_status() == 0
        steps = args.steps
        clk.start()
        t_ms, prof, launches, t_prof = timed_steps(step_nc, steps, flush, dist, "noncart_modl_infer")
        clocks = clk.stop()
        assert plan5.status() == 0 and tr.denoiser_status() == 0
        B = c5.B
        N5 = c5.H * c5.W
        normal_bytes = 8 * N5 * B * (c5.C + 2)
        gt_np = inp5["x_gt"]
        nrmse_modl = float(np.linalg.norm(tr.xs[-1].cpu().numpy() - gt_np) / np.linalg.norm(gt_np))
        # plain CG-SENSE, 30 iterations from x^0 = A^H y
        lam5 = torch.tensor([c5.lam], dtype=torch.float64, device=dev)
        xcg = torch.empty_like(AHy5)
        plan5.cg_solve(AHy5, lam5, 30, x0=AHy5, out=xcg)
        torch.cuda.synchronize()
        tc = []
        for _ in range(3):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan5.cg_solve(AHy5, lam5, 30, x0=AHy5, out=xcg)
            e1.record()
            torch.cuda.synchronize()
            tc.append(e0.elapsed_time(e1))
        nrmse_cg = float(np.linalg.norm(xcg.cpu().numpy() - gt_np) / np.linalg.norm(gt_np))
        # standalone Toeplitz normal operator
        tn5 = []
        xo5 = torch.empty_like(AHy5)
        for _ in range(10):
            flush.zero_()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            plan5.normal(AHy5, c5.lam, out=xo5)
            e1.record()
            torch.cuda.synchronize()
            tn5.append(e0.elapsed_time(e1))
        tn5m = statistics.median(tn5)
        res["noncart"] = {"toeplitz_normal_op": {"GB/s": round(normal_bytes / (tn5m * 1e-3) / 1e9, 1),
                                                 "median_us": round(tn5m * 1e3, 1), "alg_bytes": normal_bytes},
                          "cg_sense_30it": {"slices_per_s": round(B * world / (statistics.median(tc) * 1e-3), 1),
                                            "nrmse": round(nrmse_cg, 5)},
                          "modl_untrained_nrmse": round(nrmse_modl, 5),
                          "data": "x^0 = A^H y of radial samples simulated by the non-uniform DFT, noise sigma 1e-3"}
        y_h, maps_h = AHy5.cpu().pin_memory(), maps5.cpu().pin_memory()
        out_h = torch.empty(tr.xs[-1].shape, dtype=tr.xs[-1].dtype).pin_memory()
        ins = [(AHy5, y_h), (maps5, maps_h)]
        outs = [(out_h, tr.xs[-1])]
        step_fn = step_nc
        # a second device buffer set (and Toeplitz plan, same PSF) for the pipelined end-to-end
        # loop: the next batch's x^0 and maps are copied in while this one is reconstructed
        bufs = [(AHy5, maps5), (torch.empty_like(AHy5), torch.empty_like(maps5))]
        plans = [plan5, SensePlan.toeplitz(bufs[1][1], psf)]

        def step_buf_nc(k):
            tr.use_plan(plans[k])
            tr.forward_from_adjoint(bufs[k][0])
        pipe = (bufs, (y_h, maps_h), step_buf_nc, lambda: tr.xs[-1])
        value_slices = B
    elif args.workload == "varnet_train":
        from paper_2202_14005_b300.varnet import VarNetTrainer, pack_params
        c4 = synth.CONFIGS[4]
        cfg = c4
        inp4 = make_inputs(c4, slice_offset=replica_slice_offset(rank, c4.B))
        maps4 = torch.from_numpy(inp4["maps"]).to(dev)
        mask4 = torch.from_numpy(inp4["mask"]).to(dev)
        filt, rbfw, lamv = synth.varnet_weights(4000 + rank, c4.extra["T"])
        vec = torch.from_numpy(pack_params(filt, rbfw, lamv)).to(dev)
        tr = VarNetTrainer(maps4, mask4, vec, lr=1e-4, normalize=True)
        gt4 = torch.from_numpy(inp4["x_gt"]).to(dev)
        y4 = tr.plan.forward(gt4)
        y4 += torch.from_numpy(inp4["noise"]).to(dev) * mask4

        def step_vn():
            tr.train_step(y4, gt4)

        for _ in range(args.warmup):
            step_vn()
        torch.cuda.synchronize()
        assert tr.plan.status() == 0
        steps = args.steps
        clk.start()
        t_ms, prof, launches, t_prof = timed_steps(step_vn, steps, flush, dist, "varnet_train")
        clocks = clk.stop()
        assert tr.plan.status() == 0
        B = c4.B
        N4 = c4.H * c4.W
        normal_bytes = 8 * N4 * B * (c4.C + 2)
        y_h, maps_h, gt_h = y4.cpu().pin_memory(), maps4.cpu().pin_memory(), gt4.cpu().pin_memory()
        out_h = torch.empty(1, dtype=torch.float64).pin_memory()
        ins = [(y4, y_h), (maps4, maps_h), (gt4, gt_h)]
        outs = [(out_h, tr.loss)]
        step_fn = step_vn
        # a second device buffer set (and plan) for the pipelined end-to-end loop
        bufs = [(y4, maps4, gt4), (torch.empty_like(y4), torch.empty_like(maps4), torch.empty_like(gt4))]
        plans = [tr.plan, SensePlan(bufs[1][1], mask4)]

        def step_buf(k):
            tr.use_plan(plans[k])
            tr.train_step(bufs[k][0], bufs[k][2])
        pipe = (bufs, (y_h, maps_h, gt_h), step_buf, lambda: tr.loss)
        value_slices = B
        gtn = tr.gtn.cpu().numpy()
        res["varnet"] = {"loss_last_step": float(tr.loss.item()), "data_scaling": "max|x^0| = 1 per slice",
                         "nrmse_untrained_forward": round(float(np.linalg.norm(tr.xs[-1].cpu().numpy() - gtn)
                                                                / np.linalg.norm(gtn)), 5)}
    else:
        c3 = synth.CONFIGS[3]
        cfg = c3
        inp3 = make_inputs(c3, slice_offset=replica_slice_offset(rank, c3.B))
        maps3 = torch.from_numpy(inp3["maps"]).to(dev)
        mask3 = torch.from_numpy(inp3["mask"]).to(dev)
        ws, bs = synth.modl_cnn_weights(3000 + rank)
        flat = np.concatenate([np.concatenate([w.ravel(), b]) for w, b in zip(ws, bs)]).astype(np.float32)
        tr = ModlTrainer(maps3, mask3, torch.from_numpy(flat).to(dev), c3.lam, c3.extra["K"], c3.cg_iters,
                         lr=1e-4, lam_lr=1e-4)
        gt3 = torch.from_numpy(inp3["x_gt"]).to(dev)
        y3 = tr.plan.forward(gt3)
        y3 += torch.from_numpy(inp3["noise"]).to(dev) * mask3

        def step_modl():
            tr.train_step(y3, gt3)

        for _ in range(args.warmup):
            step_modl()
        torch.cuda.synchronize()
        assert tr.plan.status() == 0 and tr.denoiser_status() == 0
        steps = args.steps
        clk.start()
        t_ms, prof, launches, t_prof = timed_steps(step_modl, steps, flush, dist, "modl_train")
        clocks = clk.stop()
        assert tr.plan.status() == 0 and tr.denoiser_status() == 0
        B = c3.B
        N3 = c3.H * c3.W
        normal_bytes = 8 * N3 * B * (c3.C + 2)
        cg_bytes = 8 * N3 * B * (c3.C + 8) * c3.cg_iters
        y_h, maps_h, gt_h = y3.cpu().pin_memory(), maps3.cpu().pin_memory(), gt3.cpu().pin_memory()
        out_h = torch.empty(1, dtype=torch.float64).pin_memory()
        ins = [(y3, y_h), (maps3, maps_h), (gt3, gt_h)]
        outs = [(out_h, tr.loss)]
        step_fn = step_modl
        # a second device buffer set (and plan) for the pipelined end-to-end loop
        bufs = [(y3, maps3, gt3), (torch.empty_like(y3), torch.empty_like(maps3), torch.empty_like(gt3))]
        plans = [tr.plan, SensePlan(bufs[1][1], mask3)]

        def step_buf(k):
            tr.use_plan(plans[k])
            tr.train_step(bufs[k][0], bufs[k][2])
        pipe = (bufs, (y_h, maps_h, gt_h), step_buf, lambda: tr.loss)
        value_slices = B
        res["modl"] = {"loss_last_step": float(tr.loss.item()),
                       "nrmse_untrained_forward": round(float(np.linalg.norm(tr.xs[-1].cpu().numpy() - inp3["x_gt"])
                                                              / np.linalg.norm(inp3["x_gt"])), 5)}

    t_ms = max_over_ranks(t_ms, dist, dev)

    # per-kernel roofline inside the timed region
    Hc, Wc = cfg.H, cfg.W
    px = B * Hc * Wc
    conv_flops = 2.0 * px * 64 * 576
    vn_flops = 2.0 * px * 24 * 2 * 121  # one 2<->24 channel 11x11 convolution
    vn_store = bool(getattr(tr, "store", False)) if args.workload == "varnet_train" else False
    # FP32 arithmetic per application: the line path's ~154 FLOP per pixel and coil (two pruned
    # row transforms, coil expand and combine); the Toeplitz path's two 2H x 2W FFTs per coil
    # (5 n log2 n FLOP each)
    line_flops = 154.0 * px * cfg.C
    n4 = 4 * Hc * Wc
    tp_flops = 2 * 5.0 * n4 * math.log2(n4) * B * cfg.C
    kern = {
        "normal_lines": kernel_report("normal_lines", *prof["normal_lines"], ("hbm", normal_bytes), pk, clocks,
                                      args.workload, alu_flops=line_flops),
        "cg_lines": kernel_report("cg_lines", *prof["cg_lines"], ("hbm", cg_bytes), pk, clocks, args.workload,
                                  alu_flops=line_flops * cfg.cg_iters)
        if cg_bytes else None,
        "conv64_tc": kernel_report("conv64_tc", *prof["conv64_tc"], ("tensor", conv_flops), pk, clocks, args.workload),
        "wgrad64": kernel_report("wgrad64", *prof["wgrad64"], ("tensor", conv_flops), pk, clocks, args.workload),
        "vn_K": kernel_report("vn_K", *prof["vn_K"], ("tensor", vn_flops), pk, clocks, args.workload),
        # reverse K: K g alone when the forward's K x is kept, else K x and K g
        "vn_Kbwd": kernel_report("vn_Kbwd", *prof["vn_Kbwd"], ("tensor", (1 if vn_store else 2) * vn_flops), pk,
                                 clocks, args.workload),
        "vn_KT": kernel_report("vn_KT", *prof["vn_KT"], ("tensor", vn_flops), pk, clocks, args.workload),
        "vn_wgrad": kernel_report("vn_wgrad", *prof["vn_wgrad"], ("tensor", 2 * vn_flops), pk, clocks, args.workload),
        "toeplitz": kernel_report("toeplitz", *prof["toeplitz"], ("hbm", normal_bytes), pk, clocks, args.workload,
                                  alu_flops=tp_flops),
    }
    kern = {k: v for k, v in kern.items() if v}
    total_kernel_ms = {k: prof[k][0] for k in prof}
    breakdown = {k: {"ms_per_step": round(prof[k][0] / steps, 4), "launches_per_step": prof[k][1] // max(steps, 1),
                     "share": round(prof[k][0] / t_prof, 4)} for k in PROFILE_GROUPS if prof[k][1]}
    dominant = max(kern, key=lambda k: total_kernel_ms[k]) if kern else None
    for k in kern:
        kern[k]["share_of_step"] = round(total_kernel_ms[k] / t_prof, 4)

    # end to end through host buffers (pinned), step inputs in and result out, as a user calls it
    # (without the per-kernel events, like the step time)
    from paper_2202_14005_b300 import _lib as _l
    e2e = []
    for i in range(max(args.steps // 2, 2) + 1):
        flush.zero_()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        for d, h in ins:
            d.copy_(h, non_blocking=True)
        step_fn()
        for h, d in outs:
            h.copy_(d, non_blocking=True)
        e1.record()
        torch.cuda.synchronize()
        if i > 0:
            e2e.append(e0.elapsed_time(e1))
    e2e_ms = statistics.mean(e2e)
    e2e_mode = "serial: copy in, step, read back"
    if pipe is not None:
        n_pipe = max(args.steps, E2E_PIPELINED_STEPS)
        ms_p = e2e_pipelined(*pipe, n_pipe, flush)
        if ms_p < e2e_ms:
            e2e_ms = ms_p
            e2e_mode = (f"pipelined over {n_pipe} steps: each step's inputs copied from pinned host memory on a "
                        "second stream while the previous step runs (two device buffer sets; the first step's "
                        "copy, which nothing overlaps, counted), the step's result (loss, or the reconstruction "
                        "of an inference step) read back every step; an L2 flush (512 MB write) before every "
                        "step, counted in the time")
    _l.profile_enable(False)
    for k in PROFILE_GROUPS:
        _l.profile_read(k)  # discard the e2e loops' event times
    h2d = sum(d.numel() * d.element_size() for d, _ in ins)
    d2h = sum(h.numel() * h.element_size() for h, _ in outs)

    if rank != 0:
        return None
    value = whole_job_value(value_slices, world, steps, t_ms)
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "slices/s", "n_gpus": world,
        "steps": steps, "warmup": args.warmup, "ms_per_step": round(t_ms / steps, 4),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "c64" if args.workload == "cg_sense" else "c64+bf16",
        "data": "synthetic (seeded ellipse phantoms, Gaussian coil maps, k-space from the forward operator)",
        "config": {"workload": WORKLOADS[args.workload], "slices_per_gpu": B, "coils": cfg.C, "H": cfg.H,
                   "W": cfg.W, "R": cfg.R, "cg_iters": cfg.cg_iters, "lambda": cfg.lam,
                   "unrolled_blocks": cfg.extra.get("K") if args.workload in ("modl_train", "noncart_modl_infer") else None,
                   "stages": cfg.extra.get("T") if args.workload == "varnet_train" else None,
                   "parallelism": f"replicas x{world}", "l2": "flushed (512 MB write) between timed steps",
                   "reverse_pass": REVERSE_PASS.get(args.workload),
                   "timing": "value from K steps without the per-kernel events; kernel durations (roofline, "
                             "shares) from the same K steps run just before with them"},
        "roofline": kern.get(dominant),
        "kernels": kern,
        "time_breakdown": breakdown,
        "e2e": {"value": round(value_slices * world / (e2e_ms * 1e-3), 3), "unit": "slices/s",
                "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h, "ms_per_step": round(e2e_ms, 3),
                "mode": e2e_mode},
        "gpu_launches": launches,
        "clocks": clocks,
        "peaks": pk,
    }
    out.update(res)
    if args.workload in LEARNED and not args.no_train:
        # the learned reconstruction against CG-SENSE on the same held-out slices (untimed)
        from paper_2202_14005_b300 import train as _train
        kw = dict(LEARNED[args.workload])
        lr_res = _train.run(kw.pop("network"), kw.pop("steps"), 256, 16, kw.pop("lr"), seed=3, log_every=250,
                            **kw)
        out["nrmse_learned"] = round(lr_res["nrmse_learned"], 5)
        out["nrmse_cg_sense"] = round(lr_res["nrmse_cg_sense"], 5)
        out["learned_recon"] = lr_res
    return out


# ------------------------------------------------------------ CPU oracle
def _worker_init():
    os.environ["OMP_NUM_THREADS"] = "1"
    os.environ["OPENBLAS_NUM_THREADS"] = "1"
    os.environ["MKL_NUM_THREADS"] = "1"


def _oracle_slice(args):
    """One slice of a workload on the FP64 oracle; returns its CPU seconds."""
    import numpy as np
    import synth
    from oracle import cg as ocg
    from oracle import sense as osense
    from oracle import unrolled as ounr
    workload, s = args
    cfg = synth.CONFIGS[{"cg_sense": 2, "modl_train": 3, "varnet_train": 4, "noncart_modl_infer": 5}[workload]]
    d = synth.make_slices(cfg, [s])
    maps = d["maps"].astype(np.complex64)
    mask = d["mask"]
    gt = d["x_gt"].astype(np.complex64)
    if workload == "noncart_modl_infer":
        # one MoDL block (CNN forward + 10 CG iterations with the Toeplitz normal operator), scaled by
        # the K blocks; the PSF and x^0 = A^H A x_gt are setup, not timed
        from oracle import nn as onn
        from oracle import noncart as onc
        traj = synth.radial_trajectory(cfg.extra["spokes"], cfg.extra["samples"], cfg.H).reshape(-1, 2)
        psf = onc.toeplitz_psf(traj, cfg.H, cfg.W)
        x0 = onc.toeplitz_normal(gt, maps, psf, 0.0)
        ws, bs = synth.modl_cnn_weights(5000)
        t1 = time.perf_counter()
        z, _ = onn.modl_cnn_forward(x0, ws, bs)
        ocg.cg(lambda p: onc.toeplitz_normal(p, maps, psf, cfg.lam), x0 + cfg.lam * z, None, cfg.cg_iters)
        return cfg.extra["K"] * (time.perf_counter() - t1)
    y = (osense.forward(gt, maps, mask) + mask * d["noise"]).astype(np.complex64)
    t0 = time.perf_counter()
    rhs = osense.adjoint(y, maps, mask)
    if workload == "cg_sense":
        ocg.cg_solve(maps, mask, cfg.lam, rhs, rhs, cfg.cg_iters)
        return time.perf_counter() - t0
    t_adj = time.perf_counter() - t0
    if workload == "varnet_train":
        # VarNet: A^H y plus one gradient stage forward and reverse, scaled by T stages
        filt, rbfw, lam = synth.varnet_weights(4000, cfg.extra["T"])
        t1 = time.perf_counter()
        x1 = ounr.varnet_stage(rhs, rhs, maps, mask, filt[0], rbfw[0], lam[0])
        g = ounr.mse_loss_grad(x1, gt)
        ounr.varnet_stage_backward(g, rhs, rhs, maps, mask, filt[0], rbfw[0], lam[0])
        return t_adj + cfg.extra["T"] * (time.perf_counter() - t1)
    # MoDL: A^H y plus one unrolled block forward and reverse, scaled by K blocks
    ws, bs = synth.modl_cnn_weights(3000)
    t1 = time.perf_counter()
    x1, _ = ounr.modl_block(rhs, rhs, maps, mask, ws, bs, cfg.lam, cfg.cg_iters)
    g = ounr.mse_loss_grad(x1, gt)
    ounr.modl_block_backward(g, rhs, x1, rhs, maps, mask, ws, bs, cfg.lam, cfg.cg_iters)
    return t_adj + cfg.extra["K"] * (time.perf_counter() - t1)


def oracle_pool_run(workload, n, reps):
    cores = os.cpu_count() or 1
    ctx = mp.get_context("spawn")
    walls, per = [], []
    with ctx.Pool(processes=min(n, cores), initializer=_worker_init) as pool:
        pool.map(_oracle_slice, [("cg_sense", 0)])  # imports and FFT plans warm
        for _ in range(reps):
            t0 = time.perf_counter()
            per = pool.map(_oracle_slice, [(workload, s) for s in range(n)])
            walls.append(time.perf_counter() - t0)
    return walls, min(n, cores), per


def cpu_baseline(workload):
    """The oracle as it stands on the host cores: one process per slice."""
    n = 16 if workload == "cg_sense" else 4
    walls, used, per = oracle_pool_run(workload, n, 1)
    if workload == "cg_sense":
        wall = sum(walls)
        return {"value": round(n / wall, 5), "unit": "slices/s", "cores": used, "kind": "oracle",
                "sample": f"{n} slices, A^H y + 10 CG iterations each (FP64 NumPy, one spawn process per "
                          f"slice); wall {wall:.1f} s"}
    est = max(per)  # slices run in parallel: the step takes as long as the slowest slice
    if workload == "noncart_modl_infer":
        return {"value": round(n / est, 6), "unit": "slices/s", "cores": used, "kind": "oracle",
                "sample": f"{n} slices in parallel; per slice ONE MoDL block (CNN forward, 10 CG iterations with "
                          f"the Toeplitz normal operator, 12 coils, 512x512 embedding) timed and scaled by the "
                          f"10 blocks (FP64 NumPy, one spawn process per slice; PSF and x^0 precomputed); "
                          f"slowest slice {est:.1f} s per step"}
    if workload == "varnet_train":
        return {"value": round(n / est, 6), "unit": "slices/s", "cores": used, "kind": "oracle",
                "sample": f"{n} slices in parallel; per slice A^H y plus ONE gradient stage forward and reverse "
                          f"(24 11x11 filters, RBF, A^H A x, reverse mode with filter/RBF/lambda gradients), "
                          f"time scaled by the 10 stages of the step (FP64 NumPy, one spawn process per slice); "
                          f"slowest slice {est:.1f} s per step"}
    return {"value": round(n / est, 6), "unit": "slices/s", "cores": used, "kind": "oracle",
            "sample": f"{n} slices in parallel; per slice A^H y plus ONE unrolled block forward and reverse "
                      f"(CNN, 10-iteration CG, recomputed CNN, second CG, CNN backward), time scaled by the "
                      f"5 blocks of the step (FP64 NumPy, one spawn process per slice); slowest slice "
                      f"{est:.1f} s per step"}


def _oracle_full_step(args):
    """One slice's share of a whole step of a workload on the FP64 oracle, run in full (no
    extrapolation); returns its CPU seconds."""
    import numpy as np
    import synth
    from oracle import cg as ocg
    from oracle import sense as osense
    from oracle import unrolled as ounr
    workload, s = args
    if workload == "cg_sense":
        return _oracle_slice(args)
    cfg = synth.CONFIGS[{"modl_train": 3, "varnet_train": 4, "noncart_modl_infer": 5}[workload]]
    d = synth.make_slices(cfg, [s])
    maps = d["maps"].astype(np.complex64)
    mask = d["mask"]
    gt = d["x_gt"].astype(np.complex64)
    if workload == "noncart_modl_infer":
        from oracle import nn as onn
        from oracle import noncart as onc
        traj = synth.radial_trajectory(cfg.extra["spokes"], cfg.extra["samples"], cfg.H).reshape(-1, 2)
        psf = onc.toeplitz_psf(traj, cfg.H, cfg.W)
        x = onc.toeplitz_normal(gt, maps, psf, 0.0)  # x^0 (setup, not timed)
        ws, bs = synth.modl_cnn_weights(5000)
        t0 = time.perf_counter()
        x0 = x
        for _ in range(cfg.extra["K"]):
            z, _ = onn.modl_cnn_forward(x, ws, bs)
            x, _ = ocg.cg(lambda p: onc.toeplitz_normal(p, maps, psf, cfg.lam), x0 + cfg.lam * z, None,
                          cfg.cg_iters)
        return time.perf_counter() - t0
    y = (osense.forward(gt, maps, mask) + mask * d["noise"]).astype(np.complex64)
    t0 = time.perf_counter()
    rhs = osense.adjoint(y, maps, mask)
    if workload == "varnet_train":
        filt, rbfw, lam = synth.varnet_weights(4000, cfg.extra["T"])
        ounr.varnet_train_grads(rhs, maps, mask, gt, filt, rbfw, lam)
    else:
        ws, bs = synth.modl_cnn_weights(3000)
        ounr.modl_train_grads(rhs, maps, mask, gt, ws, bs, cfg.lam, cfg.extra["K"], cfg.cg_iters)
    return time.perf_counter() - t0


REFERENCE_BUDGET_S = 150.0  # wall time the reference arm's timed and warm-up steps may take


def run_reference(args, rank, world):
    """The FP64 oracle on the host cores, whole steps timed in full.

    A step is every slice of the sample (16 slices for CG-SENSE, one per core, at most the
    workload's batch, otherwise) going through the whole step of the workload, one spawn process
    per slice.  The first step is a warm-up; further warm-ups and the timed steps are as many of
    the requested ones as fit in REFERENCE_BUDGET_S (at least one timed step), and the line
    reports the counts actually run."""
    if rank != 0:
        return None
    import synth
    cores = os.cpu_count() or 1
    B = {"cg_sense": 16, "modl_train": synth.CONFIGS[3].B, "varnet_train": synth.CONFIGS[4].B,
         "noncart_modl_infer": synth.CONFIGS[5].B}[args.workload]
    n = 16 if args.workload == "cg_sense" else max(1, min(cores, B))
    ctx = mp.get_context("spawn")
    work = [(args.workload, s) for s in range(n)]
    with ctx.Pool(processes=min(n, cores), initializer=_worker_init) as pool:
        pool.map(_oracle_slice, [("cg_sense", 0)])  # imports and FFT plans (untimed)
        t0 = time.perf_counter()
        pool.map(_oracle_full_step, work)
        probe = time.perf_counter() - t0
        left = REFERENCE_BUDGET_S - probe
        warm = 1 + max(0, min(args.warmup - 1, int(left / probe) - args.steps))
        for _ in range(warm - 1):
            pool.map(_oracle_full_step, work)
        left = REFERENCE_BUDGET_S - warm * probe
        steps = max(1, min(args.steps, int(left / probe)))
        walls = []
        for _ in range(steps):
            t0 = time.perf_counter()
            pool.map(_oracle_full_step, work)
            walls.append(time.perf_counter() - t0)
    wall = sum(walls)
    value = n * steps / wall
    what = {"cg_sense": "A^H y + 10 CG iterations (x0 = A^H y)",
            "modl_train": "A^H y, 5 MoDL blocks forward (CNN + 10-iteration CG) and reverse (second CG, "
                          "CNN backward), loss and gradients",
            "varnet_train": "A^H y, 10 VarNet stages forward and reverse, loss and gradients",
            "noncart_modl_infer": "10 MoDL blocks (CNN + 10 CG iterations with the Toeplitz normal operator "
                                  "on the 512x512 embedding; PSF and x^0 precomputed)"}[args.workload]
    sample = (f"{n} slices per step, each the whole step: {what} (FP64 NumPy oracle, one spawn process "
              f"per slice, {min(n, cores)} of {cores} host cores); {warm} warm-up and {steps} timed steps "
              f"run in full (of {args.warmup} and {args.steps} requested; the arm's wall-time budget is "
              f"{REFERENCE_BUDGET_S:.0f} s)")
    return {"impl": "reference", "metric": METRIC, "value": round(value, 5), "unit": "slices/s",
            "n_gpus": world, "steps": steps, "warmup": warm,
            "ms_per_step": round(1e3 * wall / steps, 2), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "c128",
            "data": "synthetic", "config": {"workload": WORKLOADS[args.workload], "slices_per_step": n},
            "cpu_baseline": {"value": round(value, 5), "unit": "slices/s", "cores": min(n, cores),
                             "kind": "oracle", "sample": sample},
            "e2e": {"value": round(value, 5), "unit": "slices/s", "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}


def e2e_pipelined(bufs, host, step, loss_fn, n, flush):
    """End-to-end time per step (ms) of n steps fed from pinned host memory: the copies of step
    i + 1's inputs into device buffer set (i + 1) % 2 run on a second stream while step i runs on
    the current stream; every step's result (the loss of a training step, the reconstruction of
    an inference step) is read back to the host.  Before every step the L2 cache is flushed (a
    write larger than L2), as between the device-resident timed steps, and the flush's time
    counts.  The timed region runs from before the first copy to the completion of the last
    read-back."""
    import torch
    main = torch.cuda.current_stream()
    cs = torch.cuda.Stream()
    ev = lambda: torch.cuda.Event(enable_timing=False)
    copied, used = [ev(), ev()], [ev(), ev()]
    res = loss_fn()
    hb = [torch.empty(res.shape, dtype=res.dtype).pin_memory() for _ in range(2)]
    loss_h = [hb[i % 2] for i in range(n)]
    torch.cuda.synchronize()
    t0, t1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0.record(main)

    def copy_in(k):
        with torch.cuda.stream(cs):
            for d, h in zip(bufs[k], host):
                d.copy_(h, non_blocking=True)
            copied[k].record(cs)

    cs.wait_event(t0)
    copy_in(0)
    for i in range(n):
        k = i % 2
        if i + 1 < n:
            if i >= 1:
                cs.wait_event(used[(i + 1) % 2])  # step i - 1 has finished with that buffer set
            copy_in((i + 1) % 2)
        main.wait_event(copied[k])
        flush.zero_()
        step(k)
        loss_h[i].copy_(loss_fn(), non_blocking=True)
        used[k].record(main)
    t1.record(main)
    torch.cuda.synchronize()
    return t0.elapsed_time(t1) / n


def secondary_summary(r):
    """The main figures of another workload's line (value, e2e, dominant kernel, NRMSEs)."""
    keep = ("value", "unit", "ms_per_step", "steps", "warmup", "config", "clocks", "gpu_launches",
            "nrmse_learned", "nrmse_cg_sense", "noncart")
    out = {k: r[k] for k in keep if k in r}
    out["e2e"] = r["e2e"]["value"]
    rf = r.get("roofline") or {}
    out["dominant_kernel"] = {k: rf.get(k) for k in ("kernel", "bound", "achieved", "unit", "frac", "avg_launch_us")}
    out["kernels"] = {k: {"achieved": v["achieved"], "unit": v["unit"], "frac": v["frac"],
                          "avg_launch_us": v["avg_launch_us"]} for k, v in (r.get("kernels") or {}).items()}
    if "learned_recon" in r:
        lr = r["learned_recon"]
        out["learned_recon"] = {k: lr[k] for k in ("network", "steps", "optimizer", "nrmse_untrained",
                                                   "nrmse_learned", "nrmse_cg_sense", "nrmse_cg_sense_best",
                                                   "train_seconds") if k in lr}
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="modl_train", choices=list(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-train", action="store_true",
                    help="skip the (untimed) training and held-out NRMSE evaluation")
    ap.add_argument("--no-secondary", action="store_true",
                    help="default workload only: skip the VarNet and radial workloads measured after it")
    ap.add_argument("--profile-step", action="store_true",
                    help="run one step of the workload inside a CUDA profiler range after its warm-up, "
                         "then exit (for ncu --profile-from-start off); prints no bench line")
    args = ap.parse_args()
    global PROFILE_STEP
    if args.profile_step:
        PROFILE_STEP = args.workload
        args.no_cpu_baseline = True
    if args.impl == "ours":
        args.warmup = max(args.warmup, 3)
        args.steps = max(args.steps, 1)

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local_rank = int(os.environ.get("LOCAL_RANK", "0"))

    if args.impl == "reference":
        res = run_reference(args, rank, world)
        if res is not None:
            print(json.dumps(res), flush=True)
        return

    base = None
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        base = cpu_baseline(args.workload)  # the spawn pool runs before the first GPU call

    import torch
    if world > 1:
        torch.distributed.init_process_group("nccl", device_id=torch.device("cuda", local_rank))
    res = run_ours(args, rank, world, local_rank)
    if res is not None and world == 1 and args.workload == "modl_train" and not args.no_secondary:
        # the other two network workloads, measured the same way after the headline step and
        # reported beside it (their own lines come from --workload varnet_train / noncart_modl_infer)
        sec = {}
        for w in ("varnet_train", "noncart_modl_infer"):
            sub = argparse.Namespace(**vars(args))
            sub.workload, sub.steps = w, min(args.steps, 10)
            sec[w] = secondary_summary(run_ours(sub, rank, world, local_rank))
        res["secondary_workloads"] = sec
    if res is not None:
        res["cpu_baseline"] = base
        print(json.dumps(res), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()


if __name__ == "__main__":
    main()
