"""Seeded synthetic inputs for the SENSE / unrolled-reconstruction workloads.

This module only draws data: phantoms, coil-sensitivity maps, Cartesian
sampling masks, noise and initial network weights.  It contains none of the
method's arithmetic (no SENSE operator, no DFT of the method, no CG, no
convolution), so that both the FP64 oracle and the CUDA path can consume the
same inputs without sharing any code that computes results.

Recipe (data of the paper's Sec. "Results", simulated k-space: images times
maps, Fourier transform, subsampling, complex Gaussian noise sigma = 1e-3):

* phantom: sum of random ellipses in normalised coordinates u in [-1, 1)^2
  (centres U[-0.6, 0.6]^2, semi-axes U[0.05, 0.45], angle U[0, pi),
  intensity U[0.1, 1], additive), times exp(i*phi) with phi a smooth field of
  three random low-frequency cosines (total amplitude <= pi/2).  Optional
  band-limited texture (|k| < W/8) at 10 % amplitude.
* coil maps: Gaussian magnitude (sigma 0.4 FOV) centred on a circle of radius
  0.5 FOV, linear phase (|k| <= pi rad per FOV) plus a constant phase, then
  divided per pixel by sqrt(sum_c |S_c|^2) so that sum_c |S_c|^2 = 1.
* masks: phase-encode lines along the last axis (W), constant along H.
  n_lines = round(W / R) lines in total: n_centre contiguous centre lines and
  the rest drawn without replacement, uniformly or with Gaussian density
  exp(-d^2 / (2 (W/4)^2)) in the distance d from the centre line.
* noise: complex, real and imaginary parts each N(0, sigma^2).
* seeds: numpy.random.default_rng(1000 * config + slice).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "Config", "CONFIGS", "slice_rng", "phantom", "coil_maps", "line_mask",
    "complex_noise", "randn_complex", "he_normal", "make_slices",
    "modl_cnn_weights", "varnet_weights", "radial_trajectory",
]


@dataclass(frozen=True)
class Config:
    """One workload shape.  Fields follow the notation B, C, H, W of the method."""

    index: int
    name: str
    B: int
    C: int
    H: int
    W: int
    R: float
    n_centre: int
    density: str          # "uniform" | "gaussian"
    lam: float
    cg_iters: int
    texture: bool = False
    n_ellipses: int = 10
    extra: dict = field(default_factory=dict)


CONFIGS = {
    1: Config(1, "cg_sense_64x64_c8", B=1, C=8, H=64, W=64, R=4, n_centre=16,
              density="uniform", lam=0.01, cg_iters=10),
    2: Config(2, "cg_sense_b16_c12_256x232", B=16, C=12, H=256, W=232, R=6,
              n_centre=24, density="gaussian", lam=0.05, cg_iters=10, texture=True),
    3: Config(3, "modl_train_b4_c12_256x232", B=4, C=12, H=256, W=232, R=6,
              n_centre=24, density="gaussian", lam=0.05, cg_iters=10, texture=True,
              extra={"K": 5}),
    4: Config(4, "varnet_train_b4_c15_320x368", B=4, C=15, H=320, W=368, R=4,
              n_centre=24, density="uniform", lam=1.0, cg_iters=0,
              extra={"T": 10, "Nk": 24, "ksize": 11, "Nw": 31}),
    5: Config(5, "modl_radial_b32_c12_256x256", B=32, C=12, H=256, W=256, R=1,
              n_centre=0, density="uniform", lam=0.05, cg_iters=10,
              extra={"spokes": 96, "samples": 512, "K": 10}),
}


def slice_rng(config: int, slice_index: int, split: str = "eval") -> np.random.Generator:
    """Generator of one slice.  The "eval" split (the workloads, the tests and the held-out
    evaluation) is seeded 1000 config + slice; the "train" split draws from the seed sequence
    (7, config, slice), a stream disjoint from every integer seed, so training slices never
    repeat an evaluation slice."""
    if split == "train":
        return np.random.default_rng([7, config, slice_index])
    if split != "eval":
        raise ValueError("split must be 'eval' or 'train'")
    return np.random.default_rng(1000 * config + slice_index)


def _grid(H: int, W: int):
    """Pixel-centre-free normalised grid: u in [-1, 1), row index -> y, column -> x."""
    uy = (2.0 * np.arange(H) - H) / H
    ux = (2.0 * np.arange(W) - W) / W
    return np.meshgrid(uy, ux, indexing="ij")


def phantom(H: int, W: int, rng: np.random.Generator, n_ellipses: int = 10,
            texture: bool = False) -> np.ndarray:
    """Random-ellipse phantom with smooth phase, complex128 [H, W]."""
    Y, X = _grid(H, W)
    mag = np.zeros((H, W))
    for _ in range(n_ellipses):
        cy, cx = rng.uniform(-0.6, 0.6, size=2)
        a, b = rng.uniform(0.05, 0.45, size=2)
        th = rng.uniform(0.0, math.pi)
        val = rng.uniform(0.1, 1.0)
        dx, dy = X - cx, Y - cy
        xr = dx * math.cos(th) + dy * math.sin(th)
        yr = -dx * math.sin(th) + dy * math.cos(th)
        mag += val * ((xr / a) ** 2 + (yr / b) ** 2 <= 1.0)
    if texture:
        g = rng.standard_normal((H, W))
        G = np.fft.fft2(g)
        ky = np.fft.fftfreq(H) * H
        kx = np.fft.fftfreq(W) * W
        KY, KX = np.meshgrid(ky, kx, indexing="ij")
        G[np.sqrt(KY ** 2 + KX ** 2) >= W / 8.0] = 0.0
        t = np.real(np.fft.ifft2(G))
        t /= max(t.std(), 1e-30)
        mag = mag * (1.0 + 0.1 * t)
    amps = rng.uniform(0.0, 1.0, size=3)
    amps *= (math.pi / 2) / amps.sum()
    phi = np.zeros((H, W))
    for j in range(3):
        fy, fx = rng.uniform(-1.0, 1.0, size=2) * 0.5   # <= 1/2 cycle per unit
        ph0 = rng.uniform(0.0, 2 * math.pi)
        phi += amps[j] * np.cos(math.pi * (fy * Y + fx * X) + ph0)
    return mag * np.exp(1j * phi)


def coil_maps(C: int, H: int, W: int, rng: np.random.Generator,
              sigma: float = 0.4) -> np.ndarray:
    """Smooth Gaussian-profile coil maps normalised to sum_c |S_c|^2 = 1, complex128 [C, H, W]."""
    Y, X = _grid(H, W)
    ry, rx = Y / 2.0, X / 2.0          # FOV units, [-0.5, 0.5)
    S = np.empty((C, H, W), dtype=np.complex128)
    for c in range(C):
        ang = 2 * math.pi * c / C
        cy, cx = 0.5 * math.sin(ang), 0.5 * math.cos(ang)
        prof = np.exp(-((ry - cy) ** 2 + (rx - cx) ** 2) / (2 * sigma ** 2))
        rho = rng.uniform(0.0, 1.0)
        psi = rng.uniform(0.0, 2 * math.pi)
        ky, kx = math.pi * rho * math.sin(psi), math.pi * rho * math.cos(psi)
        ph0 = rng.uniform(0.0, 2 * math.pi)
        S[c] = prof * np.exp(1j * (ky * ry + kx * rx + ph0))
    rss = np.sqrt(np.sum(np.abs(S) ** 2, axis=0))
    return S / rss


def line_mask(W: int, R: float, n_centre: int, density: str,
              rng: np.random.Generator) -> np.ndarray:
    """Phase-encode line mask, float32 [W] of 0/1 (centred k-space index order)."""
    n_lines = int(round(W / R))
    n_centre = min(n_centre, n_lines)
    m = np.zeros(W, dtype=np.float32)
    c0 = W // 2 - n_centre // 2
    m[c0:c0 + n_centre] = 1.0
    rest = n_lines - n_centre
    if rest > 0:
        cand = np.flatnonzero(m == 0)
        if density == "gaussian":
            d = cand - W / 2.0
            p = np.exp(-d ** 2 / (2 * (W / 4.0) ** 2))
        else:
            p = np.ones(cand.size)
        p = p / p.sum()
        pick = rng.choice(cand, size=rest, replace=False, p=p)
        m[pick] = 1.0
    return m


def complex_noise(shape, sigma: float, rng: np.random.Generator) -> np.ndarray:
    return sigma * (rng.standard_normal(shape) + 1j * rng.standard_normal(shape))


def randn_complex(shape, seed: int) -> np.ndarray:
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def he_normal(shape, fan_in: int, rng: np.random.Generator) -> np.ndarray:
    return rng.standard_normal(shape) * math.sqrt(2.0 / fan_in)


def make_slices(cfg: Config, slices=None, noise_sigma: float = 1e-3, split: str = "eval") -> dict:
    """Per-slice inputs of one workload (complex128 / float32 numpy arrays).

    Returns x_gt [B,H,W], maps [B,C,H,W], mask [W] (shared by the batch and by
    both splits, drawn from its own stream of this config) and noise [B,C,H,W].
    """
    idx = list(range(cfg.B)) if slices is None else list(slices)
    xs, Ss, ns = [], [], []
    mask = line_mask(cfg.W, cfg.R, cfg.n_centre, cfg.density,
                     np.random.default_rng(1000 * cfg.index + 999))
    for s in idx:
        rng = slice_rng(cfg.index, s, split)
        xs.append(phantom(cfg.H, cfg.W, rng, cfg.n_ellipses, cfg.texture))
        Ss.append(coil_maps(cfg.C, cfg.H, cfg.W, rng))
        ns.append(complex_noise((cfg.C, cfg.H, cfg.W), noise_sigma, rng))
    return {"x_gt": np.stack(xs), "maps": np.stack(Ss), "mask": mask,
            "noise": np.stack(ns)}


def modl_cnn_weights(seed: int, chans=(2, 64, 64, 64, 64, 2), k: int = 3):
    """He-normal conv weights [Cout, Cin, k, k] (float64) and zero biases."""
    rng = np.random.default_rng(seed)
    ws, bs = [], []
    for cin, cout in zip(chans[:-1], chans[1:]):
        ws.append(he_normal((cout, cin, k, k), cin * k * k, rng))
        bs.append(np.zeros(cout))
    return ws, bs


def varnet_weights(seed: int, T: int = 10, Nk: int = 24, k: int = 11, Nw: int = 31):
    """Per-stage complex filters [Nk, k, k], RBF weights [Nk, Nw] and step sizes [T].

    Filters: zero-mean Gaussian with std 1/(k*sqrt(2)) per real component;
    RBF weights initialised to a small linear slope (w_j = 0.1 * mu_j) so that
    Phi' starts close to a scaled identity; step sizes 1.0.
    """
    rng = np.random.default_rng(seed)
    mu = np.linspace(-1.0, 1.0, Nw)
    filt = (rng.standard_normal((T, Nk, k, k)) + 1j * rng.standard_normal((T, Nk, k, k))) / (k * math.sqrt(2.0))
    filt -= filt.mean(axis=(2, 3), keepdims=True)
    rbf = np.tile(0.1 * mu, (T, Nk, 1))
    lam = np.ones(T)
    return filt, rbf, lam


def radial_trajectory(spokes: int, samples: int, N: int) -> np.ndarray:
    """Golden-angle radial k-space positions [spokes, samples, 2] in grid units, k in [-N/2, N/2)."""
    ga = math.pi * (math.sqrt(5.0) - 1.0) / 2.0
    r = (np.arange(samples) - samples / 2.0) * (N / samples)
    out = np.empty((spokes, samples, 2))
    for s in range(spokes):
        a = s * ga
        out[s, :, 0] = r * math.sin(a)
        out[s, :, 1] = r * math.cos(a)
    return out
