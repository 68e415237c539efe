"""GPU parity of the non-Cartesian SENSE path (Sec. 2.3.3): the PSF of a golden-angle
radial trajectory, the Toeplitz-embedded normal operator and CG, against the oracle
(direct non-uniform DFT sums, FP64).

Tolerances: the PSF sums M unit phasors (FP32 phasors from FP64-reduced phases, FP64
accumulation): 1e-6 relative L2.  Normal operator (FP32 FFTs of length 2H and 2W): 1e-5;
10-iteration CG: 1e-4 (the Cartesian bounds)."""
import numpy as np
import pytest
import torch

import synth
from oracle import cg as ocg
from oracle import noncart as onc

pytestmark = pytest.mark.gpu


def rel(a, b):
    a = np.asarray(a, dtype=np.complex128)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))


def dev(a):
    return torch.from_numpy(np.ascontiguousarray(a)).cuda()


def case(B, C, N, spokes, samples, seed):
    rng = np.random.default_rng(seed)
    maps = np.stack([synth.coil_maps(C, N, N, rng) for _ in range(B)]).astype(np.complex64)
    traj = synth.radial_trajectory(spokes, samples, N).reshape(-1, 2).astype(np.float32)
    return maps, traj


@pytest.mark.parametrize("N,spokes,samples", [(32, 16, 64), (48, 21, 96)])
def test_psf_and_normal_operator(N, spokes, samples):
    from paper_2202_14005_b300.sense import SensePlan, toeplitz_psf
    maps, traj = case(2, 4, N, spokes, samples, seed=N)
    psf = toeplitz_psf(dev(traj), N, N)
    torch.cuda.synchronize()
    rpsf = onc.toeplitz_psf(traj.astype(np.float64), N, N)
    assert rel(psf.cpu().numpy(), rpsf) <= 1e-6
    x = synth.randn_complex((2, N, N), 1).astype(np.complex64)
    plan = SensePlan.toeplitz(dev(maps), psf)
    out = plan.normal(dev(x), 0.1).cpu().numpy()
    ref = onc.toeplitz_normal(x, maps, rpsf, 0.1)
    assert rel(out, ref) <= 1e-5
    # the direct non-uniform DFT pair gives the same operator
    direct = onc.nudft_adjoint(onc.nudft_forward(x, maps, traj.astype(np.float64)), maps,
                               traj.astype(np.float64)) + 0.1 * x
    assert rel(out, direct) <= 1e-5
    assert plan.status() == 0


def test_cg_with_toeplitz_plan():
    from paper_2202_14005_b300.sense import SensePlan, toeplitz_psf
    N = 40
    maps, traj = case(2, 3, N, 24, 80, seed=7)
    psf = toeplitz_psf(dev(traj), N, N)
    rpsf = onc.toeplitz_psf(traj.astype(np.float64), N, N)
    plan = SensePlan.toeplitz(dev(maps), psf)
    rhs = synth.randn_complex((2, N, N), 2).astype(np.complex64)
    lam = torch.tensor([0.02], dtype=torch.float64, device="cuda")
    x = plan.cg_solve(dev(rhs), lam, 10).cpu().numpy()
    ref, _ = ocg.cg(lambda p: onc.toeplitz_normal(p, maps, rpsf, 0.02), rhs, None, 10)
    assert rel(x, ref) <= 1e-4
    assert plan.status() == 0


def test_full_size_radial_workload_sampled():
    """256 x 256, 12 coils, 96 golden-angle spokes x 512 samples: sampled PSF rows against the
    direct sum, and the normal operator against the oracle's FFT embedding of the GPU's PSF."""
    from paper_2202_14005_b300.sense import SensePlan, toeplitz_psf
    N = 256
    maps, traj = case(1, 12, N, 96, 512, seed=5)
    psf = toeplitz_psf(dev(traj), N, N)
    plan = SensePlan.toeplitz(dev(maps), psf)
    x = synth.randn_complex((1, N, N), 3).astype(np.complex64)
    out = plan.normal(dev(x), 0.0).cpu().numpy()
    g = psf.cpu().numpy().astype(np.complex128)
    t = traj.astype(np.float64)
    rows = [0, 1, 37, 255, 256, 300, 511]
    dy = np.array([r if r < N else r - 2 * N for r in rows], dtype=np.float64)
    dx = np.arange(2 * N)
    dx = np.where(dx < N, dx, dx - 2 * N)
    ref_rows = (np.exp(2j * np.pi * t[:, 0, None] * dy[None, :] / N).T
                @ np.exp(2j * np.pi * t[:, 1, None] * dx[None, :] / N)) / (N * N)
    ref_rows[:, N] = 0
    ref_rows[rows.index(256)] = 0
    assert rel(g[rows], ref_rows) <= 1e-6
    assert rel(out, onc.toeplitz_normal(x, maps, g, 0.0)) <= 1e-5


def test_toeplitz_256_rows_ragged_columns():
    """H = 256 takes the register-resident 512-point column pass; W = 250 leaves a last group of
    4 of its 8 columns (2W = 500), and two slices with their own maps."""
    from paper_2202_14005_b300.sense import SensePlan, toeplitz_psf
    B, C, H, W = 2, 3, 256, 250
    rng = np.random.default_rng(11)
    maps = np.stack([synth.coil_maps(C, H, W, rng) for _ in range(B)]).astype(np.complex64)
    traj = synth.radial_trajectory(40, 300, W).reshape(-1, 2).astype(np.float32)
    psf = toeplitz_psf(dev(traj), H, W)
    plan = SensePlan.toeplitz(dev(maps), psf)
    x = synth.randn_complex((B, H, W), 4).astype(np.complex64)
    out = plan.normal(dev(x), 0.3).cpu().numpy()
    g = psf.cpu().numpy().astype(np.complex128)
    ref = onc.toeplitz_normal(x, maps, g, 0.3)
    for b in range(B):
        assert rel(out[b], ref[b]) <= 1e-5
    assert plan.status() == 0


@pytest.mark.parametrize("B,C,H,lam", [(2, 3, 100, 0.2), (32, 2, 256, 0.0)])
def test_toeplitz_256_columns_row_passes(B, C, H, lam):
    """W = 256 takes the register-resident 512-point row passes.  H = 100 leaves a last CTA with
    4 of its 8 rows and splits the coils into groups (partial sums and the group sum); 32 slices
    of 256 rows put all coils in one group (the combine and + lambda x in the row pass)."""
    from paper_2202_14005_b300.sense import SensePlan, toeplitz_psf
    W = 256
    rng = np.random.default_rng(B + H)
    maps = np.stack([synth.coil_maps(C, H, W, rng) for _ in range(B)]).astype(np.complex64)
    traj = synth.radial_trajectory(32, 256, H).reshape(-1, 2).astype(np.float32)
    psf = toeplitz_psf(dev(traj), H, W)
    plan = SensePlan.toeplitz(dev(maps), psf)
    x = synth.randn_complex((B, H, W), 5).astype(np.complex64)
    out = plan.normal(dev(x), lam).cpu().numpy()
    g = psf.cpu().numpy().astype(np.complex128)
    ref = onc.toeplitz_normal(x, maps, g, lam)
    for b in range(B):
        assert rel(out[b], ref[b]) <= 1e-5
    assert plan.status() == 0


@pytest.mark.parametrize("B,C,N,spokes,samples", [(2, 3, 32, 16, 64), (1, 13, 40, 21, 48)])
def test_nudft_pair_against_direct_sums(B, C, N, spokes, samples):
    """The GPU non-uniform DFT pair against the oracle's direct FP64 sums (1e-5; 13 coils
    exercise a partial coil pass), the adjoint identity <A x, y> = <x, A^H y>, and A^H A of the
    pair equal to the Toeplitz normal operator of the PSF."""
    from paper_2202_14005_b300.sense import SensePlan, nudft_adjoint, nudft_forward, toeplitz_psf
    maps, traj = case(B, C, N, spokes, samples, seed=N + C)
    t64 = traj.astype(np.float64)
    x = synth.randn_complex((B, N, N), 11).astype(np.complex64)
    y = synth.randn_complex((B, C, traj.shape[0]), 12).astype(np.complex64)
    yg = nudft_forward(dev(traj), dev(maps), dev(x)).cpu().numpy()
    xg = nudft_adjoint(dev(traj), dev(maps), dev(y)).cpu().numpy()
    assert rel(yg, onc.nudft_forward(x, maps, t64)) <= 1e-5
    assert rel(xg, onc.nudft_adjoint(y, maps, t64)) <= 1e-5
    lhs = np.vdot(yg.astype(np.complex128), y)          # <A x, y>
    rhs = np.vdot(x.astype(np.complex128), xg)          # <x, A^H y>
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)
    psf = toeplitz_psf(dev(traj), N, N)
    plan = SensePlan.toeplitz(dev(maps), psf)
    n_op = plan.normal(dev(x), 0.0).cpu().numpy()
    pair = nudft_adjoint(dev(traj), dev(maps), nudft_forward(dev(traj), dev(maps), dev(x))).cpu().numpy()
    assert rel(pair, n_op) <= 1e-5


def test_nudft_full_size_sampled():
    """256 x 256, 12 coils, 96 golden-angle spokes x 512 samples: sampled outputs of both
    directions against direct FP64 sums for those entries alone."""
    from paper_2202_14005_b300.sense import nudft_adjoint, nudft_forward
    N, C = 256, 12
    maps, traj = case(1, C, N, 96, 512, seed=21)
    t64 = traj.astype(np.float64)
    x = synth.randn_complex((1, N, N), 13).astype(np.complex64)
    y = synth.randn_complex((1, C, traj.shape[0]), 14).astype(np.complex64)
    yg = nudft_forward(dev(traj), dev(maps), dev(x)).cpu().numpy()
    xg = nudft_adjoint(dev(traj), dev(maps), dev(y)).cpu().numpy()
    ny = np.arange(N) - N // 2
    u = maps[0].astype(np.complex128) * x[0].astype(np.complex128)          # [C, N, N]
    for m in (0, 1, 255, 256, 10000, traj.shape[0] - 1):
        e = np.exp(-2j * np.pi * (t64[m, 0] * ny[:, None] / N + t64[m, 1] * ny[None, :] / N))
        ref = (u * e).sum(axis=(1, 2)) / N
        assert np.linalg.norm(yg[0, :, m] - ref) <= 1e-5 * np.linalg.norm(ref)
    for (r, c) in ((0, 0), (128, 128), (17, 250), (255, 3)):
        ph = np.exp(2j * np.pi * (t64[:, 0] * (r - N // 2) / N + t64[:, 1] * (c - N // 2) / N))
        v = (y[0].astype(np.complex128) * ph[None]).sum(axis=1) / N          # [C]
        ref = np.sum(np.conj(maps[0, :, r, c].astype(np.complex128)) * v)
        assert abs(xg[0, r, c] - ref) <= 1e-5 * max(abs(ref), np.abs(v).max())


def test_cg_toeplitz_fused_dot_32_slices():
    """32 slices of 256 x 256 put every coil of a row in one CTA of the register-resident inverse
    row pass, which then also forms the rows of Re<p, S p> for the CG step (no separate dot
    pass): 5 iterations against the oracle's CG on the Toeplitz operator of the GPU's PSF, with
    residual histories."""
    from paper_2202_14005_b300.sense import SensePlan, toeplitz_psf
    B, C, N, lam_v, iters = 32, 2, 256, 0.5, 5
    maps, traj = case(B, C, N, 32, 256, seed=9)
    psf = toeplitz_psf(dev(traj), N, N)
    plan = SensePlan.toeplitz(dev(maps), psf)
    rhs = synth.randn_complex((B, N, N), 6).astype(np.complex64)
    lam = torch.tensor([lam_v], dtype=torch.float64, device="cuda")
    hist = torch.zeros((iters + 1, B), dtype=torch.float64, device="cuda")
    x = plan.cg_solve(dev(rhs), lam, iters, rr_hist=hist).cpu().numpy()
    g = psf.cpu().numpy().astype(np.complex128)
    ref, rr = ocg.cg(lambda p: onc.toeplitz_normal(p, maps, g, lam_v), rhs, None, iters)
    assert rel(x, ref) <= 1e-4
    np.testing.assert_allclose(hist.cpu().numpy(), rr, rtol=1e-3, atol=1e-12 * rr[0].max())
    assert plan.status() == 0
