"""The allocation-free inner product (sense_dot_re_noalloc) against the
workspace path.

Some callers may not allocate GPU memory once they run (a service that
reserves all device memory at start-up, or a host whose memory manager owns
the device heap).  For them the library offers one entry point whose scratch
is a fixed array inside the library.  This test calls it through the C ABI,
twice in a row (the array keeps the previous call's contents), and checks it
against the lambda gradient that cg_dc_solve_backward computes with its plan
workspace, at the CG tolerance used by the other GPU tests (1e-4 relative).
It also checks that a problem larger than the fixed scratch is refused.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

TOL = 1e-4


def _inputs(B=3, Cc=4, H=64, W=232, seed=71):
    rng = np.random.default_rng(seed)
    maps = np.stack([synth.coil_maps(Cc, H, W, rng) for _ in range(B)]).astype(np.complex64)
    mask = synth.line_mask(W, 6.0, 24, "gaussian", rng)
    x = (synth.randn_complex((B, H, W), seed + 1) * 0.3).astype(np.complex64)
    z = (synth.randn_complex((B, H, W), seed + 2) * 0.1).astype(np.complex64)
    g = (synth.randn_complex((B, H, W), seed + 3) * 0.01).astype(np.complex64)
    t = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    return t(maps), t(mask), t(x), t(z), t(g)


def _p(t):
    return C.c_void_p(t.data_ptr())


def test_noalloc_dot_matches_cg_backward_lambda_gradient():
    from paper_2202_14005_b300 import _lib
    from paper_2202_14005_b300.sense import SensePlan

    maps, mask, x, z, g = _inputs()
    B, H, W = x.shape
    plan = SensePlan(maps, mask)
    lam = torch.tensor([0.05], dtype=torch.float64, device="cuda")
    lamB = lam.repeat(B)
    v, gl_sum = plan.cg_solve_backward(g, x, z, lam, 10)
    _, gl_per = plan.cg_solve_backward(g, x, z, lamB, 10)
    torch.cuda.synchronize()
    ref_sum = gl_sum.cpu().numpy()
    ref_per = gl_per.cpu().numpy()

    L = _lib.lib()
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    for _ in range(2):  # two calls in a row share the same scratch
        out_per = torch.full((B,), float("nan"), dtype=torch.float64, device="cuda")
        out_sum = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
        assert L.sense_dot_re_noalloc(B, H, W, _p(v), _p(z), _p(x), _p(out_per), B, stream) == 0
        assert L.sense_dot_re_noalloc(B, H, W, _p(v), _p(z), _p(x), _p(out_sum), 1, stream) == 0
        torch.cuda.synchronize()
        per = out_per.cpu().numpy()
        tot = out_sum.cpu().numpy()
        np.testing.assert_allclose(per, ref_per, rtol=TOL, atol=TOL * np.abs(ref_per).max())
        assert abs(tot[0] - ref_sum[0]) <= TOL * np.abs(ref_per).sum()


def test_noalloc_refuses_problems_beyond_its_scratch():
    from paper_2202_14005_b300 import _lib

    L = _lib.lib()
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    max_rows = ((1 << 20) - 256) // 8
    # refused on the host, before any launch
    assert L.sense_dot_re_noalloc(1, max_rows + 1, 2, _p(buf), None, None, _p(out), 1, None) == -8
    assert L.sense_strerror(-8).decode().startswith("problem exceeds")
