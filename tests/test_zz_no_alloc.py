"""The allocation-free inner product (sense_dot_re_noalloc) against the
workspace path and against an FP64 sum on the host.

Some callers may not allocate GPU memory once they run: a reconstruction
service that reserves all device memory at start-up (an allocation in the
middle of streaming data can stall every stream on the device), or a host
program whose own memory manager owns the device heap.  For them the library
offers one entry point whose scratch is a fixed array inside the library.

These tests call it through the C ABI, twice in a row (the array keeps the
previous call's contents), and check that
* it returns exactly the bits of the lambda gradient that cg_dc_solve_backward
  computes with its plan workspace (same row split and order of summation),
  for a rhs term and without one (b = NULL), per slice and summed;
* it agrees with Re(sum conj(a) (b - c)) summed in float64 by numpy on the
  host copies, with b or c NULL, for B = 1 and for a problem of exactly
  SENSE_NOALLOC_MAX_ROWS rows, within the FP32 rounding of the products;
* a problem larger than the fixed scratch is refused before anything runs.
This file is collected last on purpose.
"""
import ctypes as C

import numpy as np
import pytest
import torch

import synth

pytestmark = pytest.mark.gpu

MAX_ROWS = ((1 << 20) - 256) // 8


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
    return None if t is None else C.c_void_p(t.data_ptr())


def _noalloc(a, b, c, count):
    from paper_2202_14005_b300 import _lib
    B, H, W = a.shape
    out = torch.full((count,), float("nan"), dtype=torch.float64, device="cuda")
    stream = C.c_void_p(torch.cuda.current_stream().cuda_stream)
    rc = _lib.lib().sense_dot_re_noalloc(B, H, W, _p(a), _p(b), _p(c), _p(out), count, stream)
    assert rc == 0, rc
    return out


def _host_dot(a, b, c):
    """Re(sum conj(a) (b - c)) per slice in float64 from the host copies."""
    a64 = a.cpu().numpy().astype(np.complex128)
    d = np.zeros_like(a64)
    if b is not None:
        d += b.cpu().numpy()
    if c is not None:
        d -= c.cpu().numpy()
    prod = np.conj(a64) * d
    return prod.real.sum(axis=(1, 2)), np.abs(a64).sum(axis=(1, 2)) * np.abs(d).max()


def test_noalloc_dot_equals_cg_backward_lambda_gradient_bitwise():
    from paper_2202_14005_b300.sense import SensePlan

    maps, mask, x, z, g = _inputs()
    B = x.shape[0]
    plan = SensePlan(maps, mask)
    lam = torch.tensor([0.05], dtype=torch.float64, device="cuda")
    lamB = lam.repeat(B)
    refs = {}
    for zz, key in ((z, "z"), (None, "noz")):
        v, gl_sum = plan.cg_solve_backward(g, x, zz, lam, 10)
        _, gl_per = plan.cg_solve_backward(g, x, zz, lamB, 10)
        refs[key] = (v.clone(), gl_sum.clone(), gl_per.clone())
    torch.cuda.synchronize()
    for _ in range(2):  # two calls in a row share the same scratch
        for zz, key in ((z, "z"), (None, "noz")):
            v, ref_sum, ref_per = refs[key]
            per = _noalloc(v, zz, x, B)
            tot = _noalloc(v, zz, x, 1)
            torch.cuda.synchronize()
            assert torch.equal(per, ref_per), (key, per, ref_per)
            assert torch.equal(tot, ref_sum), (key, tot, ref_sum)
            want, scale = _host_dot(v, zz, x)
            np.testing.assert_allclose(per.cpu().numpy(), want, rtol=0, atol=1e-6 * scale.max())


@pytest.mark.parametrize("null", ["b", "c"])
def test_noalloc_dot_null_operands_single_slice(null):
    _, _, x, z, g = _inputs(B=1, Cc=2, H=48, W=320, seed=81)
    b = None if null == "b" else z
    c = None if null == "c" else x
    for _ in range(2):
        out = _noalloc(g, b, c, 1)
        torch.cuda.synchronize()
        want, scale = _host_dot(g, b, c)
        assert abs(out.item() - want[0]) <= 1e-6 * scale[0]


def test_noalloc_dot_at_the_row_limit():
    # B * H exactly SENSE_NOALLOC_MAX_ROWS on a narrow grid (W = 4): the last
    # rows of the scratch are used, and the last CTA is partly filled.
    B, H, W = 3, MAX_ROWS // 3, 4
    assert B * H == MAX_ROWS
    gen = torch.Generator(device="cpu").manual_seed(5)
    mk = lambda: torch.randn((B, H, W), dtype=torch.complex64, generator=gen).cuda()
    a, b, c = mk(), mk(), mk()
    for count in (B, 1, B):
        out = _noalloc(a, b, c, count)
        torch.cuda.synchronize()
        want, scale = _host_dot(a, b, c)
        got = out.cpu().numpy()
        if count == 1:
            assert abs(got[0] - want.sum()) <= 1e-6 * scale.sum()
        else:
            np.testing.assert_allclose(got, want, rtol=0, atol=1e-6 * scale.max())


def test_noalloc_refuses_problems_beyond_its_scratch():
    from paper_2202_14005_b300 import _lib

    L = _lib.lib()
    buf = torch.zeros(16, dtype=torch.complex64, device="cuda")
    out = torch.zeros(1, dtype=torch.float64, device="cuda")
    # refused on the host, before any launch
    assert L.sense_dot_re_noalloc(1, MAX_ROWS + 1, 2, _p(buf), None, None, _p(out), 1, None) == -8
    assert L.sense_strerror(-8).decode().startswith("problem exceeds")
