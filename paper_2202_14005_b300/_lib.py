"""ctypes loader for libsense.so (the C ABI declared in include/sense.h).

The library is built in-tree by ``paper_2202_14005_b300.build``.  There is no
fallback: if the shared object is missing or fails to load, importing the
binding raises, so nothing can silently run another implementation.
"""
from __future__ import annotations

import ctypes as C
import os

HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(HERE, "libsense.so")

SENSE_OK = 0
ERRORS = {
    -1: "EINVAL_SHAPE", -2: "EINVAL_PTR", -3: "EINVAL_LAMBDA", -4: "EUNSUPPORTED",
    -5: "ECUDA", -6: "EWORKSPACE", -7: "EINVAL_ARG", -8: "ETOO_LARGE",
}
STATUS_CG_BREAKDOWN = 1
STATUS_NONFINITE = 2
STATUS_DEVICE_TIMEOUT = 4
DENOISER_MODL = 0
DENOISER_VARNET = 1

_vp = C.c_void_p
_i = C.c_int
_f = C.c_float
_dp = C.c_void_p  # device double* passed as an address

# name -> (restype, argtypes)
SIGNATURES = {
    "sense_plan_create": (_i, [C.POINTER(_vp), _i, _i, _i, _i, _vp, _vp, _i, _vp]),
    "sense_plan_create_sets": (_i, [C.POINTER(_vp), _i, _i, _i, _i, _i, _vp, _vp, _i, _vp]),
    "sense_plan_create_toeplitz": (_i, [C.POINTER(_vp), _i, _i, _i, _i, _vp, _vp, _vp]),
    "sense_toeplitz_psf": (_i, [_vp, _i, _i, _i, _vp, _vp]),
    "sense_plan_destroy": (_i, [_vp]),
    "sense_plan_set_stream": (_i, [_vp, _vp]),
    "sense_plan_workspace_bytes": (_i, [_vp, C.POINTER(C.c_size_t)]),
    "sense_plan_set_workspace": (_i, [_vp, _vp, C.c_size_t]),
    "sense_forward": (_i, [_vp, _vp, _vp]),
    "sense_adjoint": (_i, [_vp, _vp, _vp]),
    "sense_normal": (_i, [_vp, _vp, _vp, _f]),
    "cg_dc_solve": (_i, [_vp, _vp, _vp, _vp, _dp, _i, _i, _dp]),
    "cg_dc_solve_backward": (_i, [_vp, _vp, _vp, _vp, _dp, _i, _i, _vp, _dp]),
    "sense_get_status": (_i, [_vp, C.POINTER(_i)]),
    "sense_plan_set_wait_limit": (_i, [_vp, C.c_uint, _i]),
    "ipalm_update_varnet": (_i, [_vp, _vp, _vp, _i, _f, _f, _f, _f, _vp]),
    "sense_fma_probe": (_i, [_i, _i, _vp, _vp]),
    "sense_nudft_forward": (_i, [_vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "sense_nudft_adjoint": (_i, [_vp, _i, _i, _i, _i, _i, _vp, _vp, _vp, _vp]),
    "sense_profile_enable": (_i, [_i]),
    "sense_profile_read": (_i, [C.c_char_p, C.POINTER(C.c_double), C.POINTER(_i)]),
    "sense_kernel_launches": (C.c_longlong, [_i]),
    "denoiser_workspace_bytes": (C.c_size_t, [_i, _i, _i, _i]),
    "denoiser_param_count": (_i, [_i]),
    "denoiser_workspace_offsets": (_i, [_i, _i, _i, _i, C.POINTER(C.c_size_t), C.POINTER(C.c_size_t)]),
    "denoiser_forward": (_i, [_i, _vp, _vp, _vp, _vp, C.c_size_t, _i, _i, _i, _vp]),
    "denoiser_backward": (_i, [_i, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _i, _i, _i, _i, _vp]),
    "denoiser_get_status": (_i, [_vp, _i, _i, _i, _vp, C.POINTER(_i)]),
    "unrolled_step": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp, C.c_size_t]),
    "unrolled_step_backward": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp,
                                    C.c_size_t]),
    "unrolled_step_backward_ex": (_i, [_vp, _i, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _i, _vp,
                                       C.c_size_t, _i]),
    "varnet_workspace_bytes": (C.c_size_t, [_i, _i, _i]),
    "varnet_param_count": (_i, []),
    "varnet_workspace_offsets": (_i, [_i, _i, _i, C.POINTER(C.c_size_t)]),
    "varnet_stage": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t]),
    "varnet_stage_backward": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t]),
    "varnet_stage_backward_ex": (_i, [_vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, _vp, C.c_size_t, _i]),
    "sense_streams_join": (_i, [_vp]),
    "sense_mse_loss": (_i, [_vp, _vp, _vp, _vp, _vp]),
    "sense_normalize_max": (_i, [_vp, _vp, _vp, _vp]),
    "adam_update_f32": (_i, [_vp, _vp, _vp, _vp, C.c_size_t, _f, _f, _f, _f, _i, _vp]),
    "adam_update_f64": (_i, [_vp, _vp, _vp, _vp, C.c_size_t, C.c_double, C.c_double, C.c_double,
                             C.c_double, _i, C.c_double, _vp]),
    "sense_dot_re_noalloc": (_i, [_i, _i, _i, _vp, _vp, _vp, _dp, _i, _vp]),
    "sense_strerror": (C.c_char_p, [_i]),
}


class SenseError(RuntimeError):
    def __init__(self, fn: str, code: int):
        msg = _LIB.sense_strerror(code).decode() if _LIB is not None else ""
        super().__init__(f"{fn} failed: {ERRORS.get(code, code)} ({msg})")
        self.code = code


def load(path: str = LIB_PATH) -> C.CDLL:
    if not os.path.exists(path):
        raise ImportError(f"libsense.so not built at {path}: run `python -m paper_2202_14005_b300.build`")
    lib = C.CDLL(path)
    for name, (res, args) in SIGNATURES.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    return lib


_LIB = None


def lib() -> C.CDLL:
    global _LIB
    if _LIB is None:
        _LIB = load()
    return _LIB


def profile_enable(on: bool = True) -> None:
    check("sense_profile_enable", lib().sense_profile_enable(1 if on else 0))


def profile_read(name: str):
    """(ms, launches) of one kernel group since its last read."""
    ms, n = C.c_double(), C.c_int()
    check("sense_profile_read", lib().sense_profile_read(name.encode(), C.byref(ms), C.byref(n)))
    return ms.value, n.value


def kernel_launches(reset: bool = False) -> int:
    return int(lib().sense_kernel_launches(1 if reset else 0))


def check(fn: str, code: int) -> None:
    if code != SENSE_OK:
        raise SenseError(fn, code)
