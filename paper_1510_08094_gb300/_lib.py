"""ctypes binding of the C ABI in include/sphere_poisson.h (argument marshalling only).

Loading fails loudly when the compiled library is missing: there is no
fallback implementation.
"""

from __future__ import annotations

import ctypes
import os

from . import build as _build

_lib = None

SP_OK = 0
SP_WARN_NONZERO_MEAN = 1
SP_ERR_BAD_SIZE = -1
SP_ERR_NULL = -2
SP_ERR_MISALIGNED = -3
SP_ERR_WORKSPACE = -4
SP_ERR_CUDA = -5
SP_ERR_UNSUPPORTED = -6
SP_ERR_BAD_PLAN = -7
SP_ERR_BAD_ARG = -8
SP_ERR_SCRATCH_LIMIT = -9
SP_ERR_TIMEOUT = -10
SP_NOALLOC_SCRATCH_BYTES = 32 << 20

SP_FP64 = 0
SP_FP32 = 1
SP_FP32_REFINE = 2
SP_FLAG_AUTOTUNE = 1
SP_FLAG_POLES = 2

EXPORTED = (
    "sphere_poisson_plan",
    "sphere_poisson_plan_batched",
    "sphere_poisson_batch_offsets",
    "sphere_poisson_workspace_size",
    "sphere_poisson_solve",
    "sphere_poisson_solve_adjoint",
    "sphere_poisson_host_buffer_size",
    "sphere_poisson_solve_host",
    "sphere_poisson_solve_noalloc",
    "sphere_poisson_device_status",
    "sphere_poisson_wait_selftest",
    "sphere_poisson_coeffs2",
    "sphere_poisson_sample",
    "sphere_poisson_sum2",
    "sphere_poisson_gradient_workspace_size",
    "sphere_poisson_tangential_gradient",
    "sphere_poisson_curl_workspace_size",
    "sphere_poisson_set_chop",
    "sphere_poisson_divergence",
    "sphere_poisson_curl",
    "sphere_poisson_scalar_curl",
    "sphere_poisson_vorticity",
    "sphere_poisson_lowrank_workspace_size",
    "sphere_poisson_lowrank_ge",
    "sphere_poisson_solve_lowrank",
    "sphere_poisson_launch_count",
    "sphere_poisson_profile_begin",
    "sphere_poisson_profile_end",
    "sphere_poisson_stage_name",
    "sphere_poisson_pipe_rates",
    "sphere_poisson_destroy",
    "sphere_poisson_status_string",
)


class SpherePoissonError(RuntimeError):
    def __init__(self, status: int, where: str):
        self.status = status
        super().__init__(f"{where}: status {status}: {status_string(status)}")


def library_path() -> str:
    return _build.LIB_PATH


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load (building first if needed) the CUDA library."""
    global _lib
    if _lib is not None:
        return _lib
    path = library_path()
    if not os.path.exists(path) or not _build.up_to_date():
        if not build_if_missing:
            raise RuntimeError(f"CUDA library {path} is not built; run paper_1510_08094_gb300.build")
        _build.build()
    lib = ctypes.CDLL(path)
    vp, sz, i32, u32 = ctypes.c_void_p, ctypes.c_size_t, ctypes.c_int, ctypes.c_uint
    psz = ctypes.POINTER(ctypes.c_size_t)
    lib.sphere_poisson_plan.argtypes = [ctypes.POINTER(vp), i32, i32, i32, i32, u32, psz]
    lib.sphere_poisson_plan_batched.argtypes = [ctypes.POINTER(vp), i32, ctypes.POINTER(ctypes.c_int),
                                                ctypes.POINTER(ctypes.c_int), i32, i32, u32, psz]
    lib.sphere_poisson_batch_offsets.argtypes = [vp, psz]
    lib.sphere_poisson_workspace_size.argtypes = [vp, psz]
    lib.sphere_poisson_solve.argtypes = [vp, vp, vp, vp, sz, vp, vp]
    lib.sphere_poisson_solve_adjoint.argtypes = [vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_host_buffer_size.argtypes = [vp, psz]
    lib.sphere_poisson_solve_host.argtypes = [vp, vp, vp, vp, sz, vp, ctypes.POINTER(ctypes.c_double)]
    lib.sphere_poisson_solve_noalloc.argtypes = [vp, vp, vp, vp]
    lib.sphere_poisson_device_status.argtypes = [vp, vp]
    lib.sphere_poisson_wait_selftest.argtypes = [vp, u32, vp]
    lib.sphere_poisson_coeffs2.argtypes = [vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_sample.argtypes = [vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_sum2.argtypes = [vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_gradient_workspace_size.argtypes = [vp, psz]
    lib.sphere_poisson_tangential_gradient.argtypes = [vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_curl_workspace_size.argtypes = [vp, psz]
    lib.sphere_poisson_set_chop.argtypes = [vp, ctypes.c_double]
    lib.sphere_poisson_divergence.argtypes = [vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_curl.argtypes = [vp, vp, vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_scalar_curl.argtypes = [vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_vorticity.argtypes = [vp, vp, vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_lowrank_workspace_size.argtypes = [vp, i32, psz]
    lib.sphere_poisson_lowrank_ge.argtypes = [vp, vp, i32, ctypes.c_double, ctypes.c_double,
                                              ctypes.POINTER(ctypes.c_int), vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_solve_lowrank.argtypes = [vp, i32, vp, vp, vp, vp, vp, sz, vp]
    lib.sphere_poisson_launch_count.argtypes = [vp, i32, ctypes.POINTER(ctypes.c_int)]
    lib.sphere_poisson_profile_begin.argtypes = [vp, i32]
    lib.sphere_poisson_profile_end.argtypes = [vp, ctypes.POINTER(ctypes.c_double), i32,
                                               ctypes.POINTER(ctypes.c_int), ctypes.POINTER(ctypes.c_int)]
    lib.sphere_poisson_stage_name.argtypes = [vp, i32]
    lib.sphere_poisson_stage_name.restype = ctypes.c_char_p
    lib.sphere_poisson_pipe_rates.argtypes = [ctypes.POINTER(ctypes.c_double), ctypes.POINTER(ctypes.c_double)]
    lib.sphere_poisson_destroy.argtypes = [vp]
    lib.sphere_poisson_status_string.argtypes = [i32]
    lib.sphere_poisson_status_string.restype = ctypes.c_char_p
    for name in EXPORTED:
        if name not in ("sphere_poisson_status_string", "sphere_poisson_stage_name"):
            getattr(lib, name).restype = i32
    _lib = lib
    return lib


def status_string(status: int) -> str:
    return load().sphere_poisson_status_string(int(status)).decode()


def check(status: int, where: str) -> int:
    if status < 0:
        raise SpherePoissonError(status, where)
    return status
