"""Host-side checks of the C ABI library (no GPU needed): it builds, loads, exports
every function include/sphere_poisson.h declares, and validates arguments before
touching the device."""

import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names += re.findall(r"^\s*(?:int|const char\s*\*)\s*(sphere_poisson_\w+)\s*\(", src, flags=re.M)
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1510_08094_gb300 import _lib

    return _lib.load()


def test_header_declares_the_boundary():
    names = set(_declared_functions())
    for required in ("sphere_poisson_plan", "sphere_poisson_solve", "sphere_poisson_solve_adjoint",
                     "sphere_poisson_destroy", "sphere_poisson_status_string"):
        assert required in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared_functions():
        assert hasattr(lib, name), name


def test_status_strings(lib):
    from paper_1510_08094_gb300 import _lib

    for code in range(0, -9, -1):
        assert len(_lib.status_string(code)) > 5
    assert "unknown" in _lib.status_string(-999)


# the last four: just past the longest transform (12288 = 2^12 * 3 is the last
# legal length; 12800 = 2^9 * 5^2 factors but is too long; 12289 is prime)
@pytest.mark.parametrize("nt,nl", [(0, 8), (8, 0), (8, 7), (8, 1), (-1, 8), (37, 64), (8, 74),
                                   (20000, 64), (64, 40000), (12800, 64), (12289, 8), (8, 25600),
                                   (8, 24578)])
def test_plan_rejects_bad_sizes(lib, nt, nl):
    from paper_1510_08094_gb300 import _lib

    h = ctypes.c_void_p()
    ws = ctypes.c_size_t(123)
    rc = lib.sphere_poisson_plan(ctypes.byref(h), nt, nl, _lib.SP_FP64, 0, 0, ctypes.byref(ws))
    assert rc == _lib.SP_ERR_BAD_SIZE
    assert h.value is None


def test_plan_argument_checks(lib):
    from paper_1510_08094_gb300 import _lib

    assert lib.sphere_poisson_plan(None, 8, 16, 0, 0, 0, None) == _lib.SP_ERR_NULL
    h = ctypes.c_void_p()
    assert lib.sphere_poisson_plan(ctypes.byref(h), 8, 16, 7, 0, 0, None) == _lib.SP_ERR_UNSUPPORTED
    assert lib.sphere_poisson_plan(ctypes.byref(h), 8, 16, 0, 0, 5, None) == _lib.SP_ERR_BAD_ARG
    # the grid with both poles: FP64 only, 2 n_theta <= 12288
    poles = _lib.SP_FLAG_POLES
    assert lib.sphere_poisson_plan(ctypes.byref(h), 8, 16, _lib.SP_FP32, 0, poles, None) == _lib.SP_ERR_UNSUPPORTED
    assert lib.sphere_poisson_plan(ctypes.byref(h), 8, 16, _lib.SP_FP32_REFINE, 1, poles, None) == \
        _lib.SP_ERR_UNSUPPORTED
    assert lib.sphere_poisson_plan(ctypes.byref(h), 6145, 16, 0, 0, poles, None) == _lib.SP_ERR_BAD_SIZE
    assert h.value is None


def test_calls_reject_null_plan(lib):
    from paper_1510_08094_gb300 import _lib

    buf = ctypes.create_string_buffer(64)
    p = ctypes.addressof(buf)
    assert lib.sphere_poisson_solve(None, p, p, p, 64, None, None) == _lib.SP_ERR_BAD_PLAN
    assert lib.sphere_poisson_solve_adjoint(None, p, p, p, 64, None) == _lib.SP_ERR_BAD_PLAN
    assert lib.sphere_poisson_solve_host(None, p, p, p, 64, None, None) == _lib.SP_ERR_BAD_PLAN
    n = ctypes.c_size_t()
    assert lib.sphere_poisson_workspace_size(None, ctypes.byref(n)) == _lib.SP_ERR_BAD_PLAN
    assert lib.sphere_poisson_destroy(None) == _lib.SP_OK


def test_batched_plan_argument_checks(lib):
    from paper_1510_08094_gb300 import _lib

    h = ctypes.c_void_p()
    nts = (ctypes.c_int * 2)(8, 16)
    nls = (ctypes.c_int * 2)(16, 32)
    bad = (ctypes.c_int * 2)(16, 31)
    plan = lib.sphere_poisson_plan_batched
    assert plan(None, 2, nts, nls, _lib.SP_FP64, 0, 0, None) == _lib.SP_ERR_NULL
    assert plan(ctypes.byref(h), -1, nts, nls, _lib.SP_FP64, 0, 0, None) == _lib.SP_ERR_BAD_ARG
    assert plan(ctypes.byref(h), 2, None, nls, _lib.SP_FP64, 0, 0, None) == _lib.SP_ERR_NULL
    # the batched form exists in FP64 and FP32 + refinement, not in plain FP32
    assert plan(ctypes.byref(h), 2, nts, nls, _lib.SP_FP32, 0, 0, None) == _lib.SP_ERR_UNSUPPORTED
    assert plan(ctypes.byref(h), 2, nts, nls, _lib.SP_FP32_REFINE, 17, 0, None) == _lib.SP_ERR_BAD_ARG
    assert plan(ctypes.byref(h), 2, nts, nls, _lib.SP_FP32_REFINE, -1, 0, None) == _lib.SP_ERR_BAD_ARG
    assert plan(ctypes.byref(h), 2, nts, nls, _lib.SP_FP64, 0, 4, None) == _lib.SP_ERR_BAD_ARG
    assert plan(ctypes.byref(h), 2, nts, bad, _lib.SP_FP32_REFINE, 1, 0, None) == _lib.SP_ERR_BAD_SIZE
    assert h.value is None


def test_grid_on_another_device_is_refused():
    # the binding refuses a tensor that is not on the plan's device before any
    # library call (the plan's tables and kernels live on that device); the
    # library itself returns SP_ERR_BAD_ARG when the current device differs
    import torch

    from paper_1510_08094_gb300 import _check_grid

    t = torch.zeros(2, 4, dtype=torch.float64)
    with pytest.raises(ValueError, match="the plan is on cuda:0"):
        _check_grid(t, (2, 4), "f", torch.device("cuda", 0))
    with pytest.raises(ValueError, match="must be a CUDA tensor"):
        _check_grid(t, (2, 4), "f")
