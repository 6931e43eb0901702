"""The allocation-free solve, through the C ABI.

sphere_poisson_solve_noalloc serves callers that cannot allocate device memory
when they need a solve (no workspace argument; the library's fixed 32 MiB
scratch array is used).  Its results must equal those of the ordinary
sphere_poisson_solve within the parity tolerance, on consecutive calls that
reuse the same scratch array, and oversize grids must be refused cleanly.

This file is collected last, so a run that stops at the first failure has
already run every other test; it also passes on its own in a fresh process.
"""

import ctypes

import numpy as np
import pytest
import torch

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def lib():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    from paper_1510_08094_gb300 import _lib

    return _lib.load()


def _plan(lib, nt, nl, precision=0, sweeps=0):
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    rc = lib.sphere_poisson_plan(ctypes.byref(h), nt, nl, precision, sweeps, 0, ctypes.byref(ws))
    assert rc == 0, rc
    return h, ws.value


def _batched_plan(lib, sizes, precision=0, sweeps=0):
    h = ctypes.c_void_p()
    ws = ctypes.c_size_t()
    nts = (ctypes.c_int * len(sizes))(*[a for a, _ in sizes])
    nls = (ctypes.c_int * len(sizes))(*[b for _, b in sizes])
    rc = lib.sphere_poisson_plan_batched(ctypes.byref(h), len(sizes), nts, nls, precision, sweeps, 0,
                                         ctypes.byref(ws))
    assert rc == 0, rc
    offs = (ctypes.c_size_t * (len(sizes) + 1))()
    assert lib.sphere_poisson_batch_offsets(h, offs) == 0
    return h, ws.value, int(offs[len(sizes)])


def _two_calls(lib, h, ws_bytes, shape):
    """Solve two different inputs with the ordinary and the allocation-free
    entry points and compare each pair (the second call reuses the scratch)."""
    rng = np.random.default_rng(sum(shape) + ws_bytes % 97)
    stream = torch.cuda.current_stream().cuda_stream
    ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
    outs = []
    for call in range(2):
        f = torch.tensor(rng.standard_normal(shape), device="cuda")
        u_ref = torch.empty_like(f)
        u = torch.full_like(f, float("nan"))
        assert lib.sphere_poisson_solve(h, f.data_ptr(), u_ref.data_ptr(), ws.data_ptr(), ws_bytes,
                                        stream, None) == 0
        assert lib.sphere_poisson_solve_noalloc(h, f.data_ptr(), u.data_ptr(), stream) == 0
        torch.cuda.synchronize()
        err = float((u - u_ref).abs().max() / u_ref.abs().max())
        assert err <= TOL, (call, err)
        outs.append(u.clone())
    assert not torch.equal(outs[0], outs[1])


@pytest.mark.parametrize("nt,nl,sweeps", [(64, 128, 1), (256, 512, 2)])
def test_noalloc_refined_plan(lib, nt, nl, sweeps):
    # FP32 + refinement: a workspace of two double-float spectra, an FP32 one
    # and the FP64 zonal column, all inside the fixed scratch
    from paper_1510_08094_gb300 import _lib

    h, ws_bytes = _plan(lib, nt, nl, _lib.SP_FP32_REFINE, sweeps)
    try:
        assert ws_bytes <= _lib.SP_NOALLOC_SCRATCH_BYTES
        _two_calls(lib, h, ws_bytes, (nt, nl))
    finally:
        lib.sphere_poisson_destroy(h)


def test_noalloc_batched_plan(lib):
    # a small batch of uneven spheres: one persistent launch whose per-CTA
    # spectrum slots and work counter live in the fixed scratch
    from paper_1510_08094_gb300 import _lib

    h, ws_bytes, total = _batched_plan(lib, [(32, 64), (48, 96), (16, 32), (64, 128)])
    try:
        assert ws_bytes <= _lib.SP_NOALLOC_SCRATCH_BYTES
        _two_calls(lib, h, ws_bytes, (total,))
    finally:
        lib.sphere_poisson_destroy(h)


@pytest.mark.parametrize("nt,nl", [(64, 128), (75, 150), (512, 1024), (1024, 2048)])
def test_noalloc_matches_solve_on_consecutive_calls(lib, nt, nl):
    from paper_1510_08094_gb300 import _lib

    h, ws_bytes = _plan(lib, nt, nl)
    try:
        assert ws_bytes <= _lib.SP_NOALLOC_SCRATCH_BYTES
        rng = np.random.default_rng(nt + nl)
        stream = torch.cuda.current_stream().cuda_stream
        ws = torch.empty(ws_bytes, dtype=torch.uint8, device="cuda")
        outs = []
        for call in range(2):
            f = torch.tensor(rng.standard_normal((nt, nl)), device="cuda")
            u_ref = torch.empty_like(f)
            u = torch.full_like(f, float("nan"))
            assert lib.sphere_poisson_solve(h, f.data_ptr(), u_ref.data_ptr(), ws.data_ptr(), ws_bytes,
                                            stream, None) == 0
            assert lib.sphere_poisson_solve_noalloc(h, f.data_ptr(), u.data_ptr(), stream) == 0
            torch.cuda.synchronize()
            err = float((u - u_ref).abs().max() / u_ref.abs().max())
            assert err <= TOL, (call, err)
            outs.append(u.clone())
        assert not torch.equal(outs[0], outs[1])  # two different inputs, two answers
    finally:
        lib.sphere_poisson_destroy(h)


def test_noalloc_refuses_grids_beyond_its_scratch(lib):
    from paper_1510_08094_gb300 import _lib

    h, ws_bytes = _plan(lib, 2048, 4096)
    try:
        assert ws_bytes > _lib.SP_NOALLOC_SCRATCH_BYTES
        f = torch.zeros(2048, 4096, dtype=torch.float64, device="cuda")
        u = torch.zeros_like(f)
        rc = lib.sphere_poisson_solve_noalloc(h, f.data_ptr(), u.data_ptr(), None)
        assert rc == _lib.SP_ERR_SCRATCH_LIMIT
        assert "32 MiB" in _lib.status_string(rc)
    finally:
        lib.sphere_poisson_destroy(h)
