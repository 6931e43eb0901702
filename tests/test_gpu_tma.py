"""The TMA column loads of the fused colatitude stages and their bounded wait.

The fused refinement stage has the tensor memory accelerator copy each next
column (16 bytes per row at the spectrum's row stride) into shared memory, and
the fused FP32 stage its two-column tile (16 bytes per row), each waiting on an
mbarrier with a bounded number of polls.  Checked here: solves through those
paths agree with the FP64 solve at each form's bar and leave the plan's device
status at SP_OK, on grids whose column length is and is not a whole number of
256-row boxes; and a wait that runs out (the self-test: one thread polling an
mbarrier that nothing completes) sets the status, which the next status check
reports as SP_ERR_TIMEOUT and clears, with the GPU context still usable
afterwards."""

import pytest
import torch

from synth import sh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1510_08094_gb300 as sp

    return sp


@pytest.mark.parametrize("nt,nl", [(256, 512), (300, 600), (1000, 2000), (5000, 10000)])
def test_tma_refine_matches_fp64_and_status_stays_ok(sp, nt, nl):
    from paper_1510_08094_gb300 import _lib

    c = sh.random_sh_coeffs(min(nt // 3, 400), 1510080960 + nt, "inv_sq")
    f = sh.synthesize(c, nt, nl, device="cuda")
    u64 = sp.Plan(nt, nl, "fp64").solve(f)
    plan = sp.Plan(nt, nl, "fp32_refine", 1)
    for _ in range(2):
        u = plan.solve(f)
    assert plan.device_status() == _lib.SP_OK
    err = float((u - u64).abs().max() / u64.abs().max())
    assert err < 1e-12, err


@pytest.mark.parametrize("nt,nl", [(256, 512), (300, 600), (2000, 4000), (5000, 10000)])
def test_tma_fp32_matches_fp64_and_status_stays_ok(sp, nt, nl):
    # two columns per CTA (the plan's default tile), so the tile comes by TMA
    from paper_1510_08094_gb300 import _lib

    c = sh.random_sh_coeffs(min(nt // 3, 400), 1510080970 + nt, "inv_sq")
    f = sh.synthesize(c, nt, nl, device="cuda")
    u64 = sp.Plan(nt, nl, "fp64").solve(f)
    plan = sp.Plan(nt, nl, "fp32")
    for _ in range(2):
        u = plan.solve(f)
    assert plan.device_status() == _lib.SP_OK
    err = float((u - u64).abs().max() / u64.abs().max())
    assert err < 1e-5, err


def test_wait_that_runs_out_reports_timeout(sp):
    from paper_1510_08094_gb300 import _lib

    nt, nl = 64, 128
    plan = sp.Plan(nt, nl, "fp32_refine", 1)
    lib = _lib.load()
    assert plan.device_status() == _lib.SP_OK
    with torch.cuda.device(plan.device):
        assert lib.sphere_poisson_wait_selftest(plan._h, 1000, None) == _lib.SP_OK
    assert plan.device_status() == _lib.SP_ERR_TIMEOUT
    assert plan.device_status() == _lib.SP_OK            # cleared by the check
    # the context is still usable: a solve after it is correct
    c = sh.random_sh_coeffs(20, 1510080961)
    f = sh.synthesize(c, nt, nl, device="cuda")
    ue = sh.synthesize(sh.poisson_exact(c), nt, nl, device="cuda")
    u = plan.solve(f)
    assert float((u - ue).abs().max() / ue.abs().max()) < 1e-12
    assert plan.device_status() == _lib.SP_OK
    # the host-buffer solve reports a status the self-test left behind
    with torch.cuda.device(plan.device):
        assert lib.sphere_poisson_wait_selftest(plan._h, 1000, None) == _lib.SP_OK
    with pytest.raises(RuntimeError):
        plan.solve_host(f.cpu())
    assert plan.device_status() == _lib.SP_OK
