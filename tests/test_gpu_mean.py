"""The mean of f reported at the solve boundary (Section 5).

The paper's problem assumes f has zero mean over the sphere (eq.
SphericalLaplacian with eq. integralConstraint2); the solve drops the k = 0,
j = 0 equation either way.  sphere_poisson_solve can write the mean of f,
(1/4 pi) int_S f by the quadrature of eq. integrationCoeffs, to a device
pointer, and sphere_poisson_solve_host returns a warning when that mean is not
zero to rounding.  Checked against the oracle's sum2 (pinned by the paper's
worked example, 216 pi / 35) on rough input and on the worked example itself,
for every precision, on the small and the chunked host paths, and through the
C ABI's argument checks."""

import math
import os

import numpy as np
import pytest
import torch

from oracle import sphere_oracle as O
from synth import sh

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sum2_worked_example.txt")


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1510_08094_gb300 as sp

    return sp


def _golden():
    vals = {}
    for line in open(GOLDEN):
        line = line.strip()
        if line and not line.startswith("#"):
            k, v = line.split("=")
            vals[k.strip()] = float(v)
    return vals


def _worked_example(nt, nl):
    th = sh.colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    x, y, z = np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la
    return 1 + x + y ** 2 + x ** 2 * y + x ** 4 + y ** 5 + (x * y * z) ** 2


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refine"])
@pytest.mark.parametrize("nt,nl", [(1, 2), (2, 4), (5, 10), (33, 70), (64, 128), (150, 300)])
def test_device_mean_matches_oracle_sum2(sp, nt, nl, precision):
    f = np.random.default_rng(nt + nl).standard_normal((nt, nl)) + 0.25
    ref = O.sum2(f) / (4 * math.pi)
    plan = sp.Plan(nt, nl, precision)
    mean = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    ft = torch.tensor(f, device="cuda")
    u = plan.solve(ft, mean_out=mean)
    assert abs(float(mean[0]) - ref) < 1e-14 * np.abs(f).max() * max(1.0, math.sqrt(nt)), (float(mean[0]), ref)
    # the report does not change the solution
    assert torch.equal(u, plan.solve(ft))


def test_worked_example_mean(sp):
    # int_S (1 + x + y^2 + x^2 y + x^4 + y^5 + (xyz)^2) = 216 pi / 35 (Section 4,
    # Integration), so the mean is 54/35; the quadrature is exact for this degree-6
    # polynomial on a grid with n_theta > 7
    g = _golden()
    exact = g["exact_numerator_pi"] * math.pi / g["exact_denominator"] / (4 * math.pi)
    for nt, nl in [(8, 16), (40, 80), (75, 150)]:
        plan = sp.Plan(nt, nl)
        mean = torch.empty(1, dtype=torch.float64, device="cuda")
        plan.solve(torch.tensor(_worked_example(nt, nl), device="cuda"), mean_out=mean)
        assert abs(float(mean[0]) - exact) < 4e-15, (nt, float(mean[0]), exact)


@pytest.mark.parametrize("nt,nl", [(16, 32), (64, 128), (500, 1000)])
def test_host_solve_warns_on_nonzero_mean(sp, nt, nl):
    # n_theta 16: one copy each way; 64 and 500: the chunked, overlapped copies
    from paper_1510_08094_gb300 import _lib

    plan = sp.Plan(nt, nl)
    f = sh.synthesize(sh.random_sh_coeffs(min(nt // 2, 40), 5 + nt, "inv_sq"), nt, nl)
    u, mean, status = plan.solve_host(f, with_mean=True)
    assert status == _lib.SP_OK, (status, mean)
    assert abs(mean) < 1e-15 * float(f.abs().max()) * 10
    assert torch.equal(u, plan.solve_host(f))
    g = f + 3.0
    u3, mean3, status3 = plan.solve_host(g.pin_memory(), with_mean=True)
    assert status3 == _lib.SP_WARN_NONZERO_MEAN
    assert abs(mean3 - 3.0) < 1e-13
    assert "zero mean" in _lib.status_string(status3)
    # u is still written, equal to the device solve of the same f
    assert torch.equal(u3, plan.solve(g.cuda()).cpu())


def test_mean_argument_checks(sp):
    from paper_1510_08094_gb300 import _lib

    lib = _lib.load()
    plan = sp.Plan(16, 32)
    f = torch.zeros(16, 32, dtype=torch.float64, device="cuda")
    u = torch.empty_like(f)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    buf = torch.zeros(4, dtype=torch.float64, device="cuda")
    rc = lib.sphere_poisson_solve(plan._h, f.data_ptr(), u.data_ptr(), ws.data_ptr(), plan.workspace_bytes,
                                  None, buf.data_ptr() + 4)
    assert rc == _lib.SP_ERR_MISALIGNED
    rc = lib.sphere_poisson_solve(plan._h, f.data_ptr(), u.data_ptr(), ws.data_ptr(), plan.workspace_bytes,
                                  None, buf.data_ptr() + 8)
    assert rc == _lib.SP_OK
    torch.cuda.synchronize()
    assert float(buf[1]) == 0.0 and float(buf[0]) == 0.0
    bp = sp.BatchedPlan([(8, 16), (16, 32)])
    packed = torch.zeros(bp.offsets[-1], dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.SpherePoissonError) as e:
        bp.solve(packed, mean_out=buf)
    assert e.value.status == _lib.SP_ERR_UNSUPPORTED
    with pytest.raises(ValueError):
        plan.solve(f, mean_out=buf.float())


@pytest.mark.parametrize("precision", ["fp64", "fp32", "fp32_refine"])
def test_autograd_precisions(sp, precision):
    # the differentiable solve in each precision: the vector-Jacobian product
    # against a central difference of the loss <w, u(f)> along a random direction
    # (linear map, so the difference is exact up to rounding), and against the
    # FP64 adjoint; fp32_refine takes the FP64 adjoint, the transpose of the map
    # it computes to ~1e-13
    nt, nl = 32, 64
    rng = np.random.default_rng(3)
    f = torch.tensor(rng.standard_normal((nt, nl)), device="cuda", requires_grad=True)
    w = torch.tensor(rng.standard_normal((nt, nl)), device="cuda")
    d = torch.tensor(rng.standard_normal((nt, nl)), device="cuda")
    loss = (sp.poisson(f, precision, 2) * w).sum()
    loss.backward()
    tol = 1e-5 if precision == "fp32" else 1e-12
    ref = torch.tensor(O.poisson_adjoint(w.cpu().numpy()), device="cuda")
    assert float((f.grad - ref).abs().max() / ref.abs().max()) < tol
    # the map is linear, so the central difference with h = 1 is <w, S d> up to
    # the form's own rounding, which the bar scales with sum |w| |S d|
    with torch.no_grad():
        lp = float((sp.poisson(f + d, precision, 2) * w).sum())
        lm = float((sp.poisson(f - d, precision, 2) * w).sum())
        scale = float((w.abs() * sp.poisson(d).abs()).sum())
    fd = (lp - lm) / 2.0
    an = float((f.grad * d).sum())
    assert abs(fd - an) < tol * scale, (fd, an, scale)
