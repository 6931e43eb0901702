"""The solve on the grid with both poles (SP_FLAG_POLES) against the oracle.

theta_i = i pi / n_theta, i = 0..n_theta: n_theta + 1 rows, the poles
included.  The GPU path transforms each doubled column (length 2 n_theta) with
one FFT; the oracle takes the naive DFT of the doubled grid and dense or banded
LU per k (oracle.poisson_poles, pinned in test_oracle_poles.py).  Checked
element by element on rough N(0,1) input (pole rows included) from 1 x 2 to
150 x 300, with radices 2, 3, 5, 7, 8 and the large-prime passes (2 n_theta =
66 = 2 * 3 * 11, 2 n_theta = 26 = 2 * 13); against the closed form of a
band-limited series on every row up to the bench's 5000 x 10000 grid and the
largest pole grid (2 n_theta = 12288); the mean of f against the oracle's
surface integral and the paper's worked example; the host-buffer and
allocation-free calls against the device solve; the transpose (adjoint)
against the oracle's element by element, by the dot-product identity up to the
bench's grid, and through autograd against a central difference; and the
calls a pole plan refuses."""

import math

import numpy as np
import pytest
import torch

from oracle import sphere_oracle as O
from synth import sh

pytestmark = pytest.mark.gpu

TOL = 1e-12


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1510_08094_gb300 as sp

    return sp


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


SIZES = [(1, 2), (2, 4), (3, 6), (4, 8), (5, 10), (8, 16), (13, 26), (15, 30), (16, 32), (33, 70), (21, 42),
         (64, 128), (75, 150), (100, 200), (128, 64), (150, 300)]


@pytest.mark.parametrize("nt,nl", SIZES)
def test_pole_solve_matches_oracle_rough_input(sp, nt, nl):
    f = np.random.default_rng(7 * nt + nl).standard_normal((nt + 1, nl))
    u_ref = O.poisson_poles(f)
    plan = sp.Plan(nt, nl, grid="poles")
    assert plan.shape == (nt + 1, nl)
    u = plan.solve(torch.tensor(f, device="cuda")).cpu().numpy()
    if nt == 1:      # no interior row: f does not enter, u = 0
        assert np.abs(u).max() < 1e-15 and np.abs(u_ref).max() < 1e-15
        return
    assert _rel(u, u_ref) < TOL, (nt, nl, _rel(u, u_ref))


@pytest.mark.parametrize("nt,nl,lmax", [(64, 128, 20), (75, 150, 40), (512, 1024, 200)])
def test_pole_solve_matches_oracle_and_closed_form(sp, nt, nl, lmax):
    c = sh.random_sh_coeffs(lmax, 1510080950 + nt)
    f = sh.synthesize(c, nt, nl, grid="poles").numpy()
    ue = sh.synthesize(sh.poisson_exact(c), nt, nl, grid="poles").numpy()
    u = sp.Plan(nt, nl, grid="poles").solve(torch.tensor(f, device="cuda")).cpu().numpy()
    assert _rel(u, ue) < TOL
    if nt <= 128:
        assert _rel(u, O.poisson_poles(f)) < TOL


@pytest.mark.parametrize("nt,nl,lmax", [(5000, 10000, 2000), (6144, 12288, 1000)])
def test_pole_solve_closed_form_full_size(sp, nt, nl, lmax):
    # the bench's grid (2 n_theta = 10000 = 2^4 5^4) and the largest pole grid
    # (2 n_theta = 12288 = 2^12 3): every row, the poles included
    c = sh.random_sh_coeffs(lmax, 1510080942, "inv_sq")
    f = sh.synthesize(c, nt, nl, device="cuda", grid="poles")
    ue = sh.synthesize(sh.poisson_exact(c), nt, nl, device="cuda", grid="poles")
    plan = sp.Plan(nt, nl, grid="poles")
    u = plan.solve(f)
    err = float((u - ue).abs().max() / ue.abs().max())
    assert err < 5e-12, err
    # the pole rows hold the pole values: constant along the row to rounding
    for row in (u[0], u[-1]):
        assert float((row - row.mean()).abs().max()) < 1e-11 * float(ue.abs().max())


@pytest.mark.parametrize("l,m", [(1, 0), (2, 1), (10, -7), (100, 0), (100, 99), (1000, 500)])
def test_single_harmonics(sp, l, m):
    nt, nl = 1200, 2400
    f = sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl, device="cuda", grid="poles")
    u = sp.Plan(nt, nl, grid="poles").solve(f)
    exact = -f / (l * (l + 1))
    # at l = 1000, u is 1e-6 of f, and the rounding of f's zero longitude mean
    # (~1e-16 of f) passes through the k = 0 system, the worst conditioned: a
    # constant of ~1e-18 along each row, 1e-12 of u
    tol = 1e-12 if l < 1000 else 5e-12
    assert float((u - exact).abs().max() / exact.abs().max()) < tol


def test_pole_rows_of_f_do_not_enter(sp):
    nt, nl = 40, 80
    f = torch.randn(nt + 1, nl, dtype=torch.float64, device="cuda")
    g = f.clone()
    g[0] += 3.0
    g[-1] = torch.randn(nl, dtype=torch.float64, device="cuda")
    plan = sp.Plan(nt, nl, grid="poles")
    assert torch.equal(plan.solve(f), plan.solve(g))


@pytest.mark.parametrize("nt,nl", [(2, 4), (5, 10), (33, 70), (64, 128), (150, 300)])
def test_pole_mean_matches_oracle_sum2(sp, nt, nl):
    f = np.random.default_rng(nt).standard_normal((nt + 1, nl)) + 0.5
    ref = O.sum2_poles(f) / (4 * math.pi)
    mean = torch.full((1,), float("nan"), dtype=torch.float64, device="cuda")
    sp.Plan(nt, nl, grid="poles").solve(torch.tensor(f, device="cuda"), mean_out=mean)
    assert abs(float(mean[0]) - ref) < 1e-14 * max(1.0, math.sqrt(nt)) * np.abs(f).max(), (float(mean[0]), ref)


def test_pole_mean_worked_example(sp):
    # int_S (1 + x + y^2 + x^2 y + x^4 + y^5 + (xyz)^2) = 216 pi / 35 (Section 4,
    # Integration): mean 54/35, exact on grids that resolve degree 6
    for nt, nl in [(8, 16), (40, 80), (75, 150)]:
        th = sh.pole_colatitudes(nt)[:, None]
        la = sh.longitudes(nl)[None, :]
        x, y, z = np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la
        f = 1 + x + y ** 2 + x ** 2 * y + x ** 4 + y ** 5 + (x * y * z) ** 2
        mean = torch.empty(1, dtype=torch.float64, device="cuda")
        sp.Plan(nt, nl, grid="poles").solve(torch.tensor(f, device="cuda"), mean_out=mean)
        assert abs(float(mean[0]) - 54.0 / 35.0) < 4e-15, (nt, float(mean[0]))


@pytest.mark.parametrize("nt,nl", [(16, 32), (300, 600)])
def test_pole_host_and_noalloc_solves_match_device(sp, nt, nl):
    from paper_1510_08094_gb300 import _lib

    c = sh.random_sh_coeffs(min(nt // 2, 60), 11 + nt, "inv_sq")
    f = sh.synthesize(c, nt, nl, grid="poles")
    plan = sp.Plan(nt, nl, grid="poles")
    u_dev = plan.solve(f.cuda()).cpu()
    u_host, mean, status = plan.solve_host(f, with_mean=True)
    assert status == _lib.SP_OK and abs(mean) < 1e-14
    assert torch.equal(u_host, u_dev)
    out = torch.empty(nt + 1, nl, dtype=torch.float64, device="cuda")
    plan.solve_noalloc(f.cuda(), out)
    torch.cuda.synchronize()
    assert torch.equal(out.cpu(), u_dev)
    assert plan.launches() == sp.Plan(nt, nl).launches()


@pytest.mark.parametrize("nt,nl", [(1, 2), (2, 4), (3, 6), (5, 10), (8, 16), (13, 26), (33, 70), (64, 128),
                                   (75, 150)])
def test_pole_adjoint_matches_oracle(sp, nt, nl):
    g = np.random.default_rng(31 * nt + nl).standard_normal((nt + 1, nl))
    ref = O.poisson_poles_adjoint(g)
    out = sp.Plan(nt, nl, grid="poles").solve_adjoint(torch.tensor(g, device="cuda")).cpu().numpy()
    scale = max(float(np.abs(ref).max()), 1e-300)
    assert float(np.abs(out - ref).max()) / scale < TOL or float(np.abs(out - ref).max()) < 1e-15 * np.abs(g).max()


@pytest.mark.parametrize("nt,nl", [(512, 1024), (5000, 10000)])
def test_pole_adjoint_dot_product(sp, nt, nl):
    gen = torch.Generator(device="cuda").manual_seed(nt)
    f = torch.randn(nt + 1, nl, dtype=torch.float64, device="cuda", generator=gen)
    g = torch.randn(nt + 1, nl, dtype=torch.float64, device="cuda", generator=gen)
    plan = sp.Plan(nt, nl, grid="poles")
    lhs = float((plan.solve(f) * g).sum())
    rhs = float((f * plan.solve_adjoint(g)).sum())
    assert abs(lhs - rhs) < 1e-12 * abs(lhs), (lhs, rhs)


def test_pole_autograd_matches_central_difference(sp):
    # loss = <u(f), w>: its gradient is S^T w; check one directional derivative
    nt, nl = 40, 80
    gen = torch.Generator(device="cuda").manual_seed(5)
    f = torch.randn(nt + 1, nl, dtype=torch.float64, device="cuda", generator=gen).requires_grad_(True)
    w = torch.randn(nt + 1, nl, dtype=torch.float64, device="cuda", generator=gen)
    d = torch.randn(nt + 1, nl, dtype=torch.float64, device="cuda", generator=gen)
    loss = (sp.poisson(f, grid="poles") * w).sum()
    loss.backward()
    h = 1e-6
    with torch.no_grad():
        lp = float((sp.poisson(f + h * d, grid="poles") * w).sum())
        lm = float((sp.poisson(f - h * d, grid="poles") * w).sum())
    fd = (lp - lm) / (2 * h)
    an = float((f.grad * d).sum())
    assert abs(fd - an) < 1e-7 * max(abs(an), 1.0), (fd, an)


def test_pole_plan_refusals(sp):
    nt, nl = 16, 32
    plan = sp.Plan(nt, nl, grid="poles")
    f = torch.zeros(nt + 1, nl, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        plan.coeffs2(f)
    with pytest.raises(ValueError):
        plan.solve(torch.zeros(nt, nl, dtype=torch.float64, device="cuda"))   # the pole-free shape
    for prec in ("fp32", "fp32_refine"):
        with pytest.raises(RuntimeError):
            sp.Plan(nt, nl, prec, 1, grid="poles")
    with pytest.raises(RuntimeError):
        sp.Plan(6145, 12290, grid="poles")
