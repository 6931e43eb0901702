"""Vector calculus on the GPU (Section 4, vector-valued functions).

Divergence, curl, the curl of a scalar function (eq. CurlScalarF) and the
vorticity against the oracle on band-limited fields and on rough N(0,1) fields
(element by element, sizes spanning several row chunks of the division by
sin theta and a ragged tail),
and against closed forms at sizes the oracle cannot reach: the paper's
Rossby-Haurwitz stream function (Figure VectorCalculus), solid-body rotation,
and div grad = the Laplacian, inverted by the Poisson solver.

Conditioning as for the gradient: the x and y derivative terms carry the
transforms' rounding amplified by up to ~k_max m/pi through M_sin^{-1}, so
their bar is 4e-16 n_theta (n_lambda/2) relative to the field's scale."""

import numpy as np
import pytest
import torch

from oracle import sphere_oracle as O
from synth import sh

pytestmark = pytest.mark.gpu

COND = 4e-16


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1510_08094_gb300 as sp

    return sp


def _xyz(nt, nl):
    th = sh.colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    x, y, z = np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la
    return [torch.tensor(v, device="cuda") for v in (x, y, z)]


def _tol(nt, nl):
    return max(1e-12, COND * nt * (nl // 2))


def _field(nt, nl, lmax, seed):
    return [sh.synthesize(sh.random_sh_coeffs(lmax, seed + c), nt, nl).numpy() for c in range(3)]


def _close(got, ref, tol):
    got = [g.cpu().numpy() for g in got]
    scale = max(np.abs(r).max() for r in ref)
    return max(np.abs(g - r).max() for g, r in zip(got, ref)) / scale < tol


SIZES = [(12, 24, 5), (9, 20, 4), (16, 34, 7), (31, 62, 12), (65, 130, 25), (130, 260, 50)]


@pytest.mark.parametrize("nt,nl,lmax", SIZES)
def test_divergence_matches_oracle(sp, nt, nl, lmax):
    f = _field(nt, nl, lmax, 200 + nt)
    ref = O.divergence(*f)
    got = sp.Plan(nt, nl).divergence(*[torch.tensor(a, device="cuda") for a in f])
    assert _close([got], [ref], 1e-12)


@pytest.mark.parametrize("nt,nl,lmax", SIZES)
def test_curl_matches_oracle(sp, nt, nl, lmax):
    f = _field(nt, nl, lmax, 300 + nt)
    ref = O.curl(*f)
    got = sp.Plan(nt, nl).curl(*[torch.tensor(a, device="cuda") for a in f])
    assert _close(got, ref, 1e-12)


@pytest.mark.parametrize("nt,nl,lmax", SIZES)
def test_scalar_curl_and_vorticity_match_oracle(sp, nt, nl, lmax):
    plan = sp.Plan(nt, nl)
    g = sh.synthesize(sh.random_sh_coeffs(lmax, 400 + nt), nt, nl).numpy()
    assert _close(plan.scalar_curl(torch.tensor(g, device="cuda")), O.scalar_curl(g), 1e-12)
    f = _field(nt, nl, lmax, 500 + nt)
    got = plan.vorticity(*[torch.tensor(a, device="cuda") for a in f])
    assert _close([got], [O.vorticity(*f)], 1e-12)


@pytest.mark.parametrize("nt,nl,lmax", [(65, 130, 25), (130, 260, 50)])
def test_gradient_over_several_row_chunks(sp, nt, nl, lmax):
    f = sh.synthesize(sh.random_sh_coeffs(lmax, 600 + nt), nt, nl).numpy()
    got = sp.Plan(nt, nl).tangential_gradient(torch.tensor(f, device="cuda"))
    assert _close(got, O.tangential_gradient(f), 1e-12)


@pytest.mark.parametrize("nt,nl", [(40, 80), (500, 1000), (5000, 10000)])
def test_rossby_haurwitz(sp, nt, nl):
    x, y, z = _xyz(nt, nl)
    q = x ** 4 - 6 * x ** 2 * y ** 2 + y ** 4
    psi = (z + z * q).contiguous()
    px, py, pz = z * (4 * x ** 3 - 12 * x * y ** 2), z * (4 * y ** 3 - 12 * x ** 2 * y), 1 + q
    exact = [(y * pz - z * py).contiguous(), (z * px - x * pz).contiguous(), (x * py - y * px).contiguous()]
    lap = -2 * z - 30 * z * q
    plan = sp.Plan(nt, nl)
    tol = _tol(nt, nl)
    u = plan.scalar_curl(psi)
    scale = max(float(e.abs().max()) for e in exact)
    for a, b in zip(u, exact):
        assert float((a - b).abs().max()) < tol * scale
    assert float((x * u[0] + y * u[1] + z * u[2]).abs().max()) < tol * scale
    # divergence and vorticity of the exact field
    assert float(plan.divergence(*exact).abs().max()) < tol * scale
    zeta = plan.vorticity(*exact)
    assert float((zeta - lap).abs().max()) < tol * float(lap.abs().max())


@pytest.mark.parametrize("nt,nl", [(20, 40), (1000, 2000), (5000, 10000)])
def test_solid_rotation(sp, nt, nl):
    x, y, z = _xyz(nt, nl)
    f = [(-y).contiguous(), x.contiguous(), torch.zeros_like(z)]
    plan = sp.Plan(nt, nl)
    tol = _tol(nt, nl)
    c = plan.curl(*f)
    for a, b in zip(c, (x * z, y * z, 1 + z * z)):
        assert float((a - b).abs().max()) < 2 * tol
    assert float((plan.vorticity(*f) - 2 * z).abs().max()) < 2 * tol
    assert float(plan.divergence(*f).abs().max()) < tol


@pytest.mark.parametrize("nt,nl,lmax", [(64, 128, 30), (500, 1000, 200)])
def test_poisson_inverts_div_grad(sp, nt, nl, lmax):
    # div grad f = Laplacian f; the solver returns the zero-mean u with
    # Laplacian u = that, i.e. f itself for a series without the l = 0 term
    f = sh.synthesize(sh.random_sh_coeffs(lmax, 700 + nt, "inv_sq"), nt, nl, device="cuda")
    plan = sp.Plan(nt, nl)
    lap = plan.divergence(*plan.tangential_gradient(f))
    u = plan.solve(lap)
    # the second division by sin theta amplifies the first one's noise again
    # before the solve divides mode (j, k) by ~j^2 + k^2: ~eps (n_lambda/2)^2
    tol = max(1e-12, 2.5e-17 * nl ** 2)
    assert float((u - f).abs().max()) < tol * float(f.abs().max())


def test_error_paths(sp):
    from paper_1510_08094_gb300 import _lib

    z = [torch.zeros(8, 16, dtype=torch.float64, device="cuda") for _ in range(3)]
    with pytest.raises(_lib.SpherePoissonError):
        sp.Plan(8, 16, "fp32").divergence(*z)
    plan = sp.Plan(8, 16)
    small = torch.empty(plan.curl_workspace_bytes() - 16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        plan.curl(*z, workspace=small)
    with pytest.raises(ValueError):
        plan.divergence(*z, out=z[0])
    assert float(plan.divergence(*z).abs().max()) == 0.0
    assert all(float(c.abs().max()) == 0.0 for c in plan.curl(*z))
    assert all(float(c.abs().max()) == 0.0 for c in plan.scalar_curl(z[0]))
    assert float(plan.vorticity(*z).abs().max()) == 0.0
    assert plan.curl_workspace_bytes() == plan.gradient_workspace_bytes()


@pytest.mark.parametrize("nt,nl,lmax", [(16, 34, 7), (65, 130, 25), (130, 260, 50)])
def test_chop_matches_oracle(sp, nt, nl, lmax):
    f = _field(nt, nl, lmax, 800 + nt)
    plan = sp.Plan(nt, nl).set_chop(1e-14)
    ft = [torch.tensor(a, device="cuda") for a in f]
    assert _close(plan.curl(*ft), O.curl(*f, chop=1e-14), 1e-12)
    assert _close([plan.divergence(*ft)], [O.divergence(*f, chop=1e-14)], 1e-12)
    assert _close(plan.tangential_gradient(ft[0]), O.tangential_gradient(f[0], chop=1e-14), 1e-12)


@pytest.mark.parametrize("nt,nl", [(500, 1000), (5000, 10000)])
def test_chained_vorticity_of_curl_with_chop(sp, nt, nl):
    # the paper's figure computes vort(curl(psi)); chained derivatives need the
    # chop, or the first call's amplified rounding noise is differentiated again
    x, y, z = _xyz(nt, nl)
    q = x ** 4 - 6 * x ** 2 * y ** 2 + y ** 4
    psi = (z + z * q).contiguous()
    lap = -2 * z - 30 * z * q
    plan = sp.Plan(nt, nl).set_chop(1e-14)
    u = plan.scalar_curl(psi)
    scale = max(float(ui.abs().max()) for ui in u)
    zeta = plan.vorticity(*u)
    err = float((zeta - lap).abs().max() / lap.abs().max())
    div = float(plan.divergence(*u).abs().max()) / scale
    assert err < 1e-11 and div < 1e-11, (err, div)


def test_set_chop_arguments(sp):
    from paper_1510_08094_gb300 import _lib

    plan = sp.Plan(8, 16)
    for bad in (-1e-3, 1.0, float("nan"), float("inf")):
        with pytest.raises(_lib.SpherePoissonError):
            plan.set_chop(bad)
    plan.set_chop(0.0).set_chop(1e-12)
    z = [torch.zeros(8, 16, dtype=torch.float64, device="cuda") for _ in range(3)]
    assert float(plan.vorticity(*z).abs().max()) == 0.0


# Rough N(0,1) input: the maps are linear, so parity must hold for any input,
# not only for band-limited series.  The oracle divides by sin theta with the
# dense M_sin of the m-point window; the kernels form the folded part of that
# solve with the quotient's symmetry, which is all that reaches the results
# (tests/test_msin_readings.py).  Sizes: the degenerate smallest grids (one
# colatitude, 2 x 4, n_lambda = 2), small odd and even ones, and grids spanning
# one, two and three 64-row chunks of the division with ragged tails.  The bar
# is relative to the results' scale (at least the input's), 4e-16 n_theta
# n_lambda/2 as for the series (rounding amplified by the division).
ROUGH = [(1, 2), (1, 8), (2, 4), (6, 2), (3, 6), (4, 8), (5, 10), (8, 16), (33, 70), (64, 128), (65, 130),
         (130, 260)]


@pytest.mark.parametrize("nt,nl", ROUGH)
def test_rough_input_matches_oracle(sp, nt, nl):
    rng = np.random.default_rng(700 + 10 * nt + nl)
    f = [rng.standard_normal((nt, nl)) for _ in range(3)]
    t = [torch.tensor(a, device="cuda") for a in f]
    plan = sp.Plan(nt, nl)
    pairs = {"gradient": (plan.tangential_gradient(t[0]), O.tangential_gradient(f[0])),
             "divergence": ([plan.divergence(*t)], [O.divergence(*f)]),
             "curl": (plan.curl(*t), O.curl(*f)),
             "scalar curl": (plan.scalar_curl(t[0]), O.scalar_curl(f[0])),
             "vorticity": ([plan.vorticity(*t)], [O.vorticity(*f)])}
    for name, (got, ref) in pairs.items():
        got = [g.cpu().numpy() for g in got]
        scale = max(1.0, max(float(np.abs(r).max()) for r in ref))
        err = max(float(np.abs(g - r).max()) for g, r in zip(got, ref)) / scale
        assert err < _tol(nt, nl), (name, err)
