"""Tangential derivatives on the GPU (Section 4, Differentiation).

Against the oracle's coefficient-space d^t/dx, d^t/dy, d^t/dz on band-limited
spherical-harmonic series (where the division by sin theta through M_sin^{-1}
is exact) and on rough N(0,1) samples, and against closed forms at sizes the
oracle cannot reach: the paper's d^t cos(theta)/dx = -xz, projected gradients
of a polynomial, tangency and Green's identity.

Conditioning: M_sin^{-1} (eq. Msin) has norm ~m/pi and d/dlambda multiplies
column k by k, so the rounding noise the transforms leave in every coefficient
reaches the x and y components amplified by up to ~k_max m/pi; their bar is
4e-16 n_theta (n_lambda/2) (2e-9 measured at 5000 x 10000, the same growth in
a numpy model of the algorithm).  The z component has no division; d/dtheta
multiplies row j by j <= n_theta, so its bar (and that of tangency, which the
division terms do not enter) is 2e-15 n_theta (4e-12 measured at 5000)."""

COND = 4e-16

import numpy as np
import pytest
import torch

from oracle import sphere_oracle as O
from synth import sh

pytestmark = pytest.mark.gpu


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


@pytest.mark.parametrize("nt,nl,lmax", [(12, 24, 5), (16, 34, 7), (9, 20, 4), (33, 70, 14), (64, 128, 30),
                                        (22, 58, 9), (31, 62, 12)])
def test_matches_oracle_on_band_limited_series(sp, nt, nl, lmax):
    f = sh.synthesize(sh.random_sh_coeffs(lmax, 100 + nt), nt, nl).numpy()
    ref = O.tangential_gradient(f)
    got = sp.Plan(nt, nl).tangential_gradient(torch.tensor(f, device="cuda"))
    for g, r in zip(got, ref):
        assert np.abs(g.cpu().numpy() - r).max() < 1e-12 * np.abs(r).max()


@pytest.mark.parametrize("nt,nl", [(3, 6), (8, 16), (33, 70), (64, 128), (130, 260)])
def test_matches_oracle_on_rough_input(sp, nt, nl):
    # N(0,1) samples: not band-limited, so the division by sin theta meets the
    # window's boundary rows; the kernels' folded division is the part of the
    # oracle's window solve that reaches the results
    f = np.random.default_rng(900 + nt).standard_normal((nt, nl))
    ref = O.tangential_gradient(f)
    got = sp.Plan(nt, nl).tangential_gradient(torch.tensor(f, device="cuda"))
    scale = max(float(np.abs(r).max()) for r in ref)
    for g, r in zip(got, ref):
        assert np.abs(g.cpu().numpy() - r).max() < _tol_xy(nt, nl) * scale


def _tol_xy(nt, nl):
    return max(1e-12, COND * nt * (nl // 2))


def _tol_z(nt):
    return max(1e-12, 2e-15 * nt)


@pytest.mark.parametrize("nt,nl", [(40, 80), (500, 1000), (5000, 10000)])
def test_paper_example(sp, nt, nl):
    x, y, z = _xyz(nt, nl)
    gx, gy, gz = sp.Plan(nt, nl).tangential_gradient(z.contiguous())
    assert float((gx + x * z).abs().max()) < _tol_xy(nt, nl)     # -cos(l) sin(t) cos(t) = -xz
    assert float((gy + y * z).abs().max()) < _tol_xy(nt, nl)
    assert float((gz - (1 - z * z)).abs().max()) < _tol_z(nt)
    assert float((x * gx + y * gy + z * gz).abs().max()) < _tol_z(nt)


@pytest.mark.parametrize("nt,nl", [(128, 256), (1000, 2000), (5000, 10000)])
def test_polynomial_projected_gradient(sp, nt, nl):
    x, y, z = _xyz(nt, nl)
    f = 1 + x + y ** 2 + x ** 2 * y + x ** 4 + y ** 5 + (x * y * z) ** 2
    fx = 1 + 2 * x * y + 4 * x ** 3 + 2 * x * (y * z) ** 2
    fy = 2 * y + x ** 2 + 5 * y ** 4 + 2 * y * (x * z) ** 2
    fz = 2 * z * (x * y) ** 2
    rd = x * fx + y * fy + z * fz
    g = sp.Plan(nt, nl).tangential_gradient(f.contiguous())
    for c, (gi, fi, ri) in enumerate(zip(g, (fx, fy, fz), (x, y, z))):
        exact = fi - rd * ri
        tol = _tol_z(nt) if c == 2 else _tol_xy(nt, nl)
        assert float((gi - exact).abs().max() / exact.abs().max()) < tol, c
    scale = max(float(gi.abs().max()) for gi in g)
    assert float((x * g[0] + y * g[1] + z * g[2]).abs().max()) < _tol_z(nt) * scale


def test_tangency_of_series(sp):
    # a band-limited series synthesised to full accuracy (at 5000 x 10000 the
    # synthesised samples carry ~2e-9 in the top theta modes, which d/dtheta
    # would amplify; the polynomial test covers that size)
    nt, nl = 1000, 2000
    f = sh.synthesize(sh.random_sh_coeffs(400, 1510080942, "inv_sq"), nt, nl, device="cuda")
    x, y, z = _xyz(nt, nl)
    gx, gy, gz = sp.Plan(nt, nl).tangential_gradient(f)
    scale = max(float(gx.abs().max()), float(gy.abs().max()), float(gz.abs().max()))
    assert float((x * gx + y * gy + z * gz).abs().max()) < 1e-12 * scale


@pytest.mark.parametrize("l,m", [(3, 1), (10, -7), (20, 20)])
def test_green_identity(sp, l, m):
    nt, nl = 64, 128
    plan = sp.Plan(nt, nl)
    Y = sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl, device="cuda")
    gx, gy, gz = plan.tangential_gradient(Y)
    assert abs(plan.sum2(gx * gx + gy * gy + gz * gz) - l * (l + 1)) < 1e-11 * l * (l + 1)


def test_error_paths(sp):
    from paper_1510_08094_gb300 import _lib

    f = torch.zeros(8, 16, dtype=torch.float64, device="cuda")
    with pytest.raises(_lib.SpherePoissonError):
        sp.Plan(8, 16, "fp32").tangential_gradient(f)
    plan = sp.Plan(8, 16)
    small = torch.empty(16, dtype=torch.uint8, device="cuda")
    with pytest.raises(ValueError):
        plan.tangential_gradient(f, workspace=small)
    out = plan.tangential_gradient(f)
    assert all(float(o.abs().max()) == 0.0 for o in out)
