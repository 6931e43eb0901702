"""Pins of the oracle's tangential derivatives (Section 4, Differentiation).

The oracle applies eqs. diff_x, diff_y (and diff_z with the chain-rule sign)
in coefficient space, dividing by sin theta through M_sin^{-1} (eq. Msin).
Pinned against things that do not come from the oracle:
  * the paper's own example: d^t/dx of cos(theta) is -xz;
  * the projection of the 3D gradient of a polynomial onto the tangent plane,
    grad f - (r . grad f) r, evaluated pointwise;
  * tangency, x g_x + y g_y + z g_z = 0, and the printed diff_z sign failing it;
  * Green's identity for spherical harmonics, int |grad Y_l^m|^2 = l(l+1),
    through the oracle's sum2 (itself pinned by 216 pi / 35).
"""

import numpy as np
import pytest

from oracle import sphere_oracle as O
from synth import sh


def _xyz(nt, nl):
    th = sh.colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    return np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la


@pytest.mark.parametrize("nt,nl", [(8, 16), (12, 26)])
def test_paper_example_cos_theta(nt, nl):
    x, y, z = _xyz(nt, nl)
    gx, gy, gz = O.tangential_gradient(z)
    assert np.abs(gx + x * z).max() < 1e-13          # the paper: -cos(l) sin(t) cos(t) = -xz
    assert np.abs(gy + y * z).max() < 1e-13
    assert np.abs(gz - (1 - z * z)).max() < 1e-13


@pytest.mark.parametrize("nt,nl", [(16, 32), (18, 38)])
def test_polynomial_matches_projected_gradient(nt, nl):
    x, y, z = _xyz(nt, nl)
    f = 1 + x + y ** 2 + x ** 2 * y + x ** 4 + y ** 5 + (x * y * z) ** 2
    fx = 1 + 2 * x * y + 4 * x ** 3 + 2 * x * (y * z) ** 2
    fy = 2 * y + x ** 2 + 5 * y ** 4 + 2 * y * (x * z) ** 2
    fz = 2 * z * (x * y) ** 2
    rd = x * fx + y * fy + z * fz
    g = O.tangential_gradient(f)
    for gi, fi, ri in zip(g, (fx, fy, fz), (x, y, z)):
        assert np.abs(gi - (fi - rd * ri)).max() < 1e-12


def test_tangency_of_band_limited_series():
    nt, nl = 20, 40
    x, y, z = _xyz(nt, nl)
    f = sh.synthesize(sh.random_sh_coeffs(8, 17), nt, nl).numpy()
    gx, gy, gz = O.tangential_gradient(f)
    assert np.abs(x * gx + y * gy + z * gz).max() < 1e-12 * np.abs(gx).max()


def test_printed_diff_z_sign_breaks_tangency():
    # with +sin(theta) d/dtheta as printed, d^t z/dz would be -sin^2 and the
    # "gradient" of z would not be tangent: the reading is needed
    nt, nl = 12, 24
    x, y, z = _xyz(nt, nl)
    gx, gy, gz = O.tangential_gradient(z)
    assert np.abs(x * gx + y * gy + z * gz).max() < 1e-13
    assert np.abs(x * gx + y * gy - z * gz).max() > 0.1


@pytest.mark.parametrize("l,m", [(1, 0), (2, 1), (5, -3), (6, 6)])
def test_green_identity_for_harmonics(l, m):
    nt, nl = 24, 48
    Y = sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl).numpy()
    gx, gy, gz = O.tangential_gradient(Y)
    energy = O.sum2(gx ** 2 + gy ** 2 + gz ** 2)
    assert abs(energy - l * (l + 1)) < 1e-11 * l * (l + 1)
    assert abs(O.sum2(Y * Y) - 1.0) < 1e-12


def test_msin_inverse_is_exact_division():
    # (1/sin theta) applied to sin(theta) g in coefficient space returns g, for
    # g band-limited well inside the window (the M_sin^{-1} of eq. Msin)
    m = 32
    rng = np.random.default_rng(3)
    g = np.zeros(m, dtype=complex)
    g[m // 2 - 6: m // 2 + 7] = rng.standard_normal(13) + 1j * rng.standard_normal(13)
    Ms = O.op_Msin(m)
    assert np.abs(np.linalg.solve(Ms, Ms @ g) - g).max() < 1e-13
