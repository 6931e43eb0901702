"""Pins of the oracle's vector calculus (Section 4, vector-valued functions).

Divergence, curl, the curl of a scalar function (eq. CurlScalarF) and the
vorticity are combinations of the oracle's tangential derivatives; they are
pinned here by what the mathematics fixes, independently of the oracle:
  * div grad Y_l^m = -l(l+1) Y_l^m (spherical harmonics are the eigenfunctions
    of the Laplace-Beltrami operator);
  * the paper's Rossby-Haurwitz stream function psi = cos(theta) +
    sin^4(theta) cos(theta) cos(4 lambda) (Figure VectorCalculus): its curl
    n x grad psi is r x (3D gradient of the polynomial extension of psi), it is
    divergence-free, and its vorticity is the Laplacian of psi,
    -2 cos(theta) - 30 sin^4(theta) cos(theta) cos(4 lambda);
  * solid-body rotation (-y, x, 0): curl = (xz, yz, 1 + z^2) worked out from the
    projected derivatives by hand, vorticity 2z, divergence 0;
  * for any f, curl grad f = n x grad f and the vorticity of grad f is zero
    (with the degree-0 extension of f, D_j = d_j - n_j (n . grad) gives
    eps_ijk D_j d_k f = (n x grad f)_i).
Each pin fails for a swapped component, a wrong sign or a dropped term in the
corresponding combination."""

import numpy as np
import pytest

from oracle import sphere_oracle as O
from synth import sh


def _xyz(nt, nl):
    th = sh.colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    return np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la


def test_unit_normal_is_the_grid_of_the_spherical_coordinates():
    x, y, z = O.unit_normal(6, 10)
    xr, yr, zr = _xyz(6, 10)
    assert max(np.abs(a - b).max() for a, b in zip((x, y, z), (xr, yr, zr))) < 1e-15
    assert np.abs(x * x + y * y + z * z - 1).max() < 1e-15


@pytest.mark.parametrize("l,m", [(1, 0), (2, -1), (4, 3), (7, 7), (9, -5)])
def test_divergence_of_gradient_is_the_laplacian(l, m):
    nt, nl = 16, 34
    Y = sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl).numpy()
    lap = O.divergence(*O.tangential_gradient(Y))
    assert np.abs(lap + l * (l + 1) * Y).max() < 1e-11 * l * (l + 1)


def _rossby_haurwitz(nt, nl):
    x, y, z = _xyz(nt, nl)
    q = x ** 4 - 6 * x ** 2 * y ** 2 + y ** 4                 # sin^4(theta) cos(4 lambda)
    psi = z + z * q
    grad3 = (z * (4 * x ** 3 - 12 * x * y ** 2), z * (4 * y ** 3 - 12 * x ** 2 * y), 1 + q)
    lap = -2 * z - 30 * z * q                                  # l = 1 and l = 5 harmonics
    return (x, y, z), psi, grad3, lap


@pytest.mark.parametrize("nt,nl", [(12, 24), (16, 34)])
def test_rossby_haurwitz_curl_and_vorticity(nt, nl):
    (x, y, z), psi, (px, py, pz), lap = _rossby_haurwitz(nt, nl)
    u = O.scalar_curl(psi)
    exact = (y * pz - z * py, z * px - x * pz, x * py - y * px)   # r x grad psi
    for a, b in zip(u, exact):
        assert np.abs(a - b).max() < 1e-12
    assert np.abs(x * u[0] + y * u[1] + z * u[2]).max() < 1e-12   # tangent
    assert np.abs(O.divergence(*u)).max() < 1e-11
    assert np.abs(O.vorticity(*u) - lap).max() < 1e-11 * np.abs(lap).max()


def test_solid_rotation():
    nt, nl = 10, 20
    x, y, z = _xyz(nt, nl)
    c = O.curl(-y, x, 0 * z)
    for a, b in zip(c, (x * z, y * z, 1 + z * z)):
        assert np.abs(a - b).max() < 1e-12
    assert np.abs(O.vorticity(-y, x, 0 * z) - 2 * z).max() < 1e-12
    assert np.abs(O.divergence(-y, x, 0 * z)).max() < 1e-12
    # the divergence picks up the normal part of a field: div of n itself is 2
    assert np.abs(O.divergence(x, y, z) - 2).max() < 1e-12


def test_curl_of_gradient_is_the_scalar_curl():
    nt, nl = 14, 30
    f = sh.synthesize(sh.random_sh_coeffs(6, 1510080948), nt, nl).numpy()
    g = O.tangential_gradient(f)
    c, s = O.curl(*g), O.scalar_curl(f)
    scale = max(np.abs(gi).max() for gi in g)
    for a, b in zip(c, s):
        assert np.abs(a - b).max() < 1e-11 * scale
    assert np.abs(O.vorticity(*g)).max() < 1e-11 * scale


def test_chop_discards_only_the_small_coefficients():
    # a harmonic plus a 1e-10 copy of a high one: with the chop at 1e-8 the
    # gradient is that of the harmonic alone; without it the small part stays
    nt, nl = 24, 48
    Y = sh.synthesize(sh.single_sh_coeffs(3, 1), nt, nl).numpy()
    H = sh.synthesize(sh.single_sh_coeffs(20, 7), nt, nl).numpy()
    g_ref = O.tangential_gradient(Y)
    g_chop = O.tangential_gradient(Y + 1e-10 * H, chop=1e-8)
    g_plain = O.tangential_gradient(Y + 1e-10 * H)
    g_h = O.tangential_gradient(H)
    for a, b, c in zip(g_chop, O.tangential_gradient(Y, chop=1e-8), g_ref):
        assert np.abs(a - b).max() < 1e-15
        # the plain map carries the transforms' noise amplified (~1e-14 here)
        assert np.abs(a - c).max() < 1e-13
    for a, b, h in zip(g_plain, g_ref, g_h):
        assert np.abs((a - b) - 1e-10 * h).max() < 1e-13
        assert np.abs(1e-10 * h).max() > 1e-10


def test_chained_rossby_haurwitz_with_chop():
    (x, y, z), psi, _, lap = _rossby_haurwitz(16, 34)
    u = O.scalar_curl(psi, chop=1e-14)
    assert np.abs(O.vorticity(*u, chop=1e-14) - lap).max() < 1e-11 * np.abs(lap).max()
    assert np.abs(O.divergence(*u, chop=1e-14)).max() < 1e-11
