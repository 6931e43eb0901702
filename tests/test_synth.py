"""Pins of the seeded input generator (real spherical harmonics)."""

import math

import numpy as np
import pytest

from synth import sh


def _fejer1_weights(N):
    """Fejer's first rule for int_0^pi g(theta) sin(theta) dtheta on theta_i = (i+1/2)pi/N
    (exact for polynomials in cos(theta) of degree < N)."""
    th = sh.colatitudes(N)
    w = np.ones(N)
    for l in range(1, N // 2 + 1):
        w -= 2.0 * np.cos(2 * l * th) / (4 * l * l - 1)
    return w * 2.0 / N


def test_against_scipy():
    sp = pytest.importorskip("scipy.special")
    if not hasattr(sp, "sph_harm_y"):
        pytest.skip("scipy without sph_harm_y")
    nt, nl = 24, 48
    th = sh.colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    for l, m in [(0, 0), (1, 1), (1, -1), (5, 3), (7, -7), (10, -4), (11, 11)]:
        f = sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl).numpy()
        Y = sp.sph_harm_y(l, abs(m), th, la)
        if m > 0:
            ref = math.sqrt(2) * (-1) ** m * Y.real
        elif m < 0:
            ref = math.sqrt(2) * (-1) ** abs(m) * Y.imag
        else:
            ref = Y.real
        assert np.abs(f - ref).max() < 1e-14


def test_orthonormal_on_grid():
    nt, nl = 32, 64
    L = 10
    w = _fejer1_weights(nt)
    lm = [(l, m) for l in range(L + 1) for m in range(-l, l + 1)]
    Ys = np.stack([sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl).numpy() for l, m in lm])
    quad = (2 * math.pi / nl) * w[None, :, None]
    G = np.einsum("aiq,biq->ab", Ys * quad, Ys)
    assert np.abs(G - np.eye(len(lm))).max() < 1e-13


def test_high_degree_stays_finite_and_normalised():
    nt, nl = 300, 600
    c = sh.single_sh_coeffs(250, 240)
    f = sh.synthesize(c, nt, nl).numpy()
    assert np.isfinite(f).all()
    w = _fejer1_weights(nt)
    norm = (2 * math.pi / nl) * np.sum(w[:, None] * f * f)
    assert abs(norm - 1.0) < 1e-12


def test_seeded_coefficients_are_reproducible():
    a = sh.random_sh_coeffs(30, 1510080941)
    b = sh.random_sh_coeffs(30, 1510080941)
    assert np.array_equal(a, b)
    assert np.all(a[0] == 0)
    ls = np.arange(31)[:, None]
    ms = np.arange(-30, 31)[None, :]
    assert np.all(a[np.abs(ms) > ls] == 0)


def test_turning_point_values_at_degree_2048():
    # Pbar_l^m near its turning point sin(theta) ~ m/l, where the sectoral seed
    # sin^m(theta) is below the normal double range (m ~ 1000): the scaled
    # recurrence must keep full accuracy there.  Reference: mpmath's
    # hypergeometric associated Legendre function at 40 digits, normalised as
    # Pbar_l^m = sqrt((2l+1)/(4 pi) (l-m)!/(l+m)!) P_l^m, without the
    # Condon-Shortley phase.
    mp = pytest.importorskip("mpmath")
    mp.mp.dps = 40
    l, m, nt, nl = 2048, 1024, 64, 4100
    f = sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl).numpy()
    th = sh.colatitudes(nt)
    norm = mp.sqrt((2 * l + 1) / (4 * mp.pi) * mp.factorial(l - m) / mp.factorial(l + m)) * mp.sqrt(2)
    for i in range(9, 14):                    # theta from 26.7 to 37.9 degrees; turning point at 30.0
        p = mp.legenp(l, m, mp.cos(mp.mpf(th[i])), type=2)
        ref = float(abs(p) * norm) * (1.0 if p * (-1) ** m >= 0 else -1.0)
        assert abs(f[i, nl // 2] - ref) < 1e-12, (i, f[i, nl // 2], ref)   # lambda = 0: cos(m lambda) = 1
