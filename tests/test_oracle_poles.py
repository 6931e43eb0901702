"""The oracle on the grid with both poles (Section 2's DFS grid sampled on
theta in [0, pi]), pinned by what does not depend on the oracle itself.

  * Its 2D DFT on the doubled grid theta_p = -pi + 2 pi p / m returns the
    coefficients of a trigonometric polynomial evaluated directly with
    numpy's exp at those angles, and its inverse returns the samples.
  * Delta Y_l^m = -l(l+1) Y_l^m: the solve of a band-limited series sampled
    on the grid (poles included) is the closed form on every row, the pole
    rows included.
  * The samples of f on the pole rows are multiplied by sin^2 theta = 0: they
    do not change u.
  * Its surface integral of the printed polynomial is 216 pi / 35.
  * Its transpose of f -> u equals the dense matrix of the solve, built
    column by column from unit inputs, transposed.
  * u is the same function whichever grid samples f: on the rows both grids
    share no point, so the check is the interpolant, evaluated from the
    pole-grid coefficients at the pole-free colatitudes, against the
    pole-free solve of the same band-limited f.
Four plausible mistakes in the pole-grid code (the pole-free grid's phase,
the glide reflection without its half-turn in longitude, the south pole row
taken from the wrong end of the doubled grid, the transpose's fold without the
half-turn) are planted and caught."""

import math

import numpy as np
import pytest

from oracle import sphere_oracle as O
from synth import sh


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def pin_dft_of_trig_polynomial():
    m, n = 12, 10
    rng = np.random.default_rng(7)
    c = np.zeros((m, n), dtype=complex)
    c[1:, 1:] = rng.standard_normal((m - 1, n - 1)) + 1j * rng.standard_normal((m - 1, n - 1))
    th = -math.pi + 2 * math.pi * np.arange(m) / m
    la = sh.longitudes(n)
    j = np.arange(-m // 2, m // 2)
    k = np.arange(-n // 2, n // 2)
    v = np.exp(1j * np.outer(th, j)) @ c @ np.exp(1j * np.outer(k, la))
    return _rel(O.coeffs2_poles(v), c) < 1e-13 and _rel(O.sample_poles(c), v) < 1e-13


def pin_closed_forms():
    nt, nl = 16, 32
    for l, m in [(1, 0), (2, 1), (3, -2), (5, 3), (6, 0), (7, -7)]:
        f = sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl, grid="poles").numpy()
        u = O.poisson_poles(f)
        if u.shape != f.shape or _rel(u, -f / (l * (l + 1))) > 1e-12:
            return False
    return True


def pin_series():
    nt, nl = 24, 48
    c = sh.random_sh_coeffs(10, 1510080949)
    f = sh.synthesize(c, nt, nl, grid="poles").numpy()
    ue = sh.synthesize(sh.poisson_exact(c), nt, nl, grid="poles").numpy()
    return _rel(O.poisson_poles(f), ue) < 1e-12


def pin_same_function_on_both_grids():
    nt, nl = 20, 40
    c = sh.random_sh_coeffs(8, 1510080948)
    fp = sh.synthesize(c, nt, nl, grid="poles").numpy()
    fs = sh.synthesize(c, nt, nl).numpy()
    Xp = O.solve_columns(O.rhs_coefficients_poles(fp))
    us = O.poisson(fs)
    # the pole-grid interpolant at theta = (i + 1/2) pi / n_theta
    th = sh.colatitudes(nt)
    j = np.arange(-nt, nt)
    k = np.arange(-nl // 2, nl // 2)
    la = sh.longitudes(nl)
    up = (np.exp(1j * np.outer(th, j)) @ Xp @ np.exp(1j * np.outer(k, la))).real
    return _rel(up, us) < 1e-12


def pin_sum2_worked_example():
    # the printed polynomial integrates to 216 pi / 35 (Section 4, Integration);
    # exact on a grid that resolves its degree, poles included
    nt, nl = 12, 24
    th = sh.pole_colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    x, y, z = np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la
    f = 1 + x + y ** 2 + x ** 2 * y + x ** 4 + y ** 5 + (x * y * z) ** 2
    return abs(O.sum2_poles(f) - 216 * math.pi / 35) < 2e-14


def pin_dense_transpose():
    # the transpose of f -> u built column by column from the solve itself
    rng = np.random.default_rng(11)
    for nt, nl in [(3, 6), (4, 8), (8, 16)]:
        size = (nt + 1) * nl
        S = np.zeros((size, size))
        for c in range(size):
            e = np.zeros(size)
            e[c] = 1.0
            S[:, c] = O.poisson_poles(e.reshape(nt + 1, nl)).ravel()
        g = rng.standard_normal((nt + 1, nl))
        if np.abs(O.poisson_poles_adjoint(g).ravel() - S.T @ g.ravel()).max() > 1e-13 * np.abs(S).max() * size:
            return False
    return True


PINS = [pin_dft_of_trig_polynomial, pin_closed_forms, pin_series, pin_same_function_on_both_grids,
        pin_sum2_worked_example, pin_dense_transpose]


def test_pole_grid_oracle_passes_its_pins():
    for pin in PINS:
        assert pin(), pin.__name__


def test_grid_with_poles_has_both_poles():
    th = sh.pole_colatitudes(8)
    assert th.shape == (9,) and th[0] == 0.0 and th[-1] == math.pi
    assert np.array_equal(O.pole_colatitudes(8), th)


def test_pole_rows_do_not_enter():
    nt, nl = 16, 32
    rng = np.random.default_rng(3)
    f = rng.standard_normal((nt + 1, nl))
    g = f.copy()
    g[0] += rng.standard_normal(nl) * 5
    g[-1] -= 7.0
    assert np.array_equal(O.rhs_coefficients_poles(f), O.rhs_coefficients_poles(g))


def test_odd_wavenumbers_vanish_at_the_poles():
    # the doubled solution is BMC (X_{-j,k} = (-1)^k X_{j,k}), so its odd-k
    # content cancels pairwise at theta = 0 and theta = pi, for any f
    nt, nl = 16, 32
    f = np.random.default_rng(5).standard_normal((nt + 1, nl))
    u = O.poisson_poles(f)
    for row in (u[0], u[-1]):
        spec = np.fft.fft(row)
        odd = np.abs(spec[1::2]).max()
        assert odd < 1e-12 * np.abs(spec).max()


def _phase_of_pole_free_grid(m):
    return O._phase_theta(m)


def _double_without_half_turn(f):
    f = np.asarray(f, dtype=np.float64)
    nt = f.shape[0] - 1
    ft = np.empty((2 * nt, f.shape[1]))
    ft[nt:] = f[:nt]
    ft[:nt] = f[nt:0:-1]
    return ft


def _poisson_poles_south_row_from_p_last(f, reading="B", method="auto", return_all=False):
    f = np.asarray(f, dtype=np.float64)
    nt = f.shape[0] - 1
    X = O.solve_columns(O.rhs_coefficients_poles(f), reading, method)
    U = O.sample_poles(X)
    return np.concatenate([U[nt:], U[-1:]], axis=0).real


def _adjoint_fold_without_half_turn(g, reading="B"):
    g = np.asarray(g, dtype=np.float64)
    rows, n = g.shape
    nt = rows - 1
    m = 2 * nt
    Gfull = np.zeros((m, n), dtype=np.complex128)
    Gfull[nt:] = g[:nt]
    Gfull[0] += g[nt]
    Et = O._phase_theta_poles(m)
    El = O._phase_lambda(n)
    Fbar = O._solve_columns_T(Et @ Gfull @ El.T, reading)
    Fbar[m // 2, n // 2] = 0.0
    Fbar[0, :] = 0.0
    vbar = np.sin(O.dfs_theta_poles(m))[:, None] ** 2 * ((Et.conj().T @ Fbar @ El.conj()) / (m * n)).real
    out = np.zeros((rows, n))
    out[:nt] += vbar[nt:]
    out[nt:0:-1] += vbar[:nt]
    return out


MISTAKES = [
    ("_phase_theta_poles", _phase_of_pole_free_grid, {"pin_dft_of_trig_polynomial", "pin_closed_forms"}),
    ("dfs_double_poles", _double_without_half_turn, {"pin_closed_forms", "pin_series"}),
    ("poisson_poles", _poisson_poles_south_row_from_p_last, {"pin_closed_forms", "pin_series"}),
    ("poisson_poles_adjoint", _adjoint_fold_without_half_turn, {"pin_dense_transpose"}),
]


@pytest.mark.parametrize("target,mistake,must_fail", MISTAKES, ids=[m[1].__name__.lstrip("_") for m in MISTAKES])
def test_planted_mistake_is_caught(monkeypatch, target, mistake, must_fail):
    monkeypatch.setattr(O, target, mistake)
    failing = {pin.__name__ for pin in PINS if not pin()}
    assert must_fail <= failing, (target, failing)
