"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test checks the oracle against something other than itself: closed-form
solutions (spherical harmonics are Laplacian eigenfunctions), the paper's
printed worked example (216 pi / 35, Section 4), the paper's printed
eigenvalues of M_sin (Section 4 footnote), the Sylvester equation of Section 5
assembled as one dense Kronecker system, a collocation discretisation built
from textbook Fourier differentiation matrices, and invariants (BMC symmetry,
Hermitian symmetry, zero mean, transposition identities).
"""

import math
import os

import numpy as np
import pytest

from oracle import sphere_oracle as O
from synth import sh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_golden(name):
    vals = {}
    with open(os.path.join(GOLDEN, name)) as fh:
        for line in fh:
            line = line.strip()
            if not line or line.startswith("#") or "=" not in line:
                continue
            k, v = (s.strip() for s in line.split("=", 1))
            vals[k] = v
    return vals


def _series(nt, nl, lmax, seed, decay="none"):
    c = sh.random_sh_coeffs(lmax, seed, decay)
    f = sh.synthesize(c, nt, nl).numpy()
    u = sh.synthesize(sh.poisson_exact(c), nt, nl).numpy()
    return f, u


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


# --------------------------------------------------------------------------
# Closed forms: Delta Y_l^m = -l(l+1) Y_l^m
# --------------------------------------------------------------------------

@pytest.mark.parametrize("reading", ["A", "B"])
@pytest.mark.parametrize("method", ["dense", "banded"])
@pytest.mark.parametrize("nt,nl,lmax", [(16, 32, 10), (64, 128, 20), (75, 150, 40), (24, 96, 20)])
def test_sh_series_closed_form(nt, nl, lmax, reading, method):
    f, u_exact = _series(nt, nl, lmax, seed=11 + nt)
    u, F, X, imag = O.poisson(f, reading, method, return_all=True)
    assert _rel(u, u_exact) < 2e-14
    assert imag < 1e-13 * np.abs(u).max()


@pytest.mark.parametrize("l,m", [(1, 0), (1, 1), (1, -1), (2, 0), (5, -3), (12, 7), (29, 0), (29, 29),
                                 (29, -28), (20, -17)])
def test_single_harmonics(l, m):
    # resolved when l + 2 <= n_theta - 1 and |m| < n_lambda / 2
    nt, nl = 32, 64
    c = sh.single_sh_coeffs(l, m)
    f = sh.synthesize(c, nt, nl).numpy()
    u = O.poisson(f)
    # zonal harmonics live in the k = 0 column, whose system has condition number
    # ~8e3 at m = 64 (it grows like m^2.7): rounding in F is amplified accordingly
    tol = 5e-13 if m == 0 else 1e-13
    assert _rel(u, -f / (l * (l + 1))) < tol


def test_unresolved_harmonic_is_not_exact():
    # a planted-failure guard: beyond the resolution limit the closed form must fail,
    # so the closed-form tests above cannot pass vacuously.
    nt, nl = 16, 32
    c = sh.single_sh_coeffs(16, 2)
    f = sh.synthesize(c, nt, nl).numpy()
    u = O.poisson(f)
    assert _rel(u, -f / (16 * 17)) > 1e-6


# --------------------------------------------------------------------------
# The paper's printed values
# --------------------------------------------------------------------------

def test_sum2_worked_example():
    g = _read_golden("sum2_worked_example.txt")
    exact = int(g["exact_numerator_pi"]) * math.pi / int(g["exact_denominator"])
    printed = float(g["printed_value"])
    assert abs(printed - exact) == pytest.approx(float(g["printed_abs_error"]), rel=1e-3)
    for nt, nl in [(8, 16), (12, 24), (33, 70)]:
        th = sh.colatitudes(nt)[:, None]
        la = sh.longitudes(nl)[None, :]
        x = np.cos(la) * np.sin(th)
        y = np.sin(la) * np.sin(th)
        z = np.cos(th) + 0 * la
        f = 1 + x + y ** 2 + x ** 2 * y + x ** 4 + y ** 5 + (x * y * z) ** 2
        assert abs(O.sum2(f) - exact) < 4e-15 * 4


def test_sum2_of_harmonics():
    # int Y_0^0 = sqrt(4 pi); int Y_l^m = 0 for l >= 1
    nt, nl = 20, 40
    y00 = sh.synthesize(sh.single_sh_coeffs(0, 0), nt, nl).numpy()
    assert O.sum2(y00) == pytest.approx(math.sqrt(4 * math.pi), abs=1e-14)
    for l, m in [(1, 0), (2, 0), (4, 0), (3, 2), (6, -5)]:
        y = sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl).numpy()
        assert abs(O.sum2(y)) < 1e-14


@pytest.mark.parametrize("m", [4, 8, 16, 30])
def test_msin_eigenvalues(m):
    g = _read_golden("msin_eigenvalues.txt")
    assert "cos(pi*l/(m+1))" in g["formula"]
    ev = np.sort(np.linalg.eigvals(O.op_Msin(m)).real)
    ref = np.sort(np.cos(math.pi * np.arange(1, m + 1) / (m + 1)))
    assert np.abs(ev - ref).max() < 1e-13
    assert np.abs(np.linalg.eigvals(O.op_Msin(m)).imag).max() < 1e-13


# --------------------------------------------------------------------------
# Structure of the discrete problem
# --------------------------------------------------------------------------

def test_operator_readings_share_interior():
    # reading B's closed-form bands equal the literal matrix products away from
    # the truncation boundary, and the literal product has only offsets 0, +-2
    m = 24
    A = O.theta_operator_A(m)
    a, b, c = O.theta_bands_B(m)
    for r in range(2, m - 2):
        row = np.zeros(m)
        row[r] = b[r]
        row[r - 2] = a[r]
        row[r + 2] = c[r]
        assert np.allclose(A[r], row, atol=1e-12)
    offs = {j - i for i, j in zip(*np.nonzero(np.abs(A) > 1e-14))}
    assert offs <= {-2, 0, 2}


def test_block_structure_of_operator():
    # rows j >= 1 touch only columns >= 1, rows j <= -1 only columns <= -1,
    # column j = 0 has only its diagonal (this is what makes the k = 0 row replaceable)
    m = 32
    for k in [0, 1, 5]:
        L = O.theta_operator_B(m) - k * k * np.eye(m)
        j = np.arange(-m // 2, m // 2)
        pos = j >= 1
        neg = (j <= -1) & (j > -m // 2)
        assert np.all(L[np.ix_(pos, ~pos)] == 0)
        assert np.all(L[np.ix_(neg, ~neg)] == 0)
        col0 = L[:, m // 2].copy()
        col0[m // 2] = 0
        assert np.all(col0 == 0)


def test_sylvester_kronecker_bruteforce():
    # eq. SylvesterSphericalPoisson as one dense (mn x mn) system with the k = 0
    # zeroth row replaced by w^T (eq. pentdiagonalPlusRankOne), versus the per-k solve
    nt, nl = 8, 12
    m, n = 2 * nt, nl
    rng = np.random.default_rng(5)
    f = rng.standard_normal((nt, nl))
    F = O.rhs_coefficients(f)
    L = O.theta_operator_A(m)
    Dn = np.diag(1j * np.arange(-n // 2, n // 2))
    big = np.kron(np.eye(n), L) + np.kron(Dn @ Dn, np.eye(m))   # column-major vec
    rhs = F.reshape(-1, order="F").copy()
    row = (n // 2) * m + m // 2                                    # (j = 0, k = 0)
    big[row, :] = 0.0
    big[row, (n // 2) * m:(n // 2 + 1) * m] = O.integration_weights(m)
    rhs[row] = 0.0
    X = np.linalg.solve(big, rhs).reshape(m, n, order="F")
    assert np.abs(X - O.solve_columns(F, "A", "dense")).max() < 1e-13 * np.abs(X).max()


def _fourier_diff_matrices(N):
    """Trefethen, Spectral Methods in MATLAB, ch. 3: first and second derivative
    matrices on N equispaced points of a 2 pi-periodic grid (N even)."""
    h = 2 * math.pi / N
    i = np.arange(N)
    d = i[:, None] - i[None, :]
    D1 = np.zeros((N, N))
    D2 = np.zeros((N, N))
    off = d != 0
    D1[off] = 0.5 * (-1.0) ** d[off] / np.tan(d[off] * h / 2)
    D2[off] = -0.5 * (-1.0) ** d[off] / np.sin(d[off] * h / 2) ** 2
    D2[~off] = -math.pi ** 2 / (3 * h ** 2) - 1.0 / 6.0
    return D1, D2


def test_collocation_bruteforce():
    # dense collocation discretisation of eq. BMCPoisson on the DFS grid solved by
    # least squares: for resolved input it agrees with the oracle up to a constant
    nt, nl = 10, 16
    m, n = 2 * nt, nl
    f, _ = _series(nt, nl, 6, seed=3)
    th = O.dfs_theta(m)
    D1t, D2t = _fourier_diff_matrices(m)
    _, D2l = _fourier_diff_matrices(n)
    A = (np.kron(np.diag(np.sin(th) ** 2) @ D2t, np.eye(n))
         + np.kron(np.diag(np.sin(th) * np.cos(th)) @ D1t, np.eye(n))
         + np.kron(np.eye(m), D2l))
    b = (np.sin(th)[:, None] ** 2 * O.dfs_double(f)).ravel()
    U = np.linalg.lstsq(A, b, rcond=None)[0].reshape(m, n)
    u_col = U[nt:]
    u = O.poisson(f)
    shift = np.mean(u_col - u)
    assert np.abs(u_col - shift - u).max() < 1e-12 * np.abs(u).max()
    # and the oracle's DFS solution satisfies the collocation equations
    ut = O.dfs_double(u)
    assert np.abs(A @ ut.ravel() - b).max() < 1e-11 * np.abs(b).max()


def test_bmc_and_hermitian_symmetry_of_F():
    nt, nl = 12, 20
    rng = np.random.default_rng(7)
    f = rng.standard_normal((nt, nl))
    F = O.rhs_coefficients(f)
    m, n = F.shape
    for j in range(-m // 2 + 1, m // 2):
        for k in range(-n // 2 + 1, n // 2):
            a = F[j + m // 2, k + n // 2]
            assert abs(F[-j + m // 2, k + n // 2] - (-1) ** k * a) < 1e-15   # BMC fold
            assert abs(F[-j + m // 2, -k + n // 2] - np.conj(a)) < 1e-15     # real data


def test_solution_is_bmc_and_zero_mean():
    nt, nl = 20, 40
    f, _ = _series(nt, nl, 12, seed=9)
    u, F, X, _ = O.poisson(f, return_all=True)
    m, n = X.shape
    scale = np.abs(X).max()
    for j in range(1, m // 2):
        for k in range(-n // 2 + 1, n // 2):
            assert abs(X[-j + m // 2, k + n // 2] - (-1) ** k * X[j + m // 2, k + n // 2]) < 1e-14 * scale
    w = O.integration_weights(m)
    assert abs(w @ X[:, n // 2]) < 1e-15 * scale
    assert abs(O.sum2(u)) < 1e-14


def test_row0_compatibility():
    # the dropped k = 0, j = 0 equation holds for mean-zero input, not otherwise
    nt, nl = 24, 48
    f, _ = _series(nt, nl, 15, seed=21)
    u, F, X, _ = O.poisson(f, return_all=True)
    m, n = X.shape
    R = O.apply_columns(X) - F
    assert abs(R[m // 2, n // 2]) < 1e-14 * np.abs(F).max()
    u1, F1, X1, _ = O.poisson(f + 1.0, return_all=True)
    R1 = O.apply_columns(X1) - F1
    assert abs(R1[m // 2, n // 2]) > 1e-3


def test_readings_agree_for_resolved_input():
    f, _ = _series(40, 80, 30, seed=4)
    assert _rel(O.poisson(f, "A"), O.poisson(f, "B")) < 1e-14


def test_dense_and_banded_agree_on_rough_input():
    rng = np.random.default_rng(8)
    f = rng.standard_normal((30, 44))
    F = O.rhs_coefficients(f)
    for reading in ["A", "B"]:
        Xd = O.solve_columns(F, reading, "dense")
        Xb = O.solve_columns(F, reading, "banded")
        assert np.abs(Xd - Xb).max() < 1e-13 * np.abs(Xd).max()


def test_coeffs2_sample_roundtrip_and_trig_polynomial():
    m, n = 12, 10
    rng = np.random.default_rng(2)
    v = rng.standard_normal((m, n))
    assert np.abs(O.sample(O.coeffs2(v)).real - v).max() < 1e-14
    # cos(2 theta) sin(3 lambda) has coefficients -+ i/4 at (j, k) = (+-2, +-3)
    th = O.dfs_theta(m)[:, None]
    la = O.dfs_lambda(n)[None, :]
    X = O.coeffs2(np.cos(2 * th) * np.sin(3 * la))
    ref = np.zeros((m, n), dtype=complex)
    for j in (-2, 2):
        ref[j + m // 2, 3 + n // 2] = -0.25j
        ref[j + m // 2, -3 + n // 2] = 0.25j
    assert np.abs(X - ref).max() < 1e-15


def test_sampled_columns_match_full_solve():
    f, _ = _series(40, 80, 15, seed=3)
    u = O.poisson(f)
    ks = [0, 1, 2, 7, -5, 39, -39]
    U, F, X = O.sampled_columns(f, ks)
    assert np.abs(U - O.lambda_spectrum(u, ks)).max() < 1e-14


# --------------------------------------------------------------------------
# Transpose of f -> u
# --------------------------------------------------------------------------

def test_adjoint_matches_dense_transpose():
    nt, nl = 6, 12
    S = O.dense_solution_operator(nt, nl)
    rng = np.random.default_rng(0)
    g = rng.standard_normal((nt, nl))
    assert np.abs(S.T @ g.ravel() - O.poisson_adjoint(g).ravel()).max() < 1e-14


def test_adjoint_dot_product():
    nt, nl = 16, 30
    rng = np.random.default_rng(1)
    f = rng.standard_normal((nt, nl))
    g = rng.standard_normal((nt, nl))
    a = np.sum(O.poisson(f) * g)
    b = np.sum(f * O.poisson_adjoint(g))
    assert abs(a - b) < 1e-13 * abs(a)


def test_adjoint_gradient_central_difference():
    # loss(f) = ||S f - u_obs||^2 is quadratic, so central differences are exact up to rounding
    nt, nl = 8, 16
    rng = np.random.default_rng(3)
    f = rng.standard_normal((nt, nl))
    u_obs = rng.standard_normal((nt, nl))

    def loss(x):
        r = O.poisson(x) - u_obs
        return float(np.sum(r * r))

    grad = 2.0 * O.poisson_adjoint(O.poisson(f) - u_obs)
    h = 1e-6
    for _ in range(4):
        d = rng.standard_normal((nt, nl))
        fd = (loss(f + h * d) - loss(f - h * d)) / (2 * h)
        assert abs(fd - np.sum(grad * d)) < 1e-7 * max(1.0, abs(fd))
    for idx in [(0, 0), (3, 7), (7, 15)]:
        e = np.zeros((nt, nl))
        e[idx] = 1.0
        fd = (loss(f + h * e) - loss(f - h * e)) / (2 * h)
        assert abs(fd - grad[idx]) < 1e-7 * max(1.0, abs(fd))


def test_banded_adjoint_matches_dense_adjoint():
    # the banded transposed solves (used above m = 256) against dense LU
    nt, nl = 140, 40
    rng = np.random.default_rng(12)
    g = rng.standard_normal((nt, nl))
    b = O.poisson_adjoint(g)
    old = O.DENSE_MAX_M
    try:
        O.DENSE_MAX_M = 10 ** 6
        a = O.poisson_adjoint(g)
    finally:
        O.DENSE_MAX_M = old
    assert np.abs(a - b).max() < 1e-13 * np.abs(a).max()
    f = rng.standard_normal((nt, nl))
    x = np.sum(O.poisson(f) * g)
    assert abs(x - np.sum(f * b)) < 1e-12 * max(1.0, abs(x))
