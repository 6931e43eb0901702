"""Planted mistakes: the oracle's pins must catch plausible errors in it.

Each case below plants one mistake in the oracle (on the CPU, through
monkeypatch, for the duration of the test only): a dropped term, a wrong sign,
a transposed operand, a wrong index or normalisation, in the DFS doubling
(eq. BMCsphere), the 2D Fourier coefficients (eq. 2DFourierExpansion), the
banded operator (eq. SylvesterSphericalPoisson, eq. linearSystems), the
zero-mean row (eq. integrationCoeffs, eq. pentdiagonalPlusRankOne), the
transposed map, the vector calculus (Section 4), the pivot pseudoinverse and
the structure-preserving GE (Section 3), the low-rank coefficients and the
refinement reference.  It then re-runs a compact copy of the pins (closed
forms, the printed 216 pi / 35, a trigonometric polynomial's coefficients, the
zero mean, the dense transpose, div grad = Delta, the gradient of x, solid
rotation, the SVD pseudoinverse, exact recovery at the SVD rank, the dense F of
the approximant, the refinement's single-precision start and FP64 limit) at
their own tolerances, and asserts that the named pins fail.  The unmodified
oracle passes every pin (the control case)."""

import math

import numpy as np
import pytest

from oracle import sphere_oracle as O
from synth import sh


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


# --------------------------------------------------------------------------
# Compact copies of the pins; each returns True when the pin holds
# --------------------------------------------------------------------------

def pin_closed_forms(method):
    # Delta Y_l^m = -l(l+1) Y_l^m; odd and even m, zonal and sectoral
    nt, nl = 16, 32
    for l, m in [(1, 0), (3, 0), (5, -3), (6, 4), (9, 9), (2, 1)]:
        f = sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl).numpy()
        u = O.poisson(f, method=method)
        tol = 5e-13 if m == 0 else 1e-13
        if not np.all(np.isfinite(u)) or _rel(u, -f / (l * (l + 1))) > tol:
            return False
    return True


def pin_sum2_worked_example():
    # 216 pi / 35 for the printed polynomial (Section 4, Integration)
    nt, nl = 12, 24
    th = sh.colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    x, y, z = np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la
    f = 1 + x + y ** 2 + x ** 2 * y + x ** 4 + y ** 5 + (x * y * z) ** 2
    return abs(O.sum2(f) - 216 * math.pi / 35) < 1.6e-14


def pin_trig_polynomial():
    # cos(2 theta) sin(3 lambda): coefficients -+ i/4 at (j, k) = (+-2, +-3)
    m, n = 12, 10
    th = O.dfs_theta(m)[:, None]
    la = O.dfs_lambda(n)[None, :]
    X = O.coeffs2(np.cos(2 * th) * np.sin(3 * la))
    ref = np.zeros((m, n), dtype=complex)
    for j in (-2, 2):
        ref[j + m // 2, 3 + n // 2] = -0.25j
        ref[j + m // 2, -3 + n // 2] = 0.25j
    return np.abs(X - ref).max() < 1e-15


def pin_roundtrip():
    v = np.random.default_rng(2).standard_normal((12, 10))
    return np.abs(O.sample(O.coeffs2(v)).real - v).max() < 1e-14


def pin_zero_mean():
    nt, nl = 20, 40
    f = sh.synthesize(sh.random_sh_coeffs(12, 9), nt, nl).numpy()
    return abs(O.sum2(O.poisson(f))) < 1e-14


def pin_dense_transpose():
    nt, nl = 6, 12
    S = O.dense_solution_operator(nt, nl)
    g = np.random.default_rng(0).standard_normal((nt, nl))
    return np.abs(S.T @ g.ravel() - O.poisson_adjoint(g).ravel()).max() < 1e-14


def pin_div_grad():
    nt, nl = 16, 34
    for l, m in [(2, -1), (4, 3)]:
        Y = sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl).numpy()
        if np.abs(O.divergence(*O.tangential_gradient(Y)) + l * (l + 1) * Y).max() > 1e-11 * l * (l + 1):
            return False
    return True


def pin_gradient_of_x():
    # the tangential gradient of x is e_x - x n = (1 - x^2, -x y, -x z)
    nt, nl = 10, 20
    th = sh.colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    x, y, z = np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la
    g = O.tangential_gradient(x)
    return all(np.abs(a - b).max() < 1e-12 for a, b in zip(g, (1 - x * x, -x * y, -x * z)))


def pin_solid_rotation():
    nt, nl = 10, 20
    th = sh.colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    x, y, z = np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la
    c = O.curl(-y, x, 0 * z)
    ok = all(np.abs(a - b).max() < 1e-12 for a, b in zip(c, (x * z, y * z, 1 + z * z)))
    return ok and np.abs(O.vorticity(-y, x, 0 * z) - 2 * z).max() < 1e-12


def pin_pivot_pseudoinverse():
    # the epsilon-pseudoinverse of [[a, b], [b, a]] against numpy's SVD cut
    for a, b in [(1.0, 0.3), (2.0, -1.99), (-0.5, 0.5000001), (0.7, -0.7)]:
        P = O.pivot_pinv(a, b, 0.01)
        R = np.linalg.pinv(np.array([[a, b], [b, a]]), rcond=0.01)
        if not np.all(np.isfinite(P)) or np.abs(P - R).max() > 1e-12 * max(1.0, np.abs(R).max()):
            return False
    return True


def pin_ge_recovery():
    # a band-limited series is recovered after as many terms as its SVD rank
    ft = O.dfs_double(sh.synthesize(sh.random_sh_coeffs(6, 5), 24, 48).numpy())
    terms, e = O.bmc_ge(ft, max_terms=64)
    sv = np.linalg.svd(ft, compute_uv=False)
    rank = sum(int(np.linalg.matrix_rank(P)) for _, P, _, _ in terms)
    return rank == int((sv > 1e-11 * sv[0]).sum()) and float(np.abs(e).max()) < 1e-12 * float(np.abs(ft).max())


def pin_lowrank_coefficients():
    # F from the low-rank factors equals the dense F of the approximant
    nt, nl = 24, 50
    th = sh.colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    x, y, z = np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la
    ft = O.dfs_double(np.cos(1 + 2 * x + np.sin(2 * z)) * (1 + 0.5 * y))
    terms, _ = O.bmc_ge(ft)
    F_dense = O.rhs_coefficients(O.lowrank_values(terms)[nt:])
    return np.abs(O.lowrank_rhs_coefficients(terms, *ft.shape) - F_dense).max() < 1e-13 * np.abs(F_dense).max()


def pin_refinement_converges():
    nt, nl = 32, 64
    f = sh.synthesize(sh.random_sh_coeffs(14, 3), nt, nl).numpy()
    u0, u1, u2 = O.refine_reference(f, 2)
    u64 = O.poisson(f)
    e0, e2 = _rel(u0, u64), _rel(u2, u64)
    return 1e-10 < e0 < 1e-5 and e2 < 1e-13


PINS = {
    "closed forms (dense)": lambda: pin_closed_forms("dense"),
    "closed forms (banded)": lambda: pin_closed_forms("banded"),
    "sum2 worked example": pin_sum2_worked_example,
    "trigonometric polynomial": pin_trig_polynomial,
    "coeffs2/sample round trip": pin_roundtrip,
    "zero mean": pin_zero_mean,
    "dense transpose": pin_dense_transpose,
    "div grad": pin_div_grad,
    "gradient of x": pin_gradient_of_x,
    "solid rotation": pin_solid_rotation,
    "pivot pseudoinverse": pin_pivot_pseudoinverse,
    "GE recovery": pin_ge_recovery,
    "low-rank coefficients": pin_lowrank_coefficients,
    "refinement converges": pin_refinement_converges,
}


def _failing_pins():
    failed = []
    for name, pin in PINS.items():
        with np.errstate(all="ignore"):
            try:
                ok = bool(pin())
            except (np.linalg.LinAlgError, ValueError, FloatingPointError):
                ok = False
        if not ok:
            failed.append(name)
    return failed


# --------------------------------------------------------------------------
# The planted mistakes
# --------------------------------------------------------------------------

_orig = {name: getattr(O, name) for name in
         ("theta_bands_B", "system_matrix", "_bands_of", "integration_weights", "dfs_double",
          "_phase_theta", "coeffs2", "rhs_coefficients", "poisson_adjoint", "tangential_gradient",
          "curl", "pivot_pinv", "bmc_ge", "lowrank_rhs_coefficients", "_solve_columns_T",
          "_replaced_system_apply", "_solve_one_fp32")}


def _bands_swapped(m):
    a, b, c = _orig["theta_bands_B"](m)
    return c, b, a                                  # sub- and super-diagonal exchanged


def _bands_without_first_order(m):
    j = np.arange(-m // 2, m // 2, dtype=np.float64)
    return (j - 2.0) ** 2 / 4.0, -(j * j) / 2.0, (j + 2.0) ** 2 / 4.0   # sin cos d/dtheta dropped


def _system_plus_k2(m, k, reading="B"):
    L = _orig["system_matrix"](m, k, reading)
    return L + 2.0 * k * k * np.eye(m)              # +k^2 instead of -k^2


def _bands_plus_k2(m, k, reading):
    sub, d, sup = _orig["_bands_of"](m, k, reading)
    d = d + 2.0 * k * k
    d[0] = 1.0
    return sub, d, sup


def _weights_without_parity(m):
    j = np.arange(-m // 2, m // 2, dtype=np.float64)
    w = np.zeros(m)
    keep = np.abs(j) != 1
    w[keep] = 1.0 / (1.0 - j[keep] ** 2)           # the (1 + e^{i pi j}) factor dropped
    return w


def _double_without_shift(f):
    f = np.asarray(f, dtype=np.float64)
    nt, n = f.shape
    ft = np.empty((2 * nt, n))
    ft[nt:] = f
    ft[:nt] = f[::-1]                               # lambda + pi shift of the glide reflection dropped
    return ft


def _double_without_reversal(f):
    f = np.asarray(f, dtype=np.float64)
    nt, n = f.shape
    ft = np.empty((2 * nt, n))
    ft[nt:] = f
    ft[:nt] = np.roll(f, -(n // 2), axis=1)         # theta -> -theta row order not reversed
    return ft


def _phase_theta_on_wrong_grid(m):
    j = np.arange(-m // 2, m // 2, dtype=np.int64)[:, None]
    p = np.arange(m, dtype=np.int64)[None, :]
    ang = math.pi * np.mod(j * (2 * p - m), 2 * m).astype(np.float64) / m   # half-cell shift lost
    return np.cos(ang) - 1j * np.sin(ang)


def _coeffs2_half_normalised(values):
    m, n = values.shape
    return _orig["coeffs2"](values) * n              # 1/m instead of 1/(mn)


def _rhs_without_weight(f):
    return _orig["coeffs2"](O.dfs_double(f))        # sin^2(theta) factor dropped


def _adjoint_is_forward(g, reading="B"):
    return O.poisson(g, reading)                    # the map taken as its own transpose


def _adjoint_solves_untransposed(B, reading="B"):
    m, n = B.shape
    Y = np.zeros_like(B, dtype=np.complex128)
    for kk in range(n):
        # M_k instead of M_k^T in the transposed solves
        Y[:, kk] = np.linalg.solve(O.system_matrix(m, kk - n // 2, reading), B[:, kk])
    return Y


def _gradient_xy_swapped(f, chop=0.0):
    gx, gy, gz = _orig["tangential_gradient"](f, chop)
    return gy, gx, gz


def _curl_sign_flipped(f1, f2, f3, chop=0.0):
    c1, c2, c3 = _orig["curl"](f1, f2, f3, chop)
    return c1, c2, -c3


def _pinv_without_cut(a, b, alpha=0.01):
    return np.linalg.inv(np.array([[a, b], [b, a]]))  # the epsilon cut of the pseudoinverse dropped


def _ge_with_unreflected_row(ft, alpha=0.01, rtol=1e-13, max_terms=512):
    # the pivot's second row taken at theta* again instead of at -theta*
    ft = np.asarray(ft, dtype=np.float64)
    m, n = ft.shape
    N, H = m // 2, n // 2
    e = ft.copy()
    terms = []
    for _ in range(max_terms):
        if float(np.abs(e).max()) <= rtol * float(np.abs(ft).max()):
            break
        a = np.roll(e, H, axis=1)
        s1 = np.maximum(np.abs(a + e), np.abs(a - e))[N:, H:]
        i, j = np.unravel_index(int(np.argmax(s1)), s1.shape)
        p, q = N + int(i), H + int(j)
        P = O.pivot_pinv(float(e[p, q - H]), float(e[p, q]), alpha)
        cols = e[:, [q - H, q]].copy()
        rows = e[[p, p], :].copy()
        e = e - cols @ P @ rows
        terms.append((cols, P, rows, (p, q)))
    return terms, e


def _lowrank_without_weight(terms, m, n):
    Et, El = O._phase_theta(m), O._phase_lambda(n)
    F = np.zeros((m, n), dtype=complex)
    for c, P, r, _ in terms:
        F += ((Et @ c) / m) @ P @ ((El @ r.T) / n).T   # sin^2(theta) factor dropped
    return F


def _residual_sign_flipped(X, reading="B"):
    return -_orig["_replaced_system_apply"](X, reading)   # F + M X instead of F - M X


def _fp32_solve_in_fp64(Fk, m, k, reading="B"):
    return O._solve_one(Fk, m, k, reading)                  # the single-precision solve done in FP64


MISTAKES = [
    ("theta_bands_B", _bands_swapped, {"closed forms (dense)", "closed forms (banded)"}),
    ("theta_bands_B", _bands_without_first_order, {"closed forms (dense)", "closed forms (banded)"}),
    ("system_matrix", _system_plus_k2, {"closed forms (dense)"}),
    ("_bands_of", _bands_plus_k2, {"closed forms (banded)"}),
    ("integration_weights", _weights_without_parity, {"sum2 worked example", "closed forms (dense)"}),
    ("dfs_double", _double_without_shift, {"closed forms (dense)"}),
    ("dfs_double", _double_without_reversal, {"closed forms (dense)"}),
    ("_phase_theta", _phase_theta_on_wrong_grid, {"trigonometric polynomial"}),
    ("coeffs2", _coeffs2_half_normalised, {"coeffs2/sample round trip"}),
    ("rhs_coefficients", _rhs_without_weight, {"closed forms (dense)"}),
    ("poisson_adjoint", _adjoint_is_forward, {"dense transpose"}),
    ("_solve_columns_T", _adjoint_solves_untransposed, {"dense transpose"}),
    # div grad is blind to a consistent relabelling of x and y; the gradient of
    # x and the rotation are not
    ("tangential_gradient", _gradient_xy_swapped, {"gradient of x", "solid rotation"}),
    ("curl", _curl_sign_flipped, {"solid rotation"}),
    ("pivot_pinv", _pinv_without_cut, {"pivot pseudoinverse"}),
    ("bmc_ge", _ge_with_unreflected_row, {"GE recovery"}),
    ("lowrank_rhs_coefficients", _lowrank_without_weight, {"low-rank coefficients"}),
    ("_replaced_system_apply", _residual_sign_flipped, {"refinement converges"}),
    ("_solve_one_fp32", _fp32_solve_in_fp64, {"refinement converges"}),
]


def test_unmodified_oracle_passes_every_pin():
    assert _failing_pins() == []


@pytest.mark.parametrize("target,mistake,must_fail", MISTAKES, ids=[m[1].__name__.lstrip("_") for m in MISTAKES])
def test_planted_mistake_is_caught(monkeypatch, target, mistake, must_fail):
    O._theta_cache.clear()
    monkeypatch.setattr(O, target, mistake)
    try:
        failed = set(_failing_pins())
    finally:
        O._theta_cache.clear()
    assert must_fail <= failed, (target, mistake.__name__, sorted(failed))
