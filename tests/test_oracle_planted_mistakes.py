"""Planted mistakes: the oracle's pins must catch plausible errors in it.

Each case below plants one mistake in the oracle (on the CPU, through
monkeypatch, for the duration of the test only): a dropped term, a wrong sign,
a transposed operand, a wrong index or normalisation, in the DFS doubling
(eq. BMCsphere), the 2D Fourier coefficients (eq. 2DFourierExpansion), the
banded operator (eq. SylvesterSphericalPoisson, eq. linearSystems), the
zero-mean row (eq. integrationCoeffs, eq. pentdiagonalPlusRankOne), the
transposed map and the vector calculus (Section 4).  It then re-runs a compact
copy of the pins (closed forms, the printed 216 pi / 35, a trigonometric
polynomial's coefficients, the zero mean, the dense transpose, div grad =
Delta, the gradient of x, solid rotation) at their own tolerances, and asserts
that the named pins fail.  The unmodified oracle passes every pin (the control
case)."""

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
          "curl")}


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


def _gradient_xy_swapped(f, chop=0.0):
    gx, gy, gz = _orig["tangential_gradient"](f, chop)
    return gy, gx, gz


def _curl_sign_flipped(f1, f2, f3, chop=0.0):
    c1, c2, c3 = _orig["curl"](f1, f2, f3, chop)
    return c1, c2, -c3


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
    # div grad is blind to a consistent relabelling of x and y; the gradient of
    # x and the rotation are not
    ("tangential_gradient", _gradient_xy_swapped, {"gradient of x", "solid rotation"}),
    ("curl", _curl_sign_flipped, {"solid rotation"}),
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
