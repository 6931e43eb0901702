"""The division by sin theta (eq. Msin) on a numpy model, no GPU.

The oracle divides by solving M_sin x = a densely on the window
j in [-m/2, m/2 - 1].  The kernels form only the folded half j >= 0 of the
quotient, whose symmetry Q_{-j,k} = -(-1)^k Q_{j,k} a quotient by sin theta of
a function on the sphere has (Section 2, BMC functions): odd columns by the
recurrence x_{j-1} = x_{j+1} + 2i a_j run down from x_{m/2} = x_{m/2-1} = 0,
even columns (x_0 = 0) by x_{j+1} = x_{j-1} - 2i a_j run up from row 0,
-2 x_1 = 2i a_0.  This model of those recurrences is checked against the
oracle's dense window solve: equal to the part of that solve with the
quotient's symmetry on any input (rough N(0,1) fields included), equal to the
whole solve when the quotient is band-limited, and the rest of the window
solve is shown not to reach the oracle's results on theta > 0."""

import numpy as np
import pytest

from oracle import sphere_oracle as O
from synth import sh


def _coefficients(f):
    X = O.coeffs2(O.dfs_double(f))
    X[0, :] = 0.0                      # theta- and lambda-Nyquist modes dropped
    X[:, 0] = 0.0
    return X


def _dense(X):
    m, n = X.shape
    return np.linalg.solve(O.op_Msin(m), X @ O.op_Dm(n))


def _symmetric_part(q):
    """(q_{j,k} - (-1)^k q_{-j,k}) / 2 on the symmetric window, Nyquist row zero."""
    m, n = q.shape
    sign = (-1.0) ** (np.arange(-n // 2, n // 2) % 2)
    out = np.zeros_like(q)
    out[1:] = 0.5 * (q[1:] - sign[None, :] * q[:0:-1])
    return out


def _recurrence(X):
    """The kernels' folded recurrences, mirrored to j < 0 by the quotient's sign."""
    m, n = X.shape
    N = m // 2
    a = X @ O.op_Dm(n)
    x = np.zeros_like(a)
    for c in range(n):
        k = c - n // 2
        xs = np.zeros(N + 2, dtype=complex)
        if k % 2:                                        # down from xs[N] = xs[N-1] = 0
            for j in range(N - 1, 0, -1):
                xs[j - 1] = xs[j + 1] + 2j * a[j + N, c]
        else:                                            # up from xs[0] = 0 and row 0
            if N > 1:
                xs[1] = -1j * a[N, c]
            for j in range(1, N - 1):
                xs[j + 1] = xs[j - 1] - 2j * a[j + N, c]
        x[N:, c] = xs[:N]
        for j in range(1, N):
            x[N - j, c] = -((-1) ** (k % 2)) * xs[j]
    return x


@pytest.mark.parametrize("nt,nl", [(1, 2), (1, 8), (2, 4), (6, 2), (3, 6), (4, 8), (5, 10), (8, 16), (33, 70),
                                   (64, 128)])
def test_recurrences_are_the_symmetric_part_of_the_window_solve(nt, nl):
    f = np.random.default_rng(nt * 10 + nl).standard_normal((nt, nl))
    X = _coefficients(f)
    q = _symmetric_part(_dense(X))
    r = _recurrence(X)
    assert np.abs(q - r).max() <= 1e-14 * max(1.0, np.abs(q).max())


@pytest.mark.parametrize("nt,nl,lmax", [(8, 16, 5), (12, 24, 9), (16, 34, 13)])
def test_recurrences_equal_the_window_solve_on_band_limited_input(nt, nl, lmax):
    # f band-limited with (1/sin theta) d/dlambda f inside the window: the solve
    # has the quotient's symmetry already and the recurrences reproduce all of it
    f = sh.synthesize(sh.random_sh_coeffs(lmax, 40 + nt), nt, nl).numpy()
    X = _coefficients(f)
    q = _dense(X)
    q[0, :] = 0.0
    assert np.abs(q - _recurrence(X)).max() < 1e-13 * np.abs(q).max()


@pytest.mark.parametrize("nt,nl", [(3, 6), (8, 16), (33, 70)])
def test_only_the_symmetric_part_reaches_the_oracle_results(nt, nl):
    # the rest of the window solve is not small on rough input, yet the oracle's
    # results on theta > 0 are those of the symmetric part alone
    f = np.random.default_rng(nt + nl).standard_normal((nt, nl))
    X = _coefficients(f)
    q = _dense(X)
    qs = _symmetric_part(q)
    assert np.abs(q - qs).max() > 0.1 * np.abs(q).max()
    m, n = X.shape
    c = O.op_Mcos(m) @ (O.op_Dm(m) @ X)
    gx = -(qs @ O.op_Msin(n).T) + c @ O.op_Mcos(n).T
    gy = qs @ O.op_Mcos(n).T + c @ O.op_Msin(n).T
    ref = O.tangential_gradient(f)
    for G, r in zip((gx, gy), ref[:2]):
        G = G.copy()
        G[0, :] = 0.0
        G[:, 0] = 0.0
        v = O.sample(G)[nt:]
        assert np.abs(v.imag).max() < 1e-13 * np.abs(r).max()
        assert np.abs(v.real - r).max() < 1e-13 * np.abs(r).max()
