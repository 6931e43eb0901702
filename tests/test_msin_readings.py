"""The two divisions by sin theta (eq. Msin) on a numpy model, no GPU.

The oracle divides by solving M_sin x = a densely on the window
j in [-m/2, m/2 - 1]; the kernels run the recurrence x_{j-1} = x_{j+1} + 2i a_j
down the folded half j >= 0 from x_{m/2} = x_{m/2-1} = 0 (the model mirrors it
to j < 0 by the quotient's BMC sign).  This model of the recurrence checks the
reading the derivative tests rely on: the two agree to rounding when the
quotient is band-limited in the window (every test function), and on the
degenerate grids 1 x n, 2 x 4 and n x 2 for any input; for rough input on larger
grids they differ, because the two windows' boundary rows differ."""

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


def _recurrence(X):
    m, n = X.shape
    N = m // 2
    a = X @ O.op_Dm(n)
    x = np.zeros_like(a)
    for c in range(n):
        k = c - n // 2
        xs = np.zeros(N + 1, dtype=complex)          # xs[N] = xs[N-1] = 0
        for j in range(N - 1, 0, -1):
            xs[j - 1] = xs[j + 1] + 2j * a[j + N, c]
        x[N:, c] = xs[:N]
        for j in range(1, N):
            # the quotient by sin theta (odd under theta -> -theta) has the
            # opposite BMC sign: Q_{-j,k} = -(-1)^k Q_{j,k}
            x[N - j, c] = -((-1) ** (k % 2)) * xs[j]
    return x


def _diff(nt, nl, f):
    X = _coefficients(f)
    q1, q2 = _dense(X), _recurrence(X)
    q1[0, :] = 0.0
    q2[0, :] = 0.0
    return float(np.abs(q1 - q2).max()), float(np.abs(q1).max())


@pytest.mark.parametrize("nt,nl,lmax", [(8, 16, 5), (12, 24, 9), (16, 34, 13)])
def test_divisions_agree_on_band_limited_input(nt, nl, lmax):
    # f band-limited with (1/sin theta) d/dlambda f inside the window
    f = sh.synthesize(sh.random_sh_coeffs(lmax, 40 + nt), nt, nl).numpy()
    d, s = _diff(nt, nl, f)
    assert d < 1e-13 * s


@pytest.mark.parametrize("nt,nl", [(1, 2), (1, 8), (2, 4), (6, 2)])
def test_divisions_agree_on_degenerate_grids_for_any_input(nt, nl):
    f = np.random.default_rng(nt * 10 + nl).standard_normal((nt, nl))
    d, s = _diff(nt, nl, f)
    assert d < 1e-14 * max(1.0, s)


@pytest.mark.parametrize("nt,nl", [(3, 6), (4, 8), (8, 16)])
def test_divisions_differ_on_rough_input(nt, nl):
    f = np.random.default_rng(nt * 10 + nl).standard_normal((nt, nl))
    d, s = _diff(nt, nl, f)
    assert d > 1e-3 * s
