"""Numerics of the elimination order the GPU's per-k solve uses, on a numpy model.

The per-k system of eq. linearSystems splits into two chains per wavenumber
(odd j = 1, 3, ... and even j = 2, 4, ...; a_1 = a_2 = 0 decouples them from
j <= 0), tridiagonal in the chain index with the banded entries
a_j = (j-1)(j-2)/4, b_j = -j^2/2 - k^2, c_j = (j+1)(j+2)/4 (reading B, window
j <= m/2 - 1).  The kernels solve each chain by a twisted factorisation: top-down
elimination above the middle row, bottom-up elimination below it, the two
meeting at the middle row, then substitution outwards.  This model of that
order (plain numpy loops, no GPU) is compared with LAPACK's banded LU and with
top-down Thomas at m = 10^4, the bench size.  Measured: the twisted order differs
from LAPACK by <= 3e-14 for k >= 1 and by <= 2e-13 in the k = 0 chains, whose
condition numbers are ~1e9; Thomas agrees with LAPACK exactly (LAPACK does not
pivot on these diagonally dominant bands)."""

import numpy as np
import pytest
import scipy.linalg as sla


def _chain(m, k, first):
    j = np.arange(first, m // 2, 2, dtype=np.float64)
    sub = (j - 1.0) * (j - 2.0) / 4.0
    diag = -(j * j) / 2.0 - float(k * k)
    sup = (j + 1.0) * (j + 2.0) / 4.0
    sub[0] = 0.0                     # a_1 = a_2 = 0: no coupling to j <= 0
    sup[-1] = 0.0                    # X_{m/2} is outside the window
    return sub, diag, sup


def _lapack(l, d, u, r):
    ab = np.zeros((3, d.size))
    ab[0, 1:] = u[:-1]
    ab[1] = d
    ab[2, :-1] = l[1:]
    return sla.solve_banded((1, 1), ab, r)


def _thomas(l, d, u, r):
    n = d.size
    g, y = np.empty(n), np.empty(n)
    g[0], y[0] = d[0], r[0]
    for i in range(1, n):
        w = l[i] / g[i - 1]
        g[i] = d[i] - w * u[i - 1]
        y[i] = r[i] - w * y[i - 1]
    x = np.empty(n)
    x[-1] = y[-1] / g[-1]
    for i in range(n - 2, -1, -1):
        x[i] = (y[i] - u[i] * x[i + 1]) / g[i]
    return x


def _twisted(l, d, u, r):
    n = d.size
    mid = (n - 1) // 2
    g, y, e, z = np.empty(n), np.empty(n), np.empty(n), np.empty(n)
    if mid > 0:                      # top-down above the middle row
        g[0], y[0] = d[0], r[0]
        for i in range(1, mid):
            w = l[i] / g[i - 1]
            g[i] = d[i] - w * u[i - 1]
            y[i] = r[i] - w * y[i - 1]
    if mid < n - 1:                  # bottom-up below it
        e[n - 1], z[n - 1] = d[n - 1], r[n - 1]
        for i in range(n - 2, mid, -1):
            v = u[i] / e[i + 1]
            e[i] = d[i] - v * l[i + 1]
            z[i] = r[i] - v * z[i + 1]
    gm, rm = d[mid], r[mid]          # the meeting row takes both sides
    if mid > 0:
        w = l[mid] / g[mid - 1]
        gm -= w * u[mid - 1]
        rm -= w * y[mid - 1]
    if mid < n - 1:
        v = u[mid] / e[mid + 1]
        gm -= v * l[mid + 1]
        rm -= v * z[mid + 1]
    x = np.empty(n)
    x[mid] = rm / gm
    for i in range(mid - 1, -1, -1):
        x[i] = (y[i] - u[i] * x[i + 1]) / g[i]
    for i in range(mid + 1, n):
        x[i] = (z[i] - l[i] * x[i - 1]) / e[i]
    return x


def test_twisted_order_on_a_small_chain_is_exact():
    # against a dense solve on a chain short enough to check every branch
    for n_rows in (1, 2, 3, 4, 7):
        rng = np.random.default_rng(n_rows)
        d = 4.0 + rng.random(n_rows)
        l, u = rng.random(n_rows), rng.random(n_rows)
        l[0], u[-1] = 0.0, 0.0
        T = np.diag(d) + np.diag(l[1:], -1) + np.diag(u[:-1], 1)
        r = rng.standard_normal(n_rows)
        assert np.abs(_twisted(l, d, u, r) - np.linalg.solve(T, r)).max() < 1e-14


@pytest.mark.parametrize("k", [0, 1, 2, 7, 100, 2500, 4999])
def test_twisted_order_matches_lapack_at_bench_size(k):
    m = 10000
    rng = np.random.default_rng(k)
    for first in (1, 2):
        l, d, u = _chain(m, k, first)
        r = rng.standard_normal(d.size)
        ref = _lapack(l, d, u, r)
        scale = np.abs(ref).max()
        assert np.abs(_thomas(l, d, u, r) - ref).max() <= 1e-15 * scale
        bar = 1e-12 if k == 0 else 1e-13
        assert np.abs(_twisted(l, d, u, r) - ref).max() < bar * scale
