"""The transforms on their own: coeffs2 / sample / sum2 (Section 4).

coeffs2 must equal the oracle's naive 2D DFT of the doubled-up function
(same index convention, j >= 0 and the half spectrum in k); sample must
invert it on band-limited input; sum2 must reproduce the paper's worked
example, 216 pi / 35 (tests/golden/sum2_worked_example.txt)."""

import math
import os

import numpy as np
import pytest
import torch

from oracle import sphere_oracle as O
from synth import sh

pytestmark = pytest.mark.gpu
GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sum2_worked_example.txt")


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1510_08094_gb300 as sp

    return sp


@pytest.mark.parametrize("nt,nl", [(24, 48), (33, 70), (64, 128), (5, 10), (22, 58), (1, 2)])
def test_coeffs2_matches_oracle(sp, nt, nl):
    f = np.random.default_rng(nt).standard_normal((nt, nl))
    X = O.coeffs2(O.dfs_double(f))               # [j + m/2, k + n/2]
    m, n = X.shape
    C = sp.Plan(nt, nl).coeffs2(torch.tensor(f, device="cuda")).cpu().numpy()
    ref = np.empty((nt, n // 2 + 1), dtype=complex)
    ref[:, : n // 2] = X[m // 2:, n // 2:]
    ref[:, n // 2] = X[m // 2:, 0]               # k = -n/2
    got = C[:, : n // 2 + 1]
    assert np.abs(got - ref).max() < 1e-14 * max(1.0, np.abs(ref).max()) * 10


def test_sample_inverts_coeffs2_on_band_limited_input(sp):
    nt, nl = 48, 96
    c = sh.random_sh_coeffs(30, 9)
    f = sh.synthesize(c, nt, nl, device="cuda")
    plan = sp.Plan(nt, nl)
    back = plan.sample(plan.coeffs2(f))
    assert float((back - f).abs().max() / f.abs().max()) < 1e-13


def _random_sphere_coefficients(nt, nl, rng):
    """Random coefficients in the coeffs2 layout [n_theta, Kp] of a real BMC
    function: complex N(0,1) entries, except X_{0,k} = 0 for odd k (the BMC
    symmetry X_{-j,k} = (-1)^k X_{j,k} at j = 0), a real k = 0 column and a
    k = -n/2 column that is real for even n/2 and imaginary for odd n/2 (the
    aliased longitude Nyquist mode of a real function)."""
    L = nl // 2
    kp = (L + 2) // 2 * 2
    X = np.zeros((nt, kp), dtype=complex)
    X[:, : L + 1] = rng.standard_normal((nt, L + 1)) + 1j * rng.standard_normal((nt, L + 1))
    X[0, 1: L + 1: 2] = 0.0
    X[:, 0] = X[:, 0].real
    X[:, L] = X[:, L].real if L % 2 == 0 else 1j * X[:, L].imag
    if L % 2:
        X[0, L] = 0.0
    return X


def _full_window(X, nt, nl):
    """The same coefficients on the oracle's full m x n window [j + m/2, k + n/2]:
    negative j by X_{-j,k} = (-1)^k X_{j,k}, negative k by X_{j,-k} = (-1)^k conj X_{j,k},
    the theta-Nyquist row zero."""
    m, n, N, L = 2 * nt, nl, nt, nl // 2
    F = np.zeros((m, n), dtype=complex)
    for k in range(L):
        sgn = (-1.0) ** k
        F[N:, L + k] = X[:, k]
        F[N - np.arange(1, N), L + k] = sgn * X[1:, k]
        if k:
            F[:, L - k] = sgn * np.conj(F[:, L + k])
    F[N:, 0] = X[:, L]                                  # k = -n/2
    F[N - np.arange(1, N), 0] = (-1.0) ** L * X[1:, L]
    return F


@pytest.mark.parametrize("nt,nl", [(1, 2), (2, 4), (5, 10), (24, 48), (33, 70), (22, 58), (64, 130)])
def test_sample_matches_oracle_on_arbitrary_coefficients(sp, nt, nl):
    # not only the inverse of coeffs2: any coefficient array of a real function
    # on the sphere, against the oracle's inverse 2D expansion
    X = _random_sphere_coefficients(nt, nl, np.random.default_rng(nt * nl))
    F = _full_window(X, nt, nl)
    ref = O.sample(F)[nt:]
    assert np.abs(ref.imag).max() < 1e-12 * np.abs(ref.real).max()
    got = sp.Plan(nt, nl).sample(torch.tensor(X, device="cuda")).cpu().numpy()
    assert np.abs(got - ref.real).max() < 1e-13 * np.abs(ref.real).max() * max(1.0, math.log2(nt * nl))


def test_sum2_worked_example(sp):
    vals = {}
    for line in open(GOLDEN).read().splitlines():
        if "=" in line and not line.startswith("#"):
            k, v = line.split("=", 1)
            vals[k.strip()] = v.strip()
    exact = int(vals["exact_numerator_pi"]) * math.pi / int(vals["exact_denominator"])
    for nt, nl in [(8, 16), (12, 24), (33, 70)]:
        th = sh.colatitudes(nt)[:, None]
        la = sh.longitudes(nl)[None, :]
        x = np.cos(la) * np.sin(th)
        y = np.sin(la) * np.sin(th)
        z = np.cos(th) + 0 * la
        f = 1 + x + y ** 2 + x ** 2 * y + x ** 4 + y ** 5 + (x * y * z) ** 2
        got = sp.Plan(nt, nl).sum2(torch.tensor(f, device="cuda"))
        assert abs(got - exact) < 1e-13, (nt, nl, got - exact)


def test_sum2_of_harmonics(sp):
    nt, nl = 20, 40
    plan = sp.Plan(nt, nl)
    y00 = sh.synthesize(sh.single_sh_coeffs(0, 0), nt, nl, device="cuda")
    assert abs(plan.sum2(y00) - math.sqrt(4 * math.pi)) < 1e-13
    for l, m in [(1, 0), (2, 0), (3, 2), (6, -5)]:
        assert abs(plan.sum2(sh.synthesize(sh.single_sh_coeffs(l, m), nt, nl, device="cuda"))) < 1e-13
