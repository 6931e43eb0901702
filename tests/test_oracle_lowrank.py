"""Pins of the oracle's structure-preserving GE and low-rank coefficients
(Section 3, Figure GaussianElimination; Section 4, eq. 2DFourierExpansion).

Pinned against: numpy's SVD-based pseudoinverse with the same cut (the
epsilon-pseudoinverse of Definition pseudoinverse), the SVD numerical rank of
the sample matrix (Theorem BMCrankDrop: exact recovery of finite-rank BMC
functions after as many terms as their rank; spherical harmonics are rank 1),
the paper's printed ranks 23 of eq. sphereTestFunc and 12 of sin(50 xyz)
(tests/golden), the BMC
symmetry of every GE residual, and the dense coefficients of the same function.
"""

import os

import numpy as np
import pytest

from oracle import sphere_oracle as O
from synth import sh

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "sphere_test_func_rank.txt")
GOLDEN_SIN50 = os.path.join(os.path.dirname(__file__), "golden", "sin50xyz_rank.txt")


def _golden_rank(path):
    vals = {k.strip(): v.strip() for k, v in (l.split("=", 1) for l in open(path).read().splitlines()
                                              if "=" in l and not l.startswith("#"))}
    return int(vals["rank"])


def _xyz(nt, nl):
    th = sh.colatitudes(nt)[:, None]
    la = sh.longitudes(nl)[None, :]
    return np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0 * la


def _rank(P):
    return int(np.linalg.matrix_rank(P))


@pytest.mark.parametrize("a,b", [(1.0, 0.3), (2.0, -1.99), (1.0, 1.0), (-0.5, 0.5000001), (3.0, 0.0), (0.7, -0.7)])
def test_pivot_pinv_matches_svd_pseudoinverse(a, b):
    alpha = 0.01
    M = np.array([[a, b], [b, a]])
    P = O.pivot_pinv(a, b, alpha)
    assert np.abs(P - np.linalg.pinv(M, rcond=alpha)).max() < 1e-12 * max(1.0, np.abs(P).max())
    J = np.array([[0.0, 1.0], [1.0, 0.0]])
    assert np.abs(J @ P - P @ J).max() < 1e-15 * max(1.0, np.abs(P).max())   # centrosymmetric


def _bmc_error(e):
    n = e.shape[1]
    return float(np.abs(e[::-1, :] - np.roll(e, -(n // 2), axis=1)).max())


@pytest.mark.parametrize("nt,nl,lmax,seed", [(24, 48, 6, 5), (20, 44, 9, 6), (16, 30, 4, 7)])
def test_exact_recovery_of_band_limited_series(nt, nl, lmax, seed):
    f = sh.synthesize(sh.random_sh_coeffs(lmax, seed), nt, nl).numpy()
    ft = O.dfs_double(f)
    terms, e = O.bmc_ge(ft)
    sv = np.linalg.svd(ft, compute_uv=False)
    assert sum(_rank(P) for _, P, _, _ in terms) == int((sv > 1e-11 * sv[0]).sum())
    assert float(np.abs(e).max()) < 1e-12 * float(np.abs(ft).max())
    assert np.abs(O.lowrank_values(terms) - ft).max() < 1e-12 * np.abs(ft).max()


@pytest.mark.parametrize("l,m", [(3, 0), (5, 2), (7, -4)])
def test_spherical_harmonics_are_rank_one(l, m):
    ft = O.dfs_double(sh.synthesize(sh.single_sh_coeffs(l, m), 16, 32).numpy())
    terms, e = O.bmc_ge(ft)
    assert sum(_rank(P) for _, P, _, _ in terms) == 1
    assert float(np.abs(e).max()) < 1e-13 * float(np.abs(ft).max())


def test_every_step_preserves_the_bmc_structure():
    nt, nl = 20, 40
    x, y, z = _xyz(nt, nl)
    ft = O.dfs_double(np.exp(x * y + z) + np.sin(3 * x))
    terms, _ = O.bmc_ge(ft)
    e = ft.copy()
    for c, P, r, _ in terms:
        term = c @ P @ r
        assert _bmc_error(term) < 1e-13 * max(1.0, np.abs(term).max())
        e = e - term
        assert _bmc_error(e) < 1e-13 * np.abs(ft).max()


def test_paper_test_function_rank():
    vals = {k.strip(): v.strip() for k, v in (l.split("=", 1) for l in open(GOLDEN).read().splitlines()
                                              if "=" in l and not l.startswith("#"))}
    rank = int(vals["rank"].strip())
    nt, nl = 128, 256
    x, y, z = _xyz(nt, nl)
    ft = O.dfs_double(np.cos(1 + 2 * np.pi * (x + y) + 5 * np.sin(np.pi * z)))
    sv = np.linalg.svd(ft, compute_uv=False)
    assert int((sv > 1e-13 * sv[0]).sum()) == rank                 # numerical rank at 1e-13
    terms, e = O.bmc_ge(ft)
    total = sum(_rank(P) for _, P, _, _ in terms)
    assert rank <= total <= rank + 2                                # GE is near-optimal
    assert float(np.abs(e).max()) < 1e-13


@pytest.mark.parametrize("nt,nl", [(75, 150), (128, 256)])
def test_paper_poisson_example_rank(nt, nl):
    # the paper's m = n = 150 grid and a finer one
    rank = _golden_rank(GOLDEN_SIN50)
    x, y, z = _xyz(nt, nl)
    ft = O.dfs_double(np.sin(50 * x * y * z))
    terms, e = O.bmc_ge(ft)
    assert sum(_rank(P) for _, P, _, _ in terms) == rank
    assert float(np.abs(e).max()) < 1e-13
    sv = np.linalg.svd(ft, compute_uv=False)
    assert int((sv > 1e-14 * sv[0]).sum()) == rank


def test_lowrank_coefficients_equal_the_dense_ones():
    nt, nl = 24, 50
    x, y, z = _xyz(nt, nl)
    f = np.cos(1 + 2 * x + np.sin(2 * z)) * (1 + 0.5 * y)
    ft = O.dfs_double(f)
    terms, _ = O.bmc_ge(ft)
    fk = O.lowrank_values(terms)[nt:]                               # the approximant on theta > 0
    F_low = O.lowrank_rhs_coefficients(terms, *ft.shape)
    F_dense = O.rhs_coefficients(fk)
    assert np.abs(F_low - F_dense).max() < 1e-14 * np.abs(F_dense).max() * 10
    # and the Poisson solution from the low-rank F is the solution for the approximant
    X = O.solve_columns(F_low)
    u = O.sample(X)[nt:].real
    assert np.abs(u - O.poisson(fk)).max() < 1e-12 * np.abs(u).max()
