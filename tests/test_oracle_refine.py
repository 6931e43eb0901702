"""Pins of the oracle's refinement reference (refine_reference): the per-k
systems of eq. linearSystems solved in single precision, except the k = 0 column
of eq. pentdiagonalPlusRankOne in FP64, and corrected by FP64 residual sweeps.

Pinned against what the arithmetic fixes, independently of the function: the
sweeps converge to the FP64 solve (itself pinned by closed forms) and to the
closed form of a spherical-harmonic series; before any sweep the error sits at
single precision's level (so the solves really are single precision); one sweep
contracts it by orders of magnitude; and a zonal input, which lives in the FP64
k = 0 column alone, is exact to FP64 rounding without a sweep."""

import numpy as np
import pytest

from oracle import sphere_oracle as O
from synth import sh


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


@pytest.mark.parametrize("nt,nl,lmax", [(64, 128, 30), (150, 300, 60)])
def test_sweeps_converge_to_the_fp64_solve_and_the_closed_form(nt, nl, lmax):
    c = sh.random_sh_coeffs(lmax, 70 + nt, "inv_sq")
    f = sh.synthesize(c, nt, nl).numpy()
    u_exact = sh.synthesize(sh.poisson_exact(c), nt, nl).numpy()
    us = O.refine_reference(f, 2)
    u64 = O.poisson(f)
    e = [_rel(u, u64) for u in us]
    assert 1e-10 < e[0] < 1e-5              # single-precision solves
    assert e[1] < 1e-4 * e[0]               # one sweep contracts the error
    assert e[2] < 1e-13
    assert _rel(us[2], u_exact) < 1e-13


def test_zonal_input_needs_no_sweep():
    # Y_l^0 sits in the k = 0 column, which the form solves in FP64
    nt, nl = 48, 96
    f = sum(sh.synthesize(sh.single_sh_coeffs(l, 0), nt, nl).numpy() for l in (2, 5, 11))
    us = O.refine_reference(f, 0)
    assert _rel(us[0], O.poisson(f)) < 1e-13


def test_non_zonal_harmonic_is_single_precision_before_the_sweep():
    nt, nl = 48, 96
    f = sh.synthesize(sh.single_sh_coeffs(9, 4), nt, nl).numpy()
    u0, u1 = O.refine_reference(f, 1)
    ref = -f / 90.0
    assert 1e-10 < _rel(u0, ref) < 1e-5
    assert _rel(u1, ref) < 1e-13
