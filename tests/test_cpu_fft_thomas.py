"""The CPU FFT + Thomas solver that bench.py times beside the oracle
(baseline/fft_thomas.py): it must compute the oracle's solution, element by
element, on grids from one colatitude to several hundred, smooth and rough."""

import numpy as np
import pytest

from baseline import fft_thomas
from oracle import sphere_oracle as O
from synth import sh


@pytest.mark.parametrize("nt,nl", [(1, 2), (1, 8), (2, 4), (3, 6), (5, 10), (16, 2), (17, 34), (33, 70),
                                   (64, 128), (75, 150)])
def test_matches_oracle_on_rough_input(nt, nl):
    f = np.random.default_rng(nt + 7 * nl).standard_normal((nt, nl))
    ref = O.poisson(f)
    u = fft_thomas.solve(f)
    assert np.abs(u - ref).max() < 1e-12 * max(1.0, np.abs(ref).max())


def test_matches_closed_form_and_threads_agree():
    nt, nl = 96, 192
    c = sh.random_sh_coeffs(40, 11, "inv_sq")
    f = sh.synthesize(c, nt, nl).numpy()
    exact = sh.synthesize(sh.poisson_exact(c), nt, nl).numpy()
    u1 = fft_thomas.solve(f, workers=1)
    u4 = fft_thomas.solve(f, workers=4)
    assert np.abs(u1 - exact).max() < 1e-13 * np.abs(exact).max()
    assert np.abs(u1 - u4).max() < 1e-15 * np.abs(exact).max()
