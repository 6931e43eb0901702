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
