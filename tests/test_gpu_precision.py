"""GPU parity of the reduced-precision forms against the FP64 oracle.

SP_FP32: transforms and eliminations in FP32, the zonal column (k = 0, whose
system is the ill-conditioned one) in FP64 on a side stream; bar 1e-5 relative.
SP_FP32_REFINE: transforms in double-float (FP64-accurate on the FP32 pipes),
FP32 eliminations refined by a double-float residual, zonal column in FP64;
bar 1e-12 after refinement, errors recorded per sweep.
"""

import numpy as np
import pytest
import torch

from oracle import sphere_oracle as O
from synth import sh

pytestmark = pytest.mark.gpu

FP32_TOL = 1e-5
REFINED_TOL = 1e-12


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1510_08094_gb300 as sp

    return sp


def _rel(a, b):
    return float(np.abs(a - b).max() / np.abs(b).max())


def _series(nt, nl, lmax, seed, decay="inv_sq"):
    c = sh.random_sh_coeffs(lmax, seed, decay)
    return sh.synthesize(c, nt, nl).numpy(), sh.synthesize(sh.poisson_exact(c), nt, nl).numpy()


SIZES = [(64, 128), (75, 150), (48, 96), (33, 70), (5, 10), (2, 4), (256, 512)]


@pytest.mark.parametrize("nt,nl", SIZES)
def test_fp32_matches_oracle(sp, nt, nl):
    f, _ = _series(nt, nl, max(1, nt // 2), 11 + nt)
    u_ref = O.poisson(f)
    u = sp.Plan(nt, nl, "fp32").solve(torch.tensor(f, device="cuda")).cpu().numpy()
    assert _rel(u, u_ref) < FP32_TOL


@pytest.mark.parametrize("nt,nl", [(16, 32), (64, 128), (33, 70)])
def test_fp32_adjoint_matches_oracle(sp, nt, nl):
    g = np.random.default_rng(nt).standard_normal((nt, nl))
    ref = O.poisson_adjoint(g)
    out = sp.Plan(nt, nl, "fp32").solve_adjoint(torch.tensor(g, device="cuda")).cpu().numpy()
    assert _rel(out, ref) < FP32_TOL


@pytest.mark.parametrize("nt,nl", SIZES)
def test_refined_matches_oracle(sp, nt, nl):
    f, _ = _series(nt, nl, max(1, nt // 2), 21 + nt)
    u_ref = O.poisson(f)
    errs = []
    for sweeps in range(0, 4):
        u = sp.Plan(nt, nl, "fp32_refine", sweeps).solve(torch.tensor(f, device="cuda")).cpu().numpy()
        errs.append(_rel(u, u_ref))
    assert errs[0] < FP32_TOL, errs
    assert errs[2] < REFINED_TOL, errs
    assert errs[3] < REFINED_TOL, errs


@pytest.mark.parametrize("nt,nl", [(64, 128), (100, 200)])
def test_refined_rough_input(sp, nt, nl):
    f = np.random.default_rng(nt + 1).standard_normal((nt, nl))
    u_ref = O.poisson(f)
    u = sp.Plan(nt, nl, "fp32_refine", 3).solve(torch.tensor(f, device="cuda")).cpu().numpy()
    assert _rel(u, u_ref) < REFINED_TOL


@pytest.mark.parametrize("name", ["sh1024_2048x4096", "sh2000_5000x10000"])
def test_forms_at_large_size(sp, name):
    w = sh.workload(name)
    f, u_exact = w.make(device="cuda")
    u64 = sp.Plan(w.n_theta, w.n_lambda).solve(f)
    ex = float(u_exact.abs().max())
    e64 = float((u64 - u_exact).abs().max()) / ex
    u32 = sp.Plan(w.n_theta, w.n_lambda, "fp32").solve(f)
    e32 = float((u32 - u64).abs().max()) / ex
    assert e32 < FP32_TOL, e32
    for sweeps, tol in [(1, 1e-10), (2, REFINED_TOL)]:
        ur = sp.Plan(w.n_theta, w.n_lambda, "fp32_refine", sweeps).solve(f)
        er = float((ur - u64).abs().max()) / ex
        assert er < tol, (sweeps, er, e64)
