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


@pytest.mark.parametrize("nt,nl", [(16, 32), (64, 128), (33, 70), (5, 10), (2, 4), (100, 200), (75, 150)])
def test_fp32_adjoint_matches_oracle(sp, nt, nl):
    g = np.random.default_rng(nt).standard_normal((nt, nl))
    ref = O.poisson_adjoint(g)
    out = sp.Plan(nt, nl, "fp32").solve_adjoint(torch.tensor(g, device="cuda")).cpu().numpy()
    assert _rel(out, ref) < FP32_TOL


@pytest.mark.parametrize("nt,nl", [(256, 512), (1000, 2000), (5000, 10000), (6144, 12288)])
def test_fp32_adjoint_dot_product(sp, nt, nl):
    # the FP32 adjoint (its colatitude stage fused in one launch, the tile by TMA
    # where two columns fit) against the FP32 forward by <S f, g> = <f, S^T g>,
    # and against the FP64 adjoint
    gen = torch.Generator(device="cuda").manual_seed(nt)
    f = torch.randn(nt, nl, dtype=torch.float64, device="cuda", generator=gen)
    g = torch.randn(nt, nl, dtype=torch.float64, device="cuda", generator=gen)
    plan = sp.Plan(nt, nl, "fp32")
    sg = plan.solve_adjoint(g)
    sf = plan.solve(f)
    lhs = float((sf * g).sum())
    rhs = float((f * sg).sum())
    # the sums cancel heavily for random f and g: bound by the norms instead
    scale = float(sf.norm() * g.norm() + f.norm() * sg.norm())
    assert abs(lhs - rhs) < 1e-6 * scale, (lhs, rhs, scale)
    sg64 = sp.Plan(nt, nl, "fp64").solve_adjoint(g)
    assert float((sg - sg64).abs().max() / sg64.abs().max()) < FP32_TOL


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


@pytest.mark.parametrize("nt,nl,kind", [(64, 128, "series"), (150, 300, "series"), (64, 128, "rough"),
                                         (150, 300, "rough")])
def test_sweeps_follow_the_oracle_refinement_reference(sp, nt, nl, kind):
    # sweep by sweep against oracle.refine_reference (single-precision per-k
    # solves, the k = 0 column of eq. pentdiagonalPlusRankOne in FP64, FP64
    # residuals): before any sweep both are single-precision solves, so their
    # errors against the FP64 solve agree within a factor of 10 (and neither is
    # at FP64 level); from sweep 1 on the GPU form matches the reference's
    # iterate to 1e-12; the GPU error falls monotonically to the FP64 floor
    if kind == "series":
        f, _ = _series(nt, nl, nt // 2, 31 + nt)
    else:
        f = np.random.default_rng(nt).standard_normal((nt, nl))
    u64 = O.poisson(f)
    ref = O.refine_reference(f, 3)
    e_ref = [_rel(r, u64) for r in ref]
    e_gpu = []
    ft = torch.tensor(f, device="cuda")
    for sweeps in range(4):
        u = sp.Plan(nt, nl, "fp32_refine", sweeps).solve(ft).cpu().numpy()
        e_gpu.append(_rel(u, u64))
        if sweeps >= 1:
            assert _rel(u, ref[sweeps]) < REFINED_TOL, (sweeps, e_gpu, e_ref)
    assert e_ref[0] / 10 < e_gpu[0] < 10 * e_ref[0], (e_gpu, e_ref)
    assert e_gpu[0] > 1e-10, e_gpu
    assert e_gpu[1] < 1e-3 * e_gpu[0], e_gpu
    # after the first sweep the error sits at the form's FP64-level floor (2e-13
    # measured on rough input at 150 x 300) and may only jitter there
    floor = 2.0 * min(e_gpu[1:])
    for s in (1, 2):
        assert e_gpu[s + 1] <= max(e_gpu[s], floor), e_gpu


@pytest.mark.parametrize("nt,nl", [(64, 128), (100, 200)])
def test_refined_rough_input(sp, nt, nl):
    f = np.random.default_rng(nt + 1).standard_normal((nt, nl))
    u_ref = O.poisson(f)
    u = sp.Plan(nt, nl, "fp32_refine", 3).solve(torch.tensor(f, device="cuda")).cpu().numpy()
    assert _rel(u, u_ref) < REFINED_TOL


@pytest.mark.parametrize("name", ["sh1024_2048x4096", "sh2048_4096x8192", "sh2000_5000x10000"])
def test_forms_at_large_size(sp, name):
    # the FP64 solve against the series' closed form (Delta Y_l^m = -l(l+1) Y_l^m)
    # at the series bar, then the reduced-precision forms against the FP64 solve
    w = sh.workload(name)
    f, u_exact = w.make(device="cuda")
    u64 = sp.Plan(w.n_theta, w.n_lambda).solve(f)
    ex = float(u_exact.abs().max())
    e64 = float((u64 - u_exact).abs().max()) / ex
    assert e64 < 5e-12, e64
    u32 = sp.Plan(w.n_theta, w.n_lambda, "fp32").solve(f)
    e32 = float((u32 - u64).abs().max()) / ex
    assert e32 < FP32_TOL, e32
    for sweeps, tol in [(1, 1e-10), (2, REFINED_TOL)]:
        ur = sp.Plan(w.n_theta, w.n_lambda, "fp32_refine", sweeps).solve(f)
        er = float((ur - u64).abs().max()) / ex
        assert er < tol, (sweeps, er, e64)
