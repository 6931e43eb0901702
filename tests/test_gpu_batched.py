"""Batched plans: many spheres of uneven resolution in one persistent launch.

Each problem's answer must match the single-problem FP64 solve of the same
grid (same kernels up to reduction order: 1e-13) and the oracle (1e-12).
Also: the autotuned plan, a CUDA-graph capture of the launch, the empty batch.
The FP32 + refinement batched form: 1e-12 against the oracle after
refinement, the 1e-5 bar without a sweep, and agreement with the single-plan
form of the same arithmetic.
"""

import numpy as np
import pytest
import torch

from oracle import sphere_oracle as O
from synth import sh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1510_08094_gb300 as sp

    return sp


def _inputs(sizes, seed):
    rng = np.random.default_rng(seed)
    return [torch.tensor(rng.standard_normal(s), device="cuda") for s in sizes]


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


UNEVEN = [(64, 128), (2, 4), (33, 70), (48, 96), (5, 10), (100, 200), (17, 34), (64, 128), (1, 2), (128, 256)]


def test_batched_matches_single_solves(sp):
    plan = sp.BatchedPlan(UNEVEN)
    fs = _inputs(UNEVEN, 1)
    u = plan.unpack(plan.solve(plan.pack(fs)))
    for (nt, nl), f, ub in zip(UNEVEN, fs, u):
        ref = sp.Plan(nt, nl).solve(f)
        assert _rel(ub, ref) < 1e-13 or float(ref.abs().max()) < 1e-14


def test_batched_matches_oracle(sp):
    sizes = [(16, 32), (33, 70), (48, 96)]
    plan = sp.BatchedPlan(sizes)
    fs = _inputs(sizes, 2)
    u = plan.unpack(plan.solve(plan.pack(fs)))
    for f, ub in zip(fs, u):
        ref = O.poisson(f.cpu().numpy())
        assert float(np.abs(ub.cpu().numpy() - ref).max() / np.abs(ref).max()) < 1e-12


def test_batched_uneven_workload_family(sp):
    # colatitudes 16 s for s = 2..32 (prime factors up to 31), longitudes 2 n_theta,
    # spherical-harmonic series l <= n_theta/2, checked against the closed form
    sizes = [(16 * s, 32 * s) for s in range(2, 33)]
    fs, us = [], []
    for b, (nt, nl) in enumerate(sizes):
        c = sh.random_sh_coeffs(nt // 2, 1510080944 + b, "inv_sq")
        fs.append(sh.synthesize(c, nt, nl, device="cuda"))
        us.append(sh.synthesize(sh.poisson_exact(c), nt, nl, device="cuda"))
    plan = sp.BatchedPlan(sizes)
    u = plan.unpack(plan.solve(plan.pack(fs)))
    for ub, ue in zip(u, us):
        assert _rel(ub, ue) < 1e-12


def test_autotuned_plan_gives_same_answers(sp, tmp_path, monkeypatch):
    monkeypatch.setenv("SPHERE_POISSON_TUNE_CACHE", str(tmp_path / "tune.txt"))
    sizes = [(64, 128), (96, 192), (80, 160), (64, 128)]
    fs = _inputs(sizes, 3)
    a = sp.BatchedPlan(sizes)
    b = sp.BatchedPlan(sizes, autotune=True)
    ua = a.solve(a.pack(fs))
    ub = b.solve(b.pack(fs))
    assert _rel(ub, ua) < 1e-13
    lines = (tmp_path / "tune.txt").read_text().strip().splitlines()
    assert len(lines) == 3                     # one entry per distinct size
    c = sp.BatchedPlan(sizes, autotune=True)   # second plan reads the cache
    assert _rel(c.solve(c.pack(fs)), ua) < 1e-13
    assert len((tmp_path / "tune.txt").read_text().strip().splitlines()) == 3


def test_batched_launch_captured_in_cuda_graph(sp):
    sizes = [(32, 64), (48, 96), (64, 128)]
    plan = sp.BatchedPlan(sizes)
    assert plan.launches() == 1
    fs = _inputs(sizes, 4)
    f = plan.pack(fs)
    u = torch.empty_like(f)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.solve(f, u, ws)                       # warm-up outside capture
    torch.cuda.synchronize()
    ref = u.clone()
    u.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.solve(f, u, ws)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(u, ref)
    f2 = plan.pack(_inputs(sizes, 5))
    f.copy_(f2)
    g.replay()
    torch.cuda.synchronize()
    assert _rel(u, plan.solve(f2)) < 1e-15


@pytest.mark.parametrize("precision,sweeps", [("fp64", 0), ("fp32_refine", 1)])
def test_mixed_radix_groups_two_launches_in_one_graph(sp, precision, sweeps):
    # 44 = 4 * 11 and 33 = 3 * 11 need the large-prime passes, 32 and 64 do not:
    # the solve is one launch per group, and the pair captures into one graph
    sizes = [(32, 64), (44, 88), (64, 128), (33, 66), (32, 64)]
    plan = sp.BatchedPlan(sizes, precision, sweeps)
    assert plan.launches() == 2
    fs = _inputs(sizes, 12)
    f = plan.pack(fs)
    u = torch.empty_like(f)
    ws = torch.empty(plan.workspace_bytes, dtype=torch.uint8, device="cuda")
    plan.solve(f, u, ws)
    torch.cuda.synchronize()
    for b, (nt, nl) in enumerate(sizes):
        single = sp.Plan(nt, nl, precision, sweeps).solve(fs[b])
        got = u[plan.offsets[b]:plan.offsets[b + 1]].view(nt, nl)
        assert _rel(got, single) < (1e-12 if precision == "fp64" else 1e-11)
    ref = u.clone()
    u.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            plan.solve(f, u, ws)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(u, ref)


def test_empty_batch(sp):
    plan = sp.BatchedPlan([])
    assert plan.offsets == [0]
    assert plan.launches() == 0


# ---- FP32 + refinement batched form ------------------------------------------

REFINE_SIZES = [(16, 32), (33, 70), (48, 96), (5, 10), (64, 128), (1, 2), (2, 4), (31, 62)]


def test_batched_refine_matches_oracle(sp):
    plan = sp.BatchedPlan(REFINE_SIZES, precision="fp32_refine", refine_sweeps=2)
    fs = _inputs(REFINE_SIZES, 6)
    u = plan.unpack(plan.solve(plan.pack(fs)))
    for (nt, nl), f, ub in zip(REFINE_SIZES, fs, u):
        ref = O.poisson(f.cpu().numpy())
        scale = max(float(np.abs(ref).max()), float(f.abs().max()) * 1e-3)
        assert float(np.abs(ub.cpu().numpy() - ref).max()) / scale < 1e-12, (nt, nl)


def test_batched_refine_unrefined_bar(sp):
    # no sweep: FP32 eliminations of the double-float spectrum, 1e-5 bar
    plan = sp.BatchedPlan(REFINE_SIZES, precision="fp32_refine", refine_sweeps=0)
    fs = _inputs(REFINE_SIZES, 7)
    u = plan.unpack(plan.solve(plan.pack(fs)))
    errs = []
    for f, ub in zip(fs, u):
        ref = sp.Plan(*f.shape).solve(f)
        scale = max(float(ref.abs().max()), float(f.abs().max()) * 1e-3)
        errs.append(float((ub - ref).abs().max()) / scale)
    assert max(errs) < 1e-5
    assert max(errs) > 1e-13          # the FP32 eliminations are really unrefined


def test_batched_refine_matches_single_refine_plans(sp):
    sizes = [(64, 128), (96, 192), (48, 96)]
    fs = _inputs(sizes, 8)
    for sweeps in (0, 2):
        plan = sp.BatchedPlan(sizes, precision="fp32_refine", refine_sweeps=sweeps)
        u = plan.unpack(plan.solve(plan.pack(fs)))
        for f, ub in zip(fs, u):
            ref = sp.Plan(*f.shape, "fp32_refine", sweeps).solve(f)
            tol = 1e-13 if sweeps else 1e-6
            assert _rel(ub, ref) < tol, sweeps


def test_batched_refine_uneven_family_closed_form(sp):
    sizes = [(16 * s, 32 * s) for s in range(2, 33, 3)]
    fs, us = [], []
    for b, (nt, nl) in enumerate(sizes):
        c = sh.random_sh_coeffs(nt // 2, 1510080944 + b, "inv_sq")
        fs.append(sh.synthesize(c, nt, nl, device="cuda"))
        us.append(sh.synthesize(sh.poisson_exact(c), nt, nl, device="cuda"))
    plan = sp.BatchedPlan(sizes, precision="fp32_refine", refine_sweeps=1)
    u = plan.unpack(plan.solve(plan.pack(fs)))
    for ub, ue in zip(u, us):
        assert _rel(ub, ue) < 1e-12


def test_batched_refine_autotune_and_graph(sp, tmp_path, monkeypatch):
    monkeypatch.setenv("SPHERE_POISSON_TUNE_CACHE", str(tmp_path / "tune.txt"))
    sizes = [(64, 128), (80, 160), (64, 128)]
    fs = _inputs(sizes, 9)
    a = sp.BatchedPlan(sizes, precision="fp32_refine", refine_sweeps=1)
    b = sp.BatchedPlan(sizes, precision="fp32_refine", refine_sweeps=1, autotune=True)
    f = a.pack(fs)
    ua = a.solve(f)
    assert _rel(b.solve(f), ua) < 1e-13
    lines = (tmp_path / "tune.txt").read_text().strip().splitlines()
    assert len(lines) == 2 and all("fp32_refine" in ln for ln in lines)
    assert b.launches() == 1
    u = torch.empty_like(f)
    ws = torch.empty(b.workspace_bytes, dtype=torch.uint8, device="cuda")
    b.solve(f, u, ws)
    torch.cuda.synchronize()
    ref = u.clone()
    u.zero_()
    g = torch.cuda.CUDAGraph()
    s = torch.cuda.Stream()
    with torch.cuda.stream(s):
        with torch.cuda.graph(g, stream=s):
            b.solve(f, u, ws)
    g.replay()
    torch.cuda.synchronize()
    assert torch.equal(u, ref)


def test_batched_refine_empty_and_adjoint_unsupported(sp):
    plan = sp.BatchedPlan([], precision="fp32_refine", refine_sweeps=1)
    assert plan.launches() == 0
    plan = sp.BatchedPlan([(8, 16)], precision="fp32_refine", refine_sweeps=1)
    f = torch.randn(128, dtype=torch.float64, device="cuda")
    with pytest.raises(RuntimeError):
        plan.solve_adjoint(f)
