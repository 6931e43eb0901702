"""Plan-time tile tuning of single plans: the tuned plan must give the answers
of the default plan (the tiles change which CTA transforms which rows and
columns and the order of a few block sums, not the arithmetic), write one
cache entry per grid and arithmetic, and reuse it."""

import pytest
import torch

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def sp():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1510_08094_gb300 as sp

    return sp


def _rel(a, b):
    return float((a - b).abs().max() / b.abs().max())


@pytest.mark.parametrize("precision,sweeps,tol", [("fp64", 0, 1e-14), ("fp32", 0, 1e-6),
                                                  ("fp32_refine", 1, 1e-13)])
def test_tuned_plan_matches_default(sp, tmp_path, monkeypatch, precision, sweeps, tol):
    monkeypatch.setenv("SPHERE_POISSON_TUNE_CACHE", str(tmp_path / "tune.txt"))
    nt, nl = 96, 250                      # radices 2, 3 and 5, ragged tiles
    f = torch.randn(nt, nl, dtype=torch.float64, device="cuda")
    ref = sp.Plan(nt, nl, precision, sweeps).solve(f)
    tuned = sp.Plan(nt, nl, precision, sweeps, autotune=True)
    assert _rel(tuned.solve(f), ref) < tol
    if precision != "fp32_refine":     # the refined form has no adjoint
        assert _rel(tuned.solve_adjoint(f), sp.Plan(nt, nl, precision, sweeps).solve_adjoint(f)) < tol
    lines = (tmp_path / "tune.txt").read_text().strip().splitlines()
    assert len(lines) == 1 and f"|single|{precision}|" in lines[0]
    again = sp.Plan(nt, nl, precision, sweeps, autotune=True)      # served from the cache
    assert _rel(again.solve(f), ref) < tol
    assert len((tmp_path / "tune.txt").read_text().strip().splitlines()) == 1


def test_tuned_plans_share_a_cache_with_batched_plans(sp, tmp_path, monkeypatch):
    monkeypatch.setenv("SPHERE_POISSON_TUNE_CACHE", str(tmp_path / "tune.txt"))
    sp.Plan(64, 128, autotune=True)
    sp.BatchedPlan([(64, 128), (32, 64)], autotune=True)
    sp.Plan(32, 64, "fp32", autotune=True)
    lines = (tmp_path / "tune.txt").read_text().strip().splitlines()
    assert len(lines) == 4
    # a second round reads every entry back and appends nothing
    f = torch.randn(64, 128, dtype=torch.float64, device="cuda")
    u = sp.Plan(64, 128, autotune=True).solve(f)
    b = sp.BatchedPlan([(64, 128), (32, 64)], autotune=True)
    sp.Plan(32, 64, "fp32", autotune=True)
    assert len((tmp_path / "tune.txt").read_text().strip().splitlines()) == 4
    assert _rel(b.unpack(b.solve(b.pack([f, torch.randn(32, 64, dtype=torch.float64, device="cuda")])))[0], u) < 1e-13
