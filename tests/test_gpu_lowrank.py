"""Low-rank form on the GPU: the structure-preserving GE (Section 3) and the
Poisson solve with the right-hand side formed from the low-rank factors.

The GE must reproduce the oracle's pivots and approximant on generic input and
recover finite-rank functions exactly at their SVD rank (Theorem
BMCrankDrop); the low-rank solve must give the dense solve's answer (same
function, 1e-12) up to 5000 x 10000."""

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


def _xyz(nt, nl, dev="cpu"):
    th = torch.tensor(sh.colatitudes(nt), device=dev)[:, None]
    la = torch.tensor(sh.longitudes(nl), device=dev)[None, :]
    return torch.cos(la) * torch.sin(th), torch.sin(la) * torch.sin(th), torch.cos(th) + 0 * la


def _approximant(cols, piv, rows):
    """sum_t [c(theta) c(-theta)] P [r(lambda); r(lambda + pi)] on the DFS grid (numpy)."""
    cols, piv, rows = cols.cpu().numpy(), piv.cpu().numpy(), rows.cpu().numpy()
    n = rows.shape[1]
    out = 0.0
    for c, (p0, p1), r in zip(cols, piv, rows):
        C = np.stack([c, c[::-1]], axis=1)
        R = np.stack([r, np.roll(r, -(n // 2))], axis=0)
        out = out + C @ np.array([[p0, p1], [p1, p0]]) @ R
    return out


def _rank(piv):
    return sum(int(np.linalg.matrix_rank(np.array([[a, b], [b, a]]))) for a, b in piv.cpu().numpy())


@pytest.mark.parametrize("nt,nl", [(20, 40), (33, 70)])
def test_ge_matches_oracle(sp, nt, nl):
    x, y, z = _xyz(nt, nl)
    f = (torch.exp(x * y + z) + torch.sin(3 * x)).numpy()
    ft = O.dfs_double(f)
    terms, _ = O.bmc_ge(ft)
    cols, piv, rows = sp.Plan(nt, nl).lowrank_ge(torch.tensor(f, device="cuda"))
    # the first pivot is the unique global maximum: same column, row and
    # pseudoinverse; later pivots may flip between near-equal candidates with
    # rounding (a different but equally valid factorisation), so what is
    # compared there is the approximant and the rank
    scale = np.abs(ft).max()
    c, P, r, _ = terms[0]
    assert np.abs(cols[0].cpu().numpy() - c[:, 0]).max() < 1e-13 * scale
    assert np.abs(rows[0].cpu().numpy() - r[0]).max() < 1e-13 * scale
    assert abs(float(piv[0, 0]) - P[0, 0]) + abs(float(piv[0, 1]) - P[0, 1]) < 1e-13 * np.abs(P).max()
    assert abs(_rank(piv) - sum(int(np.linalg.matrix_rank(P)) for _, P, _, _ in terms)) <= 2
    approx = _approximant(cols, piv, rows)
    assert np.abs(approx - ft).max() < 1e-12 * np.abs(ft).max()
    assert np.abs(approx - O.lowrank_values(terms)).max() < 1e-12 * np.abs(ft).max()


@pytest.mark.parametrize("nt,nl", [(24, 48), (75, 150)])
def test_every_ge_term_matches_oracle_on_rough_input(sp, nt, nl):
    # rough N(0,1) samples: the largest sigma_1 of each step is separated from
    # the next by far more than rounding, so the pivot sequence is unique and
    # every term (column pair, pseudoinverse, row pair, hence pivot position)
    # must be the oracle's for the first steps
    K = 8
    f = np.random.default_rng(nt).standard_normal((nt, nl))
    ft = O.dfs_double(f)
    terms, _ = O.bmc_ge(ft, max_terms=K)
    cols, piv, rows = sp.Plan(nt, nl).lowrank_ge(torch.tensor(f, device="cuda"), max_terms=K)
    assert len(terms) == K and cols.shape[0] == K
    cols, piv, rows = cols.cpu().numpy(), piv.cpu().numpy(), rows.cpu().numpy()
    scale = np.abs(ft).max()
    H = nl // 2
    resid = ft.copy()
    for t, (c, P, r, (p, q)) in enumerate(terms):
        # the GPU's term [c(theta) c(-theta)] P [r(lambda); r(lambda + pi)] against the
        # oracle's cols @ P @ rows: c = e(., lambda* - pi), c(-theta) = e(., lambda*),
        # r = e(theta*, .), r(. + pi) = e(-theta*, .)
        assert np.abs(cols[t] - c[:, 0]).max() < 1e-12 * scale, t
        assert np.abs(cols[t][::-1] - c[:, 1]).max() < 1e-12 * scale, t
        assert np.abs(rows[t] - r[0]).max() < 1e-12 * scale, t
        assert np.abs(np.roll(rows[t], -H) - r[1]).max() < 1e-12 * scale, t
        assert np.abs(piv[t] - P[0]).max() < 1e-12 * np.abs(P).max(), t
        # the pivot position (p, q): the residual's column at lambda* - pi and row at theta*
        assert np.abs(cols[t] - resid[:, q - H]).max() < 1e-12 * scale, t
        assert np.abs(rows[t] - resid[p]).max() < 1e-12 * scale, t
        resid = resid - c @ P @ r


def test_exact_recovery_at_svd_rank(sp):
    nt, nl = 32, 64
    f = sh.synthesize(sh.random_sh_coeffs(10, 11), nt, nl).numpy()
    sv = np.linalg.svd(O.dfs_double(f), compute_uv=False)
    cols, piv, rows = sp.Plan(nt, nl).lowrank_ge(torch.tensor(f, device="cuda"))
    assert _rank(piv) == int((sv > 1e-11 * sv[0]).sum())
    assert np.abs(_approximant(cols, piv, rows) - O.dfs_double(f)).max() < 1e-12 * np.abs(f).max()


def test_paper_test_function_rank(sp):
    nt, nl = 128, 256
    x, y, z = _xyz(nt, nl, "cuda")
    f = torch.cos(1 + 2 * np.pi * (x + y) + 5 * torch.sin(np.pi * z)).contiguous()
    _, piv, _ = sp.Plan(nt, nl).lowrank_ge(f)
    assert 23 <= _rank(piv) <= 25        # the paper's spherefun reports rank 23


@pytest.mark.parametrize("nt,nl", [(24, 48), (64, 128), (26, 58), (33, 70)])
def test_lowrank_solve_matches_dense_and_oracle(sp, nt, nl):
    x, y, z = _xyz(nt, nl, "cuda")
    f = (torch.sin(5 * x * y * z) + torch.cos(2 * x + y)).contiguous()
    plan = sp.Plan(nt, nl)
    cols, piv, rows = plan.lowrank_ge(f)
    u_low = plan.solve_lowrank(cols, piv, rows)
    u = plan.solve(f)
    assert float((u_low - u).abs().max() / u.abs().max()) < 1e-12
    ref = O.poisson(f.cpu().numpy())
    assert np.abs(u_low.cpu().numpy() - ref).max() < 1e-12 * np.abs(ref).max()


def test_lowrank_solve_at_full_size(sp):
    nt, nl = 5000, 10000
    x, y, z = _xyz(nt, nl, "cuda")
    f = torch.sin(50 * x * y * z).contiguous()            # the paper's Section 5 example
    plan = sp.Plan(nt, nl)
    cols, piv, rows = plan.lowrank_ge(f, max_terms=128)
    assert _rank(piv) == 12                                  # the paper: numerical rank 12
    u_low = plan.solve_lowrank(cols, piv, rows)
    u = plan.solve(f)
    assert float((u_low - u).abs().max() / u.abs().max()) < 1e-12


def test_edges_and_errors(sp):
    from paper_1510_08094_gb300 import _lib

    plan = sp.Plan(8, 16)
    f = torch.zeros(8, 16, dtype=torch.float64, device="cuda")
    cols, piv, rows = plan.lowrank_ge(f)
    assert cols.shape[0] == 0                               # the zero function has rank 0
    assert float(plan.solve_lowrank(cols, piv, rows).abs().max()) == 0.0
    with pytest.raises(_lib.SpherePoissonError):
        plan.lowrank_ge(f, max_terms=9)                    # more than n_theta terms
    with pytest.raises(_lib.SpherePoissonError):
        sp.Plan(8, 16, "fp32").lowrank_ge(f)
