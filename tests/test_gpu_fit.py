"""Differentiation form: inverse-source fit on the 1024 x 512 grid.

loss(f) = ||u(f) - u_obs||^2 with u_obs a seeded l <= 200 series plus N(0, 1e-3)
noise.  The gradient 2 S^T (S f - u_obs) comes from the adjoint kernels through
torch.autograd; it is checked against the oracle's transpose (FP64: 1e-12, FP32:
1e-5) and against central finite differences with h = 1e-6.
"""

import numpy as np
import pytest
import torch

from oracle import sphere_oracle as O
from synth import sh

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def case():
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA device")
    import paper_1510_08094_gb300 as sp

    w = sh.workload("sh200_512x1024_noisy")
    u_obs = w.observation(device="cuda")
    rng = np.random.default_rng(55)
    f0 = torch.tensor(rng.standard_normal((w.n_theta, w.n_lambda)) * 0.1, device="cuda")
    ref_grad = 2.0 * O.poisson_adjoint(O.poisson(f0.cpu().numpy()) - u_obs.cpu().numpy())
    return sp, w, u_obs, f0, ref_grad


def _grad(sp, f0, u_obs, precision):
    f = f0.clone().requires_grad_(True)
    loss = ((sp.poisson(f, precision) - u_obs) ** 2).sum()
    loss.backward()
    return float(loss.detach()), f.grad.detach()


@pytest.mark.parametrize("precision,tol", [("fp64", 1e-12), ("fp32", 1e-5)])
def test_gradient_matches_oracle_adjoint(case, precision, tol):
    sp, w, u_obs, f0, ref = case
    _, g = _grad(sp, f0, u_obs, precision)
    err = float(np.abs(g.cpu().numpy() - ref).max() / np.abs(ref).max())
    assert err < tol, err


def test_gradient_central_differences(case):
    sp, w, u_obs, f0, _ = case
    _, g = _grad(sp, f0, u_obs, "fp64")

    def loss(x):
        return float(((sp.solve(x) - u_obs) ** 2).sum())

    h = 1e-6
    rng = np.random.default_rng(7)
    for _ in range(3):
        d = torch.tensor(rng.standard_normal(tuple(f0.shape)), device="cuda")
        fd = (loss(f0 + h * d) - loss(f0 - h * d)) / (2 * h)
        assert abs(fd - float((g * d).sum())) < 1e-6 * max(1.0, abs(fd))
    for idx in [(0, 0), (255, 511), (511, 1023)]:
        e = torch.zeros_like(f0)
        e[idx] = 1.0
        fd = (loss(f0 + h * e) - loss(f0 - h * e)) / (2 * h)
        assert abs(fd - float(g[idx])) < 1e-6 * max(1.0, abs(fd))


def test_fit_reduces_loss(case):
    # a few steps of gradient descent with exact line search on the quadratic loss
    sp, w, u_obs, f0, _ = case
    f = f0.clone()
    losses = []
    for _ in range(5):
        r = sp.solve(f) - u_obs
        losses.append(float((r * r).sum()))
        g = 2.0 * sp.solve_adjoint(r)
        sg = sp.solve(g)
        step = float((r * sg).sum()) / float((sg * sg).sum()) / 1.0
        f = f - step * g
    assert all(b < a for a, b in zip(losses, losses[1:]))
