"""Real spherical-harmonic series on the pole-free longitude-colatitude grid.

Grid (the sampling convention every part of the project uses):
  colatitude  theta_i  = (i + 1/2) * pi / n_theta,       i = 0 .. n_theta-1
  longitude   lambda_q = -pi + 2 * pi * q / n_lambda,     q = 0 .. n_lambda-1
Samples are stored row-major as f[i][q] (one row per colatitude).

Real orthonormal harmonics (integral of Y^2 over the unit sphere = 1):
  Y_l^0  = Pbar_l^0(cos theta)
  Y_l^m  = sqrt(2) Pbar_l^m(cos theta) cos(m lambda)      m > 0
  Y_l^-m = sqrt(2) Pbar_l^m(cos theta) sin(m lambda)      m > 0
where Pbar_l^m are the associated Legendre functions normalised so that
2*pi * int_0^pi Pbar^2 sin(theta) dtheta = 1, generated by the standard
forward-column recurrence of Holmes & Featherstone (J. Geodesy 76, 2002):
  Pbar_0^0 = 1/sqrt(4 pi)
  Pbar_m^m = sqrt((2m+1)/(2m)) sin(theta) Pbar_{m-1}^{m-1}
  Pbar_{m+1}^m = sqrt(2m+3) cos(theta) Pbar_m^m
  Pbar_l^m = a_lm (cos(theta) Pbar_{l-1}^m - Pbar_{l-2}^m / a_{l-1,m}),
  a_lm = sqrt((4 l^2 - 1) / (l^2 - m^2)).
The recurrences run on scaled values: each column m carries an integer power
of two per colatitude (the scaling of Holmes & Featherstone's Section 2.7),
renormalised by exact powers of two whenever a value leaves [2^-600, 2^600].
Without it the sectoral seeds Pbar_m^m ~ sin^m(theta) go subnormal for m near
1000 while, at degrees near 2048, Pbar_l^m at the same colatitude (its turning
point, sin(theta) ~ m/l) is of order one: the seeds' lost digits came out as
relative errors of 1e-9 there.  Values that stay below the double range (deep
in the evanescent zone near the poles) are zero; the true ones are smaller
than 1e-300 of the field's scale.

Coefficients are held as a dense array C of shape (L+1, 2L+1), C[l, L+m]
being the weight of Y_l^m (entries with |m| > l are ignored).  Random draws
use numpy's PCG64 with the given seed, so they are identical on every host.
"""

from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np
import torch


def colatitudes(n_theta: int) -> np.ndarray:
    """theta_i = (i + 1/2) pi / n_theta (pole-free, half-shifted grid)."""
    i = np.arange(n_theta, dtype=np.float64)
    return (i + 0.5) * math.pi / n_theta


def pole_colatitudes(n_theta: int) -> np.ndarray:
    """theta_i = i pi / n_theta, i = 0 .. n_theta (the grid with both poles:
    n_theta + 1 rows)."""
    return np.arange(n_theta + 1, dtype=np.float64) * math.pi / n_theta


def grid_colatitudes(n_theta: int, grid: str = "shifted") -> np.ndarray:
    """The colatitudes of a grid: "shifted" (pole-free, n_theta rows) or
    "poles" (n_theta + 1 rows, both poles)."""
    if grid == "shifted":
        return colatitudes(n_theta)
    if grid == "poles":
        return pole_colatitudes(n_theta)
    raise ValueError(f"unknown grid {grid!r}")


def longitudes(n_lambda: int) -> np.ndarray:
    """lambda_q = -pi + 2 pi q / n_lambda."""
    q = np.arange(n_lambda, dtype=np.float64)
    return -math.pi + 2.0 * math.pi * q / n_lambda


def random_sh_coeffs(lmax: int, seed: int, decay: str = "none", drop_l0: bool = True) -> np.ndarray:
    """Seeded N(0,1) coefficients for l <= lmax, optionally scaled by 1/(1+l)^2.

    Returns C with shape (lmax+1, 2*lmax+1); C[l, lmax+m] multiplies Y_l^m.
    The l = 0 term (the sphere mean) is zeroed when drop_l0 is set.
    """
    rng = np.random.Generator(np.random.PCG64(seed))
    c = rng.standard_normal((lmax + 1, 2 * lmax + 1))
    ls = np.arange(lmax + 1)[:, None]
    ms = np.arange(-lmax, lmax + 1)[None, :]
    c[np.abs(ms) > ls] = 0.0
    if decay == "inv_sq":
        c = c / (1.0 + ls) ** 2
    elif decay != "none":
        raise ValueError(f"unknown decay {decay!r}")
    if drop_l0:
        c[0, :] = 0.0
    return c


def single_sh_coeffs(l: int, m: int) -> np.ndarray:
    """Coefficient array holding the single harmonic Y_l^m (|m| <= l)."""
    if abs(m) > l:
        raise ValueError("need |m| <= l")
    c = np.zeros((l + 1, 2 * l + 1))
    c[l, l + m] = 1.0
    return c


def _angle_table(mmax: int, n_lambda: int, device) -> tuple[torch.Tensor, torch.Tensor]:
    """cos(m lambda_q), sin(m lambda_q) for m = 0..mmax, with the phase
    m*lambda_q = pi * (m*(2q - n)) / n reduced exactly in integers."""
    m = torch.arange(mmax + 1, dtype=torch.int64, device=device)[:, None]
    q = torch.arange(n_lambda, dtype=torch.int64, device=device)[None, :]
    r = torch.remainder(m * (2 * q - n_lambda), 2 * n_lambda).to(torch.float64)
    ang = r * (math.pi / n_lambda)
    return torch.cos(ang), torch.sin(ang)


_RENORM = 600                      # exponent step of the renormalisation
_BIG = 2.0 ** _RENORM
_SMALL = 2.0 ** -_RENORM


def _ldexp(p: torch.Tensor, e: torch.Tensor) -> torch.Tensor:
    """p * 2**e for integer-valued float64 e, in two exact halves so that no
    power of two underflows while the product is still representable."""
    h = torch.floor(e * 0.5)
    return p * torch.exp2(h) * torch.exp2(e - h)


def _legendre_columns(lmax: int, theta: torch.Tensor):
    """Yield (l, P) for l = 0..lmax, P[m, i] = Pbar_l^m(cos theta_i) for m <= l
    (the forward-column recurrence of the module docstring, on scaled values)."""
    dev = theta.device
    nt = theta.shape[0]
    x = torch.cos(theta)
    s = torch.sin(theta)
    # sectoral seeds Pbar_m^m = pm[m] * 2**pe[m]
    pm = torch.empty((lmax + 1, nt), dtype=torch.float64, device=dev)
    pe = torch.zeros((lmax + 1, nt), dtype=torch.float64, device=dev)
    cur = torch.full((nt,), 1.0 / math.sqrt(4.0 * math.pi), dtype=torch.float64, device=dev)
    ce = torch.zeros(nt, dtype=torch.float64, device=dev)
    pm[0] = cur
    for m in range(1, lmax + 1):
        cur = cur * s * math.sqrt((2.0 * m + 1.0) / (2.0 * m))
        small = cur.abs() < _SMALL
        cur = torch.where(small, cur * _BIG, cur)
        ce = torch.where(small, ce - _RENORM, ce)
        pm[m] = cur
        pe[m] = ce
    # columns m of the recurrence in l, each with its own exponent ecol[m]
    ecol = pe.clone()
    p_prev2 = torch.zeros((lmax + 1, nt), dtype=torch.float64, device=dev)
    p_prev = torch.zeros((lmax + 1, nt), dtype=torch.float64, device=dev)
    mvec = torch.arange(lmax + 1, dtype=torch.float64, device=dev)
    for l in range(0, lmax + 1):
        p_l = torch.zeros((lmax + 1, nt), dtype=torch.float64, device=dev)
        if l >= 2:
            mm = mvec[: l - 1]
            a_l = torch.sqrt((4.0 * l * l - 1.0) / (l * l - mm * mm))
            a_lm1 = torch.sqrt((4.0 * (l - 1) ** 2 - 1.0) / ((l - 1) ** 2 - mm * mm))
            p_l[: l - 1] = a_l[:, None] * (x[None, :] * p_prev[: l - 1] - p_prev2[: l - 1] / a_lm1[:, None])
        if l >= 1:
            p_l[l - 1] = math.sqrt(2.0 * l + 1.0) * x * pm[l - 1]
        p_l[l] = pm[l]
        big = p_l.abs() > _BIG
        if bool(big.any()):
            p_l = torch.where(big, p_l * _SMALL, p_l)
            p_prev = torch.where(big, p_prev * _SMALL, p_prev)
            ecol = torch.where(big, ecol + _RENORM, ecol)
        yield l, _ldexp(p_l[: l + 1], ecol[: l + 1])
        p_prev2, p_prev = p_prev, p_l


def synthesize(coeffs: np.ndarray, n_theta: int, n_lambda: int, device="cpu", grid: str = "shifted") -> torch.Tensor:
    """Sample sum_lm C[l, L+m] Y_l^m on the grid; returns float64 [rows, n_lambda]
    (rows = n_theta, or n_theta + 1 on the grid with poles)."""
    coeffs = np.asarray(coeffs, dtype=np.float64)
    lmax = coeffs.shape[0] - 1
    if coeffs.shape != (lmax + 1, 2 * lmax + 1):
        raise ValueError("coefficient array must have shape (L+1, 2L+1)")
    dev = torch.device(device)
    theta = torch.tensor(grid_colatitudes(n_theta, grid), dtype=torch.float64, device=dev)
    rows = theta.shape[0]
    cc = torch.tensor(coeffs, dtype=torch.float64, device=dev)
    # column weights: cos part (m >= 0) and sin part (m > 0)
    ccos = cc[:, lmax:]                                   # [L+1, L+1]  m = 0..L
    csin = torch.flip(cc[:, : lmax + 1], dims=[1])        # [L+1, L+1]  index m -> C[l, L-m]
    csin = csin.clone()
    csin[:, 0] = 0.0

    acc_c = torch.zeros((lmax + 1, rows), dtype=torch.float64, device=dev)
    acc_s = torch.zeros((lmax + 1, rows), dtype=torch.float64, device=dev)
    for l, p_l in _legendre_columns(lmax, theta):
        acc_c[: l + 1] += ccos[l, : l + 1, None] * p_l
        acc_s[: l + 1] += csin[l, : l + 1, None] * p_l

    scale = torch.full((lmax + 1,), math.sqrt(2.0), dtype=torch.float64, device=dev)
    scale[0] = 1.0
    acc_c = acc_c * scale[:, None]
    acc_s = acc_s * scale[:, None]
    cos_t, sin_t = _angle_table(lmax, n_lambda, dev)
    f = acc_c.transpose(0, 1) @ cos_t + acc_s.transpose(0, 1) @ sin_t
    return f.contiguous()


def synthesize_many(coeff_list, n_theta: int, n_lambda: int, device="cpu") -> torch.Tensor:
    """synthesize() for several coefficient arrays of the same degree L on the
    same grid at once; returns float64 [P, n_theta, n_lambda]."""
    P = len(coeff_list)
    lmax = coeff_list[0].shape[0] - 1
    dev = torch.device(device)
    cc = torch.tensor(np.stack([np.asarray(c, dtype=np.float64) for c in coeff_list]), dtype=torch.float64,
                      device=dev)                                    # [P, L+1, 2L+1]
    theta = torch.tensor(colatitudes(n_theta), dtype=torch.float64, device=dev)
    ccos = cc[:, :, lmax:]                                           # [P, L+1, L+1] (m = 0..L)
    csin = torch.flip(cc[:, :, : lmax + 1], dims=[2]).clone()
    csin[:, :, 0] = 0.0
    acc_c = torch.zeros((P, lmax + 1, n_theta), dtype=torch.float64, device=dev)
    acc_s = torch.zeros((P, lmax + 1, n_theta), dtype=torch.float64, device=dev)
    for l, p_l in _legendre_columns(lmax, theta):
        acc_c[:, : l + 1] += ccos[:, l, : l + 1, None] * p_l[None]
        acc_s[:, : l + 1] += csin[:, l, : l + 1, None] * p_l[None]
    scale = torch.full((lmax + 1,), math.sqrt(2.0), dtype=torch.float64, device=dev)
    scale[0] = 1.0
    acc_c = acc_c * scale[None, :, None]
    acc_s = acc_s * scale[None, :, None]
    cos_t, sin_t = _angle_table(lmax, n_lambda, dev)
    f = acc_c.transpose(1, 2) @ cos_t + acc_s.transpose(1, 2) @ sin_t
    return f.contiguous()


def batched_sizes(count: int = 4096, seed: int = 1510080944):
    """The uneven-resolution batch's sizes (n_theta = 16 s, s uniform in 2..32,
    n_lambda = 2 n_theta) and per-problem seeds, from one PCG64 stream."""
    rng = np.random.Generator(np.random.PCG64(seed))
    svals = rng.integers(2, 33, size=count)
    seeds = rng.integers(0, 2**62, size=count)
    return [(16 * int(v), 32 * int(v)) for v in svals], seeds


def batched_workload(count: int = 4096, seed: int = 1510080944, device="cpu"):
    """The uneven-resolution batch: n_theta = 16 s with s uniform in 2..32,
    n_lambda = 2 n_theta, a random series l <= n_theta/2 with N(0,1)/(1+l)^2
    coefficients per problem (seeds drawn from one PCG64 stream).  Returns
    (sizes, f list, exact-solution list)."""
    sizes, seeds = batched_sizes(count, seed)
    fs = [None] * count
    us = [None] * count
    by_size = {}
    for b, sz in enumerate(sizes):
        by_size.setdefault(sz, []).append(b)
    for (nt, nl), idx in by_size.items():
        cs = [random_sh_coeffs(nt // 2, int(seeds[b]), "inv_sq") for b in idx]
        f = synthesize_many(cs, nt, nl, device)
        u = synthesize_many([poisson_exact(c) for c in cs], nt, nl, device)
        for q, b in enumerate(idx):
            fs[b] = f[q]
            us[b] = u[q]
    return sizes, fs, us


def poisson_exact(coeffs: np.ndarray) -> np.ndarray:
    """Coefficients of the zero-mean solution of Delta u = f for f = sum C Y:
    Delta Y_l^m = -l(l+1) Y_l^m, so u has C[l]/(-l(l+1)) and no l = 0 term."""
    coeffs = np.asarray(coeffs, dtype=np.float64)
    l = np.arange(coeffs.shape[0], dtype=np.float64)[:, None]
    out = np.zeros_like(coeffs)
    out[1:] = -coeffs[1:] / (l[1:] * (l[1:] + 1.0))
    return out


@dataclass
class Workload:
    """A named synthetic workload: grid size, coefficient recipe and seed."""

    name: str
    n_theta: int
    n_lambda: int
    lmax: int
    seed: int
    decay: str = "none"
    noise_sigma: float = 0.0
    extra: dict = field(default_factory=dict)

    def coeffs(self) -> np.ndarray:
        return random_sh_coeffs(self.lmax, self.seed, self.decay)

    def make(self, device="cpu"):
        """Returns (f, u_exact) as float64 tensors of shape [n_theta, n_lambda]."""
        c = self.coeffs()
        f = synthesize(c, self.n_theta, self.n_lambda, device)
        u = synthesize(poisson_exact(c), self.n_theta, self.n_lambda, device)
        return f, u

    def observation(self, device="cpu"):
        """u_obs for the inverse-source fit: the seeded series sampled on the grid
        plus i.i.d. N(0, noise_sigma^2) noise (seed + 1), float64 [n_theta, n_lambda]."""
        c = self.coeffs()
        u = synthesize(c, self.n_theta, self.n_lambda, device)
        rng = np.random.Generator(np.random.PCG64(self.seed + 1))
        noise = rng.standard_normal((self.n_theta, self.n_lambda)) * self.noise_sigma
        return u + torch.tensor(noise, dtype=torch.float64, device=u.device)


# Seeds follow 1510080940 + workload number.
WORKLOADS = {
    "sh20_64x128": Workload("sh20_64x128", 64, 128, 20, 1510080941),
    "sh2000_5000x10000": Workload("sh2000_5000x10000", 5000, 10000, 2000, 1510080942, "inv_sq"),
    "sh1024_2048x4096": Workload("sh1024_2048x4096", 2048, 4096, 1024, 1510080943, "inv_sq"),
    "sh2048_4096x8192": Workload("sh2048_4096x8192", 4096, 8192, 2048, 1510080943, "inv_sq"),
    "sh200_512x1024_noisy": Workload("sh200_512x1024_noisy", 512, 1024, 200, 1510080945, "inv_sq", 1e-3),
    # the paper-comparable size: mn/2 = 1.03e8 unknowns (its "100 million in a minute")
    "sh2000_7168x14336": Workload("sh2000_7168x14336", 7168, 14336, 2000, 1510080946, "inv_sq"),
    # half the longitudes of the 5000 x 10000 grid: the same colatitude transforms
    # (length 5000) on a 200 MB input, the kernel-profiling case
    "sh2000_5000x5000": Workload("sh2000_5000x5000", 5000, 5000, 2000, 1510080947, "inv_sq"),
}
# the batched workload (4096 uneven spheres) is built by batched_workload()


def workload(name: str) -> Workload:
    return WORKLOADS[name]
