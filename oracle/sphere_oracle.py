"""Plain, slow CPU FP64 oracle for the double-Fourier-sphere (DFS) spectral
Poisson solver on the unit sphere (Townsend, Wilber & Wright, "Computing with
functions in spherical and polar geometries I. The sphere", Section 5).

TEST INFRASTRUCTURE ONLY.  Only tests/, __graft_entry__.smoke() and bench.py's
CPU-baseline / reference legs may import this module.  The product path (the
CUDA library and its Python binding) never calls it, and the two share no code.

What it computes, step by step in the paper's order and notation:

  1. DFS doubling (Section 2.2, eq. BMCsphere): the samples f(lambda, theta) on
     theta in (0, pi) are extended to ftilde on [-pi, pi]^2 by the glide
     reflection ftilde(lambda, -theta) = f(lambda + pi, theta).  The grid is the
     pole-free DFS grid theta_p = -pi + (p + 1/2) 2pi/m, lambda_q = -pi + 2pi q/n
     with m = 2 n_theta, n = n_lambda (the paper is silent on the grid; this is
     the pole-avoiding alternative it mentions at the end of Section 4).
  2. F = matrix of 2D Fourier coefficients of sin^2(theta) ftilde in the
     expansion of eq. 2DFourierExpansion, j in [-m/2, m/2-1], k in [-n/2, n/2-1],
     computed by a naive 2D DFT (two dense DFT-matrix products) of the sampled
     product, normalised by 1/(mn).
  3. For each k the column system of eq. linearSystems,
        (M_sin^2 D_m^2 + M_cos M_sin D_m - k^2 I) X_k = F_k,
     with D_m, M_cos (Section 5) and M_sin (eq. Msin).  The sign of the k^2
     term follows the Sylvester form (eq. SylvesterSphericalPoisson): the
     column k of X D_n^2 is -k^2 X_k.  For k = 0 the zeroth row is replaced by
     w^T X_0 = 0 (eq. pentdiagonalPlusRankOne) with the weights w of
     eq. integrationCoeffs.
     Two readings of the truncated operator:
       "A" (literal): the products of the truncated m x m matrices.
       "B" (default): the exact banded entries of the infinite operator,
           a_j = (j-1)(j-2)/4 at column j-2, b_j = -j^2/2 - k^2, c_j =
           (j+1)(j+2)/4 at column j+2, on the symmetric window
           j in [-(m/2-1), m/2-1]; the theta-Nyquist mode j = -m/2 is zero.
  4. u = real part of the inverse 2D expansion (eq. tildeuFourierExpansion)
     evaluated on the theta > 0 half of the DFS grid.

The per-k systems are solved by dense LU (numpy.linalg.solve) at small m and
by LAPACK's banded LU (scipy.linalg.solve_banded) otherwise; neither uses the
parity split or the BMC fold, which are properties the tests check.

Also here: the same solve and its transpose on the grid with both poles
(theta_i = i pi / n_theta, i = 0..n_theta; the DFS grid theta_p = -pi + 2 pi p
/ m, the same per-k systems), the structure-preserving GE of Section 3 and the low-rank form of
the coefficients F, the surface integral sum2 (Section 4, Integration, eq.
integrationCoeffs), the tangential derivatives of Section 4 (Differentiation,
eqs. diff_x..diff_z with the division by sin theta through M_sin^{-1}) and the
vector-calculus operators built from them (divergence, curl, the curl of a
scalar function of eq. CurlScalarF, vorticity), the
transpose (adjoint) of the whole linear map f -> u, both matrix-free and as a
dense matrix for tiny grids, and the single-precision per-k solves refined by
FP64 residuals (refine_reference).
"""

from __future__ import annotations

import math

import numpy as np

try:  # scipy's banded LU is used for grids too large for dense LU
    import scipy.linalg as _sla
except Exception:  # pragma: no cover - scipy is present wherever the oracle runs
    _sla = None

DENSE_MAX_M = 256  # dense LU per k up to this DFS size


# ----------------------------------------------------------------------------
# Grid and DFS doubling (Section 2)
# ----------------------------------------------------------------------------

def dfs_theta(m: int) -> np.ndarray:
    """DFS colatitudes theta_p = -pi + (p + 1/2) 2 pi / m, p = 0..m-1."""
    p = np.arange(m, dtype=np.float64)
    return -math.pi + (p + 0.5) * 2.0 * math.pi / m


def dfs_lambda(n: int) -> np.ndarray:
    """DFS longitudes lambda_q = -pi + 2 pi q / n, q = 0..n-1."""
    q = np.arange(n, dtype=np.float64)
    return -math.pi + 2.0 * math.pi * q / n


def dfs_double(f: np.ndarray) -> np.ndarray:
    """eq. BMCsphere: ftilde on the m x n DFS grid from f on n_theta x n_lambda.

    Rows p >= n_theta hold theta_p = theta_{p - n_theta} > 0, where ftilde = f.
    Rows p < n_theta hold theta_p = -theta_{n_theta-1-p} < 0, where
    ftilde(lambda, theta) = f(lambda + pi, -theta) (lambda + pi taken mod 2 pi,
    which is the grid shift q -> q + n/2).
    """
    f = np.asarray(f, dtype=np.float64)
    nt, n = f.shape
    if n % 2:
        raise ValueError("n_lambda must be even for the DFS glide reflection")
    ft = np.empty((2 * nt, n), dtype=np.float64)
    ft[nt:] = f
    shifted = np.roll(f, -(n // 2), axis=1)          # shifted[:, q] = f[:, q + n/2]
    ft[:nt] = shifted[::-1]                            # row p <- f row n_theta-1-p
    return ft


# ----------------------------------------------------------------------------
# 2D Fourier coefficients and samples (Section 4, eq. 2DFourierExpansion)
# ----------------------------------------------------------------------------

def _phase_theta(m: int) -> np.ndarray:
    """E[j + m/2, p] = exp(-i j theta_p), the exponent reduced exactly:
    j theta_p = pi * j (2p + 1 - m) / m."""
    j = np.arange(-m // 2, m // 2, dtype=np.int64)[:, None]
    p = np.arange(m, dtype=np.int64)[None, :]
    r = np.mod(j * (2 * p + 1 - m), 2 * m).astype(np.float64)
    ang = math.pi * r / m
    return np.cos(ang) - 1j * np.sin(ang)


def _phase_lambda(n: int) -> np.ndarray:
    """E[k + n/2, q] = exp(-i k lambda_q), k lambda_q = pi * k (2q - n) / n."""
    k = np.arange(-n // 2, n // 2, dtype=np.int64)[:, None]
    q = np.arange(n, dtype=np.int64)[None, :]
    r = np.mod(k * (2 * q - n), 2 * n).astype(np.float64)
    ang = math.pi * r / n
    return np.cos(ang) - 1j * np.sin(ang)


def coeffs2(values: np.ndarray) -> np.ndarray:
    """Naive 2D DFT: X[j + m/2, k + n/2] = (1/mn) sum_pq v(lambda_q, theta_p)
    exp(-i j theta_p) exp(-i k lambda_q)  (the interpolant's coefficients)."""
    m, n = values.shape
    return (_phase_theta(m) @ values @ _phase_lambda(n).T) / (m * n)


def sample(X: np.ndarray) -> np.ndarray:
    """Inverse of coeffs2: values sum_jk X_jk exp(i j theta_p) exp(i k lambda_q)
    on the m x n DFS grid (complex)."""
    m, n = X.shape
    return _phase_theta(m).conj().T @ X @ _phase_lambda(n).conj()


# ----------------------------------------------------------------------------
# Operators (Section 4 eq. Msin, Section 5)
# ----------------------------------------------------------------------------

def op_Dm(m: int) -> np.ndarray:
    """D_m = diag(i j), j = -m/2..m/2-1  (d/dtheta)."""
    return np.diag(1j * np.arange(-m // 2, m // 2, dtype=np.float64))


def op_Mcos(m: int) -> np.ndarray:
    """M_cos = (1/2) [ones on the sub- and super-diagonal]  (multiply by cos theta)."""
    return 0.5 * (np.eye(m, k=1) + np.eye(m, k=-1))


def op_Msin(m: int) -> np.ndarray:
    """M_sin = (i/2) [+1 on the super-diagonal, -1 on the sub-diagonal] (eq. Msin)."""
    return 0.5j * (np.eye(m, k=1) - np.eye(m, k=-1))


def theta_operator_A(m: int) -> np.ndarray:
    """Reading A: M_sin^2 D_m^2 + M_cos M_sin D_m from the truncated matrices
    (eq. SylvesterSphericalPoisson, left factor).  Real-valued."""
    D = op_Dm(m)
    Ms = op_Msin(m)
    Mc = op_Mcos(m)
    L = Ms @ Ms @ D @ D + Mc @ Ms @ D
    assert np.abs(L.imag).max() < 1e-12 * max(1.0, np.abs(L.real).max())
    return L.real.copy()


def theta_bands_B(m: int) -> tuple[np.ndarray, np.ndarray, np.ndarray]:
    """Reading B: entries of sin^2 d2/dtheta2 + sin cos d/dtheta on e^{ij theta}
    for j = -m/2..m/2-1: row j has a_j at column j-2, b_j (without -k^2) at j,
    c_j at column j+2.  Derived from sin^2 = 1/2 - (e^{2i t} + e^{-2i t})/4 and
    sin cos = (e^{2i t} - e^{-2i t})/(4i)."""
    j = np.arange(-m // 2, m // 2, dtype=np.float64)
    a = (j - 1.0) * (j - 2.0) / 4.0
    b = -(j * j) / 2.0
    c = (j + 1.0) * (j + 2.0) / 4.0
    return a, b, c


def theta_operator_B(m: int) -> np.ndarray:
    """Reading B as a dense m x m matrix; the Nyquist row/column j = -m/2 is
    removed from the system (its row is the identity, forcing X_{-m/2} = 0)."""
    a, b, c = theta_bands_B(m)
    L = np.diag(b) + np.diag(a[2:], k=-2) + np.diag(c[:-2], k=2)
    L[0, :] = 0.0
    L[:, 0] = 0.0
    return L


def integration_weights(m: int) -> np.ndarray:
    """eq. integrationCoeffs: w_j = (1 + e^{i pi j}) / (1 - j^2), w_{+-1} = 0,
    j = -m/2..m/2-1, so that int_0^pi c(theta) sin(theta) dtheta = sum_j w_j a_j
    for a theta-even c."""
    j = np.arange(-m // 2, m // 2, dtype=np.int64)
    w = np.zeros(m, dtype=np.float64)
    even = (j % 2) == 0
    w[even] = 2.0 / (1.0 - j[even].astype(np.float64) ** 2)
    return w


def system_matrix(m: int, k: int, reading: str = "B") -> np.ndarray:
    """Dense matrix of the k-th column system (eq. linearSystems); for k = 0
    the zeroth row is replaced by w^T (eq. pentdiagonalPlusRankOne)."""
    if reading == "A":
        L = theta_operator_A(m) - float(k * k) * np.eye(m)
    elif reading == "B":
        L = theta_operator_B(m) - float(k * k) * np.eye(m)
        L[0, 0] = 1.0  # X_{-m/2} = 0
    else:
        raise ValueError(reading)
    if k == 0:
        w = integration_weights(m)
        if reading == "B":
            w = w.copy()
            w[0] = 0.0
        L[m // 2, :] = w
    return L


def _bands_of(m: int, k: int, reading: str):
    """Diagonals (offsets -2, 0, +2) of the k-th system before the k = 0 row
    replacement.  Reading A's bands are read off the literal matrix product."""
    if reading == "A":
        L = theta_operator_A(m)
        sub = np.zeros(m)
        sup = np.zeros(m)
        sub[2:] = np.diag(L, k=-2)
        sup[:-2] = np.diag(L, k=2)
        d = np.diag(L).copy() - float(k * k)
        # the literal product has no entries off the 0, +-2 diagonals
        return sub, d, sup
    a, b, c = theta_bands_B(m)
    sub = a.copy()
    sub[:2] = 0.0
    sup = c.copy()
    sup[-2:] = 0.0
    d = b - float(k * k)
    # Nyquist row/column j = -m/2 (index 0) removed: identity row
    d[0] = 1.0
    sup[0] = 0.0
    sub[2] = 0.0
    return sub, d, sup


def _banded_solve(sub, d, sup, rhs):
    """Solve the pentadiagonal-band (offsets -2, 0, +2) system with LAPACK."""
    mm = d.shape[0]
    ab = np.zeros((5, mm), dtype=np.float64)
    ab[0, 2:] = sup[:-2]   # upper diagonal +2: ab[u + i - j, j] with u = 2
    ab[2, :] = d
    ab[4, :-2] = sub[2:]   # lower diagonal -2
    return _sla.solve_banded((2, 2), ab, rhs)


def solve_columns(F: np.ndarray, reading: str = "B", method: str = "auto") -> np.ndarray:
    """X with X_k solving the k-th system of eq. linearSystems for every k."""
    m, n = F.shape
    if method == "auto":
        method = "dense" if m <= DENSE_MAX_M else "banded"
    X = np.zeros_like(F, dtype=np.complex128)
    for kk in range(n):
        k = kk - n // 2
        if method == "dense":
            rhs = F[:, kk].astype(np.complex128).copy()
            if k == 0:
                rhs[m // 2] = 0.0
            if reading == "B":
                rhs[0] = 0.0
            X[:, kk] = np.linalg.solve(system_matrix(m, k, reading), rhs)
        else:
            X[:, kk] = _solve_one(F[:, kk], m, k, reading, banded=True)
    return X


def apply_columns(X: np.ndarray, reading: str = "B") -> np.ndarray:
    """L_k X_k for every k (the operator of eq. linearSystems, no row replaced)."""
    m, n = X.shape
    out = np.zeros_like(X, dtype=np.complex128)
    for kk in range(n):
        k = kk - n // 2
        if reading == "A":
            L = theta_operator_A(m) - float(k * k) * np.eye(m)
        else:
            L = theta_operator_B(m) - float(k * k) * np.eye(m)
        out[:, kk] = L @ X[:, kk]
    return out


# ----------------------------------------------------------------------------
# The solver (Section 5) and sum2 (Section 4)
# ----------------------------------------------------------------------------

def rhs_coefficients(f: np.ndarray) -> np.ndarray:
    """F = 2D Fourier coefficients of sin^2(theta) ftilde (eq. SylvesterSphericalPoisson)."""
    ft = dfs_double(f)
    m, _ = ft.shape
    s2 = np.sin(dfs_theta(m)) ** 2
    return coeffs2(s2[:, None] * ft)


def poisson(f: np.ndarray, reading: str = "B", method: str = "auto", return_all: bool = False):
    """u on the n_theta x n_lambda grid with Delta u = f and zero sphere mean.

    f must have zero sphere mean (the paper's assumption).  Returns u, or
    (u, F, X, imag_max) with return_all."""
    f = np.asarray(f, dtype=np.float64)
    nt, n = f.shape
    F = rhs_coefficients(f)
    X = solve_columns(F, reading, method)
    U = sample(X)[nt:]
    u = U.real.copy()
    if return_all:
        return u, F, X, float(np.abs(U.imag).max())
    return u


# ----------------------------------------------------------------------------
# The grid with both poles (Section 2: the DFS grid of a function sampled on
# theta in [0, pi], the poles included)
#
# theta_i = i pi / n_theta, i = 0..n_theta (n_theta + 1 rows, both poles);
# doubled, theta_p = -pi + 2 pi p / m, p = 0..m-1, m = 2 n_theta: row p =
# n_theta + i holds theta_i (i = 0..n_theta-1) and row p = n_theta - i holds
# -theta_i (i = 1..n_theta; p = 0 is theta = -pi, the south pole seen from the
# other side).  The per-k systems are those of the pole-free grid (they act on
# coefficients, not samples; reading B, theta-Nyquist mode dropped), only the
# samples change.
# ----------------------------------------------------------------------------

def pole_colatitudes(n_theta: int) -> np.ndarray:
    """theta_i = i pi / n_theta, i = 0..n_theta."""
    return np.arange(n_theta + 1, dtype=np.float64) * math.pi / n_theta


def dfs_theta_poles(m: int) -> np.ndarray:
    """theta_p = -pi + 2 pi p / m, p = 0..m-1."""
    return -math.pi + 2.0 * math.pi * np.arange(m, dtype=np.float64) / m


def dfs_double_poles(f: np.ndarray) -> np.ndarray:
    """eq. BMCsphere on the grid with poles: f has n_theta + 1 rows
    (theta_0 = 0 .. theta_{n_theta} = pi); ftilde has m = 2 n_theta rows.
    Rows p >= n_theta: ftilde = f row p - n_theta.  Rows p < n_theta hold
    theta_p = -theta_{n_theta - p}: ftilde(lambda, theta_p) = f(lambda + pi,
    theta_{n_theta - p}) (the shift q -> q + n/2)."""
    f = np.asarray(f, dtype=np.float64)
    rows, n = f.shape
    nt = rows - 1
    if n % 2 or nt < 1:
        raise ValueError("n_lambda must be even and n_theta >= 1")
    ft = np.empty((2 * nt, n), dtype=np.float64)
    ft[nt:] = f[:nt]
    shifted = np.roll(f, -(n // 2), axis=1)
    ft[:nt] = shifted[nt:0:-1]                     # row p <- f row n_theta - p, p = 0..n_theta-1
    return ft


def _phase_theta_poles(m: int) -> np.ndarray:
    """E[j + m/2, p] = exp(-i j theta_p), j theta_p = pi j (2p - m) / m reduced exactly."""
    j = np.arange(-m // 2, m // 2, dtype=np.int64)[:, None]
    p = np.arange(m, dtype=np.int64)[None, :]
    r = np.mod(j * (2 * p - m), 2 * m).astype(np.float64)
    ang = math.pi * r / m
    return np.cos(ang) - 1j * np.sin(ang)


def coeffs2_poles(values: np.ndarray) -> np.ndarray:
    """Naive 2D DFT of values on the m x n DFS grid with poles, normalised by 1/(mn)."""
    m, n = values.shape
    return (_phase_theta_poles(m) @ values @ _phase_lambda(n).T) / (m * n)


def sample_poles(X: np.ndarray) -> np.ndarray:
    """Inverse of coeffs2_poles: sum_jk X_jk exp(i j theta_p) exp(i k lambda_q) (complex)."""
    m, n = X.shape
    return _phase_theta_poles(m).conj().T @ X @ _phase_lambda(n).conj()


def rhs_coefficients_poles(f: np.ndarray) -> np.ndarray:
    """F of eq. SylvesterSphericalPoisson from samples on the grid with poles."""
    ft = dfs_double_poles(f)
    m, _ = ft.shape
    s2 = np.sin(dfs_theta_poles(m)) ** 2
    return coeffs2_poles(s2[:, None] * ft)


def poisson_poles(f: np.ndarray, reading: str = "B", method: str = "auto", return_all: bool = False):
    """u on the (n_theta + 1) x n_lambda grid with poles, Delta u = f, zero mean.

    The samples of f on the pole rows do not enter (sin^2 theta vanishes
    there).  u on rows i = 0..n_theta-1 is the interpolant at theta_i = theta_p,
    p = n_theta + i; on the south pole row i = n_theta it is the interpolant at
    theta = -pi, the same point as theta = pi by periodicity (no shift)."""
    f = np.asarray(f, dtype=np.float64)
    nt = f.shape[0] - 1
    F = rhs_coefficients_poles(f)
    X = solve_columns(F, reading, method)
    U = sample_poles(X)
    U = np.concatenate([U[nt:], U[:1]], axis=0)
    u = U.real.copy()
    if return_all:
        return u, F, X, float(np.abs(U.imag).max())
    return u


def sum2_poles(values_on_grid: np.ndarray) -> float:
    """sum2 on the grid with poles: 2 pi sum_j w_j A_{j,0}, A = coeffs2_poles(ftilde),
    over the symmetric window |j| <= m/2 - 1 of the solve (reading B).  On this
    grid the theta-Nyquist coefficient of a theta-even column is not zero (the
    doubled samples pair p with m - p, of the same parity), unlike the
    pole-free grid's, so the window is stated: the Nyquist term is left out."""
    ft = dfs_double_poles(values_on_grid)
    m, n = ft.shape
    A = coeffs2_poles(ft)
    w = integration_weights(m)
    w[0] = 0.0                                  # j = -m/2
    return float((2.0 * math.pi * (w @ A[:, n // 2])).real)


def sum2(values_on_grid: np.ndarray) -> float:
    """Surface integral over the unit sphere (Section 4, Integration):
    2 pi sum_j w_j A_{j,0} with A = coeffs2(ftilde)."""
    ft = dfs_double(values_on_grid)
    m, n = ft.shape
    A = coeffs2(ft)
    col0 = A[:, n // 2]
    val = 2.0 * math.pi * (integration_weights(m) @ col0)
    return float(val.real)


# ----------------------------------------------------------------------------
# Structure-preserving Gaussian elimination and low-rank coefficients
# (Section 3, Figure GaussianElimination; Section 4, eq. 2DFourierExpansion)
# ----------------------------------------------------------------------------

def pivot_pinv(a: float, b: float, alpha: float = 0.01) -> np.ndarray:
    """The epsilon-pseudoinverse (Definition pseudoinverse) of the centrosymmetric
    pivot matrix M = [[a, b], [b, a]] (eq. pivotMatrix) with eps = alpha sigma_1(M):
    M has the eigenvectors (1, 1)/sqrt2 and (1, -1)/sqrt2 with eigenvalues a + b
    and a - b, so sigma_{1,2} = max / min(|a + b|, |a - b|) (eq. SingularValues)
    and the pseudoinverse keeps the eigenpairs with |eigenvalue| > eps."""
    sig1 = max(abs(a + b), abs(a - b))
    eps = alpha * sig1
    P = np.zeros((2, 2))
    for lam, v in ((a + b, np.array([1.0, 1.0])), (a - b, np.array([1.0, -1.0]))):
        if abs(lam) > eps:
            P += np.outer(v, v) / (2.0 * lam)
    return P


def bmc_ge(ft: np.ndarray, alpha: float = 0.01, rtol: float = 1e-13, max_terms: int = 512):
    """Structure-preserving GE on the samples ft (m x n, the DFS grid) of a BMC
    function (Section 3, Figure GaussianElimination).  Step k: pick the grid
    point (lambda*, theta*) in [0, pi) x (0, pi) whose pivot matrix
    M = [[e(lambda* - pi, theta*), e(lambda*, theta*)], [e(lambda*, theta*),
    e(lambda* - pi, theta*)]] has the largest sigma_1 (the 2 x 2 analogue of
    complete pivoting, over the whole grid), then
        e <- e - [e(lambda* - pi, .)  e(lambda*, .)] M^{dagger_eps} [e(., theta*); e(., -theta*)]
    (eq. GEstructurePreservingStepPseudoinverse) with eps = alpha sigma_1(M),
    alpha = 1/100 as the paper chooses.
    Readings: the pivot search runs over the full sample grid (the paper's
    coarse-grid search is a speed device); the iteration stops when
    max |e| <= rtol max |ft| (rtol = 1e-13: "machine precision relative to the
    maximum" for a residual whose rounding floor is tens of eps), when the
    residual, already below 1e-9 max |ft|, stops decreasing for three steps
    (the rounding floor), or after max_terms steps.  The
    pole zero-out of eq. ZeroOut (for BMC-I structure) is not applied: the
    sample grid has no pole points.
    Returns (terms, residual); each term is (cols m x 2, P 2 x 2, rows 2 x n,
    (p, q)) with ft ~= sum cols @ P @ rows, p, q the pivot's row and column."""
    ft = np.asarray(ft, dtype=np.float64)
    m, n = ft.shape
    N, H = m // 2, n // 2
    e = ft.copy()
    scale = float(np.abs(ft).max())
    terms = []
    best, stall = np.inf, 0
    for _ in range(max_terms):
        r = float(np.abs(e).max())
        if r <= rtol * scale:
            break
        if r < best:
            best, stall = r, 0
        elif r < 1e-9 * scale:                        # at the rounding floor
            stall += 1
            if stall >= 3:
                break
        a = np.roll(e, H, axis=1)                     # a[p, q] = e[p, q - n/2]
        s1 = np.maximum(np.abs(a + e), np.abs(a - e))[N:, H:]
        i, j = np.unravel_index(int(np.argmax(s1)), s1.shape)
        p, q = N + int(i), H + int(j)
        P = pivot_pinv(float(e[p, q - H]), float(e[p, q]), alpha)
        cols = e[:, [q - H, q]].copy()
        rows = e[[p, m - 1 - p], :].copy()
        e = e - cols @ P @ rows
        terms.append((cols, P, rows, (p, q)))
    return terms, e


def lowrank_values(terms) -> np.ndarray:
    """sum of cols @ P @ rows: the low-rank approximant on the DFS grid."""
    return sum(c @ P @ r for c, P, r, _ in terms)


def lowrank_rhs_coefficients(terms, m: int, n: int) -> np.ndarray:
    """F of the Poisson solve (the 2D Fourier coefficients of sin^2(theta) ftilde)
    from the low-rank factors by 1D transforms only (Section 4, low-rank form of
    eq. 2DFourierExpansion): F = sum_t [DFT_theta(sin^2 c_t)] P_t [DFT_lambda(r_t)]^T,
    with the naive DFTs of coeffs2 in each variable."""
    s2 = np.sin(dfs_theta(m)) ** 2
    Et, El = _phase_theta(m), _phase_lambda(n)
    F = np.zeros((m, n), dtype=complex)
    for c, P, r, _ in terms:
        Ch = (Et @ (s2[:, None] * c)) / m            # m x 2
        Rh = (El @ r.T) / n                          # n x 2
        F += Ch @ P @ Rh.T
    return F


# ----------------------------------------------------------------------------
# Tangential derivatives (Section 4, Differentiation: eqs. diff_x, diff_y,
# diff_z, dfdx and Msin)
# ----------------------------------------------------------------------------

def tangential_gradient(f: np.ndarray, chop: float = 0.0):
    """(d^t f/dx, d^t f/dy, d^t f/dz) on the n_theta x n_lambda grid, the
    Cartesian components of the surface gradient, computed in coefficient space
    as the paper does:
        d^t/dx = -(sin lambda / sin theta) d/dlambda + cos lambda cos theta d/dtheta   (eq. diff_x)
        d^t/dy =  (cos lambda / sin theta) d/dlambda + sin lambda cos theta d/dtheta   (eq. diff_y)
        d^t/dz = -sin theta d/dtheta
    on X = coeffs2(ftilde): d/dtheta = D_m from the left, d/dlambda = D_n from
    the right, cos / sin theta = M_cos / M_sin from the left, cos / sin lambda
    the same matrices of size n acting on the k index, 1/sin theta = M_sin^{-1}
    (eq. Msin; M_sin is invertible for even m).
    Readings: (1) eq. diff_z prints +sin theta d/dtheta; with the colatitude of
    eq. sphericalCoordinates the chain rule gives e_z . theta_hat = -sin theta,
    so the sign here is minus (the tangency x g_x + y g_y + z g_z = 0 holds only
    with it).  (2) The Nyquist modes j = -m/2 and k = -n/2 of X are dropped
    before the operators act and of each result after, so the truncation is
    symmetric (as in the solver's reading B); modes the products push beyond the
    m x n window are discarded.  (3) chop > 0: coefficients with
    |X_jk| <= chop max |X| are set to zero first, the grid counterpart of the
    constructor resolving a function to a tolerance relative to its maximum
    (Section 3).  (4) The window j in [-m/2, m/2-1] of eq. Msin is not symmetric
    about j = 0: when the quotient is not band-limited inside it, the solve
    also returns a part without the symmetry q_{-j,k} = -(-1)^k q_{j,k} that a
    quotient by sin theta of a function on the sphere has (Section 2, BMC
    functions).  That part never reaches the results on theta > 0: dropping the
    theta-Nyquist row of each result and taking the real part removes it, so
    the results are those of the symmetric part alone."""
    ft = dfs_double(f)
    m, n = ft.shape
    nt = m // 2
    X = coeffs2(ft)
    X[0, :] = 0.0
    X[:, 0] = 0.0
    if chop > 0.0:
        X[np.abs(X) <= chop * np.abs(X).max()] = 0.0
    Dm, Dn = op_Dm(m), op_Dm(n)
    Mcos_t, Msin_t = op_Mcos(m), op_Msin(m)
    Mcos_l, Msin_l = op_Mcos(n), op_Msin(n)
    dth = Dm @ X                               # d/dtheta
    dla = X @ Dn                               # d/dlambda
    q = np.linalg.solve(Msin_t, dla)           # (1/sin theta) d/dlambda
    c = Mcos_t @ dth                           # cos theta d/dtheta
    gx = -(q @ Msin_l.T) + c @ Mcos_l.T        # multiplication by sin / cos lambda acts on k
    gy = q @ Mcos_l.T + c @ Msin_l.T
    gz = -(Msin_t @ dth)
    out = []
    for G in (gx, gy, gz):
        G = G.copy()
        G[0, :] = 0.0
        G[:, 0] = 0.0
        out.append(sample(G)[nt:].real.copy())
    return tuple(out)


# ----------------------------------------------------------------------------
# Vector calculus (Section 4, vector-valued functions): every operator is a
# combination of the tangential derivatives above, in the paper's formulas
# ----------------------------------------------------------------------------

def unit_normal(n_theta: int, n_lambda: int):
    """(x, y, z) of eq. sphericalCoordinates on the n_theta x n_lambda grid
    (theta > 0 half of the DFS grid): the outward unit normal n = (x, y, z)."""
    th = dfs_theta(2 * n_theta)[n_theta:][:, None]
    la = dfs_lambda(n_lambda)[None, :]
    return np.cos(la) * np.sin(th), np.sin(la) * np.sin(th), np.cos(th) + 0.0 * la


def divergence(f1: np.ndarray, f2: np.ndarray, f3: np.ndarray, chop: float = 0.0) -> np.ndarray:
    """Surface divergence of the field (f1, f2, f3): d^t f1/dx + d^t f2/dy + d^t f3/dz."""
    return (tangential_gradient(f1, chop)[0] + tangential_gradient(f2, chop)[1]
            + tangential_gradient(f3, chop)[2])


def curl(f1: np.ndarray, f2: np.ndarray, f3: np.ndarray, chop: float = 0.0):
    """Surface curl of the field (f1, f2, f3), component by component:
    (d^t f3/dy - d^t f2/dz, d^t f1/dz - d^t f3/dx, d^t f2/dx - d^t f1/dy).
    For a tangent field its normal component is the vorticity (see vorticity);
    the result is tangent only where that vanishes."""
    g1, g2, g3 = (tangential_gradient(fc, chop) for fc in (f1, f2, f3))
    return (g3[1] - g2[2], g1[2] - g3[0], g2[0] - g1[1])


def scalar_curl(f: np.ndarray, chop: float = 0.0):
    """Curl of a scalar function (eq. CurlScalarF): n x grad f, with n = (x, y, z),
    = (y d^t f/dz - z d^t f/dy, z d^t f/dx - x d^t f/dz, x d^t f/dy - y d^t f/dx)."""
    x, y, z = unit_normal(*f.shape)
    gx, gy, gz = tangential_gradient(f, chop)
    return (y * gz - z * gy, z * gx - x * gz, x * gy - y * gx)


def vorticity(f1: np.ndarray, f2: np.ndarray, f3: np.ndarray, chop: float = 0.0) -> np.ndarray:
    """Vorticity of the field, the scalar (curl f) . n."""
    x, y, z = unit_normal(*f1.shape)
    c1, c2, c3 = curl(f1, f2, f3, chop)
    return x * c1 + y * c2 + z * c3


# ----------------------------------------------------------------------------
# Transpose of the linear map f -> u (for gradients)
# ----------------------------------------------------------------------------

def _solve_columns_T(B: np.ndarray, reading: str = "B") -> np.ndarray:
    """Y with M_k^T Y_k = B_k, M_k the (row-replaced) system matrix of column k.
    Dense LU at small m; otherwise LAPACK's banded LU on the transposed bands
    (for k = 0 the transposed system has the dense column w: its row j = 0
    gives Y_0 = B_0 / w_0 first, the rest is banded)."""
    m, n = B.shape
    Y = np.zeros_like(B, dtype=np.complex128)
    for kk in range(n):
        k = kk - n // 2
        if m <= DENSE_MAX_M:
            Y[:, kk] = np.linalg.solve(system_matrix(m, k, reading).T, B[:, kk])
            continue
        sub, d, sup = _bands_of(m, k, reading)
        # (M^T)[i, i-2] = M[i-2, i] = sup[i-2],  (M^T)[i, i+2] = M[i+2, i] = sub[i+2]
        subT = np.zeros(m)
        supT = np.zeros(m)
        subT[2:] = sup[:-2]
        supT[:-2] = sub[2:]
        rhs = B[:, kk].astype(np.complex128)
        if k != 0:
            Y[:, kk] = _banded_solve(subT, d, supT, rhs)
            continue
        i0 = m // 2
        w = integration_weights(m)
        if reading == "B":
            w[0] = 0.0
        y0 = rhs[i0] / w[i0]
        keep = np.arange(m) != i0
        sub_r = subT[keep].copy()
        sup_r = supT[keep].copy()
        sub_r[i0] = 0.0
        sub_r[i0 + 1] = 0.0
        sup_r[i0 - 2] = 0.0
        sup_r[i0 - 1] = 0.0
        yr = _banded_solve(sub_r, d[keep], sup_r, rhs[keep] - w[keep] * y0)
        y = np.zeros(m, dtype=np.complex128)
        y[keep] = yr
        y[i0] = y0
        Y[:, kk] = y
    return Y


def poisson_adjoint(g: np.ndarray, reading: str = "B") -> np.ndarray:
    """S^T g for the real-linear map S: f -> u of poisson(), by transposing each
    step: restriction -> zero-extension, Re -> real embedding, complex-linear
    maps -> conjugate transposes, row replacement and Nyquist removal ->
    transposed system matrices, DFS doubling -> folding of mirrored rows."""
    g = np.asarray(g, dtype=np.float64)
    nt, n = g.shape
    m = 2 * nt
    # u = Re(sample(X))[nt:]  ->  transpose: zero-extend, then sample^H
    Gfull = np.zeros((m, n), dtype=np.complex128)
    Gfull[nt:] = g
    Et = _phase_theta(m)
    El = _phase_lambda(n)
    Xbar = Et @ Gfull @ El.T                       # (E^H)^H G (conj E)^H
    # X = M^{-1} R F (R zeroes the replaced rows of the right-hand side)
    Fbar = _solve_columns_T(Xbar, reading)
    Fbar[m // 2, n // 2] = 0.0
    if reading == "B":
        Fbar[0, :] = 0.0
    # F = coeffs2(s2 * ftilde)  ->  real part of the conjugate-transposed DFT
    Vbar = (Et.conj().T @ Fbar @ El.conj()) / (m * n)
    vbar = Vbar.real
    s2 = np.sin(dfs_theta(m)) ** 2
    vbar = s2[:, None] * vbar
    # ftilde = E f  ->  fold mirrored rows back
    out = vbar[nt:].copy()
    back = vbar[:nt][::-1]                         # row n_theta-1-p -> f row i
    out += np.roll(back, n // 2, axis=1)           # undo the q + n/2 shift
    return out


def poisson_poles_adjoint(g: np.ndarray, reading: str = "B") -> np.ndarray:
    """S^T g for the real-linear map S: f -> u of poisson_poles(), step by step
    as poisson_adjoint: the restriction to the rows p = n_theta..m-1 and p = 0
    becomes a zero-extension, the complex-linear maps their conjugate
    transposes, and the doubling with poles (rows p = n_theta + i from f row i,
    rows p = n_theta - i from f row i at lambda + pi) a fold."""
    g = np.asarray(g, dtype=np.float64)
    rows, n = g.shape
    nt = rows - 1
    m = 2 * nt
    Gfull = np.zeros((m, n), dtype=np.complex128)
    Gfull[nt:] = g[:nt]
    Gfull[0] += g[nt]
    Et = _phase_theta_poles(m)
    El = _phase_lambda(n)
    Xbar = Et @ Gfull @ El.T
    Fbar = _solve_columns_T(Xbar, reading)
    Fbar[m // 2, n // 2] = 0.0
    if reading == "B":
        Fbar[0, :] = 0.0
    Vbar = (Et.conj().T @ Fbar @ El.conj()) / (m * n)
    vbar = np.sin(dfs_theta_poles(m))[:, None] ** 2 * Vbar.real
    out = np.zeros((rows, n), dtype=np.float64)
    out[:nt] += vbar[nt:]
    out[nt:0:-1] += np.roll(vbar[:nt], n // 2, axis=1)   # row p < n_theta from f row n_theta - p
    return out


# ----------------------------------------------------------------------------
# Residual refinement of the per-k solves (the single-precision form)
# ----------------------------------------------------------------------------

def _solve_one_fp32(Fk: np.ndarray, m: int, k: int, reading: str = "B") -> np.ndarray:
    """X_k of one column system with k != 0 (eq. linearSystems) by LU in IEEE
    single precision: the bands and the right-hand side rounded to float32 /
    complex64, LAPACK's single-precision banded solve, the result widened."""
    rhs = Fk.astype(np.complex128).copy()
    if reading == "B":
        rhs[0] = 0.0
    sub, d, sup = _bands_of(m, k, reading)
    ab = np.zeros((5, m), dtype=np.float32)
    ab[0, 2:] = sup[:-2]
    ab[2, :] = d
    ab[4, :-2] = sub[2:]
    return _sla.solve_banded((2, 2), ab, rhs.astype(np.complex64)).astype(np.complex128)


def _replaced_system_apply(X: np.ndarray, reading: str = "B") -> np.ndarray:
    """M_k X_k for every k, M_k the system actually solved: the bands of
    eq. linearSystems with the Nyquist row j = -m/2 the identity (reading B) and,
    for k = 0, row j = 0 replaced by w^T (eq. pentdiagonalPlusRankOne)."""
    m, n = X.shape
    out = np.zeros_like(X, dtype=np.complex128)
    for kk in range(n):
        k = kk - n // 2
        sub, d, sup = _bands_of(m, k, reading)
        x = X[:, kk]
        y = d * x
        y[2:] += sub[2:] * x[:-2]
        y[:-2] += sup[:-2] * x[2:]
        if k == 0:
            w = integration_weights(m)
            if reading == "B":
                w[0] = 0.0
            y[m // 2] = w @ x
        out[:, kk] = y
    return out


def refine_reference(f: np.ndarray, sweeps: int, reading: str = "B"):
    """The single-precision form with residual refinement, in coefficient space:
    X_0 = S32 F and X_{s+1} = X_s + S32 (F~ - M X_s), where F~ is F of
    eq. SylvesterSphericalPoisson with the replaced rows zeroed, M the systems
    actually solved (see _replaced_system_apply), the residual formed in FP64,
    and S32 solves every k != 0 column in single precision and the
    ill-conditioned k = 0 column (eq. pentdiagonalPlusRankOne) in FP64.  F and
    the final synthesis are FP64.  Returns [u_0, u_1, ..., u_sweeps], the grid
    values after each number of sweeps."""
    f = np.asarray(f, dtype=np.float64)
    nt, n = f.shape
    m = 2 * nt
    F = rhs_coefficients(f)
    Ft = F.copy()
    Ft[m // 2, n // 2] = 0.0
    if reading == "B":
        Ft[0, :] = 0.0

    def s32(R):
        X = np.zeros_like(R, dtype=np.complex128)
        for kk in range(n):
            k = kk - n // 2
            X[:, kk] = _solve_one(R[:, kk], m, 0, reading) if k == 0 else _solve_one_fp32(R[:, kk], m, k, reading)
        return X

    X = s32(F)
    out = [sample(X)[nt:].real.copy()]
    for _ in range(sweeps):
        X = X + s32(Ft - _replaced_system_apply(X, reading))
        out.append(sample(X)[nt:].real.copy())
    return out


def dense_solution_operator(n_theta: int, n_lambda: int, reading: str = "B") -> np.ndarray:
    """The matrix S of f -> u (columns = responses to unit inputs); tiny grids."""
    N = n_theta * n_lambda
    S = np.zeros((N, N))
    for idx in range(N):
        e = np.zeros(N)
        e[idx] = 1.0
        S[:, idx] = poisson(e.reshape(n_theta, n_lambda), reading, "dense").ravel()
    return S


# ----------------------------------------------------------------------------
# Sampled columns, for grids too large for the full 2D DFT
# ----------------------------------------------------------------------------

_theta_cache: dict = {}


def _theta_phase_cached(m: int) -> np.ndarray:
    """_phase_theta(m), kept for the last size used (1.6 GB at m = 10^4)."""
    E = _theta_cache.get(m)
    if E is None:
        _theta_cache.clear()
        E = _phase_theta(m)
        _theta_cache[m] = E
    return E


def sampled_columns(f: np.ndarray, ks, reading: str = "B"):
    """For each wavenumber k in ks, the column U_k(theta_i) = sum_j X_jk e^{i j theta_i}
    of the solution on the theta > 0 rows, where X_k solves the k-th system of
    eq. linearSystems with F_k from the same naive DFT as coeffs2 restricted to
    column k.  Then u(lambda_q, theta_i) = sum_k U_k(theta_i) e^{i k lambda_q},
    so (1/n) sum_q u[i, q] e^{-i k lambda_q} = U_k(theta_i) for |k| < n/2.

    Returns (U, F, X) with shapes (n_theta, K), (m, K), (m, K)."""
    f = np.asarray(f, dtype=np.float64)
    nt, n = f.shape
    m = 2 * nt
    ks = [int(k) for k in ks]
    ft = dfs_double(f)
    s2 = np.sin(dfs_theta(m)) ** 2
    v = s2[:, None] * ft
    q = np.arange(n, dtype=np.int64)
    El = np.empty((n, len(ks)), dtype=np.complex128)
    for c, k in enumerate(ks):
        r = np.mod(k * (2 * q - n), 2 * n).astype(np.float64)
        El[:, c] = np.cos(math.pi * r / n) - 1j * np.sin(math.pi * r / n)
    G = v @ El / n                                     # lambda-DFT, (m, K)
    E = _theta_phase_cached(m)                         # E[j + m/2, p] = exp(-i j theta_p)
    F = (E @ G) / m
    X = np.zeros_like(F)
    for c, k in enumerate(ks):
        X[:, c] = _solve_one(F[:, c], m, k, reading)
    # U[i] = sum_j X_j exp(i j theta_{nt+i}) = conj(X^H E[:, nt + i])
    U = np.conj(X.conj().T @ E[:, nt:]).T
    return U, F, X


def _solve_one(Fk: np.ndarray, m: int, k: int, reading: str, banded: bool = False) -> np.ndarray:
    """X_k for one column (same systems as solve_columns)."""
    rhs = Fk.astype(np.complex128).copy()
    if k == 0:
        rhs[m // 2] = 0.0
    if reading == "B":
        rhs[0] = 0.0
    if m <= DENSE_MAX_M and not banded:
        return np.linalg.solve(system_matrix(m, k, reading), rhs)
    sub, d, sup = _bands_of(m, k, reading)
    if k != 0:
        return _banded_solve(sub, d, sup, rhs)
    keep = np.arange(m) != m // 2
    sub_r = sub[keep].copy()
    sup_r = sup[keep].copy()
    i0 = m // 2
    sub_r[i0] = 0.0
    sub_r[i0 + 1] = 0.0
    sup_r[i0 - 2] = 0.0
    sup_r[i0 - 1] = 0.0
    xr = _banded_solve(sub_r, d[keep], sup_r, rhs[keep])
    x = np.zeros(m, dtype=np.complex128)
    x[keep] = xr
    w = integration_weights(m)
    if reading == "B":
        w[0] = 0.0
    x[m // 2] = -(w[keep] @ xr) / w[m // 2]
    return x


def lambda_spectrum(u: np.ndarray, ks) -> np.ndarray:
    """(1/n) sum_q u[i, q] exp(-i k lambda_q) for each k in ks: (n_theta, K)."""
    u = np.asarray(u, dtype=np.float64)
    n = u.shape[1]
    q = np.arange(n, dtype=np.int64)
    El = np.empty((n, len(ks)), dtype=np.complex128)
    for c, k in enumerate(ks):
        r = np.mod(int(k) * (2 * q - n), 2 * n).astype(np.float64)
        El[:, c] = np.cos(math.pi * r / n) - 1j * np.sin(math.pi * r / n)
    return u @ El / n
