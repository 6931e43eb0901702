"""A fast CPU solver of the paper's spherical Poisson method, for timing only.

Section 5's algorithm as a plain CPU program: the 2D Fourier coefficients of
sin^2(theta) f~ by FFTs (a real FFT along each colatitude row, then the BMC
fold's cosine / sine transform along each longitude wavenumber column), the
per-k systems of eq. linearSystems solved by Thomas elimination on their two
parity chains (the bands have offsets 0 and +-2 only), the j = 0 row closed in
closed form (the k = 0 column by the constraint w^T X_0 = 0 of eq.
pentdiagonalPlusRankOne), then the inverse transforms.  scipy.fft does the
transforms (its `workers` threads give the multi-core timing); the eliminations
are numpy vector operations over all wavenumbers at once, one row at a time, on
one thread (threads over slices of wavenumbers were slower: the row sweeps are
short numpy calls that hold the interpreter lock).

This is the CPU baseline a user would write, not the project's product (the
CUDA library) and not its oracle (which forms F by a naive DFT and solves by
LU): neither imports it.  The tests pin it against the oracle on small grids.
Grid and truncation as the library's: theta_i = (i + 1/2) pi / n_theta,
lambda_q = -pi + 2 pi q / n_lambda, |j| <= n_theta - 1 (theta-Nyquist mode
dropped), wavenumbers k = 0 .. n_lambda/2 (the rest by Hermitian symmetry).
"""

from __future__ import annotations

import numpy as np
import scipy.fft as sfft


def _bands(N: int):
    """a_j, b_j, c_j of row j = 0..N-1 (column j-2, diagonal without -k^2, column j+2)."""
    j = np.arange(N, dtype=np.float64)
    return (j - 1.0) * (j - 2.0) / 4.0, -(j * j) / 2.0, (j + 1.0) * (j + 2.0) / 4.0


def _thomas_chain(rows, F, k2, a, b, c):
    """Solve the tridiagonal chain over the given rows (every second row j, all
    wavenumbers at once): a_j X_{j-2} + (b_j - k^2) X_j + c_j X_{j+2} = F_j with
    X = 0 outside the chain.  F: [N, K] complex; returns X on those rows."""
    nr = len(rows)
    K = F.shape[1]
    cp = np.empty((nr, K))
    dp = np.empty((nr, K), dtype=np.complex128)
    prev_c = None
    for t, j in enumerate(rows):
        diag = b[j] - k2
        lo = a[j] if t > 0 else 0.0
        if t > 0:
            denom = diag - lo * prev_c
            dp[t] = (F[j] - lo * dp[t - 1]) / denom
        else:
            denom = diag
            dp[t] = F[j] / denom
        cp[t] = (c[j] if t + 1 < nr else 0.0) / denom
        prev_c = cp[t]
    X = np.empty((nr, K), dtype=np.complex128)
    X[-1] = dp[-1]
    for t in range(nr - 2, -1, -1):
        X[t] = dp[t] - cp[t] * X[t + 1]
    return X


def solve(f: np.ndarray, workers: int = 1) -> np.ndarray:
    """u with Delta u = f and zero sphere mean on the n_theta x n_lambda grid."""
    f = np.asarray(f, dtype=np.float64)
    N, n = f.shape
    L = n // 2
    K = L + 1
    theta = (np.arange(N) + 0.5) * np.pi / N
    sgn_k = (-1.0) ** np.arange(K)                        # e^{-ik lambda_q} = (-1)^k e^{-2 pi i k q/n}
    even = (np.arange(K) % 2) == 0
    # S1-S2: sin^2 weight and the real FFT of each row, 1/n normalised
    G = sfft.rfft(f * (np.sin(theta) ** 2)[:, None], axis=1, workers=workers) * (sgn_k / n)[None, :]
    # S3: the length-2N colatitude DFT of the BMC-doubled column, folded:
    #   F_j = (1/N) sum_i G_i cos(j theta_i) (k even),  -(i/N) sum_i G_i sin(j theta_i) (k odd)
    F = np.zeros((N, K), dtype=np.complex128)
    if even.any():
        F[:, even] = sfft.dct(G[:, even], type=2, axis=0, workers=workers) / (2 * N)
    if (~even).any() and N > 1:
        F[1:, ~even] = -1j * sfft.dst(G[:, ~even], type=2, axis=0, workers=workers)[: N - 1] / (2 * N)
    # S4: the two parity chains of rows j >= 1, then row 0
    a, b, c = _bands(N)
    k2 = (np.arange(K, dtype=np.float64) ** 2)[None, :]
    X = np.zeros_like(F)
    for start in (1, 2):
        rows = np.arange(start, N, 2)
        if len(rows):
            X[rows] = _thomas_chain(rows, F, k2, a, b, c)
    ks = np.arange(1, K)
    x2 = X[2, 1:] if N > 2 else np.zeros(K - 1, dtype=np.complex128)
    X[0, 1:] = (0.5 * (1.0 + (-1.0) ** ks) * x2 - F[0, 1:]) / ks.astype(np.float64) ** 2
    je = np.arange(2, N, 2, dtype=np.float64)
    X[0, 0] = np.sum(2.0 * X[2::2, 0] / (je * je - 1.0))
    # S5: inverse colatitude transforms, u_i = X_0 + 2 sum_j X_j cos(j theta_i) or 2i sum_j X_j sin(j theta_i)
    U = np.empty((N, K), dtype=np.complex128)
    if even.any():
        U[:, even] = sfft.dct(X[:, even], type=3, axis=0, workers=workers)
    if (~even).any():
        Y = np.zeros((N, int((~even).sum())), dtype=np.complex128)
        Y[: N - 1] = X[1:, ~even]
        U[:, ~even] = 1j * sfft.dst(Y, type=3, axis=0, workers=workers)
    # S6: inverse real FFT of each row (the Nyquist column k = L enters once)
    U *= sgn_k[None, :]
    return sfft.irfft(U * n, n=n, axis=1, workers=workers)
