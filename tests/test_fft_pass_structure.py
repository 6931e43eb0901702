"""The pass structure of the library's shared-memory FFT, on a numpy model, no GPU.

The kernels transform in place by decimation in time: input q is loaded to
the digit-reversed position perm[q] (the host's digit reversal for the radix
sequence R_1 .. R_s), then pass t (sub-DFT length Ns = R_1 .. R_{t-1})
multiplies element r of butterfly (g, k) by w^(r k), w = exp(-+2 pi i/(Ns R_t)),
and applies the R_t-point DFT.  The fused FP32 colatitude stage runs its
inverse by decimation in frequency: the same passes transposed (DFT first,
the same twiddles after) in reverse order on natural-order input, which leaves
output q at position perm[q].  This model follows those index rules exactly
and checks both against numpy's FFT for the radix sequences the grids use."""

import numpy as np
import pytest


def _digit_reversal(radix):
    L = int(np.prod(radix))
    perm = np.zeros(L, dtype=int)
    for q0 in range(L):
        q, p, w = q0, 0, L
        for s in range(len(radix) - 1, -1, -1):
            w //= radix[s]
            p += (q % radix[s]) * w
            q //= radix[s]
        perm[q0] = p
    return perm


def _passes(radix):
    ns, out = 1, []
    for R in radix:
        out.append((R, ns))
        ns *= R
    return out


def _butterflies(L, R, ns):
    for g in range(L // (R * ns)):
        for k in range(ns):
            yield k, [g * ns * R + k + r * ns for r in range(R)]


def _dft(v, sign):
    a = np.arange(len(v))
    return np.exp(sign * 2j * np.pi * np.outer(a, a) / len(v)) @ v


def _dit(z, radix, sign):
    z = z.copy()
    for R, ns in _passes(radix):
        for k, idx in _butterflies(len(z), R, ns):
            z[idx] = _dft(z[idx] * np.exp(sign * 2j * np.pi * np.arange(R) * k / (ns * R)), sign)
    return z


def _dif(z, radix, sign):
    z = z.copy()
    for R, ns in reversed(_passes(radix)):
        for k, idx in _butterflies(len(z), R, ns):
            z[idx] = _dft(z[idx], sign) * np.exp(sign * 2j * np.pi * np.arange(R) * k / (ns * R))
    return z


@pytest.mark.parametrize("radix", [[5, 5, 5, 5, 8], [7, 8, 8], [5, 2, 3], [3, 4, 2], [8], [2, 2, 2], [11, 3],
                                   [13], [2]])
@pytest.mark.parametrize("sign", [-1, 1])
def test_dit_and_dif_give_the_transform(radix, sign):
    L = int(np.prod(radix))
    rng = np.random.default_rng(L)
    x = rng.standard_normal(L) + 1j * rng.standard_normal(L)
    ref = np.fft.fft(x) if sign < 0 else np.fft.ifft(x) * L
    perm = _digit_reversal(radix)
    z = np.zeros(L, dtype=complex)
    z[perm] = x                                   # the DIT load
    tol = 1e-14 * L * np.abs(ref).max()
    assert np.abs(_dit(z, radix, sign) - ref).max() < tol
    assert np.abs(_dif(x, radix, sign)[perm] - ref).max() < tol
