"""Exact DFTs in FP64: the quantities the PFT approximates.

Section 3.1.1 defines the unnormalised DFT z^_t = sum_k z_k e^{-2 pi i t k / n};
Appendix A gives the 2-D form z^[t1, t2] = sum_{k1, k2} z[k1, k2]
e^{-2 pi i t1 k1 / n1} e^{-2 pi i t2 k2 / n2}. The partial transform keeps the
lowest M1 x M2 frequencies, t_nu in [-M_nu/2, M_nu/2 - 1], returned centred
(row t1 + M1/2, column t2 + M2/2).

Three independent routes are given: the separable matrix form with integer
phase reduction (t k mod n, so every twiddle is exact to FP64 rounding), a
brute-force quadruple sum for tiny inputs, and numpy's FFT followed by a crop.
"""
from __future__ import annotations

import numpy as np

from .coeffs import freqs


def dft_matrix(n: int, t: np.ndarray) -> np.ndarray:
    """F[t, k] = exp(-2 pi i ((t k) mod n) / n) for the given rows t."""
    k = np.arange(n)
    ph = np.mod(np.outer(np.asarray(t, dtype=np.int64), k), n)
    return np.exp(-2j * np.pi * ph / n)


def partial_dft2(z: np.ndarray, M1: int, M2: int) -> np.ndarray:
    """Lowest M1 x M2 coefficients of the 2-D DFT of z[..., n1, n2] (centred)."""
    n1, n2 = z.shape[-2:]
    F1 = dft_matrix(n1, freqs(M1))
    F2 = dft_matrix(n2, freqs(M2))
    return F1 @ z @ F2.T


def partial_dft2_adjoint(y: np.ndarray, n1: int, n2: int) -> np.ndarray:
    """Conjugate transpose of partial_dft2: x = F1^H y conj(F2)."""
    M1, M2 = y.shape[-2:]
    F1 = dft_matrix(n1, freqs(M1))
    F2 = dft_matrix(n2, freqs(M2))
    return F1.conj().T @ y @ F2.conj()


def brute_partial_dft2(z: np.ndarray, M1: int, M2: int) -> np.ndarray:
    """The Appendix-A double sum written out with Python loops (tiny inputs)."""
    n1, n2 = z.shape
    out = np.zeros((M1, M2), dtype=np.complex128)
    for a, t1 in enumerate(freqs(M1)):
        for b, t2 in enumerate(freqs(M2)):
            acc = 0j
            for k1 in range(n1):
                for k2 in range(n2):
                    acc += z[k1, k2] * np.exp(-2j * np.pi * (t1 * k1 / n1 + t2 * k2 / n2))
            out[a, b] = acc
    return out


def fft_then_crop(z: np.ndarray, M1: int, M2: int) -> np.ndarray:
    """Full 2-D FFT (numpy) then the centred M1 x M2 crop of frequencies."""
    n1, n2 = z.shape[-2:]
    Z = np.fft.fft2(z, axes=(-2, -1))
    i1 = np.mod(freqs(M1), n1)
    i2 = np.mod(freqs(M2), n2)
    return Z[..., i1, :][..., :, i2]


def crop_centre(d: np.ndarray, M1: int, M2: int) -> np.ndarray:
    """d^crop: the centred M1 x M2 block of FFT-ordered data d[..., n1, n2].

    Algorithm 3 crops the centres of the (shifted) data; with data in
    FFT order this is d^crop[t1 + M1/2, t2 + M2/2] = d[t1 mod n1, t2 mod n2].
    """
    n1, n2 = d.shape[-2:]
    i1 = np.mod(freqs(M1), n1)
    i2 = np.mod(freqs(M2), n2)
    return d[..., i1, :][..., :, i2]


def full_dft2(z: np.ndarray) -> np.ndarray:
    """Unnormalised full 2-D DFT (the F of Eq. 1), numpy FFT."""
    return np.fft.fft2(z, axes=(-2, -1))


def full_idft2(y: np.ndarray) -> np.ndarray:
    """F^{-1} = F^H / (n1 n2), numpy inverse FFT."""
    return np.fft.ifft2(y, axes=(-2, -1))
