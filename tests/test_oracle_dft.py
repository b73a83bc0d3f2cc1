"""Pins for the exact partial DFT (Section 3.1.1 DFT, Appendix A 2-D DFT)."""
import numpy as np
import pytest

from oracle import dft
from oracle.coeffs import freqs


def _rand(shape, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n1,n2,M1,M2", [(4, 4, 2, 4), (8, 4, 4, 2), (6, 10, 6, 10), (8, 8, 8, 4)])
def test_brute_force_matches_matrix_and_fft_routes(n1, n2, M1, M2):
    z = _rand((n1, n2))
    b = dft.brute_partial_dft2(z, M1, M2)
    assert np.allclose(dft.partial_dft2(z, M1, M2), b, atol=1e-12 * np.abs(z).sum())
    assert np.allclose(dft.fft_then_crop(z, M1, M2), b, atol=1e-12 * np.abs(z).sum())


def test_plane_wave_and_constant():
    """A plane wave e^{2 pi i (a k1/n1 + b k2/n2)} has a single coefficient n1 n2
    at (a, b); a constant has only the DC term sum z."""
    n1, n2, M = 16, 8, 8
    k1, k2 = np.meshgrid(np.arange(n1), np.arange(n2), indexing="ij")
    a, b = -3, 2
    z = np.exp(2j * np.pi * (a * k1 / n1 + b * k2 / n2))
    y = dft.partial_dft2(z, M, M)
    expect = np.zeros((M, M), complex)
    expect[a + M // 2, b + M // 2] = n1 * n2
    assert np.allclose(y, expect, atol=1e-10)
    c = np.full((n1, n2), 0.7 - 0.2j)
    yc = dft.partial_dft2(c, M, M)
    expect = np.zeros((M, M), complex)
    expect[M // 2, M // 2] = c.sum()
    assert np.allclose(yc, expect, atol=1e-10)


def test_shift_gives_phase_ramp():
    """Circular shift by (s1, s2) multiplies coefficient t by e^{-2 pi i (t1 s1/n1 + t2 s2/n2)}."""
    n, M, s1, s2 = 16, 8, 3, -5
    z = _rand((n, n), 1)
    y0 = dft.partial_dft2(z, M, M)
    y1 = dft.partial_dft2(np.roll(z, (s1, s2), axis=(0, 1)), M, M)
    t = freqs(M)
    ramp = np.exp(-2j * np.pi * (t[:, None] * s1 + t[None, :] * s2) / n)
    assert np.allclose(y1, y0 * ramp, atol=1e-10)


def test_parseval_bessel_and_projector():
    """sum over all frequencies |z^|^2 = n1 n2 ||z||^2; a subset gives <=; and
    A^H A / (n1 n2) is an orthogonal projector for the exact partial DFT."""
    n, M = 16, 8
    z = _rand((n, n), 2)
    full = dft.partial_dft2(z, n, n)
    assert np.sum(np.abs(full) ** 2) == pytest.approx(n * n * np.sum(np.abs(z) ** 2), rel=1e-13)
    part = dft.partial_dft2(z, M, M)
    assert np.sum(np.abs(part) ** 2) <= n * n * np.sum(np.abs(z) ** 2)
    P1 = dft.partial_dft2_adjoint(part, n, n) / (n * n)
    P2 = dft.partial_dft2_adjoint(dft.partial_dft2(P1, M, M), n, n) / (n * n)
    assert np.allclose(P1, P2, atol=1e-12)


def test_adjoint_identity():
    n1, n2, M1, M2 = 16, 32, 8, 16
    x = _rand((n1, n2), 3)
    y = _rand((M1, M2), 4)
    lhs = np.vdot(y, dft.partial_dft2(x, M1, M2))
    rhs = np.vdot(dft.partial_dft2_adjoint(y, n1, n2), x)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y) * n1 * n2


def test_crop_centre_matches_shifted_crop():
    """d^crop in centred order equals the centre block of the fftshifted data."""
    n, M = 16, 6
    d = np.random.default_rng(5).random((n, n))
    sh = np.fft.fftshift(d)
    c = n // 2
    assert np.array_equal(dft.crop_centre(d, M, M), sh[c - M // 2:c + M // 2, c - M // 2:c + M // 2])
