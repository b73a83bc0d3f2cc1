"""Pins for the oracle PFT (Algorithms 2 and 5) and its adjoint."""
import numpy as np
import pytest

from oracle import coeffs, dft, pft


def _rand(shape, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


@pytest.mark.parametrize("n,M,p", [(64, 32, 16), (32, 16, 8), (64, 16, 16)])
def test_1d_error_bound(n, M, p):
    """Each twiddle is approximated to eps for |t| <= m~ (Section 3.1.1), so
    |PFT(z)_t - DFT(z)_t| <= eps ||z||_1 for every kept t."""
    P = coeffs.plan_1d(n, M, p)
    z = _rand(n, 1)
    exact = dft.dft_matrix(n, P["t"]) @ z
    got = pft.pft1(z, P)
    assert np.abs(got - exact).max() <= P["eps"] * np.abs(z).sum() * (1 + 1e-6)


@pytest.mark.parametrize("n1,n2,M1,M2,p1,p2", [(64, 64, 32, 32, 16, 16), (32, 64, 16, 32, 8, 16),
                                                (128, 128, 32, 32, 16, 16)])
def test_2d_error_bound(n1, n2, M1, M2, p1, p2):
    """Two approximated factors: |P1 P2 - E1 E2| <= (2 eps + eps^2) per term, so
    |PFT2(z) - DFT2(z)| <= (2 eps + eps^2) ||z||_1; typical rel-L2 error ~ eps."""
    P1, P2 = coeffs.plan_2d(n1, n2, M1, M2, p1, p2)
    z = _rand((n1, n2), 2)
    exact = dft.partial_dft2(z, M1, M2)
    got = pft.pft2(z, P1, P2)
    eps = P1["eps"]
    assert np.abs(got - exact).max() <= (2 * eps + eps * eps) * np.abs(z).sum() * (1 + 1e-6)
    assert np.linalg.norm(got - exact) <= 10 * eps * np.linalg.norm(exact)


def test_p_equals_n_reduces_to_fft():
    """q = 1: B = w, so C^[u, j] = w_j z^_u and PFT(z)_t = z^_{t mod n} e^{-i pi t/n} P(t/n)."""
    n, M = 16, 8
    P = coeffs.plan_1d(n, M, n, r=6)
    z = _rand(n, 3)
    t = P["t"]
    poly = np.polynomial.polynomial.polyval(t / n, P["w"])
    expect = np.fft.fft(z)[np.mod(t, n)] * np.exp(-1j * np.pi * t / n) * poly
    assert np.allclose(pft.pft1(z, P), expect, atol=1e-12 * np.abs(z).sum())


def test_2d_is_separable_in_1d_algorithm():
    """Algorithm 5 on an outer product u v^T equals Algorithm 2 on u times Algorithm 2 on v."""
    P1, P2 = coeffs.plan_2d(32, 64, 16, 32, 8, 16)
    u, v = _rand(32, 4), _rand(64, 5)
    got = pft.pft2(np.outer(u, v), P1, P2)
    assert np.allclose(got, np.outer(pft.pft1(u, P1), pft.pft1(v, P2)), atol=1e-10)


@pytest.mark.parametrize("n1,n2,M1,M2,p1,p2", [(64, 64, 32, 32, 16, 16), (32, 64, 16, 32, 8, 16)])
def test_adjoint_identity(n1, n2, M1, M2, p1, p2):
    """<A x, y> = <x, A^H y> for the approximate operator itself."""
    P1, P2 = coeffs.plan_2d(n1, n2, M1, M2, p1, p2)
    x = _rand((3, n1, n2), 6)
    y = _rand((3, M1, M2), 7)
    lhs = np.vdot(y, pft.pft2(x, P1, P2))
    rhs = np.vdot(pft.pft2_adjoint(y, P1, P2), x)
    assert abs(lhs - rhs) <= 1e-12 * np.linalg.norm(x) * np.linalg.norm(y) * n1 * n2


def test_adjoint_close_to_exact_adjoint():
    """The PFT adjoint approximates the exact partial-DFT adjoint to the same eps."""
    P1, P2 = coeffs.plan_2d(64, 64, 32, 32, 16, 16)
    y = _rand((32, 32), 8)
    got = pft.pft2_adjoint(y, P1, P2)
    exact = dft.partial_dft2_adjoint(y, 64, 64)
    assert np.abs(got - exact).max() <= (2e-7 + 1e-14) * np.abs(y).sum() * (1 + 1e-6)
