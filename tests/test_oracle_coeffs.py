"""Pins for the oracle's offline phase (Section 3.1.1, Algorithms 1 and 4)."""
import json
import math
import os

import numpy as np
import pytest
from scipy.special import jv

from oracle import coeffs

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "paper_parameters.json")


def test_r_matches_paper_value():
    """The paper prints r = 13 for eps = 1e-7 and m~/p = 1 (golden fixture)."""
    g = json.load(open(GOLDEN))["polynomial_terms"]
    assert coeffs.choose_r(g["eps"], g["m_tilde_over_p"]) == g["r"]


@pytest.mark.parametrize("eps", [1e-1, 1e-3, 1e-6])
def test_constant_polynomial_closed_form(eps):
    """r = 1: the best constant for the arc {e^{i pi x}: |x| <= xi <= 1/2} is the
    centre of its chord, cos(pi xi), with error sin(pi xi); hence
    xi(eps, 1) = arcsin(eps) / pi."""
    xi = coeffs.scope(eps, 1)
    assert xi == pytest.approx(math.asin(eps) / math.pi, rel=2e-5)
    w, err = coeffs.best_approximation(0.3, 1)
    # the error is flat (second order) in the constant near its optimum, so the
    # error is pinned tightly and the constant only loosely
    assert err == pytest.approx(math.sin(0.3 * math.pi), rel=1e-5)
    assert w[0].real == pytest.approx(math.cos(0.3 * math.pi), abs=1e-2)


@pytest.mark.parametrize("r,ratio", [(8, 0.25), (10, 0.5), (13, 1.0)])
def test_best_error_between_bessel_bounds(r, ratio):
    """Jacobi-Anger: e^{i pi xi s} = J0 + 2 sum_k i^k J_k(pi xi) T_k(s). Truncating
    after degree r-1 is one admissible polynomial, so the best error is no larger
    than the truncation's; and every degree-(r-1) polynomial leaves the T_r
    Chebyshev coefficient 2 i^r J_r untouched, which bounds its error below by
    |J_r(pi xi)| (Chebyshev coefficients are at most twice the sup norm)."""
    w, err = coeffs.best_approximation(ratio, r)
    s = np.linspace(-1, 1, 20001)
    z = math.pi * ratio
    trunc = jv(0, z) + 2 * sum((1j ** k) * jv(k, z) * np.cos(k * np.arccos(s)) for k in range(1, r))
    trunc_err = np.abs(trunc - np.exp(1j * z * s)).max()
    assert err <= trunc_err * (1 + 1e-6)
    assert err >= abs(jv(r, z)) * (1 - 1e-6)


def test_scope_is_the_supremum():
    """xi(eps, r) meets eps, and a slightly larger scope does not (definition)."""
    eps, r = 1e-7, 13
    xi, w = coeffs.coefficients(eps, r)
    assert coeffs.uniform_error(w, xi) <= eps * (1 + 1e-6)
    _, err_above = coeffs.best_approximation(xi * (1 + 1e-4), r)
    assert err_above > eps
    assert 1.0 <= xi < 1.01


def test_symmetry_and_monotonicity():
    """w_j = i^j a_j with a_j real (uniqueness + conjugate symmetry), and the
    scope grows with r (more terms never shrink it)."""
    xi, w = coeffs.coefficients(1e-7, 13)
    a = w / (1j ** np.arange(13))
    assert np.abs(a.imag).max() <= 1e-12 * np.abs(a).max()
    # Taylor-like leading terms: a_0 ~ 1, a_1 ~ pi
    assert a[0] == pytest.approx(1.0, abs=1e-6)
    assert a[1] == pytest.approx(math.pi, rel=1e-5)
    s = [coeffs.best_approximation(0.5, r)[1] for r in (6, 8, 10, 12)]
    assert all(x > y for x, y in zip(s, s[1:]))


def test_algorithm1_tables():
    """Algorithm 1: B[l, j] = w_j (1 - 2l/q)^j, W[t, j] = (t/p)^j e^{-i pi t/p};
    their product summed over j approximates each twiddle e^{-2 pi i t (l - q/2)/n}
    to eps for every kept t (Section 3.1.1, |t| <= m~)."""
    n, M, p = 64, 32, 16
    P = coeffs.plan_1d(n, M, p)
    assert (P["q"], P["r"]) == (4, 13)
    assert P["B"].shape == (4, 13) and P["W"].shape == (32, 13)
    t = P["t"][:, None]
    l = np.arange(P["q"])[None, :]
    approx = (P["W"] * np.exp(1j * np.pi * t / p)) @ P["B"].T  # sum_j (t/p)^j w_j x_l^j
    exact = np.exp(-2j * np.pi * t * (l - P["q"] / 2) / n)
    assert np.abs(approx - exact).max() <= 1e-7 * (1 + 1e-6)
