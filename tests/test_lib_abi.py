"""CPU checks of the C-ABI library: it builds, loads, exports every declared
symbol, and its host-only offline phase (Section 3.1.1) meets its definition."""
import ctypes

import numpy as np
import pytest

from paper_2408_03532_gb300 import build as libbuild
from paper_2408_03532_gb300 import pft


@pytest.fixture(scope="module")
def lib():
    libbuild.build()
    return pft.load()


def test_exports_every_declared_symbol(lib):
    names = pft.declared_functions()
    assert len(names) >= 19
    for name in names:
        assert hasattr(lib, name), name
    assert lib.pft_version() >= 10000


def test_choose_r_matches_paper_and_ratios(lib):
    """r = 13 at eps = 1e-7 and m~/p = 1 (the paper's value); fewer terms for smaller ratios."""
    assert pft.choose_r(1e-7, 1.0) == 13
    assert pft.choose_r(1e-7, 0.5) == 10
    assert pft.choose_r(1e-7, 0.25) == 8


@pytest.mark.parametrize("eps,r", [(1e-7, 13), (1e-7, 10), (1e-4, 8), (1e-2, 3)])
def test_designed_polynomial_meets_eps_on_its_scope(lib, eps, r):
    """The polynomial sum_j i^j a_j x^j is within eps of e^{i pi x} on |x| <= xi,
    measured here independently on a fine grid in FP64."""
    xi, a, err = pft.design_coefficients(eps, r)
    x = np.linspace(-xi, xi, 200001)
    w = a * (1j ** np.arange(r))
    p = np.polynomial.polynomial.polyval(x, w)
    e = np.abs(p - np.exp(1j * np.pi * x)).max()
    assert e <= eps * (1 + 1e-6)
    assert err <= eps * (1 + 1e-9)
    # the scope is close to the best-approximation scope of the oracle
    from oracle import coeffs
    assert xi == pytest.approx(coeffs.scope(eps, r), rel=2e-3)


def test_constant_term_closed_form(lib):
    """r = 1: xi(eps, 1) = arcsin(eps) / pi (best constant for an arc)."""
    xi, a, _ = pft.design_coefficients(1e-3, 1)
    assert xi == pytest.approx(np.arcsin(1e-3) / np.pi, rel=1e-6)


def test_invalid_arguments_are_reported(lib):
    with pytest.raises(pft.PftError) as e:
        pft.choose_r(0.0, 1.0)
    assert e.value.code == -1
    xi = ctypes.c_double()
    assert lib.pft_design_coefficients(1e-7, 0, ctypes.byref(xi), None, None) == -1
    assert b"NULL" in lib.pft_last_error() or b"need" in lib.pft_last_error()


def test_binding_refuses_without_library(monkeypatch, tmp_path):
    """The product path fails loudly when the CUDA library is missing."""
    monkeypatch.setattr(pft, "_lib", None)
    monkeypatch.setattr(pft, "LIB_PATH", str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        pft.load()
