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


def test_null_and_invalid_arguments_are_refused_before_any_gpu_work(lib):
    """Every entry point checks its arguments first: NULL handles, NULL outputs
    and impossible values return PFT_ERR_INVALID_ARG (-1) with a message, on a
    machine without a GPU as on one with."""
    null = None
    out = ctypes.c_void_p()
    calls = [
        lambda: lib.pft_plan_create(null, 64, 64, 32, 32, 0, 0, 1e-7, 0, 0, 0, 0),
        lambda: lib.pft_plan_create(ctypes.byref(out), 64, 64, 32, 32, 0, 0, 2.0, 0, 0, 0, 0),  # eps >= 1
        lambda: lib.pft_plan_info_get(null, null),
        lambda: lib.pft_forward(null, null, null, 1, null),
        lambda: lib.pft_adjoint(null, null, null, 1, null),
        lambda: lib.pft_fft2(null, null, 64, 1, 0, null),
        lambda: lib.pft_fft_crop(null, null, 64, 32, -1, null),
        lambda: lib.pie_ctx_info_get(null, null),
        lambda: lib.pie_ctx_colours(null, null, null),
        lambda: lib.pie_iteration(null, null, 0, 1.0, null, null),
        lambda: lib.pie_ctx_set_persistent(null, 0, 1),
        lambda: lib.pie_ctx_set_cluster(null, 0, 4),
        lambda: lib.pie_ctx_set_order(null, null, 0),
        lambda: lib.pie_iteration_blind(null, null, 0, 1.0, 1.0, 0, null, null),
        lambda: lib.pie_iteration_blind(null, null, 0, 1.0, 1.0, 7, null, null),     # unknown probe step
        lambda: lib.pie_iteration_blind(null, null, 0, 1.0, -1.0, 1, null, null),    # gamma < 0
        lambda: lib.pie_nrmse(null, null, null, null, null),
        lambda: lib.pie_amp_loss_grad(null, null, null, null, null, null, null),
        lambda: lib.pie_batch_create(ctypes.byref(out), 0, null, null, null, null, null),
        lambda: lib.pie_batch_iteration(null, null, 0, 1.0, null, null),
        lambda: lib.pie_batch_classes(null, null, null),
        lambda: lib.pie_batch_set_launch(null, 0),
        lambda: lib.pie_lf_create(ctypes.byref(out), null, null, null, null, null),
        lambda: lib.pie_lf_iteration(null, null, 1.0, null, null),
        lambda: lib.pie_lf_colours(null, null, null),
    ]
    for i, call in enumerate(calls):
        assert call() == -1, i
        assert lib.pft_last_error(), i


def test_scan_schedule_argument_checks(lib):
    pos = np.zeros((2, 2), np.int32)
    ncol, ndep = ctypes.c_int(), ctypes.c_int64()
    dep = np.zeros(0, np.int32)
    ok = lib.pie_scan_schedule(pos.ctypes.data, 2, 16, 32, 32, None, 0, ctypes.byref(ncol), None, None, None, None, 0,
                               ctypes.byref(ndep))
    assert ok == 0 and ncol.value == 2 and ndep.value == 1
    # a dep buffer too small for the lists is refused, with the count still reported
    assert lib.pie_scan_schedule(pos.ctypes.data, 2, 16, 32, 32, None, 0, ctypes.byref(ncol), None, None, None,
                                 dep.ctypes.data, 0, ctypes.byref(ndep)) == -1
    assert ndep.value == 1 and b"needed" in lib.pft_last_error()
    assert lib.pie_scan_schedule(None, 2, 16, 32, 32, None, 0, ctypes.byref(ncol), None, None, None, None, 0,
                                 ctypes.byref(ndep)) == -1
    assert lib.pie_scan_schedule(pos.ctypes.data, 2, 40, 32, 32, None, 0, ctypes.byref(ncol), None, None, None, None,
                                 0, ctypes.byref(ndep)) == -1                 # patch larger than the object
