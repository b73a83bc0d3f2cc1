"""Pins for the oracle's total-variation term."""
import numpy as np
import pytest

from oracle import grad, tv


def _rand(shape, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_difference_adjoints():
    x, u = _rand((7, 9), 1), _rand((7, 9), 2)
    u[:, -1] = 0
    assert np.vdot(u, tv.dx(x)) == pytest.approx(np.vdot(tv.dx_adjoint(u), x), rel=1e-12)
    v = _rand((7, 9), 3)
    v[-1, :] = 0
    assert np.vdot(v, tv.dy(x)) == pytest.approx(np.vdot(tv.dy_adjoint(v), x), rel=1e-12)


def test_gradient_matches_central_differences():
    z = _rand((10, 12), 4)
    g = tv.tv_grad(z, 0.3)
    rng = np.random.default_rng(5)
    for _ in range(20):
        idx = (int(rng.integers(10)), int(rng.integers(12)))
        fd = grad.finite_difference(lambda w: tv.tv(w, 0.3), z, idx, 1e-6)
        assert abs(fd - g[idx]) < 1e-6


def test_constant_and_ramp():
    """A constant has zero TV gradient and TV = H W eps; a unit ramp along x has
    |D_x z| = 1 away from the last column."""
    c = np.full((6, 8), 0.3 - 0.7j)
    assert np.allclose(tv.tv_grad(c, 0.1), 0)
    assert tv.tv(c, 0.1) == pytest.approx(6 * 8 * 0.1)
    ramp = np.tile(np.arange(8, dtype=float), (6, 1)) + 0j
    assert tv.tv(ramp, 0.0) == pytest.approx(6 * 7)
    # a step lowers TV along the negative gradient
    z = _rand((8, 8), 6)
    assert tv.tv(tv.tv_step(z, 1e-3, 0.1), 0.1) < tv.tv(z, 0.1)
