"""Pins for the oracle amplitude-loss gradient: FP64 central finite differences."""
import numpy as np
import pytest

from oracle import coeffs, grad, pie
from paper_2408_03532_gb300 import synth

EPS64 = np.finfo(np.float64).eps


def _fd_tol(g, gmax, loss, h):
    """Truncation O(h^2) is negligible at h = 1e-6; the rounding of the two loss
    values, about eps * L each, divided by 2h, is not: allow 4 eps L / h."""
    return 1e-6 * max(abs(g), 1e-3 * gmax) + 4.0 * EPS64 * loss / h


@pytest.fixture(scope="module")
def problem():
    G = synth.gradient_problem()
    P1, P2 = coeffs.plan_2d(64, 64, 32, 32, 16, 16)
    T = pie.pft_transform(P1, P2)
    d = pie.amplitudes(G["intensities"], 32)
    return G, T, d


def test_object_gradient_matches_central_differences(problem):
    """40 object entries of the 512^2 / 64^2 / 400-position problem at the seeded
    initial guess, h = 1e-6. The loss is a sum over positions and a pixel only
    enters the positions whose patch covers it, so each difference is taken on
    that partial sum (the other terms cancel exactly)."""
    G, T, d = problem
    z, probe, pos = G["init"], G["probe"], G["pos"]
    _, gz, _ = grad.amplitude_loss_grad(z, probe, pos, d, T)
    rng = np.random.default_rng(11)
    il = pie.illumination(probe, pos, z.shape)
    cand = np.argwhere(il > 1e-2 * il.max())
    for k in rng.choice(len(cand), 40, replace=False):
        r, c = cand[k]
        cover = [j for j, (a, b) in enumerate(pos) if a <= r < a + 64 and b <= c < b + 64]
        fun = lambda zz: grad.amplitude_loss(zz, probe, pos[cover], d[cover], T)
        fd = grad.finite_difference(fun, z, (r, c), 1e-6)
        assert abs(fd - gz[r, c]) <= _fd_tol(gz[r, c], np.abs(gz).max(), fun(z), 1e-6)


def test_probe_gradient_matches_central_differences(problem):
    """10 probe entries; the probe enters every position, so the check runs on the
    first 40 positions of the scan (the formula does not depend on N)."""
    G, T, d = problem
    z, probe, pos = G["init"], G["probe"], G["pos"][:40]
    dd = d[:40]
    L, _, gw = grad.amplitude_loss_grad(z, probe, pos, dd, T)
    rng = np.random.default_rng(12)
    for k in rng.choice(64 * 64, 10, replace=False):
        idx = (k // 64, k % 64)
        fun = lambda w: grad.amplitude_loss(z, w, pos, dd, T)
        fd = grad.finite_difference(fun, probe, idx, 1e-6)
        assert abs(fd - gw[idx]) <= _fd_tol(gw[idx], np.abs(gw).max(), L, 1e-6)


def test_gradient_vanishes_at_noise_free_truth_for_exact_operator():
    """With the exact partial DFT and data from the truth, L = 0 and the gradient is 0."""
    obj = synth.make_object(64)
    probe = synth.make_probe(32)
    pos = synth.raster_scan(3, 3, 16, 0)
    T = pie.partial_dft_transform(32, 32, 16, 16)
    d = np.abs(T["fwd"](probe[None] * np.stack([obj[r:r + 32, c:c + 32] for r, c in pos])))
    L, gz, gw = grad.amplitude_loss_grad(obj, probe, pos, d, T)
    assert L < 1e-20 and np.abs(gz).max() < 1e-9 and np.abs(gw).max() < 1e-9
