"""How much one PIE sweep of the oracle amplifies a perturbation of its input.

This fixes what element-wise parity can mean at the benchmarked workload (the
1024^2 object, 128^2 probe, 3600 Fermat positions, Poisson data at 1e4 peak
photons, random start of Section 4). Two perturbations of the same size are
compared with the unperturbed FP64 sweep (Eq. pie_update in colour-major
order):
  D   the start rounded once to complex64 (relative size u ~ 2.4e-8);
  D_U the object rounded to complex64 after every update, which is what FP32
      storage of the object does inside the sweep.
The full sweep amplifies the start perturbation by more than 10^4 (one
rounding moves the result by ~1.4e-3 relative), so no FP32 implementation can
match an FP64 sweep to 1e-5 there; and D_U is about D, so perturbations made
during the sweep propagate like one made at its start. The GPU parity test at
this workload bounds its error by a multiple of D derived from that.
"""
import numpy as np
import pytest

from oracle import coeffs, pie as opie
from paper_2408_03532_gb300 import synth


def _sweep(P, start, T, d, order, round_each):
    n = P["probe"].shape[0]
    z = np.array(start, dtype=np.complex128, copy=True)
    probe = P["probe"].astype(np.complex64).astype(np.complex128)
    pm2 = float(np.max(np.abs(probe) ** 2))
    for j in order:
        opie.pie_update(z, probe, P["pos"][j], d[j], T, 1.0, pm2)
        if round_each:
            r, c = P["pos"][j]
            z[r:r + n, c:c + n] = z[r:r + n, c:c + n].astype(np.complex64)
    return z


def _amplification(P, T, d):
    n = P["probe"].shape[0]
    order = opie.colour_major_order(opie.greedy_colouring(P["pos"], n, n))
    d = d.astype(np.float32).astype(np.float64)          # the data as the GPU holds them
    s64 = P["init"].astype(np.complex128)
    s32 = P["init"].astype(np.complex64).astype(np.complex128)
    a = _sweep(P, s32, T, d, order, False)
    b = _sweep(P, s64, T, d, order, False)
    c = _sweep(P, s32, T, d, order, True)
    u = np.linalg.norm(s32 - s64) / np.linalg.norm(s64)
    D = np.linalg.norm(a - b) / np.linalg.norm(a)
    DU = np.linalg.norm(c - a) / np.linalg.norm(a)
    return u, D, DU


def test_full_sweep_at_the_benchmark_size_is_ill_conditioned():
    P = synth.spiral_problem()
    u, D, DU = _amplification(P, opie.full_transform(128, 128), opie.amplitudes(P["intensities"]))
    assert 1e-8 < u < 5e-8
    assert D / u > 1e4            # measured 5.9e4 (D = 1.4e-3)
    assert 0.5 < DU / D < 2.0     # measured 1.03


def test_pft_sweep_amplifies_moderately():
    """The PFT sweep on a CPU-sized cut of the same recipe (512^2 object, 128^2
    probe, 400 Fermat positions, M = 32, Poisson 1e4): amplification 16 with
    D_U / D = 1.5 here, 90 and 0.85 at the full 3600 positions (D = 2.2e-6)."""
    P = synth.spiral_problem(side=512, n=128, count=400)
    T = opie.pft_transform(*coeffs.plan_2d(128, 128, 32, 32, 16, 16))
    u, D, DU = _amplification(P, T, opie.amplitudes(P["intensities"], 32))
    assert 5.0 < D / u < 1e3
    assert 0.3 < DU / D < 3.0
