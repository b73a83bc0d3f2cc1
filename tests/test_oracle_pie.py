"""Pins for the oracle PIE (Section 2.1), colouring, batched mode and Algorithm 3."""
import numpy as np
import pytest

from oracle import coeffs, dft, pie
from paper_2408_03532_gb300 import synth


def _rand(shape, seed=0):
    rng = np.random.default_rng(seed)
    return rng.standard_normal(shape) + 1j * rng.standard_normal(shape)


def test_full_update_is_the_modulus_projection():
    """With w = 1 and beta = 1, one FULL update replaces the patch by P_M(z)
    (Eq. 3): its spectrum is d with the phase of the old patch's spectrum
    (the modulus alone would also be d for -P_M(z))."""
    n = 16
    obj = _rand((24, 24), 1)
    probe = np.ones((n, n), complex)
    d = np.random.default_rng(2).random((n, n)) + 0.1
    z = obj.copy()
    pie.pie_update(z, probe, (3, 5), d, pie.full_transform(n, n), 1.0, 1.0)
    assert np.allclose(np.abs(np.fft.fft2(z[3:3 + n, 5:5 + n])), d, rtol=1e-12, atol=1e-12)
    old = np.fft.fft2(obj[3:3 + n, 5:5 + n])
    assert np.allclose(np.fft.fft2(z[3:3 + n, 5:5 + n]), d * old / np.abs(old), rtol=1e-12, atol=1e-12)
    # pixels outside the patch are untouched
    mask = np.ones_like(obj, bool)
    mask[3:3 + n, 5:5 + n] = False
    assert np.array_equal(z[mask], obj[mask])


def test_truth_is_a_fixed_point_and_phase_invariance():
    """Noise-free data: Phi = 0 at the truth and the sweep leaves it in place, for
    any global phase; the PFT sweep moves it only by the approximation error."""
    P = synth.small_raster_problem()
    obj, probe, pos = P["obj"], P["probe"], P["pos"]
    d = pie.amplitudes(P["intensities"])
    for ph in (1.0, np.exp(0.7j)):
        z, phi = pie.pie_sweep(obj * ph, probe, pos, d, pie.full_transform(32, 32), 1.0)
        assert phi < 1e-24 * np.sum(d ** 2) / len(pos)
        assert pie.relative_change(z, obj * ph) < 1e-13
        assert pie.nrmse(z, obj) < 1e-13
    P1, P2 = coeffs.plan_2d(32, 32, 16, 16, 8, 8)
    dc = pie.amplitudes(P["intensities"], 16)
    z, phi = pie.pie_sweep(obj, probe, pos, dc, pie.pft_transform(P1, P2), 1.0)
    assert pie.relative_change(z, obj) < 1e-6


def test_partial_dft_update_is_low_band_projection():
    """For the exact partial DFT, A^H A / (n1 n2) is the projector onto the kept
    band, so the update changes only those frequencies of the patch and sets
    their moduli to d^crop (w = 1, beta = 1)."""
    n, M = 16, 8
    obj = _rand((n, n), 3)
    d = np.random.default_rng(4).random((M, M)) + 0.1
    z = obj.copy()
    pie.pie_update(z, np.ones((n, n), complex), (0, 0), d, pie.partial_dft_transform(n, n, M, M), 1.0, 1.0)
    assert np.allclose(np.abs(dft.partial_dft2(z, M, M)), d, atol=1e-12)
    full_old, full_new = np.fft.fft2(obj), np.fft.fft2(z)
    keep = np.zeros((n, n), bool)
    idx = np.mod(np.arange(-M // 2, M // 2), n)
    keep[np.ix_(idx, idx)] = True
    assert np.allclose(full_new[~keep], full_old[~keep], atol=1e-11)


def test_colouring_is_valid_and_greedy():
    pos = synth.fermat_scan(256, 32, 200)
    col = pie.greedy_colouring(pos, 32, 32)
    for j in range(len(pos)):
        for i in range(j):
            if pie.overlaps(pos[i], pos[j], 32, 32):
                assert col[i] != col[j]
        # greedy: every smaller colour is taken by an earlier overlapping position
        earlier = {int(col[i]) for i in range(j) if pie.overlaps(pos[i], pos[j], 32, 32)}
        assert set(range(col[j])) <= earlier


def test_order_within_a_colour_does_not_matter():
    """Positions of one colour have disjoint patches, so permuting them inside
    their colour gives exactly the same sweep."""
    P = synth.small_raster_problem()
    probe, pos = P["probe"], P["pos"]
    d = pie.amplitudes(P["intensities"])
    col = pie.greedy_colouring(pos, 32, 32)
    order = pie.colour_major_order(col)
    rng = np.random.default_rng(0)
    shuffled = np.concatenate([rng.permutation(order[col[order] == c]) for c in range(col.max() + 1)])
    T = pie.full_transform(32, 32)
    z1, f1 = pie.pie_sweep(P["init"], probe, pos, d, T, 0.8, order)
    z2, f2 = pie.pie_sweep(P["init"], probe, pos, d, T, 0.8, shuffled)
    assert np.allclose(z1, z2, rtol=0, atol=1e-13)
    assert f1 == pytest.approx(f2, rel=1e-12)


def test_batched_equals_sequential_without_overlap():
    """With disjoint patches and |w| = 1 the illumination is 1 on every patch, so
    the batched update (delta = 0) equals the sequential one."""
    n = 8
    obj = _rand((32, 32), 5)
    probe = np.exp(1j * np.random.default_rng(6).random((n, n)))
    pos = synth.raster_scan(4, 4, 8, 0)
    d = np.random.default_rng(7).random((16, n, n)) + 0.1
    T = pie.full_transform(n, n)
    zs, fs = pie.pie_sweep(obj, probe, pos, d, T, 0.9)
    zb, fb = pie.batched_sweep(obj, probe, pos, d, T, 0.9, delta_rel=0.0)
    assert np.allclose(zs, zb, atol=1e-13)
    assert fs == pytest.approx(fb, rel=1e-12)


def test_batched_step_projects_a_single_exit_wave():
    """One position, delta = 0, beta = 1, FULL: the batched step divides by the
    illumination |w|^2, so z <- z - conj(w) (w z - P_M(z)) / |w|^2 makes the new
    exit wave w z exactly P_M(z) (Eq. 3) for any probe without zeros."""
    n = 16
    obj = _rand((n, n), 12)          # the patch covers the object (no unlit pixel to divide by 0)
    rng = np.random.default_rng(13)
    probe = (0.3 + rng.random((n, n))) * np.exp(2j * np.pi * rng.random((n, n)))
    d = rng.random((1, n, n)) + 0.1
    pos = np.array([[0, 0]], dtype=np.int32)
    z, _ = pie.batched_sweep(obj, probe, pos, d, pie.full_transform(n, n), 1.0, delta_rel=0.0)
    old = np.fft.fft2(probe * obj)
    new = np.fft.fft2(probe * z)
    assert np.allclose(new, d[0] * old / np.abs(old), rtol=1e-12, atol=1e-12)


def test_noise_free_recovery_up_to_global_phase():
    """FULL PIE from a random start recovers a known object up to a global phase
    on the well-lit region (noise-free data, known probe)."""
    obj = synth.make_object(96)
    probe = synth.make_probe(32)
    pos = synth.fermat_scan(96, 32, 60)
    d = pie.amplitudes(synth.simulate_intensities(obj, probe, pos))
    il = pie.illumination(probe, pos, obj.shape)
    mask = il >= 0.3 * il.max()
    z = synth.random_init(96)
    T = pie.full_transform(32, 32)
    errs = []
    for _ in range(80):
        z, _ = pie.pie_sweep(z, probe, pos, d, T, 1.0)
        errs.append(pie.nrmse(z, obj, mask))
    assert errs[-1] < 1e-2
    assert all(b <= a * 1.001 for a, b in zip(errs[10:], errs[11:]))
    # the phase-free error of Eq. rel_error is no smaller than the aligned one
    assert pie.relative_error(z[mask], obj[mask]) >= errs[-1] - 1e-15


def test_error_metrics_closed_forms():
    """Section 4's stopping rule divides by the previous iterate:
    ||2x - x|| / ||x|| = 1 (0.5 against the new one). The phase-aligned error
    of a rotated, scaled copy is |1 - s| whatever the phase, and it only sees
    the masked pixels."""
    x = _rand((12, 12), 14)
    assert pie.relative_change(2 * x, x) == pytest.approx(1.0, rel=1e-14)
    assert pie.nrmse(0.75 * np.exp(-2.1j) * x, x) == pytest.approx(0.25, rel=1e-12)
    y = x.copy()
    mask = np.zeros(x.shape, bool)
    mask[2:8, 3:9] = True
    y[~mask] += 5.0
    assert pie.nrmse(np.exp(0.4j) * y, x, mask) == pytest.approx(0.0, abs=1e-14)
    assert pie.relative_error(np.exp(0.4j) * x, x) == pytest.approx(abs(np.exp(0.4j) - 1), rel=1e-12)


def test_hybrid_runs_both_phases_and_stops_on_tolerance():
    """Algorithm 3: PFT sweeps on cropped data, then FULL sweeps; each phase
    stops on its relative-change tolerance or its sweep budget."""
    P = synth.small_raster_problem()
    P1, P2 = coeffs.plan_2d(32, 32, 16, 16, 8, 8)
    z, tr = pie.hybrid_pie(P["init"], P["probe"], P["pos"], P["intensities"], pie.pft_transform(P1, P2),
                           16, 1.0, 1.0, 0.0, 4, 0.05, 30, truth=P["obj"])
    phases = [t["phase"] for t in tr]
    assert phases[:4] == ["pft"] * 4 and phases[4] == "full"
    assert tr[-1]["change"] < 0.05 or len(tr) == 34
    assert all("nrmse" in t for t in tr)


def test_colouring_in_a_given_order():
    """Visiting order changes the greedy colouring but not its validity; the
    colour-major order keeps the visiting order inside each colour."""
    pos = synth.fermat_scan(256, 32, 120)
    order = np.random.default_rng(3).permutation(120)
    col = pie.greedy_colouring(pos, 32, 32, order)
    for a, j in enumerate(order):
        for i in order[:a]:
            if pie.overlaps(pos[i], pos[j], 32, 32):
                assert col[i] != col[j]
    cm = pie.colour_major_order(col, order)
    rank = {int(j): a for a, j in enumerate(order)}
    for x, y in zip(cm, cm[1:]):
        assert col[x] < col[y] or (col[x] == col[y] and rank[int(x)] < rank[int(y)])
    assert np.array_equal(pie.greedy_colouring(pos, 32, 32, np.arange(120)), pie.greedy_colouring(pos, 32, 32))


def test_epie_single_position_probe_step():
    """One position, one colour: the probe step equals Eq. epie_probe_update at
    the updated patch with the step gamma / (|z|^2 + delta); with gamma = 0 the
    probe is unchanged and the object step is the non-blind one."""
    n = 16
    obj = _rand((24, 24), 8)
    probe = np.exp(1j * np.random.default_rng(9).random((n, n)))
    d = np.random.default_rng(10).random((1, n, n)) + 0.1
    pos = np.array([[3, 4]], dtype=np.int32)
    T = pie.full_transform(n, n)
    col = np.zeros(1, dtype=np.int64)
    z0, w0, _ = pie.epie_colour_sweep(obj, probe, pos, d, T, 0.7, 0.0, col)
    zs, _ = pie.pie_sweep(obj, probe, pos, d, T, 0.7)
    assert np.allclose(z0, zs, atol=1e-14) and np.allclose(w0, probe, atol=0)
    z1, w1, _ = pie.epie_colour_sweep(obj, probe, pos, d, T, 0.7, 0.5, col, delta_rel=0.0)
    zj = z1[3:3 + n, 4:4 + n]
    step = np.conj(zj) * (probe * zj - np.fft.ifft2(d[0] * np.exp(1j * np.angle(np.fft.fft2(probe * zj)))))
    assert np.allclose(w1, probe - 0.5 * step / np.abs(zj) ** 2, atol=1e-12)


def test_epie_fits_the_data_up_to_blind_ambiguities():
    """Blind PIE from a perturbed probe: object and probe are only determined up
    to the ambiguities of the blind problem (z -> a z, w -> w / a, and opposite
    linear phase ramps), so the pin is on quantities they leave unchanged: the
    residual Phi falls by an order of magnitude and the exit-wave moduli
    |w . Q_j z| approach the true ones (noise-free data)."""
    obj = synth.make_object(96)
    probe = synth.make_probe(32)
    pos = synth.fermat_scan(96, 32, 60)
    d = pie.amplitudes(synth.simulate_intensities(obj, probe, pos))
    col = pie.greedy_colouring(pos, 32, 32)
    w = probe * (1 + 0.2 * np.exp(2j * np.pi * np.random.default_rng(11).random(probe.shape)))
    z = synth.random_init(96)
    T = pie.full_transform(32, 32)

    def exit_err(z, w):
        num = den = 0.0
        for r, c in pos:
            a = np.abs(w * z[r:r + 32, c:c + 32])
            b = np.abs(probe * obj[r:r + 32, c:c + 32])
            num += np.sum((a - b) ** 2)
            den += np.sum(b ** 2)
        return np.sqrt(num / den)

    phis = []
    e0 = exit_err(z, w)
    for _ in range(60):
        z, w, phi = pie.epie_colour_sweep(z, w, pos, d, T, 1.0, 0.2, col)
        phis.append(phi)
    assert phis[-1] < 0.1 * phis[0]
    assert exit_err(z, w) < 0.25 * e0


# ---------------------------------------------------------------- Eq. epie_probe_update, sequential
def test_epie_sweep_probe_step_projects_the_probe():
    """One position, beta = 0 (the patch stays c, a non-real unit constant),
    gamma = 1: Eq. epie_probe_update gives w' = w - conj(c)(c w - P_M) =
    conj(c) P_M, so the new exit wave c w' has spectrum d e^{i theta(F(c w))}:
    modulus d and the phase of the old exit wave's spectrum."""
    n = 16
    c = np.exp(0.9j)
    obj = np.full((24, 24), c)
    w = _rand((n, n), 21)
    d = np.random.default_rng(22).random((1, n, n)) + 0.1
    pos = np.array([[4, 3]], dtype=np.int32)
    z, w1, _ = pie.epie_sweep(obj, w, pos, d, pie.full_transform(n, n), 0.0, 1.0)
    assert np.array_equal(z, obj)
    old = np.fft.fft2(c * w)
    assert np.allclose(np.fft.fft2(c * w1), d[0] * old / np.abs(old), rtol=1e-12, atol=1e-12)


def test_epie_sweep_probe_step_at_the_updated_patch():
    """One position, beta = 1, a unit-modulus probe: the object step alone makes
    the exit wave P_M (w z' = |w|^2 P_M = P_M), so the probe step, evaluated at
    the updated patch z', has a zero residual and leaves the probe unchanged
    (evaluated at the old patch it would move it)."""
    n = 16
    obj = _rand((24, 24), 23)
    w = np.exp(2j * np.pi * np.random.default_rng(24).random((n, n)))
    d = np.random.default_rng(25).random((1, n, n)) + 0.1
    pos = np.array([[2, 6]], dtype=np.int32)
    z, w1, _ = pie.epie_sweep(obj, w, pos, d, pie.full_transform(n, n), 1.0, 0.7)
    assert np.allclose(np.abs(np.fft.fft2(w * z[2:2 + n, 6:6 + n])), d[0], rtol=1e-12, atol=1e-12)
    assert np.allclose(w1, w, rtol=0, atol=1e-12)


def test_epie_sweep_updates_the_probe_after_every_position():
    """Two positions on the same pixels of an all-ones object, beta = 0,
    gamma = 1/2: each step keeps the phase of F w and averages its modulus with
    that position's data, |F w| -> (|F w| + d_j)/2, so after the sweep
    |F w| = |F w0|/4 + d_1/4 + d_2/2 (the second position sees the probe the
    first one left; a summed or reordered step gives another modulus)."""
    n = 16
    obj = np.ones((20, 20), complex)
    w0 = _rand((n, n), 26)
    d = np.random.default_rng(27).random((2, n, n)) + 0.1
    pos = np.array([[1, 2], [1, 2]], dtype=np.int32)
    _, w2, _ = pie.epie_sweep(obj, w0, pos, d, pie.full_transform(n, n), 0.0, 0.5)
    F0 = np.fft.fft2(w0)
    expect = (np.abs(F0) / 4 + d[0] / 4 + d[1] / 2) * F0 / np.abs(F0)
    assert np.allclose(np.fft.fft2(w2), expect, rtol=1e-12, atol=1e-12)


def test_epie_sweep_with_gamma_zero_is_pie():
    """gamma = 0: the probe never changes and the sweep is Eq. pie_update alone,
    in the same visiting order."""
    P = synth.small_raster_problem()
    d = pie.amplitudes(P["intensities"])
    order = np.random.default_rng(28).permutation(len(P["pos"]))
    T = pie.full_transform(32, 32)
    z, w, phi = pie.epie_sweep(P["init"], P["probe"], P["pos"], d, T, 0.8, 0.0, order)
    zs, phis = pie.pie_sweep(P["init"], P["probe"], P["pos"], d, T, 0.8, order)
    assert np.array_equal(w, P["probe"].astype(np.complex128))
    assert np.allclose(z, zs, rtol=0, atol=1e-13) and phi == pytest.approx(phis, rel=1e-13)


def test_colour_sweep_with_one_position_per_colour_is_the_sequential_sweep():
    """The colour-synchronous variant with the pixel-wise normaliser off and one
    position per colour is epie_sweep in the same (random) order, exactly."""
    P = synth.small_raster_problem()
    d = pie.amplitudes(P["intensities"], 16)
    order = np.random.default_rng(29).permutation(len(P["pos"]))
    col = pie.sequential_colouring(order)
    assert np.array_equal(pie.colour_major_order(col, order), order)
    T = pie.pft_transform(*coeffs.plan_2d(32, 32, 16, 16, 8, 8))
    w0 = P["probe"] * (1 + 0.1 * _rand(P["probe"].shape, 30))
    z1, w1, p1 = pie.epie_sweep(P["init"], w0, P["pos"], d, T, 0.9, 0.05, order)
    z2, w2, p2 = pie.epie_colour_sweep(P["init"], w0, P["pos"], d, T, 0.9, 0.05, col, order, normalise=False)
    assert np.allclose(z1, z2, rtol=0, atol=1e-12) and np.allclose(w1, w2, rtol=0, atol=1e-12)
    assert p1 == pytest.approx(p2, rel=1e-12)
