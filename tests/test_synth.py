"""The seeded synthetic inputs follow their stated recipe (object ranges and
smoothness, probe disc and quadratic phase, scans inside the object, the
forward model's intensities and their Poisson scaling, the start of Section 4,
standalone frames, the uneven-batch sizes) and are reproducible."""
import math

import numpy as np
import pytest

from paper_2408_03532_gb300 import synth


def test_object_ranges_smoothness_and_seeding():
    z = synth.make_object(256)
    amp, pha = np.abs(z), np.angle(z)
    assert amp.min() == pytest.approx(0.5, abs=1e-12) and amp.max() == pytest.approx(1.0, abs=1e-12)
    assert pha.min() == pytest.approx(-math.pi / 2, abs=1e-12) and pha.max() == pytest.approx(math.pi / 2, abs=1e-12)
    # Gaussian smoothing (sigma = 2 px): neighbours are strongly correlated
    a = amp - amp.mean()
    corr = float(np.sum(a[:, 1:] * a[:, :-1]) / np.sum(a * a))
    assert corr > 0.9
    assert np.array_equal(z, synth.make_object(256))
    assert not np.allclose(z, synth.make_object(256, seed=synth.SEED_OBJECT + 1))


@pytest.mark.parametrize("n", [32, 128])
def test_probe_disc_edge_and_quadratic_phase(n):
    w = synth.make_probe(n)
    R = 12.0 * n / 32.0
    c = (n - 1) / 2.0
    yy, xx = np.meshgrid(np.arange(n) - c, np.arange(n) - c, indexing="ij")
    rho = np.hypot(yy, xx)
    inside = rho <= R
    assert np.allclose(np.abs(w[inside]), 1.0)
    out = ~inside
    assert np.allclose(np.abs(w[out]), np.exp(-((rho[out] - R) ** 2) / 8.0))
    # phase pi a rho^2 / R^2 with one a in (-1, 1): recover a where the phase has not wrapped
    small = inside & (rho > 1.0) & (rho < 0.5 * R)
    a = np.angle(w[small]) / (math.pi * rho[small] ** 2 / R ** 2)
    assert np.ptp(a) < 1e-9 and -1.0 < a[0] < 1.0


def test_raster_and_spiral_scans_stay_inside_the_object():
    pos = synth.raster_scan(8, 8, 12, 6)
    assert pos.shape == (64, 2) and pos.min() == 6 and pos.max() == 6 + 7 * 12
    assert (pos[1] - pos[0]).tolist() == [0, 12]
    side, n, N = 1024, 128, 3600
    pos = synth.fermat_scan(side, n, N)
    assert pos.shape == (N, 2) and pos.min() >= 0 and pos.max() <= side - n
    other = synth.fermat_scan(side, n, N, seed=synth.SEED_SCAN + 1)       # same spiral, other jitter
    d = np.abs(pos.astype(int) - other.astype(int))
    assert d.max() <= 2 and d.max() > 0                                     # jitter in {-1, 0, 1} per draw
    assert len(np.unique(pos, axis=0)) > 0.99 * N


def test_intensities_follow_the_forward_model_and_its_noise():
    obj = synth.make_object(96)
    w = synth.make_probe(32)
    pos = synth.raster_scan(3, 3, 24, 8)
    I = synth.simulate_intensities(obj, w, pos)
    for j, (r, c) in enumerate(pos):
        psi = w * obj[r:r + 32, c:c + 32]
        assert I[j].sum() == pytest.approx(32 * 32 * np.sum(np.abs(psi) ** 2), rel=1e-12)   # Parseval
        assert I[j, 0, 0] == pytest.approx(abs(psi.sum()) ** 2, rel=1e-12)                  # FFT order: DC first
    Ip = synth.simulate_intensities(obj, w, pos, peak_photons=1e4)
    for j in range(len(pos)):
        s = 1e4 / I[j].max()
        counts = Ip[j] * s
        assert np.allclose(counts, np.rint(counts), atol=1e-6)             # integer counts, scaled back
        assert abs(counts.max() - 1e4) < 5 * math.sqrt(1e4)


def test_start_frames_and_batch_recipe():
    z = synth.random_init(64)
    assert np.abs(z).max() < 1.0 and np.angle(z).min() >= 0.0 and np.angle(z).max() < math.pi / 2
    f = synth.random_frames(16, 64)
    assert f.dtype == np.complex64
    for part in (f.real, f.imag):
        assert abs(float(part.mean())) < 0.02 and abs(float(part.var()) - 1.0) < 0.03
    specs = synth.uneven_batch_recipe(64)
    assert len(specs) == 64 and specs == synth.uneven_batch_recipe(64)
    for sp in specs:
        assert sp["side"] in (256, 512, 1024, 2048) and sp["n"] in (64, 128, 256)
        assert sp["n"] < sp["side"] and sp["M"] in (16, 32, 64) and sp["M"] <= sp["n"]
        assert 50 <= sp["npos"] <= 2000


def test_torch_object_recipe():
    """The torch version of the object recipe (for the 16384^2 workload): the same
    ranges, a smooth field (neighbouring pixels close, as after a sigma = 2 px
    Gaussian), and the same draw for the same seed."""
    torch = pytest.importorskip("torch")
    a = synth.make_object_torch(256, "cpu")
    b = synth.make_object_torch(256, "cpu")
    assert a.dtype == torch.complex64 and torch.equal(a, b)
    amp, pha = a.abs(), a.angle()
    assert abs(amp.min().item() - 0.5) < 1e-5 and abs(amp.max().item() - 1.0) < 1e-5
    assert abs(pha.min().item() + np.pi / 2) < 1e-5 and abs(pha.max().item() - np.pi / 2) < 1e-5
    step = (amp[:, 1:] - amp[:, :-1]).abs().mean().item()
    ref = np.abs(np.diff(np.abs(synth.make_object(256)), axis=1)).mean()
    assert 0.5 * ref < step < 2.0 * ref
    assert not torch.equal(a, synth.make_object_torch(256, "cpu", seed=9))
