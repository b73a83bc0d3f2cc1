"""Seeded synthetic inputs shaped like the paper's ptychography workloads.

This module is shared by the FP64 oracle tests and by the GPU library's tests
and benchmark. It only draws and shapes inputs: objects, probes, scan
positions, initial guesses, standalone frames, and the simulated diffraction
intensities of the forward model (Eq. 1, d_j = |F(w . Q_j z)|), which use
numpy's FFT as a library routine. It holds no part of the reconstruction
method (no PFT, no partial DFT, no PIE update, no projection), so neither side
of a parity test borrows arithmetic from the other through it.

Recipes (the paper's baboon/cameraman images are not available, so these
synthetic stand-ins replace them):

* object: i.i.d. uniform noise for amplitude and phase, each smoothed by a
  Gaussian of sigma = 2 px (truncated at 4 sigma, reflecting boundary), then
  min-max rescaled to amplitude [0.5, 1] and phase [-pi/2, pi/2];
* probe: a disc of radius R (12 px for a 32 px frame, scaled with the frame
  side) with a Gaussian edge of 2 px and a random quadratic phase
  pi * a * rho^2 / R^2, a ~ U(-1, 1);
* scans: rasters with a given stride and offset, or a Fermat spiral
  (rho_k = c sqrt(k), theta_k = k * 137.508 deg) with uniform integer jitter
  in {-1, 0, 1} per axis, clamped so that every patch lies in the object;
* intensities: I_j = |FFT2(probe * patch_j)|^2 in FFT order (not shifted),
  optionally Poisson-sampled at a given peak photon count per frame;
* initial guess: magnitude U[0, 1], phase U[0, pi/2] (Section 4);
* standalone frames: real and imaginary parts i.i.d. N(0, 1).
"""
from __future__ import annotations

import math

import numpy as np

GOLDEN_ANGLE_DEG = 137.508

# Seeds used by the benchmark and the tests (object, probe, scan jitter,
# Poisson noise, initial guess, standalone frames).
SEED_OBJECT = 1
SEED_PROBE = 2
SEED_SCAN = 3
SEED_POISSON = 4
SEED_INIT = 5
SEED_FRAMES = 0


def _gaussian_smooth(a: np.ndarray, sigma: float) -> np.ndarray:
    from scipy.ndimage import gaussian_filter

    return gaussian_filter(a, sigma=sigma, mode="reflect", truncate=4.0)


def _minmax(a: np.ndarray, lo: float, hi: float) -> np.ndarray:
    amin, amax = float(a.min()), float(a.max())
    if amax == amin:
        return np.full_like(a, 0.5 * (lo + hi))
    return lo + (hi - lo) * (a - amin) / (amax - amin)


def make_object(side: int, seed: int = SEED_OBJECT, sigma: float = 2.0) -> np.ndarray:
    """Smooth random complex object, amplitude in [0.5, 1], phase in [-pi/2, pi/2]."""
    rng = np.random.default_rng(seed)
    amp = _minmax(_gaussian_smooth(rng.random((side, side)), sigma), 0.5, 1.0)
    pha = _minmax(_gaussian_smooth(rng.random((side, side)), sigma), -math.pi / 2, math.pi / 2)
    return amp * np.exp(1j * pha)


def make_object_torch(side: int, device, seed: int = SEED_OBJECT, sigma: float = 2.0):
    """The make_object recipe drawn and smoothed with torch on `device` (complex64),
    for objects too large for the numpy route (the 16384^2 large-scale workload):
    uniform noise, a separable Gaussian of sigma px truncated at 4 sigma with
    reflecting edges, min-max to amplitude [0.5, 1] and phase [-pi/2, pi/2]. Same
    distribution as make_object, not the same draw."""
    import torch
    import torch.nn.functional as F
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    rad = int(4.0 * sigma + 0.5)
    x = torch.arange(-rad, rad + 1, device=device, dtype=torch.float32)
    k = torch.exp(-0.5 * (x / sigma) ** 2)
    k = k / k.sum()

    def smooth(a):
        a = a[None, None]
        a = F.conv2d(F.pad(a, (rad, rad, 0, 0), mode="reflect"), k.view(1, 1, 1, -1))
        a = F.conv2d(F.pad(a, (0, 0, rad, rad), mode="reflect"), k.view(1, 1, -1, 1))
        return a[0, 0]

    def minmax(a, lo, hi):
        return lo + (hi - lo) * (a - a.min()) / (a.max() - a.min())

    amp = minmax(smooth(torch.rand(side, side, generator=g, device=device)), 0.5, 1.0)
    pha = minmax(smooth(torch.rand(side, side, generator=g, device=device)), -math.pi / 2, math.pi / 2)
    return torch.polar(amp, pha)


def make_probe(n: int, seed: int = SEED_PROBE, radius: float | None = None,
               edge: float = 2.0) -> np.ndarray:
    """Disc probe with a Gaussian edge and a random quadratic phase (complex128 [n, n])."""
    if radius is None:
        radius = 12.0 * n / 32.0
    rng = np.random.default_rng(seed)
    a = rng.uniform(-1.0, 1.0)
    c = (n - 1) / 2.0
    yy, xx = np.meshgrid(np.arange(n) - c, np.arange(n) - c, indexing="ij")
    rho = np.hypot(yy, xx)
    amp = np.where(rho <= radius, 1.0, np.exp(-((rho - radius) ** 2) / (2.0 * edge * edge)))
    return amp * np.exp(1j * math.pi * a * rho * rho / (radius * radius))


def raster_scan(ny: int, nx: int, stride: int, offset: int) -> np.ndarray:
    """Top-left (row, col) offsets of an ny x nx raster, row by row (int32 [N, 2])."""
    r = offset + stride * np.arange(ny)
    c = offset + stride * np.arange(nx)
    rr, cc = np.meshgrid(r, c, indexing="ij")
    return np.stack([rr.ravel(), cc.ravel()], axis=1).astype(np.int32)


def fermat_scan(obj_side: int, n: int, count: int, seed: int = SEED_SCAN,
                jitter: int = 1) -> np.ndarray:
    """Fermat-spiral scan with integer jitter; every n x n patch lies in the object."""
    rng = np.random.default_rng(seed)
    hi = obj_side - n
    centre = hi / 2.0
    rho_max = max(hi / 2.0 - jitter, 0.0)
    c = rho_max / math.sqrt(max(count - 1, 1))
    k = np.arange(count)
    rho = c * np.sqrt(k)
    th = np.deg2rad(GOLDEN_ANGLE_DEG) * k
    r = np.rint(centre + rho * np.sin(th)).astype(np.int64)
    s = np.rint(centre + rho * np.cos(th)).astype(np.int64)
    if jitter:
        r = r + rng.integers(-jitter, jitter + 1, size=count)
        s = s + rng.integers(-jitter, jitter + 1, size=count)
    r = np.clip(r, 0, hi)
    s = np.clip(s, 0, hi)
    return np.stack([r, s], axis=1).astype(np.int32)


def simulate_intensities(obj: np.ndarray, probe: np.ndarray, positions: np.ndarray,
                         peak_photons: float | None = None,
                         seed: int = SEED_POISSON) -> np.ndarray:
    """Far-field intensities |FFT2(probe * patch_j)|^2, FFT order, float64 [N, n, n].

    With ``peak_photons`` each frame j is scaled by s_j = peak / max(I_j),
    Poisson-sampled, and scaled back by 1 / s_j, so that the returned data
    live on the same scale as the noise-free model.
    """
    n1, n2 = probe.shape
    out = np.empty((len(positions), n1, n2), dtype=np.float64)
    for j, (r, c) in enumerate(np.asarray(positions)):
        psi = probe * obj[r:r + n1, c:c + n2]
        out[j] = np.abs(np.fft.fft2(psi)) ** 2
    if peak_photons is not None:
        rng = np.random.default_rng(seed)
        for j in range(len(out)):
            s = peak_photons / out[j].max()
            out[j] = rng.poisson(out[j] * s).astype(np.float64) / s
    return out


def random_init(side: int, seed: int = SEED_INIT) -> np.ndarray:
    """Initial guess with magnitude U[0, 1] and phase U[0, pi/2] (Section 4)."""
    rng = np.random.default_rng(seed)
    mag = rng.random((side, side))
    pha = rng.random((side, side)) * (math.pi / 2)
    return mag * np.exp(1j * pha)


def random_frames(batch: int, n1: int, n2: int | None = None,
                  seed: int = SEED_FRAMES) -> np.ndarray:
    """Standalone frames, real and imaginary parts i.i.d. N(0, 1) (complex64)."""
    n2 = n1 if n2 is None else n2
    rng = np.random.default_rng(seed)
    out = np.empty((batch, n1, n2), dtype=np.complex64)
    out.real = rng.standard_normal((batch, n1, n2), dtype=np.float32)
    out.imag = rng.standard_normal((batch, n1, n2), dtype=np.float32)
    return out


# ---------------------------------------------------------------------------
# Workload recipes (sizes of the paper-shaped configurations)
# ---------------------------------------------------------------------------

def small_raster_problem(noise: bool = False, seed_shift: int = 0) -> dict:
    """128^2 object, 32^2 probe, 8 x 8 raster of stride 12 (offset 6), M = 16.

    ``seed_shift`` draws another instance (object, noise and start move; the
    probe and the raster stay)."""
    obj = make_object(128, seed=SEED_OBJECT + seed_shift)
    probe = make_probe(32)
    pos = raster_scan(8, 8, 12, 6)
    inten = simulate_intensities(obj, probe, pos, 1e4 if noise else None, seed=SEED_POISSON + seed_shift)
    return dict(obj=obj, probe=probe, pos=pos, intensities=inten, M=16,
                init=random_init(128, seed=SEED_INIT + seed_shift))


def spiral_problem(side: int = 1024, n: int = 128, count: int = 3600,
                   peak_photons: float | None = 1e4, M: int = 32, seed_shift: int = 0) -> dict:
    """Fermat-spiral reconstruction (default: 1024^2 object, 128^2 probe, 3600 positions).

    ``seed_shift`` draws another instance of the same recipe (object, scan
    jitter, Poisson noise and start move by the shift; the probe is the
    instrument and stays)."""
    obj = make_object(side, seed=SEED_OBJECT + seed_shift)
    probe = make_probe(n)
    pos = fermat_scan(side, n, count, seed=SEED_SCAN + seed_shift)
    inten = simulate_intensities(obj, probe, pos, peak_photons, seed=SEED_POISSON + seed_shift)
    return dict(obj=obj, probe=probe, pos=pos, intensities=inten, M=M,
                init=random_init(side, seed=SEED_INIT + seed_shift))


def gradient_problem() -> dict:
    """512^2 object, 64^2 probe, 20 x 20 raster of stride 16 (offset 72)."""
    obj = make_object(512)
    probe = make_probe(64)
    pos = raster_scan(20, 20, 16, 72)
    inten = simulate_intensities(obj, probe, pos, None)
    return dict(obj=obj, probe=probe, pos=pos, intensities=inten, M=32,
                init=random_init(512))


def uneven_batch_recipe(count: int = 64, seed: int = 6, max_side: int = 2048,
                        sides=(256, 512, 1024, 2048), probes=(64, 128, 256), Ms=(16, 32, 64),
                        npos=(50, 2000)) -> list[dict]:
    """Sizes of `count` independent reconstructions: object side uniform in
    `sides` (<= max_side), probe side uniform in `probes` (< object side), M
    uniform in `Ms` with M <= probe side, and a uniform number of Fermat-spiral
    positions in [npos[0], npos[1]]. Each entry also carries its own seeds."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        side = int(rng.choice([s for s in sides if s <= max_side]))
        n = int(rng.choice([p for p in probes if p < side]))
        M = int(rng.choice([m for m in Ms if m <= n]))
        N = int(rng.integers(npos[0], npos[1] + 1))
        out.append(dict(side=side, n=n, M=M, npos=N, seed=100 + 7 * i))
    return out


def make_instance(spec: dict) -> dict:
    """Object, probe and scan of one recipe entry (intensities are left to the
    caller, who may compute them on whichever device suits the size)."""
    s = spec["seed"]
    return dict(obj=make_object(spec["side"], seed=s), probe=make_probe(spec["n"], seed=s + 1),
                pos=fermat_scan(spec["side"], spec["n"], spec["npos"], seed=s + 2),
                init=random_init(spec["side"], seed=s + 3), M=spec["M"])


def simulate_intensities_torch(obj, probe, positions, chunk: int = 256):
    """|FFT2(probe * patch_j)|^2 (FFT order, float32) computed with torch on the
    tensors' device; for inputs too large for the numpy route (test input
    synthesis only)."""
    import torch
    n = probe.shape[-1]
    idx = torch.as_tensor(np.asarray(positions, dtype=np.int64), device=obj.device)
    ar = torch.arange(n, device=obj.device)
    out = torch.empty(len(idx), n, n, dtype=torch.float32, device=obj.device)
    for s in range(0, len(idx), chunk):
        part = idx[s:s + chunk]
        rows = part[:, 0, None] + ar[None, :]
        cols = part[:, 1, None] + ar[None, :]
        patches = obj[rows[:, :, None], cols[:, None, :]]
        out[s:s + chunk] = (torch.abs(torch.fft.fft2(probe[None] * patches)) ** 2).float()
    return out
