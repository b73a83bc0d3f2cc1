"""PIE with a full or partial Fourier transform, and the hybrid of Algorithm 3.

Section 2.1: with psi = w . Q_j z and the modulus projection (Eq. 3)
    P_M(z) = F^{-1}[ d_j . exp(i theta(F psi)) ],
the PIE object update (Eq. pie_update) is
    z_j <- z_j - beta conj(w) (w . z_j - P_M(z_j)),
written back into the pixels of patch Q_j. The objective (Eq. 4) is
    Phi = (1/N) sum_j || w . Q_j z - P_M(z) ||^2.

Readings used here (the paper leaves these open):
* theta(0) = 0, so a zero coefficient is replaced by d (torch.angle's value);
* step normalisation: beta conj(w) / max|w|^2 (the classical ePIE scaling;
  for a probe with max |w| = 1 it is the paper's formula unchanged);
* with the PFT the operator A (M1 M2 x n1 n2) has no inverse; following the
  gradient reading of PIE (Section 2.1: the iterates are gradient steps on
  Phi) and differentiation through the operator (Section 1),
      w . z_j - P_M(z_j) := A^H (A psi - d^crop . exp(i theta(A psi))) / (n1 n2),
  which for A = F is exactly the expression above (F^{-1} = F^H / (n1 n2));
* Phi is accumulated during a sweep as (1/N) sum_j || R_j ||^2 / (n1 n2)
  with R_j = A psi_j - d_j exp(i theta(A psi_j)) (Parseval makes this Eq. 4
  for A = F);
* order: positions are visited in a given order (sequential j = 1..N by
  default). The GPU visits them colour by colour; in a colouring no two
  patches of one colour overlap, so any order within a colour gives the same
  result, and the colour-major order below is an ordinary PIE order;
* batched mode (all positions read the same object, updates summed and
  divided by the illumination sum_j |w_j|^2 + delta) is a different, parallel
  algorithm, given here so the GPU's batched mode has a reference.
"""
from __future__ import annotations

import numpy as np

from . import dft as _dft
from . import pft as _pft


# ---------------------------------------------------------------------------
# transforms: (forward, adjoint) pairs on [..., n1, n2] frames
# ---------------------------------------------------------------------------

def full_transform(n1: int, n2: int) -> dict:
    """A = F, the full unnormalised 2-D DFT; A^H = n1 n2 F^{-1}."""
    return dict(kind="full", n1=n1, n2=n2,
                fwd=lambda x: _dft.full_dft2(x),
                adj=lambda y: _dft.full_idft2(y) * (n1 * n2))


def pft_transform(plan1: dict, plan2: dict) -> dict:
    """A = the 2-D PFT of Algorithm 5 with the given Algorithm-4 tables."""
    return dict(kind="pft", n1=plan1["n"], n2=plan2["n"], M1=plan1["M"], M2=plan2["M"],
                fwd=lambda x: _pft.pft2(x, plan1, plan2),
                adj=lambda y: _pft.pft2_adjoint(y, plan1, plan2))


def partial_dft_transform(n1: int, n2: int, M1: int, M2: int) -> dict:
    """A = the exact partial DFT (lowest M1 x M2 frequencies)."""
    return dict(kind="partial", n1=n1, n2=n2, M1=M1, M2=M2,
                fwd=lambda x: _dft.partial_dft2(x, M1, M2),
                adj=lambda y: _dft.partial_dft2_adjoint(y, n1, n2))


def amplitudes(intensities: np.ndarray, M: int | None = None) -> np.ndarray:
    """d_j = sqrt(I_j) (FFT order); with M, the centred crop d_j^crop (the cropped data of Algorithm 3)."""
    d = np.sqrt(np.maximum(np.asarray(intensities, dtype=np.float64), 0.0))
    return d if M is None else _dft.crop_centre(d, M, M)


# ---------------------------------------------------------------------------
# one update, one sweep
# ---------------------------------------------------------------------------

def residual(Psi: np.ndarray, d: np.ndarray) -> np.ndarray:
    """R = Psi - d . exp(i theta(Psi)) with theta(0) = 0 (Eq. 3)."""
    mag = np.abs(Psi)
    phase = np.where(mag > 0.0, Psi / np.where(mag > 0.0, mag, 1.0), 1.0)
    return Psi - d * phase


def pie_update(obj: np.ndarray, probe: np.ndarray, pos, d: np.ndarray, T: dict,
               beta: float, probe_max2: float) -> float:
    """Eq. pie_update at one position, in place on obj; returns ||R||^2/(n1 n2)."""
    n1, n2 = probe.shape
    r, c = int(pos[0]), int(pos[1])
    patch = obj[r:r + n1, c:c + n2]
    psi = probe * patch
    R = residual(T["fwd"](psi), d)
    dpsi = T["adj"](R) / (n1 * n2)          # w . z_j - P_M(z_j)
    obj[r:r + n1, c:c + n2] = patch - beta * np.conj(probe) / probe_max2 * dpsi
    return float(np.sum(np.abs(R) ** 2)) / (n1 * n2)


def pie_sweep(obj: np.ndarray, probe: np.ndarray, positions: np.ndarray, data: np.ndarray,
              T: dict, beta: float, order=None) -> tuple[np.ndarray, float]:
    """One sweep of sequential PIE over the positions in ``order``; returns (z, Phi)."""
    z = np.array(obj, dtype=np.complex128, copy=True)
    probe_max2 = float(np.max(np.abs(probe) ** 2))
    order = range(len(positions)) if order is None else order
    tot = 0.0
    for j in order:
        tot += pie_update(z, probe, positions[j], data[j], T, beta, probe_max2)
    return z, tot / len(positions)


def batched_sweep(obj: np.ndarray, probe: np.ndarray, positions: np.ndarray, data: np.ndarray,
                  T: dict, beta: float, delta_rel: float = 1e-3) -> tuple[np.ndarray, float]:
    """Parallel variant: every position reads the same z;
    z <- z - beta * sum_j Q_j^T(conj(w) dpsi_j) / (sum_j Q_j^T|w|^2 + delta),
    delta = delta_rel * max of the illumination sum_j Q_j^T |w|^2."""
    n1, n2 = probe.shape
    z = np.asarray(obj, dtype=np.complex128)
    acc = np.zeros_like(z)
    illum = illumination(probe, positions, z.shape)
    tot = 0.0
    for j, (r, c) in enumerate(positions):
        psi = probe * z[r:r + n1, c:c + n2]
        R = residual(T["fwd"](psi), data[j])
        tot += float(np.sum(np.abs(R) ** 2)) / (n1 * n2)
        acc[r:r + n1, c:c + n2] += np.conj(probe) * T["adj"](R) / (n1 * n2)
    denom = illum + delta_rel * illum.max()
    return z - beta * acc / denom, tot / len(positions)


def illumination(probe: np.ndarray, positions: np.ndarray, shape) -> np.ndarray:
    """sum_j Q_j^T |w|^2 over the object grid."""
    n1, n2 = probe.shape
    out = np.zeros(shape, dtype=np.float64)
    p2 = np.abs(probe) ** 2
    for r, c in positions:
        out[r:r + n1, c:c + n2] += p2
    return out


def epie_sweep(obj: np.ndarray, probe: np.ndarray, positions: np.ndarray, data: np.ndarray,
               T: dict, beta: float, gamma: float, order=None) -> tuple[np.ndarray, np.ndarray, float]:
    """Blind PIE as Section 2.1 states it: one sweep of Eq. pie_update and Eq.
    epie_probe_update, the probe refined after every position.

    Positions are visited in ``order`` (index order by default; the blind
    experiments of Section 4.2 draw a uniformly random order without
    replacement). At position j, with the current probe w^k:
      1. z_j^{k+1} = z_j^k - beta conj(w^k)/max|w^k|^2 (w^k z_j^k - P_M(z_j^k))
         (the object step with reading R8's normalisation);
      2. w^{k+1} = w^k - gamma conj(z_j^{k+1}) (w^k z_j^{k+1} - P_M(z_j^{k+1})),
         the projection taken with w^k (the modulus set of Eq. epie_probe_update
         is the one of w^k) and gamma a plain scalar, as printed.
    w z - P_M(z) is A^H R / (n1 n2) (reading R4). Returns (z, w, Phi), Phi from
    the object steps."""
    n1, n2 = probe.shape
    z = np.array(obj, dtype=np.complex128, copy=True)
    w = np.array(probe, dtype=np.complex128, copy=True)
    order = range(len(positions)) if order is None else order
    tot = 0.0
    for j in order:
        tot += pie_update(z, w, positions[j], data[j], T, beta, float(np.max(np.abs(w) ** 2)))
        r, c = int(positions[j][0]), int(positions[j][1])
        zj = z[r:r + n1, c:c + n2]                       # z_j^{k+1}
        R = residual(T["fwd"](w * zj), data[j])
        w = w - gamma * np.conj(zj) * (T["adj"](R) / (n1 * n2))
    return z, w, tot / len(positions)


def epie_colour_sweep(obj: np.ndarray, probe: np.ndarray, positions: np.ndarray, data: np.ndarray,
                      T: dict, beta: float, gamma: float, colours: np.ndarray, order=None,
                      delta_rel: float = 1e-3, normalise: bool = True) -> tuple[np.ndarray, np.ndarray, float]:
    """Blind PIE, colour-synchronous: a parallel variant of epie_sweep (reading R14).

    The probe is shared by every position, so positions that run together
    cannot each see the probe left by the previous one. Within a colour every
    position uses the probe w of the colour's start and updates its patch
    (Eq. pie_update); then the probe step of Eq. epie_probe_update is evaluated
    at the updated patch z_j^{k+1},
        g_j = conj(z_j^{k+1}) . (w . z_j^{k+1} - P_M(z_j^{k+1})),
    and the colour's steps are summed. With ``normalise`` (the default) the sum
    is divided pixel by pixel,
        w <- w - gamma * sum_j g_j / (sum_j |z_j^{k+1}|^2 + delta),
    delta = delta_rel * max of that sum; without it w <- w - gamma sum_j g_j,
    the scalar step of Eq. epie_probe_update, and with one position per colour
    the sweep is then epie_sweep in colour-major order. Returns (z, w, Phi)."""
    n1, n2 = probe.shape
    z = np.array(obj, dtype=np.complex128, copy=True)
    w = np.array(probe, dtype=np.complex128, copy=True)
    cm = colour_major_order(colours, order)
    tot = 0.0
    for c in range(int(colours.max()) + 1):
        members = [j for j in cm if colours[j] == c]
        wmax2 = float(np.max(np.abs(w) ** 2))
        for j in members:
            tot += pie_update(z, w, positions[j], data[j], T, beta, wmax2)
        acc = np.zeros_like(w)
        den = np.zeros(w.shape)
        for j in members:
            r, cc = positions[j]
            zj = z[r:r + n1, cc:cc + n2]
            R = residual(T["fwd"](w * zj), data[j])
            acc += np.conj(zj) * T["adj"](R) / (n1 * n2)
            den += np.abs(zj) ** 2
        w = w - gamma * (acc / (den + delta_rel * den.max()) if normalise else acc)
    return z, w, tot / len(positions)


def sequential_colouring(order) -> np.ndarray:
    """One position per colour, colours in visiting order: colour-major order
    is then the visiting order itself (exact sequential PIE)."""
    order = np.asarray(order)
    col = np.empty(len(order), dtype=np.int64)
    col[order] = np.arange(len(order))
    return col


# ---------------------------------------------------------------------------
# position colouring (overlap-free classes)
# ---------------------------------------------------------------------------

def overlaps(a, b, n1: int, n2: int) -> bool:
    """Two n1 x n2 patches with top-left corners a and b share a pixel."""
    return abs(int(a[0]) - int(b[0])) < n1 and abs(int(a[1]) - int(b[1])) < n2


def greedy_colouring(positions: np.ndarray, n1: int, n2: int, order=None) -> np.ndarray:
    """Greedy colouring: positions are visited in ``order`` (index order by
    default) and each takes the smallest colour not used by an earlier-visited
    position whose patch overlaps its own."""
    N = len(positions)
    order = np.arange(N) if order is None else np.asarray(order)
    col = np.full(N, -1, dtype=np.int64)
    for a, j in enumerate(order):
        used = set()
        for i in order[:a]:
            if overlaps(positions[i], positions[j], n1, n2):
                used.add(int(col[i]))
        k = 0
        while k in used:
            k += 1
        col[j] = k
    return col


def colour_major_order(colours: np.ndarray, order=None) -> np.ndarray:
    """Positions sorted by colour, in visiting order (index order by default)
    within a colour."""
    N = len(colours)
    rank = np.empty(N, dtype=np.int64)
    rank[np.arange(N) if order is None else np.asarray(order)] = np.arange(N)
    return np.lexsort((rank, colours))


# ---------------------------------------------------------------------------
# metrics and the hybrid driver
# ---------------------------------------------------------------------------

def relative_change(new: np.ndarray, old: np.ndarray) -> float:
    """||z^{k+1} - z^k|| / ||z^k|| (the stopping rule of Section 4)."""
    return float(np.linalg.norm(new - old) / np.linalg.norm(old))


def relative_error(z: np.ndarray, truth: np.ndarray) -> float:
    """Eq. rel_error: ||z - z_true|| / ||z_true|| (no phase alignment)."""
    return float(np.linalg.norm(z - truth) / np.linalg.norm(truth))


def illuminated_mask(probe: np.ndarray, positions: np.ndarray, shape,
                     thresh: float = 1e-3) -> np.ndarray:
    """Pixels whose illumination is at least thresh times its maximum."""
    il = illumination(probe, positions, shape)
    return il >= thresh * il.max()


def nrmse(z: np.ndarray, truth: np.ndarray, mask: np.ndarray | None = None) -> float:
    """min over a global phase phi of ||e^{i phi} z - z_true|| / ||z_true|| on the mask.

    The optimal phase is the argument of <z, z_true> = sum conj(z) z_true.
    """
    if mask is not None:
        z, truth = z[mask], truth[mask]
    ip = np.vdot(z, truth)
    ph = ip / abs(ip) if abs(ip) > 0 else 1.0
    return float(np.linalg.norm(ph * z - truth) / np.linalg.norm(truth))


def hybrid_pie(init: np.ndarray, probe: np.ndarray, positions: np.ndarray,
               intensities: np.ndarray, T_pft: dict, M: int, beta_pft: float, beta_full: float,
               tol_pft: float, max_pft: int, tol_full: float, max_full: int,
               order=None, truth: np.ndarray | None = None, tv_pft: float = 0.0, tv_full: float = 0.0,
               tv_eps: float = 1e-3) -> tuple[np.ndarray, list]:
    """Algorithm 3: crop the data, PFT-PIE until tol_pft or max_pft sweeps,
    then full-FFT PIE from that point until tol_full or max_full sweeps. With
    a TV weight, each sweep of that phase is followed by one TV gradient step
    (Section 4 regularises both phases, the PFT phase more strongly).

    Returns (z, trace) with one dict per sweep: phase, Phi, relative change and
    (with a truth) the phase-aligned error on the illuminated mask.
    """
    n1, n2 = probe.shape
    d_full = amplitudes(intensities)
    d_crop = _dft.crop_centre(d_full, M, M)                  # cropped data for the PFT phase
    T_full = full_transform(n1, n2)
    mask = illuminated_mask(probe, positions, init.shape) if truth is not None else None
    z = np.array(init, dtype=np.complex128, copy=True)
    trace = []
    from . import tv as _tv
    for phase, T, data, beta, tol, mx, lam in (("pft", T_pft, d_crop, beta_pft, tol_pft, max_pft, tv_pft),
                                                ("full", T_full, d_full, beta_full, tol_full, max_full, tv_full)):
        for _ in range(mx):                                  # the PFT phase, then the full phase
            z_new, phi = pie_sweep(z, probe, positions, data, T, beta, order)
            if lam > 0.0:
                z_new = _tv.tv_step(z_new, lam, tv_eps)
            ch = relative_change(z_new, z)
            z = z_new
            rec = dict(phase=phase, phi=phi, change=ch)
            if truth is not None:
                rec["nrmse"] = nrmse(z, truth, mask)
            trace.append(rec)
            if ch < tol:
                break
    return z, trace

