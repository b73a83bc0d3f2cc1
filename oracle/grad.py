"""Amplitude loss through a Fourier operator, its gradient, and finite differences.

Section 1 of the paper motivates a differentiable PFT so that gradient methods
can run through it. The loss here is
    L(z, w) = sum_j || |A(w . Q_j z)| - d_j ||^2,
with A the PFT (or any linear operator with an adjoint) and d_j the cropped
amplitudes. With Psi_j = A psi_j and R_j = Psi_j - d_j sgn(Psi_j)
(sgn(0) = 0), the gradients in the convention dL/dRe + i dL/dIm are
    g_psi_j = 2 A^H R_j,
    grad_z = sum_j Q_j^T ( conj(w) . g_psi_j ),
    grad_w = sum_j conj(Q_j z) . g_psi_j.
"""
from __future__ import annotations

import numpy as np


def _patches(z: np.ndarray, positions: np.ndarray, n1: int, n2: int) -> np.ndarray:
    return np.stack([z[r:r + n1, c:c + n2] for r, c in positions])


def amplitude_loss(z: np.ndarray, probe: np.ndarray, positions: np.ndarray, d: np.ndarray,
                   T: dict) -> float:
    """L(z, w) = sum_j || |A(w . Q_j z)| - d_j ||^2."""
    n1, n2 = probe.shape
    Psi = T["fwd"](probe[None] * _patches(z, positions, n1, n2))
    return float(np.sum((np.abs(Psi) - d) ** 2))


def amplitude_loss_grad(z: np.ndarray, probe: np.ndarray, positions: np.ndarray, d: np.ndarray,
                        T: dict) -> tuple[float, np.ndarray, np.ndarray]:
    """(L, grad_z, grad_w) with grad = dL/dRe + i dL/dIm."""
    n1, n2 = probe.shape
    P = _patches(z, positions, n1, n2)
    Psi = T["fwd"](probe[None] * P)
    mag = np.abs(Psi)
    sgn = np.where(mag > 0.0, Psi / np.where(mag > 0.0, mag, 1.0), 0.0)
    R = Psi - d * sgn
    loss = float(np.sum((mag - d) ** 2))
    g_psi = 2.0 * T["adj"](R)
    grad_z = np.zeros_like(z, dtype=np.complex128)
    for j, (r, c) in enumerate(positions):
        grad_z[r:r + n1, c:c + n2] += np.conj(probe) * g_psi[j]
    grad_w = np.sum(np.conj(P) * g_psi, axis=0)
    return loss, grad_z, grad_w


def finite_difference(fun, x: np.ndarray, index, h: float = 1e-6) -> complex:
    """Central differences of a real function of a complex array at one entry:
    (f(x + h) - f(x - h)) / 2h + i (f(x + ih) - f(x - ih)) / 2h."""
    def at(delta):
        y = np.array(x, dtype=np.complex128, copy=True)
        y[index] += delta
        return fun(y)
    re = (at(h) - at(-h)) / (2.0 * h)
    im = (at(1j * h) - at(-1j * h)) / (2.0 * h)
    return complex(re, im)
