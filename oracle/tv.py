"""Total-variation regularisation of the object (Section 4: the reconstructions
use TV regularisation, with a larger weight in the PFT phase).

The paper does not spell the TV term out. Reading: the smoothed isotropic TV
of the complex object with forward differences and zero flux at the far edge,
    D_x z[i, j] = z[i, j+1] - z[i, j]  (0 in the last column),
    D_y z[i, j] = z[i+1, j] - z[i, j]  (0 in the last row),
    TV(z) = sum_ij sqrt(|D_x z|^2 + |D_y z|^2 + eps^2),
whose gradient (dTV/dRe + i dTV/dIm) is
    g = D_x^H (D_x z / s) + D_y^H (D_y z / s),  s = sqrt(|D_x z|^2 + |D_y z|^2 + eps^2),
and the regularised PIE takes one gradient step z <- z - lambda g after each
sweep.
"""
from __future__ import annotations

import numpy as np


def dx(z: np.ndarray) -> np.ndarray:
    out = np.zeros_like(z)
    out[:, :-1] = z[:, 1:] - z[:, :-1]
    return out


def dy(z: np.ndarray) -> np.ndarray:
    out = np.zeros_like(z)
    out[:-1, :] = z[1:, :] - z[:-1, :]
    return out


def dx_adjoint(u: np.ndarray) -> np.ndarray:
    """Conjugate transpose of dx (u's last column is ignored, as dx never fills it)."""
    u = np.array(u, copy=True)
    u[:, -1] = 0
    out = np.zeros_like(u)
    out[:, 1:] += u[:, :-1]
    out[:, :-1] -= u[:, :-1]
    return out


def dy_adjoint(v: np.ndarray) -> np.ndarray:
    v = np.array(v, copy=True)
    v[-1, :] = 0
    out = np.zeros_like(v)
    out[1:, :] += v[:-1, :]
    out[:-1, :] -= v[:-1, :]
    return out


def tv(z: np.ndarray, eps: float) -> float:
    a, b = dx(z), dy(z)
    return float(np.sum(np.sqrt(np.abs(a) ** 2 + np.abs(b) ** 2 + eps * eps)))


def tv_grad(z: np.ndarray, eps: float) -> np.ndarray:
    a, b = dx(z), dy(z)
    s = np.sqrt(np.abs(a) ** 2 + np.abs(b) ** 2 + eps * eps)
    return dx_adjoint(a / s) + dy_adjoint(b / s)


def tv_step(z: np.ndarray, lam: float, eps: float) -> np.ndarray:
    """One gradient step z - lambda grad TV(z)."""
    return z - lam * tv_grad(z, eps)
