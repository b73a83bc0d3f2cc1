"""Online phase of the PFT (Algorithms 2 and 5) and the adjoint of Algorithm 5.

1-D (Algorithm 2), with the tables of Algorithm 1, B (q x r) and W (M x r):
    Z = z.reshape(p, q);  C = Z B;  C^[:, j] = FFT_p(C[:, j]);
    z^_PFT[t] = sum_j C^[t mod p, j] W[t, j].

2-D (Algorithm 5), with one table pair per axis:
    Z = z.reshape(p1, q1, p2, q2).permute(0, 2, 1, 3)        -> [p1, p2, q1, q2]
    C[k1, k2] = B1^T Z[k1, k2] B2                           (plain transpose)
    C^[:, :, j1, j2] = FFT2(C[:, :, j1, j2])
    z^_PFT[t1, t2] = sum_{j1, j2} C^[t1 mod p1, t2 mod p2, j1, j2] W1[t1, j1] W2[t2, j2]
(W of Algorithm 4 is separable: W[t1, t2, j1, j2] = W1[t1, j1] W2[t2, j2].)

The adjoint is not printed in the paper; the paper differentiates through the
operator (Section 1). Reversing each linear step of Algorithm 5 gives, per axis,
    H[u, j]  = sum_{t = u mod p} conj(W[t, j]) y[t]     (scatter by residue)
    E[k, j]  = sum_u e^{+2 pi i u k / p} H[u, j]        (= p * inverse FFT_p)
    x[q k + l] = sum_j conj(B[l, j]) E[k, j],
applied on both axes.
"""
from __future__ import annotations

import numpy as np


def pft1(z: np.ndarray, plan: dict) -> np.ndarray:
    """Algorithm 2 on a vector z (length n); returns M values for t = -M/2 .. M/2-1."""
    p, q, t = plan["p"], plan["q"], plan["t"]
    Z = z.reshape(p, q)                       # p blocks of q consecutive values
    C = Z @ plan["B"]                         # compress every block with B
    Chat = np.fft.fft(C, axis=0)              # length-p FFT of each column
    out = np.zeros(t.size, dtype=np.complex128)
    for a, tt in enumerate(t):                # combine with W at residue t mod p
        out[a] = np.sum(Chat[tt % p, :] * plan["W"][a, :])
    return out


def pft2(z: np.ndarray, plan1: dict, plan2: dict, chunk: int = 16) -> np.ndarray:
    """Algorithm 5 on z[..., n1, n2] (any leading batch); centred [..., M1, M2] output.

    Frames are processed ``chunk`` at a time only to bound the memory of step 9.
    """
    lead = z.shape[:-2]
    flat = z.reshape(-1, *z.shape[-2:])
    out = np.empty((flat.shape[0], plan1["M"], plan2["M"]), dtype=np.complex128)
    for s in range(0, flat.shape[0], chunk):
        out[s:s + chunk] = _pft2_frames(flat[s:s + chunk], plan1, plan2)
    return out.reshape(*lead, plan1["M"], plan2["M"])


def _pft2_frames(z: np.ndarray, plan1: dict, plan2: dict) -> np.ndarray:
    p1, q1 = plan1["p"], plan1["q"]
    p2, q2 = plan2["p"], plan2["q"]
    B1, B2, W1, W2 = plan1["B"], plan2["B"], plan1["W"], plan2["W"]
    lead = z.shape[:-2]
    Z = z.reshape(*lead, p1, q1, p2, q2)                      # blocks of q1 x q2
    Z = np.moveaxis(Z, -3, -2)                                # -> [.., p1, p2, q1, q2]
    # compression: C[k1, k2] = B1^T Z[k1, k2] B2 for every block (k1, k2)
    C = np.einsum("lj,...abls,sk->...abjk", B1, Z, B2, optimize=True)
    Chat = np.fft.fft2(C, axes=(-4, -3))                      # p1 x p2 FFT per (j1, j2)
    t1, t2 = plan1["t"], plan2["t"]
    G = Chat[..., np.mod(t1, p1), :, :, :][..., np.mod(t2, p2), :, :]   # [.., M1, M2, r1, r2]
    return np.einsum("...abjk,aj,bk->...ab", G, W1, W2, optimize=True)  # combine with W1, W2


def pft2_adjoint(y: np.ndarray, plan1: dict, plan2: dict, chunk: int = 16) -> np.ndarray:
    """Conjugate transpose of pft2: y[..., M1, M2] -> x[..., n1, n2]."""
    lead = y.shape[:-2]
    flat = y.reshape(-1, *y.shape[-2:])
    out = np.empty((flat.shape[0], plan1["n"], plan2["n"]), dtype=np.complex128)
    for s in range(0, flat.shape[0], chunk):
        out[s:s + chunk] = _pft2_adjoint_frames(flat[s:s + chunk], plan1, plan2)
    return out.reshape(*lead, plan1["n"], plan2["n"])


def _pft2_adjoint_frames(y: np.ndarray, plan1: dict, plan2: dict) -> np.ndarray:
    p1, q1, r1 = plan1["p"], plan1["q"], plan1["r"]
    p2, q2, r2 = plan2["p"], plan2["q"], plan2["r"]
    B1, B2, W1, W2 = plan1["B"], plan2["B"], plan1["W"], plan2["W"]
    t1, t2 = plan1["t"], plan2["t"]
    lead = y.shape[:-2]
    # adjoint of the W combine: G[t1, t2, j1, j2] = conj(W1) conj(W2) y, summed by residue
    G = np.einsum("...ab,aj,bk->...abjk", y, W1.conj(), W2.conj(), optimize=True)
    H = np.zeros((*lead, p1, p2, r1, r2), dtype=np.complex128)
    for a, u1 in enumerate(np.mod(t1, p1)):
        for b, u2 in enumerate(np.mod(t2, p2)):
            H[..., u1, u2, :, :] += G[..., a, b, :, :]
    # adjoint of the p1 x p2 FFT: the unnormalised DFT's adjoint is p1 p2 * inverse DFT
    E = np.fft.ifft2(H, axes=(-4, -3)) * (p1 * p2)
    # adjoint of the compression: Z[k1, k2] = conj(B1) E[k1, k2] B2^H
    Z = np.einsum("lj,...abjk,sk->...abls", B1.conj(), E, B2.conj(), optimize=True)
    # adjoint of the blocking (a permutation): back to [n1, n2]
    return np.moveaxis(Z, -2, -3).reshape(*lead, p1 * q1, p2 * q2)
