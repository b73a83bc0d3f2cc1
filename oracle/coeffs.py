"""Offline phase of the PFT: minimax polynomial for e^{i pi x} and the tables.

Section 3.1.1 defines P_{alpha, xi} as the best uniform approximation to
e^{i pi x} on |x| <= xi among polynomials of degree <= alpha, the scope

    xi(eps, r) = sup{ xi >= 0 : || P_{r-1, xi}(x) - e^{i pi x} ||_{|x|<=xi} <= eps },

and writes P_{r-1, xi(eps, r)}(x) = sum_{j<r} w_{eps,r,j} x^j. The paper takes
w from a precomputed database that is not available; this module computes the
best approximation itself as a discrete complex Chebyshev problem on a dense
grid, solved as a linear program (a minimax algorithm in the sense of the
survey the paper cites), in FP64.

Algorithm 1 (1-D) and Algorithm 4 (2-D, one factor per axis) then give

    q = n / p,  r = min{ r : xi(eps, r) >= m~ / p },
    B[l, j] = w_j (1 - 2 l / q)^j,               l in [q], j in [r],
    W[t, j] = (t / p)^j exp(-i pi t / p),          t in the kept range.

Reading of the output range: the kept frequencies are t in [-M/2, M/2 - 1]
(M values per axis, m~ = M/2); the polynomial must cover |t|/p <= M/(2p).
"""
from __future__ import annotations

import functools
import math

import numpy as np
from numpy.polynomial import chebyshev as _cheb

_GRID = 241          # grid points on [0, xi] (Chebyshev-clustered towards xi)
_DIRS = 8            # initial polygon directions bounding the complex modulus
_CUT_TOL = 1e-5      # stop when max |e| on the grid <= delta * (1 + _CUT_TOL)
_CHECK_GRID = 20001  # denser grid used to report the uniform error


def _lobatto(k: int) -> np.ndarray:
    return np.cos(np.pi * np.arange(k) / (k - 1))


@functools.lru_cache(maxsize=None)
def best_approximation(xi: float, r: int) -> tuple[np.ndarray, float]:
    """Best uniform approximation of e^{i pi x} on |x| <= xi by degree r-1.

    Returns (w, err): the monomial coefficients w[j] of P(x) = sum_j w[j] x^j
    (complex128, length r) and the uniform error on a dense check grid.

    Method (discrete complex Chebyshev approximation, solved as a sequence of
    linear programs):
    * symmetry: e^{i pi x} maps to its conjugate under x -> -x, so by
      uniqueness the best approximation has w_j = i^j a_j with a_j real; it is
      written as sum_j i^j b_j T_j(x / xi) with b real, and the error modulus
      is even, so only x in [0, xi] is sampled;
    * start from the least-squares fit on the grid and solve for a correction
      scaled by the start's error, so the LP works with O(1) numbers;
    * the cone |e(x_k)| <= delta is imposed through its tangent half-planes
      Re(e^{-i theta} e(x_k)) <= delta: a few fixed directions first, then at
      every grid point that still violates the cone a cut along the direction
      of its current error (Kelley's cutting-plane method), until the grid
      error meets delta to a relative 1e-5. HiGHS solves each LP.
    """
    from scipy.optimize import linprog

    if r < 1 or xi <= 0.0:
        raise ValueError("need r >= 1 and xi > 0")
    s = np.cos(0.5 * np.pi * np.arange(_GRID) / (_GRID - 1))  # 1 ... 0
    T = _cheb.chebvander(s, r - 1) * (1j ** np.arange(r))[None, :]  # [G, r]
    f = np.exp(1j * np.pi * xi * s)
    # least-squares start (real unknowns b)
    Tr = np.vstack([T.real, T.imag])
    fr = np.concatenate([f.real, f.imag])
    b0, *_ = np.linalg.lstsq(Tr, fr, rcond=None)
    g = f - T @ b0
    scale = float(np.abs(g).max())
    if scale == 0.0:
        return _to_monomial(b0, xi, r), uniform_error(_to_monomial(b0, xi, r), xi)
    g = g / scale
    # cuts: rows (point index, direction)
    th = 2.0 * np.pi * np.arange(_DIRS) / _DIRS
    pts = np.repeat(np.arange(s.size), _DIRS)
    dirs = np.tile(np.exp(-1j * th), s.size)
    cost = np.zeros(r + 1)
    cost[-1] = 1.0
    bounds = [(None, None)] * r + [(0.0, None)]
    db = np.zeros(r)
    for _ in range(200):
        A = (dirs[:, None] * T[pts, :]).real
        rhs = (dirs * g[pts]).real
        A_ub = np.hstack([A, -np.ones((A.shape[0], 1))])
        res = linprog(cost, A_ub=A_ub, b_ub=rhs, bounds=bounds, method="highs")
        if res.status != 0:
            raise RuntimeError("minimax LP failed: " + str(res.message))
        db, delta = res.x[:r], res.x[r]
        e = T @ db - g
        ae = np.abs(e)
        viol = np.nonzero(ae > delta * (1.0 + _CUT_TOL))[0]
        if viol.size == 0:
            break
        pts = np.concatenate([pts, viol])
        dirs = np.concatenate([dirs, np.conj(e[viol]) / ae[viol]])
    w = _to_monomial(b0 + scale * db, xi, r)
    return w, uniform_error(w, xi)


def _to_monomial(b: np.ndarray, xi: float, r: int) -> np.ndarray:
    """sum_j i^j b_j T_j(x / xi)  ->  monomial coefficients in x."""
    c = b * (1j ** np.arange(r))
    d = _cheb.cheb2poly(c)
    d = np.concatenate([d, np.zeros(r - d.size, dtype=complex)]) if d.size < r else d[:r]
    return (d / xi ** np.arange(r)).astype(np.complex128)


def uniform_error(w: np.ndarray, xi: float) -> float:
    """max_{|x| <= xi} |sum_j w_j x^j - e^{i pi x}| on a dense grid (both grids)."""
    x = np.concatenate([xi * _lobatto(_CHECK_GRID), np.linspace(-xi, xi, _CHECK_GRID)])
    p = np.polynomial.polynomial.polyval(x, w)
    return float(np.abs(p - np.exp(1j * np.pi * x)).max())


@functools.lru_cache(maxsize=None)
def scope(eps: float, r: int) -> float:
    """xi(eps, r): the largest xi whose best degree-(r-1) error is <= eps.

    The best error grows monotonically with xi, roughly like xi^r, so
    xi(eps, r) is the root of g(u) = log err(e^u) - log eps, nearly linear in
    u = log xi with slope r. Newton steps with slope r bracket the root, then
    the Illinois variant of regula falsi closes the bracket to a relative
    width of 1e-7; the lower end (error <= eps) is returned.
    """
    def g(u):
        return math.log(best_approximation(math.exp(u), r)[1]) - math.log(eps)

    u = math.log(0.5)
    gu = g(u)
    lo = hi = None  # (u, g) with g <= 0 and g > 0
    for _ in range(80):
        if gu <= 0.0:
            lo = (u, gu)
        else:
            hi = (u, gu)
        if lo is None or hi is None:
            step = max(min(-gu / r, math.log(4.0)), -math.log(4.0))
            u = u + step
            if u > math.log(64.0):
                raise ValueError("scope beyond 64: eps too large for this r")
            if u < math.log(1e-9):
                raise ValueError("eps below the reachable accuracy for this r")
            gu = g(u)
            continue
        break
    side = 0
    for _ in range(80):
        if hi[0] - lo[0] < 1e-7:
            break
        u = lo[0] - lo[1] * (hi[0] - lo[0]) / (hi[1] - lo[1])
        gu = g(u)
        if gu <= 0.0:
            lo = (u, gu)
            if side == -1:
                hi = (hi[0], 0.5 * hi[1])
            side = -1
        else:
            hi = (u, gu)
            if side == 1:
                lo = (lo[0], 0.5 * lo[1])
            side = 1
    return math.exp(lo[0])


def coefficients(eps: float, r: int) -> tuple[float, np.ndarray]:
    """(xi(eps, r), w_{eps, r, .}) -- the precomputed pair of Section 3.1.1."""
    xi = scope(eps, r)
    w, _ = best_approximation(xi, r)
    return xi, w


def choose_r(eps: float, ratio: float, r_max: int = 40) -> int:
    """r = min{ r : xi(eps, r) >= ratio }, ratio = m~ / p (the choice of r in Algorithm 1).

    Since the best error grows with xi, xi(eps, r) >= ratio exactly when the
    best approximation on |x| <= ratio already meets eps.
    """
    for r in range(1, r_max + 1):
        if best_approximation(float(ratio), r)[1] <= eps:
            return r
    raise ValueError("no r <= r_max reaches eps")


def freqs(M: int) -> np.ndarray:
    """Kept frequencies t = -M/2, ..., M/2 - 1 (output row t + M/2)."""
    if M % 2:
        raise ValueError("M must be even")
    return np.arange(-(M // 2), M // 2)


def plan_1d(n: int, M: int, p: int, eps: float = 1e-7, r: int | None = None) -> dict:
    """Algorithm 1: the 1-D offline tables B (q x r) and W (M x r)."""
    if n % p:
        raise ValueError("p must divide n")
    q = n // p
    if r is None:
        r = choose_r(eps, (M / 2) / p)
    xi, w = coefficients(eps, r)
    j = np.arange(r)
    x = 1.0 - 2.0 * np.arange(q) / q
    B = w[None, :] * x[:, None] ** j[None, :]
    t = freqs(M)
    W = (t[:, None] / p) ** j[None, :] * np.exp(-1j * np.pi * t / p)[:, None]
    return dict(n=n, M=M, p=p, q=q, r=r, xi=xi, w=w, B=B, W=W, t=t, eps=eps)


def plan_2d(n1: int, n2: int, M1: int, M2: int, p1: int, p2: int,
            eps: float = 1e-7, r1: int | None = None, r2: int | None = None) -> tuple[dict, dict]:
    """Algorithm 4: one Algorithm-1 factor per axis; W is their outer product."""
    return plan_1d(n1, M1, p1, eps, r1), plan_1d(n2, M2, p2, eps, r2)
