"""FP64 CPU oracle for the action of the matrix exponential on a block of
vectors by Leja-point interpolation: the `expleja` step of the paper's
low-rank algorithms (§3: e^{hA} L for skinny L, Alg. 1-2), here with a sparse A.

TEST INFRASTRUCTURE ONLY (see ``dme_oracle``).

Method (Newton interpolation at Leja points, as in the works the paper cites
for `expleja`; written from the method's definition):

* Spectral interval.  Gershgorin: every eigenvalue of A lies in a disc centred
  at a_ii of radius R_i = sum_{j != i} |a_ij|, so its real part lies in
  [a, b] = [min_i (a_ii - R_i), max_i (a_ii + R_i)] and |Im| <= max_i R_i.
  With c = (a + b) / 2 and g = (b - a) / 4 the map A = c I + g X sends the
  interval to [-2, 2].
* Leja points on [-2, 2]: x_0 = 2, x_k = argmax_{x in [-2, 2]} prod_{i<k} |x - x_i|
  (maximised over a fine uniform grid; the first ones are 2, -2, 0, ...).
* Over a substep t (t = tau / s), exp(t A) v = e^{t c} exp(t g X) v, and
  exp(t g x) is interpolated at the Leja points: with divided differences
  d_k = f[x_0, ..., x_k] of f(x) = exp(t g x), p(X) v = sum_k d_k w_k with
  w_0 = v, w_{k+1} = (X - x_k I) w_k.  The divided differences are the first
  column of f(Z) = exp(t g Z) with Z lower bidiagonal (x_k on the diagonal,
  ones below; Opitz's theorem), evaluated by this oracle's own Pade exponential.
* s is the smallest number of substeps with t g <= RHO_MAX; the series stops
  when the last two terms |d_k| ||w_k|| are below tol times the sum's norm.

Readings where the paper is silent (its reference implementation is not
described): RHO_MAX = 4, at most 80 terms per substep, tol = 1e-15, a grid of
20001 points for the Leja points.
"""
from __future__ import annotations

import math

import numpy as np

from .dme_oracle import expm

__all__ = ["leja_points", "divided_differences_exp", "gershgorin_interval", "leja_action", "RHO_MAX",
           "LEJA_MAX_TERMS"]

RHO_MAX = 4.0
LEJA_MAX_TERMS = 80


def leja_points(m: int, grid: int = 20001) -> np.ndarray:
    """The first m Leja points of [-2, 2] starting at 2 (greedy maximisation of
    the product of distances over a uniform grid; ties go to the first grid
    point)."""
    xs = np.linspace(-2.0, 2.0, grid)
    pts = [2.0]
    with np.errstate(divide="ignore"):
        logprod = np.log(np.abs(xs - 2.0))
    for _ in range(1, m):
        k = int(np.argmax(logprod))
        pts.append(float(xs[k]))
        with np.errstate(divide="ignore"):
            logprod = logprod + np.log(np.abs(xs - xs[k]))
    return np.array(pts)


def divided_differences_exp(x: np.ndarray, scale: float = 1.0) -> np.ndarray:
    """f[x_0], f[x_0, x_1], ..., f[x_0..x_{m-1}] for f(x) = exp(scale x): the
    first column of f(Z) = exp(scale Z), Z lower bidiagonal with x on the
    diagonal and ones below it (Opitz)."""
    m = len(x)
    Z = np.diag(np.asarray(x, dtype=np.float64)) + np.diag(np.ones(m - 1), -1)
    return expm(scale * Z)[:, 0].copy()


def gershgorin_interval(A):
    """[a, b] containing the real parts of A's eigenvalues (Gershgorin), for a
    dense array or a scipy sparse matrix."""
    if hasattr(A, "tocsr"):
        A = A.tocsr()
        d = A.diagonal()
        R = np.asarray(abs(A).sum(axis=1)).ravel() - np.abs(d)
    else:
        A = np.asarray(A, dtype=np.float64)
        d = np.diag(A)
        R = np.abs(A).sum(axis=1) - np.abs(d)
    return float(np.min(d - R)), float(np.max(d + R))


def leja_action(A, V, tau: float, tol: float = 1e-15, interval=None):
    """exp(tau A) V for a dense or sparse A (n x n) and a block V (n x r)."""
    V = np.array(V, dtype=np.float64, copy=True)
    if V.ndim == 1:
        V = V[:, None]
    a, b = interval if interval is not None else gershgorin_interval(A)
    c = 0.5 * (a + b)
    g = 0.25 * (b - a)
    if g <= 0.0:                               # A = c I
        return math.exp(tau * c) * V
    s = max(1, int(math.ceil(tau * g / RHO_MAX)))
    t = tau / s
    xi = leja_points(LEJA_MAX_TERMS)
    dd = divided_differences_exp(xi, t * g)
    scale = math.exp(t * c)

    def Xmul(W):                               # (A - c I) W / g
        return (A @ W - c * W) / g

    for _ in range(s):
        P = dd[0] * V
        W = V
        small = 0
        for k in range(1, LEJA_MAX_TERMS):
            W = Xmul(W) - xi[k - 1] * W
            term = dd[k] * W
            P = P + term
            if np.linalg.norm(term) <= tol * np.linalg.norm(P):
                small += 1
                if small == 2:
                    break
            else:
                small = 0
        V = scale * P
    return V
