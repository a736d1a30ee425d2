"""FP64 CPU oracle for the dense splitting schemes of Mena, Pfurtscheller &
Stillfjord, "GPU acceleration of splitting schemes applied to differential
matrix equations" (arXiv:1805.08990).

TEST INFRASTRUCTURE ONLY.  Nothing on the product path imports, calls or links
this module: only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU
baseline / reference arm use it.  It shares no code with the CUDA path; its only
common dependency is the seeded input generator module ``dme_workloads``.

Everything here is the plain definition in float64 with numpy: matrix products
are ``@``, linear systems are ``numpy.linalg.solve`` (LAPACK LU with partial
pivoting).  No blocking, fusion or reordering beyond what each definition or
algorithm states.  Notation is the paper's:

    dP/dt = A^T P + P A + Q + G(P),  P(0) = P0                        (§1)
    G = 0 (DLE, Eq. lyap), G(P) = -P B R^{-1} B^T P (DRE, Eq. ricc),
    + S P S^T (generalised forms, Eq. lyapGen and §2.4).

Sub-flows T_k(tau) are the exact (or, for T_4, midpoint/Euler) solution
operators of dP/dt = F_k(P) over [0, tau] (§2):
    T_1(tau) P = e^{tau A^T} P e^{tau A}                              (§2.1)
    T_2(tau) P = P + tau Q                                            (§2.1)
    T_12(tau) P = e^{tau A^T} P e^{tau A} + int_0^tau e^{sA^T} Q e^{sA} ds   (Eq. full)
    T_3(tau) P = (I + tau P B R^{-1} B^T)^{-1} P                      (Eq. nonlinear)
    T_4(tau) P ~ P + tau S (P + tau/2 S P S^T) S^T  (midpoint), or
                 P + tau S P S^T (explicit Euler, enough for Lie)     (§2.3)

Lie / Strang compositions (§2, §3): the operators are listed in the order they
are applied.  Lie "Fa Fb Fc" = T_c(h) T_b(h) T_a(h); Strang "Fa Fb Fc" =
T_a(h/2) T_b(h/2) T_c(h) T_b(h/2) T_a(h/2); two-term Strang "Fa Fb" =
T_a(h/2) T_b(h) T_a(h/2).

The integral term of T_12 is taken from Van Loan's block exponential
(C. Van Loan, "Computing integrals involving the matrix exponential", IEEE
TAC 23(3), 1978): with M = [[-A^T, Q], [0, A]], e^{tau M} = [[F11, F12],
[0, F22]], F22 = e^{tau A} and F22^T F12 = int_0^tau e^{sA^T} Q e^{sA} ds.  The
exponential is Higham's [13/13] Pade scaling-and-squaring (N. J. Higham, "The
scaling and squaring method for the matrix exponential revisited", SIAM J.
Matrix Anal. Appl. 26(4), 2005, Alg. 2.3 restricted to m = 13).

Readings where the paper is silent: the paper approximates the integral by an
unnamed quadrature (§3, Alg. 2); here it is exact to rounding.  The block
exponential is evaluated at a step t with ||t A||_1 <= 1 and doubled to tau
with the semigroup law of Eq. full (see van_loan).  After every sub-flow the
state is symmetrised, P <- (P + P^T)/2.

Every function below is pinned by ``tests/test_oracle_*.py`` against closed
forms, library routines (scipy) or brute force; none is "parity unpinned".
"""
from __future__ import annotations

import math
from fractions import Fraction

import numpy as np

__all__ = [
    "pade13_coefficients", "THETA13", "norm1", "expm", "van_loan",
    "flow_T1", "flow_T2", "flow_T12", "flow_T3", "flow_T4", "symmetrize",
    "step_sequence", "Plan", "solve", "extrapolation_weights", "solve_extrapolated",
    "mass_transform", "lqr_gain", "rel_fro",
]

# theta_13 of Higham (2005), Table 2.3: the largest ||X||_1 for which the
# [13/13] approximant has backward error below the unit roundoff 2^-53.
THETA13 = 5.371920351148152


def pade13_coefficients() -> list[float]:
    """Coefficients c_j of the [m/m] Pade numerator of e^x, m = 13:
    c_j = (2m - j)! m! / ((2m)! j! (m - j)!), p(x) = sum_j c_j x^j and
    q(x) = p(-x) (Higham 2005, Eq. 2.2 and the line after it)."""
    m = 13
    f = math.factorial
    return [float(Fraction(f(2 * m - j) * f(m), f(2 * m) * f(j) * f(m - j))) for j in range(m + 1)]


def norm1(M: np.ndarray) -> float:
    """Matrix 1-norm: maximum absolute column sum."""
    if M.size == 0:
        return 0.0
    return float(np.abs(M).sum(axis=0).max())


def expm(M: np.ndarray) -> np.ndarray:
    """e^M by [13/13] Pade scaling and squaring (Higham 2005, Alg. 2.3 with
    m = 13 only): s = max(0, ceil(log2(||M||_1 / theta_13))), X = M / 2^s,
    r_13(X) = q(X)^{-1} p(X) with p = V + U, q = V - U (U the odd part, V the
    even part, evaluated with X^2, X^4, X^6), then s squarings."""
    M = np.asarray(M, dtype=np.float64)
    n = M.shape[0]
    if n == 0:
        return M.copy()
    c = pade13_coefficients()
    nrm = norm1(M)
    s = 0 if nrm <= THETA13 else int(math.ceil(math.log2(nrm / THETA13)))
    X = M / (2.0 ** s)
    I = np.eye(n)
    X2 = X @ X
    X4 = X2 @ X2
    X6 = X4 @ X2
    U = X @ (X6 @ (c[13] * X6 + c[11] * X4 + c[9] * X2)
             + c[7] * X6 + c[5] * X4 + c[3] * X2 + c[1] * I)
    V = (X6 @ (c[12] * X6 + c[10] * X4 + c[8] * X2)
         + c[6] * X6 + c[4] * X4 + c[2] * X2 + c[0] * I)
    R = np.linalg.solve(V - U, V + U)
    for _ in range(s):
        R = R @ R
    return R


def van_loan(A: np.ndarray, Q: np.ndarray, tau: float):
    """E = e^{tau A} and W = int_0^tau e^{s A^T} Q e^{s A} ds (the integral of
    Eq. full) from the 2n x 2n exponential of t [[-A^T, Q], [0, A]]:
    E_t = F22, W_t = F22^T F12.

    The block exponential is taken at t = tau / 2^j with ||t A||_1 <= 1 and
    brought to tau by the semigroup law of Eq. full, E_{2t} = E_t^2,
    W_{2t} = W_t + E_t^T W_t E_t.  At large tau ||A|| the (1,1) block
    e^{-tau A^T} of a stable A grows like e^{tau ||A||}, and W = F22^T F12 then
    loses every digit to cancellation; at ||t A||_1 <= 1 no block grows."""
    n = A.shape[0]
    nA = norm1(A) * abs(tau)
    j = 0 if nA <= 1.0 else int(math.ceil(math.log2(nA)))
    t = tau / (2.0 ** j)
    M = np.zeros((2 * n, 2 * n))
    M[:n, :n] = -A.T
    M[:n, n:] = Q
    M[n:, n:] = A
    F = expm(t * M)
    E = F[n:, n:].copy()
    W = E.T @ F[:n, n:]
    for _ in range(j):
        W = W + E.T @ W @ E
        E = E @ E
    return E, W


def symmetrize(P: np.ndarray) -> np.ndarray:
    return 0.5 * (P + P.T)


def flow_T1(P, E):
    """T_1(tau) P = e^{tau A^T} P e^{tau A} = E^T P E  (§2.1), E = e^{tau A}."""
    return symmetrize(E.T @ P @ E)


def flow_T2(P, Q, tau):
    """T_2(tau) P = P + tau Q  (§2.1)."""
    return symmetrize(P + tau * Q)


def flow_T12(P, E, W):
    """T_12(tau) P = E^T P E + W, the exact flow of F_12 = A^T P + P A + Q
    (Eq. full with t = tau)."""
    return symmetrize(E.T @ P @ E + W)


def flow_T3(P, BRB, tau):
    """T_3(tau) P = (I + tau P B R^{-1} B^T)^{-1} P, the exact flow of
    F_3 = -P B R^{-1} B^T P (Eq. nonlinear), taken literally as one dense
    n x n solve.  BRB = B R^{-1} B^T."""
    n = P.shape[0]
    return symmetrize(np.linalg.solve(np.eye(n) + tau * (P @ BRB), P))


def flow_T4(P, S, tau, rule="midpoint"):
    """T_4(tau) P for F_4 = S P S^T (§2.3): the midpoint rule
    P + tau S (P + tau/2 S P S^T) S^T, or explicit Euler P + tau S P S^T,
    which suffices for a first-order (Lie) scheme."""
    if rule == "midpoint":
        return symmetrize(P + tau * (S @ (P + 0.5 * tau * (S @ P @ S.T)) @ S.T))
    if rule == "euler":
        return symmetrize(P + tau * (S @ P @ S.T))
    raise ValueError(rule)


def step_sequence(comp: str, flows: list[str], h: float):
    """One step of a composition as (flow, tau) pairs in application order.

    comp = "lie":    [(a, h), (b, h), (c, h)]                  (§2, L_h)
    comp = "strang": [(a, h/2), (b, h/2), (c, h), (b, h/2), (a, h/2)]
                     and [(a, h/2), (b, h), (a, h/2)] for two flows   (§2, S_h)
    A single flow (the unsplit F12 of the DLE) is [(a, h)] for both."""
    if len(flows) == 1:
        return [(flows[0], h)]
    if comp == "lie":
        return [(f, h) for f in flows]
    if comp == "strang":
        half = [(f, 0.5 * h) for f in flows[:-1]]
        return half + [(flows[-1], h)] + half[::-1]
    raise ValueError(comp)


class Plan:
    """Problem data plus the per-tau cache of (E_tau, W_tau): the matrices the
    paper builds once per step size (§4, 'one-time')."""

    def __init__(self, A, Q, B=None, R=None, S=None):
        self.A = np.asarray(A, dtype=np.float64)
        self.Q = np.asarray(Q, dtype=np.float64)
        self.n = self.A.shape[0]
        self.S = None if S is None else np.asarray(S, dtype=np.float64)
        if B is not None:
            B = np.asarray(B, dtype=np.float64)
            R = np.eye(B.shape[1]) if R is None else np.asarray(R, dtype=np.float64)
            self.BRB = B @ np.linalg.solve(R, B.T)      # B R^{-1} B^T
        else:
            self.BRB = None
        self._ew = {}

    def EW(self, tau: float):
        key = float(tau)
        if key not in self._ew:
            self._ew[key] = van_loan(self.A, self.Q, key)
        return self._ew[key]

    def apply(self, flow: str, tau: float, P: np.ndarray, t4_rule: str = "midpoint"):
        if flow == "F1":
            return flow_T1(P, self.EW(tau)[0])
        if flow == "F2":
            return flow_T2(P, self.Q, tau)
        if flow == "F12":
            E, W = self.EW(tau)
            return flow_T12(P, E, W)
        if flow == "F3":
            if self.BRB is None:
                raise ValueError("F3 needs B")
            return flow_T3(P, self.BRB, tau)
        if flow == "F4":
            if self.S is None:
                raise ValueError("F4 needs S")
            return flow_T4(P, self.S, tau, t4_rule)
        raise ValueError(flow)

    def step(self, P, comp, flows, h, t4_rule=None):
        rule = t4_rule or ("midpoint" if comp == "strang" else "euler")
        for f, tau in step_sequence(comp, flows, h):
            P = self.apply(f, tau, P, rule)
        return P


def solve(A, Q, P0, T, nsteps, comp="strang", flows=("F12",), B=None, R=None, S=None,
          t4_rule=None, plan: Plan | None = None):
    """P(T) ~ P_N by N = nsteps steps of the composition, h = T/N (§2:
    P_{k+1} = L_h P_k or S_h P_k, P_0 = P0)."""
    plan = plan or Plan(A, Q, B, R, S)
    h = T / nsteps
    P = np.array(P0, dtype=np.float64, copy=True)
    for _ in range(nsteps):
        P = plan.step(P, comp, list(flows), h, t4_rule)
    return P


def extrapolation_weights(q: int) -> list[float]:
    """Weights gamma_1..gamma_q of the extrapolated Strang scheme of order 2q
    (the higher-order schemes mentioned in §2).  Strang of exact flows is
    symmetric, so its global error expands in even powers of h; combining the
    results of k steps of size h/k, k = 1..q, with weights that reproduce the
    value at x = h^2 -> 0 of every polynomial of degree < q in x = (h/k)^2 is
    the Lagrange basis at 0 on the nodes x_k = 1/k^2:
    gamma_k = prod_{j != k} x_j / (x_j - x_k) = prod_{j != k} k^2 / (k^2 - j^2)."""
    out = []
    for k in range(1, q + 1):
        g = Fraction(1)
        for j in range(1, q + 1):
            if j != k:
                g *= Fraction(k * k, k * k - j * j)
        out.append(float(g))
    return out


def solve_extrapolated(A, Q, P0, T, nsteps, q, flows=("F12", "F3"), B=None, R=None, plan: Plan | None = None):
    """P(T) by N = nsteps steps of the extrapolated Strang scheme of order 2q:
    P_{j+1} = sum_k gamma_k (S_{h/k})^k P_j, h = T/N.  Needs exact sub-flows
    (no F4, whose midpoint rule is not symmetric)."""
    if "F4" in flows:
        raise ValueError("extrapolation needs a symmetric base scheme (no F4)")
    plan = plan or Plan(A, Q, B, R)
    gam = extrapolation_weights(q)
    h = T / nsteps
    P = np.array(P0, dtype=np.float64, copy=True)
    for _ in range(nsteps):
        acc = np.zeros_like(P)
        for k in range(1, q + 1):
            Y = P
            for _ in range(k):
                Y = plan.step(Y, "strang", list(flows), h / k)
            acc = acc + gam[k - 1] * Y
        P = acc
    return P


def mass_transform(M, A, Q):
    """Generalised state space (Example 4, §5.1.4): M^T P' M = A^T P M + M^T P A + Q
    - M^T P B R^-1 B^T P M is, after cancelling M^T and M,
    P' = M^-T A^T P + P A M^-1 + M^-T Q M^-1 - P B R^-1 B^T P: the standard DRE with
    A~ = A M^-1 and Q~ = M^-T Q M^-1 (the displayed equation; its A M^-1 is
    read literally).  Returns (A~, Q~)."""
    M = np.asarray(M, dtype=np.float64)
    At = np.linalg.solve(M.T, np.asarray(A, dtype=np.float64).T).T     # A M^-1
    Y = np.linalg.solve(M.T, np.asarray(Q, dtype=np.float64))          # M^-T Q
    Qt = np.linalg.solve(M.T, Y.T).T                                    # M^-T Q M^-1
    return At, 0.5 * (Qt + Qt.T)


def lqr_gain(P, B, R):
    """K = R^{-1} B^T P: the optimal LQR input is u(t) = -K(T - t) x(t) with
    K built from the DRE solution P (§1)."""
    return np.linalg.solve(np.asarray(R, dtype=np.float64), np.asarray(B, dtype=np.float64).T @ P)


def rel_fro(X, Y) -> float:
    """||X - Y||_F / ||Y||_F (the relative error of §5.2; the norm is a reading)."""
    d = np.linalg.norm(np.asarray(X) - np.asarray(Y))
    r = np.linalg.norm(np.asarray(Y))
    return float(d / r) if r > 0 else float(d)
