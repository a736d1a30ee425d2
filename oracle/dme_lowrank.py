"""FP64 CPU oracle for the low-rank (LDL^T) form of the splitting schemes of
Mena, Pfurtscheller & Stillfjord (arXiv:1805.08990), §2.1-2.3 and Alg. 1-4.

TEST INFRASTRUCTURE ONLY, like ``dme_oracle``: only ``tests/``,
``__graft_entry__.smoke()`` and ``bench.py``'s CPU legs use it; it shares no
code with the CUDA path.

The state is P = L D L^T with L n x r and D r x r symmetric.  Each sub-flow
acts on the factors without forming P:

    T_1(tau):  L <- e^{tau A^T} L                                 (Eq. F_sol_LDL)
    T_2(tau):  L <- [L, L_Q],  D <- blkdiag(D, tau D_Q)           (§2.1), Q = L_Q D_Q L_Q^T
    T_3(tau):  D <- (I + tau D L^T B R^{-1} B^T L)^{-1} D          (§2.2; Alg. 3 prints the
               product without B^T, a misprint: the §2.2 form is used)
    T_4(tau):  midpoint: L <- [L, sqrt(tau) S L, tau/sqrt(2) S^2 L], D <- blkdiag(D, D, D);
               Euler:    L <- [L, sqrt(tau) S L],                   D <- blkdiag(D, D)
               (§2.3, with S^2 L_0 where the text writes S^2 L)
    T_12(tau): L <- [e^{tau A^T} L, L_I], D <- blkdiag(D, D_I), with
               W_tau ~ L_I D_I L_I^T from a quadrature of the integral of Eq. full
               (Alg. 2): L_I = [e^{s_k A^T} L_Q], D_I = blkdiag(w_k D_Q), compressed.

Column compression (Alg. 1, 2, 4; §3): a reduced SVD L = U Sigma V^T, then the
diagonalisation of the small system Sigma V^T D V Sigma = Y Lambda Y^T, and
L <- U Y, D <- Lambda; eigenvalues with |lambda| <= tol * max |lambda| are
dropped.  It is applied after every sub-flow that appends columns.

Readings where the paper is silent: the quadrature is Gauss-Legendre with q
nodes on [0, tau] (default q = 7); the truncation is relative to the largest
eigenvalue of the compressed system with tol = 1e-13 by default.  e^{s A^T} L
is either the dense exponential of ``dme_oracle.expm`` times L (action
"dense") or, as in the paper, the Leja interpolation of ``dme_leja`` applied to
L with A dense or sparse (action "leja"); the two agree to the interpolation's
tolerance.
"""
from __future__ import annotations

import math

import numpy as np

from .dme_oracle import expm, step_sequence

__all__ = [
    "lr_T1", "lr_T2", "lr_T3", "lr_T4", "compress", "gauss_legendre", "quadrature_factor", "lr_T12",
    "LowRankPlan", "solve_lowrank", "ldl_product",
]


def ldl_product(L, D):
    """P = L D L^T."""
    return L @ D @ L.T


def lr_T1(L, D, tau, A):
    """T_1(tau) on factors: e^{tau A^T} L (Eq. F_sol_LDL)."""
    return expm(tau * np.asarray(A, dtype=np.float64).T) @ L, D


def lr_T2(L, D, LQ, DQ, tau):
    """T_2(tau) on factors: [L, L_Q], blkdiag(D, tau D_Q) (§2.1)."""
    r, p = D.shape[0], DQ.shape[0]
    Dn = np.zeros((r + p, r + p))
    Dn[:r, :r] = D
    Dn[r:, r:] = tau * DQ
    return np.hstack([L, LQ]), Dn


def lr_T3(L, D, B, R, tau):
    """T_3(tau) on factors (§2.2): D <- (I + tau D L^T B R^{-1} B^T L)^{-1} D."""
    G = L.T @ B                                   # r x m
    K = G @ np.linalg.solve(R, G.T)               # L^T B R^{-1} B^T L
    r = D.shape[0]
    Dn = np.linalg.solve(np.eye(r) + tau * D @ K, D)
    return L, 0.5 * (Dn + Dn.T)


def lr_T4(L, D, S, tau, rule="midpoint"):
    """T_4(tau) on factors (§2.3): midpoint [L, sqrt(t) S L, t/sqrt(2) S^2 L] with
    blkdiag(D, D, D); explicit Euler [L, sqrt(t) S L] with blkdiag(D, D)."""
    SL = S @ L
    r = D.shape[0]
    if rule == "euler":
        blocks = [L, math.sqrt(tau) * SL]
    else:
        blocks = [L, math.sqrt(tau) * SL, (tau / math.sqrt(2.0)) * (S @ SL)]
    k = len(blocks)
    Dn = np.zeros((k * r, k * r))
    for i in range(k):
        Dn[i * r:(i + 1) * r, i * r:(i + 1) * r] = D
    return np.hstack(blocks), Dn


def compress(L, D, tol=1e-13):
    """Column compression (§3): reduced SVD of L, diagonalisation of the small
    system, truncation of eigenvalues with |lambda| <= tol * max |lambda|.
    Returns (L, D) with D diagonal and L with orthonormal columns."""
    if L.shape[1] == 0:
        return L, D
    U, sig, Vt = np.linalg.svd(L, full_matrices=False)
    M = (sig[:, None] * (Vt @ D @ Vt.T)) * sig[None, :]
    lam, Y = np.linalg.eigh(0.5 * (M + M.T))
    amax = np.max(np.abs(lam)) if lam.size else 0.0
    keep = np.abs(lam) > tol * amax if amax > 0 else np.zeros(lam.shape, dtype=bool)
    order = np.argsort(-np.abs(lam[keep]))
    lam_k = lam[keep][order]
    Y_k = Y[:, keep][:, order]
    return U @ Y_k, np.diag(lam_k)


def gauss_legendre(q, tau):
    """Nodes and weights of the q-point Gauss-Legendre rule on [0, tau]."""
    x, w = np.polynomial.legendre.leggauss(q)
    return 0.5 * tau * (x + 1.0), 0.5 * tau * w


def quadrature_factor(A, LQ, DQ, tau, q=7, tol=1e-13):
    """Alg. 2's integral term: W_tau ~ sum_k w_k e^{s_k A^T} Q e^{s_k A}
    = L_I D_I L_I^T with L_I = [e^{s_k A^T} L_Q], D_I = blkdiag(w_k D_Q), compressed."""
    s, w = gauss_legendre(q, tau)
    At = np.asarray(A, dtype=np.float64).T
    p = DQ.shape[0]
    LI = np.hstack([expm(sk * At) @ LQ for sk in s])
    DI = np.zeros((q * p, q * p))
    for k in range(q):
        DI[k * p:(k + 1) * p, k * p:(k + 1) * p] = w[k] * DQ
    return compress(LI, DI, tol)


def lr_T12(L, D, E, LI, DI):
    """T_12(tau) on factors (Alg. 2): [e^{tau A^T} L, L_I], blkdiag(D, D_I)."""
    r, k = D.shape[0], DI.shape[0]
    Dn = np.zeros((r + k, r + k))
    Dn[:r, :r] = D
    Dn[r:, r:] = DI
    return np.hstack([E.T @ L, LI]), Dn


class LowRankPlan:
    """Problem data (A, Q = C^T C as L_Q = C^T, D_Q = I, B, R, S) and the per-tau
    caches of e^{tau A} and of the quadrature factor of W_tau."""

    def __init__(self, A, C, B=None, R=None, S=None, q=7, tol=1e-13, action="dense"):
        # action "dense": e^{tau A^T} L with the dense exponential; "leja": by
        # Leja interpolation (dme_leja.leja_action), A dense or scipy sparse
        self.action = action
        self.A = A if (action == "leja" and hasattr(A, "tocsr")) else np.asarray(A, dtype=np.float64)
        C = np.asarray(C, dtype=np.float64)
        self.LQ = C.T.copy()
        self.DQ = np.eye(C.shape[0])
        self.B = None if B is None else np.asarray(B, dtype=np.float64)
        self.R = None if R is None else np.asarray(R, dtype=np.float64)
        self.S = None if S is None else (S.tocsr() if hasattr(S, "tocsr") else np.asarray(S, dtype=np.float64))
        self.q, self.tol = q, tol
        self._E, self._W = {}, {}

    def E(self, tau):
        key = float(tau)
        if key not in self._E:
            self._E[key] = expm(key * self.A)
        return self._E[key]

    def expAT(self, tau, L):
        """e^{tau A^T} L (Eq. F_sol_LDL)."""
        if self.action == "leja":
            from .dme_leja import leja_action
            return leja_action(self.A.T, L, tau) if L.shape[1] else L
        return self.E(tau).T @ L

    def W(self, tau):
        key = float(tau)
        if key not in self._W:
            if self.action == "leja":
                s, w = gauss_legendre(self.q, key)
                p = self.DQ.shape[0]
                LI = np.hstack([self.expAT(sk, self.LQ) for sk in s])
                DI = np.zeros((self.q * p, self.q * p))
                for k in range(self.q):
                    DI[k * p:(k + 1) * p, k * p:(k + 1) * p] = w[k] * self.DQ
                self._W[key] = compress(LI, DI, self.tol)
            else:
                self._W[key] = quadrature_factor(self.A, self.LQ, self.DQ, key, self.q, self.tol)
        return self._W[key]

    def apply(self, flow, tau, L, D, t4_rule="midpoint"):
        if flow == "F1":
            return self.expAT(tau, L), D
        if flow == "F2":
            return compress(*lr_T2(L, D, self.LQ, self.DQ, tau), self.tol)
        if flow == "F12":
            LI, DI = self.W(tau)
            r, k = D.shape[0], DI.shape[0]
            Dn = np.zeros((r + k, r + k))
            Dn[:r, :r] = D
            Dn[r:, r:] = DI
            return compress(np.hstack([self.expAT(tau, L), LI]), Dn, self.tol)
        if flow == "F3":
            return lr_T3(L, D, self.B, self.R, tau)
        if flow == "F4":
            return compress(*lr_T4(L, D, self.S, tau, t4_rule), self.tol)
        raise ValueError(flow)

    def step(self, L, D, comp, flows, h, t4_rule=None):
        rule = t4_rule or ("midpoint" if comp == "strang" else "euler")
        for f, tau in step_sequence(comp, flows, h):
            L, D = self.apply(f, tau, L, D, rule)
        return L, D


def solve_lowrank(A, C, L0, D0, T, nsteps, comp="strang", flows=("F1", "F2"), B=None, R=None, S=None,
                  q=7, tol=1e-13, t4_rule=None, plan: LowRankPlan | None = None, action="dense"):
    """(L, D) with L D L^T ~ P(T) after N = nsteps steps of the composition on
    the factors (Alg. 1-4), h = T/N, P_0 = L0 D0 L0^T."""
    plan = plan or LowRankPlan(A, C, B, R, S, q, tol, action)
    L = np.array(L0, dtype=np.float64, copy=True).reshape(A.shape[0], -1)
    D = np.array(D0, dtype=np.float64, copy=True).reshape(L.shape[1], L.shape[1])
    h = T / nsteps
    for _ in range(nsteps):
        L, D = plan.step(L, D, comp, list(flows), h, t4_rule)
    return L, D
