"""Error metrics that pin the CPU oracle to things other than itself: closed
forms, published tables, library routines (scipy, called, not retyped) and
brute force.  Each takes the oracle module so the planted-mistake tests can
run the same pin against a deliberately broken copy."""
from __future__ import annotations

import math

import numpy as np
import scipy.integrate as si
import scipy.linalg as sla

import dme_workloads as W

# Higham (2005), Alg. 2.3: the [13/13] numerator coefficients normalised to b_13 = 1.
HIGHAM_B13 = [64764752532480000, 32382376266240000, 7771770303897600, 1187353796428800,
              129060195264000, 10559470521600, 670442572800, 33522128640, 1323241920,
              40840800, 960960, 16380, 182, 1]


def pade_table_error(orc) -> float:
    c = orc.pade13_coefficients()
    return max(abs(c[j] / c[13] - HIGHAM_B13[j]) / HIGHAM_B13[j] for j in range(14))


def expm_scipy_error(orc, seed=0, n=12, scales=(1e-3, 0.3, 3.0, 40.0, 900.0)) -> float:
    """Max relative error of orc.expm against scipy.linalg.expm over random
    matrices whose 1-norms span s = 0 .. about 8 squarings."""
    rng = np.random.default_rng(seed)
    worst = 0.0
    for sc in scales:
        M = rng.standard_normal((n, n))
        M *= sc / np.abs(M).sum(axis=0).max()
        ref = sla.expm(M)
        worst = max(worst, np.linalg.norm(orc.expm(M) - ref) / np.linalg.norm(ref))
    return worst


def laplacian_eigen(nx: int):
    """Closed-form eigenpairs of the 5-point Dirichlet Laplacian: sine
    products V = V1 (x) V1, V1[i,k] = sqrt(2/(nx+1)) sin(k pi i dx), and
    lambda = lambda_k + lambda_l with lambda_k = (2/dx^2)(cos(k pi dx) - 1)."""
    dx = 1.0 / (nx + 1)
    idx = np.arange(1, nx + 1)
    V1 = math.sqrt(2.0 * dx) * np.sin(np.pi * np.outer(idx, idx) * dx)
    lam1 = (2.0 / dx ** 2) * (np.cos(idx * np.pi * dx) - 1.0)
    V = np.kron(V1, V1)
    lam = (lam1[:, None] + lam1[None, :]).ravel()
    return V, lam


def dle_exact_symmetric(V, lam, Q, P0, t):
    """Exact DLE solution for A = V diag(lam) V^T, V orthogonal (Eq. full in
    the eigenbasis): P~_ij = P0~_ij e^{(l_i+l_j)t} + Q~_ij (e^{(l_i+l_j)t} - 1)/(l_i+l_j)."""
    L = lam[:, None] + lam[None, :]
    Qt = V.T @ Q @ V
    Pt = V.T @ P0 @ V
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = np.where(np.abs(L) > 0, np.expm1(L * t) / L, t)
    return V @ (Pt * np.exp(L * t) + Qt * phi) @ V.T


def van_loan_diag_error(orc, seed=1, n=7, tau=0.37) -> float:
    """Diagonal A: E = diag(e^{a_i tau}), W_ij = Q_ij (e^{(a_i+a_j)tau}-1)/(a_i+a_j)."""
    rng = np.random.default_rng(seed)
    a = -rng.uniform(0.1, 5.0, n)
    a[0] = 0.8                         # one unstable mode, and a pair summing to 0
    a[1] = -0.8
    G = rng.standard_normal((3, n))
    Q = G.T @ G
    E, Wm = orc.van_loan(np.diag(a), Q, tau)
    L = a[:, None] + a[None, :]
    with np.errstate(divide="ignore", invalid="ignore"):
        phi = np.where(np.abs(L) > 1e-14, np.expm1(L * tau) / L, tau)
    We = Q * phi
    Ee = np.diag(np.exp(a * tau))
    return max(np.linalg.norm(E - Ee) / np.linalg.norm(Ee), np.linalg.norm(Wm - We) / np.linalg.norm(We))


def van_loan_stiff_diag_error(orc, seed=13, n=9, tau=0.5) -> float:
    """Stiff diagonal A (tau a_i down to -400): the closed form of
    van_loan_diag_error, where e^{-tau A^T} would reach e^{400}."""
    rng = np.random.default_rng(seed)
    a = -rng.uniform(1.0, 800.0, n)
    G = rng.uniform(0.0, 1.0, (3, n))
    Q = G.T @ G
    E, Wm = orc.van_loan(np.diag(a), Q, tau)
    L = a[:, None] + a[None, :]
    We = Q * np.expm1(L * tau) / L
    Ee = np.diag(np.exp(a * tau))
    return max(np.linalg.norm(E - Ee) / np.linalg.norm(Ee), np.linalg.norm(Wm - We) / np.linalg.norm(We))


def van_loan_lyapunov_error(orc, nx=10, tau=1.0 / 16, seed=14) -> float:
    """Differentiating the integrand of Eq. full: A^T W + W A = E^T Q E - Q.
    W from scipy.linalg.solve_continuous_lyapunov (Bartels-Stewart) on a stiff
    non-normal convection-diffusion A (tau ||A||_1 ~ 60)."""
    A = W.convection_diffusion_2d(nx)
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, (3, A.shape[0]))
    Q = C.T @ C
    E, Wm = orc.van_loan(A, Q, tau)
    Wl = sla.solve_continuous_lyapunov(A.T, E.T @ Q @ E - Q)
    Ee = sla.expm(tau * A)
    return max(np.linalg.norm(Wm - Wl) / np.linalg.norm(Wl), np.linalg.norm(E - Ee) / np.linalg.norm(Ee))


def van_loan_quadrature_error(orc, seed=2, n=6, tau=0.5) -> float:
    """Non-normal A: W against 40-point Gauss-Legendre quadrature of
    int_0^tau e^{sA^T} Q e^{sA} ds, each e^{sA} from scipy.linalg.expm."""
    rng = np.random.default_rng(seed)
    A = rng.standard_normal((n, n)) - 2.0 * np.eye(n)
    G = rng.standard_normal((2, n))
    Q = G.T @ G
    E, Wm = orc.van_loan(A, Q, tau)
    x, w = np.polynomial.legendre.leggauss(40)
    s = 0.5 * tau * (x + 1.0)
    Wq = sum(0.5 * tau * wk * (sla.expm(sk * A).T @ Q @ sla.expm(sk * A)) for sk, wk in zip(s, w))
    Ee = sla.expm(tau * A)
    return max(np.linalg.norm(Wm - Wq) / np.linalg.norm(Wq), np.linalg.norm(E - Ee) / np.linalg.norm(Ee))


def ode_reference(A, Q, P0, T, BRB=None, S=None, rtol=1e-13, atol=1e-15):
    """P(T) of dP/dt = A^T P + P A + Q - P BRB P + S P S^T by scipy's DOP853 on
    vec(P) (the vectorised reference of §5.2, with an explicit RK in place of ode15s)."""
    n = A.shape[0]

    def rhs(_t, y):
        P = y.reshape(n, n)
        F = A.T @ P + P @ A + Q
        if BRB is not None:
            F = F - P @ BRB @ P
        if S is not None:
            F = F + S @ P @ S.T
        return F.ravel()

    sol = si.solve_ivp(rhs, (0.0, T), np.asarray(P0, float).ravel(), method="DOP853", rtol=rtol, atol=atol)
    assert sol.success, sol.message
    return sol.y[:, -1].reshape(n, n)


def scalar_dre_exact(a, b, q, r, t):
    """p(t) for p' = 2 a p + q - (b^2/r) p^2, p(0) = 0:
    p = q tanh(beta t) / (beta - a tanh(beta t)), beta = sqrt(a^2 + q b^2 / r)."""
    beta = math.sqrt(a * a + q * b * b / r)
    th = math.tanh(beta * t)
    return q * th / (beta - a * th)


def scalar_dre_errors(orc, scheme, comp, ks=(3, 4, 5, 6), a=-1.0, b=1.0, q=2.0, r=1.0, T=1.0):
    A = np.array([[a]])
    Q = np.array([[q]])
    B = np.array([[b]])
    R = np.array([[r]])
    exact = scalar_dre_exact(a, b, q, r, T)
    errs = []
    for k in ks:
        P = orc.solve(A, Q, np.zeros((1, 1)), T, 2 ** k, comp, W.SCHEMES[scheme], B=B, R=R)
        errs.append(abs(P[0, 0] - exact) / abs(exact))
    return errs


def observed_orders(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


def small_dre(seed=3, n=5, m=2, p=2, with_S=False, rscale=1.0):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n)) / math.sqrt(n)
    A = M - (np.abs(M).sum(axis=0).max() * 0.5 + 0.5) * np.eye(n)
    B = rng.standard_normal((n, m))
    C = rng.uniform(0.0, 1.0, (p, n))
    S = 0.5 * rng.standard_normal((n, n)) / math.sqrt(n) if with_S else None
    R = rscale * np.eye(m)
    return A, C.T @ C, B, R, S


def scheme_errors_vs_ode(orc, scheme, comp, ks=(3, 4, 5), seed=3, with_S=False, T=1.0, rscale=1.0):
    A, Q, B, R, S = small_dre(seed=seed, with_S=with_S, rscale=rscale)
    flows = W.SCHEMES[scheme]
    uses_B = "F3" in flows
    BRB = B @ np.linalg.solve(R, B.T) if uses_B else None
    n = A.shape[0]
    ref = ode_reference(A, Q, np.zeros((n, n)), T, BRB=BRB, S=S if "F4" in flows else None)
    errs = []
    for k in ks:
        P = orc.solve(A, Q, np.zeros((n, n)), T, 2 ** k, comp, flows,
                      B=B if uses_B else None, R=R if uses_B else None,
                      S=S if "F4" in flows else None)
        errs.append(orc.rel_fro(P, ref))
    return errs


def t12_vs_ode_error(orc, nx=3, tau=0.05, seed=4) -> float:
    """T_12 is the exact DLE flow: one application on a non-symmetric
    (convection-diffusion) A from a random PSD state against the ODE."""
    A = W.convection_diffusion_2d(nx)
    n = A.shape[0]
    rng = np.random.default_rng(seed)
    C = rng.uniform(0, 1, (2, n))
    Q = C.T @ C
    P0 = W.random_psd(n, seed)
    E, Wm = orc.van_loan(A, Q, tau)
    P = orc.flow_T12(P0, E, Wm)
    ref = ode_reference(A, Q, P0, tau)
    return orc.rel_fro(P, ref)


def t3_closed_form_scalar_error(orc) -> float:
    """Scalar T_3: p / (1 + tau (b^2/r) p)."""
    worst = 0.0
    for p, b, r, tau in [(0.7, 1.3, 2.0, 0.4), (5.0, 0.2, 1e-3, 0.01), (1e-3, 3.0, 1.0, 2.0)]:
        got = orc.flow_T3(np.array([[p]]), np.array([[b * b / r]]), tau)[0, 0]
        exact = p / (1.0 + tau * (b * b / r) * p)
        worst = max(worst, abs(got - exact) / abs(exact))
    return worst


def t3_vs_ode_error(orc, seed=5, n=6, m=3, tau=0.3) -> float:
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, m))
    BRB = B @ B.T
    P0 = W.random_psd(n, seed)
    ref = ode_reference(np.zeros((n, n)), np.zeros((n, n)), P0, tau, BRB=BRB)
    return orc.rel_fro(orc.flow_T3(P0, BRB, tau), ref)


def t4_local_errors(orc, rule, taus=(0.2, 0.1, 0.05), seed=6, n=5):
    """T_4 against the exact flow of dP/dt = S P S^T, vec(P(t)) = expm(t S(x)S) vec(P0)
    (scipy expm on the n^2 x n^2 Kronecker operator)."""
    rng = np.random.default_rng(seed)
    S = rng.standard_normal((n, n)) / math.sqrt(n)
    P0 = W.random_psd(n, seed)
    K = np.kron(S, S)
    errs = []
    for tau in taus:
        exact = (sla.expm(tau * K) @ P0.ravel()).reshape(n, n)
        errs.append(orc.rel_fro(orc.flow_T4(P0, S, tau, rule), exact))
    return errs


def mass_ode_reference(M, A, Q, P0, T, BRB=None, rtol=1e-13, atol=1e-15):
    """P(T) of the generalised form M^T P' M = A^T P M + M^T P A + Q - M^T P BRB P M
    (Example 4, before any cancellation), vec(P) with DOP853; P' is obtained
    from the right-hand side by two solves with M^T and M."""
    n = A.shape[0]

    def rhs(_t, y):
        P = y.reshape(n, n)
        F = A.T @ P @ M + M.T @ P @ A + Q
        if BRB is not None:
            F = F - M.T @ P @ BRB @ P @ M
        return np.linalg.solve(M.T, np.linalg.solve(M.T, F.T).T).ravel()

    sol = si.solve_ivp(rhs, (0.0, T), np.asarray(P0, float).ravel(), method="DOP853", rtol=rtol, atol=atol)
    assert sol.success, sol.message
    return sol.y[:, -1].reshape(n, n)


def dle_exact_apply_stencil_laplacian(nx, c, t, X, chunk=1024):
    """P(t) X for the DLE with A = the unscaled 5-point Dirichlet stencil on an
    nx x nx grid (x index fastest; eigenvalues 2cos(k pi h) + 2cos(l pi h) - 4,
    h = 1/(nx+1)), Q = c c^T and P0 = 0, without forming P: in the sine basis
    V (the orthonormal DST-I in each direction), P = V (q q^T o Phi) V^T with
    q = V^T c and Phi_ij = expm1((l_i + l_j) t) / (l_i + l_j), applied in row
    chunks of Phi."""
    import scipy.fft as sf
    n = nx * nx
    h = 1.0 / (nx + 1)
    k = np.arange(1, nx + 1)
    l1 = 2.0 * np.cos(k * np.pi * h) - 2.0
    lam = (l1[:, None] + l1[None, :]).ravel()        # index (iy, ix) -> iy * nx + ix

    def vt(v):
        return sf.dstn(v.reshape(nx, nx), type=1, norm="ortho").ravel()

    q = vt(np.asarray(c, dtype=np.float64))
    X = np.atleast_2d(np.asarray(X, dtype=np.float64).T).T
    out = np.empty_like(X)
    for j in range(X.shape[1]):
        y = q * vt(X[:, j])
        z = np.empty(n)
        for i0 in range(0, n, chunk):
            L = lam[i0:i0 + chunk, None] + lam[None, :]
            with np.errstate(divide="ignore", invalid="ignore"):
                phi = np.where(np.abs(L) > 0, np.expm1(L * t) / L, t)
            z[i0:i0 + chunk] = phi @ y
        out[:, j] = vt(q * z)      # V is symmetric: V = V^T
    return out
