"""Pins of the low-rank (LDL^T) oracle against the dense oracle (itself pinned to
closed forms and library routines), Van Loan's exact integral, and linear
algebra identities.  CPU only."""
import math

import numpy as np
import pytest

import dme_workloads as W
import oracle as O


def _lowrank_state(n=12, r=3, seed=0):
    rng = np.random.default_rng(seed)
    L = rng.standard_normal((n, r))
    d = rng.uniform(0.5, 2.0, r)
    return L, np.diag(d)


def _problem(n=12, m=2, p=2, seed=1):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n)) / math.sqrt(n)
    A = M - (np.abs(M).sum(axis=0).max() + 0.5) * np.eye(n)
    B = rng.standard_normal((n, m))
    C = rng.uniform(0.0, 1.0, (p, n))
    S = 0.4 * rng.standard_normal((n, n)) / math.sqrt(n)
    return A, B, C, S


def test_factor_flows_equal_dense_flows():
    A, B, C, S = _problem()
    L, D = _lowrank_state()
    P = O.ldl_product(L, D)
    tau = 0.3
    E = O.expm(tau * A)
    assert O.rel_fro(O.ldl_product(*O.lr_T1(L, D, tau, A)), O.flow_T1(P, E)) < 1e-13
    Q = C.T @ C
    assert O.rel_fro(O.ldl_product(*O.lr_T2(L, D, C.T, np.eye(2), tau)), O.flow_T2(P, Q, tau)) < 1e-14
    R = np.array([[2.0, 0.3], [0.3, 1.0]])
    BRB = B @ np.linalg.solve(R, B.T)
    assert O.rel_fro(O.ldl_product(*O.lr_T3(L, D, B, R, tau)), O.flow_T3(P, BRB, tau)) < 1e-12
    for rule in ("midpoint", "euler"):
        assert O.rel_fro(O.ldl_product(*O.lr_T4(L, D, S, tau, rule)), O.flow_T4(P, S, tau, rule)) < 1e-13


def test_compress_is_an_eigendecomposition_of_P():
    L, D = _lowrank_state(n=15, r=4)
    Lx = np.hstack([L, L[:, :2] @ np.array([[1.0, 2.0], [0.5, -1.0]]), np.zeros((15, 1))])   # dependent columns
    Dx = np.zeros((7, 7))
    Dx[:4, :4] = D
    Dx[4:6, 4:6] = np.array([[1.0, 0.2], [0.2, 3.0]])
    P = O.ldl_product(Lx, Dx)
    Lc, Dc = O.compress(Lx, Dx, tol=1e-12)
    assert Lc.shape[1] == np.linalg.matrix_rank(P) == 4
    assert O.rel_fro(O.ldl_product(Lc, Dc), P) < 1e-14
    assert np.allclose(Lc.T @ Lc, np.eye(4), atol=1e-13)
    assert np.count_nonzero(Dc - np.diag(np.diag(Dc))) == 0
    ev = np.linalg.eigvalsh(P)
    top = ev[np.argsort(-np.abs(ev))][:4]
    assert np.allclose(np.diag(Dc), top, rtol=1e-12)


def test_compress_truncates_only_below_tolerance():
    L, D = _lowrank_state(n=10, r=3)
    D[2, 2] = 1e-15 * D[0, 0]
    Lq, _ = np.linalg.qr(L)
    Lc, Dc = O.compress(Lq, D, tol=1e-13)
    assert Lc.shape[1] == 2
    assert O.rel_fro(O.ldl_product(Lc, Dc), O.ldl_product(Lq, D)) < 1e-14


def test_gauss_legendre_on_interval_is_exact_for_degree_2q_minus_1():
    for q in (1, 3, 7):
        s, w = O.gauss_legendre(q, 0.37)
        for j in range(2 * q):
            assert abs(np.dot(w, s ** j) - 0.37 ** (j + 1) / (j + 1)) < 1e-15


@pytest.mark.parametrize("tau,q,bound", [(1 / 256, 7, 1e-13), (1 / 16, 16, 1e-10), (1 / 16, 24, 1e-12)])
def test_quadrature_factor_converges_to_van_loan(tau, q, bound):
    pr = W.dre_convdiff(nx=6, m=2, p=3)
    _, Wx = O.van_loan(pr.A, pr.Q, tau)
    LI, DI = O.quadrature_factor(pr.A, pr.C.T, np.eye(3), tau, q)
    assert O.rel_fro(O.ldl_product(LI, DI), Wx) < bound


def test_quadrature_error_falls_with_nodes():
    pr = W.dre_convdiff(nx=6, m=2, p=3)
    _, Wx = O.van_loan(pr.A, pr.Q, 1 / 16)
    errs = [O.rel_fro(O.ldl_product(*O.quadrature_factor(pr.A, pr.C.T, np.eye(3), 1 / 16, q)), Wx)
            for q in (4, 7, 10)]
    assert errs[0] > 10 * errs[1] > 100 * errs[2]


@pytest.mark.parametrize("flows,comp", [(["F1", "F2"], "strang"), (["F1", "F2", "F3"], "strang"),
                                        (["F1", "F3", "F2"], "lie"), (["F1", "F2"], "lie")])
def test_lowrank_schemes_equal_dense_schemes(flows, comp):
    pr = W.dre_convdiff(nx=6, m=2, p=3)
    n = pr.n
    N = 8
    L, D = O.solve_lowrank(pr.A, pr.C, np.zeros((n, 0)), np.zeros((0, 0)), pr.T, N, comp, flows,
                           B=pr.B, R=pr.R, tol=1e-15)
    uses_B = "F3" in flows
    ref = O.solve(pr.A, pr.Q, np.zeros((n, n)), pr.T, N, comp, flows, B=pr.B if uses_B else None,
                  R=pr.R if uses_B else None)
    assert O.rel_fro(O.ldl_product(L, D), ref) < 1e-12


def test_lowrank_generalised_scheme_equals_dense():
    A, B, C, S = _problem(n=10)
    L0, D0 = _lowrank_state(n=10, r=2, seed=4)
    for rule, comp in (("midpoint", "strang"), ("euler", "lie")):
        L, D = O.solve_lowrank(A, C, L0, D0, 0.5, 4, comp, ["F1", "F2", "F4"], S=S, tol=1e-15, t4_rule=rule)
        ref = O.solve(A, C.T @ C, O.ldl_product(L0, D0), 0.5, 4, comp, ["F1", "F2", "F4"], S=S, t4_rule=rule)
        assert O.rel_fro(O.ldl_product(L, D), ref) < 1e-12


def test_lowrank_quadrature_scheme_approaches_dense_t12():
    pr = W.dre_convdiff(nx=6, m=2, p=3)
    n = pr.n
    ref = O.solve(pr.A, pr.Q, np.zeros((n, n)), pr.T, 8, "strang", ["F12", "F3"], B=pr.B, R=pr.R)
    L, D = O.solve_lowrank(pr.A, pr.C, np.zeros((n, 0)), np.zeros((0, 0)), pr.T, 8, "strang", ["F12", "F3"],
                           B=pr.B, R=pr.R, q=24, tol=1e-15)
    assert O.rel_fro(O.ldl_product(L, D), ref) < 1e-10


def test_lowrank_rank_stays_low_on_heat_dle():
    pr = W.dle_heat(nx=12)
    L, D = O.solve_lowrank(pr.A, pr.C, np.zeros((pr.n, 0)), np.zeros((0, 0)), pr.T, 20, "strang", ["F1", "F2"])
    assert L.shape[1] < pr.n // 4
    ref = O.solve(pr.A, pr.Q, np.zeros((pr.n, pr.n)), pr.T, 20, "strang", ["F1", "F2"])
    assert O.rel_fro(O.ldl_product(L, D), ref) < 1e-11


# ---------------------------------------------------------------- planted mistakes (CPU, in the oracle)
def _t4_without_sqrt(L, D, S, tau, rule="midpoint"):
    SL = S @ L
    blocks = [L, tau * SL, (tau / math.sqrt(2.0)) * (S @ SL)]
    r = D.shape[0]
    Dn = np.zeros((3 * r, 3 * r))
    for i in range(3):
        Dn[i * r:(i + 1) * r, i * r:(i + 1) * r] = D
    return np.hstack(blocks), Dn


def _t3_wrong_side(L, D, B, R, tau):
    G = L.T @ B
    K = G @ np.linalg.solve(R, G.T)
    Dn = np.linalg.solve(np.eye(D.shape[0]) + tau * K @ D, D)     # K D instead of D K
    return L, 0.5 * (Dn + Dn.T)


def _compress_without_sigma(L, D, tol=1e-13):
    U, sig, Vt = np.linalg.svd(L, full_matrices=False)
    lam, Y = np.linalg.eigh(Vt @ D @ Vt.T)
    return U @ Y, np.diag(lam)


def _t4_transposed_S(L, D, S, tau, rule="midpoint"):
    St = np.ascontiguousarray(S.T)                                  # S^T L instead of S L
    SL = St @ L
    blocks = [L, math.sqrt(tau) * SL, (tau / math.sqrt(2.0)) * (St @ SL)]
    r = D.shape[0]
    Dn = np.zeros((3 * r, 3 * r))
    for i in range(3):
        Dn[i * r:(i + 1) * r, i * r:(i + 1) * r] = D
    return np.hstack(blocks), Dn


def _t4_s2_of_new_block(L, D, S, tau, rule="midpoint"):
    SL = S @ L
    blocks = [L, math.sqrt(tau) * SL, (tau / math.sqrt(2.0)) * (S @ (math.sqrt(tau) * SL))]   # S^2 of the scaled block
    r = D.shape[0]
    Dn = np.zeros((3 * r, 3 * r))
    for i in range(3):
        Dn[i * r:(i + 1) * r, i * r:(i + 1) * r] = D
    return np.hstack(blocks), Dn


@pytest.mark.parametrize("name,fn", [("lr_T4", _t4_without_sqrt), ("lr_T3", _t3_wrong_side),
                                     ("compress", _compress_without_sigma), ("lr_T4", _t4_transposed_S),
                                     ("lr_T4", _t4_s2_of_new_block)])
def test_pins_catch_planted_lowrank_mistakes(monkeypatch, name, fn):
    import oracle.dme_lowrank as lr
    monkeypatch.setattr(lr, name, fn)
    A, B, C, S = _problem()
    L, D = _lowrank_state()
    P = O.ldl_product(L, D)
    tau = 0.3
    if name == "lr_T4":
        got = O.ldl_product(*lr.lr_T4(L, D, S, tau))
        ref = O.flow_T4(P, S, tau, "midpoint")
    elif name == "lr_T3":
        R = np.array([[2.0, 0.3], [0.3, 1.0]])
        got = O.ldl_product(*lr.lr_T3(L, D, B, R, tau))
        ref = O.flow_T3(P, B @ np.linalg.solve(R, B.T), tau)
    else:
        got = O.ldl_product(*lr.compress(L, D))
        ref = P
    assert O.rel_fro(got, ref) > 1e-6
