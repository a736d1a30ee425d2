"""The CPU oracle against what the paper and the mathematics fix: closed
forms, published coefficient tables, library routines and brute force.
(The paper prints no worked-example values: its error figures are absent.)"""
import math

import numpy as np
import pytest
import scipy.linalg as sla

import dme_workloads as W
import oracle as O
import pins


# ---- exponential and Van Loan integral (plan step) -------------------------------

def test_pade13_coefficients_match_published_table():
    assert pins.pade_table_error(O) < 1e-15


def test_expm_matches_scipy_over_scaling_range():
    assert pins.expm_scipy_error(O) < 1e-13


def test_expm_special_cases():
    d = np.array([-3.0, 0.0, 1.5, 7.0])
    assert np.allclose(O.expm(np.diag(d)), np.diag(np.exp(d)), rtol=1e-14, atol=0)
    # strictly upper triangular (nilpotent): the Taylor series terminates
    rng = np.random.default_rng(0)
    N = np.triu(rng.standard_normal((5, 5)), 1) * 3.0
    taylor = sum(np.linalg.matrix_power(N, k) / math.factorial(k) for k in range(5))
    assert np.linalg.norm(O.expm(N) - taylor) / np.linalg.norm(taylor) < 1e-13
    # e^M e^{-M} = I and e^{2M} = (e^M)^2
    M = rng.standard_normal((6, 6)) * 2.0
    assert np.linalg.norm(O.expm(M) @ O.expm(-M) - np.eye(6)) < 1e-11
    assert np.linalg.norm(O.expm(2 * M) - O.expm(M) @ O.expm(M)) / np.linalg.norm(O.expm(2 * M)) < 1e-12
    assert O.expm(np.zeros((0, 0))).shape == (0, 0)


def test_van_loan_diagonal_closed_form():
    assert pins.van_loan_diag_error(O) < 1e-14


def test_van_loan_stiff_diagonal_closed_form():
    assert pins.van_loan_stiff_diag_error(O) < 1e-13


def test_van_loan_stiff_nonnormal_lyapunov_identity():
    assert pins.van_loan_lyapunov_error(O) < 1e-11


def test_van_loan_against_quadrature_nonnormal():
    assert pins.van_loan_quadrature_error(O) < 1e-13


def test_van_loan_semigroup():
    """E_{2t} = E_t^2 and W_{2t} = W_t + E_t^T W_t E_t (Eq. full at 2t)."""
    A = W.convection_diffusion_2d(4)
    rng = np.random.default_rng(7)
    C = rng.uniform(0, 1, (3, 16))
    Q = C.T @ C
    E1, W1 = O.van_loan(A, Q, 0.01)
    E2, W2 = O.van_loan(A, Q, 0.02)
    assert np.linalg.norm(E1 @ E1 - E2) / np.linalg.norm(E2) < 1e-13
    assert np.linalg.norm(W1 + E1.T @ W1 @ E1 - W2) / np.linalg.norm(W2) < 1e-13


# ---- sub-flows --------------------------------------------------------------------

def test_T12_is_exact_dle_flow_nonsymmetric_A():
    assert pins.t12_vs_ode_error(O) < 1e-11


def test_T1_T2_are_exact_subflows():
    A = W.convection_diffusion_2d(3)
    n = A.shape[0]
    P0 = W.random_psd(n, 1)
    tau = 0.03
    E, _ = O.van_loan(A, np.zeros((n, n)), tau)
    ref = pins.ode_reference(A, np.zeros((n, n)), P0, tau)
    assert O.rel_fro(O.flow_T1(P0, E), ref) < 1e-11
    Q = W.random_psd(n, 2)
    assert np.allclose(O.flow_T2(P0, Q, tau), P0 + tau * Q, rtol=1e-15)


def test_T3_scalar_closed_form():
    assert pins.t3_closed_form_scalar_error(O) < 1e-15


def test_T3_against_ode():
    assert pins.t3_vs_ode_error(O) < 1e-11


def test_T3_equals_woodbury_form():
    """(I + t P B R^-1 B^T)^-1 P = P - t P Bt (I + t Bt^T P Bt)^-1 Bt^T P, Bt = B L^-T, R = L L^T."""
    rng = np.random.default_rng(8)
    n, m = 9, 3
    P = W.random_psd(n, 8)
    B = rng.standard_normal((n, m))
    G = rng.standard_normal((m, m))
    R = G @ G.T + m * np.eye(m)
    L = np.linalg.cholesky(R)
    Bt = np.linalg.solve(L, B.T).T
    tau = 0.7
    Z = P @ Bt
    wood = P - tau * Z @ np.linalg.solve(np.eye(m) + tau * Bt.T @ Z, Z.T)
    got = O.flow_T3(P, B @ np.linalg.solve(R, B.T), tau)
    assert O.rel_fro(got, wood) < 1e-13


def test_T3_semigroup():
    rng = np.random.default_rng(9)
    n = 7
    B = rng.standard_normal((n, 2))
    BRB = B @ B.T
    P = W.random_psd(n, 9)
    a = O.flow_T3(O.flow_T3(P, BRB, 0.3), BRB, 0.5)
    b = O.flow_T3(P, BRB, 0.8)
    assert O.rel_fro(a, b) < 1e-13


def test_T4_midpoint_third_order_euler_second_order_local():
    em = pins.t4_local_errors(O, "midpoint")
    ee = pins.t4_local_errors(O, "euler")
    for o in pins.observed_orders(em):
        assert 2.6 < o < 3.4
    for o in pins.observed_orders(ee):
        assert 1.7 < o < 2.3


# ---- compositions: closed forms and observed order ---------------------------------

def test_step_sequences():
    assert O.step_sequence("lie", ["F1", "F2", "F3"], 1.0) == [("F1", 1.0), ("F2", 1.0), ("F3", 1.0)]
    assert O.step_sequence("strang", ["F1", "F2"], 1.0) == [("F1", 0.5), ("F2", 1.0), ("F1", 0.5)]
    assert O.step_sequence("strang", ["F12", "F3", "F4"], 1.0) == [
        ("F12", 0.5), ("F3", 0.5), ("F4", 1.0), ("F3", 0.5), ("F12", 0.5)]
    assert O.step_sequence("lie", ["F12"], 0.25) == [("F12", 0.25)]


def test_dle_heat_n256_F12_matches_eigenbasis_closed_form():
    pr = W.dle_heat(16)
    V, lam = pins.laplacian_eigen(16)
    assert np.linalg.norm(pr.A @ V - V * lam) / np.linalg.norm(pr.A) < 1e-13
    exact = pins.dle_exact_symmetric(V, lam, pr.Q, pr.P0, pr.T)
    P = O.solve(pr.A, pr.Q, pr.P0, pr.T, 100, "strang", ["F12"])
    assert O.rel_fro(P, exact) < 1e-12


def test_dle_heat_n256_strang_F1F2_second_order():
    pr = W.dle_heat(16)
    V, lam = pins.laplacian_eigen(16)
    exact = pins.dle_exact_symmetric(V, lam, pr.Q, pr.P0, pr.T)
    errs = [O.rel_fro(O.solve(pr.A, pr.Q, pr.P0, pr.T, N, "strang", ["F1", "F2"]), exact)
            for N in (50, 100, 200)]
    for o in pins.observed_orders(errs):
        assert 1.85 < o < 2.15


@pytest.mark.parametrize("scheme", ["F12F3", "F1F2F3", "F1F3F2"])
def test_scalar_dre_tanh_orders(scheme):
    lie = pins.observed_orders(pins.scalar_dre_errors(O, scheme, "lie"))
    strang = pins.observed_orders(pins.scalar_dre_errors(O, scheme, "strang"))
    assert all(0.85 < o < 1.15 for o in lie), lie
    assert all(1.9 < o < 2.1 for o in strang), strang


def test_scalar_dre_small_R_inverse():
    """R^-1 = 1e-3 (the nonlinear term is weak, §5.2): still order 2."""
    e = pins.scalar_dre_errors(O, "F1F2F3", "strang", r=1e3)
    assert all(1.9 < o < 2.1 for o in pins.observed_orders(e))


@pytest.mark.parametrize("scheme,comp,with_S,lo,hi", [
    ("F12F3", "strang", False, 1.9, 2.1), ("F1F2F3", "strang", False, 1.9, 2.1),
    ("F1F3F2", "strang", False, 1.9, 2.1), ("F12F3", "lie", False, 0.9, 1.15),
    ("F12F4", "strang", True, 1.9, 2.1), ("F1F2F4", "strang", True, 1.9, 2.1),
    ("F1F4F2", "strang", True, 1.9, 2.1), ("F12F3F4", "strang", True, 1.9, 2.1),
    ("F12F4", "lie", True, 0.9, 1.15), ("F1F2F3F4", "strang", True, 1.9, 2.1),
])
def test_matrix_schemes_order_against_ode(scheme, comp, with_S, lo, hi):
    errs = pins.scheme_errors_vs_ode(O, scheme, comp, with_S=with_S)
    assert all(lo < o < hi for o in pins.observed_orders(errs)), errs


def test_two_term_more_accurate_when_nonlinear_term_weak():
    """§5.2: with R^-1 = 1e-3 the two-term F12F3 is clearly more accurate
    than the three-term splittings."""
    e2 = pins.scheme_errors_vs_ode(O, "F12F3", "strang", ks=(4,), rscale=1e3)[0]
    e3 = pins.scheme_errors_vs_ode(O, "F1F2F3", "strang", ks=(4,), rscale=1e3)[0]
    assert e2 * 3 < e3


def test_special_cases_where_splitting_is_exact():
    A = W.convection_diffusion_2d(3)
    n = A.shape[0]
    rng = np.random.default_rng(11)
    C = rng.uniform(0, 1, (2, n))
    Q = C.T @ C
    # B = 0: the Riccati flow is the identity and F12F3 collapses to F12
    P_a = O.solve(A, Q, np.zeros((n, n)), 0.2, 8, "strang", ["F12", "F3"], B=np.zeros((n, 1)))
    P_b = O.solve(A, Q, np.zeros((n, n)), 0.2, 8, "strang", ["F12"])
    assert O.rel_fro(P_a, P_b) < 1e-13
    # A = 0, Q = 0: only the Riccati flow remains, which T3 solves exactly
    B = rng.standard_normal((n, 2))
    P0 = W.random_psd(n, 11)
    P_c = O.solve(np.zeros((n, n)), np.zeros((n, n)), P0, 0.5, 4, "strang", ["F12", "F3"], B=B)
    ref = pins.ode_reference(np.zeros((n, n)), np.zeros((n, n)), P0, 0.5, BRB=B @ B.T)
    assert O.rel_fro(P_c, ref) < 1e-11


def test_invariants_symmetric_psd():
    pr = W.dre_convdiff(nx=6, m=2, p=3)
    P = O.solve(pr.A, pr.Q, pr.P0, pr.T, 16, "strang", ["F12", "F3"], B=pr.B, R=pr.R)
    assert np.array_equal(P, P.T)
    assert np.linalg.eigvalsh(P).min() >= -1e-12 * np.linalg.norm(P)


def test_padded_rows_stay_zero():
    pr = W.gdre_convdiff_padded(nx=4, n_pad=20, m=2, p=2)
    P = O.solve(pr.A, pr.Q, pr.P0, pr.T, 4, "strang", ["F12", "F3", "F4"], B=pr.B, R=pr.R, S=pr.S)
    na = pr.meta["n_active"]
    assert np.all(P[na:, :] == 0) and np.all(P[:, na:] == 0)
    assert np.linalg.norm(P[:na, :na]) > 0


def test_long_horizon_reaches_algebraic_riccati_solution():
    """P(T) -> the stabilising ARE solution A^T X + X A + Q - X B R^-1 B^T X = 0
    (scipy.linalg.solve_continuous_are); the Strang steady state is O(h^2) off."""
    A, Q, B, R, _ = pins.small_dre(seed=12, n=4, m=2)
    X = sla.solve_continuous_are(A, B, Q, R)
    errs = []
    for N in (200, 400):
        P = O.solve(A, Q, np.zeros((4, 4)), 20.0, N, "strang", ["F12", "F3"], B=B, R=R)
        errs.append(O.rel_fro(P, X))
    assert errs[1] < 1e-3
    assert 1.8 < math.log2(errs[0] / errs[1]) < 2.2


def test_large_dre_shape_at_T1_approaches_the_are_solution_at_order_two():
    """The large dense DRE's shape (Laplacian, B n x 8, C 8 x n, P0 = 0, T = 1)
    on an 8 x 8 grid: the exact state at T = 1 is the stabilising ARE solution
    up to e^(-2 * 2 pi^2) ~ 1e-17, so the Strang F12F3 state's distance to it is
    the splitting error, O(h^2): it shrinks about four-fold per halving of h."""
    pr = W.dre_heat_large(nx=8)
    X = sla.solve_continuous_are(pr.A, pr.B, pr.Q, pr.R)
    errs = [O.rel_fro(O.solve(pr.A, pr.Q, pr.P0, pr.T, N, "strang", ["F12", "F3"], B=pr.B, R=pr.R), X)
            for N in (128, 256, 512)]
    assert errs[2] < 1e-3
    for a, b in zip(errs, errs[1:]):
        assert 1.8 < math.log2(a / b) < 2.2


def test_lqr_gain_scalar_steady_state_closes_the_loop():
    """§1: u = -R^-1 B^T P x.  For the scalar DRE at steady state, p = (a + beta)/s
    (s = b^2/r, beta = sqrt(a^2 + q s)), so the closed-loop pole a - b k is -beta."""
    a, b, q, r = 0.7, 1.3, 2.0, 0.5
    beta = math.sqrt(a * a + q * b * b / r)
    p = pins.scalar_dre_exact(a, b, q, r, 40.0)
    k = O.lqr_gain(np.array([[p]]), np.array([[b]]), np.array([[r]]))[0, 0]
    assert abs(k - b * p / r) < 1e-14 * abs(k)
    assert abs((a - b * k) + beta) < 1e-12


def test_lqr_gain_from_long_horizon_stabilises():
    A, Q, B, R, _ = pins.small_dre(seed=21, n=5, m=2)
    A = A - (np.linalg.eigvals(A).real.max() - 0.5) * np.eye(5)    # open loop unstable (max Re = 0.5)
    P = O.solve(A, Q, np.zeros((5, 5)), 15.0, 600, "strang", ["F12", "F3"], B=B, R=R)
    K = O.lqr_gain(P, B, R)
    assert np.linalg.eigvals(A).real.max() > 0
    assert np.linalg.eigvals(A - B @ K).real.max() < 0


def test_mass_transform_identity_and_ode():
    """M = I leaves (A, Q) unchanged; with a finite-element mass matrix, Strang
    F12F3 on (A M^-1, M^-T Q M^-1) converges with order 2 to the ODE solution of
    the untransformed generalised form (which tells A M^-1 from M^-1 A)."""
    pr = W.fe_heat_mass(nx=3, m=2, p=2, T=0.2)
    At, Qt = O.mass_transform(np.eye(pr.n), pr.A, pr.Q)
    assert np.allclose(At, pr.A, rtol=1e-15) and np.allclose(Qt, pr.Q, rtol=1e-15)
    M = pr.meta["M"]
    At, Qt = O.mass_transform(M, pr.A, pr.Q)
    BRB = pr.B @ pr.B.T
    ref = pins.mass_ode_reference(M, pr.A, pr.Q, pr.P0, pr.T, BRB=BRB)
    errs = [O.rel_fro(O.solve(At, Qt, pr.P0, pr.T, N, "strang", ["F12", "F3"], B=pr.B, R=pr.R), ref)
            for N in (32, 64, 128)]
    assert all(1.85 < o < 2.15 for o in pins.observed_orders(errs)), errs
    # the other reading (M^-1 A) solves a different equation
    Aw = np.linalg.solve(M, pr.A)
    wrong = O.solve(Aw, Qt, pr.P0, pr.T, 128, "strang", ["F12", "F3"], B=pr.B, R=pr.R)
    assert O.rel_fro(wrong, ref) > 100 * errs[-1]


# ---------------------------------------------------------------- higher-order (extrapolated Strang)
def test_extrapolation_weights_solve_the_moment_conditions():
    """The weights reproduce constants and cancel the h^2, ..., h^(2q-2) error
    terms: an independent Vandermonde solve of sum_k g_k k^(-2j) = [j == 0]."""
    for q in (1, 2, 3, 4):
        g = np.array(O.extrapolation_weights(q))
        V = np.array([[float(k) ** (-2 * j) for k in range(1, q + 1)] for j in range(q)])
        rhs = np.zeros(q)
        rhs[0] = 1.0
        assert np.allclose(g, np.linalg.solve(V, rhs), rtol=1e-13, atol=1e-13)
    assert O.extrapolation_weights(2) == [-1.0 / 3.0, 4.0 / 3.0]


@pytest.mark.parametrize("q,order", [(1, 2), (2, 4), (3, 6)])
def test_extrapolated_strang_order_on_scalar_dre(q, order):
    A, Q, B, R = (np.array([[v]]) for v in (-1.0, 2.0, 1.0, 1.0))
    exact = pins.scalar_dre_exact(-1.0, 1.0, 2.0, 1.0, 1.0)
    errs = [abs(O.solve_extrapolated(A, Q, np.zeros((1, 1)), 1.0, 2 ** k, q, B=B, R=R)[0, 0] - exact) / exact
            for k in (2, 3, 4)]
    ords = pins.observed_orders(errs)
    assert all(abs(o - order) < 0.25 for o in ords), (errs, ords)


def test_extrapolated_strang_order_on_matrix_dre():
    A, Q, B, R, _ = pins.small_dre(seed=3)
    n = A.shape[0]
    ref = pins.ode_reference(A, Q, np.zeros((n, n)), 1.0, BRB=B @ np.linalg.solve(R, B.T))
    errs = [O.rel_fro(O.solve_extrapolated(A, Q, np.zeros((n, n)), 1.0, 2 ** k, 2, B=B, R=R), ref)
            for k in (2, 3, 4)]
    ords = pins.observed_orders(errs)
    assert all(abs(o - 4.0) < 0.35 for o in ords), (errs, ords)
    with pytest.raises(ValueError):
        O.solve_extrapolated(A, Q, np.zeros((n, n)), 1.0, 2, 2, flows=("F12", "F4"))
