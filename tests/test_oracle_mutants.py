"""Planted mistakes in the CPU oracle (on the CPU only): each plausible slip
must be caught by at least one pin, so the pins are known to bite."""
import types

import numpy as np
import pytest

import oracle as O
import oracle.dme_oracle as core
import pins


def mutant(**overrides):
    m = types.ModuleType("oracle_mutant")
    m.__dict__.update({k: getattr(core, k) for k in dir(core) if not k.startswith("__")})
    m.__dict__.update(overrides)
    # Plan / solve look functions up in their module globals: rebind them to the mutant
    src_plan = core.Plan

    class Plan(src_plan):
        def EW(self, tau):
            key = float(tau)
            if key not in self._ew:
                self._ew[key] = m.van_loan(self.A, self.Q, key)
            return self._ew[key]

        def apply(self, flow, tau, P, t4_rule="midpoint"):
            if flow == "F12":
                E, Wm = self.EW(tau)
                return m.flow_T12(P, E, Wm)
            if flow == "F3":
                return m.flow_T3(P, self.BRB, tau)
            if flow == "F1":
                return m.flow_T1(P, self.EW(tau)[0])
            return src_plan.apply(self, flow, tau, P, t4_rule)

        def step(self, P, comp, flows, h, t4_rule=None):
            rule = t4_rule or ("midpoint" if comp == "strang" else "euler")
            for f, tau in m.step_sequence(comp, flows, h):
                P = self.apply(f, tau, P, rule)
            return P

    def solve(A, Q, P0, T, nsteps, comp="strang", flows=("F12",), B=None, R=None, S=None,
              t4_rule=None, plan=None):
        plan = plan or Plan(A, Q, B, R, S)
        P = np.array(P0, dtype=np.float64, copy=True)
        for _ in range(nsteps):
            P = plan.step(P, comp, list(flows), T / nsteps, t4_rule)
        return P

    m.Plan = Plan
    m.solve = solve
    return m


def _vl_missing_E(A, Q, tau):
    n = A.shape[0]
    M = np.zeros((2 * n, 2 * n))
    M[:n, :n] = -A.T
    M[:n, n:] = Q
    M[n:, n:] = A
    F = core.expm(tau * M)
    return F[n:, n:].copy(), F[:n, n:].copy()          # W = F12 (drops F22^T)


def _vl_sign(A, Q, tau):
    n = A.shape[0]
    M = np.zeros((2 * n, 2 * n))
    M[:n, :n] = A.T                                     # +A^T instead of -A^T
    M[:n, n:] = Q
    M[n:, n:] = A
    F = core.expm(tau * M)
    E = F[n:, n:].copy()
    return E, E.T @ F[:n, n:]


def _expm_one_squaring_short(M):
    import math
    c = core.pade13_coefficients()
    nrm = core.norm1(M)
    s = 0 if nrm <= core.THETA13 else int(math.ceil(math.log2(nrm / core.THETA13)))
    X = M / 2.0 ** s
    I = np.eye(M.shape[0])
    X2 = X @ X
    X4 = X2 @ X2
    X6 = X4 @ X2
    U = X @ (X6 @ (c[13] * X6 + c[11] * X4 + c[9] * X2) + c[7] * X6 + c[5] * X4 + c[3] * X2 + c[1] * I)
    V = X6 @ (c[12] * X6 + c[10] * X4 + c[8] * X2) + c[6] * X6 + c[4] * X4 + c[2] * X2 + c[0] * I
    R = np.linalg.solve(V - U, V + U)
    for _ in range(max(s - 1, 0)):
        R = R @ R
    return R


def _vl_literal_block(A, Q, tau):
    """The unscaled literal block exponential: unstable at large tau ||A||."""
    n = A.shape[0]
    M = np.zeros((2 * n, 2 * n))
    M[:n, :n] = -A.T
    M[:n, n:] = Q
    M[n:, n:] = A
    F = core.expm(tau * M)
    E = F[n:, n:].copy()
    return E, E.T @ F[:n, n:]


def _vl_doubling_sign(A, Q, tau):
    E, Wm = core.van_loan(A, Q, tau / 2)
    return E @ E, Wm - E.T @ Wm @ E


def _pade_shifted():
    c = core.pade13_coefficients()
    return c[1:] + [c[13] / 27.0]


def _strang_full_steps(comp, flows, h):
    if len(flows) == 1 or comp == "lie":
        return [(f, h) for f in flows]
    half = [(f, h) for f in flows[:-1]]                 # h where h/2 belongs
    return half + [(flows[-1], h)] + half[::-1]


def _strang_wrong_order(comp, flows, h):
    seq = core.step_sequence(comp, flows, h)
    return seq[::-1] if comp == "lie" else seq[1:] + seq[:1]


@pytest.mark.parametrize("name,mut,pin,bound", [
    ("W drops E^T", dict(van_loan=_vl_missing_E), lambda m: pins.van_loan_diag_error(m), 1e-6),
    ("sign of A^T block", dict(van_loan=_vl_sign), lambda m: pins.van_loan_quadrature_error(m), 1e-6),
    ("unscaled block exponential", dict(van_loan=_vl_literal_block), lambda m: pins.van_loan_lyapunov_error(m), 1e-6),
    ("doubling sign", dict(van_loan=_vl_doubling_sign), lambda m: pins.van_loan_lyapunov_error(m), 1e-6),
    ("T12 transposed congruence", dict(flow_T12=lambda P, E, Wm: core.symmetrize(E @ P @ E.T + Wm)),
     lambda m: pins.t12_vs_ode_error(m), 1e-6),
    ("T3 sign", dict(flow_T3=lambda P, BRB, t: core.symmetrize(
        np.linalg.solve(np.eye(P.shape[0]) - t * (P @ BRB), P))),
     lambda m: pins.t3_closed_form_scalar_error(m), 1e-6),
    ("T3 operand order", dict(flow_T3=lambda P, BRB, t: core.symmetrize(
        np.linalg.solve(np.eye(P.shape[0]) + t * (BRB @ P), P.T).T)),
     lambda m: pins.t3_vs_ode_error(m), 1e-6),
    ("T4 midpoint drops 1/2", dict(flow_T4=lambda P, S, t, rule="midpoint": core.symmetrize(
        P + t * (S @ (P + t * (S @ P @ S.T)) @ S.T))),
     lambda m: max(pins.observed_orders(pins.t4_local_errors(m, "midpoint"))) < 2.6 and 1.0 or 0.0, 0.5),
    ("one squaring short", dict(expm=_expm_one_squaring_short), lambda m: pins.expm_scipy_error(m), 1e-6),
    ("Pade index shift", dict(pade13_coefficients=_pade_shifted), lambda m: pins.pade_table_error(m), 1e-6),
])
def test_pin_catches_planted_mistake(name, mut, pin, bound):
    good = pin(mutant())
    bad = pin(mutant(**mut))
    assert good < bound, (name, good)
    assert bad > bound, (name, bad)


def test_order_pin_catches_wrong_strang_half_steps():
    bad = pins.scalar_dre_errors(mutant(step_sequence=_strang_full_steps), "F12F3", "strang")
    good = pins.scalar_dre_errors(mutant(), "F12F3", "strang")
    assert good[-1] < 1e-4 and bad[-1] > 1e-2


def test_order_pin_catches_rotated_strang_sequence():
    orders = pins.observed_orders(pins.scalar_dre_errors(mutant(step_sequence=_strang_wrong_order),
                                                          "F1F2F3", "strang"))
    assert min(orders) < 1.5


def _weights_on_h_not_h2(q):
    # the slip: Lagrange nodes 1/k (odd error terms) instead of 1/k^2
    out = []
    for k in range(1, q + 1):
        g = 1.0
        for j in range(1, q + 1):
            if j != k:
                g *= k / (k - j)
        out.append(g)
    return out


def test_order_pin_catches_extrapolation_weights_on_h(monkeypatch):
    import math
    monkeypatch.setattr(core, "extrapolation_weights", _weights_on_h_not_h2)
    A, Q, B, R = (np.array([[v]]) for v in (-1.0, 2.0, 1.0, 1.0))
    exact = pins.scalar_dre_exact(-1.0, 1.0, 2.0, 1.0, 1.0)
    errs = [abs(O.solve_extrapolated(A, Q, np.zeros((1, 1)), 1.0, 2 ** k, 2, B=B, R=R)[0, 0] - exact) / exact
            for k in (2, 3, 4)]
    ords = pins.observed_orders(errs)
    assert not all(abs(o - 4.0) < 0.25 for o in ords), ords
    assert all(math.isfinite(e) for e in errs)
