"""Pins of the Leja-interpolation oracle (the exponential's action on a block
of vectors) against closed forms, scipy's dense exponential and sparse
expm_multiply, eigenvalues, and the dense low-rank path.  CPU only."""
import math

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spl

import dme_workloads as W
import oracle as O


def test_first_leja_points():
    x = O.leja_points(5)
    assert list(x[:3]) == [2.0, -2.0, 0.0]
    # the fourth maximises |x - 2| |x + 2| |x| = |x (4 - x^2)|: x = +-2/sqrt(3)
    assert abs(abs(x[3]) - 2 / math.sqrt(3)) < 4.0 / 20000
    assert len(set(np.round(x, 12))) == 5


def test_divided_differences_closed_forms():
    for scale in (0.3, 1.0, 3.0):
        x = np.array([0.5, -1.2])
        dd = O.divided_differences_exp(x, scale)
        assert abs(dd[0] - math.exp(scale * 0.5)) < 1e-15 * math.exp(scale * 0.5)
        ref = (math.exp(scale * -1.2) - math.exp(scale * 0.5)) / (-1.2 - 0.5)
        assert abs(dd[1] - ref) < 1e-14 * abs(ref)
    # confluent limit: all points equal -> scale^k e^{scale x} / k!
    dd = O.divided_differences_exp(np.full(6, 0.7), 2.0)
    ref = [2.0 ** k * math.exp(1.4) / math.factorial(k) for k in range(6)]
    assert np.allclose(dd, ref, rtol=1e-13)


def test_gershgorin_interval_contains_the_spectrum():
    pr = W.dre_convdiff(nx=6)
    a, b = O.gershgorin_interval(pr.A)
    ev = np.linalg.eigvals(pr.A)
    assert np.all(ev.real >= a - 1e-9) and np.all(ev.real <= b + 1e-9)


@pytest.mark.parametrize("tau", [1e-3, 1 / 64, 0.25])
def test_leja_action_matches_dense_exponential(tau):
    pr = W.dre_convdiff(nx=10)
    V = np.random.default_rng(0).standard_normal((pr.n, 5))
    ref = sla.expm(tau * pr.A.T) @ V
    got = O.leja_action(pr.A.T, V, tau)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_leja_action_sparse_matches_expm_multiply():
    pr = W.dle_heat(nx=40)
    A = sp.csr_matrix(pr.A)
    V = np.random.default_rng(1).standard_normal((pr.n, 3))
    ref = spl.expm_multiply((1 / 512) * A.tocsc(), V)
    got = O.leja_action(A, V, 1 / 512)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-12


def test_lowrank_with_leja_action_equals_dense_lowrank():
    pr = W.dre_convdiff(nx=8, m=2, p=3)
    n = pr.n
    for flows in (["F1", "F2", "F3"], ["F12", "F3"]):
        L1, D1 = O.solve_lowrank(pr.A, pr.C, np.zeros((n, 0)), np.zeros((0, 0)), pr.T, 6, "strang", flows,
                                 B=pr.B, R=pr.R, tol=1e-15)
        L2, D2 = O.solve_lowrank(sp.csr_matrix(pr.A), pr.C, np.zeros((n, 0)), np.zeros((0, 0)), pr.T, 6, "strang",
                                 flows, B=pr.B, R=pr.R, tol=1e-15, action="leja")
        assert O.rel_fro(O.ldl_product(L2, D2), O.ldl_product(L1, D1)) < 1e-12


def test_pin_catches_unscaled_divided_differences(monkeypatch):
    import oracle.dme_leja as lj

    def unscaled(x, scale=1.0):          # the slip: ones below the diagonal not scaled
        m = len(x)
        Z = np.diag(scale * np.asarray(x)) + np.diag(np.ones(m - 1), -1)
        return O.expm(Z)[:, 0].copy()

    monkeypatch.setattr(lj, "divided_differences_exp", unscaled)
    pr = W.dre_convdiff(nx=10)
    V = np.random.default_rng(0).standard_normal((pr.n, 5))
    ref = sla.expm(pr.A.T / 64) @ V
    got = O.leja_action(pr.A.T, V, 1 / 64)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) > 1e-3


def test_stencil_laplacian_dle_closed_form_helper():
    """The DST-based exact DLE product used at large n, against the dense
    eigenbasis closed form at a small size."""
    import pins
    nx = 6
    A = W.laplacian_2d(nx) / (nx + 1) ** 2
    c = np.random.default_rng(2).uniform(0, 1, nx * nx)
    lam, V = np.linalg.eigh(A)
    P = pins.dle_exact_symmetric(V, lam, np.outer(c, c), np.zeros_like(A), 0.7)
    X = np.random.default_rng(3).standard_normal((nx * nx, 2))
    got = pins.dle_exact_apply_stencil_laplacian(nx, c, 0.7, X)
    assert np.linalg.norm(got - P @ X) / np.linalg.norm(P @ X) < 1e-13


def test_sparse_generalised_factored_oracle_equals_dense_form():
    """The factored oracle with sparse A and S (Leja action, sparse S L) against
    the same oracle with dense A and S and the dense exponential (Example 2's
    structure, GDRE, Strang F12 F3 F4)."""
    import dme_workloads as W
    from oracle.dme_lowrank import solve_lowrank, ldl_product
    A, B, S, C, T = W.stochastic_heat_csr(6, True)
    n = A.shape[0]
    z, z0 = np.zeros((n, 0)), np.zeros((0, 0))
    flows = ["F12", "F3", "F4"]
    Ls, Ds = solve_lowrank(A, C, z, z0, T, 4, "strang", flows, B=B, R=np.eye(1), S=S, tol=1e-15, action="leja")
    Ld, Dd = solve_lowrank(A.toarray(), C, z, z0, T, 4, "strang", flows, B=B, R=np.eye(1), S=S.toarray(),
                           tol=1e-15, action="dense")
    Ps, Pd = ldl_product(Ls, Ds), ldl_product(Ld, Dd)
    assert np.linalg.norm(Ps - Pd) / np.linalg.norm(Pd) < 1e-11


def test_stochastic_heat_data_structure():
    """Generator shape checks: A symmetric with the Robin diagonal on the east
    edge only, S diagonal on that edge, B on the west edge, C the mean."""
    import dme_workloads as W
    nx = 7
    A, B, S, C, T = W.stochastic_heat_csr(nx, True)
    Ad = A.toarray()
    dx = 1.0 / (nx + 1)
    assert np.allclose(Ad, Ad.T)
    east = [nx - 1 + nx * j for j in range(nx)]
    d = np.diag(Ad) * dx * dx
    assert np.allclose(d[east], -3.0 + 0.25 * dx)
    assert np.allclose(np.delete(d, east), -4.0)
    assert S.nnz == nx and np.allclose(S.diagonal()[east], 0.5 / dx)
    assert np.count_nonzero(B) == nx and np.allclose(B[::nx, 0], 1.0 / (dx * dx))
    assert np.isclose(C.sum(), 1.0) and T == 0.5
    assert W.stochastic_heat_csr(nx, False)[1] is None
