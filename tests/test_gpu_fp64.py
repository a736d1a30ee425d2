"""FP64 CUDA path against the CPU oracle, element by element, through the C ABI.
Sizes span several 64-wide tiles and ragged tails; bar: relative Frobenius
error <= 1e-11 (and exact symmetry of every GPU state)."""
import math

import numpy as np
import pytest
import torch

import dme_workloads as W
import oracle as O
import paper_1805_08990_gb300 as dme
from gpu_util import FP64_TOL, dev, host, plan_for, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


# ---------------------------------------------------------------- plan: E_t, W_t
@pytest.mark.parametrize("n,kind,tau", [(1, "random", 0.3), (37, "random", 0.05), (100, "convdiff", 1e-3),
                                        (130, "random", 2.0), (256, "laplace", 5e-4)])
def test_expm_van_loan_matches_oracle(n, kind, tau):
    rng = np.random.default_rng(n)
    if kind == "convdiff":
        A = W.convection_diffusion_2d(int(math.isqrt(n)))
    elif kind == "laplace":
        A = W.laplacian_2d(int(math.isqrt(n)))
    else:
        M = rng.standard_normal((n, n)) / math.sqrt(n)
        A = M - (np.abs(M).sum(axis=0).max() * 0.5) * np.eye(n)
    C = rng.uniform(0, 1, (3, n))
    Q = C.T @ C
    E_ref, W_ref = O.van_loan(A, Q, tau)
    plan = dme.Plan(dev(A), C=dev(C), h=tau, flows=["F12"])
    E = torch.empty(n, n, dtype=torch.float64, device="cuda")
    Wd = torch.empty_like(E)
    plan.expm(tau, E, Wd)
    assert rel(host(E), E_ref) < FP64_TOL
    assert rel(host(Wd), W_ref) < FP64_TOL
    assert torch.equal(Wd, Wd.T)
    # host output pointers work too
    Eh = np.empty((n, n))
    plan.expm(tau, Eh, None)
    assert rel(Eh, E_ref) < FP64_TOL


# ---------------------------------------------------------------- single sub-flows
def _problem(n, m=3, with_S=True, seed=0):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n)) / math.sqrt(n)
    A = M - (np.abs(M).sum(axis=0).max() * 0.5 + 0.5) * np.eye(n)
    C = rng.uniform(0, 1, (2, n))
    B = rng.standard_normal((n, m))
    G = rng.standard_normal((m, m))
    R = G @ G.T + m * np.eye(m)
    S = 0.3 * rng.standard_normal((n, n)) / math.sqrt(n) if with_S else None
    return W.Problem("t", A, C, np.zeros((n, n)), 1.0, B=B, R=R, S=S)


@pytest.mark.parametrize("n", [1, 37, 64, 130])
@pytest.mark.parametrize("flow", ["F1", "F2", "F12", "F3", "F4"])
def test_single_subflow_matches_oracle(n, flow):
    pr = _problem(n, m=3)
    tau = 0.07
    plan = plan_for(pr, ["F12", "F3", "F4"], "strang", tau)
    P0 = W.random_psd(n, 5 + n)
    P = dev(P0)
    plan.apply(flow, tau, P)
    op = O.Plan(pr.A, pr.Q, pr.B, pr.R, pr.S)
    ref = op.apply(flow, tau, P0, "midpoint")
    assert rel(host(P), ref) < FP64_TOL, flow
    assert torch.equal(P, P.T)


@pytest.mark.parametrize("m", [1, 2, 8, 11])
def test_riccati_flow_m_sizes(m):
    n = 97
    pr = _problem(n, m=m, with_S=False, seed=m)
    plan = plan_for(pr, ["F12", "F3"], "strang", 0.1)
    P0 = W.random_psd(n, m, scale=3.0)
    P = dev(P0)
    plan.apply("F3", 0.4, P)
    ref = O.flow_T3(P0, pr.B @ np.linalg.solve(pr.R, pr.B.T), 0.4)
    assert rel(host(P), ref) < FP64_TOL


def test_t4_euler_rule_for_lie():
    pr = _problem(50)
    plan = plan_for(pr, ["F12", "F4"], "lie", 0.1)
    P0 = W.random_psd(50, 1)
    P = dev(P0)
    plan.apply("F4", 0.1, P)
    assert rel(host(P), O.flow_T4(P0, pr.S, 0.1, "euler")) < FP64_TOL


# ---------------------------------------------------------------- compositions
def _oracle_solve(pr, flows, comp, N, T=None, t4_rule=None):
    T = pr.T if T is None else T
    uses_B = "F3" in flows
    return O.solve(pr.A, pr.Q, pr.P0, T, N, comp, flows, B=pr.B if uses_B else None,
                   R=pr.R if uses_B else None, S=pr.S if "F4" in flows else None, t4_rule=t4_rule)


@pytest.mark.parametrize("scheme,comp", [("F1F2", "strang"), ("F12", "strang"), ("F1F2", "lie")])
def test_dle_heat_n256_full_config(scheme, comp):
    """Plain DLE, n = 256 Laplacian, Q = all-ones, T = 0.1, h = T/100."""
    pr = W.dle_heat(16)
    N = 100
    flows = W.SCHEMES[scheme]
    plan = plan_for(pr, flows, comp, pr.T / N)
    out = np.empty((pr.n, pr.n))
    plan.solve(pr.P0, pr.T, N, out)
    ref = _oracle_solve(pr, flows, comp, N)
    assert rel(out, ref) < FP64_TOL
    assert np.array_equal(out, out.T)


@pytest.mark.parametrize("scheme", ["F12F3", "F1F2F3", "F1F3F2"])
@pytest.mark.parametrize("comp", ["lie", "strang"])
def test_dre_convdiff_small_schemes(scheme, comp):
    pr = W.dre_convdiff(nx=10, m=2, p=3)        # n = 100: two 64-tiles, ragged
    N = 16
    flows = W.SCHEMES[scheme]
    plan = plan_for(pr, flows, comp, pr.T / N)
    P = dev(pr.P0)
    plan.step(P, N)
    assert rel(host(P), _oracle_solve(pr, flows, comp, N)) < FP64_TOL


@pytest.mark.parametrize("scheme,comp", [("F12F3F4", "strang"), ("F12F4F3", "lie"), ("F12F4", "strang"),
                                         ("F1F2F4", "strang"), ("F1F4F2", "strang"), ("F1F4F2", "lie"),
                                         ("F1F2F3F4", "strang"), ("F1F2F3F4", "lie")])
def test_generalised_schemes_padded(scheme, comp):
    pr = W.gdre_convdiff_padded(nx=8, n_pad=72, m=2, p=3)
    N = 8
    flows = W.SCHEMES[scheme]
    plan = plan_for(pr, flows, comp, pr.T / N)
    P = dev(pr.P0)
    plan.step(P, N)
    got = host(P)
    assert rel(got, _oracle_solve(pr, flows, comp, N)) < FP64_TOL
    na = pr.meta["n_active"]
    assert np.all(got[na:, :] == 0) and np.all(got[:, na:] == 0)


def test_dre_convdiff_n1024_full_size():
    """DRE config at full size (n = 1024), FP64, Strang F12F3, h = T/16."""
    pr = W.dre_convdiff()
    N = 16
    plan = plan_for(pr, ["F12", "F3"], "strang", pr.T / N)
    P = dev(pr.P0)
    plan.step(P, N)
    ref = _oracle_solve(pr, ["F12", "F3"], "strang", N)
    assert rel(host(P), ref) < FP64_TOL


def test_scalar_dre_against_tanh_closed_form():
    a, b, q = -1.0, 1.0, 2.0
    A, C, B, R = np.array([[a]]), np.array([[math.sqrt(q)]]), np.array([[b]]), np.array([[1.0]])
    beta = math.sqrt(a * a + q * b * b)
    exact = q * math.tanh(beta) / (beta - a * math.tanh(beta))
    errs = []
    for N in (32, 64):
        plan = dme.Plan(dev(A), C=dev(C), h=1.0 / N, flows=["F12", "F3"], comp="strang", B=dev(B), R=dev(R))
        out = np.zeros((1, 1))
        plan.solve(np.zeros((1, 1)), 1.0, N, out)
        errs.append(abs(out[0, 0] - exact) / exact)
    assert errs[1] < 1e-4 and 1.9 < math.log2(errs[0] / errs[1]) < 2.1


def test_step_replay_equals_repeated_single_steps():
    pr = W.dre_convdiff(nx=8, m=2, p=3)
    plan = plan_for(pr, ["F12", "F3"], "strang", 0.05)
    P1 = dev(W.random_psd(pr.n, 3))
    P2 = P1.clone()
    plan.step(P1, 3)
    for _ in range(3):
        plan.step(P2, 1)
    assert torch.equal(P1, P2)


def test_solve_host_and_device_buffers_agree():
    pr = W.dre_convdiff(nx=8, m=2, p=3)
    plan = plan_for(pr, ["F12", "F3"], "strang", 0.1)
    Ph = np.empty((pr.n, pr.n))
    plan.solve(pr.P0, 1.0, 10, Ph)
    Pd = torch.empty(pr.n, pr.n, dtype=torch.float64, device="cuda")
    plan.solve(dev(pr.P0), 1.0, 10, Pd)
    assert np.array_equal(Ph, host(Pd))
    # a different h than the plan's rebuilds E, W for the new step lengths
    plan.solve(pr.P0, 1.0, 20, Ph)
    assert rel(Ph, _oracle_solve(pr, ["F12", "F3"], "strang", 20)) < FP64_TOL


# ---------------------------------------------------------------- errors
def test_non_spd_R_is_reported():
    pr = _problem(20, m=2, with_S=False)
    with pytest.raises(dme.DmeError) as ei:
        dme.Plan(dev(pr.A), C=dev(pr.C), h=0.1, flows=["F12", "F3"], B=dev(pr.B), R=dev(-np.eye(2)))
    assert ei.value.status == dme.DME_ENOTSPD


def test_invalid_descriptors_are_rejected():
    A = dev(np.eye(4))
    C = dev(np.ones((1, 4)))
    with pytest.raises(dme.DmeError) as ei:
        dme.Plan(A, C=C, h=-1.0)
    assert ei.value.status == dme.DME_EINVAL
    d = dme.make_desc(0, eq=dme.DME_DLE, flows=("F12",), h=0.1, q_is_factor=True, p=1)
    with pytest.raises(dme.DmeError):
        dme.dme_plan(d, A, C)
    d = dme.make_desc(4, eq=dme.DME_DLE, flows=("F12", "F3"), h=0.1, q_is_factor=True, p=1)
    with pytest.raises(dme.DmeError):                      # F3 in a DLE
        dme.dme_plan(d, A, C)


def test_riccati_not_spd_on_device_is_reported():
    """M = I + t Bt^T P Bt fails its Cholesky when P is strongly indefinite."""
    pr = _problem(16, m=2, with_S=False)
    plan = plan_for(pr, ["F12", "F3"], "strang", 0.1)
    P = dev(-50.0 * np.eye(16))
    with pytest.raises(dme.DmeError) as ei:
        plan.apply("F3", 1.0, P)
    assert ei.value.status == dme.DME_ENOTSPD
    # the plan stays usable afterwards
    P = dev(W.random_psd(16, 1))
    plan.apply("F3", 0.1, P)


@pytest.mark.parametrize("n,m", [(1, 1), (130, 3), (257, 8)])
def test_lqr_gain_matches_oracle(n, m):
    pr = _problem(n, m=m, with_S=False, seed=n)
    plan = plan_for(pr, ["F12", "F3"], "strang", 0.1)
    P0 = W.random_psd(n, 2 * n, scale=2.0)
    K = np.empty((m, n))
    plan.gain(dev(P0), K)
    assert rel(K, O.lqr_gain(P0, pr.B, pr.R)) < FP64_TOL
    with pytest.raises(dme.DmeError):
        dle = dme.Plan(dev(pr.A), C=dev(pr.C), h=0.1, flows=["F12"])
        dle.gain(dev(P0), K)


@pytest.mark.parametrize("nx,prec", [(8, "fp64"), (11, "fp64"), (11, "split_bf16")])
def test_mass_matrix_dre_matches_oracle(nx, prec):
    """Example 4's generalised state space: the plan forms A M^-1 and M^-T Q M^-1
    on the device; the solve matches the oracle's transform + scheme."""
    pr = W.fe_heat_mass(nx=nx, m=2, p=3, T=0.2)
    M = pr.meta["M"]
    N = 16
    plan = dme.Plan(dev(pr.A), C=dev(pr.C), h=pr.T / N, flows=["F12", "F3"], comp="strang", B=dev(pr.B),
                    R=dev(pr.R), M=dev(M), prec=prec)
    out = np.empty((pr.n, pr.n))
    plan.solve(pr.P0, pr.T, N, out)
    At, Qt = O.mass_transform(M, pr.A, pr.Q)
    ref = O.solve(At, Qt, pr.P0, pr.T, N, "strang", ["F12", "F3"], B=pr.B, R=pr.R)
    assert rel(out, ref) < (FP64_TOL if prec == "fp64" else 1e-7)


@pytest.mark.parametrize("nx", [7, 12])
def test_mass_matrix_needing_row_exchanges(nx):
    """A mass matrix with its rows reversed (zero diagonal away from the middle):
    the device's Gauss-Jordan inversion must exchange rows at almost every
    column.  The plan's (E_t, W_t) for A M^-1 and M^-T Q M^-1 against the
    oracle's transform (LU solves) and Van Loan exponential."""
    pr = W.fe_heat_mass(nx=nx, m=2, p=3)
    M = np.ascontiguousarray(pr.meta["M"][::-1])
    assert np.count_nonzero(np.diag(M)) < pr.n // 2
    tau = 1e-3
    plan = dme.Plan(dev(pr.A), C=dev(pr.C), h=tau, flows=["F12"], M=dev(M))
    E = np.empty((pr.n, pr.n))
    Wm = np.empty((pr.n, pr.n))
    plan.expm(tau, E, Wm)
    At, Qt = O.mass_transform(M, pr.A, pr.Q)
    E_ref, W_ref = O.van_loan(At, Qt, tau)
    assert rel(E, E_ref) < FP64_TOL
    assert rel(Wm, W_ref) < FP64_TOL


def test_mass_matrix_plan_rejections():
    pr = W.fe_heat_mass(nx=5, m=2, p=3)
    M = pr.meta["M"].copy()
    M[-1, :] = 0.0                                   # singular mass matrix
    with pytest.raises(dme.DmeError) as ei:
        dme.Plan(dev(pr.A), C=dev(pr.C), h=0.01, flows=["F12", "F3"], B=dev(pr.B), R=dev(pr.R), M=dev(M))
    assert ei.value.status == dme.DME_EINVAL
    with pytest.raises(dme.DmeError):
        dme.Plan(dev(pr.A), C=dev(pr.C), h=0.01, flows=["F12", "F3", "F4"], B=dev(pr.B), R=dev(pr.R),
                 S=dev(np.eye(pr.n)), M=dev(pr.meta["M"]))


# ---------------------------------------------------------------- FSAL merging, extrapolated Strang
@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
@pytest.mark.parametrize("scheme,N", [("F12F3", 12), ("F1F2F3", 7), ("F1F3F2", 2), ("F12F3", 1)])
def test_fsal_matches_unmerged_oracle(prec, scheme, N):
    """Merging T_a(h/2) T_a(h/2) of neighbouring Strang steps into T_a(h) is
    exact for exact outer flows: the result is the unmerged scheme's."""
    pr = W.dre_convdiff(nx=10, m=2, p=3)
    flows = W.SCHEMES[scheme]
    plan = plan_for(pr, flows, "strang", pr.T / N, prec=prec, fsal=True)
    P = dev(pr.P0)
    plan.step(P, N)
    got = host(P)
    ref = _oracle_solve(pr, flows, "strang", N)
    assert rel(got, ref) < (FP64_TOL if prec == "fp64" else 1e-7)
    assert np.array_equal(got, got.T)
    if N >= 2:
        plain = plan_for(pr, flows, "strang", pr.T / N, prec=prec)
        plain.step(dev(pr.P0), 1)
        assert plan.kernels_per_step < plain.kernels_per_step


def test_fsal_dle_and_rejections():
    pr = W.dle_heat(nx=9)
    N = 10
    plan = plan_for(pr, ["F1", "F2"], "strang", pr.T / N, fsal=True)
    P = dev(pr.P0)
    plan.step(P, N)
    assert rel(host(P), _oracle_solve(pr, ["F1", "F2"], "strang", N)) < FP64_TOL
    g = W.gdre_convdiff_padded(nx=5, n_pad=32, m=2, p=2)
    for flows, comp in [(["F12", "F3"], "lie"), (["F12"], "strang"), (["F4", "F12"], "strang")]:
        with pytest.raises(dme.DmeError):
            plan_for(g, flows, comp, 0.01, fsal=True)


@pytest.mark.parametrize("prec", ["fp64", "split_bf16"])
@pytest.mark.parametrize("q,scheme,N", [(2, "F12F3", 6), (3, "F12F3", 3), (4, "F1F2F3", 2), (2, "F1F2", 5)])
def test_extrapolated_strang_matches_oracle(prec, q, scheme, N):
    pr = W.dre_convdiff(nx=9, m=2, p=3) if "F3" in W.SCHEMES[scheme] else W.dle_heat(nx=9)
    flows = W.SCHEMES[scheme]
    plan = plan_for(pr, flows, "strang", pr.T / N, prec=prec, extrap=q)
    P = dev(pr.P0)
    plan.step(P, N)
    got = host(P)
    uses_B = "F3" in flows
    ref = O.solve_extrapolated(pr.A, pr.Q, pr.P0, pr.T, N, q, flows=flows, B=pr.B if uses_B else None,
                               R=pr.R if uses_B else None)
    assert rel(got, ref) < (FP64_TOL if prec == "fp64" else 1e-7)
    assert np.array_equal(got, got.T)


def test_extrapolation_rejections():
    g = W.gdre_convdiff_padded(nx=5, n_pad=32, m=2, p=2)
    for flows, comp, q, fsal in [(["F12", "F3"], "lie", 2, False), (["F12", "F3", "F4"], "strang", 2, False),
                                 (["F12", "F3"], "strang", 5, False), (["F12", "F3"], "strang", 2, True)]:
        with pytest.raises(dme.DmeError):
            plan_for(g, flows, comp, 0.01, extrap=q, fsal=fsal)


# ---------------------------------------------------------------- the dense solve of the Pade step
@pytest.mark.parametrize("n,nrhs", [(1, 3), (37, 5), (200, 300), (64, 26000), (1100, 40), (4100, 3)])
def test_dense_solve_matches_numpy(n, nrhs):
    """Blocked Gauss-Jordan with partial pivoting (the plan's Pade solves) against
    numpy's LU solve: one panel and a ragged one (37), several (200), a trailing
    block far wider than M (64, 26000), a cluster of 8 CTAs per panel (1100), and
    above 4096 the single cooperative launch (4100)."""
    rng = np.random.default_rng(n + nrhs)
    M = rng.standard_normal((n, n)) + n ** 0.5 * np.eye(n)
    B = rng.standard_normal((n, nrhs))
    X = B.copy()
    dme.dme_dense_solve(M, X)
    ref = np.linalg.solve(M, B)
    assert rel(X, ref) < 1e-12
    Md, Xd = dev(M), dev(B)
    dme.dme_dense_solve(Md, Xd)
    assert rel(host(Xd), ref) < 1e-12
    assert np.array_equal(host(Md), M)


def test_dense_solve_pivots_and_rejects_singular():
    n = 50
    rng = np.random.default_rng(3)
    P = np.eye(n)[rng.permutation(n)]
    M = P @ (3.0 * np.eye(n) + 0.1 * rng.standard_normal((n, n)))   # dominant entries off the diagonal
    assert np.count_nonzero(np.argmax(np.abs(M), axis=0) != np.arange(n)) > n // 2
    B = rng.standard_normal((n, 4))
    X = B.copy()
    dme.dme_dense_solve(M, X)
    assert rel(X, np.linalg.solve(M, B)) < 1e-11
    S = M.copy()
    S[:, 7] = 0.0                                          # a zero column: singular
    with pytest.raises(dme.DmeError) as ei:
        dme.dme_dense_solve(S, B.copy())
    assert ei.value.status == dme.DME_EINVAL


def test_bounded_device_wait_gives_up_and_reports():
    """A grid-barrier wait that nothing releases (the wait of the persistent
    kernels) stops at its poll limit with DEV_TIMEOUT; the context stays usable."""
    assert dme.dme_wait_selftest()
    X = np.eye(3)
    dme.dme_dense_solve(2.0 * np.eye(3), X)
    assert np.allclose(X, 0.5 * np.eye(3))


# ---------------------------------------------------------------- golden fixtures (tests/golden/)
def test_cuda_path_reproduces_golden_fixtures():
    """The stored oracle values of tests/golden/ (scalar DRE, Lie and Strang
    F12F3 at N = 8..64; the 3 x 3-grid DLE after 10 F12 steps) from the CUDA
    path: FP64 to 1e-11, the split path to 1e-7."""
    import test_golden as G
    p, _, vals = G.load_scalar()
    A, C, B, R = (np.array([[p["a"]]]), np.array([[math.sqrt(p["q"])]]), np.array([[p["b"]]]),
                  np.array([[p["r"]]]))
    for (comp, N), v in vals.items():
        plan = dme.Plan(dev(A), C=dev(C), h=p["T"] / N, flows=["F12", "F3"], comp=comp, B=dev(B), R=dev(R))
        out = np.zeros((1, 1))
        plan.solve(np.zeros((1, 1)), p["T"], N, out)
        assert abs(out[0, 0] - v) <= FP64_TOL * abs(v), (comp, N)
    P = G.load_dle()
    pr = W.dle_heat(nx=3, T=0.1)
    for prec, tol in (("fp64", FP64_TOL), ("split_bf16", 1e-7)):
        plan = dme.Plan(dev(pr.A), C=dev(pr.C), h=pr.T / 10, flows=["F12"], comp="strang", prec=prec)
        out = np.empty((9, 9))
        plan.solve(pr.P0, pr.T, 10, out)
        assert rel(out, P) < tol, prec
