"""Low-rank (LDL^T) CUDA path against the low-rank CPU oracle through the C ABI:
P = L D L^T compared element by element (bar 1e-11, the FP64 path's), the rank
and the kept eigenvalues, a general P0 = L0 D0 L0^T, and the error paths."""
import numpy as np
import pytest

import dme_workloads as W
import oracle as O
import paper_1805_08990_gb300 as dme
from gpu_util import FP64_TOL, SPLIT_TOL, dev, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _run(pr, flows, comp, N, q=7, tol=1e-13, L0=None, D0=None, T=None, prec="fp64"):
    T = pr.T if T is None else T
    uses_B = "F3" in flows
    uses_S = "F4" in flows
    B = pr.B if uses_B else None
    R = pr.R if uses_B else None
    S = pr.S if uses_S else None
    plan = dme.LowRankPlan(dev(pr.A), dev(pr.C), h=T / N, flows=flows, comp=comp,
                           B=None if B is None else dev(B), R=None if R is None else dev(R),
                           S=None if S is None else dev(S), quad_nodes=q, tol=tol, prec=prec)
    P = np.empty((pr.n, pr.n))
    r = plan.solve(T, N, L0=L0, D0=D0, P_out=P)
    L, d = plan.factors()
    n = pr.n
    Lo, Do = O.solve_lowrank(pr.A, pr.C, np.zeros((n, 0)) if L0 is None else L0,
                             np.zeros((0, 0)) if D0 is None else D0, T, N, comp, flows, B=B, R=R, S=S,
                             q=q, tol=tol)
    return P, r, L, d, Lo, Do


CASES = [
    ("dle", ["F1", "F2"], "strang", 10),
    ("dle", ["F1", "F2"], "lie", 6),
    ("dre", ["F1", "F2", "F3"], "strang", 6),
    ("dre", ["F12", "F3"], "strang", 5),
    ("dre", ["F1", "F3", "F2"], "lie", 4),
    ("dre", ["F12", "F3"], "lie", 3),
    ("gdre", ["F12", "F3", "F4"], "strang", 3),
    ("gdle", ["F1", "F2", "F4"], "lie", 3),
]


def _problem(kind):
    if kind == "dle":
        return W.dle_heat(nx=9)
    if kind == "dre":
        return W.dre_convdiff(nx=8, m=2, p=3)
    return W.gdre_convdiff_padded(nx=6, n_pad=40, m=2, p=2)


@pytest.mark.parametrize("kind,flows,comp,N", CASES)
def test_lowrank_matches_oracle(kind, flows, comp, N):
    pr = _problem(kind)
    P, r, L, d, Lo, Do = _run(pr, flows, comp, N)
    ref = O.ldl_product(Lo, Do)
    assert rel(P, ref) < FP64_TOL
    assert abs(r - Lo.shape[1]) <= 1
    assert rel(L @ np.diag(d) @ L.T, P) < 1e-13
    assert np.all(d > 0)


def test_lowrank_kept_eigenvalues_match_oracle():
    pr = W.dre_convdiff(nx=8, m=2, p=3)
    P, r, L, d, Lo, Do = _run(pr, ["F1", "F3", "F2"], "lie", 4)    # each Lie step ends with T2 (compressed)
    assert r == Lo.shape[1]
    assert np.allclose(d, np.diag(Do), rtol=1e-10, atol=1e-13 * d.max())
    assert np.allclose(L.T @ L, np.eye(r), atol=1e-10)


def test_lowrank_general_initial_state():
    pr = W.dre_convdiff(nx=7, m=2, p=2)
    rng = np.random.default_rng(11)
    L0 = rng.standard_normal((pr.n, 5))
    G = rng.standard_normal((5, 5))
    D0 = G @ G.T / 5 + 0.1 * np.eye(5)
    P, r, L, d, Lo, Do = _run(pr, ["F12", "F3"], "strang", 4, L0=L0, D0=D0)
    assert rel(P, O.ldl_product(Lo, Do)) < FP64_TOL


def test_lowrank_equals_dense_gpu_path():
    """With exact sub-flows (no quadrature) the factored scheme is the dense scheme."""
    pr = W.dre_convdiff(nx=8, m=2, p=3)
    flows, N = ["F1", "F2", "F3"], 8
    P, *_ = _run(pr, flows, "strang", N, tol=1e-15)
    dense = dme.Plan(dev(pr.A), C=dev(pr.C), h=pr.T / N, flows=flows, B=dev(pr.B), R=dev(pr.R))
    Pd = np.empty((pr.n, pr.n))
    dense.solve(pr.P0, pr.T, N, Pd)
    assert rel(P, Pd) < 1e-11


def test_lowrank_errors():
    pr = W.dre_convdiff(nx=6, m=2, p=3)
    with pytest.raises(dme.DmeError) as ei:
        plan = dme.LowRankPlan(dev(pr.A), dev(pr.C), h=0.1, flows=["F12", "F3"], B=dev(pr.B), R=dev(pr.R), rmax=8)
        plan.solve(1.0, 10, P_out=np.empty((pr.n, pr.n)))
    assert ei.value.status in (dme.DME_ENOMEM,)
    d = dme.make_desc(pr.n, m=2, p=3, eq=dme.DME_DRE, flows=["F12", "F3"], prec=7, h=0.1, q_is_factor=True)
    with pytest.raises(dme.DmeError):
        dme.dme_lr_plan(d, pr.A, pr.C, pr.B, pr.R)
    d = dme.make_desc(pr.n, m=2, p=3, eq=dme.DME_DRE, flows=["F12", "F3"], h=0.1, q_is_factor=False)
    with pytest.raises(dme.DmeError):
        dme.dme_lr_plan(d, pr.A, pr.Q, pr.B, pr.R)


@pytest.mark.parametrize("kind,flows,comp,N", [("dle", ["F1", "F2"], "strang", 10), ("dre", ["F12", "F3"], "strang", 5),
                                               ("gdre", ["F12", "F3", "F4"], "strang", 3),
                                               ("dre", ["F1", "F3", "F2"], "lie", 4)])
def test_lowrank_split_precision_matches_oracle(kind, flows, comp, N):
    """The products with E_t and S on the tensor cores (bf16 slices, exact
    accumulation), the rest in FP64: within the split-precision bar."""
    pr = _problem(kind)
    P, r, L, d, Lo, Do = _run(pr, flows, comp, N, prec="split_bf16")
    assert rel(P, O.ldl_product(Lo, Do)) < SPLIT_TOL
    assert abs(r - Lo.shape[1]) <= 1


def test_lowrank_split_at_full_size_matches_fp64_lowrank():
    """n = 4096 (the large DRE): split-precision factored steps against the FP64
    factored steps on the GPU (both parity-tested against the oracle above)."""
    pr = W.dre_heat_large()
    h = 1 / 256
    out = {}
    for prec in ("fp64", "split_bf16"):
        plan = dme.LowRankPlan(dev(pr.A), dev(pr.C), h=h, flows=["F1", "F2", "F3"], B=dev(pr.B), R=dev(pr.R),
                               prec=prec)
        P = np.empty((pr.n, pr.n))
        out[prec] = (plan.solve(8 * h, 8, P_out=P), P)
        plan.close()
    assert abs(out["fp64"][0] - out["split_bf16"][0]) <= 1
    assert rel(out["split_bf16"][1], out["fp64"][1]) < SPLIT_TOL


# ---------------------------------------------------------------- sparse A: Leja interpolation
import scipy.sparse as sp   # noqa: E402


def _csr_run(pr, flows, comp, N, q=7, tol=1e-13):
    A = sp.csr_matrix(pr.A)
    uses_B = "F3" in flows
    B = pr.B if uses_B else None
    R = pr.R if uses_B else None
    plan = dme.LowRankPlan.from_csr(A, pr.C, h=pr.T / N, flows=flows, comp=comp, B=B, R=R, quad_nodes=q, tol=tol)
    P = np.empty((pr.n, pr.n))
    r = plan.solve(pr.T, N, P_out=P)
    Lo, Do = O.solve_lowrank(A, pr.C, np.zeros((pr.n, 0)), np.zeros((0, 0)), pr.T, N, comp, flows, B=B, R=R,
                             q=q, tol=tol, action="leja")
    return P, r, Lo, Do, plan


@pytest.mark.parametrize("kind,flows,comp,N", [("dle", ["F1", "F2"], "strang", 10), ("dre", ["F12", "F3"], "strang", 5),
                                               ("dre", ["F1", "F3", "F2"], "lie", 4), ("dre", ["F1", "F2", "F3"], "strang", 6)])
def test_sparse_lowrank_matches_leja_oracle(kind, flows, comp, N):
    pr = _problem(kind)
    P, r, Lo, Do, _ = _csr_run(pr, flows, comp, N)
    assert rel(P, O.ldl_product(Lo, Do)) < FP64_TOL
    assert abs(r - Lo.shape[1]) <= 1


def test_sparse_lowrank_equals_dense_lowrank_gpu():
    pr = W.dre_convdiff(nx=8, m=2, p=3)
    P, *_ = _csr_run(pr, ["F1", "F2", "F3"], "strang", 6, tol=1e-15)
    Pd, *_ = _run(pr, ["F1", "F2", "F3"], "strang", 6, tol=1e-15)
    assert rel(P, Pd) < 1e-11


def test_sparse_lowrank_beyond_the_dense_limit_matches_closed_form():
    """n = 130^2 = 16900 (past the dense path's 16384): the DLE for the unscaled
    5-point stencil with Q = c c^T, T12 steps (exact flow, W by quadrature), the
    factored result applied to random vectors against the exact solution in the
    sine basis (DST)."""
    import pins
    nx = 130
    n = nx * nx
    T1 = sp.diags([np.full(nx - 1, 1.0), np.full(nx, -2.0), np.full(nx - 1, 1.0)], [-1, 0, 1])
    I1 = sp.identity(nx)
    A = (sp.kron(I1, T1) + sp.kron(T1, I1)).tocsr()
    c = np.random.default_rng(5).uniform(0.0, 1.0, n)
    T, N = 0.5, 5
    plan = dme.LowRankPlan.from_csr(A, c[None, :], h=T / N, flows=["F12"], comp="strang", quad_nodes=7)
    r = plan.solve(T, N)
    L, d = plan.factors()
    assert 1 <= r <= 224 and np.all(d > 0)
    X = np.random.default_rng(6).standard_normal((n, 1))
    got = L @ (d[:, None] * (L.T @ X))
    ref = pins.dle_exact_apply_stencil_laplacian(nx, c, T, X)
    assert np.linalg.norm(got - ref) / np.linalg.norm(ref) < 1e-10
    with pytest.raises(dme.DmeError):
        plan.solve(T, N, P_out=np.empty((1, 1)))


@pytest.mark.parametrize("control,flows,comp,N", [(True, ["F12", "F3", "F4"], "strang", 4),
                                                  (True, ["F1", "F2", "F3", "F4"], "lie", 5),
                                                  (False, ["F1", "F2", "F4"], "strang", 4)])
def test_sparse_generalised_lowrank_matches_leja_oracle(control, flows, comp, N):
    """Example 2's structure (stochastic heat transfer): sparse A and sparse S
    (the Robin-edge noise), B on the control edge, C the mean."""
    A, B, S, C, T = W.stochastic_heat_csr(8, control)
    R = np.eye(1) if control else None
    plan = dme.LowRankPlan.from_csr(A, C, h=T / N, flows=flows, comp=comp, B=B, R=R, S_csr=S, tol=1e-13)
    n = A.shape[0]
    P = np.empty((n, n))
    r = plan.solve(T, N, P_out=P)
    Lo, Do = O.solve_lowrank(A, C, np.zeros((n, 0)), np.zeros((0, 0)), T, N, comp, flows, B=B, R=R, S=S,
                             tol=1e-13, action="leja")
    assert rel(P, O.ldl_product(Lo, Do)) < FP64_TOL
    assert abs(r - Lo.shape[1]) <= 1


def test_sparse_generalised_lowrank_equals_dense_lowrank_gpu():
    pr = W.gdre_stochastic_heat(8, True)
    A, B, S, C, T = W.stochastic_heat_csr(8, True)
    plan = dme.LowRankPlan.from_csr(A, C, h=T / 5, flows=["F12", "F3", "F4"], B=B, R=np.eye(1), S_csr=S, tol=1e-15)
    P = np.empty((pr.n, pr.n))
    plan.solve(T, 5, P_out=P)
    Pd, *_ = _run(pr, ["F12", "F3", "F4"], "strang", 5, tol=1e-15)
    assert rel(P, Pd) < 1e-11


def test_sparse_lowrank_rejects_malformed_csr():
    pr = W.dre_convdiff(nx=5, m=2, p=2)
    A = sp.csr_matrix(pr.A)
    bad = A.indices.copy()
    bad[3] = pr.n + 7
    d = dme.make_desc(pr.n, m=2, p=2, eq=dme.DME_DRE, flows=["F12", "F3"], h=0.1, q_is_factor=True)
    with pytest.raises(dme.DmeError) as ei:
        dme.dme_lr_plan_csr(d, A.indptr, bad, A.data, pr.C, pr.B, pr.R)
    assert ei.value.status == dme.DME_EINVAL
    d4 = dme.make_desc(pr.n, m=2, p=2, eq=dme.DME_GDRE, flows=["F12", "F3", "F4"], h=0.1, q_is_factor=True)
    with pytest.raises(dme.DmeError):
        dme.dme_lr_plan_csr(d4, A.indptr, A.indices, A.data, pr.C, pr.B, pr.R)     # S missing
    with pytest.raises(dme.DmeError) as ei:
        dme.dme_lr_plan_csr(d4, A.indptr, A.indices, A.data, pr.C, pr.B, pr.R, S_csr=(A.indptr, bad, A.data))
    assert ei.value.status == dme.DME_EINVAL
    d1 = dme.make_desc(pr.n, m=2, p=2, eq=dme.DME_DRE, flows=["F12", "F3", "F4"], h=0.1, q_is_factor=True)
    with pytest.raises(dme.DmeError):
        dme.dme_lr_plan_csr(d1, A.indptr, A.indices, A.data, pr.C, pr.B, pr.R)     # F4 needs GDLE / GDRE
