"""Split-precision (bf16 slices on tcgen05) path against exact products and
the CPU oracle.  Bar: relative Frobenius error <= 1e-7 (the path is built
for ~1e-8 per product)."""
import math

import numpy as np
import pytest
import torch

import dme_workloads as W
import oracle as O
import paper_1805_08990_gb300 as dme
from gpu_util import SPLIT_TOL, dev, host, plan_for, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def gemm_split(A, B):
    C = torch.empty(A.shape[0], B.shape[0], dtype=torch.float64, device="cuda")
    dme.dme_gemm_split(dev(A), dev(B), C)
    torch.cuda.synchronize()
    return host(C)


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (256, 384, 512), (100, 37, 70), (1, 1, 1), (130, 260, 4096)])
def test_tensor_core_products_of_small_integers_are_exact(M, N, K):
    """Integers in [-63, 63] fit the first slice exactly, so C = A B^T must be
    bit-exact: checks the TMA/UMMA tile layouts and the exact fp32 accumulation."""
    rng = np.random.default_rng(M * 7 + N * 3 + K)
    A = rng.integers(-63, 64, size=(M, K)).astype(np.float64)
    B = rng.integers(-63, 64, size=(N, K)).astype(np.float64)
    A[:, 0] = 63.0        # every row uses the full first-slice range
    B[:, 0] = -63.0
    C = gemm_split(A, B)
    assert np.array_equal(C, A @ B.T)


def test_tensor_core_exact_at_accumulator_limit():
    """All-64 rows at K = 4096: level-0 sums reach exactly 2^24 units."""
    K = 4096
    A = np.full((128, K), 1.0)
    B = np.full((128, K), 1.0)
    A[1::2] = -1.0
    C = gemm_split(A, B)
    assert np.array_equal(C, A @ B.T)


@pytest.mark.parametrize("M,N,K", [(64, 64, 64), (200, 150, 333), (512, 512, 4096)])
def test_split_gemm_random_accuracy(M, N, K):
    rng = np.random.default_rng(K)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    ref = A @ B.T
    C = gemm_split(A, B)
    # entrywise bound ~ 2^-27 of the row scales times sqrt(K) (random signs)
    assert rel(C, ref) < SPLIT_TOL
    bound = 4 * 2.0 ** -27 * np.abs(A).max(1)[:, None] * np.abs(B).max(1)[None, :] * math.sqrt(K)
    assert np.all(np.abs(C - ref) <= bound + 1e-300)


def test_split_gemm_wide_dynamic_range_rows():
    rng = np.random.default_rng(3)
    A = rng.uniform(0, 1, (96, 256)) * np.logspace(-20, 20, 96)[:, None]
    B = rng.uniform(0, 1, (80, 256)) * np.logspace(15, -15, 80)[:, None]
    ref = A @ B.T
    C = gemm_split(A, B)
    assert np.max(np.abs(C - ref) / np.abs(ref)) < 1e-7


def test_split_gemm_rejects_long_k():
    with pytest.raises(dme.DmeError):
        gemm_split(np.ones((4, 4097)), np.ones((4, 4097)))


# ---------------------------------------------------------------- sub-flows and schemes
def _problem(n, m=3, seed=0):
    rng = np.random.default_rng(seed)
    M = rng.standard_normal((n, n)) / math.sqrt(n)
    A = M - (np.abs(M).sum(axis=0).max() * 0.5 + 0.5) * np.eye(n)
    C = rng.uniform(0, 1, (2, n))
    B = rng.standard_normal((n, m))
    S = 0.3 * rng.standard_normal((n, n)) / math.sqrt(n)
    return W.Problem("t", A, C, np.zeros((n, n)), 1.0, B=B, R=np.eye(m), S=S)


@pytest.mark.parametrize("n", [1, 37, 130, 300])
@pytest.mark.parametrize("flow", ["F1", "F12", "F4"])
def test_split_subflows_match_oracle(n, flow):
    pr = _problem(n)
    tau = 0.05
    plan = plan_for(pr, ["F12", "F3", "F4"], "strang", tau, prec="split_bf16")
    P0 = W.random_psd(n, 3 + n)
    P = dev(P0)
    plan.apply(flow, tau, P)
    ref = O.Plan(pr.A, pr.Q, pr.B, pr.R, pr.S).apply(flow, tau, P0, "midpoint")
    assert rel(host(P), ref) < SPLIT_TOL
    assert torch.equal(P, P.T)


def _oracle_solve(pr, flows, comp, N):
    uses_B = "F3" in flows
    return O.solve(pr.A, pr.Q, pr.P0, pr.T, N, comp, flows, B=pr.B if uses_B else None,
                   R=pr.R if uses_B else None, S=pr.S if "F4" in flows else None)


@pytest.mark.parametrize("scheme,comp", [("F12F3", "strang"), ("F1F2F3", "strang"), ("F1F3F2", "lie")])
def test_split_dre_convdiff_n1024(scheme, comp):
    """DRE config at full size, split precision, 64 steps."""
    pr = W.dre_convdiff()
    N = 64
    flows = W.SCHEMES[scheme]
    plan = plan_for(pr, flows, comp, pr.T / N, prec="split_bf16")
    P = dev(pr.P0)
    plan.step(P, N)
    assert rel(host(P), _oracle_solve(pr, flows, comp, N)) < SPLIT_TOL


def test_split_dle_heat_n256_full_config():
    pr = W.dle_heat(16)
    plan = plan_for(pr, ["F1", "F2"], "strang", pr.T / 100, prec="split_bf16")
    P = dev(pr.P0)
    plan.step(P, 100)
    assert rel(host(P), _oracle_solve(pr, ["F1", "F2"], "strang", 100)) < SPLIT_TOL


@pytest.mark.parametrize("scheme,comp", [("F12F3F4", "strang"), ("F12F4", "lie"), ("F1F2F3F4", "strang")])
def test_split_generalised_padded(scheme, comp):
    pr = W.gdre_convdiff_padded(nx=12, n_pad=160, m=2, p=3)
    N = 8
    flows = W.SCHEMES[scheme]
    plan = plan_for(pr, flows, comp, pr.T / N, prec="split_bf16")
    P = dev(pr.P0)
    plan.step(P, N)
    got = host(P)
    assert rel(got, _oracle_solve(pr, flows, comp, N)) < SPLIT_TOL
    na = pr.meta["n_active"]
    assert np.all(got[na:, :] == 0) and np.all(got[:, na:] == 0)


def test_split_rejects_n_above_4096():
    A = torch.zeros(1, dtype=torch.float64, device="cuda")
    d = dme.make_desc(4097, eq=dme.DME_DLE, flows=("F12",), h=0.1, prec="split_bf16", q_is_factor=True, p=1)
    with pytest.raises(dme.DmeError):
        dme.dme_plan(d, A, A)


def test_split_k_tail_tiles_match_oracle_and_repeat():
    """n = 1664: the full GEMM has 169 tiles, so its last 17 run split in two
    K halves whose sums meet in a workspace; the result must match the oracle
    and repeat bit for bit."""
    n = 1664
    pr = _problem(n, seed=4)
    tau = 0.01
    plan = plan_for(pr, ["F12", "F3"], "strang", tau, prec="split_bf16")
    P0 = W.random_psd(n, 21, rank=32)
    P1, P2 = dev(P0), dev(P0)
    plan.apply("F12", tau, P1)
    plan.apply("F12", tau, P2)
    assert torch.equal(P1, P2)
    E, Wm = O.van_loan(pr.A, pr.Q, tau)
    assert rel(host(P1), O.flow_T12(P0, E, Wm)) < SPLIT_TOL


# ---------------------------------------------------------------- accurate mode (Pade products)
def gemm_split_acc(A, B):
    C = torch.empty(A.shape[0], B.shape[0], dtype=torch.float64, device="cuda")
    dme.dme_gemm_split_acc(dev(A), dev(B), C)
    torch.cuda.synchronize()
    return host(C)


@pytest.mark.parametrize("M,N,K", [(128, 128, 32), (130, 260, 700), (256, 128, 4096), (1, 3, 1)])
def test_accurate_products_of_small_integers_are_exact(M, N, K):
    """Integers in [-63, 63] are one 7-bit digit: every chunk of 512 sums them
    exactly and the chunks add exactly in fp64, so C = A B^T bit for bit
    (K = 700 and 4096 cross chunk boundaries; K = 4096 is eight chunks)."""
    rng = np.random.default_rng(M + 5 * N + 11 * K)
    A = rng.integers(-63, 64, size=(M, K)).astype(np.float64)
    B = rng.integers(-63, 64, size=(N, K)).astype(np.float64)
    A[:, 0] = 63.0
    B[:, 0] = -63.0
    assert np.array_equal(gemm_split_acc(A, B), A @ B.T)


@pytest.mark.parametrize("M,N,K", [(200, 150, 333), (512, 512, 4096)])
def test_accurate_products_reach_two_to_the_minus_39(M, N, K):
    """Six 7-bit slices leave 2^-42 of each row scale; the dropped levels >= 6 and
    the fp32 rounding of the shared level-3 accumulator stay near 2^-39 of the
    row scales' product per term, so |C - AB^T| <= 8 * 2^-39 sA sB sqrt(K)."""
    rng = np.random.default_rng(K + 1)
    A = rng.standard_normal((M, K))
    B = rng.standard_normal((N, K))
    ref = A @ B.T
    C = gemm_split_acc(A, B)
    sa = 2.0 ** np.ceil(np.log2(np.abs(A).max(1) * (1 + 2 ** -52)))
    sb = 2.0 ** np.ceil(np.log2(np.abs(B).max(1) * (1 + 2 ** -52)))
    bound = 8 * 2.0 ** -39 * sa[:, None] * sb[None, :] * math.sqrt(K)
    assert np.all(np.abs(C - ref) <= bound)
    assert rel(C, ref) < 1e-10


# ---------------------------------------------------------------- slice-pair configurations
@pytest.mark.parametrize("pairs", [10, 13, 14])
@pytest.mark.parametrize("n", [37, 300])
def test_every_pair_configuration_matches_oracle(n, pairs):
    pr = _problem(n)
    tau = 0.05
    plan = plan_for(pr, ["F12", "F3", "F4"], "strang", tau, prec="split_bf16", pairs=pairs)
    assert plan.split_choice[0] == pairs
    P0 = W.random_psd(n, 5 + n)
    ref = O.Plan(pr.A, pr.Q, pr.B, pr.R, pr.S)
    for flow in ("F12", "F4"):
        P = dev(P0)
        plan.apply(flow, tau, P)
        assert rel(host(P), ref.apply(flow, tau, P0, "midpoint")) < SPLIT_TOL
        assert torch.equal(P, P.T)


def test_more_pairs_are_more_accurate_on_one_congruence():
    """The one-application error falls as pairs are added (dropped levels and the
    fixed operand's fifth slice), each against the oracle's T12."""
    n = 300
    pr = _problem(n, seed=9)
    tau = 0.05
    P0 = W.random_psd(n, 77)
    E, Wm = O.van_loan(pr.A, pr.Q, tau)
    ref = O.flow_T12(P0, E, Wm)
    errs = {}
    for pairs in (10, 13, 14):
        plan = plan_for(pr, ["F12"], "strang", tau, prec="split_bf16", pairs=pairs)
        P = dev(P0)
        plan.apply("F12", tau, P)
        errs[pairs] = rel(host(P), ref)
        plan.close()
    assert errs[14] <= errs[13] * 1.5 and errs[13] < errs[10]
    assert errs[10] < 1e-8


def test_plan_choice_is_reported_and_within_its_target():
    """pairs = 0: the plan keeps the cheapest configuration whose estimate
    4 N e (N = congruences over the horizon) meets tol; the estimate is reported,
    and the solve over that horizon meets tol against the oracle."""
    pr = W.dre_convdiff()
    N = 64
    flows = W.SCHEMES["F12F3"]
    plan = plan_for(pr, flows, "strang", pr.T / N, prec="split_bf16", horizon=N)
    pairs, est = plan.split_choice
    assert pairs in (10, 13, 14)
    if pairs < 14:
        assert 0 < est <= 1e-7
    errs, rho = plan.split_probe
    k = [10, 13, 14].index(pairs)
    assert all(e > 0 for e in errs[:k + 1]) and all(e == -1 for e in errs[k + 1:])   # tried in order
    assert 0.0 < rho < 1.0                      # the convection-diffusion flow damps
    c = 2                                       # Strang F12F3: two congruences per step
    est_of = lambda e: 4 * e * c * (1 - rho ** N) / (1 - rho)     # noqa: E731
    assert math.isclose(est, est_of(errs[k]), rel_tol=1e-9)
    for q in range(k):
        assert est_of(errs[q]) > 1e-7           # every cheaper configuration missed the target
    P = dev(pr.P0)
    plan.step(P, N)
    assert rel(host(P), _oracle_solve(pr, flows, "strang", N)) < SPLIT_TOL


def test_explicit_pairs_are_validated():
    A = torch.zeros(4, 4, dtype=torch.float64, device="cuda")
    d = dme.make_desc(4, eq=dme.DME_DLE, flows=("F12",), h=0.1, prec="split_bf16", q_is_factor=False, pairs=11)
    with pytest.raises(dme.DmeError):
        dme.dme_plan(d, A, A)


# ---------------------------------------------------------------- Pade chain on the tensor cores
@pytest.mark.parametrize("n,tau", [(600, 0.01), (1024, 1.0 / 512)])
def test_split_plan_exponential_from_tensor_pade_chain(n, tau):
    """Split plans of n >= 512 form the Pade products of E_t and W_t in the
    accurate tensor mode (denominator solves and squarings in FP64): E and W
    stay within 1e-10 of the oracle's 2n x 2n exponential."""
    if n == 1024:
        pr = W.dre_convdiff()
    else:
        pr = _problem(n, seed=2)
    plan = plan_for(pr, ["F12"], "strang", tau, prec="split_bf16")
    E = torch.empty(n, n, dtype=torch.float64, device="cuda")
    Wt = torch.empty_like(E)
    plan.expm(tau, E, Wt)
    Eo, Wo = O.van_loan(pr.A, pr.Q, tau)
    assert rel(host(E), Eo) < 1e-10
    assert rel(host(Wt), Wo) < 1e-10
    assert torch.equal(Wt, Wt.T)
