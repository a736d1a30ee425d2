"""Serving (continuous batching with grouped kernels) through the C ABI:
results against the oracle and the single-plan path, bit-identical alone and
in a mix, HBM-budget admission, poll timeouts, and failures made on the host
(a non-SPD R, an over-budget request) that leave the server serving."""
import json
import math
import time

import numpy as np
import pytest
import torch

import dme_workloads as W
import oracle as O
import paper_1805_08990_gb300 as dme
from gpu_util import FP64_TOL, SPLIT_TOL, dev, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


def _desc(pr, nsteps, flows=("F12", "F3"), prec="fp64"):
    ric = "F3" in flows
    return dme.make_desc(pr.n, m=pr.B.shape[1] if ric else 0, p=pr.C.shape[0],
                         eq=dme.DME_DRE if ric else dme.DME_DLE, comp="strang", flows=flows,
                         h=pr.T / nsteps, q_is_factor=True, prec=prec)


def _submit(srv, pr, nsteps, flows=("F12", "F3"), prec="fp64"):
    ric = "F3" in flows
    return dme.dme_submit(srv, _desc(pr, nsteps, flows, prec), pr.A, pr.C, pr.B if ric else None,
                          pr.R if ric else None, None, pr.P0, pr.T, nsteps)


def _poll(srv, tk, n, timeout_us=-1):
    out = np.empty((n, n))
    s = dme.dme_poll(srv, tk, out, timeout_us)
    return s, out


def _requests():
    specs = W.serving_requests(8, seed=5, n_max=160, steps=(5, 12), horizon=(0.1, 1.0))
    return [(W.materialize(sp), sp["steps"]) for sp in specs]


@pytest.fixture
def server():
    srv = dme.dme_server_create(8 << 30, 16)
    yield srv
    dme.dme_server_destroy(srv)


def test_serving_results_match_oracle_and_single_plan(server):
    reqs = _requests()
    tickets = [_submit(server, pr, N) for pr, N in reqs]
    for (pr, N), tk in zip(reqs, tickets):
        s, got = _poll(server, tk, pr.n)
        assert s == dme.DME_OK
        ref = O.solve(pr.A, pr.Q, pr.P0, pr.T, N, "strang", ["F12", "F3"], B=pr.B, R=pr.R)
        assert rel(got, ref) < FP64_TOL
        plan = dme.Plan(dev(pr.A), C=dev(pr.C), h=pr.T / N, flows=["F12", "F3"], B=dev(pr.B), R=dev(pr.R))
        single = np.empty((pr.n, pr.n))
        plan.solve(pr.P0, pr.T, N, single)
        assert np.array_equal(got, single)
    st = json.loads(dme.dme_server_stats(server))
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["p99_ms"] >= st["p50_ms"] > 0
    # rounds ran from captured graphs, and the FP64 tile autotuner saw every group size class
    assert 1 <= st["graph_builds"] <= st["rounds"]
    assert st["tuned_groups"] >= 1


def test_result_is_identical_alone_and_in_a_mix(server):
    target = W.dre_convdiff(nx=11, m=3, p=2, seed=9)
    N = 10
    s, alone = _poll(server, _submit(server, target, N), target.n)
    assert s == dme.DME_OK
    others = _requests()
    tks = [_submit(server, pr, n) for pr, n in others[:3]]
    tk = _submit(server, target, N)
    tks += [_submit(server, pr, n) for pr, n in others[3:]]
    s, mixed = _poll(server, tk, target.n)
    assert s == dme.DME_OK
    assert np.array_equal(alone, mixed)
    for (pr, _), t in zip(others, tks):
        assert _poll(server, t, pr.n)[0] == dme.DME_OK


def test_tiny_budget_admits_one_request_at_a_time():
    reqs = _requests()[:4]
    biggest = max(pr.n for pr, _ in reqs)
    budget = int((6 + 2 + 17) * 8 * biggest * biggest + (1 << 21))
    srv = dme.dme_server_create(budget, 4)
    try:
        tks = [_submit(srv, pr, N) for pr, N in reqs]
        for (pr, N), tk in zip(reqs, tks):
            s, got = _poll(srv, tk, pr.n)
            assert s == dme.DME_OK
            ref = O.solve(pr.A, pr.Q, pr.P0, pr.T, N, "strang", ["F12", "F3"], B=pr.B, R=pr.R)
            assert rel(got, ref) < FP64_TOL
        big = W.dre_convdiff(nx=40)
        with pytest.raises(dme.DmeError) as ei:
            _submit(srv, big, 4)
        assert ei.value.status == dme.DME_ENOMEM
    finally:
        dme.dme_server_destroy(srv)


def test_poll_timeout_and_not_ready(server):
    pr = W.dre_convdiff(nx=32)
    tk = _submit(server, pr, 60)
    s, _ = _poll(server, tk, pr.n, timeout_us=0)
    assert s == dme.DME_ENOTREADY
    s, _ = _poll(server, tk, pr.n, timeout_us=1000)
    assert s == dme.DME_ETIMEOUT
    s, got = _poll(server, tk, pr.n, timeout_us=-1)
    assert s == dme.DME_OK and np.isfinite(got).all()


def test_failed_request_is_reported_and_server_keeps_serving(server):
    bad = W.dre_convdiff(nx=6, m=2, p=2)
    bad.R = -np.eye(2)                       # not SPD: the plan's Cholesky of R fails
    good = W.dre_convdiff(nx=7, m=2, p=2)
    tb = _submit(server, bad, 5)
    tg = _submit(server, good, 5)
    with pytest.raises(dme.DmeError) as ei:
        _poll(server, tb, bad.n)
    assert ei.value.status == dme.DME_ENOTSPD
    s, got = _poll(server, tg, good.n)
    assert s == dme.DME_OK
    ref = O.solve(good.A, good.Q, good.P0, good.T, 5, "strang", ["F12", "F3"], B=good.B, R=good.R)
    assert rel(got, ref) < FP64_TOL
    st = json.loads(dme.dme_server_stats(server))
    assert st["failed"] >= 1


def test_split_precision_requests_in_a_mix(server):
    """Split-precision requests (grouped tcgen05 GEMMs) beside FP64 ones: each
    matches the oracle at its bar, and the split ones equal the single-plan
    split path bit for bit."""
    reqs = _requests()
    precs = ["split_bf16" if i % 2 == 0 else "fp64" for i in range(len(reqs))]
    tickets = [_submit(server, pr, N, prec=pc) for (pr, N), pc in zip(reqs, precs)]
    for (pr, N), pc, tk in zip(reqs, precs, tickets):
        s, got = _poll(server, tk, pr.n)
        assert s == dme.DME_OK
        ref = O.solve(pr.A, pr.Q, pr.P0, pr.T, N, "strang", ["F12", "F3"], B=pr.B, R=pr.R)
        assert rel(got, ref) < (SPLIT_TOL if pc == "split_bf16" else FP64_TOL)
        if pc == "split_bf16":
            # the server gives a request the horizon of its own solve (nsteps steps)
            plan = dme.Plan(dev(pr.A), C=dev(pr.C), h=pr.T / N, flows=["F12", "F3"], B=dev(pr.B), R=dev(pr.R),
                            prec="split_bf16", horizon=N)
            single = np.empty((pr.n, pr.n))
            plan.solve(pr.P0, pr.T, N, single)
            assert np.array_equal(got, single)


def test_submit_rejections(server):
    pr = W.dre_convdiff(nx=5)
    d = _desc(pr, 4)
    d.prec = 7
    with pytest.raises(dme.DmeError):
        dme.dme_submit(server, d, pr.A, pr.C, pr.B, pr.R, None, pr.P0, pr.T, 4)
    with pytest.raises(dme.DmeError):
        dme.dme_submit(server, _desc(pr, 4), pr.A, pr.C, pr.B, pr.R, None, pr.P0, -1.0, 4)
    with pytest.raises(dme.DmeError):
        dme.dme_poll(server, 987654321, None, 0)


def test_back_to_back_requests_get_their_own_round(server):
    """One request at a time, each polled (and freed) before the next is
    submitted: every result equals its single-plan solve bit for bit (a round
    captured for an earlier request must never serve a later one, even when the
    later request's bookkeeping lands at the freed address)."""
    for k in range(6):
        pr = W.dre_convdiff(nx=7, m=2, p=2, seed=20 + k)
        N = 4 + k % 3
        s, got = _poll(server, _submit(server, pr, N), pr.n)
        assert s == dme.DME_OK
        plan = dme.Plan(dev(pr.A), C=dev(pr.C), h=pr.T / N, flows=["F12", "F3"], B=dev(pr.B), R=dev(pr.R))
        single = np.empty((pr.n, pr.n))
        plan.solve(pr.P0, pr.T, N, single)
        assert np.array_equal(got, single), k


def test_gain_history_in_serving(server):
    """dme_submit_gain: the gains K_k = R^-1 B^T P_k after every step, recorded on
    the device inside the captured rounds; against the single plan's states and
    its dme_gain (bit for bit) and against the oracle's gain of the oracle's
    states; a mix of gain and plain requests; a DLE is refused."""
    pr = W.dre_convdiff(nx=8, m=3, p=2, seed=4)
    N = 6
    d = _desc(pr, N)
    tk = dme.dme_submit_gain(server, d, pr.A, pr.C, pr.B, pr.R, None, pr.P0, pr.T, N)
    others = [_submit(server, q, n) for q, n in _requests()[:3]]
    Pout = np.empty((pr.n, pr.n))
    K = np.empty((N, pr.B.shape[1], pr.n))
    assert dme.dme_poll_gain(server, tk, Pout, K, -1) == dme.DME_OK
    plan = dme.Plan(dev(pr.A), C=dev(pr.C), h=pr.T / N, flows=["F12", "F3"], B=dev(pr.B), R=dev(pr.R))
    P = dev(pr.P0)
    Kk = torch.empty(pr.B.shape[1], pr.n, dtype=torch.float64, device=P.device)
    Po = pr.P0.copy()
    for k in range(N):
        plan.step(P, 1)
        plan.gain(P, Kk)
        assert np.array_equal(K[k], Kk.cpu().numpy()), k
        Po = O.solve(pr.A, pr.Q, Po, pr.T / N, 1, "strang", ["F12", "F3"], B=pr.B, R=pr.R)
        ref = O.lqr_gain(Po, pr.B, pr.R)
        assert rel(K[k], ref) < FP64_TOL
    assert np.array_equal(Pout, P.cpu().numpy())
    for t in others:
        assert dme.dme_poll(server, t, None, -1) == dme.DME_OK
    dl = W.dle_heat(nx=5)
    with pytest.raises(dme.DmeError):
        dme.dme_submit_gain(server, _desc(dl, 4, flows=("F12",)), dl.A, dl.C, None, None, None, dl.P0, dl.T, 4)
