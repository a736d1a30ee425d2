"""Observed convergence orders on the GPU at the DRE order-study size (n = 1024
convection-diffusion, T = 1): Lie F12F3 order 1, Strang F12F3 order 2, against a
GPU reference 16x finer than the finest step of the sweep.  Split precision (its error, <= 1e-9 here, is far below the
splitting errors measured).  The extrapolated scheme is checked for its gain over
Strang (its order 4 is pinned on smooth problems in the oracle tests)."""
import math

import numpy as np
import pytest

import dme_workloads as W
from gpu_util import dev, host, plan_for, rel, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(autouse=True, scope="module")
def _gpu():
    require_gpu()


@pytest.fixture(scope="module")
def problem():
    return W.dre_convdiff()          # n = 1024, B 1024 x 2, C 3 x 1024, T = 1


def _solve(pr, comp, N, extrap=0):
    plan = plan_for(pr, ["F12", "F3"], comp, pr.T / N, prec="split_bf16", extrap=extrap)
    P = dev(pr.P0)
    plan.step(P, N)
    return host(P)


@pytest.fixture(scope="module")
def reference(problem):
    return _solve(problem, "strang", 4096)


def _orders(errs):
    return [math.log2(errs[i] / errs[i + 1]) for i in range(len(errs) - 1)]


@pytest.mark.parametrize("comp,order,Ns", [("lie", 1.0, (32, 64, 128, 256)), ("strang", 2.0, (32, 64, 128, 256))])
def test_observed_order(problem, reference, comp, order, Ns):
    errs = [rel(_solve(problem, comp, N), reference) for N in Ns]
    ords = _orders(errs)
    assert abs(ords[-1] - order) < 0.25, (errs, ords)
    assert all(o > order - 0.45 for o in ords), (errs, ords)


def test_extrapolated_strang_on_the_stiff_problem(problem):
    """Extrapolated Strang (q = 2) is order 4 on smooth problems (oracle pins);
    on this stiff convection-diffusion DRE it shows order reduction to about
    2.4 (the oracle shows the same at n = 100), while still beating plain Strang
    at the same step by an order of magnitude."""
    ref = _solve(problem, "strang", 256, extrap=2)
    errs = [rel(_solve(problem, "strang", N, extrap=2), ref) for N in (8, 16, 32)]
    ords = _orders(errs)
    assert all(o > 2.0 for o in ords), (errs, ords)
    plain = rel(_solve(problem, "strang", 32), ref)
    assert errs[-1] < plain / 4, (errs, plain)
