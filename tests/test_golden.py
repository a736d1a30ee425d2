"""The golden fixtures of tests/golden/ (written by tests/golden/make_golden.py
from the CPU oracle and the scalar closed form; see their headers): the oracle
still reproduces them, the stored scheme values converge to the stored exact
value at the orders the splittings have (§2: Lie 1, Strang 2), and the stored
DLE state agrees with the exact solution in the sine basis.  The GPU
counterparts are in test_gpu_fp64.py."""
import math
import os

import numpy as np

import dme_workloads as W
import oracle as O
import pins

GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def load_scalar():
    vals, params, exact = {}, {}, None
    for ln in open(os.path.join(GOLDEN, "scalar_dre.txt")):
        if ln.startswith("#") or not ln.strip():
            continue
        parts = ln.split()
        if parts[0] == "params":
            params = {k: float(v) for k, v in (p.split("=") for p in parts[1:])}
        elif parts[0] == "exact":
            exact = float(parts[1])
        else:
            vals[(parts[0], int(parts[2].split("=")[1]))] = float(parts[3])
    return params, exact, vals


def load_dle():
    rows = [ln.split() for ln in open(os.path.join(GOLDEN, "dle_laplacian_n9.txt")) if not ln.startswith("#")]
    return np.array([[float(v) for v in r] for r in rows if r])


def test_scalar_golden_exact_is_the_closed_form():
    p, exact, _ = load_scalar()
    assert abs(exact - pins.scalar_dre_exact(p["a"], p["b"], p["q"], p["r"], p["T"])) < 1e-15


def test_scalar_golden_orders():
    _, exact, vals = load_scalar()
    for comp, order in (("lie", 1), ("strang", 2)):
        errs = [abs(vals[(comp, N)] - exact) for N in (8, 16, 32, 64)]
        for e0, e1 in zip(errs, errs[1:]):
            assert abs(math.log2(e0 / e1) - order) < 0.15


def test_oracle_reproduces_scalar_golden():
    p, _, vals = load_scalar()
    A, B, R = np.array([[p["a"]]]), np.array([[p["b"]]]), np.array([[p["r"]]])
    Q = np.array([[p["q"]]])
    for (comp, N), v in vals.items():
        got = O.solve(A, Q, np.zeros((1, 1)), p["T"], N, comp, ["F12", "F3"], B=B, R=R)[0, 0]
        assert abs(got - v) <= 1e-14 * abs(v)


def test_dle_golden_is_exact_and_reproduced():
    P = load_dle()
    pr = W.dle_heat(nx=3, T=0.1)
    assert P.shape == (9, 9) and np.array_equal(P, P.T)
    got = O.solve(pr.A, pr.Q, pr.P0, pr.T, 10, "strang", ["F12"])
    assert np.abs(got - P).max() <= 1e-14 * np.abs(P).max()
    # F12 is the exact flow: the stored state is the DLE's solution.  With A = S / dx^2 (S the
    # unscaled stencil), P(t) = dx^2 P_S(t / dx^2), P_S the sine-basis closed form for S.
    dx2 = (1.0 / 4.0) ** 2
    ref = dx2 * pins.dle_exact_apply_stencil_laplacian(3, np.ones(9), 0.1 / dx2, np.eye(9))
    assert np.abs(ref - P).max() <= 1e-13 * np.abs(P).max()
