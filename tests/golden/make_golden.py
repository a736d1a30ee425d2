"""Writes the golden fixtures of this folder.  Calls only the CPU oracle
(``oracle/``) and the closed form below; nothing here runs the CUDA path.

    python tests/golden/make_golden.py

* scalar_dre.txt: the scalar DRE p' = 2 a p + q - (b^2 / r) p^2, p(0) = 0
  (Eq. ricc with n = m = 1), its exact solution
  p(t) = q tanh(beta t) / (beta - a tanh(beta t)), beta = sqrt(a^2 + q b^2 / r)
  (separation of variables), and the oracle's Lie and Strang F12F3 results
  (§2) for N = 8, 16, 32, 64 steps on [0, T].
* dle_laplacian_n9.txt: the DLE of the 5-point Laplacian on a 3 x 3 grid
  (Example 1's operator, Eq. lyap), Q = C^T C with C a row of ones, P0 = 0,
  T = 0.1, the oracle's F12 result after 10 steps (F12 is the exact flow of
  the DLE, Eq. full), all 81 entries row by row.
"""
import math
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))

import dme_workloads as W  # noqa: E402
import oracle as O  # noqa: E402

SCALAR = dict(a=-1.0, b=1.0, q=2.0, r=1.0, T=1.0)


def scalar_exact(a, b, q, r, T):
    beta = math.sqrt(a * a + q * b * b / r)
    th = math.tanh(beta * T)
    return q * th / (beta - a * th)


def main():
    a, b, q, r, T = (SCALAR[k] for k in ("a", "b", "q", "r", "T"))
    A, B, R = np.array([[a]]), np.array([[b]]), np.array([[r]])
    Q = np.array([[q]])
    lines = ["# scalar DRE p' = 2 a p + q - (b^2/r) p^2, p(0) = 0 (Eq. ricc, n = m = 1)",
             "# exact: p(T) = q tanh(beta T) / (beta - a tanh(beta T)), beta = sqrt(a^2 + q b^2 / r)",
             "# written by tests/golden/make_golden.py from the CPU oracle",
             f"params a={a!r} b={b!r} q={q!r} r={r!r} T={T!r}",
             f"exact {scalar_exact(a, b, q, r, T)!r}"]
    for comp in ("lie", "strang"):
        for N in (8, 16, 32, 64):
            P = O.solve(A, Q, np.zeros((1, 1)), T, N, comp, ["F12", "F3"], B=B, R=R)
            lines.append(f"{comp} F12F3 N={N} {float(P[0, 0])!r}")
    with open(os.path.join(HERE, "scalar_dre.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")

    pr = W.dle_heat(nx=3, T=0.1)
    P = O.solve(pr.A, pr.Q, pr.P0, pr.T, 10, "strang", ["F12"])
    out = ["# DLE of the 5-point Laplacian on a 3 x 3 grid (Eq. lyap), Q = C^T C, C = row of ones,",
           "# P0 = 0, T = 0.1, 10 steps of F12 (the exact flow, Eq. full); P(T) row by row",
           "# written by tests/golden/make_golden.py from the CPU oracle"]
    out += [" ".join(repr(float(v)) for v in row) for row in P]
    with open(os.path.join(HERE, "dle_laplacian_n9.txt"), "w") as f:
        f.write("\n".join(out) + "\n")


if __name__ == "__main__":
    main()
