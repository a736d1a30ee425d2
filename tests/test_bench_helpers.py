"""Host-side helpers of bench.py (no GPU): the serving work model and its
roofline fraction, the sparse low-rank problem, the peaks file fallback, and
the serving request stream's determinism and ranges."""
import math

import numpy as np
import pytest

import bench
import dme_workloads as W


def test_serving_work_counts_each_request():
    specs = [{"n": 10, "m": 2, "steps": 3}, {"n": 100, "m": 8, "steps": 50}]
    f64, tens = bench.serving_work(specs)
    assert f64 == 3 * (6 * 10 ** 3 + 3 * 10 ** 2 * 2) + 50 * (6 * 100 ** 3 + 3 * 100 ** 2 * 8)
    assert tens == 3 * 36 * 10 ** 3 + 50 * 36 * 100 ** 3


def test_serving_roofline_fractions():
    peaks = {"bf16_tflops_sustained": 1600.0}
    st = {"work_fp64_flops": 2.0e12, "work_tensor_flops": 8.0e14, "wall_s": 2.0}
    r = bench.serving_roofline(st, "split_bf16", peaks)
    assert r["bound"] == "tensor" and math.isclose(r["achieved"], 400.0) and math.isclose(r["frac"], 0.25)
    assert math.isclose(r["fp64_equiv_tflops"], 1.0)
    r = bench.serving_roofline(st, "fp64", peaks)
    assert r["bound"] == "fp64" and math.isclose(r["achieved"], 1.0)
    assert math.isclose(r["frac"], 1.0 / bench.FP64_NOMINAL_TFLOPS)


def test_sparse_problem_is_the_unscaled_stencil():
    nx = 7
    A, B, C = bench.sparse_problem(nx)
    n = nx * nx
    assert A.shape == (n, n) and B.shape == (n, 4) and C.shape == (2, n)
    Ad = A.toarray()
    assert np.allclose(Ad, Ad.T) and np.allclose(np.diag(Ad), -4.0)
    assert np.count_nonzero(Ad) == 5 * n - 4 * nx
    assert np.all(C >= 0.0) and np.all(C <= 1.0)


def test_load_peaks_reports_its_source():
    peaks, src = bench.load_peaks()
    assert src in ("measured", "fallback")
    for k in ("hbm_gbs", "bf16_tflops", "bf16_tflops_sustained"):
        assert peaks[k] > 0


@pytest.mark.parametrize("seed", [0, 3])
def test_serving_stream_is_seeded_and_in_range(seed):
    a = W.serving_requests(200, seed=seed, rate=5.0)
    b = W.serving_requests(200, seed=seed, rate=5.0)
    assert a == b
    arrivals = [s["arrival"] for s in a]
    assert all(x < y for x, y in zip(arrivals, arrivals[1:]))
    for s in a:
        assert 32 <= s["n"] <= 1024 + 64                      # a Laplacian rounds n to nx^2
        assert 1 <= s["m"] <= 8 and 1 <= s["p"] <= 8 and 50 <= s["steps"] <= 500 and 0.1 <= s["T"] <= 10.0
        if s["family"] == "laplacian":
            assert math.isqrt(s["n"]) ** 2 == s["n"]
    # log-uniform n: about half of the requests below the geometric midpoint sqrt(32 * 1024) = 181
    below = sum(s["n"] < 181 for s in a) / len(a)
    assert 0.35 < below < 0.65


def test_split_roofline_counts_the_algorithmic_products():
    """frac uses 6 bf16 products per FP64 product (9 n^3 per launch on average);
    the pairs the kernel issues only enter slice_pipe_*."""
    n, ms = 4096, 0.8312
    r = bench.roofline_split(n, ms, 14, 1920.7, "measured", None, 1.8, 0.12)
    assert math.isclose(r["achieved"], 9.0 * n ** 3 / (ms / 1e3) / 1e12)
    assert math.isclose(r["frac"], r["achieved"] / 1920.7)
    assert 0.38 < r["frac"] < 0.40                      # the figure recomputed by hand for 0.8312 ms
    assert math.isclose(r["slice_pipe_tflops"], 14 / 6 * r["achieved"])
    assert math.isclose(r["fp64_equivalent_tflops"], r["achieved"] / 6)


def test_are_residual_is_zero_at_the_care_solution():
    """The diagnostic is the relative residual of the algebraic Riccati equation:
    zero (to rounding) at scipy's stabilising solution."""
    import scipy.linalg as sl
    import torch
    rng = np.random.default_rng(5)
    n, m = 12, 3
    A = W.laplacian_2d(4) if n == 16 else -np.eye(n) * 3 + 0.3 * rng.standard_normal((n, n))
    Bt = rng.standard_normal((n, m))
    C = rng.uniform(0, 1, (2, n))
    Q = C.T @ C
    X = sl.solve_continuous_are(A, Bt, Q, np.eye(m))
    t = lambda x: torch.as_tensor(x, dtype=torch.float64)    # noqa: E731
    assert bench.are_residual(t(X), t(A), t(Q), t(Bt)) < 1e-12
    assert bench.are_residual(t(X * 1.01), t(A), t(Q), t(Bt)) > 1e-4


def test_serving_oracle_baseline_solves_the_stream_prefix():
    """The serving CPU baseline times the oracle on the first requests of the
    stream; with small n it runs in well under a second here, reports its
    sample and equals the count over its wall time."""
    out = bench.serving_oracle_run(2, seed=3, n_max=40)
    specs = W.serving_requests(2, seed=3, n_max=40)
    assert out["kind"] == "oracle" and out["unit"] == "solves/s" and out["requests"] == 2
    assert out["steps_total"] == sum(sp["steps"] for sp in specs)
    assert out["n_max"] == max(sp["n"] for sp in specs) <= 40
    assert math.isclose(out["value"], 2 / out["wall_s"], rel_tol=1e-12)
    assert 0 <= out["plan_s"] <= out["wall_s"]
