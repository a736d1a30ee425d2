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
    assert tens == 3 * 112 * 10 ** 3 + 50 * 112 * 100 ** 3


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
