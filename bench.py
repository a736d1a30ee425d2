"""Benchmark: Strang steps/s of the large dense DRE (n = 4096) on one GB300.

Workload (the metric's configuration): A = 5-point Dirichlet Laplacian on a
64 x 64 grid (n = 4096), B = N(0,1) n x 8, R = I_8, C = U(0,1) 8 x n
(Q = C^T C), P0 = 0, T = 1, h = T/256, Strang F12F3:
T12(h/2) T3(h) T12(h/2) per step.  One step = one pass of the whole hot path
(two congruences E^T P E + W and one Riccati update).  All data are seeded
synthetic inputs; the P, E, W, X working set (4 x 134 MB) exceeds the 129 MB
L2, so no flush is needed between timed steps.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--prec fp64|split|both]
    python bench.py --impl reference      # the CPU FP64 oracle on the same workload

With N > 1 (torchrun) every rank runs an independent replica (the path has no
exchange step); value = steps of all ranks / max over ranks of the time.
Prints ONE JSON line on rank 0.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import dme_workloads as W  # noqa: E402

METRIC = "Strang steps/s at n=4096 (FP64 vs split-prec @1e-7); mixed-n solves/s, p99 ms"
WORKLOAD = ("large dense DRE: 5-point Laplacian 64x64 (n=4096), B 4096x8 N(0,1), R=I_8, C 8x4096 U(0,1), "
            "P0=0, T=1, h=1/256, Strang F12F3")
NOMINAL_FP64_TFLOPS = 1.25    # GB300 FP64 (non-tensor and tensor), the profiling recipe's nominal figure


FP64_MAX_STEPS = 16

# DRAM bytes (read + write) per launch of the tensor kernel in the congruence at n = 4096
# (10 slice products), the mean of its two launches (U = G P: 872.1 + 157.5 MB; the
# triangle G U^T: 657.0 + 121.7 MB), from the ncu capture summarised in
# profiles/ozaki_gemm_n4096_ncu.md; None while the kernel has changed since that capture.
OZAKI_LAUNCH_DRAM_BYTES = 0.5 * ((872.1 + 157.5) + (657.0 + 121.7)) * 1e6


def load_peaks():
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


class ClockSampler:
    """nvidia-smi samples during the timed region (SM clock, throttle reasons)."""
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,clocks_event_reasons.hw_slowdown,"
         "clocks_event_reasons.hw_thermal_slowdown,clocks_event_reasons.sw_thermal_slowdown,"
         "clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                                          "-lms", "200", "-i", str(self.index)], stdout=subprocess.PIPE,
                                         stderr=subprocess.DEVNULL, text=True)
            time.sleep(0.3)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            time.sleep(0.25)
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for name, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    ws = int(os.environ.get("WORLD_SIZE", "1"))
    if ws <= 1:
        return 0, 1, 0, None
    import torch
    import torch.distributed as dist
    rank = int(os.environ["RANK"])
    local = int(os.environ.get("LOCAL_RANK", rank))
    torch.cuda.set_device(local)
    dist.init_process_group("nccl" if torch.cuda.is_available() else "gloo")
    return rank, ws, local, dist


def replica_max_ms(ms_local: float, dist, device=None) -> float:
    """Timed-region length of the slowest rank (every rank runs an independent
    replica; there is no data-path collective, only this timing reduction)."""
    if dist is None:
        return float(ms_local)
    import torch
    t = torch.tensor([float(ms_local)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(steps_per_rank: int, ms_max: float, world_size: int) -> float:
    """Whole-job steps/s: the steps of all replicas over the slowest rank's time."""
    return world_size * steps_per_rank / (ms_max / 1e3)


FP64_NOMINAL_TFLOPS = 1.25     # GB300 FP64 (nominal; no measured figure in the peaks file)


def serving_work(specs):
    """Algorithmic work of the stepping of these requests (Strang F12F3, one
    step = two congruences and T3): FP64 flops 6 n^3 + 3 n^2 m per step (the
    congruence 2 n^3 + n^3 with the symmetric half, Z = P Bt and the update
    of T3); tensor flops of the split path: the same congruences as 6 bf16
    products each (the algorithmic count of the headline roofline), 36 n^3
    per step."""
    f64 = sum(sp["steps"] * (6.0 * sp["n"] ** 3 + 3.0 * sp["n"] ** 2 * sp["m"]) for sp in specs)
    tens = sum(sp["steps"] * 36.0 * sp["n"] ** 3 for sp in specs)
    return f64, tens


def serving_roofline(st, prec, peaks):
    """Fraction of the roofline the served stepping work reaches over a run's wall
    time (planning overlaps it and is not counted as work)."""
    if prec == "fp64":
        ach = st["work_fp64_flops"] / st["wall_s"] / 1e12
        return {"bound": "fp64", "achieved": ach, "peak": FP64_NOMINAL_TFLOPS, "unit": "TFLOP/s",
                "frac": ach / FP64_NOMINAL_TFLOPS, "peak_source": "GB300 FP64 nominal"}
    ach = st["work_tensor_flops"] / st["wall_s"] / 1e12
    pk = peaks["bf16_tflops_sustained"]
    return {"bound": "tensor", "achieved": ach, "peak": pk, "unit": "TFLOP/s", "frac": ach / pk,
            "fp64_equiv_tflops": st["work_fp64_flops"] / st["wall_s"] / 1e12,
            "peak_source": "bf16 dense sustained, MEASURED_PEAKS.json"}


def serving_run(count: int, seed: int, rate: float | None, prec: str = "fp64"):
    """Submit `count` requests of the serving stream (n log-uniform 32..1024,
    Laplacian or stable random A, m, p ~ U{1..8}, T ~ U[0.1, 10], 50-500 Strang
    F12F3 steps) to a server, at Poisson arrival times (rate req/s) or all at
    once (rate None); wait for all.  Returns the server's statistics."""
    import paper_1805_08990_gb300 as dme
    specs = W.serving_requests(count, seed=seed, rate=rate or 1.0)
    probs = [W.materialize(sp) for sp in specs]
    srv = dme.dme_server_create(64 << 30, 32)
    try:
        t0 = time.perf_counter()
        tickets = []
        for sp, pr in zip(specs, probs):
            if rate is not None:
                delay = sp["arrival"] - (time.perf_counter() - t0)
                if delay > 0:
                    time.sleep(delay)
            d = dme.make_desc(pr.n, m=pr.B.shape[1], p=pr.C.shape[0], eq=dme.DME_DRE, comp="strang",
                              flows=("F12", "F3"), h=pr.T / sp["steps"], q_is_factor=True, prec=prec)
            tickets.append((dme.dme_submit(srv, d, pr.A, pr.C, pr.B, pr.R, None, pr.P0, pr.T, sp["steps"]), pr.n))
        for tk, n in tickets:
            out = np.empty((n, n))
            assert dme.dme_poll(srv, tk, out, -1) == dme.DME_OK
        wall = time.perf_counter() - t0
        st = json.loads(dme.dme_server_stats(srv))
        st["wall_s"] = wall
        st["steps_total"] = int(sum(sp["steps"] for sp in specs))
        st["work_fp64_flops"], st["work_tensor_flops"] = serving_work(specs)
        return st
    finally:
        dme.dme_server_destroy(srv)


def serving_stream(count: int, seed: int, rate: float, prec: str):
    """Poisson stream of `count` serving requests at `rate` req/s, each built
    from its spec only when it is submitted; a second thread collects the
    results as they finish.  Returns the server's statistics."""
    import threading
    import paper_1805_08990_gb300 as dme
    specs = W.serving_requests(count, seed=seed, rate=rate)
    srv = dme.dme_server_create(64 << 30, 32)
    tickets: list = []
    cv = threading.Condition()
    failures = []
    busy = [0]

    def reap():
        i = 0
        while i < count:
            with cv:
                while len(tickets) <= i:
                    cv.wait()
                tk, n = tickets[i]
            out = np.empty((n, n))
            if dme.dme_poll(srv, tk, out, -1) != dme.DME_OK:
                failures.append(tk)
            i += 1

    th = threading.Thread(target=reap)
    th.start()
    try:
        t0 = time.perf_counter()
        for sp in specs:
            pr = W.materialize(sp)
            delay = sp["arrival"] - (time.perf_counter() - t0)
            if delay > 0:
                time.sleep(delay)
            d = dme.make_desc(pr.n, m=pr.B.shape[1], p=pr.C.shape[0], eq=dme.DME_DRE, comp="strang",
                              flows=("F12", "F3"), h=pr.T / sp["steps"], q_is_factor=True, prec=prec)
            while True:          # a full queue pushes back: retry until the server takes the request
                try:
                    tk = dme.dme_submit(srv, d, pr.A, pr.C, pr.B, pr.R, None, pr.P0, pr.T, sp["steps"])
                    break
                except dme.DmeError as e:
                    if e.status != dme.DME_EBUSY:
                        raise
                    busy[0] += 1
                    time.sleep(0.005)
            with cv:
                tickets.append((tk, pr.n))
                cv.notify()
        th.join()
        st = json.loads(dme.dme_server_stats(srv))
        st["wall_s"] = time.perf_counter() - t0
        st["client_failures"] = len(failures)
        st["busy_retries"] = busy[0]
        st["work_fp64_flops"], st["work_tensor_flops"] = serving_work(specs)
        return st
    finally:
        dme.dme_server_destroy(srv)


def run_config_suite(args):
    """Steps/s of the other workload configurations (FP64 and split precision),
    with the work per step and the rate it corresponds to: the plain DLE
    (n = 256, Strang F1F2, h = T/100), the DRE order-study operator (n = 1024,
    Strang and Lie F12F3, h = T/256), and the padded generalised DRE (n = 2048,
    Strang F12F3F4, h = T/128).  Device-timed with CUDA events; one line of JSON."""
    import torch
    import paper_1805_08990_gb300 as dme
    from paper_1805_08990_gb300 import build
    build.build()
    dev = torch.device("cuda", 0)
    torch.cuda.set_device(dev)
    stream = torch.cuda.Stream(device=dev)

    def t(x):
        return None if x is None else torch.as_tensor(x, dtype=torch.float64, device=dev)

    cases = [
        ("plain DLE, Laplacian 16x16 (n=256), Strang F1F2, h = T/100", W.dle_heat(), ["F1", "F2"], "strang", 100,
         lambda n: 2 * 3.0 * n ** 3),
        ("DRE, convection-diffusion 32x32 (n=1024), Strang F12F3, h = T/256", W.dre_convdiff(), ["F12", "F3"],
         "strang", 256, lambda n: 2 * 3.0 * n ** 3),
        ("DRE, convection-diffusion 32x32 (n=1024), Lie F12F3, h = T/256", W.dre_convdiff(), ["F12", "F3"], "lie",
         256, lambda n: 3.0 * n ** 3),
        ("GDRE, convection-diffusion 45x45 padded to n=2048, Strang F12F3F4, h = T/128", W.gdre_convdiff_padded(),
         ["F12", "F3", "F4"], "strang", 128, lambda n: 4 * 3.0 * n ** 3),
    ]
    rows = []
    for name, pr, flows, comp, N, flops in cases:
        row = {"workload": name, "n": pr.n}
        for prec, kprec in (("fp64", "fp64"), ("split", "split_bf16")):
            uses_B, uses_S = "F3" in flows, "F4" in flows
            with torch.cuda.stream(stream):
                plan = dme.Plan(t(pr.A), C=t(pr.C), h=pr.T / N, flows=flows, comp=comp,
                                B=t(pr.B) if uses_B else None, R=t(pr.R) if uses_B else None,
                                S=t(pr.S) if uses_S else None, prec=kprec, stream=stream, horizon=N)
            P = torch.zeros(pr.n, pr.n, dtype=torch.float64, device=dev)
            steps = min(N, 32) if prec == "fp64" else N
            plan.step(P, 3)
            torch.cuda.synchronize(dev)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            plan.step(P, steps)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms = e0.elapsed_time(e1) / steps
            row[prec] = {"steps_per_s": 1e3 / ms, "ms_per_step": ms, "kernels_per_step": plan.kernels_per_step,
                         "slice_pairs": plan.split_choice[0],
                         "congruence_flop_per_step": flops(pr.n),
                         "fp64_equivalent_tflops": flops(pr.n) / (ms / 1e3) / 1e12}
            plan.close()
        rows.append(row)
    print(json.dumps({"config_suite": rows, "note": "flop counts are the congruences' 3 n^3 each (P E and the "
                      "upper triangle of E^T X); split rows run slice_pairs bf16 products per congruence flop"}))


def run_serving_suite(args):
    """The serving configuration at several loads: saturation from a burst, then
    Poisson streams at 0.5, 0.9 and 1.2 times it (split precision and FP64)."""
    import torch
    from paper_1805_08990_gb300 import build
    build.build()
    torch.cuda.set_device(0)
    out = {}
    for prec, count, burst_n in (("split_bf16", args.serving_suite, 256),
                                 ("fp64", args.serving_suite_fp64 or max(args.serving_suite // 8, 64), 64)):
        serving_run(8, seed=4, rate=None, prec=prec)       # warm-up (module loading, first launches), untimed
        burst = serving_run(burst_n, seed=1, rate=None, prec=prec)
        sat = burst["completed"] / burst["wall_s"]
        peaks, _ = load_peaks()
        rows = []
        for load in (0.5, 0.9, 1.2):
            st = serving_stream(count, seed=3, rate=load * sat, prec=prec)
            rows.append({"load": load, "offered_per_s": load * sat, "solves_per_s": st["completed"] / st["wall_s"],
                         "p50_ms": st["p50_ms"], "p99_ms": st["p99_ms"], "completed": st["completed"],
                         "failed": st["failed"] + st["client_failures"], "wall_s": st["wall_s"],
                         "graph_builds": st.get("graph_builds"), "rounds": st.get("rounds"),
                         "graph_build_ms": st.get("graph_build_ms"), "round_wait_ms": st.get("round_wait_ms"),
                         "busy_retries": st.get("busy_retries"), "plan_ms_mean": st.get("plan_ms_mean"),
                         "split_pairs_10_13_14": st.get("split_pairs_10_13_14"),
                         "roofline": serving_roofline(st, prec, peaks)})
        out[prec] = {"requests_per_load": count, "saturation_solves_per_s": sat, "burst_requests": burst_n,
                     "burst_plan_ms_mean": burst.get("plan_ms_mean"),
                     "burst_split_pairs_10_13_14": burst.get("split_pairs_10_13_14"),
                     "saturation_roofline": serving_roofline(burst, prec, peaks), "loads": rows}
    if args.serving_oracle > 0:
        out["cpu_baseline"] = serving_oracle_run(args.serving_oracle)
    print(json.dumps({"serving_suite": out, "workload": "n log-uniform 32..1024 (Laplacian or stable random A), "
                      "m, p ~ U{1..8}, R = I_m, T ~ U[0.1, 10], 50-500 Strang F12F3 steps, P0 = 0, Poisson arrivals",
                      "max_slots": 32}))


# ------------------------------------------------------------------ oracle (CPU)
def oracle_steps(pr, nsteps, E=None, Wm=None):
    """Time nsteps oracle Strang F12F3 steps of the workload; returns (seconds, E, W)."""
    import oracle as O
    h = pr.T / 256
    plan = O.Plan(pr.A, pr.Q, pr.B, pr.R)
    if E is None:
        E, Wm = O.van_loan(pr.A, pr.Q, 0.5 * h)
    plan._ew[float(0.5 * h)] = (E, Wm)
    P = np.array(pr.P0)
    t0 = time.perf_counter()
    for _ in range(nsteps):
        P = plan.step(P, "strang", ["F12", "F3"], h)
    return time.perf_counter() - t0, E, Wm


def run_reference(args):
    rank, ws, _, dist = dist_init()
    if rank != 0:
        return 0
    pr = W.dre_heat_large()
    t0 = time.perf_counter()
    _, E, Wm = oracle_steps(pr, 0)
    plan_s = time.perf_counter() - t0
    oracle_steps(pr, args.warmup, E, Wm)
    secs, _, _ = oracle_steps(pr, args.steps, E, Wm)
    v = args.steps / secs
    line = {"impl": "reference", "metric": METRIC, "value": v, "unit": "steps/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * secs / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "impl": "CPU FP64 oracle (numpy/OpenBLAS)"},
            "cpu_baseline": {"value": v, "unit": "steps/s", "cores": os.cpu_count(), "kind": "oracle",
                             "sample": f"{args.steps} oracle Strang F12F3 steps at n=4096 after {args.warmup} "
                                       f"warm-up steps; oracle plan (2n x 2n Pade expm) {plan_s:.1f} s untimed"},
            "e2e": {"value": v, "unit": "steps/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


def serving_oracle_run(count: int, seed: int = 3, n_max: int = 1024):
    """CPU baseline of the serving configuration: the oracle (numpy/OpenBLAS, FP64,
    all host threads) solving the first `count` requests of the same stream
    (seed 3, as the serving suite's Poisson streams) one after another, each
    with its own 2n x 2n exponential for E, W and its Strang F12F3 steps from
    P0 = 0.  A bounded sample: the oracle is slow, the GPU server serves
    10,000 such requests per load."""
    import oracle as O
    specs = W.serving_requests(count, seed=seed, n_max=n_max)
    t_plan = 0.0
    t0 = time.perf_counter()
    for sp in specs:
        pr = W.materialize(sp)
        tp = time.perf_counter()
        plan = O.Plan(pr.A, pr.Q, pr.B, pr.R)
        plan.EW(0.5 * pr.T / sp["steps"])
        t_plan += time.perf_counter() - tp
        O.solve(pr.A, pr.Q, pr.P0, pr.T, sp["steps"], "strang", ["F12", "F3"], B=pr.B, R=pr.R, plan=plan)
    wall = time.perf_counter() - t0
    ns = [sp["n"] for sp in specs]
    return {"value": count / wall, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "wall_s": wall, "plan_s": t_plan, "requests": count,
            "steps_total": int(sum(sp["steps"] for sp in specs)),
            "n_median": float(statistics.median(ns)), "n_max": int(max(ns)),
            "sample": f"the first {count} requests of the serving stream (seed {seed}: n log-uniform "
                      f"32..{n_max}, 50-500 Strang F12F3 steps), solved one after another by the oracle "
                      "with all host threads, its 2n x 2n exponential included"}


# ------------------------------------------------------------------ GPU arm
FULL_STEPS = 256          # the configuration's whole solve: T = 1, h = T/256


def roofline_split(n, avg_ms, pairs, peak, peak_src, traffic, cong_ms, slice_ms):
    """Roofline of the split tensor kernel.  Algorithmic work (the measurement
    table's count for the bf16 split path): 6 bf16 products per FP64 product,
    i.e. per congruence 6 x (2 n^3 + n^3) tensor flops over its two launches
    (P E full, E^T X upper triangle), 9 n^3 per launch on average.  The slice
    products the kernel actually issues (pairs x 3 n^3 per congruence) give the
    tensor-pipe figure, reported beside it as slice_pipe_*."""
    per_launch = 6 * 3.0 * n ** 3 / 2
    achieved = per_launch / (avg_ms / 1e3) / 1e12
    pipe = pairs * 3.0 * n ** 3 / 2 / (avg_ms / 1e3) / 1e12
    return {"bound": "tensor", "achieved": achieved, "peak": peak, "unit": "TFLOP/s", "frac": achieved / peak,
            "traffic": traffic,
            "traffic_of": "dram__bytes_read.sum + dram__bytes_write.sum per launch of the tensor kernel in the "
                          "n = 4096 congruence (mean of U = G P and the triangle G U^T; ncu, "
                          "profiles/ozaki_gemm_n4096_ncu.md); algorithmic bytes per launch: slices of A and B "
                          "268 MB + output 134 MB",
            "kernel": "ozaki_gemm_kernel (tcgen05 kind::f16, 2 launches per congruence)",
            "work": "algorithmic: 6 bf16 products x (2n^3 + n^3) per congruence = 9 n^3 tensor flops per launch",
            "peak_source": f"bf16 dense burst, {peak_src} (MEASURED_PEAKS.json)",
            "avg_launch_ms": avg_ms, "slice_pairs": pairs, "slice_pipe_tflops": pipe, "slice_pipe_frac": pipe / peak,
            "fp64_equivalent_tflops": 3.0 * n ** 3 / (2 * avg_ms / 1e3) / 1e12,
            "congruence_ms": cong_ms, "slice_ms_per_congruence": slice_ms}


def are_residual(P, A, Q, Bt):
    """Relative algebraic Riccati residual ||A^T P + P A + Q - P Bt Bt^T P||_F / ||Q||_F
    (diagnostic of the state at T = 1, computed with torch in float64)."""
    import torch
    Z = P @ Bt
    R = A.T @ P + P @ A + Q - Z @ Z.T
    return (torch.linalg.norm(R) / torch.linalg.norm(Q)).item()


def run_ours(args):
    import torch
    rank, ws, local, dist = dist_init()
    import paper_1805_08990_gb300 as dme
    from paper_1805_08990_gb300 import build
    build.build()
    dev = torch.device("cuda", local)
    torch.cuda.set_device(dev)
    peaks, peaks_src = load_peaks()
    pr = W.dre_heat_large()
    n = pr.n
    K, Wu = args.steps, args.warmup
    h = pr.T / FULL_STEPS
    stream = torch.cuda.Stream(device=dev)

    def to_dev(x):
        return torch.as_tensor(x, dtype=torch.float64, device=dev)

    def barrier():
        if dist is not None:
            dist.barrier()

    def ev():
        return torch.cuda.Event(enable_timing=True)

    results = {}
    states = {}
    precs = ["fp64", "split"] if args.prec == "both" else [args.prec]
    head = "split" if "split" in precs else "fp64"
    for prec in precs:
        kprec = "fp64" if prec == "fp64" else "split_bf16"
        t0 = time.perf_counter()
        with torch.cuda.stream(stream):
            plan = dme.Plan(to_dev(pr.A), C=to_dev(pr.C), h=h, flows=["F12", "F3"], comp="strang",
                            B=to_dev(pr.B), R=to_dev(pr.R), prec=kprec, stream=stream, horizon=FULL_STEPS)
        plan_s = time.perf_counter() - t0
        pairs, pair_est = plan.split_choice
        probe = plan.split_probe if prec == "split" else None
        P = torch.zeros(n, n, dtype=torch.float64, device=dev)
        # the headline (split) arm times exactly K steps; the FP64 comparison arm (about 0.36 s
        # per step at n = 4096) at most FP64_MAX_STEPS of them, reported under its own key
        steps = min(K, FP64_MAX_STEPS) if prec == "fp64" else (args.split_steps or K)
        plan.step(P, Wu)
        torch.cuda.synchronize(dev)
        barrier()
        torch.cuda.synchronize(dev)
        # one CUDA event after every step (graph replays enqueued back to back, no host sync)
        evs = [ev() for _ in range(steps + 1)]
        full = []
        with ClockSampler(local) as clk:
            torch.cuda.nvtx.range_push("timed")
            evs[0].record(stream)
            for i in range(steps):
                plan.step_async(P, 1)
                evs[i + 1].record(stream)
            torch.cuda.synchronize(dev)
            torch.cuda.nvtx.range_pop()
            plan.sync()
            barrier()
            torch.cuda.synchronize(dev)
            if prec == head:
                # the configuration's whole solve (T = 1, 256 steps from P0 = 0), median of
                # args.solve_reps CUDA-event windows enqueued back to back
                for _ in range(args.solve_reps if prec == "split" else 1):
                    a, b = ev(), ev()
                    with torch.cuda.stream(stream):
                        P.zero_()
                    a.record(stream)
                    plan.step_async(P, FULL_STEPS)
                    b.record(stream)
                    full.append((a, b))
                torch.cuda.synchronize(dev)
                plan.sync()
        window_ms = evs[0].elapsed_time(evs[-1])
        per_step = [evs[i].elapsed_time(evs[i + 1]) for i in range(steps)]
        ms = replica_max_ms(window_ms, dist, dev)
        full_ms = [a.elapsed_time(b) for a, b in full]
        if prec != head:
            plan.step(P, FULL_STEPS - Wu - steps)     # continue the same trajectory to T = 1 (untimed)
        torch.cuda.synchronize(dev)
        states[prec] = P.clone()
        kps = plan.kernels_per_step
        # dominant kernel: the congruence E^T P E (+ W) applied alone; the library brackets each of
        # its launches with CUDA events on the plan's stream (profiling mode), read back per kind
        R = 3 if prec == "fp64" else 20
        Pc = P.clone()
        plan.apply_async("F12", 0.5 * h, Pc)
        plan.sync()
        plan.profile(True)
        for kind in range(4):
            plan.timing(kind)
        c0, c1 = ev(), ev()
        c0.record(stream)
        for _ in range(R):
            plan.apply_async("F12", 0.5 * h, Pc)
        c1.record(stream)
        plan.sync()
        plan.profile(False)
        cong_ms = c0.elapsed_time(c1) / R
        kind = dme.DME_KIND_FP64_GEMM if prec == "fp64" else dme.DME_KIND_SPLIT_GEMM
        k_ms, k_launch = plan.timing(kind)
        s_ms, s_launch = plan.timing(dme.DME_KIND_SLICE)
        e2e_s = None
        if prec == head:
            # end to end through the C ABI with host buffers: H2D of P0, K steps, D2H of P(T)
            P0h = torch.zeros(n, n, dtype=torch.float64).pin_memory()
            Ph = torch.empty(n, n, dtype=torch.float64).pin_memory()
            plan.solve(P0h, steps * h, steps, Ph)        # E, W for this h already cached
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            plan.solve(P0h, steps * h, steps, Ph)
            e2e_s = time.perf_counter() - t0
        results[prec] = {"ms": ms, "steps": steps, "kps": kps, "cong_ms": cong_ms, "plan_s": plan_s,
                         "e2e_s": e2e_s, "clocks": clk.summary(), "bytes": plan.nbytes,
                         "kernel_ms": k_ms, "kernel_launches": k_launch, "slice_ms": s_ms, "slice_launches": s_launch,
                         "R": R, "per_step_ms": per_step, "full_ms": full_ms, "pairs": pairs, "pair_est": pair_est,
                         "probe": probe}
        plan.close()

    r = results[head]
    value = replica_value(r["steps"], r["ms"], ws)
    cong_flops = 3.0 * n ** 3          # P E (2n^3) + upper triangle of E^T X (n^3)
    if head == "fp64":
        achieved = cong_flops / (r["cong_ms"] / 1e3) / 1e12
        roof = {"bound": "alu", "achieved": achieved, "peak": NOMINAL_FP64_TFLOPS, "unit": "TFLOP/s",
                "frac": achieved / NOMINAL_FP64_TFLOPS, "traffic": None,
                "kernel": "gemm64_batch_kernel (congruence, 2 launches)",
                "peak_source": "nominal GB300 FP64 rate (profiling recipe table)"}
    else:
        avg_ms = r["kernel_ms"] / max(r["kernel_launches"], 1)
        roof = roofline_split(n, avg_ms, r["pairs"], peaks["bf16_tflops"], peaks_src, OZAKI_LAUNCH_DRAM_BYTES,
                              r["cong_ms"], r["slice_ms"] / max(r["R"], 1))
    med_step = statistics.median(r["per_step_ms"])
    line = {
        "metric": METRIC, "value": value, "unit": "steps/s", "n_gpus": ws, "steps": r["steps"], "warmup": Wu,
        "ms_per_step": r["ms"] / r["steps"], "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
        "dtype": "f64" if head == "fp64" else f"bf16 slices, {r['pairs']} slice products (exact f32 leading level) -> f64",
        "data": "synthetic (seeded generators; no datasets or weights)",
        "config": {"workload": WORKLOAD, "prec": head, "parallelism": f"replicas x{ws}" if ws > 1 else "single GPU",
                   "l2": "working set P,E,W,X = 536 MB > L2 (no flush)", "plan_s": r["plan_s"],
                   "device_bytes": r["bytes"]},
        "roofline": roof,
        "e2e": {"value": r["steps"] / r["e2e_s"], "unit": "steps/s", "h2d_bytes_per_step": 8 * n * n / r["steps"],
                "d2h_bytes_per_step": 8 * n * n / r["steps"],
                "what": f"dme_solve with pinned host P0 and P_out, {r['steps']} steps per call"},
        "gpu_launches": r["kps"] * r["steps"],
        "clocks": r["clocks"],
        "median_step_ms": med_step,
        "median_steps_per_s": 1e3 / med_step,
        "timing": f"value = K steps / one CUDA-event window around K graph replays on the plan's stream; "
                  f"median_step_ms = median of the K per-step event intervals",
    }
    if r["full_ms"]:
        fm = statistics.median(r["full_ms"])
        line["full_solve"] = {"steps": FULL_STEPS, "T": pr.T, "windows": len(r["full_ms"]), "median_ms": fm,
                              "min_ms": min(r["full_ms"]), "max_ms": max(r["full_ms"]),
                              "steps_per_s": FULL_STEPS / (fm / 1e3), "solves_per_s": 1e3 / fm,
                              "what": "P0 = 0 to T = 1 (256 Strang F12F3 steps), median of CUDA-event windows "
                                      "around dme_step_async, clocks sampled over all windows"}
    for prec, rr in results.items():
        line[f"{prec}_steps_per_s"] = replica_value(rr["steps"], rr["ms"], ws)
        line[f"{prec}_steps_timed"] = rr["steps"]
        line[f"{prec}_plan_s"] = rr["plan_s"]
    line["peaks_source"] = peaks_src
    # accuracy at the configuration's horizon: both states are P(T = 1) from P0 = 0 after 256 steps
    Ad, Qd, Bd = to_dev(pr.A), to_dev(pr.Q), to_dev(pr.B)
    acc = {"steps": FULL_STEPS, "T": pr.T}
    for prec, Pt in states.items():
        acc[f"{prec}_are_residual"] = are_residual(Pt, Ad, Qd, Bd)
    if "fp64" in states and "split" in states:
        a, b = states["split"], states["fp64"]
        acc["split_rel_err_vs_fp64"] = (torch.linalg.norm(a - b) / torch.linalg.norm(b)).item()
    if "split" in results:
        acc["split_pairs"] = results["split"]["pairs"]
        acc["split_pair_estimate"] = results["split"]["pair_est"]
        errs, rho = results["split"]["probe"]
        acc["split_probe"] = {"one_congruence_err": {k: e for k, e in zip(("10", "13", "14"), errs) if e >= 0},
                              "step_contraction": rho,
                              "rule": "cheapest pairs with 4 e c (1 + rho + ... + rho^255) <= 1e-7, c = 2 "
                                      "congruences per step"}
    acc["what"] = ("relative Frobenius distance of the split-precision state from the FP64 GPU state at T = 1 "
                   "(256 steps each from P0 = 0; the FP64 path is tied to the oracle at this size by the parity "
                   "tests), and ||A^T P + P A + Q - P B R^-1 B^T P||_F / ||Q||_F of each")
    line["accuracy"] = acc
    if args.extras and rank == 0:
        line["extras"] = extras_run(args, dme, pr, h, to_dev, stream, dev)
    if args.serving_requests > 0:
        line["serving"] = {"requests": args.serving_requests, "scheme": "strang F12F3", "max_slots": 32,
                           "workload": "n log-uniform 32..1024 (Laplacian or stable random A), m,p ~ U{1..8}, "
                                       "T ~ U[0.1,10], 50-500 steps, R = I_m, P0 = 0; burst: all submitted at t=0; "
                                       "live: Poisson arrivals at 0.9x the burst throughput"}
        for prec, kprec in (("fp64", "fp64"), ("split", "split_bf16")):
            serving_run(8, seed=4, rate=None, prec=kprec)      # warm-up, untimed
            burst = serving_run(args.serving_requests, seed=1, rate=None, prec=kprec)
            sat = burst["completed"] / burst["wall_s"]
            live = serving_run(args.serving_requests, seed=2, rate=0.9 * sat, prec=kprec)
            line["serving"][prec] = {
                "saturation_solves_per_s": sat, "poisson_rate": 0.9 * sat,
                "solves_per_s": live["completed"] / live["wall_s"], "p50_ms": live["p50_ms"],
                "p99_ms": live["p99_ms"], "burst_p50_ms": burst["p50_ms"], "burst_p99_ms": burst["p99_ms"],
                "plan_ms_mean": burst.get("plan_ms_mean"), "split_pairs_10_13_14": burst.get("split_pairs_10_13_14"),
                "roofline": serving_roofline(burst, prec, peaks)}
    if rank == 0 and ws == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline_run(pr, args)
    if rank == 0:
        print(json.dumps(line), flush=True)
    if dist is not None:
        dist.destroy_process_group()
    return 0


def cpu_baseline_run(pr, args):
    """The oracle timed on the host cores: its own 2n x 2n exponential for E, W
    (all threads, untimed), then, in a fresh process per thread count (1 and
    nproc, set through OMP/OpenBLAS variables before numpy loads), one warm-up
    Strang F12F3 step and args.cpu_runs timed steps; the median step time."""
    import shutil
    import tempfile
    import oracle as O
    h = pr.T / FULL_STEPS
    t0 = time.perf_counter()
    E, Wm = O.van_loan(pr.A, pr.Q, 0.5 * h)
    plan_s = time.perf_counter() - t0
    d = tempfile.mkdtemp(prefix="dme_oracle_")
    try:
        np.save(os.path.join(d, "E.npy"), E)
        np.save(os.path.join(d, "W.npy"), Wm)
        nproc = os.cpu_count() or 1
        runs = {}
        for threads in (1, nproc):
            env = dict(os.environ)
            for k in ("OMP_NUM_THREADS", "OPENBLAS_NUM_THREADS", "MKL_NUM_THREADS"):
                env[k] = str(threads)
            out = subprocess.run([sys.executable, os.path.abspath(__file__), "--cpu-worker", d,
                                  "--cpu-runs", str(args.cpu_runs)], env=env, capture_output=True, text=True,
                                 timeout=1200)
            if out.returncode != 0:
                raise RuntimeError(f"oracle worker failed: {out.stderr[-400:]}")
            runs[threads] = json.loads(out.stdout.strip().splitlines()[-1])["step_s"]
    finally:
        shutil.rmtree(d, ignore_errors=True)
    med = {t: statistics.median(v) for t, v in runs.items()}
    return {"value": 1.0 / med[nproc], "unit": "steps/s", "cores": nproc, "kind": "oracle",
            "sample": f"the oracle (numpy/OpenBLAS, FP64) on the n = 4096 Strang F12F3 workload: 1 warm-up step, "
                      f"then the median of {args.cpu_runs} single timed steps, in a fresh process per thread "
                      f"count; its own 2n x 2n exponential for E, W ({plan_s:.1f} s, all threads) untimed",
            "single_thread": {"value": 1.0 / med[1], "unit": "steps/s", "cores": 1, "step_s": runs[1]},
            "step_s": runs[nproc]}


def cpu_worker(args):
    """Child process of cpu_baseline_run: time oracle steps with E, W from disk."""
    import oracle as O
    pr = W.dre_heat_large()
    h = pr.T / FULL_STEPS
    E = np.load(os.path.join(args.cpu_worker, "E.npy"))
    Wm = np.load(os.path.join(args.cpu_worker, "W.npy"))
    plan = O.Plan(pr.A, pr.Q, pr.B, pr.R)
    plan._ew[float(0.5 * h)] = (E, Wm)
    P = plan.step(np.array(pr.P0), "strang", ["F12", "F3"], h)        # warm-up
    times = []
    for _ in range(args.cpu_runs):
        t0 = time.perf_counter()
        P = plan.step(P, "strang", ["F12", "F3"], h)
        times.append(time.perf_counter() - t0)
    print(json.dumps({"step_s": times}), flush=True)
    return 0


def extras_run(args, dme, pr, h, to_dev, stream, dev):
    """Separately reported variants of the same workload (never the headline):
    FSAL-merged Strang steps on the split path (same scheme up to rounding), and
    the low-rank factored path (F1F2F3 Strang, no quadrature) with its final rank."""
    import torch
    out = {}
    n = pr.n
    K = args.split_steps or args.steps
    with torch.cuda.stream(stream):
        plan = dme.Plan(to_dev(pr.A), C=to_dev(pr.C), h=h, flows=["F12", "F3"], comp="strang", B=to_dev(pr.B),
                        R=to_dev(pr.R), prec="split_bf16", stream=stream, fsal=True)
    P = torch.zeros(n, n, dtype=torch.float64, device=dev)
    plan.step(P, 4)
    torch.cuda.synchronize(dev)
    e0 = torch.cuda.Event(enable_timing=True)
    e1 = torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    plan.step(P, K)
    e1.record(stream)
    torch.cuda.synchronize(dev)
    out["fsal_split"] = {"steps_per_s": K / (e0.elapsed_time(e1) / 1e3), "steps": K,
                         "what": "Strang F12F3 with T12(h/2) T12(h/2) of neighbouring steps merged into T12(h)"}
    plan.close()
    t0 = time.perf_counter()
    lr = dme.LowRankPlan(to_dev(pr.A), to_dev(pr.C), h=h, flows=["F1", "F2", "F3"], comp="strang",
                         B=to_dev(pr.B), R=to_dev(pr.R), stream=stream)
    plan_s = time.perf_counter() - t0
    N = args.lowrank_steps
    lr.solve(N * h, 4)                    # warm-up (and the rank the state settles at)
    torch.cuda.synchronize(dev)
    t0 = time.perf_counter()
    r = lr.solve(N * h, N)
    torch.cuda.synchronize(dev)
    dt = time.perf_counter() - t0
    out["lowrank_fp64"] = {"steps_per_s": N / dt, "steps": N, "final_rank": r, "plan_s": plan_s,
                           "what": "factored P = L diag(d) L^T, Strang F1F2F3 from P0 = 0, tol 1e-13, "
                                   "host-timed (a rank read-back per compression)"}
    lr.close()
    # the factored path past the dense limit: sparse A, e^{tA^T} L by Leja interpolation
    try:
        nx = args.sparse_nx
        As, Bs, Cs = sparse_problem(nx)
        ns = nx * nx
        hs = 0.01
        t0 = time.perf_counter()
        sl = dme.LowRankPlan.from_csr(As, Cs, h=hs, flows=["F1", "F2", "F3"], comp="strang", B=Bs, R=np.eye(4),
                                      stream=stream)
        plan_s = time.perf_counter() - t0
        sl.solve(4 * hs, 4)
        torch.cuda.synchronize(dev)
        Ns = 8
        t0 = time.perf_counter()
        r = sl.solve(Ns * hs, Ns)
        torch.cuda.synchronize(dev)
        dt = time.perf_counter() - t0
        out["lowrank_sparse_fp64"] = {
            "steps_per_s": Ns / dt, "steps": Ns, "n": ns, "final_rank": r, "plan_s": plan_s,
            "what": f"factored Strang F1F2F3 for the unscaled 5-point stencil on a {nx} x {nx} grid (sparse A, "
                    "e^{tA^T} L by Leja interpolation), B n x 4 N(0,1), R = I, C 2 x n U(0,1), h = 0.01, from P0 = 0"}
        sl.close()
    except Exception as e:            # reported, never fatal to the bench line
        out["lowrank_sparse_fp64"] = {"error": str(e)[:200]}
    # Example 2's shape (stochastic heat transfer: sparse A and S) at the paper's
    # largest size, whole solves T = 1/2 with h = 0.005 (100 steps) from P0 = 0
    for key, control, flows in (("example2_gdre_f12f3f4", True, ["F12", "F3", "F4"]),
                                ("example2_gdle_f1f2f4", False, ["F1", "F2", "F4"])):
        try:
            A2, B2, S2, C2, T2 = W.stochastic_heat_csr(args.example2_nx, control)
            N2 = int(round(T2 / 0.005))
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            p2 = dme.LowRankPlan.from_csr(A2, C2, h=T2 / N2, flows=flows, comp="strang", B=B2,
                                          R=np.eye(1) if control else None, S_csr=S2, stream=stream)
            plan_s = time.perf_counter() - t0
            t0 = time.perf_counter()
            r = p2.solve(T2, N2)
            torch.cuda.synchronize(dev)
            dt = time.perf_counter() - t0
            out[key] = {"solve_s": dt, "plan_s": plan_s, "steps": N2, "n": A2.shape[0], "final_rank": r,
                        "what": f"factored Strang {''.join(flows)} on a {args.example2_nx} x {args.example2_nx} grid "
                                "(sparse A and S, Leja action, quadrature W with 7 nodes), T = 1/2, h = 0.005, "
                                "from P0 = 0; the first solve on a fresh plan (includes its one-off W quadrature)"}
            p2.close()
        except Exception as e:
            out[key] = {"error": str(e)[:200]}
    return out


def sparse_problem(nx):
    """The sparse low-rank extra's DRE: the unscaled 5-point stencil on an nx x nx
    grid, B n x 4 N(0,1), R = I, C 2 x n U(0,1) (seed 0)."""
    import scipy.sparse as sps
    T1 = sps.diags([np.full(nx - 1, 1.0), np.full(nx, -2.0), np.full(nx - 1, 1.0)], [-1, 0, 1])
    I1 = sps.identity(nx)
    As = (sps.kron(I1, T1) + sps.kron(T1, I1)).tocsr()
    rng = np.random.default_rng(0)
    Bs = rng.standard_normal((nx * nx, 4))
    Cs = rng.uniform(0.0, 1.0, (2, nx * nx))
    return As, Bs, Cs


def run_lowrank_only(args):
    """Profile target: one low-rank configuration alone, its timed steps inside the
    NVTX range "lr".  fp64 / split: the large dense DRE (n = 4096, Strang F1F2F3,
    h = 1/256, FP64 or split-precision products), 8 warm-up steps; sparse: the
    sparse DRE of sparse_problem (n = sparse_nx^2, Strang F1F2F3, h = 0.01), 4
    warm-up steps.  Then --lowrank-steps timed steps."""
    import torch
    import paper_1805_08990_gb300 as dme
    from paper_1805_08990_gb300 import build
    build.build()
    mode = args.lowrank_only
    if mode == "sparse":
        As, Bs, Cs = sparse_problem(args.sparse_nx)
        h, warm = 0.01, 4
        lr = dme.LowRankPlan.from_csr(As, Cs, h=h, flows=["F1", "F2", "F3"], comp="strang", B=Bs, R=np.eye(4))
        n = As.shape[0]
    else:
        pr = W.dre_heat_large()
        h, warm = 1.0 / 256, 8
        dev = torch.device("cuda")
        to_dev = lambda x: torch.from_numpy(np.ascontiguousarray(x)).to(dev)   # noqa: E731
        lr = dme.LowRankPlan(to_dev(pr.A), to_dev(pr.C), h=h, flows=["F1", "F2", "F3"], comp="strang",
                             B=to_dev(pr.B), R=to_dev(pr.R), prec="split_bf16" if mode == "split" else "fp64")
        n = pr.n
    lr.solve(warm * h, warm)
    torch.cuda.synchronize()
    N = args.lowrank_steps
    torch.cuda.nvtx.range_push("lr")
    t0 = time.perf_counter()
    r = lr.solve(N * h, N)
    torch.cuda.synchronize()
    dt = time.perf_counter() - t0
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"lowrank_only": mode, "n": n, "steps": N, "ms_per_step": dt / N * 1e3, "rank": r}))
    lr.close()
    return 0


def run_cong_only(args):
    """Profile target: the split plan of the bench workload (n = 4096, its slice
    products chosen for the 256-step horizon, or --pairs) applying one sub-flow
    --reps times to a PSD state, inside the NVTX range "cong": --flow F12 (the
    congruence T12(h/2), E^T P E + W: two tensor-kernel launches) or F3 (the
    Riccati flow: Z^T = Bt^T P and P - t Y Y^T on the tensor kernel)."""
    import torch
    import paper_1805_08990_gb300 as dme
    from paper_1805_08990_gb300 import build
    build.build()
    dev = torch.device("cuda")
    pr = W.dre_heat_large()
    h = pr.T / FULL_STEPS
    t = lambda x: torch.as_tensor(x, dtype=torch.float64, device=dev)   # noqa: E731
    plan = dme.Plan(t(pr.A), C=t(pr.C), h=h, flows=["F12", "F3"], comp="strang", B=t(pr.B), R=t(pr.R),
                    prec="split_bf16", horizon=FULL_STEPS, pairs=args.pairs)
    P = t(W.random_psd(pr.n, 3, rank=64))
    tau = 0.5 * h if args.flow == "F12" else h
    plan.apply(args.flow, tau, P)
    torch.cuda.synchronize()
    torch.cuda.nvtx.range_push("cong")
    t0 = time.perf_counter()
    for _ in range(args.reps):
        plan.apply_async(args.flow, tau, P)
    plan.sync()
    dt = (time.perf_counter() - t0) / args.reps
    torch.cuda.nvtx.range_pop()
    print(json.dumps({"cong_only": pr.n, "flow": args.flow, "pairs": plan.split_choice[0],
                      "ms_per_application": dt * 1e3}))
    plan.close()
    return 0


def run_gemm_only(args):
    """The split-precision tensor-core product alone: C = A B^T, A, B seeded
    N(0,1) of size N x N (inputs and their slices exceed L2 at N = 4096)."""
    import torch
    import paper_1805_08990_gb300 as dme
    from paper_1805_08990_gb300 import build
    build.build()
    N = args.gemm_only
    g = torch.Generator(device="cpu").manual_seed(0)
    A = torch.randn(N, N, generator=g, dtype=torch.float64).cuda()
    B = torch.randn(N, N, generator=g, dtype=torch.float64).cuda()
    C = torch.empty(N, N, dtype=torch.float64, device="cuda")
    dme.dme_gemm_split(A, B, C)
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    for _ in range(args.reps):
        dme.dme_gemm_split(A, B, C)
    torch.cuda.synchronize()
    dt = (time.perf_counter() - t0) / args.reps
    err = (torch.linalg.norm(C - A @ B.T) / torch.linalg.norm(A @ B.T)).item()
    print(json.dumps({"gemm_only": N, "ms_per_call_with_slicing_and_alloc": dt * 1e3, "rel_err_vs_fp64": err}))
    return 0


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=32)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="both", choices=["fp64", "split", "both"])
    ap.add_argument("--split-steps", type=int, default=0, help="override K for the split arm (0: K)")
    ap.add_argument("--cpu-runs", type=int, default=3, help="timed oracle steps per thread count (median)")
    ap.add_argument("--cpu-worker", default="", help=argparse.SUPPRESS)
    ap.add_argument("--solve-reps", type=int, default=10, help="CUDA-event windows of the whole 256-step solve")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--gemm-only", type=int, default=0, help="profile target: split GEMM of this size alone")
    ap.add_argument("--reps", type=int, default=3)
    ap.add_argument("--cong-only", action="store_true", help="profile target: the split congruence at n = 4096")
    ap.add_argument("--pairs", type=int, default=0, help="--cong-only: slice products (0: the plan's choice)")
    ap.add_argument("--flow", default="F12", choices=["F12", "F3"], help="--cong-only: the sub-flow applied")
    ap.add_argument("--lowrank-only", default="", choices=["", "fp64", "split", "sparse"],
                    help="profile target: one low-rank configuration alone (--lowrank-steps timed steps)")
    ap.add_argument("--serving-requests", type=int, default=32, help="serving sample size (0: skip)")
    ap.add_argument("--no-extras", dest="extras", action="store_false", help="skip the FSAL and low-rank lines")
    ap.add_argument("--config-suite", action="store_true",
                    help="run only the steps/s of the other workload configurations")
    ap.add_argument("--serving-suite", type=int, default=0,
                    help="run only the serving loads 0.5/0.9/1.2 x saturation with this many split requests")
    ap.add_argument("--serving-oracle", type=int, default=0,
                    help="--serving-suite: also time the CPU oracle on this many requests of the stream")
    ap.add_argument("--serving-suite-fp64", type=int, default=0,
                    help="FP64 requests per load of the serving suite (0: an eighth of the split count)")
    ap.add_argument("--lowrank-steps", type=int, default=32)
    ap.add_argument("--sparse-nx", type=int, default=1000, help="grid of the sparse low-rank extra (n = nx^2)")
    ap.add_argument("--example2-nx", type=int, default=150, help="grid of the stochastic heat extras (n = nx^2)")
    args = ap.parse_args()
    if args.warmup < 3:
        args.warmup = 3
    if args.cpu_worker:
        return cpu_worker(args)
    if args.impl == "reference":
        return run_reference(args)
    if args.lowrank_only:
        return run_lowrank_only(args)
    if args.gemm_only:
        return run_gemm_only(args)
    if args.cong_only:
        return run_cong_only(args)
    if args.serving_suite:
        return run_serving_suite(args)
    if args.serving_oracle:
        # the serving configuration's CPU baseline alone (no GPU work)
        print(json.dumps({"serving_cpu_baseline": serving_oracle_run(args.serving_oracle)}), flush=True)
        return 0
    if args.config_suite:
        return run_config_suite(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
