"""Helpers for the GPU parity tests (CUDA path through the C ABI vs oracle)."""
from __future__ import annotations

import numpy as np
import torch

import paper_1805_08990_gb300 as dme
from paper_1805_08990_gb300 import build

FP64_TOL = 1e-11      # relative Frobenius error bound of the FP64 path
SPLIT_TOL = 1e-7      # relative Frobenius error bound of the split-precision path

_built = False


def require_gpu():
    global _built
    assert torch.cuda.is_available(), "GPU tests need a CUDA device"
    if not _built:
        build.build()
        _built = True


def dev(x):
    return torch.as_tensor(np.ascontiguousarray(x), dtype=torch.float64, device="cuda")


def host(t):
    return t.detach().cpu().numpy()


def rel(x, y):
    x = np.asarray(x)
    y = np.asarray(y)
    d = np.linalg.norm(x - y)
    r = np.linalg.norm(y)
    return float(d / r) if r > 0 else float(d)


def plan_for(pr, flows, comp, h, prec="fp64", t4_rule=dme.DME_T4_AUTO, pairs=0, fsal=False, extrap=0, horizon=0):
    """A dme plan for a dme_workloads.Problem with Q = C^T C."""
    return dme.Plan(dev(pr.A), C=dev(pr.C), h=h, flows=flows, comp=comp,
                    B=None if pr.B is None or "F3" not in flows else dev(pr.B),
                    R=None if pr.R is None or "F3" not in flows else dev(pr.R),
                    S=None if pr.S is None or "F4" not in flows else dev(pr.S),
                    prec=prec, t4_rule=t4_rule, pairs=pairs, fsal=fsal, extrap=extrap,
                    horizon=horizon)
