"""Host-side argument validation of the C ABI, without a GPU: every case below
is rejected with DME_EINVAL before the library makes any CUDA call, so these
run on a machine with no device.  (The GPU tests cover the checks that need
device data, such as a malformed CSR matrix or a singular mass matrix.)"""
import os
import shutil

import numpy as np
import pytest

import paper_1805_08990_gb300 as dme
from paper_1805_08990_gb300 import build


@pytest.fixture(scope="module", autouse=True)
def _lib():
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("nvcc not available")
    build.build()


N = 6
A = np.zeros((N, N))
C = np.ones((1, N))
B = np.ones((N, 2))
R = np.eye(2)
S = np.eye(N)


def _einval(fn, *args, **kw):
    with pytest.raises(dme.DmeError) as ei:
        fn(*args, **kw)
    assert ei.value.status == dme.DME_EINVAL
    return str(ei.value)


def _desc(**kw):
    base = dict(m=2, p=1, eq=dme.DME_DRE, comp="strang", flows=("F12", "F3"), h=0.1, q_is_factor=True)
    base.update(kw)
    n = base.pop("n", N)
    return dme.make_desc(n, **base)


@pytest.mark.parametrize("kw,msg", [
    (dict(n=0), "n must be"),
    (dict(n=16385), "n must be"),
    (dict(h=0.0), "h must be"),
    (dict(h=float("nan")), "h must be"),
    (dict(eq=dme.DME_DLE), "F3 needs"),                          # F3 without a Riccati term
    (dict(flows=("F12", "F4")), "F4 needs"),                     # F4 without S P S^T
    (dict(m=0), "1 <= m <= 32"),
    (dict(m=33), "1 <= m <= 32"),
])
def test_plan_descriptor_rejections(kw, msg):
    assert msg in _einval(dme.dme_plan, _desc(**kw), A, C, B, R, None)


def test_plan_rejections_by_field():
    d = _desc()
    d.nflows = 0
    assert "nflows" in _einval(dme.dme_plan, d, A, C, B, R, None)
    d = _desc()
    d.flows[1] = 9
    assert "flow id" in _einval(dme.dme_plan, d, A, C, B, R, None)
    d = _desc()
    d.comp = 7
    assert "comp" in _einval(dme.dme_plan, d, A, C, B, R, None)
    d = _desc()
    d.prec = 5
    assert "prec" in _einval(dme.dme_plan, d, A, C, B, R, None)
    d = _desc(eq=dme.DME_GDRE, flows=("F12", "F3", "F4"))
    assert "need S" in _einval(dme.dme_plan, d, A, C, B, R, None)          # S missing
    d = _desc()
    d.extrap = 5
    assert "extrap" in _einval(dme.dme_plan, d, A, C, B, R, None)
    d = _desc(comp="lie")
    d.fsal = 1
    assert "fsal" in _einval(dme.dme_plan, d, A, C, B, R, None)
    d = _desc(eq=dme.DME_GDRE, flows=("F12", "F3", "F4"))
    d.extrap = 2
    assert "extrapolation" in _einval(dme.dme_plan, d, A, C, B, R, S)      # F4 is not an exact flow
    d = _desc(prec="split_bf16", n=4097)
    assert "4096" in _einval(dme.dme_plan, d, A, C, B, R, None)
    d = _desc(prec="split_tf32")
    assert "DME_SPLIT_TF32 is not built" in _einval(dme.dme_plan, d, A, C, B, R, None)


def test_plan_requires_data():
    assert "required" in _einval(dme.dme_plan, _desc(), None, C, B, R, None)
    assert "B, R" in _einval(dme.dme_plan, _desc(), A, C, None, R, None)


def test_lowrank_plan_rejections():
    assert "q_is_factor" in _einval(dme.dme_lr_plan, _desc(q_is_factor=False), A, C, B, R, None)
    d = _desc()
    d.fsal = 1
    assert "fsal" in _einval(dme.dme_lr_plan, d, A, C, B, R, None)
    assert "rmax" in _einval(dme.dme_lr_plan, _desc(), A, C, B, R, None, rmax=500)
    assert "quad_nodes" in _einval(dme.dme_lr_plan, _desc(), A, C, B, R, None, quad_nodes=65)
    assert "p exceeds" in _einval(dme.dme_lr_plan, _desc(p=9), A, np.ones((9, N)), B, R, None, rmax=8)


def test_server_and_solve_rejections():
    assert "max_slots" in _einval(dme.dme_server_create, 1 << 30, 0)
    assert "budget" in _einval(dme.dme_server_create, 0, 4)
    assert "nrhs" in _einval(dme.dme_dense_solve, np.zeros((0, 0)), np.zeros((0, 1)))


def test_split_gemm_bindings_reject_bad_operands_before_any_call():
    """dme_gemm_split and dme_gemm_split_noalloc take only float64 contiguous
    CUDA tensors of matching shapes; anything else is refused on the host
    (a host pointer or a short C_out would otherwise reach device kernels)."""
    import torch
    a = torch.zeros(4, 3, dtype=torch.float64)
    b = torch.zeros(5, 3, dtype=torch.float64)
    c = torch.zeros(4, 5, dtype=torch.float64)
    for f in (dme.dme_gemm_split, dme.dme_gemm_split_noalloc):
        for args in ((a, b, c), (a.numpy(), b, c), (a, b, c.float()), (a, b, c[:, :4]), (a, b[:, :2], c),
                     (a.t(), b, c)):
            with pytest.raises(dme.DmeError) as ei:
                f(*args)
            assert ei.value.status == dme.DME_EINVAL
