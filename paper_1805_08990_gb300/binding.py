"""ctypes binding of libdme.so (include/dme.h).  Argument marshalling only:
every step of the splitting schemes runs in the library's CUDA kernels.

Matrices are passed as torch tensors (CUDA or CPU) or numpy arrays; they must
be float64 and C-contiguous (they are made so, which copies if needed).  The
library itself decides host vs device per pointer.  There is no fallback:
if libdme.so is missing, every call raises ``LibraryNotBuilt``.
"""
from __future__ import annotations

import ctypes as C
import os
import re
import threading

PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(PKG, "lib", "libdme.so")
HEADER = os.path.join(os.path.dirname(PKG), "include", "dme.h")

DME_OK, DME_EINVAL, DME_ENOMEM, DME_ENOTSPD, DME_ECUDA, DME_ETIMEOUT, DME_EBUSY, DME_ENOTREADY = range(8)
STATUS_NAMES = ["DME_OK", "DME_EINVAL", "DME_ENOMEM", "DME_ENOTSPD", "DME_ECUDA", "DME_ETIMEOUT",
                "DME_EBUSY", "DME_ENOTREADY"]
DME_DLE, DME_DRE, DME_GDLE, DME_GDRE = range(4)
DME_F1, DME_F2, DME_F12, DME_F3, DME_F4 = 1, 2, 3, 4, 5
DME_LIE, DME_STRANG = 1, 2
DME_FP64, DME_SPLIT_TF32, DME_SPLIT_BF16 = 0, 1, 2
DME_T4_AUTO, DME_T4_MIDPOINT, DME_T4_EULER = 0, 1, 2
DME_KIND_SPLIT_GEMM, DME_KIND_SLICE, DME_KIND_FP64_GEMM, DME_KIND_RICCATI = 0, 1, 2, 3

FLOW_IDS = {"F1": DME_F1, "F2": DME_F2, "F12": DME_F12, "F3": DME_F3, "F4": DME_F4}
COMP_IDS = {"lie": DME_LIE, "strang": DME_STRANG}
PREC_IDS = {"fp64": DME_FP64, "split_tf32": DME_SPLIT_TF32, "split_bf16": DME_SPLIT_BF16}


class LibraryNotBuilt(RuntimeError):
    pass


class DmeError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        self.status = status
        name = STATUS_NAMES[status] if 0 <= status < len(STATUS_NAMES) else str(status)
        super().__init__(f"{where}: {name}: {msg}")


class dme_plan_desc(C.Structure):
    _fields_ = [("n", C.c_int), ("m", C.c_int), ("p", C.c_int), ("eq", C.c_int), ("comp", C.c_int),
                ("nflows", C.c_int), ("flows", C.c_int * 4), ("prec", C.c_int), ("h", C.c_double),
                ("q_is_factor", C.c_int), ("t4_rule", C.c_int), ("pairs", C.c_int), ("fsal", C.c_int),
                ("extrap", C.c_int), ("horizon", C.c_int), ("tol", C.c_double)]


class dme_lr_opts(C.Structure):
    _fields_ = [("quad_nodes", C.c_int), ("rmax", C.c_int), ("tol", C.c_double)]


_lib = None
_lock = threading.Lock()

_SIGS = {
    "dme_plan": (C.c_int, [C.POINTER(dme_plan_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                           C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "dme_plan_mass": (C.c_int, [C.POINTER(dme_plan_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                                C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_void_p)]),
    "dme_expm": (C.c_int, [C.c_void_p, C.c_double, C.c_void_p, C.c_void_p]),
    "dme_lr_plan": (C.c_int, [C.POINTER(dme_plan_desc), C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p,
                              C.c_void_p, C.POINTER(dme_lr_opts), C.c_void_p, C.POINTER(C.c_void_p)]),
    "dme_lr_plan_csr": (C.c_int, [C.POINTER(dme_plan_desc), C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.POINTER(dme_lr_opts), C.c_void_p, C.POINTER(C.c_void_p)]),
    "dme_lr_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_double, C.c_int, C.c_void_p,
                               C.POINTER(C.c_int)]),
    "dme_lr_factors": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p, C.POINTER(C.c_int)]),
    "dme_lr_destroy": (C.c_int, [C.c_void_p]),
    "dme_apply": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p]),
    "dme_apply_async": (C.c_int, [C.c_void_p, C.c_int, C.c_double, C.c_void_p]),
    "dme_sync": (C.c_int, [C.c_void_p]),
    "dme_plan_kernels_per_step": (C.c_int, [C.c_void_p]),
    "dme_plan_profile": (C.c_int, [C.c_void_p, C.c_int]),
    "dme_plan_timing": (C.c_int, [C.c_void_p, C.c_int, C.POINTER(C.c_double), C.POINTER(C.c_int)]),
    "dme_step": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dme_step_async": (C.c_int, [C.c_void_p, C.c_void_p, C.c_int]),
    "dme_solve": (C.c_int, [C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.c_void_p]),
    "dme_plan_bytes": (C.c_size_t, [C.c_void_p]),
    "dme_plan_split_choice": (C.c_int, [C.c_void_p, C.POINTER(C.c_int), C.POINTER(C.c_double)]),
    "dme_plan_split_probe": (C.c_int, [C.c_void_p, C.POINTER(C.c_double), C.POINTER(C.c_double)]),
    "dme_gemm_split_acc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dme_gain": (C.c_int, [C.c_void_p, C.c_void_p, C.c_void_p]),
    "dme_plan_destroy": (C.c_int, [C.c_void_p]),
    "dme_server_create": (C.c_int, [C.c_size_t, C.c_int, C.POINTER(C.c_void_p)]),
    "dme_submit": (C.c_int, [C.c_void_p, C.POINTER(dme_plan_desc), C.c_void_p, C.c_void_p, C.c_void_p,
                             C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_uint64)]),
    "dme_poll": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_int64]),
    "dme_submit_gain": (C.c_int, [C.c_void_p, C.POINTER(dme_plan_desc), C.c_void_p, C.c_void_p, C.c_void_p,
                                  C.c_void_p, C.c_void_p, C.c_void_p, C.c_double, C.c_int, C.POINTER(C.c_uint64)]),
    "dme_poll_gain": (C.c_int, [C.c_void_p, C.c_uint64, C.c_void_p, C.c_void_p, C.c_int64]),
    "dme_server_stats": (C.c_char_p, [C.c_void_p]),
    "dme_server_destroy": (C.c_int, [C.c_void_p]),
    "dme_last_error": (C.c_char_p, []),
    "dme_gemm_split": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]),
    "dme_dense_solve": (C.c_int, [C.c_void_p, C.c_int, C.c_void_p, C.c_int, C.c_void_p]),
    "dme_wait_selftest": (C.c_int, [C.POINTER(C.c_int)]),
    "dme_gemm_split_noalloc": (C.c_int, [C.c_int, C.c_int, C.c_int, C.c_void_p, C.c_void_p, C.c_void_p,
                                         C.c_void_p]),
}


def header_functions() -> list[str]:
    """Names of the functions include/dme.h declares."""
    txt = open(HEADER).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(dme_[a-z_]+)\s*\(", txt)))


def lib():
    """Load libdme.so (once).  Raises LibraryNotBuilt if it is absent."""
    global _lib
    if _lib is None:
        with _lock:
            if _lib is None:
                if not os.path.exists(LIB_PATH):
                    raise LibraryNotBuilt(f"{LIB_PATH} is missing: run paper_1805_08990_gb300.build.build()")
                L = C.CDLL(LIB_PATH)
                for name, (res, args) in _SIGS.items():
                    f = getattr(L, name)
                    f.restype = res
                    f.argtypes = args
                _lib = L
    return _lib


def last_error() -> str:
    return (lib().dme_last_error() or b"").decode()


def _check(status: int, where: str):
    if status != DME_OK:
        raise DmeError(status, where, last_error())


def _ptr(x, keep: list):
    """Raw pointer of a float64 C-contiguous matrix (torch tensor or numpy array)."""
    if x is None:
        return None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.float64 or not x.is_contiguous():
                x = x.to(torch.float64).contiguous()
            keep.append(x)
            return x.data_ptr()
    except ImportError:
        pass
    import numpy as np
    a = np.ascontiguousarray(x, dtype=np.float64)
    keep.append(a)
    return a.ctypes.data


def make_desc(n, *, m=0, p=0, eq=DME_DLE, comp="strang", flows=("F12",), prec="fp64", h=1e-3,
              q_is_factor=False, t4_rule=DME_T4_AUTO, pairs=0, fsal=False, extrap=0, horizon=0,
              tol=0.0) -> dme_plan_desc:
    d = dme_plan_desc()
    d.n, d.m, d.p, d.eq = n, m, p, eq
    d.comp = COMP_IDS[comp] if isinstance(comp, str) else comp
    fl = [FLOW_IDS[f] if isinstance(f, str) else f for f in flows]
    d.nflows = len(fl)
    for i, f in enumerate(fl):
        d.flows[i] = f
    d.prec = PREC_IDS[prec] if isinstance(prec, str) else prec
    d.h = float(h)
    d.q_is_factor = int(bool(q_is_factor))
    d.t4_rule = t4_rule
    d.pairs = int(pairs)
    d.fsal = int(bool(fsal))
    d.extrap = int(extrap)
    d.horizon = int(horizon)
    d.tol = float(tol)
    return d


# ------------------------------------------------------------------ C-ABI mirrors
def dme_plan(desc: dme_plan_desc, A, QorC, B=None, R=None, S=None, stream=None) -> int:
    keep: list = []
    out = C.c_void_p()
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().dme_plan(C.byref(desc), _ptr(A, keep), _ptr(QorC, keep), _ptr(B, keep), _ptr(R, keep),
                          _ptr(S, keep), st, C.byref(out)), "dme_plan")
    return out.value


def dme_plan_mass(desc: dme_plan_desc, M, A, QorC, B=None, R=None, S=None, stream=None) -> int:
    keep: list = []
    out = C.c_void_p()
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().dme_plan_mass(C.byref(desc), _ptr(M, keep), _ptr(A, keep), _ptr(QorC, keep), _ptr(B, keep),
                               _ptr(R, keep), _ptr(S, keep), st, C.byref(out)), "dme_plan_mass")
    return out.value


def dme_lr_plan(desc: dme_plan_desc, A, C_factor, B=None, R=None, S=None, quad_nodes=0, rmax=0, tol=0.0,
                stream=None) -> int:
    keep: list = []
    out = C.c_void_p()
    opts = dme_lr_opts(int(quad_nodes), int(rmax), float(tol))
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().dme_lr_plan(C.byref(desc), _ptr(A, keep), _ptr(C_factor, keep), _ptr(B, keep), _ptr(R, keep),
                             _ptr(S, keep), C.byref(opts), st, C.byref(out)), "dme_lr_plan")
    return out.value


def _iptr(x, keep: list):
    """Raw pointer of an int32 C-contiguous array (torch tensor or numpy array)."""
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.int32 or not x.is_contiguous():
                x = x.to(torch.int32).contiguous()
            keep.append(x)
            return x.data_ptr()
    except ImportError:
        pass
    import numpy as np
    a = np.ascontiguousarray(x, dtype=np.int32)
    keep.append(a)
    return a.ctypes.data


def dme_lr_plan_csr(desc: dme_plan_desc, indptr, indices, data, C_factor, B=None, R=None, quad_nodes=0, rmax=0,
                    tol=0.0, stream=None, S_csr=None) -> int:
    """S_csr: (indptr, indices, data) of S for the generalised equations, else None."""
    keep: list = []
    out = C.c_void_p()
    opts = dme_lr_opts(int(quad_nodes), int(rmax), float(tol))
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    nnz = int(len(data))
    nnz_s, sp, si, sv = 0, None, None, None
    if S_csr is not None:
        nnz_s = int(len(S_csr[2]))
        sp = _iptr(S_csr[0], keep)
        si = _iptr(S_csr[1], keep) if nnz_s else None
        sv = _ptr(S_csr[2], keep) if nnz_s else None
    _check(lib().dme_lr_plan_csr(C.byref(desc), nnz, _iptr(indptr, keep), _iptr(indices, keep) if nnz else None,
                                 _ptr(data, keep) if nnz else None, _ptr(C_factor, keep), _ptr(B, keep),
                                 _ptr(R, keep), nnz_s, sp, si, sv, C.byref(opts), st, C.byref(out)),
           "dme_lr_plan_csr")
    return out.value


def dme_lr_solve(plan: int, L0, D0, r0: int, T: float, nsteps: int, P_out=None) -> int:
    keep: list = []
    r = C.c_int(0)
    _check(lib().dme_lr_solve(plan, _ptr(L0, keep) if r0 else None, _ptr(D0, keep) if r0 else None, int(r0),
                              float(T), int(nsteps), _out_ptr(P_out), C.byref(r)), "dme_lr_solve")
    return r.value


def dme_lr_factors(plan: int, L_out=None, d_out=None) -> int:
    r = C.c_int(0)
    _check(lib().dme_lr_factors(plan, _out_ptr(L_out), _out_ptr(d_out), C.byref(r)), "dme_lr_factors")
    return r.value


def dme_lr_destroy(plan: int):
    lib().dme_lr_destroy(plan)


def dme_expm(plan: int, t: float, E_out=None, W_out=None):
    _check(lib().dme_expm(plan, float(t), _out_ptr(E_out), _out_ptr(W_out)), "dme_expm")


def dme_apply(plan: int, flow, t: float, P):
    f = FLOW_IDS[flow] if isinstance(flow, str) else flow
    _check(lib().dme_apply(plan, f, float(t), _out_ptr(P)), "dme_apply")


def dme_apply_async(plan: int, flow, t: float, P):
    f = FLOW_IDS[flow] if isinstance(flow, str) else flow
    _check(lib().dme_apply_async(plan, f, float(t), _out_ptr(P)), "dme_apply_async")


def dme_sync(plan: int):
    _check(lib().dme_sync(plan), "dme_sync")


def dme_plan_kernels_per_step(plan: int) -> int:
    return int(lib().dme_plan_kernels_per_step(plan))


def dme_plan_profile(plan: int, enable: bool):
    _check(lib().dme_plan_profile(plan, int(bool(enable))), "dme_plan_profile")


def dme_plan_timing(plan: int, kind: int):
    """(milliseconds, launches) accumulated for one kernel kind since the last call."""
    ms = C.c_double()
    cnt = C.c_int()
    _check(lib().dme_plan_timing(plan, int(kind), C.byref(ms), C.byref(cnt)), "dme_plan_timing")
    return ms.value, cnt.value


def dme_step(plan: int, P, nsteps: int):
    _check(lib().dme_step(plan, _out_ptr(P), int(nsteps)), "dme_step")


def dme_step_async(plan: int, P, nsteps: int):
    _check(lib().dme_step_async(plan, _out_ptr(P), int(nsteps)), "dme_step_async")


def dme_solve(plan: int, P0, T: float, nsteps: int, P_out):
    keep: list = []
    _check(lib().dme_solve(plan, _ptr(P0, keep), float(T), int(nsteps), _out_ptr(P_out)), "dme_solve")


def dme_gain(plan: int, P, K_out):
    """K_out (m x n) = R^{-1} B^T P, the LQR feedback gain."""
    _check(lib().dme_gain(plan, _out_ptr(P), _out_ptr(K_out)), "dme_gain")


def dme_plan_split_choice(plan: int):
    """(slice products per output, the estimate that chose them) of a plan."""
    pairs = C.c_int(0)
    est = C.c_double(0.0)
    _check(lib().dme_plan_split_choice(plan, C.byref(pairs), C.byref(est)), "dme_plan_split_choice")
    return pairs.value, est.value


def dme_plan_split_probe(plan: int):
    """([err of 10, 13, 14 slice products for one congruence], step contraction rho)."""
    err = (C.c_double * 3)()
    rho = C.c_double(0.0)
    _check(lib().dme_plan_split_probe(plan, err, C.byref(rho)), "dme_plan_split_probe")
    return list(err), rho.value


def dme_plan_bytes(plan: int) -> int:
    return int(lib().dme_plan_bytes(plan))


def dme_plan_destroy(plan: int):
    if plan:
        _check(lib().dme_plan_destroy(plan), "dme_plan_destroy")


def dme_server_create(hbm_budget_bytes: int, max_slots: int) -> int:
    out = C.c_void_p()
    _check(lib().dme_server_create(int(hbm_budget_bytes), int(max_slots), C.byref(out)), "dme_server_create")
    return out.value


def dme_submit(srv: int, desc: dme_plan_desc, A, QorC, B, R, S, P0, T: float, nsteps: int) -> int:
    keep: list = []
    tk = C.c_uint64()
    _check(lib().dme_submit(srv, C.byref(desc), _ptr(A, keep), _ptr(QorC, keep), _ptr(B, keep), _ptr(R, keep),
                            _ptr(S, keep), _ptr(P0, keep), float(T), int(nsteps), C.byref(tk)), "dme_submit")
    return tk.value


def dme_poll(srv: int, ticket: int, P_out=None, timeout_us: int = -1) -> int:
    """Returns DME_OK when done (P_out filled); DME_ENOTREADY / DME_ETIMEOUT otherwise."""
    s = lib().dme_poll(srv, C.c_uint64(ticket), _out_ptr(P_out), C.c_int64(timeout_us))
    if s in (DME_OK, DME_ENOTREADY, DME_ETIMEOUT):
        return s
    raise DmeError(s, "dme_poll", last_error())


def dme_submit_gain(srv: int, desc: dme_plan_desc, A, QorC, B, R, S, P0, T: float, nsteps: int) -> int:
    keep: list = []
    tk = C.c_uint64()
    _check(lib().dme_submit_gain(srv, C.byref(desc), _ptr(A, keep), _ptr(QorC, keep), _ptr(B, keep),
                                 _ptr(R, keep), _ptr(S, keep), _ptr(P0, keep), float(T), int(nsteps), C.byref(tk)),
           "dme_submit_gain")
    return tk.value


def dme_poll_gain(srv: int, ticket: int, P_out=None, K_out=None, timeout_us: int = -1) -> int:
    """As dme_poll; K_out (nsteps x m x n) receives the gains K_k = R^-1 B^T P_k."""
    s = lib().dme_poll_gain(srv, C.c_uint64(ticket), _out_ptr(P_out), _out_ptr(K_out), C.c_int64(timeout_us))
    if s in (DME_OK, DME_ENOTREADY, DME_ETIMEOUT):
        return s
    raise DmeError(s, "dme_poll_gain", last_error())


def dme_server_stats(srv: int) -> str:
    return (lib().dme_server_stats(srv) or b"{}").decode()


def dme_server_destroy(srv: int):
    if srv:
        _check(lib().dme_server_destroy(srv), "dme_server_destroy")


def _gemm_operands(where: str, A, B, C_out):
    """(M, N, K) of C_out = A @ B.T after checking that A (M x K), B (N x K) and
    C_out (M x N) are float64 C-contiguous CUDA tensors on the current device.
    Anything else raises DmeError(DME_EINVAL) before the library is called: a
    host pointer or a smaller C_out would otherwise reach the device kernels,
    and a silent conversion would allocate."""
    import torch

    def bad(msg):
        return DmeError(DME_EINVAL, where, msg)

    for name, x in (("A", A), ("B", B), ("C_out", C_out)):
        if not isinstance(x, torch.Tensor):
            raise bad(f"{name} must be a torch CUDA tensor")
        if x.dtype != torch.float64 or not x.is_contiguous() or x.dim() != 2:
            raise bad(f"{name} must be a contiguous 2-D float64 tensor")
        if not x.is_cuda or x.device.index != torch.cuda.current_device():
            raise bad(f"{name} must live on the current CUDA device")
    M, K = A.shape
    N = B.shape[0]
    if B.shape[1] != K:
        raise bad(f"A is {M} x {K} but B is {tuple(B.shape)}: both need K = {K} columns")
    if tuple(C_out.shape) != (M, N):
        raise bad(f"C_out is {tuple(C_out.shape)}, expected ({M}, {N})")
    return int(M), int(N), int(K)


def dme_gemm_split(A, B, C_out, stream=None):
    """C_out = A @ B.T on the split-precision tensor-core path (device tensors)."""
    M, N, K = _gemm_operands("dme_gemm_split", A, B, C_out)
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().dme_gemm_split(M, N, K, A.data_ptr(), B.data_ptr(), C_out.data_ptr(), st), "dme_gemm_split")


def dme_gemm_split_acc(A, B, C_out, stream=None):
    """C_out = A @ B.T in the accurate split mode (7-bit digits, 6 slices per
    operand, exact K chunks of 512 combined in fp64; device tensors)."""
    M, N, K = _gemm_operands("dme_gemm_split_acc", A, B, C_out)
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().dme_gemm_split_acc(M, N, K, A.data_ptr(), B.data_ptr(), C_out.data_ptr(), st),
           "dme_gemm_split_acc")


def dme_dense_solve(M, B_inout, stream=None):
    """B_inout <- M^{-1} B_inout (Gauss-Jordan with partial pivoting on the
    device; M n x n, B n x nrhs, float64, host or device; M is not modified)."""
    n = int(M.shape[0])
    nrhs = int(B_inout.shape[1]) if len(B_inout.shape) == 2 else 1
    keep: list = []
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().dme_dense_solve(_ptr(M, keep), n, _out_ptr(B_inout), nrhs, st), "dme_dense_solve")


def dme_wait_selftest() -> bool:
    """True when a device wait that can never be satisfied gave up with its
    timeout status (the bounded waits of the persistent kernels)."""
    t = C.c_int(0)
    _check(lib().dme_wait_selftest(C.byref(t)), "dme_wait_selftest")
    return bool(t.value)


def dme_gemm_split_noalloc(A, B, C_out, stream=None):
    """C_out = A @ B.T like dme_gemm_split, with the library's fixed 8 MiB
    device scratch instead of any allocation (see include/dme.h).  The operands
    are passed as they are (never converted or copied)."""
    M, N, K = _gemm_operands("dme_gemm_split_noalloc", A, B, C_out)
    st = None if stream is None else (stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream))
    _check(lib().dme_gemm_split_noalloc(M, N, K, A.data_ptr(), B.data_ptr(), C_out.data_ptr(), st),
           "dme_gemm_split_noalloc")


def dme_last_error() -> str:
    return last_error()


def _out_ptr(x):
    """Pointer of an output buffer, which must already be float64 and contiguous."""
    if x is None:
        return None
    try:
        import torch
        if isinstance(x, torch.Tensor):
            if x.dtype != torch.float64 or not x.is_contiguous():
                raise ValueError("output tensors must be float64 and contiguous")
            return x.data_ptr()
    except ImportError:
        pass
    import numpy as np
    if not (isinstance(x, np.ndarray) and x.dtype == np.float64 and x.flags.c_contiguous):
        raise ValueError("output arrays must be float64 and C-contiguous")
    return x.ctypes.data
