"""GB300-native dense splitting schemes for differential Lyapunov and Riccati
equations (Mena, Pfurtscheller & Stillfjord, arXiv:1805.08990).

The compute path is libdme.so (CUDA for sm_103a, C ABI in include/dme.h);
this package only marshals arguments to it.  Importing the package does not
load the library; the first call does, and fails loudly if it is not built.
"""
from .binding import (  # noqa: F401
    DME_DLE, DME_DRE, DME_GDLE, DME_GDRE, DME_F1, DME_F2, DME_F12, DME_F3, DME_F4,
    DME_LIE, DME_STRANG, DME_FP64, DME_SPLIT_TF32, DME_SPLIT_BF16, DME_T4_AUTO, DME_T4_MIDPOINT, DME_T4_EULER,
    DME_KIND_SPLIT_GEMM, DME_KIND_SLICE, DME_KIND_FP64_GEMM, DME_KIND_RICCATI, dme_plan_profile, dme_plan_timing,
    DME_OK, DME_EINVAL, DME_ENOMEM, DME_ENOTSPD, DME_ECUDA, DME_ETIMEOUT, DME_EBUSY, DME_ENOTREADY,
    DmeError, LibraryNotBuilt, dme_plan_desc, make_desc, lib, header_functions,
    dme_plan, dme_plan_mass, dme_lr_plan, dme_lr_plan_csr, dme_lr_solve, dme_lr_factors, dme_lr_destroy, dme_expm, dme_apply, dme_apply_async, dme_sync, dme_plan_kernels_per_step, dme_step, dme_step_async, dme_solve, dme_plan_bytes, dme_plan_split_choice, dme_plan_split_probe, dme_plan_destroy, dme_gain,
    dme_server_create, dme_submit, dme_poll, dme_submit_gain, dme_poll_gain, dme_server_stats, dme_server_destroy,
    dme_last_error,
    dme_gemm_split, dme_gemm_split_acc, dme_gemm_split_noalloc, dme_dense_solve, dme_wait_selftest,
)

EQ_IDS = {"dle": DME_DLE, "dre": DME_DRE, "gdle": DME_GDLE, "gdre": DME_GDRE}


class Plan:
    """Owning wrapper of a dme_plan_t.

    ``Plan(A, C, h, scheme=["F12", "F3"], comp="strang", B=B, R=R)`` with
    Q = C^T C (``q_is_factor``) or ``Q=...`` for a dense Q."""

    def __init__(self, A, C=None, h=1e-3, flows=("F12",), comp="strang", B=None, R=None, S=None,
                 Q=None, prec="fp64", t4_rule=DME_T4_AUTO, pairs=0, stream=None, M=None, fsal=False, extrap=0,
                 horizon=0, tol=0.0):
        n = int(A.shape[0])
        m = 0 if B is None else int(B.shape[1])
        eq = ("g" if S is not None else "") + ("dre" if B is not None else "dle")
        if Q is None and C is None:
            raise ValueError("give C (Q = C^T C) or Q")
        self.n, self.m = n, m
        self.desc = make_desc(n, m=m, p=0 if C is None else int(C.shape[0]), eq=EQ_IDS[eq], comp=comp,
                              flows=flows, prec=prec, h=h, q_is_factor=Q is None, t4_rule=t4_rule, pairs=pairs,
                              fsal=fsal, extrap=extrap, horizon=horizon, tol=tol)
        if M is None:
            self.handle = dme_plan(self.desc, A, C if Q is None else Q, B, R, S, stream)
        else:
            self.handle = dme_plan_mass(self.desc, M, A, C if Q is None else Q, B, R, S, stream)

    def expm(self, t, E_out=None, W_out=None):
        dme_expm(self.handle, t, E_out, W_out)

    def apply(self, flow, t, P):
        dme_apply(self.handle, flow, t, P)

    def apply_async(self, flow, t, P):
        dme_apply_async(self.handle, flow, t, P)

    def sync(self):
        dme_sync(self.handle)

    def profile(self, enable=True):
        dme_plan_profile(self.handle, enable)

    def timing(self, kind):
        return dme_plan_timing(self.handle, kind)

    @property
    def kernels_per_step(self):
        return dme_plan_kernels_per_step(self.handle)

    def step(self, P, nsteps=1):
        dme_step(self.handle, P, nsteps)

    def step_async(self, P, nsteps=1):
        dme_step_async(self.handle, P, nsteps)

    def solve(self, P0, T, nsteps, P_out):
        dme_solve(self.handle, P0, T, nsteps, P_out)

    def gain(self, P, K_out):
        dme_gain(self.handle, P, K_out)

    @property
    def split_choice(self):
        """(slice products per output, estimate that chose them)."""
        return dme_plan_split_choice(self.handle)

    @property
    def split_probe(self):
        """([one-congruence errors of 10, 13, 14 slice products], step contraction)."""
        return dme_plan_split_probe(self.handle)

    @property
    def nbytes(self):
        return dme_plan_bytes(self.handle)

    def close(self):
        if self.handle:
            dme_plan_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class LowRankPlan:
    """Owning wrapper of a dme_lr_t: the factored (LDL^T) schemes.

    ``LowRankPlan(A, C, h, flows=["F12", "F3"], B=B, R=R)``; ``solve(T, N, P_out=P)``
    runs N steps from P0 = L0 D0 L0^T (0 if L0 is None), writes L diag(d) L^T to P_out
    when given, and returns the final rank; ``factors()`` returns (L, d)."""

    def __init__(self, A, C, h=1e-3, flows=("F1", "F2"), comp="strang", B=None, R=None, S=None,
                 t4_rule=DME_T4_AUTO, quad_nodes=0, rmax=0, tol=0.0, stream=None, prec="fp64"):
        n = int(A.shape[0])
        m = 0 if B is None else int(B.shape[1])
        eq = ("g" if S is not None else "") + ("dre" if B is not None else "dle")
        self.n, self.m = n, m
        self.desc = make_desc(n, m=m, p=int(C.shape[0]), eq=EQ_IDS[eq], comp=comp, flows=flows, prec=prec, h=h,
                              q_is_factor=True, t4_rule=t4_rule)
        self.handle = dme_lr_plan(self.desc, A, C, B, R, S, quad_nodes, rmax, tol, stream)

    @classmethod
    def from_csr(cls, A_csr, C, h=1e-3, flows=("F1", "F2"), comp="strang", B=None, R=None, S_csr=None,
                 t4_rule=DME_T4_AUTO, quad_nodes=0, rmax=0, tol=0.0, stream=None):
        """The factored path for a sparse A (and, for the generalised equations,
        a sparse S; scipy.sparse matrices or anything with indptr / indices /
        data): e^{t A^T} L by Leja interpolation, S L by a sparse product."""
        self = cls.__new__(cls)
        A_csr = A_csr.tocsr() if hasattr(A_csr, "tocsr") else A_csr
        n = int(A_csr.shape[0])
        m = 0 if B is None else int(B.shape[1])
        self.n, self.m = n, m
        eq = ("g" if S_csr is not None else "") + ("dre" if B is not None else "dle")
        self.desc = make_desc(n, m=m, p=int(C.shape[0]), eq=EQ_IDS[eq], comp=comp, flows=flows, prec="fp64", h=h,
                              q_is_factor=True, t4_rule=t4_rule)
        s3 = None
        if S_csr is not None:
            S_csr = S_csr.tocsr() if hasattr(S_csr, "tocsr") else S_csr
            s3 = (S_csr.indptr, S_csr.indices, S_csr.data)
        self.handle = dme_lr_plan_csr(self.desc, A_csr.indptr, A_csr.indices, A_csr.data, C, B, R, quad_nodes, rmax,
                                      tol, stream, S_csr=s3)
        return self

    def solve(self, T, nsteps, L0=None, D0=None, P_out=None):
        r0 = 0 if L0 is None else int(L0.shape[1])
        return dme_lr_solve(self.handle, L0, D0, r0, T, nsteps, P_out)

    def factors(self):
        import numpy as np
        r = dme_lr_factors(self.handle)
        L = np.empty((self.n, r))
        d = np.empty(r)
        if r:
            dme_lr_factors(self.handle, L, d)
        return L, d

    def close(self):
        if getattr(self, "handle", None):
            dme_lr_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
