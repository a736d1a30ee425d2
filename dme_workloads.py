"""Seeded synthetic inputs for the differential matrix equations
dP/dt = A^T P + P A + Q + G(P)   (Mena, Pfurtscheller & Stillfjord, §1).

This module only builds problem data (A, B, R, C, S, P0, horizons, arrival
streams).  It holds none of the splitting method's arithmetic, and it is the
one module that both the CUDA path's tests/bench and the CPU oracle import.

All randomness comes from ``numpy.random.default_rng(seed)`` (PCG64); the
order of the draws is fixed in each generator so a seed names one input.

Matrices are float64, C-contiguous, row-major, index ``i + nx*j`` for grid
point (x_i, y_j) (x fastest), which is the lexicographic ordering of the
5-point finite-difference discretisation of Example 1 (§5.1.1).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field

import numpy as np

__all__ = [
    "laplacian_2d", "convection_diffusion_2d", "zero_pad", "Problem",
    "dle_heat", "dre_convdiff", "gdre_convdiff_padded", "dre_heat_large",
    "random_psd", "serving_requests", "materialize", "fe_heat_mass", "SCHEMES",
    "stochastic_heat_csr", "gdre_stochastic_heat",
]


def _tridiag(nx: int, lo: float, mid: float, hi: float) -> np.ndarray:
    T = np.zeros((nx, nx))
    idx = np.arange(nx)
    T[idx, idx] = mid
    T[idx[1:], idx[:-1]] = lo
    T[idx[:-1], idx[1:]] = hi
    return T


def laplacian_2d(nx: int) -> np.ndarray:
    """5-point Dirichlet Laplacian on the unit square, nx interior points per
    direction, dx = 1/(nx+1):  A = (T (x) I + I (x) T)/dx^2, T = tridiag(1,-2,1)
    (Example 1, §5.1.1).  Symmetric negative definite, n = nx^2."""
    dx = 1.0 / (nx + 1)
    T = _tridiag(nx, 1.0, -2.0, 1.0)
    I = np.eye(nx)
    return (np.kron(I, T) + np.kron(T, I)) / (dx * dx)


def convection_diffusion_2d(nx: int, v=(10.0, 10.0)) -> np.ndarray:
    """u_t = Laplace(u) - v . grad(u) with centred differences, Dirichlet
    boundary, nx interior points per direction:
    A = Lap - (v_x D_x + v_y D_y),  D = tridiag(-1, 0, 1)/(2 dx).
    The convection part is skew-symmetric, so A + A^T = 2 Lap < 0."""
    dx = 1.0 / (nx + 1)
    D1 = _tridiag(nx, -1.0, 0.0, 1.0) / (2.0 * dx)
    I = np.eye(nx)
    Dx = np.kron(I, D1)          # acts on the x index (fastest)
    Dy = np.kron(D1, I)
    return laplacian_2d(nx) - (v[0] * Dx + v[1] * Dy)


def zero_pad(M: np.ndarray, rows: int, cols: int) -> np.ndarray:
    out = np.zeros((rows, cols))
    out[: M.shape[0], : M.shape[1]] = M
    return out


def random_psd(n: int, seed: int, rank: int | None = None, scale: float = 1.0) -> np.ndarray:
    """A seeded symmetric positive semi-definite matrix G G^T * scale/k with
    G ~ U(0,1) of size n x k (k = rank or n): a stand-in state P for
    single-step checks.  Entrywise positive, like the DLE/DRE solutions with
    Q = C^T C, C >= 0 and a heat-kernel e^{tA}."""
    rng = np.random.default_rng(seed)
    k = n if rank is None else rank
    G = rng.uniform(0.0, 1.0, size=(n, k))
    P = (G @ G.T) * (scale / max(k, 1))
    return 0.5 * (P + P.T)


# Scheme names follow the paper's legend convention (§5.2): flows listed in the
# order they are applied.  Strang "Fa Fb Fc" = T_a(h/2) T_b(h/2) T_c(h) T_b(h/2) T_a(h/2).
SCHEMES = {
    "F12": ["F12"], "F1F2": ["F1", "F2"],
    "F12F3": ["F12", "F3"], "F1F2F3": ["F1", "F2", "F3"], "F1F3F2": ["F1", "F3", "F2"],
    "F12F4": ["F12", "F4"], "F1F2F4": ["F1", "F2", "F4"], "F1F4F2": ["F1", "F4", "F2"],
    "F12F3F4": ["F12", "F3", "F4"], "F12F4F3": ["F12", "F4", "F3"],
    "F1F2F3F4": ["F1", "F2", "F3", "F4"],
}


@dataclass
class Problem:
    """One DLE/DRE/GDLE/GDRE instance.  Q = C^T C.  B, R, S may be None."""
    name: str
    A: np.ndarray
    C: np.ndarray
    P0: np.ndarray
    T: float
    B: np.ndarray | None = None
    R: np.ndarray | None = None
    S: np.ndarray | None = None
    meta: dict = field(default_factory=dict)

    @property
    def n(self) -> int:
        return self.A.shape[0]

    @property
    def Q(self) -> np.ndarray:
        return self.C.T @ self.C


def dle_heat(nx: int = 16, T: float = 0.1, seed: int = 0) -> Problem:
    """Plain DLE: Laplacian (n = nx^2), C = 1 x n row of ones (Q = all-ones),
    P0 = 0, T = 0.1.  Default nx = 16 gives n = 256."""
    n = nx * nx
    A = laplacian_2d(nx)
    C = np.ones((1, n))
    return Problem("dle_heat", A, C, np.zeros((n, n)), T, meta={"nx": nx, "seed": seed})


def dre_convdiff(nx: int = 32, m: int = 2, p: int = 3, T: float = 1.0, seed: int = 0) -> Problem:
    """DRE on the convection-diffusion operator, v = (10, 10):
    B = n x m N(0,1), R = I_m, C = p x n U(0,1), P0 = 0, T = 1.
    Draw order: B then C.  Default nx = 32 gives n = 1024."""
    n = nx * nx
    rng = np.random.default_rng(seed)
    A = convection_diffusion_2d(nx)
    B = rng.standard_normal((n, m))
    C = rng.uniform(0.0, 1.0, size=(p, n))
    return Problem("dre_convdiff", A, C, np.zeros((n, n)), T, B=B, R=np.eye(m),
                   meta={"nx": nx, "seed": seed})


def gdre_convdiff_padded(nx: int = 45, n_pad: int = 2048, m: int = 4, p: int = 5,
                         s_scale: float = 0.1, T: float = 1.0, seed: int = 0) -> Problem:
    """Generalised DRE: convection-diffusion on an nx x nx grid (2025 unknowns
    at nx = 45) zero-padded to n_pad; S = s_scale * N(0,1)/sqrt(n_pad) dense on
    the active block; B = N(0,1) n x m; R = I_m; C = U(0,1) p x n; P0 = 0.
    Padded rows/columns of A, B, C and S are zero.  Draw order: S, B, C."""
    na = nx * nx
    n = max(n_pad, na)
    rng = np.random.default_rng(seed)
    S_a = s_scale * rng.standard_normal((na, na)) / math.sqrt(n)
    B_a = rng.standard_normal((na, m))
    C_a = rng.uniform(0.0, 1.0, size=(p, na))
    A = zero_pad(convection_diffusion_2d(nx), n, n)
    return Problem("gdre_convdiff_padded", A, zero_pad(C_a, p, n), np.zeros((n, n)), T,
                   B=zero_pad(B_a, n, m), R=np.eye(m), S=zero_pad(S_a, n, n),
                   meta={"nx": nx, "n_active": na, "seed": seed})


def stochastic_heat_csr(nx: int, control: bool = True):
    """Sparse data in the shape of the stochastic heat transfer problem of
    Example 2 (§5.1.2), on an nx x nx interior grid (dx = 1/(nx+1), n = nx^2):
    no randomness is drawn.

    * Laplacian with homogeneous Dirichlet conditions on the south (j = 0) and
      north (j = nx-1) edges.
    * West edge (i = 0): the control enters as the boundary value x = u, so
      B (n x 1) holds 1/dx^2 in the west-edge rows.  Without control (the
      generalised DLE of the example) B is None and that edge is homogeneous
      Dirichlet, which leaves A unchanged.
    * East edge (i = nx-1): the Robin condition n . grad x = 0.5 (0.5 + dW/dt) x
      with a ghost value; its deterministic part gives the diagonal
      (-3 + 0.25 dx)/dx^2 there, its noise part S = diag(0.5/dx) on the
      east-edge rows (nx nonzeros), zero elsewhere.
    * C = (1/n) (1, ..., 1), the mean; T = 1/2.

    Returns (A, B, S, C, T) with A and S scipy.sparse CSR matrices."""
    import scipy.sparse as sp
    n = nx * nx
    dx = 1.0 / (nx + 1)
    T1 = sp.diags([np.ones(nx - 1), -2.0 * np.ones(nx), np.ones(nx - 1)], [-1, 0, 1])
    I = sp.identity(nx)
    east = np.arange(nx) * nx + (nx - 1)
    west = np.arange(nx) * nx
    # the east diagonal moves from -4/dx^2 to (-3 + 0.25 dx)/dx^2
    A = (sp.kron(I, T1, format="csr") + sp.kron(T1, I, format="csr")) / (dx * dx)
    A = (A + sp.csr_matrix((np.full(nx, (1.0 + 0.25 * dx) / (dx * dx)), (east, east)), shape=(n, n))).tocsr()
    A.eliminate_zeros()
    A.sort_indices()
    S = sp.csr_matrix((np.full(nx, 0.5 / dx), (east, east)), shape=(n, n))
    B = None
    if control:
        B = np.zeros((n, 1))
        B[west, 0] = 1.0 / (dx * dx)
    C = np.full((1, n), 1.0 / n)
    return A, B, S, C, 0.5


def gdre_stochastic_heat(nx: int = 10, control: bool = True) -> Problem:
    """``stochastic_heat_csr`` as a dense Problem (GDRE with R = I_1, or the
    GDLE when control is False); P0 = 0."""
    A, B, S, C, T = stochastic_heat_csr(nx, control)
    n = nx * nx
    return Problem("gdre_stochastic_heat" if control else "gdle_stochastic_heat", A.toarray(), C,
                   np.zeros((n, n)), T, B=B, R=np.eye(1) if control else None, S=S.toarray(),
                   meta={"nx": nx, "control": control})


def dre_heat_large(nx: int = 64, m: int = 8, p: int = 8, T: float = 1.0, seed: int = 0) -> Problem:
    """Large dense DRE: Laplacian on nx x nx (n = 4096 at nx = 64), B = N(0,1)
    n x m, R = I_m, C = U(0,1) p x n, P0 = 0, T = 1.  Draw order: B then C."""
    n = nx * nx
    rng = np.random.default_rng(seed)
    A = laplacian_2d(nx)
    B = rng.standard_normal((n, m))
    C = rng.uniform(0.0, 1.0, size=(p, n))
    return Problem("dre_heat_large", A, C, np.zeros((n, n)), T, B=B, R=np.eye(m),
                   meta={"nx": nx, "seed": seed})


def fe_heat_mass(nx: int = 10, m: int = 2, p: int = 3, T: float = 0.5, seed: int = 0,
                 v: float = 5.0) -> Problem:
    """Linear finite elements for u_t = Laplace(u) - v u_x on the unit square (nx
    interior nodes per direction, tensor-product P1 basis): M x' = A x + B u with
    M = M1 (x) M1, A = -(K1 (x) M1 + M1 (x) K1) - v M1 (x) G1,
    M1 = dx tridiag(1/6, 2/3, 1/6), K1 = tridiag(-1, 2, -1)/dx,
    G1 = tridiag(-1/2, 0, 1/2) (x index fastest).  The convection term makes A
    non-symmetric and not commuting with M.  A synthetic stand-in for Example
    4's mass and stiffness matrices.  The mass matrix is returned in meta["M"].
    Draw order: B then C."""
    dx = 1.0 / (nx + 1)
    M1 = dx * _tridiag(nx, 1.0 / 6.0, 2.0 / 3.0, 1.0 / 6.0)
    K1 = _tridiag(nx, -1.0, 2.0, -1.0) / dx
    G1 = _tridiag(nx, -0.5, 0.0, 0.5)
    M = np.kron(M1, M1)
    A = -(np.kron(K1, M1) + np.kron(M1, K1)) - v * np.kron(M1, G1)
    n = nx * nx
    rng = np.random.default_rng(seed)
    B = rng.standard_normal((n, m))
    C = rng.uniform(0.0, 1.0, size=(p, n)) * dx
    return Problem("fe_heat_mass", A, C, np.zeros((n, n)), T, B=B, R=np.eye(m),
                   meta={"nx": nx, "M": M, "seed": seed})


def serving_requests(count: int, seed: int = 0, n_min: int = 32, n_max: int = 1024,
                     rate: float = 1.0, horizon=(0.1, 10.0), steps=(50, 500)):
    """Arrival stream of LQR/DRE requests (Strang F12F3, P0 = 0, R = I_m).

    The stream generator draws, per request and in this order: inter-arrival
    Exp(rate); n = round(exp(U(ln n_min, ln n_max))); the family bit (Laplacian
    with nx = round(sqrt n), n = nx^2, or the stable random A = M - (||M||_1+1) I,
    M = N(0,1)/sqrt(n)); m ~ U{1..8}; p ~ U{1..8}; T ~ U[horizon];
    steps ~ U{steps}; a 63-bit sub-seed.  Matrices are built lazily from the
    sub-seed by ``materialize`` so a 10 000-request stream stays small.
    Returns a list of spec dicts (arrival time in seconds)."""
    rng = np.random.default_rng(seed)
    t = 0.0
    out = []
    for r in range(count):
        t += rng.exponential(1.0 / rate)
        n = int(round(math.exp(rng.uniform(math.log(n_min), math.log(n_max)))))
        lap = bool(rng.integers(0, 2))
        if lap:
            nx = max(2, int(round(math.sqrt(n))))
            n = nx * nx
        m = int(rng.integers(1, 9))
        p = int(rng.integers(1, 9))
        T = float(rng.uniform(*horizon))
        N = int(rng.integers(steps[0], steps[1] + 1))
        sub = int(rng.integers(0, 2**63 - 1))
        out.append({"id": r, "arrival": t, "n": n, "m": m, "p": p, "T": T, "steps": N,
                    "family": "laplacian" if lap else "random", "seed": sub})
    return out


def materialize(spec: dict) -> Problem:
    """Build A, B, C, R for one serving spec.  Draw order from the sub-seed:
    (random family only) M, then B, then C."""
    n, m, p = spec["n"], spec["m"], spec["p"]
    rng = np.random.default_rng(spec["seed"])
    if spec["family"] == "laplacian":
        A = laplacian_2d(int(round(math.sqrt(n))))
    else:
        Mr = rng.standard_normal((n, n)) / math.sqrt(n)
        A = Mr - (np.abs(Mr).sum(axis=0).max() + 1.0) * np.eye(n)
    B = rng.standard_normal((n, m))
    C = rng.uniform(0.0, 1.0, size=(p, n))
    return Problem("serving", A, C, np.zeros((n, n)), spec["T"], B=B, R=np.eye(m),
                   meta={"steps": spec["steps"], "id": spec["id"]})
