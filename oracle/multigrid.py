"""The Laplace preconditioner L^-1: one symmetric V-cycle (oracle; test infrastructure only).

The paper applies an algebraic multigrid cycle as its Laplace preconditioner
S-hat^-1 (Sec. 3.2, the AMG line of Algorithm "Gauss-Newton with iterative
solver") and treats it as a black box. On the structured grids used here the
black box is a geometric V-cycle, defined as follows (every choice below is
the same on the CUDA side, which implements it independently):

* Coarsening. Q1 vertex grids: per axis with n >= 3 vertices, the coarse
  vertices are the even indices plus the last vertex; 1D linear interpolation
  P1; the coarse operator is the Galerkin product P^T A P. FV cell grids: per
  axis with an even n >= 4 cells, 2:1 cell agglomeration; 1D cell-centred
  linear interpolation with weights 3/4 and 1/4 (constant extrapolation at
  the boundary); the coarse operator is the same FV operator rediscretized on
  the coarse grid. Restriction R = P^T. Coarsening stops when the level has at
  most 512 unknowns or no axis can be coarsened.
* Smoother: degree-k Chebyshev iteration (k = 2) preconditioned by the
  diagonal D of the level operator, on the interval [lam/r, lam], lam the
  Gershgorin bound max_i sum_j |A_ij| / A_ii of D^-1 A, with r = 10 on FV cell
  grids and r = 6 on Q1 vertex grids (the ratios that gave the fewest PCG
  iterations over isotropic and anisotropic grids of both kinds; the paper
  leaves the smoother to the AMG black box).
* Cycle: pre-smooth from zero, residual, restrict, recurse, prolongate and
  add, post-smooth with the same polynomial. The coarsest level is solved
  exactly by a dense Cholesky factorization.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .discretization import fv_assemble, q1_assemble

COARSE_MAX = 512
CHEB_DEGREE = 2
CHEB_RATIO = {"fv": 10.0, "q1": 6.0}


def q1_prolongation_1d(n: int):
    """Linear interpolation from the coarse vertex set onto n fine vertices.

    Coarse vertices: even fine indices, plus the last vertex when n - 1 is odd.
    Returns (P of shape (n, nc), nc), or (None, n) when n < 3.
    """
    if n < 3:
        return None, n
    coarse = list(range(0, n, 2))
    if coarse[-1] != n - 1:
        coarse.append(n - 1)
    nc = len(coarse)
    P = np.zeros((n, nc))
    pos = {f: c for c, f in enumerate(coarse)}
    for f in range(n):
        if f in pos:
            P[f, pos[f]] = 1.0
        else:  # odd interior vertex between two coarse vertices f-1, f+1
            P[f, pos[f - 1]] = 0.5
            P[f, pos[f + 1]] = 0.5
    return sp.csr_matrix(P), nc


def fv_prolongation_1d(n: int):
    """Cell-centred linear interpolation from n/2 coarse cells onto n fine cells.

    Fine cell 2I + s takes 3/4 of coarse cell I and 1/4 of its neighbour on the
    same side (I - 1 for s = 0, I + 1 for s = 1); a missing neighbour is
    replaced by I itself. Returns (P, nc) or (None, n) when n is odd or < 4.
    """
    if n % 2 or n < 4:
        return None, n
    nc = n // 2
    P = np.zeros((n, nc))
    for f in range(n):
        I, s = divmod(f, 2)
        J = I - 1 if s == 0 else I + 1
        if 0 <= J < nc:
            P[f, I] += 0.75
            P[f, J] += 0.25
        else:
            P[f, I] += 1.0
    return sp.csr_matrix(P), nc


def gershgorin_bound(A: sp.csr_matrix) -> float:
    """max_i sum_j |A_ij| / A_ii, an upper bound on the spectrum of D^-1 A."""
    absrow = np.asarray(abs(A).sum(axis=1)).ravel()
    return float(np.max(absrow / A.diagonal()))


@dataclass
class Level:
    A: sp.csr_matrix
    n: tuple
    h: tuple
    dinv: np.ndarray
    lam: float
    P: sp.csr_matrix | None = None  # to the next coarser level
    chol: object = None             # coarsest only


@dataclass
class Hierarchy:
    disc: str
    levels: list = field(default_factory=list)

    @property
    def N(self) -> int:
        return self.levels[0].A.shape[0]


def _kron_axes(Ps):
    """Kronecker product of per-axis operators with x fastest (Ps[0] is x)."""
    out = Ps[0]
    for P in Ps[1:]:
        out = sp.kron(P, out, format="csr")
    return out


def build_hierarchy(disc: str, n: tuple[int, ...], h: tuple[float, ...]) -> Hierarchy:
    """Level operators, transfers and the coarsest Cholesky factor."""
    n = tuple(int(v) for v in n)
    h = tuple(float(v) for v in h)
    if disc == "q1":
        K, _, Ml = q1_assemble(n[0], n[1], h[0], h[1])
        A = (K + sp.diags(Ml)).tocsr()
    elif disc == "fv":
        K, M = fv_assemble(n[0], n[1], n[2], h[0], h[1], h[2])
        A = (K + sp.diags(M)).tocsr()
    else:
        raise ValueError(disc)
    H = Hierarchy(disc)
    while True:
        lev = Level(A=A, n=n, h=h, dinv=1.0 / A.diagonal(), lam=gershgorin_bound(A))
        H.levels.append(lev)
        if A.shape[0] <= COARSE_MAX:
            break
        Ps, nc, hc = [], [], []
        for ax in range(len(n)):
            P1, ncax = (q1_prolongation_1d if disc == "q1" else fv_prolongation_1d)(n[ax])
            if P1 is None:
                Ps.append(sp.identity(n[ax], format="csr"))
                nc.append(n[ax])
                hc.append(h[ax])
            else:
                Ps.append(P1)
                nc.append(ncax)
                hc.append(2.0 * h[ax])
        if tuple(nc) == n:
            break
        P = _kron_axes(Ps)
        lev.P = P
        if disc == "q1":
            A = (P.T @ A @ P).tocsr()
        else:
            Kc, Mc = fv_assemble(nc[0], nc[1], nc[2], hc[0], hc[1], hc[2])
            A = (Kc + sp.diags(Mc)).tocsr()
        n, h = tuple(nc), tuple(hc)
    last = H.levels[-1]
    if last.A.shape[0] > 1024:
        raise ValueError("coarsest level too large for the dense solve")
    last.chol = sla.cho_factor(last.A.toarray(), lower=True)
    return H


def chebyshev(A, dinv, lam, b, x, ratio, degree=CHEB_DEGREE):
    """Degree-k Chebyshev iteration for A x = b with Jacobi preconditioning on
    [lam/ratio, lam]; the error is multiplied by T_k((theta - mu)/delta) / T_k(theta/delta)
    for each eigenvalue mu of D^-1 A."""
    lo, hi = lam / ratio, lam
    theta = 0.5 * (hi + lo)
    delta = 0.5 * (hi - lo)
    sigma = theta / delta
    r = b - A @ x
    d = dinv * r / theta
    x = x + d
    rho_prev = 1.0 / sigma
    for _ in range(1, degree):
        r = r - A @ d
        rho = 1.0 / (2.0 * sigma - rho_prev)
        d = rho * rho_prev * d + (2.0 * rho / delta) * dinv * r
        x = x + d
        rho_prev = rho
    return x


def vcycle(H: Hierarchy, b: np.ndarray, level: int = 0) -> np.ndarray:
    """One V-cycle applied to b (zero initial guess): x = L-hat^-1 b."""
    lev = H.levels[level]
    if lev.chol is not None:
        return sla.cho_solve(lev.chol, b)
    r_cheb = CHEB_RATIO[H.disc]
    x = chebyshev(lev.A, lev.dinv, lev.lam, b, np.zeros_like(b), r_cheb)
    r = b - lev.A @ x
    xc = vcycle(H, lev.P.T @ r, level + 1)
    x = x + lev.P @ xc
    return chebyshev(lev.A, lev.dinv, lev.lam, b, x, r_cheb)


def vcycle_matrix(H: Hierarchy) -> np.ndarray:
    """Dense matrix of the V-cycle operator (tiny grids only)."""
    N = H.N
    out = np.empty((N, N))
    for j in range(N):
        e = np.zeros(N)
        e[j] = 1.0
        out[:, j] = vcycle(H, e)
    return out
