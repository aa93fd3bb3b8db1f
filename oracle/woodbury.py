"""Woodbury capacitance, preconditioner apply, direct solve and PCG (oracle; test infrastructure only).

Notation (paper -> here): beta -> alpha, S-hat^-1 -> L-hat^-1 (one V-cycle on
K + M), M measurements -> m rows of J.

* Algorithm "MINRES with the Laplace-Woodbury preconditioner": line H builds
  H = L-hat^-1 J^T (here one V-cycle per column), line C forms
  C = I + alpha^-1 J H, line chol factors C = L L^T.
* Sec. 3.2, preconditioner P-hat: with P = alpha L-hat + J^T J, the
  Sherman-Morrison-Woodbury formula gives
  P^-1 r = alpha^-1 [ L-hat^-1 r - alpha^-1 H C^-1 H^T r ].
* Sec. 3.1: with the exact inverse of K + M in place of L-hat^-1 the same
  formula is the direct solve (Algorithm "Gauss-Newton with direct solver").
* Stopping rule: Euclidean ||r_k|| <= tol ||b|| from x_0 = 0 (Sec. 4, the
  Matlab MINRES criterion); here for PCG on the SPD primal system.
"""
from __future__ import annotations

import numpy as np
import scipy.linalg as sla

from . import multigrid as mg


def gn_rhs(A_reg, alpha, m_minus_mref, J, d):
    """b = -alpha (K + M)(m - m_ref) - J^T (g - g_obs): Eq. (2.9) scaled by beta, with mass."""
    return -alpha * (A_reg @ m_minus_mref) - J.T @ d


def apply_operator(A_reg, alpha, J, p):
    """q = alpha (K + M) p + J^T (J p); J^T J is never formed."""
    return alpha * (A_reg @ p) + J.T @ (J @ p)


def hhat(H: mg.Hierarchy, J: np.ndarray) -> np.ndarray:
    """H-hat = L-hat^-1 J^T, one V-cycle per measurement (N x m)."""
    return np.stack([mg.vcycle(H, J[i]) for i in range(J.shape[0])], axis=1) if J.shape[0] else \
        np.zeros((J.shape[1], 0))


def capacitance(J: np.ndarray, Hh: np.ndarray, alpha: float) -> np.ndarray:
    """C = I + alpha^-1 J H-hat, symmetrized as (C + C^T)/2."""
    m = J.shape[0]
    C = np.eye(m) + (J @ Hh) / alpha
    return 0.5 * (C + C.T)


class WoodburyPreconditioner:
    """P^-1 r = alpha^-1 [ L^-1 r - alpha^-1 H C^-1 H^T r ] for a given L^-1."""

    def __init__(self, apply_Linv, J: np.ndarray, alpha: float, Hh: np.ndarray | None = None):
        self.apply_Linv = apply_Linv
        self.alpha = alpha
        self.J = J
        m = J.shape[0]
        if Hh is None:
            Hh = np.stack([apply_Linv(J[i]) for i in range(m)], axis=1) if m else np.zeros((J.shape[1], 0))
        self.Hh = Hh
        self.C = capacitance(J, Hh, alpha)
        self.L = np.linalg.cholesky(self.C) if m else np.zeros((0, 0))

    def __call__(self, r: np.ndarray) -> np.ndarray:
        z0 = self.apply_Linv(r)
        if self.J.shape[0] == 0:
            return z0 / self.alpha
        s = self.Hh.T @ r
        y = sla.solve_triangular(self.L, s, lower=True)
        v = sla.solve_triangular(self.L.T, y, lower=False)
        return (z0 - (self.Hh @ v) / self.alpha) / self.alpha


def woodbury_direct(A_reg_dense: np.ndarray, J: np.ndarray, alpha: float, b: np.ndarray) -> np.ndarray:
    """Direct solve of (alpha A + J^T J) x = b through the Woodbury formula with
    the exact inverse of A (Sec. 3.1)."""
    Ainv = np.linalg.inv(A_reg_dense)
    P = WoodburyPreconditioner(lambda v: Ainv @ v, J, alpha)
    return P(b)


def pcg(apply_A, apply_P, b: np.ndarray, rtol: float, maxit: int, max_restarts: int = 3):
    """Preconditioned CG from x_0 = 0.

    Stops when the recursively updated residual satisfies ||r|| <= rtol ||b||;
    then the true residual b - A x is formed and, if it fails the test, the
    iteration restarts from r = b - A x (at most ``max_restarts`` times).
    Returns (x, iterations, true relative residual).
    """
    bnorm = float(np.linalg.norm(b))
    x = np.zeros_like(b)
    if bnorm == 0.0:
        return x, 0, 0.0
    r = b.copy()
    it = 0
    for _ in range(max_restarts + 1):
        z = apply_P(r)
        p = z.copy()
        rz = float(r @ z)
        while it < maxit and np.linalg.norm(r) > rtol * bnorm:
            q = apply_A(p)
            a = rz / float(p @ q)
            x = x + a * p
            r = r - a * q
            it += 1
            if np.linalg.norm(r) <= rtol * bnorm:
                break
            z = apply_P(r)
            rz_new = float(r @ z)
            p = z + (rz_new / rz) * p
            rz = rz_new
        r = b - apply_A(x)
        rel = float(np.linalg.norm(r)) / bnorm
        if rel <= rtol or it >= maxit:
            return x, it, rel
    return x, it, rel
