"""Gauss-Newton steps on the ERT model (oracle; test infrastructure only).

Algorithm "Gauss-Newton with iterative solver": at the iterate m, evaluate g_m
and J_m (``oracle.ert``), take the step dm that minimizes the linearized
objective

    1/2 ||g_m - g_obs + J_m dm||^2 + alpha/2 (m - m_ref + dm)^T (K + M) (m - m_ref + dm),

i.e. (alpha (K + M) + J^T J) dm = -alpha (K + M)(m - m_ref) - J^T (g_m - g_obs)
(Eq. 2.9 scaled by beta, with the mass term), and set m := m + dm. Here the
system is solved densely. K + M is the finite-volume operator of
``oracle.discretization`` on the same grid.
"""
from __future__ import annotations

import numpy as np

from . import discretization as disc
from . import ert


def objective(n, h, alpha, m, m_ref, cells, abmn, k, dirichlet, g_obs, A_reg=None) -> float:
    """1/2 ||g(m) - g_obs||^2 + alpha/2 (m - m_ref)^T (K + M) (m - m_ref)."""
    A_reg = disc.regularization_operator("fv", n, h) if A_reg is None else A_reg
    g, _ = ert.forward(n, h, m, cells, abmn, k, dirichlet)
    r = m - m_ref
    return 0.5 * float(np.sum((g - g_obs) ** 2)) + 0.5 * alpha * float(r @ (A_reg @ r))


def gn_step(n, h, alpha, m, m_ref, cells, abmn, k, dirichlet, g_obs):
    """(dm, g_m, J_m) of one Gauss-Newton step, dense normal-equations solve."""
    A_reg = disc.regularization_operator("fv", n, h).toarray()
    g, U = ert.forward(n, h, m, cells, abmn, k, dirichlet)
    J = ert.jacobian(n, h, m, U, abmn, k, dirichlet)
    b = -alpha * A_reg @ (m - m_ref) - J.T @ (g - g_obs)
    dm = np.linalg.solve(alpha * A_reg + J.T @ J, b)
    return dm, g, J
