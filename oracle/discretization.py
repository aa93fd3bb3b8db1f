"""Assembly of the regularization operator K + M (oracle; test infrastructure only).

The paper's H1 regularization term int |grad(m - m_ref)|^2 gives the operator
L of Eq. (2.8) (Sec. 2.2); with the mass term added, the Gauss-Newton system of
Eq. (2.9) scaled by beta reads (alpha (K + M) + J^T J) x = b with alpha the
paper's beta. Boundary conditions: natural (zero-flux) on every face.

* 2D: bilinear Q1 elements on an nx x ny vertex grid, element matrices by
  exact 2 x 2 Gauss quadrature, row-sum lumped mass.
* 3D: cell-centred finite volumes on an nx x ny x nz cell grid; face
  transmissibility (face area / centre distance) between neighbours, none
  across the boundary; M = cell volume. On a Cartesian grid this is the
  lowest-order Raviart-Thomas Schur complement D diag(Q)^-1 D^T that the paper
  uses as its Laplace approximation S-hat (Sec. 3.2).

Vectors are indexed x fastest: p = (k * ny + j) * nx + i.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def q1_element_matrices(hx: float, hy: float) -> tuple[np.ndarray, np.ndarray]:
    """Stiffness and consistent mass of one hx x hy bilinear element.

    Local node a = ii + 2 jj sits at (ii hx, jj hy). Integrals by 2 x 2 Gauss
    quadrature, exact for these bilinear products.
    """
    g = np.array([0.5 - 0.5 / np.sqrt(3.0), 0.5 + 0.5 / np.sqrt(3.0)])
    Ke = np.zeros((4, 4))
    Me = np.zeros((4, 4))
    for xi in g:
        for eta in g:
            w = 0.25 * hx * hy
            phi = np.empty(4)
            dx = np.empty(4)
            dy = np.empty(4)
            for a in range(4):
                ii, jj = a % 2, a // 2
                fx = xi if ii else 1.0 - xi
                fy = eta if jj else 1.0 - eta
                dfx = 1.0 if ii else -1.0
                dfy = 1.0 if jj else -1.0
                phi[a] = fx * fy
                dx[a] = dfx * fy / hx
                dy[a] = fx * dfy / hy
            Ke += w * (np.outer(dx, dx) + np.outer(dy, dy))
            Me += w * np.outer(phi, phi)
    return Ke, Me


def q1_assemble(nx: int, ny: int, hx: float, hy: float):
    """Assemble Q1 stiffness K, consistent mass Mc and lumped mass diagonal Ml."""
    Ke, Me = q1_element_matrices(hx, hy)
    ex, ey = np.meshgrid(np.arange(nx - 1), np.arange(ny - 1), indexing="xy")
    ex, ey = ex.ravel(), ey.ravel()
    nodes = np.stack([(ey + a // 2) * nx + (ex + a % 2) for a in range(4)], axis=1)
    rows = np.repeat(nodes, 4, axis=1).ravel()
    cols = np.tile(nodes, (1, 4)).ravel()
    N = nx * ny
    K = sp.coo_matrix((np.tile(Ke.ravel(), len(ex)), (rows, cols)), shape=(N, N)).tocsr()
    Mc = sp.coo_matrix((np.tile(Me.ravel(), len(ex)), (rows, cols)), shape=(N, N)).tocsr()
    K.sum_duplicates()
    Mc.sum_duplicates()
    Ml = np.asarray(Mc.sum(axis=1)).ravel()
    return K, Mc, Ml


def fv_assemble(nx: int, ny: int, nz: int, hx: float, hy: float, hz: float):
    """Assemble the cell-centred FV stiffness K and the mass diagonal M."""
    N = nx * ny * nz
    T = (hy * hz / hx, hx * hz / hy, hx * hy / hz)
    idx = np.arange(N).reshape(nz, ny, nx)
    rows, cols, vals = [], [], []
    for axis, t in zip((2, 1, 0), T):  # array axis 2 is x, 1 is y, 0 is z
        lo = [slice(None)] * 3
        hi = [slice(None)] * 3
        lo[axis] = slice(0, idx.shape[axis] - 1)
        hi[axis] = slice(1, None)
        a = idx[tuple(lo)].ravel()
        b = idx[tuple(hi)].ravel()
        rows += [a, b, a, b]
        cols += [a, b, b, a]
        vals += [np.full(a.size, t), np.full(a.size, t), np.full(a.size, -t), np.full(a.size, -t)]
    if rows:
        K = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                          shape=(N, N)).tocsr()
    else:
        K = sp.csr_matrix((N, N))
    K.sum_duplicates()
    M = np.full(N, hx * hy * hz)
    return K, M


def regularization_operator(disc: str, n: tuple[int, ...], h: tuple[float, ...]) -> sp.csr_matrix:
    """K + M as a CSR matrix (Q1 with lumped mass, or FV with cell volumes)."""
    if disc == "q1":
        K, _, Ml = q1_assemble(n[0], n[1], h[0], h[1])
        return (K + sp.diags(Ml)).tocsr()
    if disc == "fv":
        K, M = fv_assemble(n[0], n[1], n[2], h[0], h[1], h[2])
        return (K + sp.diags(M)).tocsr()
    raise ValueError(disc)
