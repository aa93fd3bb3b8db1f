"""ERT forward model and its Jacobian (oracle; test infrastructure only).

The model of Sec. 4.1 (Eqs. 4.1-4.5) on a cell-centred finite-volume grid:

* potential equation -div(sigma grad u) = f, sigma = exp(m) per cell;
* the face conductance between neighbouring cells a, b along axis k is
  G_k * 2 sigma_a sigma_b / (sigma_a + sigma_b) (harmonic mean of the two
  cells' conductivities), G_k = face area / centre distance;
* a face of the box listed as Dirichlet (the paper's gamma_D, u = 0) couples
  its boundary cell to a ghost value 0 at distance h_k / 2, conductance
  2 G_k sigma_a; every other box face is zero-flux (gamma_N);
* electrode e injects a unit current into one cell c_e, so its pole field is
  u_e = A^-1 e_{c_e}, and the voltage at electrode f is u(c_f);
* measurement i with electrodes (A, B, M, N), any of them -1 for "at
  infinity", is g_i = k_i <e_M - e_N, A^-1 (e_A - e_B)> (Eq. 4.3 scaled by
  the geometric factor of Eq. 4.5), i.e. g_i = k_i (v(c_M) - v(c_N)) with
  v = u_A - u_B;
* its derivative with respect to m_c (Eq. 4.4, discretely: dA^-1 =
  -A^-1 dA A^-1 and reciprocity A^-1 (e_M - e_N) = u_M - u_N = w) is
  J_ic = -k_i w^T (dA / dm_c) v.

Vectors are indexed x fastest: p = (k * ny + j) * nx + i. Box faces are
numbered 0..5 = x-, x+, y-, y+, z-, z+; bit f of ``dirichlet`` marks face f
as Dirichlet. Pins: the Jacobian against central differences of g, the 1D
column against its series-resistance closed form, reciprocity, and the
homogeneous half-space against the apparent-resistivity normalisation of
Eq. 4.5 under refinement.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla


def _index(n):
    nx, ny, nz = n
    k, j, i = np.meshgrid(np.arange(nz), np.arange(ny), np.arange(nx), indexing="ij")
    return i.ravel(), j.ravel(), k.ravel()


def faces(n, h, dirichlet: int):
    """Interior faces (a, b, G) and Dirichlet boundary faces (a, G) of the grid.

    a < b are the two cells of an interior face; G = face area / distance of
    the two centres. A boundary face's G is its area / (h_k / 2)."""
    nx, ny, nz = n
    i, j, k = _index(n)
    p = np.arange(nx * ny * nz)
    area = (h[1] * h[2], h[0] * h[2], h[0] * h[1])
    coord = (i, j, k)
    stride = (1, nx, nx * ny)
    inner_a, inner_b, inner_g = [], [], []
    bnd_a, bnd_g = [], []
    for ax in range(3):
        last = n[ax] - 1
        sel = coord[ax] < last
        inner_a.append(p[sel])
        inner_b.append(p[sel] + stride[ax])
        inner_g.append(np.full(int(sel.sum()), area[ax] / h[ax]))
        for side, at in ((0, 0), (1, last)):
            if dirichlet >> (2 * ax + side) & 1:
                cells = p[coord[ax] == at]
                bnd_a.append(cells)
                bnd_g.append(np.full(cells.size, area[ax] / (0.5 * h[ax])))
    cat = lambda xs, dt: np.concatenate(xs).astype(dt) if xs else np.zeros(0, dt)
    return (cat(inner_a, np.int64), cat(inner_b, np.int64), cat(inner_g, float),
            cat(bnd_a, np.int64), cat(bnd_g, float))


def face_conductances(n, h, logsigma, dirichlet: int):
    """Conductance of every interior face (harmonic mean) and Dirichlet face."""
    a, b, g, ba, bg = faces(n, h, dirichlet)
    s = np.exp(np.asarray(logsigma, dtype=float))
    t = g * 2.0 * s[a] * s[b] / (s[a] + s[b])
    tb = bg * s[ba]
    return (a, b, t), (ba, tb)


def ert_matrix(n, h, logsigma, dirichlet: int) -> sp.csr_matrix:
    """A = sum over faces of t (e_a - e_b)(e_a - e_b)^T + sum over Dirichlet faces t e_a e_a^T."""
    N = int(np.prod(n))
    (a, b, t), (ba, tb) = face_conductances(n, h, logsigma, dirichlet)
    rows = np.concatenate([a, b, a, b, ba])
    cols = np.concatenate([a, b, b, a, ba])
    vals = np.concatenate([t, t, -t, -t, tb])
    return sp.csr_matrix((vals, (rows, cols)), shape=(N, N))


def fields(n, h, logsigma, cells, dirichlet: int) -> np.ndarray:
    """Pole fields u_e = A^-1 e_{c_e} for every electrode, by a sparse LU solve: (n_e, N)."""
    A = ert_matrix(n, h, logsigma, dirichlet).tocsc()
    N = A.shape[0]
    rhs = np.zeros((N, len(cells)))
    rhs[np.asarray(cells), np.arange(len(cells))] = 1.0
    return np.ascontiguousarray(spla.splu(A).solve(rhs).T)


def _combo(U, e1, e2):
    """u_e1 - u_e2 with -1 meaning 'at infinity' (no field)."""
    out = np.zeros(U.shape[1])
    if e1 >= 0:
        out = out + U[e1]
    if e2 >= 0:
        out = out - U[e2]
    return out


def measurements(U, cells, abmn, k) -> np.ndarray:
    """g_i = k_i (v(c_M) - v(c_N)), v = u_A - u_B (Eq. 4.3 with Eq. 4.5's factor)."""
    cells = np.asarray(cells)
    g = np.empty(len(abmn))
    for i, (ea, eb, em, en) in enumerate(np.asarray(abmn)):
        v = _combo(U, ea, eb)
        val = (v[cells[em]] if em >= 0 else 0.0) - (v[cells[en]] if en >= 0 else 0.0)
        g[i] = k[i] * val
    return g


def jacobian(n, h, logsigma, U, abmn, k, dirichlet: int) -> np.ndarray:
    """J_ic = -k_i w^T (dA / dm_c) v (Eq. 4.4), v = u_A - u_B, w = u_M - u_N: (m, N).

    dA/dm_c has a term from every face of cell c: for an interior face with
    conductance t = G 2 s_a s_b / (s_a + s_b), d t / d m_a = G 2 s_a s_b^2 / (s_a + s_b)^2
    (s = exp(m)); for a Dirichlet face t = 2 G s_a and d t / d m_a = t."""
    a, b, g, ba, bg = faces(n, h, dirichlet)
    s = np.exp(np.asarray(logsigma, dtype=float))
    den = (s[a] + s[b]) ** 2
    dta = g * 2.0 * s[a] * s[b] ** 2 / den
    dtb = g * 2.0 * s[b] * s[a] ** 2 / den
    dtd = bg * s[ba]
    N = U.shape[1]
    J = np.zeros((len(abmn), N))
    for i, (ea, eb, em, en) in enumerate(np.asarray(abmn)):
        v = _combo(U, ea, eb)
        w = _combo(U, em, en)
        prod = (v[a] - v[b]) * (w[a] - w[b])
        row = np.zeros(N)
        np.add.at(row, a, dta * prod)
        np.add.at(row, b, dtb * prod)
        np.add.at(row, ba, dtd * v[ba] * w[ba])
        J[i] = -k[i] * row
    return J


def forward(n, h, logsigma, cells, abmn, k, dirichlet: int):
    """(g, U) for one conductivity model."""
    U = fields(n, h, logsigma, cells, dirichlet)
    return measurements(U, cells, abmn, k), U


def top_cell(n, h, x: float, y: float) -> int:
    """Index of the cell of the top layer (k = 0, the z- face) under the point (x, y)."""
    i = min(int(x / h[0]), n[0] - 1)
    j = min(int(y / h[1]), n[1] - 1)
    return j * n[0] + i
