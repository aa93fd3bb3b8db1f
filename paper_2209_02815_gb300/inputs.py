"""Seeded synthetic inputs for the Gauss-Newton linear solve.

This module only draws random numbers and evaluates the synthetic data model
(a Gaussian random log-conductivity field, surface electrode layouts and
analytic half-space sensitivities standing in for the ERT Jacobian). It holds
none of the solver's arithmetic: no stiffness or mass operator, no multigrid,
no Woodbury algebra. Both the CUDA path and the CPU oracle consume what it
returns, so neither side needs the other.

Workload shapes follow the paper's ERT experiments (Sec. 4): the parameter is a
log-conductivity m = log(sigma), measurements are pole-dipole apparent
resistivities whose sensitivity rows follow Eq. (4.4) with the geometric
factors of Eq. (4.5) (B electrode at infinity), and the Jacobian J is a dense
m x N matrix, one row per measurement.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np
import torch

# Seeds: 0 = J / random field, 1 = right-hand side / noise, 2 = batch draws.
SEED_FIELD = 0
SEED_RHS = 1
SEED_BATCH = 2


# ----------------------------------------------------------------------------
# Plain Gaussian problems (2D Q1 vertex grids)
# ----------------------------------------------------------------------------

@dataclass
class GaussianProblem:
    """A 2D Q1 problem with i.i.d. Gaussian J and b.

    J has shape (m, N) with entries N(0,1)/sqrt(N); b has shape (N,) with
    entries N(0,1). N = nx * ny vertices, x fastest.
    """
    nx: int
    ny: int
    m: int
    alpha: float
    J: np.ndarray
    b: np.ndarray

    @property
    def N(self) -> int:
        return self.nx * self.ny

    @property
    def h(self) -> tuple[float, float]:
        return (1.0 / (self.nx - 1), 1.0 / (self.ny - 1))


def gaussian_problem(nx: int, ny: int, m: int, alpha: float,
                     seed_j: int = SEED_FIELD, seed_b: int = SEED_RHS) -> GaussianProblem:
    """2D unit-square Q1 problem: J ~ N(0,1)/sqrt(N), b ~ N(0,1) (seeded)."""
    N = nx * ny
    rj = np.random.default_rng(seed_j)
    rb = np.random.default_rng(seed_b)
    J = rj.standard_normal((m, N)) / math.sqrt(N)
    b = rb.standard_normal(N)
    return GaussianProblem(nx, ny, m, alpha, J, b)


def small_c1_problem() -> GaussianProblem:
    """64 x 64 vertices on [0,1]^2, m = 16, alpha = 1e-2, J ~ N(0,1)/64."""
    return gaussian_problem(64, 64, 16, 1e-2)


# ----------------------------------------------------------------------------
# Gaussian random field (exponential covariance), circulant embedding
# ----------------------------------------------------------------------------

def gaussian_random_field(shape: tuple[int, ...], h: tuple[float, ...], corr_len: float,
                          mean: float, std: float, seed: int = SEED_FIELD) -> tuple[np.ndarray, float]:
    """Sample a stationary field with covariance std^2 exp(-r / corr_len).

    Circulant embedding on a periodic grid padded to twice the size along
    each axis; negative eigenvalues of the embedding are clamped to zero. The
    returned array has ``shape`` with axis 0 the slowest (z, y, x for 3D).
    Returns (field, clamped_fraction): the second value is the share of the
    embedding's eigenvalue mass that was clamped.
    """
    pad = tuple(2 * s for s in shape)
    grids = []
    for ax, (s, hh) in enumerate(zip(pad, h)):
        k = np.arange(s)
        d = np.minimum(k, s - k) * hh
        grids.append(d)
    r2 = np.zeros(pad)
    for ax, d in enumerate(grids):
        sh = [1] * len(pad)
        sh[ax] = pad[ax]
        r2 = r2 + (d.reshape(sh)) ** 2
    cov = (std ** 2) * np.exp(-np.sqrt(r2) / corr_len)
    lam = np.real(np.fft.fftn(cov))
    neg = float(-lam[lam < 0].sum() / np.abs(lam).sum())
    lam = np.maximum(lam, 0.0)
    rng = np.random.default_rng(seed)
    w = rng.standard_normal(pad) + 1j * rng.standard_normal(pad)
    total = float(np.prod(pad))
    f = np.fft.fftn(np.sqrt(lam / total) * w)
    sl = tuple(slice(0, s) for s in shape)
    return mean + np.real(f)[sl].copy(), neg


# ----------------------------------------------------------------------------
# ERT electrode layouts and measurement protocols
# ----------------------------------------------------------------------------

def line_electrodes(n_cells: int, n_e: int, h: float) -> np.ndarray:
    """n_e electrodes on the top face z = 0 along x at the cell-face centre row
    closest to y = 1/2, equispaced in x. Returns (n_e, 3) coordinates."""
    step = n_cells // n_e
    ix = step // 2 + step * np.arange(n_e)
    jy = n_cells // 2
    xs = (ix + 0.5) * h
    return np.stack([xs, np.full(n_e, (jy + 0.5) * h), np.zeros(n_e)], axis=1)


def grid_electrodes(n_cells: int, ex: int, ey: int, h: float) -> np.ndarray:
    """ex x ey electrodes on the top face at equispaced cell-face centres."""
    sx, sy = n_cells // ex, n_cells // ey
    ix = sx // 2 + sx * np.arange(ex)
    iy = sy // 2 + sy * np.arange(ey)
    X, Y = np.meshgrid((ix + 0.5) * h, (iy + 0.5) * h, indexing="xy")
    return np.stack([X.ravel(), Y.ravel(), np.zeros(X.size)], axis=1)


def pair_protocol(n_e: int) -> np.ndarray:
    """Pole-dipole pairs: for p < q, A = p, B at infinity, M = q and N the next
    electrode after q (cyclically) that is not p. Gives n_e (n_e - 1) / 2
    measurements as an (m, 3) integer array of (A, M, N)."""
    rows = []
    for p in range(n_e):
        for q in range(p + 1, n_e):
            nn = (q + 1) % n_e
            if nn == p:
                nn = (nn + 1) % n_e
            rows.append((p, q, nn))
    return np.asarray(rows, dtype=np.int64)


def dipole_dipole_grid(ex: int, ey: int, m_max: int) -> np.ndarray:
    """Dipole-dipole on an ex x ey electrode grid: dipoles are the adjacent
    x- and y-pairs; measurements are (source s, receiver r) with r > s and
    disjoint electrodes, in lexicographic order, truncated to m_max. Returns
    (m, 4) arrays (A, B, M, N)."""
    dip = []
    for j in range(ey):
        for i in range(ex - 1):
            dip.append((j * ex + i, j * ex + i + 1))
    for j in range(ey - 1):
        for i in range(ex):
            dip.append((j * ex + i, (j + 1) * ex + i))
    rows = []
    for s in range(len(dip)):
        for r in range(s + 1, len(dip)):
            if len({*dip[s], *dip[r]}) == 4:
                rows.append((*dip[s], *dip[r]))
                if len(rows) == m_max:
                    return np.asarray(rows, dtype=np.int64)
    return np.asarray(rows, dtype=np.int64)


def electrode_cells(n_cells: int, electrodes: np.ndarray, h: float) -> np.ndarray:
    """Index of the top-layer (z = 0) cell under each surface electrode (x, y, 0)."""
    i = np.minimum((electrodes[:, 0] / h).astype(np.int64), n_cells - 1)
    j = np.minimum((electrodes[:, 1] / h).astype(np.int64), n_cells - 1)
    return (j * n_cells + i).astype(np.int32)


# Dirichlet (u = 0) on every box face but the surface z = 0 (bits x-, x+, y-, y+, z+)
ERT_DIRICHLET_ALL_BUT_TOP = 0b101111


def ert_survey(n: int, n_e_line: int = 32, grid: tuple[int, int] | None = None,
               m_rows: int | None = None):
    """Electrode cells, (A, B, M, N) rows (-1 = at infinity) and geometric factors of
    the surveys used by ``ert_problem``: the line pair protocol (B at infinity) or
    the dipole-dipole grid. Returns (cells, abmn, k, electrodes)."""
    h = 1.0 / n
    if grid is None:
        el = line_electrodes(n, n_e_line, h)
        prot = pair_protocol(n_e_line)
        if m_rows is not None:
            prot = prot[:m_rows]
        abmn = np.stack([prot[:, 0], np.full(len(prot), -1), prot[:, 1], prot[:, 2]], axis=1)
        k = geometric_factor_pole_dipole(el[prot[:, 0]], el[prot[:, 1]], el[prot[:, 2]])
    else:
        el = grid_electrodes(n, grid[0], grid[1], h)
        abmn = dipole_dipole_grid(grid[0], grid[1], m_rows or 10 ** 9)
        k = geometric_factor_dipole_dipole(el[abmn[:, 0]], el[abmn[:, 1]], el[abmn[:, 2]], el[abmn[:, 3]])
    return electrode_cells(n, el, h), abmn.astype(np.int32), k, el


def gn_truth(n: int, sigma_bg: float = 0.01, factors=(10.0, 0.1),
             centres=((0.35, 0.5, 0.18), (0.65, 0.5, 0.18)), width: float = 0.08) -> np.ndarray:
    """Log-conductivity of the inversion workload: a background of sigma_bg with two
    Gaussian anomalies of peak conductivity factors ``factors`` (one conductive, one
    resistive) below the surface z = 0; cell centres of an n^3 grid on the unit cube,
    x fastest."""
    c = (np.arange(n) + 0.5) / n
    z, y, x = np.meshgrid(c, c, c, indexing="ij")
    ls = np.full(x.shape, math.log(sigma_bg))
    for f, (cx, cy, cz) in zip(factors, centres):
        ls += math.log(f) * np.exp(-((x - cx) ** 2 + (y - cy) ** 2 + (z - cz) ** 2) / (2 * width ** 2))
    return ls.reshape(-1)


def gn_survey(n: int, ex: int = 6, ey: int = 8, m_rows: int | None = 1000):
    """Surface electrodes on an ex x ey grid with the pair protocol over them (A, B at
    infinity, M, N), the first m_rows rows whose geometric factor is defined: on a grid
    the protocol's N can be as far from A as M is, which makes 1/|AM| - 1/|AN| vanish,
    and those rows are skipped. Returns (cells, abmn, k, electrodes)."""
    h = 1.0 / n
    el = grid_electrodes(n, ex, ey, h)
    prot = pair_protocol(len(el))
    am = np.linalg.norm(el[prot[:, 0]] - el[prot[:, 1]], axis=1)
    an = np.linalg.norm(el[prot[:, 0]] - el[prot[:, 2]], axis=1)
    prot = prot[np.abs(1.0 / am - 1.0 / an) > 1e-9 / am]
    if m_rows is not None:
        prot = prot[:m_rows]
    abmn = np.stack([prot[:, 0], np.full(len(prot), -1), prot[:, 1], prot[:, 2]], axis=1)
    k = geometric_factor_pole_dipole(el[prot[:, 0]], el[prot[:, 1]], el[prot[:, 2]])
    return electrode_cells(n, el, h), abmn.astype(np.int32), k, el


def noisy(g_true: np.ndarray, noise: float = 0.02, seed: int = SEED_RHS) -> np.ndarray:
    """Observed data g_true (1 + noise eps), eps ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    return g_true * (1.0 + noise * rng.standard_normal(g_true.shape))


def geometric_factor_pole_dipole(xa, xm, xn) -> np.ndarray:
    """3D geometric factor with B at infinity (limit of Eq. 4.5)."""
    am = np.linalg.norm(xa - xm, axis=-1)
    an = np.linalg.norm(xa - xn, axis=-1)
    return 2.0 * np.pi / (1.0 / am - 1.0 / an)


def geometric_factor_dipole_dipole(xa, xb, xm, xn) -> np.ndarray:
    """3D geometric factor of Eq. 4.5 for four finite electrodes."""
    d = lambda u, v: np.linalg.norm(u - v, axis=-1)
    return 2.0 * np.pi / (1.0 / d(xa, xm) - 1.0 / d(xb, xm) - 1.0 / d(xa, xn) + 1.0 / d(xb, xn))


# ----------------------------------------------------------------------------
# Analytic half-space sensitivities (stand-in for the ERT Jacobian)
# ----------------------------------------------------------------------------

@dataclass
class ErtProblem:
    """One synthetic 3D ERT Gauss-Newton step on an n^3 cell-centred grid.

    logsigma: (N,) current iterate m = log(sigma), x fastest.
    m_ref: scalar reference value log(sigma_ref).
    J: (m, N) sensitivity matrix (numpy on CPU or torch on a device).
    d: (m,) data residual g_m - g_obs.
    """
    n: int
    alpha: float
    logsigma: np.ndarray
    m_ref: float
    J: object
    d: np.ndarray
    electrodes: np.ndarray
    protocol: np.ndarray
    k: np.ndarray
    clamped: float

    @property
    def N(self) -> int:
        return self.n ** 3

    @property
    def h(self) -> float:
        return 1.0 / self.n


def _cell_centres(n: int, h: float, device, dtype):
    c = (torch.arange(n, device=device, dtype=dtype) + 0.5) * h
    z, y, x = torch.meshgrid(c, c, c, indexing="ij")
    return x.reshape(-1), y.reshape(-1), z.reshape(-1)


def half_space_gradients(n: int, h: float, electrodes: np.ndarray, sigma0: float,
                         device="cpu", dtype=torch.float64) -> torch.Tensor:
    """Gradient of the unit-current half-space potential u_e = 1/(2 pi sigma0 |x - x_e|)
    at every cell centre, for every electrode: tensor (n_e, 3, N)."""
    x, y, z = _cell_centres(n, h, device, dtype)
    out = torch.empty((len(electrodes), 3, n ** 3), device=device, dtype=dtype)
    c = -1.0 / (2.0 * math.pi * sigma0)
    for e, xe in enumerate(electrodes):
        dx, dy, dz = x - float(xe[0]), y - float(xe[1]), z - float(xe[2])
        r3 = (dx * dx + dy * dy + dz * dz) ** 1.5
        out[e, 0] = c * dx / r3
        out[e, 1] = c * dy / r3
        out[e, 2] = c * dz / r3
    return out


def ert_problem(n: int, n_e_line: int = 32, alpha: float = 1e-3, m_rows: int | None = None,
                device="cpu", corr_len: float = 0.1, sigma_bg: float = 0.01,
                noise: float = 0.02, grid: tuple[int, int] | None = None) -> ErtProblem:
    """Synthetic ERT step on an n^3 cell grid over the unit cube (z = 0 is the
    top face). The log-conductivity is a Gaussian random field (exponential
    covariance, correlation length ``corr_len``, mean log(sigma_bg), std 1).

    Line layout (default): n_e_line electrodes and the pole-dipole pair
    protocol, m = n_e (n_e - 1) / 2. Grid layout (``grid=(ex, ey)``):
    dipole-dipole over adjacent pairs, truncated to ``m_rows``.

    J_ic = -k_i sigma_c grad u_A . grad(u_M - u_N) h^3 (Eq. 4.4 evaluated with
    homogeneous half-space potentials); the data residual is
    d = g - g_obs = -noise * eps / sigma_bg with eps ~ N(0,1) (seed 1).
    """
    h = 1.0 / n
    field, clamped = gaussian_random_field((n, n, n), (h, h, h), corr_len,
                                           math.log(sigma_bg), 1.0, SEED_FIELD)
    logsigma = field.reshape(-1)
    if grid is None:
        el = line_electrodes(n, n_e_line, h)
        prot = pair_protocol(n_e_line)
        if m_rows is not None:
            prot = prot[:m_rows]
        k = geometric_factor_pole_dipole(el[prot[:, 0]], el[prot[:, 1]], el[prot[:, 2]])
        a_idx, b_idx, m_idx, n_idx = prot[:, 0], None, prot[:, 1], prot[:, 2]
    else:
        el = grid_electrodes(n, grid[0], grid[1], h)
        prot = dipole_dipole_grid(grid[0], grid[1], m_rows or 10 ** 9)
        k = geometric_factor_dipole_dipole(el[prot[:, 0]], el[prot[:, 1]], el[prot[:, 2]], el[prot[:, 3]])
        a_idx, b_idx, m_idx, n_idx = prot[:, 0], prot[:, 1], prot[:, 2], prot[:, 3]
    m = len(prot)
    G = half_space_gradients(n, h, el, sigma_bg, device=device)
    sig = torch.exp(torch.as_tensor(logsigma, device=device))
    J = torch.empty((m, n ** 3), device=device, dtype=torch.float64)
    vol = h ** 3
    for i in range(m):
        ga = G[a_idx[i]]
        if b_idx is not None:
            ga = ga - G[b_idx[i]]
        gmn = G[m_idx[i]] - G[n_idx[i]]
        J[i] = (-float(k[i]) * vol) * sig * (ga * gmn).sum(0)
    del G
    rng = np.random.default_rng(SEED_RHS)
    d = -noise * rng.standard_normal(m) / sigma_bg
    return ErtProblem(n, alpha, logsigma, math.log(sigma_bg), J if device != "cpu" else J.numpy(),
                      d, el, prot, k, clamped)


# ----------------------------------------------------------------------------
# Batched 2D instances of uneven size
# ----------------------------------------------------------------------------

def batch_instances(count: int = 64, sides=(128, 256, 512, 1024), ms=(8, 32, 64, 256),
                    alpha_range=(1e-4, 1e-1), seed: int = SEED_BATCH) -> list[dict]:
    """Descriptors of ``count`` independent 2D Q1 problems: side s (vertices),
    m and alpha drawn i.i.d. (alpha log-uniform). J and b are drawn per
    instance with seeds derived from ``seed``."""
    rng = np.random.default_rng(seed)
    out = []
    for i in range(count):
        s = int(rng.choice(sides))
        m = int(rng.choice(ms))
        a = float(math.exp(rng.uniform(math.log(alpha_range[0]), math.log(alpha_range[1]))))
        out.append({"n": s, "m": m, "alpha": a, "seed_j": 1000 + 2 * i, "seed_b": 1001 + 2 * i})
    return out


def batch_instance_data(desc: dict, device="cpu"):
    """J (m x N, i.i.d. N(0,1)/sqrt(N)) and b (N, i.i.d. N(0,1)) of one batch
    instance, N = n^2 vertices, from the instance's own seeds."""
    n, m = desc["n"], desc["m"]
    N = n * n
    g = torch.Generator(device=device)
    g.manual_seed(desc["seed_j"])
    J = torch.randn((m, N), generator=g, dtype=torch.float64, device=device) / math.sqrt(N)
    g.manual_seed(desc["seed_b"])
    b = torch.randn(N, generator=g, dtype=torch.float64, device=device)
    return J, b


def paper_pole_dipole(n_e: int) -> np.ndarray:
    """The paper's 1D pole-dipole sequence (Fig. 4.1): for spacings s = 2, 4, 8
    and each direction along the line, electrode triples (A, M, N) at positions
    (i, i + s, i + 2s); B is at infinity. Gives M = 6 n_e - 56 measurements.
    Returns an (M, 3) array of 0-based electrode indices."""
    rows = []
    for s in (2, 4, 8):
        for i in range(n_e - 2 * s):
            rows.append((i, i + s, i + 2 * s))
        for i in range(n_e - 2 * s):
            j = n_e - 1 - i
            rows.append((j, j - s, j - 2 * s))
    return np.asarray(rows, dtype=np.int64)
