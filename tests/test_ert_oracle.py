"""Pins of the ERT forward-model oracle (Sec. 4.1, Eqs. 4.1-4.5), CPU only.

Each test ties ``oracle.ert`` to something other than itself: central
differences of the discrete measurements, the series-resistance closed form of
a 1D column, reciprocity of the symmetric operator, the degree -1 homogeneity
of g in sigma, and the apparent-resistivity normalisation of the homogeneous
half space.
"""
import numpy as np
import pytest

from oracle import ert


ALL_BUT_TOP = 0b101111   # every box face Dirichlet except z- (the surface)


def _small_case(seed, dirichlet):
    rng = np.random.default_rng(seed)
    n, h = (4, 3, 5), (0.3, 0.25, 0.2)
    N = int(np.prod(n))
    logsigma = np.log(0.01) + rng.standard_normal(N)
    cells = [0, 2, 5, 7, 11]          # four in the top layer, one below it
    cells[-1] = 11 + n[0] * n[1]
    abmn = np.array([[0, -1, 1, 2], [1, 3, 0, 4], [2, -1, 4, -1], [3, 0, 2, 1]])
    k = rng.uniform(0.5, 2.0, len(abmn))
    return n, h, logsigma, cells, abmn, k, dirichlet


@pytest.mark.parametrize("dirichlet", [ALL_BUT_TOP, 0b100000, 0b000011])
def test_jacobian_matches_central_differences(dirichlet):
    n, h, ls, cells, abmn, k, dm = _small_case(3, dirichlet)
    g, U = ert.forward(n, h, ls, cells, abmn, k, dm)
    J = ert.jacobian(n, h, ls, U, abmn, k, dm)
    eps = 1e-5
    fd = np.empty_like(J)
    for c in range(ls.size):
        e = np.zeros_like(ls)
        e[c] = eps
        gp, _ = ert.forward(n, h, ls + e, cells, abmn, k, dm)
        gm, _ = ert.forward(n, h, ls - e, cells, abmn, k, dm)
        fd[:, c] = (gp - gm) / (2 * eps)
    scale = np.abs(J).max(axis=1, keepdims=True)
    assert np.abs(fd - J).max() / scale.min() < 1e-7


def test_column_series_resistance():
    """A 1 x 1 x nz column, Dirichlet only at the bottom: all current flows down,
    so the source cell's potential is the series resistance from its centre to the
    ghost, (hz / (hx hy)) (1 / (2 s_0) + sum_{k >= 1} 1 / s_k), and its derivative
    in m_k is -(hz / (hx hy)) / (2 s_0) for k = 0 and -(hz / (hx hy)) / s_k else."""
    n, h = (1, 1, 7), (0.5, 0.4, 0.1)
    rng = np.random.default_rng(5)
    ls = rng.standard_normal(7)
    s = np.exp(ls)
    c = h[2] / (h[0] * h[1])
    abmn, k = np.array([[0, -1, 0, -1]]), np.array([1.0])
    g, U = ert.forward(n, h, ls, [0], abmn, k, 0b100000)
    assert g[0] == pytest.approx(c * (0.5 / s[0] + np.sum(1.0 / s[1:])), rel=1e-13)
    J = ert.jacobian(n, h, ls, U, abmn, k, 0b100000)
    want = -c / s
    want[0] *= 0.5
    np.testing.assert_allclose(J[0], want, rtol=1e-12)


def test_reciprocity():
    n, h, ls, cells, _, _, dm = _small_case(7, ALL_BUT_TOP)
    U = ert.fields(n, h, ls, cells, dm)
    V = U[:, cells]                        # V[a, b] = u_a(c_b)
    np.testing.assert_allclose(V, V.T, rtol=1e-12)


@pytest.mark.parametrize("dirichlet", [ALL_BUT_TOP, 0b000011])
def test_homogeneity(dirichlet):
    """sigma -> e^t sigma scales A by e^t and g by e^-t, so sum_c J_ic = -g_i."""
    n, h, ls, cells, abmn, k, dm = _small_case(11, dirichlet)
    g, U = ert.forward(n, h, ls, cells, abmn, k, dm)
    J = ert.jacobian(n, h, ls, U, abmn, k, dm)
    np.testing.assert_allclose(J.sum(axis=1), -g, rtol=1e-11)


@pytest.mark.parametrize("n", [16, 24])
def test_half_space_apparent_resistivity(n):
    """Pole-dipole on a homogeneous unit cube, surface electrodes spaced 1/8 apart:
    with the geometric factor of Eq. 4.5 (B at infinity) g is the apparent
    resistivity, 1 / sigma_0 for the half space; the discrete box model gives it
    within a few percent."""
    h = (1.0 / n,) * 3
    s0 = 0.01
    ls = np.full(n ** 3, np.log(s0))
    cells = [ert.top_cell((n, n, n), h, x + 0.5 / n, 0.5 + 0.5 / n) for x in (0.375, 0.5, 0.625)]
    P = np.array([[(c % n + 0.5) / n, (c // n + 0.5) / n, 0.0] for c in cells])
    k = 2 * np.pi / (1 / np.linalg.norm(P[0] - P[1]) - 1 / np.linalg.norm(P[0] - P[2]))
    g, _ = ert.forward((n, n, n), h, ls, cells, np.array([[0, -1, 1, 2]]), [k], ALL_BUT_TOP)
    assert abs(g[0] * s0 - 1.0) < 0.05


# ---- Gauss-Newton steps (Algorithm "Gauss-Newton with iterative solver") ----------

from oracle import discretization as odisc  # noqa: E402
from oracle import gn as ogn  # noqa: E402


def _gn_case(alpha):
    n, h = (6, 5, 4), (1 / 6, 1 / 5, 1 / 4)
    N = int(np.prod(n))
    rng = np.random.default_rng(21)
    m_ref = np.full(N, np.log(0.01))
    m = m_ref + 0.3 * rng.standard_normal(N)
    m_true = m_ref + 0.5 * rng.standard_normal(N)
    cells = [0, 2, 4, 12, 16, 27]
    abmn = np.array([(p, -1, q, (q + 1) % 6 if (q + 1) % 6 != p else (q + 2) % 6)
                     for p in range(6) for q in range(p + 1, 6)])
    k = np.linspace(1.0, 2.0, len(abmn))
    g_true, _ = ert.forward(n, h, m_true, cells, abmn, k, ALL_BUT_TOP)
    return n, h, alpha, m, m_ref, cells, abmn, k, ALL_BUT_TOP, g_true * 1.01


def test_gn_step_is_the_least_squares_minimizer():
    """The step minimizes 1/2||d + J dm||^2 + alpha/2 ||R (m - m_ref + dm)||^2 with
    K + M = R^T R: solved here as a stacked least-squares problem by QR (numpy lstsq)
    instead of the normal equations."""
    n, h, alpha, m, m_ref, cells, abmn, k, dm_, g_obs = _gn_case(1e-3)
    dm, g, J = ogn.gn_step(n, h, alpha, m, m_ref, cells, abmn, k, dm_, g_obs)
    R = np.linalg.cholesky(odisc.regularization_operator("fv", n, h).toarray()).T
    A = np.vstack([J, np.sqrt(alpha) * R])
    rhs = -np.concatenate([g - g_obs, np.sqrt(alpha) * R @ (m - m_ref)])
    ls = np.linalg.lstsq(A, rhs, rcond=None)[0]
    assert np.abs(dm - ls).max() / np.abs(ls).max() < 1e-9


def test_gn_step_descends():
    n, h, alpha, m, m_ref, cells, abmn, k, dm_, g_obs = _gn_case(1e-3)
    dm, _, _ = ogn.gn_step(n, h, alpha, m, m_ref, cells, abmn, k, dm_, g_obs)
    f0 = ogn.objective(n, h, alpha, m, m_ref, cells, abmn, k, dm_, g_obs)
    f1 = ogn.objective(n, h, alpha, m + 1e-3 * dm, m_ref, cells, abmn, k, dm_, g_obs)
    assert f1 < f0


def test_gn_step_large_alpha_returns_to_reference():
    """With the regularization dominating, the step is m_ref - m."""
    n, h, alpha, m, m_ref, cells, abmn, k, dm_, g_obs = _gn_case(1e8)
    dm, _, _ = ogn.gn_step(n, h, alpha, m, m_ref, cells, abmn, k, dm_, g_obs)
    assert np.abs(dm + (m - m_ref)).max() / np.abs(m - m_ref).max() < 1e-6
