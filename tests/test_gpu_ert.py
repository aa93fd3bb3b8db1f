"""ERT forward model and Jacobian on the GPU (h1w_forward / h1w_adjoint) against the
oracle (Sec. 4.1, Eqs. 4.1-4.5).

Small grids are compared element by element with ``oracle.ert`` (sparse LU
fields): pole fields, measurements, Jacobian rows and J^T r, with ragged tiles
(cell counts not a multiple of the 32-cell Jacobian tile) and multi-level
hierarchies. At the 128^3 size of the Gauss-Newton workload, where the oracle's
direct solve is out of reach, the tests check properties that hold at any size:
reciprocity, the homogeneity sum_c J_ic = -g_i, and J^T r against the stored rows.
"""
import numpy as np
import pytest
import torch

from oracle import ert as oert
from paper_2209_02815_gb300 import h1w, inputs

pytestmark = pytest.mark.gpu

DEV = "cuda"
ALL_BUT_TOP = inputs.ERT_DIRICHLET_ALL_BUT_TOP


def _solver(n, h):
    return h1w.Solver(h1w.H1W_FV_CELL, n, h, 1e-3, 1, device=DEV)


def _random_survey(n, n_e, m, seed, dirichlet=ALL_BUT_TOP, with_b=True):
    rng = np.random.default_rng(seed)
    N = int(np.prod(n))
    cells = rng.choice(n[0] * n[1], size=n_e, replace=False)      # top layer
    cells[-1] = N - 1 - int(rng.integers(0, n[0]))                   # one at the bottom
    rows = []
    for _ in range(m):
        a, b, mm, nn = rng.choice(n_e, size=4, replace=False)
        rows.append((a, b if with_b and rng.random() < 0.5 else -1, mm, nn if rng.random() < 0.8 else -1))
    k = rng.uniform(0.5, 3.0, m)
    return h1w.Survey(cells, np.array(rows), k, dirichlet)


def _logsigma(n, seed):
    rng = np.random.default_rng(seed)
    return np.log(0.01) + rng.standard_normal(int(np.prod(n)))


CASES = [
    ((20, 18, 14), (1 / 20, 1 / 18, 1 / 14), ALL_BUT_TOP),    # 5040 cells: two levels, ragged tile
    ((24, 16, 12), (0.05, 0.06, 0.08), 0b110000),             # anisotropic, Dirichlet top and bottom
    ((9, 7, 5), (0.1, 0.1, 0.1), 0b000001),                   # one level (dense solve), one Dirichlet face
    ((32, 32, 32), (1 / 32,) * 3, ALL_BUT_TOP),               # three levels
    ((21, 16, 12), (1 / 21, 1 / 16, 1 / 12), ALL_BUT_TOP),    # odd x: x not coarsened (one-cell transfers)
]


@pytest.mark.parametrize("n,h,dirichlet", CASES)
def test_forward_and_jacobian_match_oracle(n, h, dirichlet):
    N = int(np.prod(n))
    sv = _random_survey(n, 6, 9, seed=N, dirichlet=dirichlet)
    ls = _logsigma(n, N + 1)
    s = _solver(n, h)
    lst = torch.tensor(ls, device=DEV)
    g, U, info = s.forward(sv, lst, rtol=1e-13, maxit=300)
    assert info.rel_res_true < 1e-12
    g0, U0 = oert.forward(n, h, ls, sv.cells, sv.abmn, sv.k, dirichlet)
    Ug = U.cpu().numpy()
    scale = np.abs(U0).max(axis=1, keepdims=True)
    assert np.abs(Ug - U0).max(axis=1, keepdims=True).max() / scale.min() < 1e-9
    np.testing.assert_allclose(g.cpu().numpy(), g0, rtol=1e-9, atol=1e-9 * np.abs(g0).max())
    JTr, J = s.adjoint(sv, lst, U, r=torch.tensor(np.linspace(-1, 2, sv.m), device=DEV), rows=True)
    J0 = oert.jacobian(n, h, ls, U0, sv.abmn, sv.k, dirichlet)
    Jg = J.cpu().numpy()
    row_scale = np.abs(J0).max(axis=1)
    assert (np.abs(Jg - J0).max(axis=1) / row_scale).max() < 1e-8
    r = np.linspace(-1, 2, sv.m)
    jtr0 = J0.T @ r
    assert np.abs(JTr.cpu().numpy() - jtr0).max() / np.abs(jtr0).max() < 1e-8
    # J^T r formed without J agrees with the stored rows of the same fields
    jtr_rows = Jg.T @ r
    assert np.abs(JTr.cpu().numpy() - jtr_rows).max() / np.abs(jtr_rows).max() < 1e-13
    # and so does J p
    pv = np.cos(np.arange(N) * 0.37)
    Jp = s.jvp(sv, lst, U, torch.tensor(pv, device=DEV)).cpu().numpy()
    assert np.abs(Jp - Jg @ pv).max() / np.abs(Jg @ pv).max() < 1e-12
    assert np.abs(Jp - J0 @ pv).max() / np.abs(J0 @ pv).max() < 1e-8


def test_jacobian_is_derivative_of_forward_on_gpu():
    """Central differences of the GPU measurements along a random direction d
    against J d and against the autograd backward pass."""
    n, h = (20, 18, 14), (1 / 20, 1 / 18, 1 / 14)
    N = int(np.prod(n))
    sv = _random_survey(n, 5, 7, seed=3)
    s = _solver(n, h)
    ls = torch.tensor(_logsigma(n, 4), device=DEV)
    d = torch.tensor(np.random.default_rng(5).standard_normal(N), device=DEV)
    eps = 1e-4
    gp, _, _ = s.forward(sv, ls + eps * d, rtol=1e-13, maxit=300)
    gm, _, _ = s.forward(sv, ls - eps * d, rtol=1e-13, maxit=300)
    fd = ((gp - gm) / (2 * eps)).cpu().numpy()
    x = ls.clone().requires_grad_(True)
    g = h1w.ErtForward.apply(x, s, sv, 1e-13, 300)
    w = torch.tensor(np.random.default_rng(6).standard_normal(sv.m), device=DEV)
    (g * w).sum().backward()
    _, U, _ = s.forward(sv, ls, rtol=1e-13, maxit=300)
    _, J = s.adjoint(sv, ls, U, rows=True)
    Jd = (J @ d).cpu().numpy()
    assert np.abs(fd - Jd).max() / np.abs(Jd).max() < 1e-6
    np.testing.assert_allclose(x.grad.cpu().numpy(), (J.T @ w).cpu().numpy(), rtol=1e-12,
                               atol=1e-13 * float(torch.abs(J.T @ w).max()))


def test_edge_cases():
    n, h = (12, 10, 8), (0.1, 0.1, 0.1)
    s = _solver(n, h)
    N = int(np.prod(n))
    ls = torch.tensor(_logsigma(n, 9), device=DEV)
    # one electrode, no measurements: fields only
    sv = h1w.Survey([5], np.zeros((0, 4), dtype=np.int32), np.zeros(0), ALL_BUT_TOP)
    g, U, info = s.forward(sv, ls, rtol=1e-12)
    assert g.numel() == 0 and info.rel_res_true < 1e-11
    U0 = oert.fields(n, h, ls.cpu().numpy(), [5], ALL_BUT_TOP)
    assert np.abs(U.cpu().numpy() - U0).max() / np.abs(U0).max() < 1e-9
    # a measurement at its own source cell (M = A, N at infinity)
    sv = h1w.Survey([5, 17], [[0, -1, 0, -1], [1, 0, 1, 0]], [1.0, 2.0], ALL_BUT_TOP)
    g, U, _ = s.forward(sv, ls, rtol=1e-13)
    g0, _ = oert.forward(n, h, ls.cpu().numpy(), [5, 17], sv.abmn, sv.k, ALL_BUT_TOP)
    np.testing.assert_allclose(g.cpu().numpy(), g0, rtol=1e-9)
    # invalid surveys fail on the host with H1W_EINVAL
    for bad in (h1w.Survey([N], [[0, -1, 0, -1]], [1.0], ALL_BUT_TOP),       # cell out of range
                h1w.Survey([3], [[0, -1, 1, -1]], [1.0], ALL_BUT_TOP),       # electrode index out of range
                h1w.Survey([3], [[0, -1, 0, -1]], [1.0], 0)):                # no Dirichlet face
        with pytest.raises(h1w.H1wError) as ei:
            s.forward(bad, ls)
        assert ei.value.status == h1w.H1W_EINVAL
    # a Q1 context has no ERT model
    q = h1w.Solver(h1w.H1W_Q1_VERTEX, (33, 33), (1 / 32, 1 / 32), 1e-2, 1, device=DEV)
    assert h1w.h1w_ert_workspace_size(q.ctx, 1, 1) == 0


@pytest.mark.parametrize("grid", [None, (8, 8)])
def test_full_size_properties(grid):
    """128^3, the Gauss-Newton workload's grid and survey (32-electrode line pair
    protocol, m = 496; or the 8 x 8 dipole-dipole grid, first 1024 rows): reciprocity
    of the fields, sum_c J_ic = -g_i, and J^T r against the stored rows."""
    n = 128
    cells, abmn, k, _ = inputs.ert_survey(n, grid=grid, m_rows=None if grid is None else 1024)
    sv = h1w.Survey(cells, abmn, k, ALL_BUT_TOP)
    s = _solver((n, n, n), (1 / n,) * 3)
    field, _ = inputs.gaussian_random_field((n, n, n), (1 / n,) * 3, 0.1, np.log(0.01), 1.0, 0)
    ls = torch.tensor(field.reshape(-1), device=DEV)
    # Both identities hold up to the reciprocity error of the computed fields, which
    # follows the solve's residual: at rtol 1e-10 the 64-electrode survey showed 3e-9.
    g, U, info = s.forward(sv, ls, rtol=1e-12, maxit=200)
    assert info.rel_res_true < 1e-11
    V = U[:, torch.tensor(cells, device=DEV, dtype=torch.long)].cpu().numpy()
    np.testing.assert_allclose(V, V.T, rtol=1e-9, atol=1e-11 * np.abs(V).max())
    r = torch.tensor(np.random.default_rng(2).standard_normal(sv.m), device=DEV)
    JTr, J = s.adjoint(sv, ls, U, r=r, rows=True)
    rs = J.sum(dim=1)
    assert float(torch.abs(rs + g).max() / torch.abs(g).max()) < 1e-9
    jr = J.T @ r
    assert float(torch.abs(JTr - jr).max() / torch.abs(jr).max()) < 1e-12
    pv = torch.cos(torch.arange(n ** 3, device=DEV, dtype=torch.float64) * 0.37)
    Jp = s.jvp(sv, ls, U, pv)
    jp = J @ pv
    assert float(torch.abs(Jp - jp).max() / torch.abs(jp).max()) < 1e-11


def test_gn_steps_match_oracle():
    """Two passes of h1w_gn_step (forward, J, Laplace-Woodbury PCG, update) against the
    oracle's Gauss-Newton steps with a dense solve."""
    from oracle import gn as ogn
    n, h = (16, 12, 8), (1 / 16, 1 / 12, 1 / 8)
    N = int(np.prod(n))
    alpha = 1e-2
    rng = np.random.default_rng(8)
    cells = rng.choice(n[0] * n[1], size=8, replace=False)
    prot = inputs.pair_protocol(8)
    abmn = np.stack([prot[:, 0], np.full(len(prot), -1), prot[:, 1], prot[:, 2]], axis=1)
    k = rng.uniform(1.0, 3.0, len(abmn))
    m_ref = np.full(N, np.log(0.01))
    m_true = m_ref + 0.8 * rng.standard_normal(N)
    g_true, _ = oert.forward(n, h, m_true, cells, abmn, k, ALL_BUT_TOP)
    g_obs = inputs.noisy(g_true)
    sv = h1w.Survey(cells, abmn, k, ALL_BUT_TOP)
    s = h1w.Solver(h1w.H1W_FV_CELL, n, h, alpha, sv.m, device=DEV)
    m_dev = torch.tensor(m_ref, device=DEV)
    m_host = m_ref.copy()
    for step in range(2):
        hist, g, _ = s.gn_inversion(sv, torch.tensor(g_obs, device=DEV), torch.tensor(m_ref, device=DEV), m_dev, 1,
                                    rtol_fwd=1e-13, rtol=1e-12)
        dm, g0, _ = ogn.gn_step(n, h, alpha, m_host, m_ref, cells, abmn, k, ALL_BUT_TOP, g_obs)
        # the second step's data follow the first update, on which the GPU's PCG (rtol 1e-12)
        # and the oracle's dense solve agree to cond * rtol: small entries are compared
        # against the largest datum
        np.testing.assert_allclose(g.cpu().numpy(), g0, rtol=1e-9, atol=1e-9 * np.abs(g0).max())
        m_host = m_host + dm
        err = np.abs(m_dev.cpu().numpy() - m_host).max() / np.abs(dm).max()
        assert err < 1e-7, (step, err)
        # the misfit is that of the returned data (which the line above compares with the oracle's)
        assert hist[0].misfit == pytest.approx(np.linalg.norm(g.cpu().numpy() - g_obs), rel=1e-11)
        assert abs(hist[0].misfit - np.linalg.norm(g0 - g_obs)) <= 1.01 * np.linalg.norm(g.cpu().numpy() - g0)


def test_gn_inversion_reduces_misfit():
    """Three Gauss-Newton steps of the inversion workload's design (two Gaussian
    anomalies, 6 x 8 surface electrodes, pair protocol, 2 % noise) on a 32^3 grid."""
    n = 32
    cells, abmn, k, _ = inputs.gn_survey(n, m_rows=1000)
    sv = h1w.Survey(cells, abmn, k, ALL_BUT_TOP)
    s = h1w.Solver(h1w.H1W_FV_CELL, (n,) * 3, (1 / n,) * 3, 100.0, sv.m, device=DEV)
    ls_true = torch.tensor(inputs.gn_truth(n), device=DEV)
    g_true, _, _ = s.forward(sv, ls_true, rtol=1e-12)
    g_obs = torch.tensor(inputs.noisy(g_true.cpu().numpy()), device=DEV)
    m_ref = torch.full((n ** 3,), np.log(0.01), dtype=torch.float64, device=DEV)
    m = m_ref.clone()
    hist, _, _ = s.gn_inversion(sv, g_obs, m_ref, m, 3)
    mis = [h_.misfit for h_ in hist]
    assert mis[1] < mis[0] and mis[2] < 0.3 * mis[0], mis
    assert all(h_.rel_res_true < 1e-7 for h_ in hist)


def test_gn_inversion_checkpoint_resume(tmp_path):
    """Two steps written to a checkpoint, then a fresh context resumes to step three: the
    iterate equals that of three uninterrupted steps bit for bit (the checkpoint keeps the
    pole fields, so the resumed forward solve starts warm as the uninterrupted one does)."""
    n = 16
    cells, abmn, k, _ = inputs.gn_survey(n, m_rows=200)
    sv = h1w.Survey(cells, abmn, k, ALL_BUT_TOP)
    mk = lambda: h1w.Solver(h1w.H1W_FV_CELL, (n,) * 3, (1 / n,) * 3, 100.0, sv.m, device=DEV)
    s = mk()
    ls_true = torch.tensor(inputs.gn_truth(n), device=DEV)
    g_true, _, _ = s.forward(sv, ls_true, rtol=1e-12)
    g_obs = torch.tensor(inputs.noisy(g_true.cpu().numpy()), device=DEV)
    m_ref = torch.full((n ** 3,), np.log(0.01), dtype=torch.float64, device=DEV)
    m_straight = m_ref.clone()
    hist3, _, _ = s.gn_inversion(sv, g_obs, m_ref, m_straight, 3)
    ck = str(tmp_path / "gn.pt")
    m_a = m_ref.clone()
    hist2, _, _ = mk().gn_inversion(sv, g_obs, m_ref, m_a, 2, checkpoint=ck)
    assert len(hist2) == 2 and torch.equal(m_a, torch.load(ck, weights_only=True)["m"].to(DEV))
    m_b = torch.full_like(m_ref, 123.0)                    # overwritten from the checkpoint
    hist_b, _, _ = mk().gn_inversion(sv, g_obs, m_ref, m_b, 3, checkpoint=ck)
    assert len(hist_b) == 3 and [h_.gn_iters for h_ in hist_b] == [h_.gn_iters for h_ in hist3]
    assert torch.equal(m_b, m_straight)
    assert torch.load(ck, weights_only=True)["step"] == 3


def test_forward_warm_start():
    """From the fields of a nearby model the forward solve reaches the same fields in
    fewer iterations (H1W_FORWARD_WARM_START)."""
    n, h = (24, 16, 12), (0.05, 0.06, 0.08)
    sv = _random_survey(n, 6, 9, seed=12)
    s = _solver(n, h)
    ls = torch.tensor(_logsigma(n, 13), device=DEV)
    ls2 = ls + 0.05 * torch.tensor(np.random.default_rng(14).standard_normal(ls.numel()), device=DEV)
    _, U, _ = s.forward(sv, ls, rtol=1e-12)
    g_cold, U_cold, i_cold = s.forward(sv, ls2, rtol=1e-12)
    g_warm, U_warm, i_warm = s.forward(sv, ls2, rtol=1e-12, U=U.clone(), warm=True)
    assert i_warm.iters < i_cold.iters and i_warm.rel_res_true < 1e-11
    gc = g_cold.cpu().numpy()
    np.testing.assert_allclose(g_warm.cpu().numpy(), gc, rtol=1e-9, atol=1e-9 * np.abs(gc).max())
    assert float(torch.abs(U_warm - U_cold).max() / torch.abs(U_cold).max()) < 1e-9


def test_gn_step_and_direct_argument_checks():
    n, h = (12, 10, 8), (0.1, 0.1, 0.1)
    N = int(np.prod(n))
    sv = _random_survey(n, 4, 6, seed=31)
    s = h1w.Solver(h1w.H1W_FV_CELL, n, h, 1.0, 3, device=DEV)   # m_max = 3 < survey.m
    t = lambda k: torch.zeros(k, dtype=torch.float64, device=DEV)
    ws = s.ert_workspace(sv)
    with pytest.raises(h1w.H1wError) as ei:
        h1w.h1w_gn_step(s.ctx, sv, t(sv.m), t(N), t(N), t(sv.n_e * N), t(sv.m * N), t(sv.m), t(3 * N + sv.m), ws,
                        1e-10, 1e-8, 100, N)
    assert ei.value.status == h1w.H1W_EINVAL
    with pytest.raises(h1w.H1wError) as ei:   # no capacitance call yet
        s.solve_direct(t(N))
    assert ei.value.status == h1w.H1W_ESTATE
    with pytest.raises(h1w.H1wError) as ei:   # unknown forward flag
        h1w.h1w_forward(s.ctx, sv, t(N), t(sv.n_e * N), t(sv.m), ws, 1e-10, 100, N, flags=2)
    assert ei.value.status == h1w.H1W_EINVAL


def test_max_electrodes():
    """H1W_ERT_MAX_ELECTRODES = 128 electrodes: the Jacobian kernel stages 128 x 6 face
    jumps for 32 cells (about 200 KB of shared memory per block). Fields, measurements,
    J rows, J^T r and J p against the oracle; 129 electrodes are refused."""
    n, h = (24, 20, 16), (1 / 24, 1 / 20, 1 / 16)
    N = int(np.prod(n))
    rng = np.random.default_rng(61)
    ne = 128
    cells = rng.choice(n[0] * n[1], size=ne, replace=False)
    rows = []
    for _ in range(300):
        a, b, mm, nn = rng.choice(ne, size=4, replace=False)
        rows.append((a, b if rng.random() < 0.5 else -1, mm, nn))
    sv = h1w.Survey(cells, np.array(rows), rng.uniform(0.5, 2.0, 300), ALL_BUT_TOP)
    s = _solver(n, h)
    ls = _logsigma(n, 62)
    lst = torch.tensor(ls, device=DEV)
    g, U, info = s.forward(sv, lst, rtol=1e-13, maxit=300)
    g0, U0 = oert.forward(n, h, ls, sv.cells, sv.abmn, sv.k, ALL_BUT_TOP)
    assert np.abs(U.cpu().numpy() - U0).max() / np.abs(U0).max() < 1e-9
    np.testing.assert_allclose(g.cpu().numpy(), g0, rtol=1e-9, atol=1e-9 * np.abs(g0).max())
    r = np.sin(np.arange(sv.m))
    JTr, J = s.adjoint(sv, lst, U, r=torch.tensor(r, device=DEV), rows=True)
    J0 = oert.jacobian(n, h, ls, U0, sv.abmn, sv.k, ALL_BUT_TOP)
    assert (np.abs(J.cpu().numpy() - J0).max(axis=1) / np.abs(J0).max(axis=1)).max() < 1e-8
    assert np.abs(JTr.cpu().numpy() - J0.T @ r).max() / np.abs(J0.T @ r).max() < 1e-8
    pv = np.cos(np.arange(N) * 0.11)
    Jp = s.jvp(sv, lst, U, torch.tensor(pv, device=DEV)).cpu().numpy()
    assert np.abs(Jp - J0 @ pv).max() / np.abs(J0 @ pv).max() < 1e-8
    too_many = h1w.Survey(np.arange(129), [[0, -1, 1, 2]], [1.0], ALL_BUT_TOP)
    assert h1w.h1w_ert_workspace_size(s.ctx, 129, 1) == 0
    with pytest.raises(h1w.H1wError) as ei:
        s.forward(too_many, lst, ws=torch.empty(1 << 20, dtype=torch.uint8, device=DEV))
    assert ei.value.status == h1w.H1W_EINVAL
