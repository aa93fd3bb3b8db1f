"""Failure paths of the bounded device waits and of line chol, on the GPU without a fault.

Each bounded wait (the tensor-core GEMM's mbarrier waits, the cooperative C^-1 solve's
flag waits) is made to run out by withholding the one signal it waits for
(h1w_inject_stall: the GEMM's copy warp issues no copies; the first block of the
C^-1 solve publishes no result). The waits give up after a short limit, the kernels
return, the call reports H1W_ETIMEOUT, and the same context then solves normally.
A non-positive-definite matrix handed to h1w_cholesky gives H1W_ENOTSPD with text.
"""
import time

import numpy as np
import pytest
import torch

from oracle import discretization as disc
from paper_2209_02815_gb300 import h1w

pytestmark = pytest.mark.gpu
DEV = "cuda"
WAIT_NS = 20_000_000   # 20 ms per wait


def _case(m=40, n=(16, 16, 16), alpha=1e-2, seed=5):
    h = tuple(1.0 / v for v in n)
    N = int(np.prod(n))
    rng = np.random.default_rng(seed)
    J = rng.standard_normal((m, N)) / np.sqrt(N)
    b = rng.standard_normal(N)
    S = h1w.Solver(h1w.H1W_FV_CELL, n, h, alpha, m, device=DEV)
    return S, J, b, n, h, alpha


def _dense_solution(J, b, n, h, alpha):
    A = disc.regularization_operator("fv", n, h).toarray()
    return np.linalg.solve(alpha * A + J.T @ J, b)


def test_capacitance_gemm_wait_runs_out_and_context_recovers():
    S, J, b, n, h, alpha = _case()
    Jt = torch.as_tensor(J, device=DEV)
    S.inject_stall(h1w.H1W_STALL_CAP_GEMM, WAIT_NS)
    t0 = time.perf_counter()
    with pytest.raises(h1w.H1wError) as ei:
        S.capacitance(Jt)
    elapsed = time.perf_counter() - t0
    assert ei.value.status == h1w.H1W_ETIMEOUT
    assert "wait" in str(ei.value)
    assert elapsed < 10.0
    # a timed-out capacitance leaves none: PCG refuses until line H, C, chol run again
    with pytest.raises(h1w.H1wError) as ei2:
        S.pcg(torch.as_tensor(b, device=DEV), 1e-10, 100)
    assert ei2.value.status == h1w.H1W_ESTATE
    S.inject_stall(h1w.H1W_STALL_NONE, 0)
    S.capacitance(Jt)
    x, info = S.pcg(torch.as_tensor(b, device=DEV), 1e-12, 200)
    torch.cuda.synchronize()
    x_ref = _dense_solution(J, b, n, h, alpha)
    assert np.linalg.norm(x.cpu().numpy() - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


def test_preconditioner_solve_wait_runs_out_and_context_recovers():
    S, J, b, n, h, alpha = _case(m=70)
    S.capacitance(torch.as_tensor(J, device=DEV))
    bt = torch.as_tensor(b, device=DEV)
    S.inject_stall(h1w.H1W_STALL_PREC_SOLVE, WAIT_NS)
    t0 = time.perf_counter()
    with pytest.raises(h1w.H1wError) as ei:
        S.pcg(bt, 1e-12, 3)
    assert ei.value.status == h1w.H1W_ETIMEOUT
    assert time.perf_counter() - t0 < 10.0
    S.inject_stall(h1w.H1W_STALL_NONE, 0)
    x, info = S.pcg(bt, 1e-12, 200)
    torch.cuda.synchronize()
    x_ref = _dense_solution(J, b, n, h, alpha)
    assert np.linalg.norm(x.cpu().numpy() - x_ref) <= 1e-9 * np.linalg.norm(x_ref)


@pytest.mark.parametrize("n", [1, 31, 32, 33, 100, 257])
def test_cholesky_matches_numpy(n):
    S, *_ = _case(m=4, n=(8, 8, 8))
    rng = np.random.default_rng(n)
    B = rng.standard_normal((n, n))
    A = B @ B.T + n * np.eye(n)
    At = torch.as_tensor(A, device=DEV)
    S.cholesky(At)
    torch.cuda.synchronize()
    L = At.cpu().numpy()
    assert np.all(np.triu(L, 1) == 0.0)
    L_ref = np.linalg.cholesky(A)
    assert np.abs(L - L_ref).max() <= 1e-12 * np.abs(L_ref).max()


@pytest.mark.parametrize("n,bad", [(5, 0), (70, 40), (200, 199)])
def test_cholesky_reports_not_spd(n, bad):
    """A symmetric matrix with one negative eigenvalue: the pivot of row `bad` (or an
    earlier one) is not positive."""
    S, J, b, nn, h, alpha = _case(m=8, n=(8, 8, 8))
    rng = np.random.default_rng(3)
    Q, _ = np.linalg.qr(rng.standard_normal((n, n)))
    lam = np.linspace(1.0, 2.0, n)
    lam[bad] = -0.5
    A = (Q * lam) @ Q.T
    A = 0.5 * (A + A.T)
    with pytest.raises(h1w.H1wError) as ei:
        S.cholesky(torch.as_tensor(A, device=DEV))
    assert ei.value.status == h1w.H1W_ENOTSPD
    assert "not positive" in str(ei.value)
    # the context is still usable
    S.capacitance(torch.as_tensor(J, device=DEV))
    x, info = S.pcg(torch.as_tensor(b, device=DEV), 1e-12, 200)
    assert info.rel_res_true <= 1e-12
