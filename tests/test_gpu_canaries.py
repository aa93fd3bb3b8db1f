"""Out-of-bounds writes, found without compute-sanitizer: every buffer the library writes
(the caller's workspace, the ERT workspace and the output vectors) sits inside a larger
allocation whose guard bands hold a fixed canary pattern, and the bands are checked after
each call. Inputs, including the borrowed J, get guard bands too and must come back
unchanged. Grids are small and ragged (axes that are not multiples of the kernels' tiles,
odd axes that are not coarsened), with both the default double-float path and the plain FP64
form, on FV cells and Q1 vertices."""
import numpy as np
import pytest
import torch

from paper_2209_02815_gb300 import h1w, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda"
GUARD_BYTES = 4096                # before and after the workspace (keeps its 256-byte alignment)
GUARD = 512                       # float64 entries before and after each vector
CANARY_BYTE = 0xA5
CANARY_BITS = 0x7FF4DEADBEEF0001  # a NaN with a payload no kernel writes


def _guarded_vec(n, fill=None):
    """(whole, view): a float64 vector of n entries inside canary bands."""
    whole = torch.full((n + 2 * GUARD,), CANARY_BITS, dtype=torch.int64, device=DEV).view(torch.float64)
    view = whole[GUARD:GUARD + n]
    if fill is not None:
        view.copy_(fill)
    return whole, view


def _bands_intact(whole, n):
    bits = whole.view(torch.int64)
    return bool((bits[:GUARD] == CANARY_BITS).all()) and bool((bits[GUARD + n:] == CANARY_BITS).all())


def _guarded_ws(size):
    whole = torch.full((size + 2 * GUARD_BYTES,), CANARY_BYTE, dtype=torch.uint8, device=DEV)
    return whole, whole[GUARD_BYTES:GUARD_BYTES + size]


def _ws_intact(whole, size):
    return bool((whole[:GUARD_BYTES] == CANARY_BYTE).all()) and bool((whole[GUARD_BYTES + size:] == CANARY_BYTE).all())


@pytest.mark.parametrize("disc,n,m,fp64_form", [
    (h1w.H1W_FV_CELL, (24, 14, 10), 37, False),
    (h1w.H1W_FV_CELL, (24, 14, 10), 37, True),
    (h1w.H1W_FV_CELL, (33, 20, 16), 5, False),     # an odd axis: not coarsened
    (h1w.H1W_Q1_VERTEX, (37, 29), 13, False),
    (h1w.H1W_Q1_VERTEX, (37, 29), 13, True),
])
def test_solver_writes_stay_in_bounds(disc, n, m, fp64_form):
    h = tuple(1.0 / v for v in n)
    alpha = 3e-3
    grid = h1w.make_grid(disc, n, h, alpha)
    opt = h1w.h1w_default_options()
    if fp64_form:
        opt.cap_gemm = 1
        opt.mg_arith = 1
    size = h1w.h1w_workspace_size(grid, m, opt)
    assert size > 0
    ws_whole, ws = _guarded_ws(size)
    N = int(np.prod(n))
    g = torch.Generator(device=DEV).manual_seed(11)
    J_ref = torch.randn(m * N, dtype=torch.float64, device=DEV, generator=g) / N ** 0.5
    b_ref = torch.randn(N, dtype=torch.float64, device=DEV, generator=g)
    J_whole, J = _guarded_vec(m * N, J_ref)
    b_whole, b = _guarded_vec(N, b_ref)
    x_whole, x = _guarded_vec(N)
    z_whole, z = _guarded_vec(N)
    q_whole, q = _guarded_vec(N)
    stream = torch.cuda.current_stream()
    ctx = h1w.h1w_setup(grid, m, opt, ws, stream)
    try:
        h1w.h1w_capacitance(ctx, m, J, N)
        torch.cuda.synchronize()
        assert _ws_intact(ws_whole, size), "capacitance wrote outside the workspace"
        h1w.h1w_apply_prec(ctx, b, z, N)
        h1w.h1w_apply_op(ctx, b, q, N)
        info = h1w.h1w_pcg(ctx, b, x, 1e-10, 300, N)
        torch.cuda.synchronize()
    finally:
        h1w.h1w_destroy(ctx)
    assert info.rel_res_true <= 1e-10
    assert _ws_intact(ws_whole, size), "a call wrote outside the workspace"
    for whole, nn, name in ((J_whole, m * N, "J"), (b_whole, N, "b"), (x_whole, N, "x"), (z_whole, N, "z"),
                            (q_whole, N, "q")):
        assert _bands_intact(whole, nn), f"a write landed outside {name}"
    assert torch.equal(J, J_ref) and torch.equal(b, b_ref), "an input was modified"
    for v in (x, z, q):
        assert torch.isfinite(v).all()


def test_ert_writes_stay_in_bounds():
    n, h = (20, 12, 10), (0.05, 1 / 12, 0.1)
    N = int(np.prod(n))
    rng = np.random.default_rng(4)
    n_e = 6
    cells = rng.choice(n[0] * n[1], size=n_e, replace=False)
    prot = inputs.pair_protocol(n_e)
    abmn = np.stack([prot[:, 0], np.full(len(prot), -1), prot[:, 1], prot[:, 2]], axis=1)
    k = rng.uniform(1.0, 3.0, len(abmn))
    sv = h1w.Survey(cells, abmn, k, inputs.ERT_DIRICHLET_ALL_BUT_TOP)
    S = h1w.Solver(h1w.H1W_FV_CELL, n, h, 1e-2, sv.m, device=DEV)
    size = h1w.h1w_ert_workspace_size(S.ctx, sv.n_e, sv.m)
    ws_whole, ws = _guarded_ws(size)
    ls_ref = torch.tensor(np.log(0.01) + 0.5 * rng.standard_normal(N), device=DEV)
    ls_whole, ls = _guarded_vec(N, ls_ref)
    U_whole, U = _guarded_vec(sv.n_e * N)
    g_whole, gv = _guarded_vec(sv.m)
    r_whole, r = _guarded_vec(sv.m, torch.ones(sv.m, dtype=torch.float64, device=DEV))
    JTr_whole, JTr = _guarded_vec(N)
    Jr_whole, Jrows = _guarded_vec(sv.m * N)
    info = h1w.h1w_forward(S.ctx, sv, ls, U, gv, ws, 1e-10, 200, N)
    h1w.h1w_adjoint(S.ctx, sv, ls, U, r, JTr, Jrows, ws, N)
    torch.cuda.synchronize()
    assert info.rel_res_true <= 1e-9
    assert _ws_intact(ws_whole, size), "the ERT calls wrote outside their workspace"
    for whole, nn, name in ((ls_whole, N, "logsigma"), (U_whole, sv.n_e * N, "U"), (g_whole, sv.m, "g"),
                            (r_whole, sv.m, "r"), (JTr_whole, N, "JTr"), (Jr_whole, sv.m * N, "J")):
        assert _bands_intact(whole, nn), f"a write landed outside {name}"
    assert torch.equal(ls, ls_ref)
    for v in (U, gv, JTr, Jrows):
        assert torch.isfinite(v).all()
