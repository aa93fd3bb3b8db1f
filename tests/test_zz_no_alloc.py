"""The allocation-free operator apply, h1w_apply_op_static.

It serves callers that cannot call cudaMalloc (their device memory belongs to
another allocator, such as a framework's caching pool or a fixed arena), so it
keeps its scratch in a fixed file-scope device array instead of a
caller-provided workspace. This file checks, through the C ABI, that it
returns what the workspace-based h1w_apply_op returns, on two calls in a row
(the second call reuses the array the first one left behind), and that sizes
beyond the array are refused. It is named to be collected last.
"""
import numpy as np
import pytest
import torch

from paper_2209_02815_gb300 import h1w

pytestmark = pytest.mark.gpu
DEV = "cuda"
RTOL = 1e-12  # the operator-apply tolerance of the parity tests


def _rel(a, b):
    a, b = a.double().cpu().numpy(), b.double().cpu().numpy()
    return float(np.linalg.norm(a - b) / np.linalg.norm(b))


@pytest.mark.parametrize("disc,n,h", [
    (h1w.H1W_FV_CELL, (40, 24, 20), (1 / 40, 1 / 24, 1 / 20)),
    (h1w.H1W_Q1_VERTEX, (130, 67), (1 / 129, 1 / 66)),
])
def test_static_apply_matches_workspace_apply_twice(disc, n, h):
    alpha, m = 3e-3, 37
    S = h1w.Solver(disc, n, h, alpha, m, device=DEV)
    g = torch.Generator(device=DEV).manual_seed(7)
    J = torch.randn(m, S.N, dtype=torch.float64, device=DEV, generator=g) / S.N ** 0.5
    S.capacitance(J)
    grid = h1w.make_grid(disc, n, h, alpha)
    for call in range(2):
        p = torch.randn(S.N, dtype=torch.float64, device=DEV, generator=g)
        q_ref = S.apply_op(p)
        q = torch.full_like(p, float("nan"))
        h1w.h1w_apply_op_static(grid, m, J, p, q, S.N)
        torch.cuda.synchronize()
        assert torch.isfinite(q).all(), f"call {call}"
        assert _rel(q, q_ref) <= RTOL, f"call {call}"


def test_static_apply_rejects_sizes_beyond_scratch():
    """256^3 cells with 4000 rows need 4096 * 4000 partial sums, more than the
    2^20-double array: refused on the host before any launch (J is never read)."""
    n = (256, 256, 256)
    grid = h1w.make_grid(h1w.H1W_FV_CELL, n, (1 / 256,) * 3, 1e-3)
    N = 256 ** 3
    J = torch.zeros(8, dtype=torch.float64, device=DEV)
    p = torch.zeros(N, dtype=torch.float64, device=DEV)
    q = torch.zeros_like(p)
    st = h1w.load().h1w_apply_op_static(grid, 4000, J.data_ptr(), p.data_ptr(), q.data_ptr(), None)
    assert st == h1w.H1W_EINVAL
    assert "static scratch" in h1w.h1w_last_error(None)
    assert float(q.abs().max()) == 0.0
