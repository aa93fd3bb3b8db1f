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


@pytest.mark.parametrize("disc,n,h,m", [
    (h1w.H1W_FV_CELL, (40, 24, 20), (1 / 40, 1 / 24, 1 / 20), 37),
    (h1w.H1W_FV_CELL, (32, 32, 32), (1 / 32,) * 3, 37),      # isotropic: the equal-T stencil branch
    (h1w.H1W_FV_CELL, (24, 16, 20), (1 / 24, 1 / 16, 1 / 20), 0),
    (h1w.H1W_Q1_VERTEX, (130, 67), (1 / 129, 1 / 66), 37),
    (h1w.H1W_Q1_VERTEX, (64, 64), (1 / 63,) * 2, 0),
])
def test_static_apply_matches_workspace_apply_twice(disc, n, h, m):
    alpha = 3e-3
    S = h1w.Solver(disc, n, h, alpha, max(m, 1), device=DEV)
    g = torch.Generator(device=DEV).manual_seed(7)
    J = torch.randn(m, S.N, dtype=torch.float64, device=DEV, generator=g) / S.N ** 0.5 if m else None
    S.capacitance(J)
    grid = h1w.make_grid(disc, n, h, alpha)
    ps = [torch.randn(S.N, dtype=torch.float64, device=DEV, generator=g) for _ in range(2)]
    qs = [torch.full_like(ps[0], float("nan")) for _ in range(2)]
    refs = [S.apply_op(p) for p in ps]
    torch.cuda.synchronize()
    for call in range(2):
        if call == 1:  # the entry point allocates nothing: device memory is the same after the call
            free0 = torch.cuda.mem_get_info()[0]
            alloc0 = torch.cuda.memory_allocated()
        h1w.h1w_apply_op_static(grid, m, J, ps[call], qs[call], S.N)
        torch.cuda.synchronize()
        if call == 1:
            assert torch.cuda.mem_get_info()[0] == free0
            assert torch.cuda.memory_allocated() == alloc0
        assert torch.isfinite(qs[call]).all(), f"call {call}"
        assert _rel(qs[call], refs[call]) <= RTOL, f"call {call}"


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
