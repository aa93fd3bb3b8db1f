"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/h1w.h declares. No GPU needed (no compute call is made)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared(header: str) -> list[str]:
    text = open(os.path.join(ROOT, "include", header)).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(h1w_[a-z_0-9]+)\s*\(", text)))


def test_library_exports_every_declared_symbol():
    from paper_2209_02815_gb300 import build
    path = build.build()
    lib = ctypes.CDLL(path)
    names = []
    for hdr in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if hdr.endswith(".h"):
            names += _declared(hdr)
    assert "h1w_pcg" in names and "h1w_capacitance" in names
    for n in names:
        assert hasattr(lib, n), n


def test_host_side_validation_without_gpu():
    """Workspace sizing and argument checks run on the host only."""
    from paper_2209_02815_gb300 import h1w
    g = h1w.make_grid(h1w.H1W_FV_CELL, (128, 128, 128), (1 / 128,) * 3, 1e-3)
    size = h1w.h1w_workspace_size(g, 496)
    N = 128 ** 3
    assert size > 496 * N * 8  # H as double-floats plus the multigrid vectors
    bad = h1w.make_grid(h1w.H1W_FV_CELL, (33, 33, 33), (1 / 33,) * 3, 1e-3)
    assert h1w.h1w_workspace_size(bad, 4) == 0  # cannot coarsen to <= 1024 unknowns
    neg = h1w.make_grid(h1w.H1W_Q1_VERTEX, (64, 64), (1 / 63,) * 2, -1.0)
    assert h1w.h1w_workspace_size(neg, 4) == 0
    o = h1w.h1w_default_options()
    assert (o.cheb_degree, o.rhs_block, o.max_restarts, o.j_digits) == (2, 128, 3, 1)
    # J's digits for every K panel are kept when they fit: a larger workspace than with j_digits = 0
    o0 = h1w.h1w_default_options()
    o0.j_digits = 0
    assert size > h1w.h1w_workspace_size(g, 496, o0) + 496 * N * 8
    o0.j_digits = 2
    assert h1w.h1w_workspace_size(g, 496, o0) == 0


def test_rhs_block_buffers_capped_at_m_max():
    """A context never batches more right-hand sides than it has rows of J, so its
    V-cycle block buffers are sized for min(rhs_block, m_max)."""
    from paper_2209_02815_gb300 import h1w
    g = h1w.make_grid(h1w.H1W_Q1_VERTEX, (256, 256), (1 / 255,) * 2, 1e-3)
    sizes = {}
    for rb in (8, 64, 128):
        o = h1w.h1w_default_options()
        o.rhs_block = rb
        sizes[rb] = h1w.h1w_workspace_size(g, 8, o)
    assert sizes[8] == sizes[64] == sizes[128] > 0
    o = h1w.h1w_default_options()
    o.rhs_block = 4
    assert 0 < h1w.h1w_workspace_size(g, 8, o) < sizes[8]


def test_new_entry_points_reject_null_context_without_gpu():
    """The ERT, Gauss-Newton and direct-solve entry points check their context on the
    host; the options default to the Laplace-Woodbury preconditioner."""
    from paper_2209_02815_gb300 import h1w
    lib = h1w.load()
    assert lib.h1w_ert_workspace_size(None, 4, 10) == 0
    assert lib.h1w_direct_workspace_size(None) == 0
    sv = h1w.Survey([0], [[0, -1, 0, -1]], [1.0], 0b101111)
    assert lib.h1w_forward(None, ctypes.byref(sv.c), None, None, None, None, 0, 1e-10, 10, 0, None) == h1w.H1W_EINVAL
    assert lib.h1w_adjoint(None, ctypes.byref(sv.c), None, None, None, None, None, None, 0) == h1w.H1W_EINVAL
    assert lib.h1w_ert_jvp(None, ctypes.byref(sv.c), None, None, None, None, None, 0) == h1w.H1W_EINVAL
    assert lib.h1w_solve_direct(None, None, None, None, 0) == h1w.H1W_EINVAL
    assert lib.h1w_pcg_host(None, None, None, 1e-8, 10, None) == h1w.H1W_EINVAL
    assert lib.h1w_gn_step(None, ctypes.byref(sv.c), None, None, None, None, None, None, None, None, 0, 1e-10, 1e-8,
                           10, 0, None) == h1w.H1W_EINVAL
    assert h1w.h1w_default_options().precond == 0
    bad = h1w.h1w_default_options()
    bad.precond = 2
    g = h1w.make_grid(h1w.H1W_FV_CELL, (32, 32, 32), (1 / 32,) * 3, 1e-3)
    assert h1w.h1w_workspace_size(g, 8, bad) == 0
