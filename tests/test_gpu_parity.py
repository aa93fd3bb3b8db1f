"""Parity of the CUDA path (through the C ABI) with the FP64 CPU oracle.

Sizes span several 256-thread blocks and multigrid levels with ragged tails
(grid sides that are not multiples of the tile or of powers of two), plus the
degenerate cases m = 0 and m = 1.

Tolerances (FP64 throughout). Both sides evaluate the same formulas in FP64
but with different summation orders, so each elementary result differs by a
few units of roundoff, amplified by the conditioning of the step:
* V-cycle, operator apply, right-hand side: 1e-12 relative (norm-wise), the
  operators have O(1)-conditioned rounding (tens of flops per entry).
* capacitance C: 1e-11 relative, a sum of N products (error ~ sqrt(N) eps).
* Cholesky factor and preconditioner apply: 1e-9 relative, the error of C is
  amplified by at most cond(C) (<= 1e3 for the cases here).
* solution of the system: 1e-9 relative to the dense direct solve, the
  bound stated for FP64 paths; PCG is run to rtol 1e-12 (C1) so that
  cond(A) * rtol stays below it.
"""
import numpy as np
import pytest
import torch

from oracle import ccg
from oracle import discretization as disc
from oracle import multigrid as mg
from oracle import woodbury as wb
from paper_2209_02815_gb300 import h1w, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda"

Q1_CASES = [(29, 23), (64, 64), (37, 41), (130, 67)]
FV_CASES = [(16, 8, 12), (24, 24, 24), (20, 12, 28)]


def _q1(n):
    return "q1", tuple(n), tuple(1.0 / (v - 1) for v in n)


def _fv(n):
    return "fv", tuple(n), tuple(1.0 / v for v in n)


def _gpu(d, n, h, alpha, m_max, **opt):
    o = None
    if opt:
        o = h1w.h1w_default_options()
        for k, v in opt.items():
            setattr(o, k, v)
    code = h1w.H1W_Q1_VERTEX if d == "q1" else h1w.H1W_FV_CELL
    return h1w.Solver(code, n, h, alpha, m_max, device=DEV, opt=o)


def _t(a):
    return torch.as_tensor(np.ascontiguousarray(a), dtype=torch.float64, device=DEV)


def _rel(a, b):
    return float(np.linalg.norm(np.asarray(a) - np.asarray(b)) / max(np.linalg.norm(np.asarray(b)), 1e-300))


ALL = [_q1(n) for n in Q1_CASES] + [_fv(n) for n in FV_CASES]


@pytest.mark.parametrize("case", ALL, ids=lambda c: f"{c[0]}{'x'.join(map(str, c[1]))}")
def test_hierarchy_matches_oracle(case):
    d, n, h = case
    H = mg.build_hierarchy(d, n, h)
    S = _gpu(d, n, h, 1e-2, 4)
    lv = S.levels()
    want = [tuple(list(l.n) + [1] * (3 - len(l.n))) for l in H.levels]
    assert lv == want


VC_CASES = [(c, a) for c in ALL for a in (0, 1)]


@pytest.mark.parametrize("case,mg_arith", VC_CASES,
                         ids=lambda v: f"{v[0]}{'x'.join(map(str, v[1]))}" if isinstance(v, tuple)
                         else ("df64" if v == 0 else "fp64"))
def test_vcycle_parity(case, mg_arith):
    """FP64 cycle and double-float cycle (FP32 pairs of about 48 bits: errors
    of a few 1e-15 per operation, ~1e-13 over a cycle), on Q1 and FV grids,
    against the oracle's V-cycle, relative error 1e-12."""
    d, n, h = case
    H = mg.build_hierarchy(d, n, h)
    N = H.N
    rng = np.random.default_rng(21)
    B = rng.standard_normal((3, N))
    S = _gpu(d, n, h, 1e-2, 4, rhs_block=2, mg_arith=mg_arith)  # 3 right-hand sides: blocks of 2 and 1
    X = S.vcycle(_t(B)).cpu().numpy()
    for r in range(3):
        ref = mg.vcycle(H, B[r])
        assert _rel(X[r], ref) <= 1e-12


# Grids for the fused double-float legs: ragged xy tiles (sides not multiples of
# 32 x 16 fine cells), several z segments, a level that is coarsened along two axes
# only (a 9-cell side), and a coarsest level reached after semi-coarsening.
FUSED_GRIDS = [(16, 8, 12), (24, 24, 24), (20, 12, 28), (72, 40, 36), (24, 9, 16), (64, 64, 64), (48, 100, 20)]


@pytest.mark.parametrize("n", FUSED_GRIDS, ids=lambda n: "x".join(map(str, n)))
def test_fused_cycle_matches_unfused(n):
    """The fused legs evaluate the two Chebyshev steps in collapsed form (the same
    linear map as the one-kernel-per-step recurrence, different rounding), so the
    cycles agree to double-float accuracy: relative 1e-13. Within the fused path
    every cell is computed by the same operations whichever block owns it, so
    blocks of 4 and of 1 right-hand sides (different z segmentations and halo
    overlaps) agree bit for bit."""
    d, n, h = _fv(n)
    N = int(np.prod(n))
    rng = np.random.default_rng(31)
    B = _t(rng.standard_normal((5, N)))
    a = _gpu(d, n, h, 1e-2, 4, rhs_block=4, mg_unfused=0).vcycle(B)
    b = _gpu(d, n, h, 1e-2, 4, rhs_block=4, mg_unfused=1).vcycle(B)
    for r in range(5):
        assert _rel(a[r].cpu().numpy(), b[r].cpu().numpy()) <= 1e-13
    c1 = _gpu(d, n, h, 1e-2, 4, rhs_block=1, mg_unfused=0).vcycle(B)
    assert torch.equal(a, c1)


@pytest.mark.parametrize("n", [(72, 40, 36), (48, 100, 20)], ids=lambda n: "x".join(map(str, n)))
def test_fused_cycle_parity_larger_grids(n):
    """Fused double-float cycle against the oracle's FP64 V-cycle, relative 1e-12."""
    d, n, h = _fv(n)
    H = mg.build_hierarchy(d, n, h)
    rng = np.random.default_rng(32)
    B = rng.standard_normal((2, H.N))
    X = _gpu(d, n, h, 1e-2, 4).vcycle(_t(B)).cpu().numpy()
    for r in range(2):
        assert _rel(X[r], mg.vcycle(H, B[r])) <= 1e-12


@pytest.mark.parametrize("case", ALL, ids=lambda c: f"{c[0]}{'x'.join(map(str, c[1]))}")
def test_apply_op_and_rhs_parity(case):
    d, n, h = case
    A = disc.regularization_operator(d, n, h)
    N = A.shape[0]
    rng = np.random.default_rng(22)
    m, alpha = 7, 3e-3
    J = rng.standard_normal((m, N)) / np.sqrt(N)
    p = rng.standard_normal(N)
    S = _gpu(d, n, h, alpha, m)
    Jt = _t(J)
    S.capacitance(Jt)
    q = S.apply_op(_t(p)).cpu().numpy()
    assert _rel(q, wb.apply_operator(A, alpha, J, p)) <= 1e-12
    dm = rng.standard_normal(N)
    dd = rng.standard_normal(m)
    b = S.gn_rhs(_t(dm), _t(dd)).cpu().numpy()
    assert _rel(b, wb.gn_rhs(A, alpha, dm, J, dd)) <= 1e-12


@pytest.mark.parametrize("case", ALL, ids=lambda c: f"{c[0]}{'x'.join(map(str, c[1]))}")
@pytest.mark.parametrize("m", [1, 13, 70])
@pytest.mark.parametrize("cap_gemm", [0, 1], ids=["tensor", "fp64"])
def test_capacitance_and_prec_parity(case, m, cap_gemm):
    """C, its Cholesky factor and the preconditioner, with line C on the tensor
    cores (49-bit digit split per 512-entry chunk: error below about 2^-48 of the
    chunk maxima, i.e. far below 1e-11 of ||C|| for these Gaussian rows) or on the
    FP64 CUDA cores."""
    d, n, h = case
    H = mg.build_hierarchy(d, n, h)
    N = H.N
    rng = np.random.default_rng(23 + m)
    alpha = 1e-2
    J = rng.standard_normal((m, N)) / np.sqrt(N)
    P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), J, alpha)
    S = _gpu(d, n, h, alpha, m, rhs_block=16, cap_gemm=cap_gemm)
    S.capacitance(_t(J))
    C, L = (t.cpu().numpy() for t in S.factors())
    assert np.array_equal(C, C.T)
    assert _rel(C, P.C) <= 1e-11
    assert _rel(L, np.linalg.cholesky(P.C)) <= 1e-9
    r = rng.standard_normal(N)
    z = S.apply_prec(_t(r)).cpu().numpy()
    assert _rel(z, P(r)) <= 1e-9


@pytest.mark.parametrize("case", [_fv((24, 24, 24)), _fv((20, 12, 28)), _q1((130, 67))],
                         ids=lambda c: f"{c[0]}{'x'.join(map(str, c[1]))}")
@pytest.mark.parametrize("m", [13, 150])
def test_j_digits_in_line_h_equal_per_panel_split(case, m):
    """j_digits = 1 splits J into the GEMM's digits while line H converts it (digits of every
    K panel kept), j_digits = 0 splits it per panel in line C: the same digits, so C, L and
    the PCG solution (whose passes read the double-float copy of J written by either path)
    agree bit for bit; with more than one 128-row block (m = 150) the padding rows of the
    last block are zero in both."""
    d, n, h = case
    N = int(np.prod(n))
    rng = np.random.default_rng(61 + m)
    J = _t(rng.standard_normal((m, N)) / np.sqrt(N))
    b = _t(rng.standard_normal(N))
    out = []
    for jd in (1, 0):
        S = _gpu(d, n, h, 1e-2, m, j_digits=jd, rhs_block=64)
        S.capacitance(J)
        C, L = S.factors()
        x, info = S.pcg(b, 1e-11, 300)
        out.append((C.clone(), L.clone(), x.clone(), info.iters))
    assert torch.equal(out[0][0], out[1][0]) and torch.equal(out[0][1], out[1][1])
    assert torch.equal(out[0][2], out[1][2]) and out[0][3] == out[1][3]


def test_m0_prec_is_scaled_vcycle():
    d, n, h = _fv((16, 8, 12))
    H = mg.build_hierarchy(d, n, h)
    S = _gpu(d, n, h, 0.25, 4)
    S.capacitance(None)
    r = np.random.default_rng(5).standard_normal(H.N)
    z = S.apply_prec(_t(r)).cpu().numpy()
    assert _rel(z, mg.vcycle(H, r) / 0.25) <= 1e-12


def test_pcg_small_2d_matches_dense_solve():
    """The 64 x 64 Q1 problem: J ~ N(0,1)/64 (16 rows), alpha = 1e-2, rtol 1e-12."""
    pr = inputs.small_c1_problem()
    A = disc.regularization_operator("q1", (pr.nx, pr.ny), pr.h)
    x_ref = np.linalg.solve(pr.alpha * A.toarray() + pr.J.T @ pr.J, pr.b)
    H = mg.build_hierarchy("q1", (pr.nx, pr.ny), pr.h)
    P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), pr.J, pr.alpha)
    _, it_ref, _ = wb.pcg(lambda v: wb.apply_operator(A, pr.alpha, pr.J, v), P, pr.b, 1e-12, 200)
    S = _gpu("q1", (pr.nx, pr.ny), pr.h, pr.alpha, pr.J.shape[0])
    S.capacitance(_t(pr.J))
    x, info = S.pcg(_t(pr.b), 1e-12, 200)
    x = x.cpu().numpy()
    assert info.rel_res_true <= 1e-12
    assert _rel(x, x_ref) <= 1e-9
    assert abs(info.iters - it_ref) <= 1


@pytest.mark.parametrize("case", [_fv((24, 24, 24)), _q1((130, 67)), _fv((20, 12, 28))],
                         ids=["fv24", "q1_130x67", "fv20x12x28"])
@pytest.mark.parametrize("alpha,rtol,xtol", [(1e-1, 1e-11, 1e-9), (1e-2, 1e-11, 1e-9), (1e-4, 1e-8, None)])
def test_pcg_matches_oracle_pcg(case, alpha, rtol, xtol):
    """rtol is chosen above the attainable accuracy eps * cond(A) of each case
    (alpha = 1e-4 on the FV grids has cond(A) ~ 1e8); where cond(A) * rtol
    exceeds 1e-9 only the residual and the iteration count are compared."""
    d, n, h = case
    A = disc.regularization_operator(d, n, h)
    N = A.shape[0]
    rng = np.random.default_rng(31)
    m = 40
    J = rng.standard_normal((m, N)) / np.sqrt(N)
    b = rng.standard_normal(N)
    H = mg.build_hierarchy(d, n, h)
    P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), J, alpha)
    x_ref, it_ref, rel_ref = wb.pcg(lambda v: wb.apply_operator(A, alpha, J, v), P, b, rtol, 300)
    assert rel_ref <= rtol
    S = _gpu(d, n, h, alpha, m)
    S.capacitance(_t(J))
    x, info = S.pcg(_t(b), rtol, 300)
    assert info.rel_res_true <= rtol
    if xtol is not None:
        assert _rel(x.cpu().numpy(), x_ref) <= xtol
    assert abs(info.iters - it_ref) <= 1
    # the true residual agrees with the C oracle's operator
    op = ccg.CsrOperator(A, alpha, J)
    rt = b - op.apply(x.cpu().numpy())
    assert np.linalg.norm(rt) <= 1.5 * rtol * np.linalg.norm(b)


def test_ert_small_gn_step():
    """A 32^3 ERT step (analytic half-space sensitivities, 8 line electrodes):
    b from Eq. 2.9, solution vs the oracle's PCG."""
    pr = inputs.ert_problem(32, n_e_line=8, alpha=1e-3)
    n = (32, 32, 32)
    h = (pr.h,) * 3
    A = disc.regularization_operator("fv", n, h)
    dm = pr.logsigma - pr.m_ref
    b_ref = wb.gn_rhs(A, pr.alpha, dm, pr.J, pr.d)
    H = mg.build_hierarchy("fv", n, h)
    P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), pr.J, pr.alpha)
    x_ref, it_ref, _ = wb.pcg(lambda v: wb.apply_operator(A, pr.alpha, pr.J, v), P, b_ref, 1e-10, 300)
    S = _gpu("fv", n, h, pr.alpha, pr.J.shape[0])
    S.capacitance(_t(pr.J))
    b = S.gn_rhs(_t(dm), _t(pr.d))
    assert _rel(b.cpu().numpy(), b_ref) <= 1e-12
    x, info = S.pcg(b, 1e-10, 300)
    assert info.rel_res_true <= 1e-10
    xg = x.cpu().numpy()
    op = ccg.CsrOperator(A, pr.alpha, pr.J)
    assert np.linalg.norm(b_ref - op.apply(xg)) <= 1.5e-10 * np.linalg.norm(b_ref)
    # both iterates satisfy the same residual bound; their difference is at
    # most cond(A) * rtol and is printed for the record
    print("ert32: iters gpu/oracle", info.iters, it_ref, "rel diff", _rel(xg, x_ref))
    assert abs(info.iters - it_ref) <= 2


def test_status_codes():
    d, n, h = _fv((16, 8, 12))
    S = _gpu(d, n, h, 1e-2, 4)
    b = torch.randn(S.N, dtype=torch.float64, device=DEV)
    with pytest.raises(h1w.H1wError) as e:
        S.pcg(b, 1e-8)
    assert e.value.status == h1w.H1W_ESTATE
    J = torch.randn(4, S.N, dtype=torch.float64, device=DEV) / S.N ** 0.5
    S.capacitance(J)
    x, info = S.pcg(b, 1e-14, maxit=1, raise_on_notconv=False)
    assert info.iters == 1 and info.rel_res_true > 1e-14
    with pytest.raises(h1w.H1wError) as e:
        S.pcg(b, 1e-14, maxit=1)
    assert e.value.status == h1w.H1W_ENOTCONV
    with pytest.raises(h1w.H1wError) as e:
        h1w.h1w_capacitance(S.ctx, 5, torch.zeros(5 * S.N, dtype=torch.float64, device=DEV), S.N)
    assert e.value.status == h1w.H1W_EINVAL
    g = h1w.make_grid(h1w.H1W_FV_CELL, n, h, 1e-2)
    small = torch.empty(1024, dtype=torch.uint8, device=DEV)
    with pytest.raises(h1w.H1wError) as e:
        h1w.h1w_setup(g, 4, None, small)
    assert e.value.status == h1w.H1W_ENOMEM
    bad = h1w.make_grid(h1w.H1W_FV_CELL, (33, 33, 33), (1 / 33,) * 3, 1e-2)
    with pytest.raises(h1w.H1wError) as e:
        h1w.h1w_setup(bad, 4, None, torch.empty(1 << 20, dtype=torch.uint8, device=DEV))
    assert e.value.status == h1w.H1W_EUNSUPPORTED
    # zero right-hand side: x = 0, no iterations
    x, info = S.pcg(torch.zeros_like(b), 1e-8)
    assert info.iters == 0 and float(x.abs().max()) == 0.0


@pytest.mark.parametrize("n,m", [((72, 64, 64), 150), ((40, 36, 20), 300), ((96, 96, 96), 40)],
                         ids=["2panels_m150", "m300", "4panels_m40"])
def test_tensor_capacitance_matches_fp64(n, m):
    """Line C on the tensor cores against the FP64 CUDA-core GEMM on the same
    GPU-built H (more than one 262144-wide K panel, up to four, ragged tiles): the
    digit split keeps 49 bits of every chunk of a row, so C agrees to ~1e-11 of ||C||."""
    h = tuple(1.0 / v for v in n)
    N = int(np.prod(n))
    rng = np.random.default_rng(41)
    J = _t(rng.standard_normal((m, N)) * rng.uniform(0.1, 10.0, size=(m, 1)) / np.sqrt(N))
    Cs = []
    for mode in (0, 1):
        S = _gpu("fv", n, h, 1e-3, m, cap_gemm=mode)
        S.capacitance(J)
        C, L = S.factors()
        Cs.append(C.cpu().numpy())
    assert np.array_equal(Cs[0], Cs[0].T)
    assert np.linalg.norm(Cs[0] - Cs[1]) <= 1e-11 * np.linalg.norm(Cs[1])


def test_tensor_capacitance_on_peaked_ert_rows():
    """ERT sensitivity rows peak sharply at the electrodes and C reaches ~1e9.
    The preconditioner stays within a few percent of the exact one only if
    the absolute error of C is far below 1; the chunk-scaled digit split keeps
    ||C_tensor - C_fp64||_2 of order 1e-3 or less here (an exact CPU emulation of
    the base-64 split gave 1.6e-3 at 64^3; the base-128 one is more accurate),
    checked against 2e-2."""
    n = 48
    pr = inputs.ert_problem(n, n_e_line=32, alpha=1e-3, device=DEV)
    Cs = []
    for mode in (0, 1):
        S = _gpu("fv", (n,) * 3, (1.0 / n,) * 3, 1e-3, pr.J.shape[0], cap_gemm=mode)
        S.capacitance(pr.J)
        Cs.append(S.factors()[0].cpu().numpy())
        del S
    E = Cs[0] - Cs[1]
    assert np.linalg.norm(Cs[1], 2) > 1e8          # the ill-conditioned regime
    assert np.linalg.norm(E, 2) <= 2e-2


@pytest.mark.parametrize("rhs_block", [32, 5])
def test_capacitance_from_host_equals_device_path(rhs_block):
    """J streamed from pinned host memory in row batches under line H gives the
    same C and Cholesky factor, bit for bit, as the device entry point, and
    leaves an exact copy of J in the destination buffer."""
    d, n, h = _fv((24, 24, 24))
    N = int(np.prod(n))
    m = 70
    rng = np.random.default_rng(41)
    Jh = torch.as_tensor(rng.standard_normal((m, N)) / np.sqrt(N)).pin_memory()
    Jd = Jh.to(DEV)
    a = _gpu(d, n, h, 1e-2, m, rhs_block=rhs_block)
    a.capacitance(Jd)
    Ca, La = a.factors()
    b = _gpu(d, n, h, 1e-2, m, rhs_block=rhs_block)
    Jdst = torch.empty_like(Jd)
    b.capacitance_from_host(Jh, Jdst)
    Cb, Lb = b.factors()
    assert torch.equal(Jdst, Jd)
    assert torch.equal(Ca, Cb) and torch.equal(La, Lb)


@pytest.mark.parametrize("rhs_block", [128, 20])
def test_prefetched_capacitance_from_host_equals_device_path(rhs_block):
    """Double-buffered prefetch (h1w_prefetch_J) of the next system's J during the current
    solve: three systems in a row, each capacitance bit-identical to the device entry point,
    the solutions equal, and the per-batch copy profile is ordered (each batch's cycles
    start after the copy of its rows ended). A prefetched J is consumed in rhs_block
    batches; with 20 they straddle the copy's batches (16, 20, 20, 14 rows)."""
    d, n, h = _fv((24, 24, 24))
    N = int(np.prod(n))
    m = 70
    rng = np.random.default_rng(43)
    Jhs = [torch.as_tensor(rng.standard_normal((m, N)) / np.sqrt(N)).pin_memory() for _ in range(3)]
    b = _t(rng.standard_normal(N))
    ref = _gpu(d, n, h, 1e-2, m, rhs_block=rhs_block)
    S = _gpu(d, n, h, 1e-2, m, rhs_block=rhs_block)
    bufs = [torch.empty((m, N), dtype=torch.float64, device=DEV) for _ in range(2)]
    S.prefetch_J(Jhs[0], bufs[0])
    for k in range(3):
        if k + 1 < 3:
            S.prefetch_J(Jhs[k + 1], bufs[(k + 1) % 2])
        S.capacitance_from_host(Jhs[k], bufs[k % 2])
        prof = S.copy_profile()
        assert sum(p["rows"] for p in prof) == m
        for p in prof:
            assert p["copy_end"] >= p["copy_begin"]
            assert p["cycle_begin"] >= p["copy_end"] - 1e-3
        C, L = S.factors()
        x, _ = S.pcg(b, 1e-12, 200)
        ref.capacitance(Jhs[k].to(DEV))
        Cr, Lr = ref.factors()
        xr, _ = ref.pcg(b, 1e-12, 200)
        assert torch.equal(bufs[k % 2], Jhs[k].to(DEV))
        assert torch.equal(C, Cr) and torch.equal(L, Lr)
        assert torch.equal(x, xr)


@pytest.mark.parametrize("pcg_mode", [0, 1])
def test_pcg_host_equals_device_pcg(pcg_mode):
    """h1w_pcg_host (b read from, x written to pinned host memory by kernels) gives bit for bit
    the solution and iteration count of h1w_pcg on device vectors, in both loop forms, with the
    next system's J prefetched beside it; pageable host memory is refused with H1W_EINVAL."""
    d, n, h = _fv((24, 16, 20))
    N = int(np.prod(n))
    m = 33
    rng = np.random.default_rng(44)
    Jh = torch.as_tensor(rng.standard_normal((m, N)) / np.sqrt(N)).pin_memory()
    b = _t(rng.standard_normal(N))
    S = _gpu(d, n, h, 1e-2, m, pcg_mode=pcg_mode)
    bufs = [torch.empty((m, N), dtype=torch.float64, device=DEV) for _ in range(2)]
    S.capacitance_from_host(Jh, bufs[0])
    xd, infod = S.pcg(b, 1e-11, 300)
    xd = xd.clone()
    b_host = b.cpu().pin_memory()
    x_host = torch.full((N,), float("nan"), dtype=torch.float64).pin_memory()
    S.prefetch_J(Jh, bufs[1])
    info = S.pcg_host(b_host, x_host, 1e-11, 300)
    assert info.iters == infod.iters and info.rel_res_true == infod.rel_res_true
    assert torch.equal(x_host, xd.cpu())
    S.capacitance_from_host(Jh, bufs[1])
    info2 = S.pcg_host(b_host, x_host, 1e-11, 300)
    assert info2.iters == infod.iters and torch.equal(x_host, xd.cpu())
    pageable = torch.zeros(N, dtype=torch.float64)
    st = h1w.load().h1w_pcg_host(S.ctx, pageable.data_ptr(), x_host.data_ptr(), 1e-11, 300, None)
    assert st == h1w.H1W_EINVAL
    assert "page-locked" in h1w.h1w_last_error(S.ctx)


def test_prefetch_rejects_a_third_pending_copy():
    d, n, h = _fv((16, 8, 12))
    N = int(np.prod(n))
    m = 9
    S = _gpu(d, n, h, 1e-2, m)
    Jh = torch.zeros((m, N), dtype=torch.float64).pin_memory()
    bufs = [torch.empty((m, N), dtype=torch.float64, device=DEV) for _ in range(3)]
    S.prefetch_J(Jh, bufs[0])
    S.prefetch_J(Jh, bufs[1])
    with pytest.raises(h1w.H1wError) as ei:
        S.prefetch_J(Jh, bufs[2])
    assert ei.value.status == h1w.H1W_ESTATE
    S.capacitance_from_host(Jh, bufs[0])
    S.capacitance_from_host(Jh, bufs[1])


def test_solve_batch_matches_individual_solves():
    """Systems of different grids, discretizations and measurement counts
    (including m = 0), solved together by h1w_solve_batch on their own streams,
    give bit for bit the solutions of solving each alone."""
    cases = [(_q1((64, 64)), 16), (_fv((24, 24, 24)), 30), (_q1((37, 41)), 5), (_fv((16, 8, 12)), 0),
             (_fv((20, 12, 28)), 9)]
    rng = np.random.default_rng(51)
    solvers, Js, bs, xs, refs = [], [], [], [], []
    for (d, n, h), m in cases:
        N = int(np.prod(n))
        J = _t(rng.standard_normal((m, N)) / np.sqrt(N)) if m else None
        b = _t(rng.standard_normal(N))
        code = h1w.H1W_Q1_VERTEX if d == "q1" else h1w.H1W_FV_CELL
        solvers.append(h1w.Solver(code, n, h, 1e-2, max(m, 1), device=DEV, stream=torch.cuda.Stream()))
        Js.append(J)
        bs.append(b)
        xs.append(torch.empty_like(b))
        R = _gpu(d, n, h, 1e-2, max(m, 1))
        R.capacitance(J)
        xr, _ = R.pcg(b, 1e-10)
        refs.append(xr)
    torch.cuda.synchronize()
    infos, sts = h1w.solve_batch(solvers, Js, bs, xs, 1e-10, threads=3)
    assert all(s == h1w.H1W_OK for s in sts)
    for x, xr, inf in zip(xs, refs, infos):
        assert torch.equal(x, xr)
        assert inf.rel_res_true <= 1e-10


def test_cholesky_under_concurrent_load():
    """The capacitance Cholesky (several 32-row panels) while another stream keeps the
    SMs busy, so that the blocks of a panel start at different times: the factor must
    equal numpy's Cholesky of the returned C every time. (A block that started after
    the diagonal block was written back would factor L11 instead of A11.)"""
    d, n, h = _q1((128, 128))
    m = 256
    rng = np.random.default_rng(61)
    J = _t(rng.standard_normal((m, n[0] * n[1])) / n[0])
    S = _gpu(d, n, h, 1e-3, m, rhs_block=m)
    side = torch.cuda.Stream()
    A = torch.randn(4096, 4096, device=DEV)
    for _ in range(6):
        with torch.cuda.stream(side):
            for _ in range(8):
                A = torch.tanh(A @ A * 1e-3)
        S.capacitance(J)
        C, L = (t.cpu().numpy() for t in S.factors())
        assert _rel(L, np.linalg.cholesky(C)) <= 1e-10
    torch.cuda.synchronize()


def test_solve_batch_orders_streams():
    """Solvers on their own streams, created right after their J was generated on
    the current stream (no synchronize in between), and more systems than host
    threads: every system must succeed and match solving it alone on the same
    context bit for bit. The binding orders each context's stream after the current
    one, so neither the inputs nor memory the caching allocator recycles into a
    workspace can be read or overwritten early."""
    descs = inputs.batch_instances(12, sides=(128, 256), ms=(32, 256), alpha_range=(1e-4, 1e-3), seed=77)
    solvers, Js, bs, xs = [], [], [], []
    for d in descs:
        n = d["n"]
        J, b = inputs.batch_instance_data(d, device=DEV)
        solvers.append(h1w.Solver(h1w.H1W_Q1_VERTEX, (n, n), (1.0 / (n - 1),) * 2, d["alpha"], d["m"], device=DEV,
                                  stream=torch.cuda.Stream()))
        Js.append(J)
        bs.append(b)
        xs.append(torch.empty_like(b))
    infos, sts = h1w.solve_batch(solvers, Js, bs, xs, 1e-8, threads=4)
    assert all(s_ == h1w.H1W_OK for s_ in sts)
    for S, J, b, x, inf in zip(solvers, Js, bs, xs, infos):
        assert inf.rel_res_true <= 1e-8
        S.capacitance(J)
        xr, _ = S.pcg(b, 1e-8)
        assert torch.equal(x, xr)


@pytest.mark.parametrize("cap_gemm,mg_arith", [(0, 0), (1, 1)], ids=["mixed", "fp64_form"])
def test_dipole_grid_solution_error_vs_oracle(cap_gemm, mg_arith):
    """The precision configuration at small size: a 32^3 ERT step with a 4 x 4
    electrode grid and the dipole-dipole protocol (60 measurements). The default
    path (double-float cycle and passes, BF16-digit GEMM, FP64 outer residual) and
    the plain FP64 form are solved to a true residual of 1e-12 and compared with
    the oracle's FP64 PCG solution (residual 1e-12, near the FP64 floor of this
    system): relative error at most 1e-7 after refinement, the bound for
    mixed-precision paths."""
    pr = inputs.ert_problem(32, grid=(4, 4), m_rows=60, alpha=1e-3)
    n = (32, 32, 32)
    h = (pr.h,) * 3
    A = disc.regularization_operator("fv", n, h)
    dm = pr.logsigma - pr.m_ref
    b_ref = wb.gn_rhs(A, pr.alpha, dm, pr.J, pr.d)
    H = mg.build_hierarchy("fv", n, h)
    P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), pr.J, pr.alpha)
    x_ref, _, rel_ref = wb.pcg(lambda v: wb.apply_operator(A, pr.alpha, pr.J, v), P, b_ref, 1e-12, 400)
    assert rel_ref <= 1e-12
    S = _gpu("fv", n, h, pr.alpha, pr.J.shape[0], cap_gemm=cap_gemm, mg_arith=mg_arith)
    S.capacitance(_t(pr.J))
    x, info = S.pcg(_t(b_ref), 1e-12, 400)
    assert info.rel_res_true <= 1e-12
    xn = x.cpu().numpy()
    err = _rel(xn, x_ref)
    err_max = float(np.abs(xn - x_ref).max() / np.abs(x_ref).max())
    print(f"dipole grid 32^3 m=60 ({'mixed' if cap_gemm == 0 else 'fp64'}): iters {info.iters}, "
          f"restarts {info.restarts}, rel error vs oracle {err:.2e}, max entry error {err_max:.2e}")
    assert err <= 1e-7
    # entry by entry too: a localised error (e.g. at a tile edge) could hide under the norm
    assert err_max <= 1e-7


def test_ert_64cube_m496_converges_like_fp64_form():
    """A 64^3 ERT step with the full 496-measurement protocol, where C spans ~1e9:
    the default path (double-float cycle and passes, tensor-core C) reaches a true
    residual of 1e-8 within one PCG iteration of the plain FP64 form. Catches
    precision losses that only show when C is ill-conditioned."""
    pr = inputs.ert_problem(64, n_e_line=32, alpha=1e-3, device=DEV)
    n = (64, 64, 64)
    h = (1.0 / 64,) * 3
    m = pr.J.shape[0]
    dm = torch.as_tensor(pr.logsigma - pr.m_ref, device=DEV)
    d = torch.as_tensor(pr.d, device=DEV)
    its = []
    for opt in ({}, {"cap_gemm": 1, "mg_arith": 1}):
        S = _gpu("fv", n, h, pr.alpha, m, **opt)
        S.capacitance(pr.J)
        C, _ = S.factors()
        b = S.gn_rhs(dm, d)
        x, info = S.pcg(b, 1e-8, 60)
        assert info.rel_res_true <= 1e-8
        its.append(info.iters)
        del S
    assert float(torch.linalg.matrix_norm(C, 2)) > 1e8
    assert abs(its[0] - its[1]) <= 1, its


@pytest.mark.parametrize("case", [_q1((65, 65)), _fv((32, 32, 32))], ids=["q1_65", "fv32"])
def test_laplace_only_preconditioner(case):
    """The paper's variant without the capacitance matrix (precond = 1, P^-1 = alpha^-1
    L-hat^-1): the same solution as with the Laplace-Woodbury preconditioner, iteration
    counts as the oracle's PCG with that preconditioner, and the behaviour Sec. 3.2 and the
    timing experiments describe: its iterations grow with m and as alpha falls, while the
    Laplace-Woodbury counts stay flat."""
    d, n, h = case
    A = disc.regularization_operator(d, n, h)
    N = A.shape[0]
    H = mg.build_hierarchy(d, n, h)
    rng = np.random.default_rng(41)
    J_all = rng.standard_normal((32, N)) / np.sqrt(N)
    b = rng.standard_normal(N)
    its = {}
    for m in (4, 32):
        J = J_all[:m]
        for alpha in (1e-1, 1e-2):
            S0 = _gpu(d, n, h, alpha, m)
            S0.capacitance(_t(J))
            x0, i0 = S0.pcg(_t(b), 1e-11, 3000)
            S1 = _gpu(d, n, h, alpha, m, precond=1)
            S1.capacitance(_t(J))
            x1, i1 = S1.pcg(_t(b), 1e-11, 3000)
            assert i0.rel_res_true <= 1e-11 and i1.rel_res_true <= 1e-11
            assert _rel(x1.cpu().numpy(), x0.cpu().numpy()) <= 1e-8
            _, it_ref, _ = wb.pcg(lambda v: wb.apply_operator(A, alpha, J, v), lambda v: mg.vcycle(H, v) / alpha,
                                  b, 1e-11, 3000)
            # without the capacitance term the preconditioned system is far worse conditioned,
            # and at rtol 1e-11 the 48-bit cycle and the oracle's FP64 one part by a few
            # iterations (35 against 32 for m = 4, alpha = 1e-2 on the Q1 grid)
            assert abs(i1.iters - it_ref) <= max(3, it_ref // 10), (m, alpha, i1.iters, it_ref)
            its[(m, alpha)] = (i0.iters, i1.iters)
    assert its[(32, 1e-2)][1] > its[(4, 1e-2)][1] and its[(32, 1e-2)][1] > its[(32, 1e-1)][1], its
    wood = [v[0] for v in its.values()]
    assert max(wood) <= min(wood) + 3, its
    with pytest.raises(h1w.H1wError):
        S1.factors()


@pytest.mark.parametrize("case", [_q1((33, 33)), _q1((64, 64)), _fv((16, 12, 8)), _fv((16, 16, 16))],
                         ids=["q1_33", "q1_64", "fv16x12x8", "fv16"])
def test_direct_solve_matches_oracle(case):
    """h1w_solve_direct (dense alpha (K + M) + J^T J, blocked Cholesky, two triangular
    solves) against the oracle's dense solve, and against the PCG solution."""
    d, n, h = case
    A = disc.regularization_operator(d, n, h).toarray()
    N = A.shape[0]
    rng = np.random.default_rng(51)
    m, alpha = 24, 1e-2
    J = rng.standard_normal((m, N)) / np.sqrt(N)
    b = rng.standard_normal(N)
    x_ref = np.linalg.solve(alpha * A + J.T @ J, b)
    S = _gpu(d, n, h, alpha, m)
    S.capacitance(_t(J))
    x = S.solve_direct(_t(b))
    assert _rel(x.cpu().numpy(), x_ref) <= 1e-10
    xp, _ = S.pcg(_t(b), 1e-12, 300)
    assert _rel(xp.cpu().numpy(), x.cpu().numpy()) <= 1e-9
    # m = 0: the regularization operator alone; b and x may coincide
    S0 = _gpu(d, n, h, alpha, 1)
    S0.capacitance(None)
    bb = _t(b)
    S0.solve_direct(bb, bb)
    assert _rel(bb.cpu().numpy(), np.linalg.solve(alpha * A, b)) <= 1e-10


def test_direct_solve_refuses_large_grids():
    S = _gpu("fv", (32, 32, 32), (1 / 32,) * 3, 1e-2, 1)
    S.capacitance(None)
    with pytest.raises(h1w.H1wError) as ei:
        S.solve_direct(_t(np.ones(32 ** 3)))
    assert ei.value.status == h1w.H1W_EUNSUPPORTED
