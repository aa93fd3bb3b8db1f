"""The PCG loop driven from the device (a CUDA graph with a conditional while node,
pcg_mode = 0) and the multi-system batch as one graph (h1w_solve_batch_graph).

* The graph loop performs the same kernels in the same order as the host loop
  (pcg_mode = 1), so solutions and iteration counts are identical, bit for bit.
* The batch graph gives each system exactly the solution of solving it alone, and
  replaying the cached graph gives the same again.
* Two systems shaped like the 64-instance batch workload (2D Q1, side 1024 with m = 256;
  side 128 with m = 8) are checked against the oracle: the oracle's FP64 operator
  recomputes the true residual, and the solution is compared with the FP64 GPU form
  solved to 1e-12 (norm-wise and entry by entry), within the mixed-path bound 1e-7.
"""
import numpy as np
import pytest
import torch

from oracle import ccg
from oracle import discretization as disc
from paper_2209_02815_gb300 import h1w, inputs

pytestmark = pytest.mark.gpu
DEV = "cuda"


def _solver(d, n, alpha, m_max, stream=None, **opt):
    o = h1w.h1w_default_options()
    for k, v in opt.items():
        setattr(o, k, v)
    code = h1w.H1W_Q1_VERTEX if d == "q1" else h1w.H1W_FV_CELL
    h = tuple(1.0 / (v - 1) for v in n) if d == "q1" else tuple(1.0 / v for v in n)
    return h1w.Solver(code, n, h, alpha, m_max, device=DEV, opt=o, stream=stream)


CASES = [("q1", (64, 64), 16, {}), ("fv", (24, 24, 24), 30, {}), ("q1", (37, 41), 5, {}),
         ("fv", (16, 8, 12), 0, {}), ("fv", (20, 12, 28), 40, {"mg_arith": 1, "cap_gemm": 1}),
         ("fv", (24, 16, 16), 12, {"precond": 1})]


@pytest.mark.parametrize("case", CASES, ids=lambda c: f"{c[0]}{'x'.join(map(str, c[1]))}m{c[2]}{len(c[3])}")
def test_graph_loop_equals_host_loop(case):
    d, n, m, opt = case
    N = int(np.prod(n))
    rng = np.random.default_rng(71)
    J = torch.as_tensor(rng.standard_normal((m, N)) / np.sqrt(N), device=DEV) if m else None
    b = torch.as_tensor(rng.standard_normal(N), device=DEV)
    S = _solver(d, n, 1e-2, max(m, 1), **opt)
    S.capacitance(J)
    S.set_pcg_mode(1)
    xh, ih = S.pcg(b, 1e-10, 500)
    xh = xh.clone()
    S.set_pcg_mode(0)
    xg, ig = S.pcg(b, 1e-10, 500)
    xg2, ig2 = S.pcg(b, 1e-10, 500)   # the cached graph, replayed
    torch.cuda.synchronize()
    assert ig.iters == ih.iters == ig2.iters
    assert torch.equal(xg, xh) and torch.equal(xg2, xh)
    assert ig.rel_res_true <= 1e-10
    assert S.timings().launches_pcg > 0


def test_graph_cache_with_alternating_J_buffers():
    """Two device copies of J used in turn (the double-buffered host-copy pattern) and a third
    one: each system's graph is looked up by J's address among the two cached ones, and the
    solutions stay bit-identical to the host loop's. Different J contents in the buffers
    catch a graph replayed with the other buffer's address."""
    n, m = (24, 16, 20), 21
    N = int(np.prod(n))
    rng = np.random.default_rng(74)
    Ja = torch.as_tensor(rng.standard_normal((m, N)) / np.sqrt(N), device=DEV)
    Jb = torch.as_tensor(rng.standard_normal((m, N)) / np.sqrt(N), device=DEV)
    Jc = Ja.clone()
    b = torch.as_tensor(rng.standard_normal(N), device=DEV)
    S = _solver("fv", n, 1e-2, m)
    ref = {}
    S.set_pcg_mode(1)
    for name, J in (("a", Ja), ("b", Jb)):
        S.capacitance(J)
        x, info = S.pcg(b, 1e-10, 300)
        ref[name] = (x.clone(), info.iters)
    S.set_pcg_mode(0)
    for name, J in (("a", Ja), ("b", Jb), ("a", Ja), ("b", Jb), ("a", Jc), ("b", Jb), ("a", Ja)):
        S.capacitance(J)
        x, info = S.pcg(b, 1e-10, 300)
        torch.cuda.synchronize()
        assert info.iters == ref[name][1]
        assert torch.equal(x, ref[name][0]), f"J buffer {name}"
        assert info.rel_res_true <= 1e-10


def test_graph_loop_zero_rhs_and_maxit():
    S = _solver("fv", (16, 16, 16), 1e-2, 8)
    rng = np.random.default_rng(72)
    J = torch.as_tensor(rng.standard_normal((8, 4096)) / 64.0, device=DEV)
    S.capacitance(J)
    x, info = S.pcg(torch.zeros(4096, dtype=torch.float64, device=DEV), 1e-10, 50)
    assert info.iters == 0 and float(x.abs().max()) == 0.0
    b = torch.as_tensor(rng.standard_normal(4096), device=DEV)
    with pytest.raises(h1w.H1wError) as ei:
        S.pcg(b, 1e-14, 2)
    assert ei.value.status == h1w.H1W_ENOTCONV


def test_batch_graph_matches_individual_solves():
    cases = [("q1", (64, 64), 16), ("fv", (24, 24, 24), 30), ("q1", (37, 41), 5), ("fv", (16, 8, 12), 0),
             ("fv", (20, 12, 28), 9), ("q1", (130, 67), 40)]
    rng = np.random.default_rng(73)
    solvers, Js, bs, xs, refs = [], [], [], [], []
    for d, n, m in cases:
        N = int(np.prod(n))
        J = torch.as_tensor(rng.standard_normal((m, N)) / np.sqrt(N), device=DEV) if m else None
        b = torch.as_tensor(rng.standard_normal(N), device=DEV)
        solvers.append(_solver(d, n, 1e-2, max(m, 1), stream=torch.cuda.Stream()))
        Js.append(J)
        bs.append(b)
        xs.append(torch.empty_like(b))
        R = _solver(d, n, 1e-2, max(m, 1))
        R.capacitance(J)
        xr, _ = R.pcg(b, 1e-10)
        refs.append(xr)
    torch.cuda.synchronize()
    for rep in range(2):   # capture, then replay
        for x in xs:
            x.fill_(float("nan"))
        infos, sts = h1w.solve_batch(solvers, Js, bs, xs, 1e-10, graph=True)
        assert all(s == h1w.H1W_OK for s in sts)
        for x, xr, inf in zip(xs, refs, infos):
            assert torch.equal(x, xr)
            assert inf.rel_res_true <= 1e-10


@pytest.mark.parametrize("side,m,alpha", [(1024, 256, 1e-3), (128, 8, 0.1)])
def test_batch_shaped_instances_against_oracle(side, m, alpha):
    """C3-shaped systems through the batch graph: oracle residual and entry-wise error."""
    n = (side, side)
    N = side * side
    dsc = {"n": side, "m": m, "alpha": alpha, "seed_j": 7 + side, "seed_b": 8 + side}
    J, b = inputs.batch_instance_data(dsc, device=DEV)
    S = _solver("q1", n, alpha, m, stream=torch.cuda.Stream())
    x = torch.empty_like(b)
    infos, sts = h1w.solve_batch([S], [J], [b], [x], 1e-8, graph=True)
    assert sts[0] == h1w.H1W_OK
    # the oracle's FP64 operator (C, CSR K + M, J on the host) recomputes the residual
    A = disc.regularization_operator("q1", n, tuple(1.0 / (v - 1) for v in n))
    Jn, bn, xn = J.cpu().numpy(), b.cpu().numpy(), x.cpu().numpy()
    op = ccg.CsrOperator(A, alpha, Jn)
    res = np.linalg.norm(bn - op.apply(xn)) / np.linalg.norm(bn)
    assert res <= 1e-8 * 1.01, res
    # against the plain FP64 form solved to 1e-12
    F = _solver("q1", n, alpha, m, mg_arith=1, cap_gemm=1)
    F.capacitance(J)
    xf, inf = F.pcg(b, 1e-12, 1000)
    xf = xf.cpu().numpy()
    assert np.linalg.norm(xn - xf) <= 1e-7 * np.linalg.norm(xf)
    assert np.abs(xn - xf).max() <= 1e-7 * np.abs(xf).max()


def test_autotune_picks_a_block_and_caches_it():
    """h1w_autotune times line H's batched cycle for each candidate rhs_block and returns
    one of them; the second call comes from the cache; the tuned context solves to the
    same bits as the default one (each right-hand side's cycle does not depend on the batch)."""
    import time
    n, m, alpha = (96, 80), 40, 1e-2
    h = tuple(1.0 / (v - 1) for v in n)
    g = h1w.make_grid(h1w.H1W_Q1_VERTEX, n, h, alpha)
    opt, ms = h1w.h1w_autotune(g, m, device=DEV)
    assert opt.rhs_block in (8, 16, 32, 40) and ms > 0.0
    t0 = time.perf_counter()
    opt2, ms2 = h1w.h1w_autotune(g, m, device=DEV)
    assert time.perf_counter() - t0 < 0.5
    assert opt2.rhs_block == opt.rhs_block and ms2 == ms
    N = n[0] * n[1]
    rng = np.random.default_rng(74)
    J = torch.as_tensor(rng.standard_normal((m, N)) / np.sqrt(N), device=DEV)
    b = torch.as_tensor(rng.standard_normal(N), device=DEV)
    T = h1w.Solver(h1w.H1W_Q1_VERTEX, n, h, alpha, m, device=DEV, opt=opt)
    D = _solver("q1", n, alpha, m)
    T.capacitance(J)
    D.capacitance(J)
    xt, _ = T.pcg(b, 1e-10)
    xd, _ = D.pcg(b, 1e-10)
    assert torch.equal(xt, xd)
