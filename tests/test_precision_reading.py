"""Why the inner arithmetic is ~48 bits and not FP32.

On ERT sensitivities the capacitance matrix C = I + J H-hat / alpha has an
eigenvalue spread of ~1e10. The Woodbury preconditioner then subtracts two
nearly equal operators in the directions where J is large, so a relative
inconsistency delta between H-hat (and the C built from it) and the V-cycle
that P^-1 applies becomes an error of size delta * ||C|| in P^-1. This test
takes the oracle's V-cycle, rounds H-hat to a given number of significand
bits, rebuilds C consistently from the rounded H-hat and runs the oracle PCG:
48 bits (the double-float cycle and passes) keep the FP64 iteration count,
while FP32 storage (24 bits) no longer converges.
"""
import numpy as np
import pytest

from oracle import discretization as disc
from oracle import multigrid as mg
from oracle import woodbury as wb
from paper_2209_02815_gb300 import inputs


def _round_bits(X, bits):
    f, e = np.frexp(X)
    s = 2.0 ** bits
    return np.ldexp(np.round(f * s) / s, e)


@pytest.fixture(scope="module")
def ert24():
    n, alpha = 24, 1e-3
    pr = inputs.ert_problem(n, n_e_line=16, alpha=alpha)
    J = np.asarray(pr.J)
    h = (1.0 / n,) * 3
    H = mg.build_hierarchy("fv", (n, n, n), h)
    A = disc.regularization_operator("fv", (n, n, n), h)
    Hh = wb.hhat(H, J)
    b = wb.gn_rhs(A, alpha, pr.logsigma - pr.m_ref, J, pr.d)
    return H, A, J, alpha, Hh, b


def _iters(ert, Hx, maxit):
    H, A, J, alpha, _, b = ert
    P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), J, alpha, Hh=Hx)
    _, it, rel = wb.pcg(lambda p: wb.apply_operator(A, alpha, J, p), P, b, 1e-8, maxit, max_restarts=0)
    return it, rel


def test_capacitance_spread_is_large(ert24):
    _, _, J, alpha, Hh, _ = ert24
    ev = np.linalg.eigvalsh(wb.capacitance(J, Hh, alpha))
    assert ev[0] >= 1.0 - 1e-6 and ev[-1] > 1e9


def test_48_bits_keep_the_fp64_count_fp32_does_not_converge(ert24):
    Hh = ert24[4]
    it64, rel64 = _iters(ert24, Hh, 60)
    it48, rel48 = _iters(ert24, _round_bits(Hh, 48), 60)
    it24, rel24 = _iters(ert24, Hh.astype(np.float32).astype(np.float64), 60)
    assert rel64 <= 1e-8 and it64 <= 12
    assert rel48 <= 1e-8 and abs(it48 - it64) <= 1
    assert rel24 > 1e-6  # 60 iterations do not reach the tolerance
