"""Low-rank capacitance (the paper's outlook, Sec. 5: data-sparse or randomized low-rank
approximation of the capacitance equation), evaluated on the oracle before any GPU path.

The preconditioner keeps the Woodbury form but projects the data term on the top-k
eigenvectors Q of G = J L-hat^-1 J^T / alpha: P_k = alpha L-hat + J^T Q Q^T J, i.e. the
Woodbury apply with J_k = Q^T J (k rows), H_k = L-hat^-1 J_k^T and C_k = I + alpha^-1 J_k H_k.
Exact eigenvectors are the best case for any randomized sketch of the same rank. The
directions left out stay in the operator and CG must resolve them, so the iteration count
depends on how many eigenvalues of G / alpha exceed O(1): on ERT sensitivities they spread
over ten decades, and below that count the iterations rise steeply.

Run as a script for the 32^3 table (m = 496, the 32-electrode pair protocol):
    python -m tests.test_low_rank_capacitance 32 32
"""
import sys

import numpy as np
import pytest

from oracle import discretization as disc
from oracle import multigrid as mg
from oracle import woodbury as wb
from paper_2209_02815_gb300 import inputs


def low_rank_table(n, n_e, ks_frac, alpha=1e-3, maxit=400):
    pr = inputs.ert_problem(n, n_e_line=n_e, alpha=alpha)
    J = np.asarray(pr.J)
    m = J.shape[0]
    h = (1.0 / n,) * 3
    H = mg.build_hierarchy("fv", (n, n, n), h)
    A = disc.regularization_operator("fv", (n, n, n), h)
    Hh = wb.hhat(H, J)
    b = wb.gn_rhs(A, alpha, pr.logsigma - pr.m_ref, J, pr.d)
    G = J @ Hh
    ev, V = np.linalg.eigh(0.5 * (G + G.T) / alpha)
    ev, V = ev[::-1], V[:, ::-1]
    counts = {t: int((ev > t).sum()) for t in (1e6, 1e3, 10.0, 1.0, 0.1)}
    rows = []
    for f in ks_frac:
        k = int(round(f * m))
        Q = V[:, :k]
        P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), Q.T @ J, alpha, Hh=Hh @ Q)
        _, it, rel = wb.pcg(lambda p: wb.apply_operator(A, alpha, J, p), P, b, 1e-8, maxit, max_restarts=0)
        rows.append((k, it, rel))
    return m, float(ev[0]), counts, rows


def test_low_rank_capacitance_needs_the_large_eigenvalues():
    m, top, counts, rows = low_rank_table(24, 16, (0.5, 0.75, 1.0), maxit=120)
    assert m == 120 and top > 1e9
    full_it = rows[-1][1]
    (k2, it2, _), (k3, it3, rel3) = rows[0], rows[1]
    assert rows[-1][2] <= 1e-8 and full_it <= 12
    # rank 3m/4 covers every eigenvalue above 1 (81 of 120) and keeps the count
    assert counts[1.0] <= k3 and rel3 <= 1e-8 and it3 <= full_it + 1
    # rank m/2 leaves about 20 eigenvalues above 10 to CG: many more iterations
    assert counts[10.0] > k2 and it2 >= 3 * full_it


if __name__ == "__main__":
    n, ne = int(sys.argv[1]), int(sys.argv[2])
    m, top, counts, rows = low_rank_table(n, ne, (0.0, 1 / 16, 1 / 8, 1 / 4, 1 / 2, 3 / 4, 1.0))
    print(f"{n}^3, m = {m}: largest eigenvalue of G/alpha {top:.3g}; counts above 1e6, 1e3, 10, 1, 0.1: "
          + ", ".join(str(counts[t]) for t in (1e6, 1e3, 10.0, 1.0, 0.1)))
    for k, it, rel in rows:
        print(f"k = {k:4d}: {it:4d} PCG iterations, true relative residual {rel:.1e}")
