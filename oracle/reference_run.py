"""Full oracle solve of the 128^3 ERT Gauss-Newton step (test infrastructure only).

Runs the oracle's Woodbury-preconditioned PCG (the same method in plain CPU
code: scipy-sparse V-cycles, numpy products) on the 128^3 cell grid with the
32-electrode pole-dipole protocol (m = 496, alpha = 1e-3) to the Euclidean
relative residual 1e-8, and writes the iteration count, the true relative
residual and per-phase wall times to ``reference_run.json`` beside this file.

bench.py reads the iteration count to extrapolate its bounded CPU samples to
one full solve. Usage: python -m oracle.reference_run [n] [n_e]
"""
from __future__ import annotations

import json
import os
import platform
import sys
import time

import numpy as np

from . import ccg
from . import discretization as disc
from . import multigrid as mg
from . import woodbury as wb

HERE = os.path.dirname(os.path.abspath(__file__))


def main(n: int = 128, n_e: int = 32, rtol: float = 1e-8) -> dict:
    from paper_2209_02815_gb300 import inputs

    t0 = time.perf_counter()
    pr = inputs.ert_problem(n, n_e_line=n_e, alpha=1e-3, device="cpu")
    J = np.ascontiguousarray(pr.J)
    t_inputs = time.perf_counter() - t0
    h = (1.0 / n,) * 3
    A = disc.regularization_operator("fv", (n, n, n), h)
    H = mg.build_hierarchy("fv", (n, n, n), h)
    dm = pr.logsigma - pr.m_ref
    b = wb.gn_rhs(A, pr.alpha, dm, J, pr.d)
    t1 = time.perf_counter()
    Hh = wb.hhat(H, J)
    t_H = time.perf_counter() - t1
    t1 = time.perf_counter()
    P = wb.WoodburyPreconditioner(lambda v: mg.vcycle(H, v), J, pr.alpha, Hh=Hh)
    t_C_chol = time.perf_counter() - t1
    op = ccg.CsrOperator(A, pr.alpha, J)
    t1 = time.perf_counter()
    x, it, rel = wb.pcg(op.apply, P, b, rtol, 1000)
    t_pcg = time.perf_counter() - t1
    out = {
        "workload": f"3D FV {n}^3, m={J.shape[0]}, alpha={pr.alpha}, rtol={rtol}",
        "iterations": it,
        "rel_res_true": rel,
        "t_inputs_s": t_inputs,
        "t_H_s": t_H,
        "t_C_chol_s": t_C_chol,
        "t_pcg_s": t_pcg,
        "threads": ccg.threads(),
        "machine": platform.machine(),
        "processor": platform.processor(),
        "nproc": os.cpu_count(),
        "x_norm": float(np.linalg.norm(x)),
    }
    return out


if __name__ == "__main__":
    n = int(sys.argv[1]) if len(sys.argv) > 1 else 128
    ne = int(sys.argv[2]) if len(sys.argv) > 2 else 32
    res = main(n, ne)
    path = os.path.join(HERE, "reference_run.json" if n == 128 else f"reference_run_{n}.json")
    with open(path, "w") as f:
        json.dump(res, f, indent=1)
    print(json.dumps(res, indent=1))
