#!/usr/bin/env python
"""Benchmark: Gauss-Newton linear solves per second on one GB300.

One step = one full GN linear solve of (alpha (K + M) + J^T J) x = b on the
128^3 cell-centred FV grid with m = 496 measurements (32 line electrodes,
pole-dipole pairs, analytic half-space sensitivities, alpha = 1e-3, FP64):
lines H, C and chol of the Laplace-Woodbury algorithm (h1w_capacitance)
followed by PCG from x0 = 0 to ||r||_2 <= 1e-8 ||b||_2 with the FP64 true
residual check (h1w_pcg). This matches the paper's t_norm, which includes
lines H, C and chol.

Prints one JSON line (rank 0). With torchrun (N > 1) every rank solves its
own independent GN step (replicas; no collective on the data path) and the
value is the whole-job rate.

--impl reference times the FP64 CPU oracle (the same method written plainly
with scipy/numpy) on the host cores, on bounded samples extrapolated to one
solve with the oracle's own iteration count.
"""
from __future__ import annotations

import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

N_SIDE = 128
N_E = 32
ALPHA = 1e-3
RTOL = 1e-8
ACC_RTOL = 1e-11   # the FP64 form's tolerance for the accuracy comparison (near its attainable floor)
MAXIT = 1000
METRIC = "GN linear solves/s at rel-res 1e-8"
# FP32 instructions per fine cell of the fused double-float legs (isotropic 7-point operator;
# double-float product 7, product with a float 6, cascaded-sum term 8 (the first term of a sum
# is free), sum result 3):
# down 7 (g) + 68 (two Chebyshev steps, T folded into gamma) + 76 (residual)
#   + 43 (separable restriction: x pass 51 per half cell, y pass 51 per quarter cell, z taps 20
#   per quarter cell);
# up 41 (separable prolongation: x pass 19 per quarter cell, y pass 19 per half cell, z taps and
#   the add 27) + 83 (r0, d0) + 76 (final update, T folded into kappa)
FP32_OPS_DOWN = 194
FP32_OPS_UP = 200
# Algorithmic HBM bytes per fine cell and right-hand side of the finest-level fused legs
# (double-float vectors, 8 bytes per entry; the coarse level has 1/8 of the cells):
#   down leg: b in, x out, the restricted residual out      = 8 + 8 + 1 = 17
#   up leg:   x in, b in, the coarse correction in, y out  = 8 + 8 + 1 + 8 = 25
HBM_BYTES_DOWN = 17.0
HBM_BYTES_UP = 25.0
# ncu DRAM read + write bytes per fine cell and right-hand side of the finest up leg, from one
# capture of the 64^3 case with 128 right-hand sides (the kernel build these figures belong to
# is named by NCU_TRAFFIC_BUILD; traffic is reported only while it matches FUSED_BUILD)
NCU_BYTES_PER_CELL_RHS = {"k_post_fused": (599.148544e6 + 242.237184e6) / (262144 * 128),
                          "k_pre_fused": (285.612544e6 + 255.360512e6) / (262144 * 128)}
NCU_TRAFFIC_BUILD = "df-legs-v3"
FUSED_BUILD = "df-legs-v3"
DTYPE_MIXED = "mixed(df48+bf16-digit, fp64 outer)"


def workload(n, m, grid=None, alpha=ALPHA):
    proto = "pole-dipole" if grid is None else "dipole-dipole %dx%d grid" % grid
    return ("3D ERT GN step, %d^3 cell-centred FV, m=%d %s, alpha=%g, true FP64 relative residual "
            "<= 1e-8" % (n, m, proto, alpha))


def electrode_grid(args):
    if not args.grid:
        return None
    ex, ey = (int(v) for v in args.grid.lower().split("x"))
    return (ex, ey)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--n", type=int, default=N_SIDE)
    ap.add_argument("--alpha", type=float, default=ALPHA, help="regularization weight of the GN step")
    ap.add_argument("--ne", type=int, default=N_E)
    ap.add_argument("--grid", default=None,
                    help="electrode grid EXxEY on the top face with the dipole-dipole protocol (e.g. 8x8)")
    ap.add_argument("--m-rows", type=int, default=None, help="truncate the protocol to this many measurements")
    ap.add_argument("--ert", action="store_true",
                    help="time the ERT model evaluation (h1w_forward + h1w_adjoint J rows) instead")
    ap.add_argument("--precond", default="woodbury", choices=["woodbury", "laplace"],
                    help="laplace: the paper's variant without the capacitance matrix (comparison only)")
    ap.add_argument("--maxit", type=int, default=MAXIT)
    ap.add_argument("--gn-steps", type=int, default=0,
                    help="time this many Gauss-Newton steps of the ERT inversion workload instead")
    ap.add_argument("--batch", type=int, default=0,
                    help="instead of the ERT step: a batch of this many independent 2D Q1 systems "
                         "(sides 128..1024, m 8..256, alpha log-uniform 1e-4..1e-1) solved by h1w_solve_batch")
    ap.add_argument("--batch-mode", default="graph", choices=["graph", "threads"],
                    help="--batch: one CUDA graph for all systems (h1w_solve_batch_graph) or a pool of host "
                         "threads (h1w_solve_batch)")
    ap.add_argument("--no-autotune", action="store_true", help="--batch: default rhs_block for every instance")
    ap.add_argument("--accuracy", action="store_true",
                    help="after timing: the solution's error against the plain FP64 GPU form solved to 1e-12 "
                         "(frees the mixed workspace first; for the largest sizes)")
    ap.add_argument("--e2e-steps", type=int, default=10)
    ap.add_argument("--no-oracle-check", action="store_true",
                    help="skip the oracle's FP64 residual of the timed solution (rank 0)")
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--rhs-block", type=int, default=0, help="right-hand sides per batched V-cycle (0: default)")
    ap.add_argument("--cheb-degree", type=int, default=0, help="Chebyshev smoother degree (0: default 2)")
    ap.add_argument("--cheb-ratio", type=float, default=0.0,
                    help="Chebyshev interval [lambda / ratio, lambda] (0: the discretization default, 10 FV / 6 Q1)")
    ap.add_argument("--pcg-mode", type=int, default=0,
                    help="0: PCG loop driven from the device (CUDA graph, default); 1: host loop")
    ap.add_argument("--arith", default="mixed", choices=["mixed", "fp64"],
                    help="timed path: mixed (double-float cycle and passes, tensor-core C; default) or the "
                         "plain FP64 form (FP64 cycle and passes, CUDA-core C)")
    ap.add_argument("--fp64-form-steps", type=int, default=5,
                    help="steps of the plain FP64 GPU form (FP64 V-cycle, CUDA-core GEMM) timed for comparison")
    ap.add_argument("--cpu-sample-s", type=float, default=20.0)
    ap.add_argument("--cpu-full-solve", action="store_true",
                    help="cpu_baseline: time one complete oracle solve of the workload on the host cores "
                         "(minutes at 128^3) instead of the bounded, extrapolated sample")
    return ap.parse_args()


# ----------------------------------------------------------------------------
# clocks sampled during the timed region
# ----------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.f = tempfile.NamedTemporaryFile("w+", suffix=".csv", delete=False)
        self.p = None

    def start(self):
        try:
            self.p = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.FIELDS}",
                                       "--format=csv,noheader,nounits", "-lms", "200"],
                                      stdout=self.f, stderr=subprocess.DEVNULL)
        except FileNotFoundError:
            self.p = None

    def stop(self) -> dict:
        if self.p is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.p.terminate()
        try:
            self.p.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.p.kill()
        self.f.flush()
        rows = []
        with open(self.f.name) as fh:
            for line in fh:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.f.name)
        if not rows:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["no samples"]}
        sm = [float(r[1]) for r in rows if r[1].replace(".", "").isdigit()]
        mx = [float(r[2]) for r in rows if r[2].replace(".", "").isdigit()]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for nm, v in zip(names, r[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(mx) if mx else None,
                "power_w_max": max(float(r[3]) for r in rows if r[3].replace(".", "").isdigit())
                if any(r[3].replace(".", "").isdigit() for r in rows) else None,
                "samples": len(rows), "reasons": sorted(reasons)}


# ----------------------------------------------------------------------------
# distributed plumbing (replicas)
# ----------------------------------------------------------------------------

def dist_init(args):
    import torch
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        if torch.cuda.is_available():
            torch.cuda.set_device(local)
        dist.init_process_group(backend=backend)
    elif torch.cuda.is_available():
        torch.cuda.set_device(local)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def allmax(world, v: float) -> float:
    if world == 1:
        return v
    import torch
    import torch.distributed as dist
    t = torch.tensor([v], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ----------------------------------------------------------------------------
# CPU oracle timing on bounded samples (cpu_baseline and --impl reference)
# ----------------------------------------------------------------------------

def oracle_sample(J_host, logsigma, m_ref, d, n, budget_s: float, iters_fallback=None, default_case=True) -> dict:
    """Times the oracle's phases on bounded samples and extrapolates to one solve:
    t = m * t_vcycle + t_gemm(m x N x m) + iters * t_iteration. The iteration count
    comes from the oracle's own full solve of this workload (oracle/reference_run.json)."""
    import numpy as np
    from oracle import ccg
    from oracle import discretization as disc
    from oracle import multigrid as mg
    from oracle import woodbury as wb

    h = (1.0 / n,) * 3
    m = J_host.shape[0]
    A = disc.regularization_operator("fv", (n, n, n), h)
    H = mg.build_hierarchy("fv", (n, n, n), h)
    op = ccg.CsrOperator(A, ALPHA, J_host)  # the operator's cost does not depend on alpha
    rng = np.random.default_rng(0)
    v = rng.standard_normal(A.shape[0])
    t0 = time.perf_counter()
    nv = 0
    while nv < 2 or (time.perf_counter() - t0 < 0.25 * budget_s and nv < 8):
        mg.vcycle(H, v)
        nv += 1
    t_v = (time.perf_counter() - t0) / nv
    t0 = time.perf_counter()
    na = 0
    while na < 1 or (time.perf_counter() - t0 < 0.25 * budget_s and na < 4):
        op.apply(v)
        na += 1
    t_apply = (time.perf_counter() - t0) / na          # J p, J^T w and the stencil
    t0 = time.perf_counter()
    s = J_host @ v
    t_jpass = time.perf_counter() - t0                 # one pass over an m x N matrix
    # GEMM sample k x N x k (line C is m x N x m); a 256-row block runs at close to the
    # full product's BLAS efficiency (a 64-row one ran 11x slower per flop on the box)
    k = min(m, 256)
    t0 = time.perf_counter()
    _ = J_host[:k] @ J_host[:k].T
    t_g = time.perf_counter() - t0
    t_gemm = t_g * (m / k) ** 2
    path = os.path.join(ROOT, "oracle", "reference_run.json")
    iters = None
    iters_from = "oracle"
    if os.path.exists(path) and n == N_SIDE and default_case:
        with open(path) as f:
            iters = json.load(f).get("iterations")
    if iters is None and iters_fallback is not None:
        iters, iters_from = int(iters_fallback), "gpu"
    # one PCG iteration: operator apply + V-cycle + H^T r + H v (two more m x N passes)
    t_it = t_apply + t_v + 2 * t_jpass
    t_solve = m * t_v + t_gemm + (iters or 0) * t_it
    return {"t_vcycle_s": t_v, "t_apply_s": t_apply, "t_jpass_s": t_jpass, "t_gemm_s": t_gemm,
            "t_iteration_s": t_it, "iterations": iters, "iterations_from": iters_from, "t_solve_s": t_solve,
            "threads": ccg.threads(), "vcycles_timed": nv, "applies_timed": na}


# ----------------------------------------------------------------------------
# batch of independent 2D systems (multi-instance workload)
# ----------------------------------------------------------------------------

def run_batch(args):
    import torch
    from paper_2209_02815_gb300 import h1w, inputs

    world, rank, local = dist_init(args)
    dev = torch.device("cuda", local)
    descs = inputs.batch_instances(args.batch)
    solvers, Js, bs, xs = [], [], [], []
    tuned = {}
    t_tune = time.perf_counter()
    for dsc in descs:
        n = dsc["n"]
        J, b = inputs.batch_instance_data(dsc, device=dev)
        g = h1w.make_grid(h1w.H1W_Q1_VERTEX, (n, n), (1.0 / (n - 1),) * 2, dsc["alpha"])
        opt = None
        if not args.no_autotune:
            # rhs_block of line H's batched V-cycle per instance shape (cached per side and m)
            opt, ms_rhs = h1w.h1w_autotune(g, dsc["m"], device=dev)
            tuned["%dx%d m=%d" % (n, n, dsc["m"])] = {"rhs_block": int(opt.rhs_block),
                                                       "vcycle_ms_per_rhs": ms_rhs}
        solvers.append(h1w.Solver(h1w.H1W_Q1_VERTEX, (n, n), (1.0 / (n - 1),) * 2, dsc["alpha"], dsc["m"],
                                  device=dev, stream=torch.cuda.Stream(dev), opt=opt))
        Js.append(J)
        bs.append(b)
        xs.append(torch.empty_like(b))
    torch.cuda.synchronize()
    t_tune = time.perf_counter() - t_tune
    graph = args.batch_mode == "graph"
    for _ in range(args.warmup):
        infos, _ = h1w.solve_batch(solvers, Js, bs, xs, RTOL, MAXIT, graph=graph)
    barrier(world)
    torch.cuda.synchronize()
    clk = ClockSampler(local)
    clk.start()
    t0 = time.perf_counter()
    launches = 0
    for _ in range(args.steps):
        infos, _ = h1w.solve_batch(solvers, Js, bs, xs, RTOL, MAXIT, graph=graph)
        launches += sum(int(S_.timings().launches_capacitance + S_.timings().launches_pcg) for S_ in solvers)
    torch.cuda.synchronize()
    dt = allmax(world, (time.perf_counter() - t0) * 1e3)
    clocks = clk.stop()
    value = world * len(descs) * args.steps / (dt / 1e3)
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": dt / args.steps, "higher_is_better": True, "scaling": "weak",
           "vs_baseline": None, "dtype": DTYPE_MIXED, "data": "synthetic",
           "config": {"workload": "%d independent 2D Q1 systems per step (sides 128-1024, m 8-256, "
                                  "alpha log-uniform 1e-4..1e-1), %s" %
                                  (len(descs), "h1w_solve_batch_graph (one CUDA graph)" if graph else
                                   "h1w_solve_batch (host thread pool)"),
                      "dof_total": int(sum(d["n"] ** 2 for d in descs)),
                      "J_entries": int(sum(d["n"] ** 2 * d["m"] for d in descs)),
                      "parallelism": "replicas" if world > 1 else "single GPU"},
           "pcg_iters": [int(i.iters) for i in infos], "max_rel_res_true": max(float(i.rel_res_true) for i in infos),
           "clocks": clocks, "timing": "host wall clock around whole batches (each call synchronizes)",
           "gpu_launches": launches, "autotune": tuned or None,
           "phases_ms_sum_over_systems": ({k_: round(sum(float(getattr(S_.timings(), k_)) for S_ in solvers), 2)
                                           for k_ in ("t_H_ms", "t_C_ms", "t_chol_ms", "t_pcg_ms")}
                                          if not graph else None),
           "setup_and_autotune_s": t_tune, "impl": "ours"}
    if rank == 0:
        print(json.dumps(out))


# ----------------------------------------------------------------------------
# ERT model evaluation: pole fields, measurements and all rows of J (Sec. 4.1)
# ----------------------------------------------------------------------------

ERT_RTOL = 1e-10
# regularization weight of the inversion workload: on the 16^3 oracle inversion of the same
# design, full Gauss-Newton steps diverge for alpha <= 0.1 and reach the noise level in 3-4
# steps for alpha = 10..100 (100: smallest model error)
GN_ALPHA = 100.0
# ncu DRAM read + write bytes per J entry of k_jacobian<rows> (64^3, 32 electrodes, m = 496):
# (1102.789 + 69.838) MB / (496 * 262144)
NCU_BYTES_PER_J_ENTRY = (1102.789e6 + 69.83808e6) / (496 * 262144)


def ert_oracle_sample(n_side: int, ne: int, budget_s: float) -> dict:
    """The oracle's evaluation (sparse LU pole fields, g, J rows) on an n_side^3 grid
    with the same survey design, timed on the host cores."""
    import numpy as np
    from oracle import ert as oert
    from paper_2209_02815_gb300 import inputs
    cells, abmn, k, _ = inputs.ert_survey(n_side, n_e_line=ne)
    field, _ = inputs.gaussian_random_field((n_side,) * 3, (1.0 / n_side,) * 3, 0.1, math.log(0.01), 1.0, 0)
    ls = field.reshape(-1)
    h = (1.0 / n_side,) * 3
    t0 = time.perf_counter()
    g, U = oert.forward((n_side,) * 3, h, ls, cells, abmn, k, inputs.ERT_DIRICHLET_ALL_BUT_TOP)
    t1 = time.perf_counter()
    rows = max(1, min(len(abmn), int(len(abmn) * budget_s / max(1e-3, 4 * (t1 - t0)))))
    oert.jacobian((n_side,) * 3, h, ls, U, abmn[:rows], k[:rows], inputs.ERT_DIRICHLET_ALL_BUT_TOP)
    t2 = time.perf_counter()
    return {"fields_s": t1 - t0, "rows_timed": rows, "rows_s": t2 - t1,
            "eval_s": (t1 - t0) + (t2 - t1) * len(abmn) / rows, "m": int(len(abmn)), "n": n_side}


def run_ert(args):
    import numpy as np
    import torch
    from paper_2209_02815_gb300 import h1w, inputs

    world, rank, local = dist_init(args)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    n = args.n
    N = n ** 3
    grid = electrode_grid(args)
    cells, abmn, k, _ = inputs.ert_survey(n, n_e_line=args.ne, grid=grid, m_rows=args.m_rows)
    sv = h1w.Survey(cells, abmn, k, inputs.ERT_DIRICHLET_ALL_BUT_TOP)
    field, _ = inputs.gaussian_random_field((n,) * 3, (1.0 / n,) * 3, 0.1, math.log(0.01), 1.0, inputs.SEED_FIELD)
    with torch.cuda.stream(stream):
        o_ert = None
        if args.cheb_ratio > 0:
            o_ert = h1w.h1w_default_options()
            o_ert.cheb_ratio = args.cheb_ratio
        S = h1w.Solver(h1w.H1W_FV_CELL, (n, n, n), (1.0 / n,) * 3, ALPHA, 1, device=dev, opt=o_ert, stream=stream)
        ls = torch.as_tensor(field.reshape(-1), device=dev)
        ws = S.ert_workspace(sv)
        U = torch.empty((sv.n_e, N), dtype=torch.float64, device=dev)
        J = torch.empty((sv.m, N), dtype=torch.float64, device=dev)
        g = torch.empty(sv.m, dtype=torch.float64, device=dev)

        def step():
            info = h1w.h1w_forward(S.ctx, sv, ls, U, g, ws, ERT_RTOL, 200, N)
            h1w.h1w_adjoint(S.ctx, sv, ls, U, None, None, J, ws, N)
            return info

        for _ in range(args.warmup):
            info = step()
        torch.cuda.synchronize()
        barrier(world)
        clk = ClockSampler(local)
        clk.start()
        ev = [torch.cuda.Event(enable_timing=True) for _ in range(2 * args.steps + 1)]
        ev[0].record(stream)
        iters = []
        for i in range(args.steps):
            info = h1w.h1w_forward(S.ctx, sv, ls, U, g, ws, ERT_RTOL, 200, N)
            ev[2 * i + 1].record(stream)
            h1w.h1w_adjoint(S.ctx, sv, ls, U, None, None, J, ws, N)
            ev[2 * i + 2].record(stream)
            iters.append(int(info.iters))
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = allmax(world, ev[0].elapsed_time(ev[-1]))
        fwd = [ev[2 * i].elapsed_time(ev[2 * i + 1]) for i in range(args.steps)]
        jac = [ev[2 * i + 1].elapsed_time(ev[2 * i + 2]) for i in range(args.steps)]

        # the data term from the fields (no J stored: J^T r of h1w_adjoint, J p of h1w_ert_jvp)
        # against the same products with the stored J (library FP64 GEMV), one pass each
        r = torch.ones(sv.m, dtype=torch.float64, device=dev)
        pv = torch.ones(N, dtype=torch.float64, device=dev)
        fe = [torch.cuda.Event(enable_timing=True) for _ in range(5)]
        fe[0].record(stream)
        JTr = S.adjoint(sv, ls, U, r=r, ws=ws)[0]
        fe[1].record(stream)
        S.jvp(sv, ls, U, pv, ws=ws)
        fe[2].record(stream)
        torch.mv(J.t(), r)
        fe[3].record(stream)
        torch.mv(J, pv)
        fe[4].record(stream)
        torch.cuda.synchronize()
        fields_ms = {"JTr_from_fields": fe[0].elapsed_time(fe[1]), "Jp_from_fields": fe[1].elapsed_time(fe[2]),
                     "JTr_stored_J_gemv": fe[2].elapsed_time(fe[3]), "Jp_stored_J_gemv": fe[3].elapsed_time(fe[4])}
        del JTr

        # end to end through the public API: logsigma from pinned host memory, g back to it
        ls_host = torch.empty(N, dtype=torch.float64, pin_memory=True)
        ls_host.copy_(ls)
        g_host = torch.empty(sv.m, dtype=torch.float64, pin_memory=True)
        ls_dev = torch.empty_like(ls)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(args.e2e_steps):
            ls_dev.copy_(ls_host, non_blocking=True)
            h1w.h1w_forward(S.ctx, sv, ls_dev, U, g, ws, ERT_RTOL, 200, N)
            h1w.h1w_adjoint(S.ctx, sv, ls_dev, U, None, None, J, ws, N)
            g_host.copy_(g, non_blocking=True)
        e1.record(stream)
        torch.cuda.synchronize()
        e2e_ms = allmax(world, e0.elapsed_time(e1)) if args.e2e_steps else None

    m = sv.m
    new_src = np.concatenate([[True], np.any(np.diff(abmn[:, :2], axis=0) != 0, axis=1)])
    src_b = int(np.sum(new_src & (abmn[:, 1] >= 0)))
    src_a = int(np.sum(new_src)) - src_b
    n_full = int(np.sum((abmn[:, 2] >= 0) & (abmn[:, 3] >= 0)))
    # FP32 instructions of the double-float J-row kernel (FMA counted once): per row and cell
    # 6 faces x (difference 20 + product 7 + sum term 8) + 3 to renormalize (6 x (7 + 8) + 3
    # when one receiver electrode is at infinity); per new source and cell 6 x (20 + 7), or
    # 6 x 7 without a B electrode
    fp32_inst = N * (n_full * 213 + (m - n_full) * 93 + src_b * 162 + src_a * 42)
    jac_ms = float(np.median(jac))
    ach = fp32_inst / (jac_ms / 1e3) / 1e12
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    alu_peak = 152 * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    value = world * args.steps / (ms / 1e3)
    out = {"metric": "ERT model evaluations/s (pole fields, g and all rows of J)", "value": value,
           "unit": "evaluations/s", "n_gpus": world, "steps": args.steps, "warmup": args.warmup,
           "ms_per_step": ms / args.steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": "mixed(fp32 cycle, df48 J rows, fp64 PCG)", "data": "synthetic",
           "config": {"workload": "ERT forward model and Jacobian, %d^3 FV cells, %d electrodes, m = %d "
                                  "(%s), GRF log-conductivity, PCG rtol %g" %
                                  (n, sv.n_e, m, "dipole-dipole grid" if grid else "line pair protocol",
                                   ERT_RTOL),
                      "n": [n, n, n], "n_e": sv.n_e, "m": m, "l2": "inputs larger than L2 (fields "
                      "%.1f GB, J %.1f GB)" % (sv.n_e * N * 8 / 1e9, m * N * 8 / 1e9)},
           "forward_ms": float(np.median(fwd)), "jacobian_rows_ms": jac_ms, "pcg_iters": iters,
           "data_term_ms": fields_ms,
           "rel_res_true": float(info.rel_res_true),
           "roofline": {"bound": "alu", "achieved": ach, "peak": alu_peak, "unit": "T FP32 inst/s",
                        "frac": ach / alu_peak, "traffic": NCU_BYTES_PER_J_ENTRY * m * N,
                        "traffic_note": "ncu 64^3 capture (32 electrodes, m = 496), scaled by J entries per launch",
                        "kernel": "k_jacobian<rows>",
                        "note": "FP32 instructions of the double-float J-row kernel (%d per launch) / its "
                                "event time; peak = FP32 issue rate (152 SMs x 128 lanes x max SM clock)"
                                % fp32_inst},
           "clocks": clocks, "impl": "ours"}
    if e2e_ms:
        out["e2e"] = {"value": world * args.e2e_steps / (e2e_ms / 1e3), "unit": "evaluations/s",
                      "h2d_bytes_per_step": N * 8, "d2h_bytes_per_step": m * 8, "steps": args.e2e_steps}
    if rank == 0 and not args.no_cpu_baseline:
        smp = ert_oracle_sample(32, args.ne if grid is None else args.ne, args.cpu_sample_s)
        out["cpu_baseline"] = {"value": 1.0 / (smp["eval_s"] * N / 32 ** 3), "unit": "evaluations/s",
                               "kind": "oracle", "cores": os.cpu_count(),
                               "sample": "oracle on a 32^3 grid with the same survey design (sparse LU "
                                         "fields, g, %d of %d J rows timed), scaled linearly in cells to "
                                         "%d^3: an upper bound, since the LU grows faster than linearly"
                                         % (smp["rows_timed"], smp["m"], n), "detail": smp}
    if rank == 0:
        print(json.dumps(out))


# ----------------------------------------------------------------------------
# Gauss-Newton inversion: Algorithm "Gauss-Newton with iterative solver"
# ----------------------------------------------------------------------------

def run_gn(args):
    import numpy as np
    import torch
    from paper_2209_02815_gb300 import h1w, inputs

    world, rank, local = dist_init(args)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    n = args.n
    N = n ** 3
    cells, abmn, k, _ = inputs.gn_survey(n, m_rows=args.m_rows or 1000)
    sv = h1w.Survey(cells, abmn, k, inputs.ERT_DIRICHLET_ALL_BUT_TOP)
    with torch.cuda.stream(stream):
        S = h1w.Solver(h1w.H1W_FV_CELL, (n, n, n), (1.0 / n,) * 3, GN_ALPHA, sv.m, device=dev, stream=stream)
        ls_true = torch.as_tensor(inputs.gn_truth(n), device=dev)
        g_true, _, _ = S.forward(sv, ls_true, rtol=1e-12)
        g_obs = torch.as_tensor(inputs.noisy(g_true.cpu().numpy()), device=dev)
        m_ref = torch.full((N,), math.log(0.01), dtype=torch.float64, device=dev)
        m = m_ref.clone()
        if args.warmup:
            S.gn_inversion(sv, g_obs, m_ref, m, min(args.warmup, 2), rtol_fwd=ERT_RTOL, rtol=RTOL, maxit=MAXIT)
        m.copy_(m_ref)
        torch.cuda.synchronize()
        barrier(world)
        clk = ClockSampler(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        hist, g, _ = S.gn_inversion(sv, g_obs, m_ref, m, args.gn_steps, rtol_fwd=ERT_RTOL, rtol=RTOL, maxit=MAXIT)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        ms = allmax(world, e0.elapsed_time(e1))
        t = S.timings()
        err_true = float(torch.linalg.norm(m - ls_true) / torch.linalg.norm(ls_true - m_ref))
    value = world * args.gn_steps / (ms / 1e3)
    out = {"metric": "Gauss-Newton steps/s (ERT inversion: forward, J, Laplace-Woodbury PCG, update)",
           "value": value, "unit": "GN steps/s", "n_gpus": world, "steps": args.gn_steps, "warmup": args.warmup,
           "ms_per_step": ms / args.gn_steps, "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
           "dtype": DTYPE_MIXED, "data": "synthetic",
           "config": {"workload": "ERT inversion, %d^3 FV cells, two Gaussian anomalies (10x and 0.1x of "
                                  "0.01 S/m), %d surface electrodes (6 x 8), pair protocol m = %d, 2 %% noise, "
                                  "alpha = %g, m_0 = m_ref" % (n, sv.n_e, sv.m, GN_ALPHA),
                      "n": [n, n, n], "n_e": sv.n_e, "m": sv.m, "rtol_forward": ERT_RTOL, "rtol_gn": RTOL},
           "misfit": [float(h_.misfit) for h_ in hist], "final_misfit": float(torch.linalg.norm(
               S.forward(sv, m, rtol=ERT_RTOL)[0] - g_obs)),
           "noise_level": float(torch.linalg.norm(g_obs - g_true)),
           "rel_model_error": err_true,
           "fwd_iters": [int(h_.fwd_iters) for h_ in hist], "gn_iters": [int(h_.gn_iters) for h_ in hist],
           "last_step_phases_ms": {"t_H_ms": t.t_H_ms, "t_C_ms": t.t_C_ms, "t_chol_ms": t.t_chol_ms,
                                   "t_pcg_ms": t.t_pcg_ms},
           "roofline": None,
           "roofline_note": "a GN step runs the kernels of the default line (GN solve, about 70 % of the step) "
                            "and of --ert (forward and J rows); their rooflines are reported there",
           "clocks": clocks, "impl": "ours"}
    if rank == 0:
        print(json.dumps(out))


# ----------------------------------------------------------------------------
# our arm
# ----------------------------------------------------------------------------

def run_ours(args):
    import numpy as np
    import torch
    from paper_2209_02815_gb300 import h1w, inputs

    world, rank, local = dist_init(args)
    dev = torch.device("cuda", local)
    stream = torch.cuda.Stream(dev)
    n = args.n
    with torch.cuda.stream(stream):
        pr = inputs.ert_problem(n, n_e_line=args.ne, alpha=args.alpha, device=dev, m_rows=args.m_rows,
                                grid=electrode_grid(args))
        J = pr.J
        m, N = J.shape
        o_main = None
        if args.arith == "fp64" or args.rhs_block > 0 or args.precond == "laplace" or args.cheb_degree > 0 or \
                args.pcg_mode != 0 or args.cheb_ratio > 0:
            o_main = h1w.h1w_default_options()
            if args.cheb_ratio > 0:
                o_main.cheb_ratio = args.cheb_ratio
            if args.cheb_degree > 0:
                o_main.cheb_degree = args.cheb_degree
            o_main.pcg_mode = args.pcg_mode
            if args.precond == "laplace":
                o_main.precond = 1
            if args.arith == "fp64":
                o_main.cap_gemm = 1
                o_main.mg_arith = 1
            if args.rhs_block > 0:
                o_main.rhs_block = args.rhs_block
        S = h1w.Solver(h1w.H1W_FV_CELL, (n, n, n), (1.0 / n,) * 3, args.alpha, m, device=dev, stream=stream,
                       opt=o_main)
        dm = torch.as_tensor(pr.logsigma - pr.m_ref, device=dev)
        d = torch.as_tensor(pr.d, device=dev)
        S.capacitance(J)
        b = S.gn_rhs(dm, d)
        x = torch.empty_like(b)
        for _ in range(args.warmup):
            S.capacitance(J)
            _, info = S.pcg(b, RTOL, args.maxit, x=x, raise_on_notconv=args.precond != "laplace")
        stream.synchronize()
        barrier(world)
        torch.cuda.synchronize()
        clk = ClockSampler(local)
        clk.start()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        phase = {"t_H_ms": [], "t_C_ms": [], "t_chol_ms": [], "t_pcg_ms": []}
        kern = {k_: [0.0, 0] for k_ in ("gemm_kernel", "jdot", "op", "hdot", "hupd", "vc_down", "vc_up",
                                        "split_j", "split_h", "d2df")}
        launches = 0
        iters = []
        e0.record(stream)
        for _ in range(args.steps):
            S.capacitance(J)
            _, info = S.pcg(b, RTOL, args.maxit, x=x, raise_on_notconv=args.precond != "laplace")
            t = S.timings()
            for k_ in phase:
                phase[k_].append(getattr(t, k_))
            for k_ in kern:
                kern[k_][0] += getattr(t, "t_" + k_ + "_ms")
                kern[k_][1] += getattr(t, "n_" + k_)
            launches += t.launches_capacitance + t.launches_pcg
            iters.append(info.iters)
        e1.record(stream)
        torch.cuda.synchronize()
        clocks = clk.stop()
        barrier(world)
        ms = e0.elapsed_time(e1)
        ms_max = allmax(world, ms)
        rel_true = info.rel_res_true
        x_timed = x.clone()   # the e2e and FP64-form legs below reuse x
        pcg_graph = args.pcg_mode == 0
        if pcg_graph:
            # the device-driven loop times no individual kernels: one more solve, untimed, with
            # the host loop gives the per-kernel times of the PCG passes (same kernels, same order)
            S.set_pcg_mode(1)
            _, info_h = S.pcg(b, RTOL, args.maxit, x=x, raise_on_notconv=args.precond != "laplace")
            th = S.timings()
            S.set_pcg_mode(0)
            for k_ in ("jdot", "op", "hdot", "hupd"):
                kern[k_][0] = getattr(th, "t_" + k_ + "_ms") * args.steps
                kern[k_][1] = getattr(th, "n_" + k_) * args.steps

        # end to end: host buffers in, host result out, through the public API
        e2e = None
        if args.e2e_steps > 0:
            J_host = torch.empty(J.shape, dtype=torch.float64, pin_memory=True)
            J_host.copy_(J)
            b_host = torch.empty(b.shape, dtype=torch.float64, pin_memory=True)
            b_host.copy_(b)
            x_host = torch.empty_like(b_host).pin_memory()
            J_dev = torch.empty_like(J)
            # the plain host-to-device copy rate of J, for reference
            c0 = torch.cuda.Event(enable_timing=True)
            c1 = torch.cuda.Event(enable_timing=True)
            c0.record(stream)
            J_dev.copy_(J_host, non_blocking=True)
            c1.record(stream)
            torch.cuda.synchronize()
            h2d_gbs = J.numel() * 8 / (c0.elapsed_time(c1) / 1e3) / 1e9
            J_dev2 = torch.empty_like(J)

            def copy_waits():
                # time line H's stream waited for rows of J, and the host-link rate of the step's
                # whole copy of J (first batch's start to last batch's end; the copy runs without
                # gaps, so this is the link's rate)
                prof = S.copy_profile()
                wait, prev = 0.0, 0.0
                for pb in prof:
                    wait += max(0.0, pb["cycle_begin"] - prev)
                    prev = pb["cycle_end"]
                rate = None
                if prof:
                    dt_ = prof[-1]["copy_end"] - prof[0]["copy_begin"]
                    if dt_ > 0:
                        rate = sum(pb["rows"] for pb in prof) * N * 8 / (dt_ / 1e3) / 1e9
                return wait, rate

            def e2e_run(steps, pipelined):
                # one step: b in, J in (row batches, overlapped with line H), solve, x out. Pipelined:
                # the copy of the next step's J into the other device buffer (h1w_prefetch_J) starts
                # once this step's capacitance has returned, so it runs beside this step's PCG and
                # is done, or nearly, when the next step's line H needs its rows. The first step's
                # J is copied by its own capacitance call, batch by batch under line H.
                ev = [torch.cuda.Event(enable_timing=True) for _ in range(steps + 1)]
                waits = []
                phases_k = []
                ev[0].record(stream)
                bufs = (J_dev, J_dev2)
                for k_ in range(steps):
                    # b and x go through h1w_pcg_host, which reads and writes the pinned host
                    # vectors with kernels: a host copy queued on the solver's stream while a
                    # copy of J ran on the copy stream held the stream's next work back until
                    # all of J had arrived (measured, about 40 ms per step)
                    S.capacitance_from_host(J_host, bufs[k_ % 2] if pipelined else J_dev)
                    if pipelined and k_ + 1 < steps:
                        S.prefetch_J(J_host, bufs[(k_ + 1) % 2])
                    waits.append(copy_waits())
                    S.pcg_host(b_host, x_host, RTOL, MAXIT)
                    ev[k_ + 1].record(stream)
                    t_ = S.timings()
                    phases_k.append([round(float(getattr(t_, p_)), 2) for p_ in phase])
                torch.cuda.synchronize()
                step_ms = [ev[k_].elapsed_time(ev[k_ + 1]) for k_ in range(steps)]
                total = allmax(world, ev[0].elapsed_time(ev[-1]))
                srt = sorted(step_ms)
                return {"value": world * steps / (total / 1e3), "unit": "solves/s", "steps": steps,
                        "median_step_ms": float(statistics.median(step_ms)), "min_step_ms": srt[0],
                        "max_step_ms": srt[-1], "median_value": world * 1e3 / float(statistics.median(step_ms)),
                        "step_ms": step_ms,
                        "lineH_copy_wait_ms": [w[0] for w in waits],
                        "phases_ms_per_step (H, C, chol, pcg)": phases_k,
                        "link_gb_per_s": [w[1] for w in waits]}

            e2e_run(1, False)  # untimed: the first call creates the copy stream and its events
            e2e_run(2, True)
            barrier(world)
            te0 = e2e_run(args.e2e_steps, False)
            te = S.timings()
            e2e = e2e_run(args.e2e_steps, True)
            e2e.update({"h2d_bytes_per_step": int(J.numel() * 8 + b.numel() * 8),
                        "d2h_bytes_per_step": int(x.numel() * 8), "h2d_copy_gb_per_s": h2d_gbs,
                        "api": "Solver.capacitance_from_host + prefetch_J + pcg_host (h1w_capacitance_from_host, "
                               "h1w_prefetch_J of the next J, h1w_pcg_host), J double-buffered on the device",
                        "unpipelined": {k_: te0[k_] for k_ in ("value", "median_value", "median_step_ms",
                                                              "min_step_ms", "max_step_ms", "step_ms",
                                                              "lineH_copy_wait_ms",
                                                              "link_gb_per_s")},
                        "last_step_phases_ms": {k_: float(getattr(te, k_)) for k_ in phase}})
            del J_dev2
            del J_host, J_dev

        # the plain FP64 GPU form of the same step (FP64 V-cycle and Krylov passes, FP64
        # CUDA-core capacitance GEMM), same inputs, for comparison with the headline
        fp64_form = None
        accuracy = None
        x64_keep = None
        if (args.fp64_form_steps > 0 or args.accuracy) and args.arith == "mixed":
            o64 = h1w.h1w_default_options()
            o64.cap_gemm = 1
            o64.mg_arith = 1
            if args.accuracy:   # both workspaces do not fit at the largest sizes
                x_tight, i_tight = S.pcg(b, ACC_RTOL, 4 * MAXIT, x=torch.empty_like(x), raise_on_notconv=False)
                S.close()
                del S
                torch.cuda.synchronize()
                torch.cuda.empty_cache()
            S64 = h1w.Solver(h1w.H1W_FV_CELL, (n, n, n), (1.0 / n,) * 3, args.alpha, m, device=dev, stream=stream,
                             opt=o64)
            S64.capacitance(J)                      # untimed warm-up solve
            S64.pcg(b, RTOL, MAXIT, x=x)
            if args.accuracy:
                # the timed mixed-precision solution against the plain FP64 form solved to 1e-12;
                # the FP64 form's own solution at the bench's rtol (in x) shows how far any
                # solution at that residual is from the converged one
                x_fp64_at_rtol = x.clone()
                x64, i64 = S64.pcg(b, ACC_RTOL, 4 * MAXIT, x=torch.empty_like(x), raise_on_notconv=False)
                dx = x_timed - x64
                dx64 = x_fp64_at_rtol - x64
                accuracy = {"rel_err_vs_fp64_form": float(torch.linalg.norm(dx) / torch.linalg.norm(x64)),
                            "max_abs_err_over_max_abs": float(dx.abs().max() / x64.abs().max()),
                            "fp64_form_rtol": ACC_RTOL, "fp64_form_iters": int(i64.iters),
                            "fp64_form_rel_res_true": float(i64.rel_res_true),
                            "mixed_rtol": RTOL,
                            "fp64_form_at_mixed_rtol": {
                                "rel_err_vs_fp64_form": float(torch.linalg.norm(dx64) / torch.linalg.norm(x64)),
                                "max_abs_err_over_max_abs": float(dx64.abs().max() / x64.abs().max())},
                            "bound_after_refinement": 1e-7,
                            "mixed_at_fp64_form_rtol": {
                                "rel_err_vs_fp64_form": float(torch.linalg.norm(x_tight - x64) / torch.linalg.norm(x64)),
                                "max_abs_err_over_max_abs": float((x_tight - x64).abs().max() / x64.abs().max()),
                                "iters": int(i_tight.iters), "restarts": int(i_tight.restarts),
                                "rel_res_true": float(i_tight.rel_res_true)}}
                x64_keep = x64
            torch.cuda.synchronize()
            if args.fp64_form_steps > 0:
                g0 = torch.cuda.Event(enable_timing=True)
                g1 = torch.cuda.Event(enable_timing=True)
                g0.record(stream)
                for _ in range(args.fp64_form_steps):
                    S64.capacitance(J)
                    _, inf64 = S64.pcg(b, RTOL, MAXIT, x=x)
                g1.record(stream)
                torch.cuda.synchronize()
                gms = allmax(world, g0.elapsed_time(g1))
                fp64_form = {"value": world * args.fp64_form_steps / (gms / 1e3), "unit": "solves/s",
                             "ms_per_step": gms / args.fp64_form_steps, "steps": args.fp64_form_steps,
                             "pcg_iters": int(inf64.iters), "rel_res_true": float(inf64.rel_res_true),
                             "options": "cap_gemm=1 (FP64 CUDA-core GEMM), mg_arith=1 (FP64 V-cycle and passes)"}
            del S64

    value = world * args.steps / (ms_max / 1e3)
    if fp64_form:
        fp64_form["headline_over_fp64_form"] = value / fp64_form["value"]
    mean = {k_: float(np.mean(v_)) for k_, v_ in phase.items()}
    peaks = {}
    try:
        with open(os.path.join(ROOT, "MEASURED_PEAKS.json")) as f:
            peaks = json.load(f)
    except OSError:
        pass
    hbm = float(peaks.get("hbm_gbs", 6746.0))
    bf16_sus = float(peaks.get("bf16_tflops_sustained", 1715.2))
    # per-kernel rates from CUDA events on the library's stream (h1w_get_timings)
    tiles = sum(max(0, (m + 63) // 64 - 2 * I) for I in range((m + 127) // 128))
    kp = min(((N + 2047) // 2048) * 2048, 262144)
    panels = (N + kp - 1) // kp
    gemm_flops_launch = tiles * 28 * 2.0 * 128 * 64 * kp        # digit-pair products per panel launch
    table = {}
    def rate(name, total_ms, n, per_launch, unit, bound, peak, note):
        if n == 0 or total_ms <= 0:
            return
        avg = total_ms / n
        ach = per_launch / (avg / 1e3) / (1e12 if unit == "TFLOP/s" else 1e9)
        table[name] = {"bound": bound, "achieved": ach, "peak": peak, "unit": unit, "frac": ach / peak,
                       "avg_launch_ms": avg, "launches_per_step": n / args.steps,
                       "ms_per_step": total_ms / args.steps, "algorithmic_per_launch": per_launch, "note": note}
    mat = 8.0 * m * N
    rate("k_ozaki_gemm", kern["gemm_kernel"][0], kern["gemm_kernel"][1], gemm_flops_launch, "TFLOP/s", "tensor",
         bf16_sus, "BF16 digit-pair products of one 262144-wide K panel; peak = measured sustained BF16")
    rate("k_rows_dot_df (J z)", kern["jdot"][0], kern["jdot"][1], mat + 8.0 * N, "GB/s", "hbm", hbm,
         "bytes of J (double-float) and z per pass")
    rate("k_apply_op_df<FV> (stencil + J^T w)", kern["op"][0], kern["op"][1], mat + 16.0 * N, "GB/s", "hbm", hbm,
         "bytes of J (double-float), p and q per pass")
    # fused V-cycle legs on the finest level, against HBM with their algorithmic bytes per
    # fine cell and right-hand side; beside it the FP32 issue fraction: algorithmic FP32
    # instructions per fine cell (FMA counted once) of the double-float operations the legs
    # require, halo recomputation excluded, against 152 SMs x 128 FP32 lanes x the maximum
    # SM clock. The legs are bound by instruction issue (double-float arithmetic), so the
    # issue fraction explains the HBM one.
    alu_peak = 152 * 128 * float(peaks.get("sm_max_mhz", 2070.0)) * 1e6 / 1e12
    n_up = kern["vc_up"][1]
    for key, name, byts, ops in (("vc_down", "k_pre_fused (finest level: smoothing + residual + restriction)",
                                  HBM_BYTES_DOWN, FP32_OPS_DOWN),
                                 ("vc_up", "k_post_fused (finest level: prolongation + smoothing)", HBM_BYTES_UP,
                                  FP32_OPS_UP)):
        n_ = kern[key][1]
        if n_:
            cell_rhs = float(m) * N * args.steps / n_      # fine cells x right-hand sides per launch
            rate(name, kern[key][0], n_, byts * cell_rhs, "GB/s", "hbm", hbm,
                 "%d bytes per fine cell and right-hand side (b, x, y in and out as double-floats, the coarse "
                 "vector at 1/8)" % byts)
            t_ = table[name]
            t_["issue_bound"] = {"achieved": ops * cell_rhs / (t_["avg_launch_ms"] / 1e3) / 1e12,
                                 "peak": alu_peak, "unit": "T FP32 inst/s",
                                 "frac": ops * cell_rhs / (t_["avg_launch_ms"] / 1e3) / 1e12 / alu_peak,
                                 "note": "%d algorithmic FP32 instructions per fine cell and right-hand side "
                                         "(double-float arithmetic, halo excluded); peak = FP32 issue rate"
                                         % ops}
    rate("k_rows_dot_df (H^T r)", kern["hdot"][0], kern["hdot"][1], mat + 8.0 * N, "GB/s", "hbm", hbm,
         "bytes of H (double-float) and r per pass")
    rate("k_woodbury_update_df (z update)", kern["hupd"][0], kern["hupd"][1], mat + 32.0 * N, "GB/s", "hbm", hbm,
         "bytes of H, z0, r and z per pass")
    # operand preparation of line C and line H: per panel, the split of J (FP64 in) and of H
    # (double-float in) writes seven BF16 digits (14 bytes) per entry plus one exponent per
    # 512-entry chunk; the conversion of J to double-floats reads 8 and writes 8 bytes per entry
    kw_avg = float(N) / panels
    rate("k_split_digits<double> (J digits)", kern["split_j"][0], kern["split_j"][1], 22.0 * m * kw_avg, "GB/s",
         "hbm", hbm, "8 bytes of J in, 14 bytes of digits out per entry of one K panel")
    rate("k_split_digits<df> (H digits)", kern["split_h"][0], kern["split_h"][1], 22.0 * m * kw_avg, "GB/s",
         "hbm", hbm, "8 bytes of H (double-float) in, 14 bytes of digits out per entry of one K panel")
    if kern["d2df"][1] and kern["split_j"][1] == 0 and args.arith == "mixed":
        # J's digits split in line H together with its double-float copy (the full-K digit
        # buffer): per row batch 8 bytes in, 8 + 14 bytes out per entry; line C splits only H
        rate("k_split_digits<double> + double-float copy (J, line H)", kern["d2df"][0], kern["d2df"][1],
             30.0 * m * N * args.steps / kern["d2df"][1], "GB/s", "hbm", hbm,
             "8 bytes of J in, 8 bytes of double-float copy and 14 bytes of digits out per entry of the row batch")
    elif kern["d2df"][1]:
        rate("k_d2df (J to double-floats, line H)", kern["d2df"][0], kern["d2df"][1],
             16.0 * m * N * args.steps / kern["d2df"][1], "GB/s", "hbm", hbm,
             "8 bytes in, 8 bytes out per entry of J's row batch")
    dom = max(table, key=lambda k_: table[k_]["ms_per_step"]) if table else None
    roofline = dict(table[dom], kernel=dom, traffic=None) if dom else None
    # DRAM bytes per launch from one ncu capture of the same kernel build on the 64^3 case
    # (dram__bytes_read.sum + dram__bytes_write.sum of the finest up leg), scaled by the cells x
    # right-hand sides of an average launch here: reads equal the algorithmic x, b and
    # coarse-vector bytes there, so traffic grows in proportion
    for key_, n_key in (("k_post_fused", "vc_up"), ("k_pre_fused", "vc_down")):
        if roofline and dom.startswith(key_) and kern[n_key][1] and NCU_TRAFFIC_BUILD == FUSED_BUILD:
            roofline["traffic"] = NCU_BYTES_PER_CELL_RHS[key_] * float(m) * N * args.steps / kern[n_key][1]
            roofline["traffic_note"] = "ncu 64^3 x 128 RHS capture, scaled by cell-RHS per launch"
    if roofline:
        roofline["peak_note"] = "of measured (MEASURED_PEAKS.json)" if peaks else "of fallback"
    # independent check of the timed solution: the oracle's FP64 operator (C, CSR K + M,
    # J in FP64 on the host) recomputes ||b - A x|| / ||b||
    oracle_check = None
    J_np = None
    if rank == 0 and not args.no_oracle_check and args.precond == "woodbury":
        from oracle import ccg
        from oracle import discretization as odisc
        J_np = J.cpu().numpy()
        x_np = x_timed.cpu().numpy()
        b_np = b.cpu().numpy()
        t0_ = time.perf_counter()
        op = ccg.CsrOperator(odisc.regularization_operator("fv", (n, n, n), (1.0 / n,) * 3), args.alpha, J_np)
        res = b_np - op.apply(x_np)
        oracle_check = {"rel_res_true_oracle": float(np.linalg.norm(res) / np.linalg.norm(b_np)),
                        "rel_res_true_gpu": float(rel_true), "seconds": time.perf_counter() - t0_,
                        "fp64_form_1e-12_rel_res_true_oracle": (
                            float(np.linalg.norm(b_np - op.apply(x64_keep.cpu().numpy())) / np.linalg.norm(b_np))
                            if accuracy else None),
                        "note": "||b - A x||/||b|| of the last timed solution, A applied by the oracle "
                                "(CSR K + M and FP64 J on the host)"}
    out = {
        "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_max / args.steps, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": DTYPE_MIXED if args.arith == "mixed" else "f64",
        "data": "synthetic",
        "config": {"workload": workload(n, m, electrode_grid(args), args.alpha), "n": [n, n, n], "N": N, "m": m, "alpha": args.alpha,
                   "rtol": RTOL, "precond": args.precond,
                   "parallelism": "replicas" if world > 1 else "single GPU",
                   "l2": "inputs larger than L2 (J is %.1f GB)" % (J.numel() * 8 / 1e9)},
        "phases_ms": mean, "pcg_iters": iters, "rel_res_true": rel_true,
        "mg_dof_per_s": float(m) * N / (mean["t_H_ms"] / 1e3),
        "pcg_only_solves_per_s": world * 1e3 / mean["t_pcg_ms"],
        "arith": ({"operator_and_krylov": "f64", "true_residual": "f64",
                   "vcycle": "double-float (FP32 pairs, ~48 bits)",
                   "capacitance_gemm": "BF16 tensor cores on an exact 48-bit digit split, FP64 accumulation",
                   "cholesky": "f64", "woodbury_passes": "double-float", "krylov_J_passes": "double-float"}
                  if args.arith == "mixed" else
                  {"everything": "f64 (plain FP64 form: FP64 cycle and passes, CUDA-core C)"}),
        "pcg_loop": "device-driven (CUDA graph with a conditional while node)" if args.pcg_mode == 0 else "host loop",
        "roofline": roofline, "kernels": table, "clocks": clocks, "gpu_launches": int(launches), "e2e": e2e,
        "fp64_form": fp64_form, "accuracy": accuracy, "oracle_check": oracle_check,
        "impl": "ours",
    }
    if rank == 0 and world == 1 and not args.no_cpu_baseline and args.cpu_full_solve:
        from oracle import reference_run
        del J_np
        full = reference_run.main(n, args.ne)
        t_full = full["t_H_s"] + full["t_C_chol_s"] + full["t_pcg_s"]
        out["cpu_baseline"] = {"value": 1.0 / t_full, "unit": "solves/s", "cores": full["threads"],
                               "kind": "oracle", "sample": "full solve (lines H, C, chol and PCG to the "
                                                          "FP64 true residual 1e-8, timed, not extrapolated)",
                               "detail": full}
    elif rank == 0 and world == 1 and not args.no_cpu_baseline:
        J_host = J.cpu().numpy() if J_np is None else J_np
        s = oracle_sample(J_host, pr.logsigma, pr.m_ref, pr.d, n, args.cpu_sample_s, iters_fallback=iters[-1],
                          default_case=(args.grid is None and args.m_rows is None and args.ne == N_E
                                        and args.alpha == ALPHA))
        out["cpu_baseline"] = {"value": (1.0 / s["t_solve_s"]) if s["iterations"] else None,
                               "unit": "solves/s", "cores": s["threads"], "kind": "oracle",
                               "sample": ("oracle phases timed on bounded samples and extrapolated: "
                                          f"{s['vcycles_timed']} scipy V-cycles (x m), "
                                          f"{s['applies_timed']} operator applies, one 256-row GEMM "
                                          "(scaled by (m/256)^2), iterations from the oracle's full "
                                          "solve of this workload"), "detail": s}
    if rank == 0:
        print(json.dumps(out))
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


def run_reference(args):
    import numpy as np
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from paper_2209_02815_gb300 import inputs
    n = args.n
    pr = inputs.ert_problem(n, n_e_line=args.ne, alpha=args.alpha, device="cpu", m_rows=args.m_rows,
                            grid=electrode_grid(args))
    J = np.ascontiguousarray(pr.J)
    vals = []
    last = None
    budget = max(5.0, min(args.cpu_sample_s, 120.0 / max(1, args.steps + args.warmup)))
    wall = []
    for i in range(args.warmup + args.steps):
        t0 = time.perf_counter()
        s = oracle_sample(J, pr.logsigma, pr.m_ref, pr.d, n, budget,
                          default_case=(args.grid is None and args.m_rows is None and args.ne == N_E
                                        and args.alpha == ALPHA))
        if i >= args.warmup:
            vals.append(s["t_solve_s"])
            wall.append(time.perf_counter() - t0)
        last = s
    t = statistics.median(vals)
    value = 1.0 / t if last["iterations"] else None
    # ms_per_step is the wall time of one step as run (one bounded sample); the solve time
    # that the sample extrapolates to is reported beside it
    out = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
           "warmup": args.warmup, "ms_per_step": statistics.median(wall) * 1e3,
           "extrapolated_ms_per_solve": t * 1e3, "extrapolated": True, "higher_is_better": True,
           "scaling": "weak",
           "vs_baseline": None, "dtype": "f64", "data": "synthetic",
           "config": {"workload": workload(n, int(J.shape[0]), electrode_grid(args), args.alpha), "n": [n, n, n],
                      "m": int(J.shape[0]), "alpha": args.alpha,
                      "rtol": RTOL},
           "impl": "reference",
           "cpu_baseline": {"value": value, "unit": "solves/s", "kind": "oracle", "cores": last["threads"],
                            "sample": "EXTRAPOLATED: each step times the oracle's phases on bounded "
                                      "samples (scipy V-cycles, C operator applies, a 256-row GEMM) and "
                                      "extrapolates them to one full solve with the oracle's own "
                                      "iteration count; ms_per_step is the sample's wall time",
                            "detail": last},
           "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(out))


if __name__ == "__main__":
    a = parse()
    if a.impl == "reference":
        run_reference(a)
    elif a.ert:
        run_ert(a)
    elif a.gn_steps > 0:
        run_gn(a)
    elif a.batch > 0:
        run_batch(a)
    else:
        run_ours(a)
