"""Python binding of the h1w C ABI (argument marshalling only).

Every function here has the name of the C entry point it calls and does no
arithmetic of its own: tensors are checked for device, dtype, contiguity and
size, and their data pointers are passed through ctypes. PyTorch supplies
device memory (the workspace and the vectors) and the CUDA stream.

The shared library is built in-tree by ``paper_2209_02815_gb300.build``. If it
is missing or cannot be loaded, ``load()`` raises: there is no CPU fallback.
"""
from __future__ import annotations

import ctypes
import os

import torch

from . import build as _build

H1W_OK, H1W_EINVAL, H1W_ENOMEM, H1W_ECUDA, H1W_ENOTCONV = 0, 1, 2, 3, 4
H1W_ENOTSPD, H1W_ETIMEOUT, H1W_EUNSUPPORTED, H1W_ESTATE = 5, 6, 7, 8
H1W_Q1_VERTEX, H1W_FV_CELL = 1, 2
H1W_STALL_NONE, H1W_STALL_CAP_GEMM, H1W_STALL_PREC_SOLVE = 0, 1, 2

_STATUS_NAMES = {0: "H1W_OK", 1: "H1W_EINVAL", 2: "H1W_ENOMEM", 3: "H1W_ECUDA", 4: "H1W_ENOTCONV",
                 5: "H1W_ENOTSPD", 6: "H1W_ETIMEOUT", 7: "H1W_EUNSUPPORTED", 8: "H1W_ESTATE"}


class H1wError(RuntimeError):
    def __init__(self, status: int, msg: str):
        super().__init__(f"{_STATUS_NAMES.get(status, status)}: {msg}")
        self.status = status


class Grid(ctypes.Structure):
    _fields_ = [("dim", ctypes.c_int32), ("disc", ctypes.c_int32), ("n", ctypes.c_int32 * 3),
                ("h", ctypes.c_double * 3), ("alpha", ctypes.c_double)]


class Options(ctypes.Structure):
    _fields_ = [("cheb_degree", ctypes.c_int32), ("rhs_block", ctypes.c_int32),
                ("max_restarts", ctypes.c_int32), ("cap_gemm", ctypes.c_int32),
                ("mg_arith", ctypes.c_int32), ("mg_unfused", ctypes.c_int32), ("precond", ctypes.c_int32),
                ("pcg_mode", ctypes.c_int32), ("cheb_ratio", ctypes.c_double), ("j_digits", ctypes.c_int32)]


class Timings(ctypes.Structure):
    _fields_ = [("t_H_ms", ctypes.c_float), ("t_C_ms", ctypes.c_float), ("t_chol_ms", ctypes.c_float),
                ("t_pcg_ms", ctypes.c_float), ("launches_capacitance", ctypes.c_int64),
                ("launches_pcg", ctypes.c_int64), ("t_gemm_kernel_ms", ctypes.c_float),
                ("t_jdot_ms", ctypes.c_float), ("t_op_ms", ctypes.c_float), ("t_hdot_ms", ctypes.c_float),
                ("t_hupd_ms", ctypes.c_float), ("n_gemm_kernel", ctypes.c_int32), ("n_jdot", ctypes.c_int32),
                ("n_op", ctypes.c_int32), ("n_hdot", ctypes.c_int32), ("n_hupd", ctypes.c_int32),
                ("reserved", ctypes.c_int32), ("t_vc_down_ms", ctypes.c_float), ("t_vc_up_ms", ctypes.c_float),
                ("n_vc_down", ctypes.c_int32), ("n_vc_up", ctypes.c_int32), ("t_split_j_ms", ctypes.c_float),
                ("t_split_h_ms", ctypes.c_float), ("t_d2df_ms", ctypes.c_float), ("n_split_j", ctypes.c_int32),
                ("n_split_h", ctypes.c_int32), ("n_d2df", ctypes.c_int32), ("reserved2", ctypes.c_int32)]


class Info(ctypes.Structure):
    _fields_ = [("iters", ctypes.c_int32), ("restarts", ctypes.c_int32),
                ("rel_res_true", ctypes.c_double), ("rel_res_rec", ctypes.c_double)]


class SurveyC(ctypes.Structure):
    _fields_ = [("n_e", ctypes.c_int32), ("cell", ctypes.POINTER(ctypes.c_int32)), ("m", ctypes.c_int32),
                ("abmn", ctypes.POINTER(ctypes.c_int32)), ("k", ctypes.POINTER(ctypes.c_double)),
                ("dirichlet", ctypes.c_uint32)]


class GnInfo(ctypes.Structure):
    _fields_ = [("fwd_iters", ctypes.c_int32), ("gn_iters", ctypes.c_int32), ("misfit", ctypes.c_double),
                ("rel_res_true", ctypes.c_double), ("step_norm", ctypes.c_double)]


_lib = None


def load(build_if_missing: bool = True) -> ctypes.CDLL:
    """Load libh1w.so (building it first when asked). Raises when unavailable."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_missing and (not os.path.exists(path) or _build._stale([])):
        _build.build()
    if not os.path.exists(path):
        raise RuntimeError(f"h1w CUDA library not found at {path}; run __graft_entry__.build()")
    lib = ctypes.CDLL(path)
    P, I32, D, SZ = ctypes.c_void_p, ctypes.c_int32, ctypes.c_double, ctypes.c_size_t
    G, O, IN = ctypes.POINTER(Grid), ctypes.POINTER(Options), ctypes.POINTER(Info)
    sig = {
        "h1w_default_options": (None, [O]),
        "h1w_workspace_size": (SZ, [G, I32, O]),
        "h1w_setup": (I32, [G, I32, O, P, SZ, P, ctypes.POINTER(P)]),
        "h1w_capacitance": (I32, [P, I32, P]),
        "h1w_capacitance_from_host": (I32, [P, I32, P, P]),
        "h1w_apply_prec": (I32, [P, P, P]),
        "h1w_apply_op": (I32, [P, P, P]),
        "h1w_vcycle": (I32, [P, I32, P, P]),
        "h1w_gn_rhs": (I32, [P, P, P, P]),
        "h1w_pcg": (I32, [P, P, P, D, I32, IN]),
        "h1w_pcg_host": (I32, [P, P, P, D, I32, IN]),
        "h1w_capacitance_factors": (I32, [P, P, P]),
        "h1w_level_info": (I32, [P, I32, ctypes.POINTER(I32), ctypes.POINTER(I32)]),
        "h1w_get_timings": (I32, [P, ctypes.POINTER(Timings)]),
        "h1w_apply_op_static": (I32, [G, I32, P, P, P, P]),
        "h1w_solve_batch": (I32, [ctypes.POINTER(P), I32, ctypes.POINTER(I32), ctypes.POINTER(P),
                                  ctypes.POINTER(P), ctypes.POINTER(P), D, I32, I32, IN, ctypes.POINTER(I32)]),
        "h1w_solve_batch_graph": (I32, [ctypes.POINTER(P), I32, ctypes.POINTER(I32), ctypes.POINTER(P),
                                        ctypes.POINTER(P), ctypes.POINTER(P), D, I32, IN, ctypes.POINTER(I32)]),
        "h1w_autotune_workspace_size": (SZ, [G, I32, O]),
        "h1w_autotune": (I32, [G, I32, O, P, SZ, P, O, ctypes.POINTER(ctypes.c_float)]),
        "h1w_ert_workspace_size": (SZ, [P, I32, I32]),
        "h1w_forward": (I32, [P, ctypes.POINTER(SurveyC), P, P, P, P, SZ, D, I32, ctypes.c_uint32, IN]),
        "h1w_adjoint": (I32, [P, ctypes.POINTER(SurveyC), P, P, P, P, P, P, SZ]),
        "h1w_ert_jvp": (I32, [P, ctypes.POINTER(SurveyC), P, P, P, P, P, SZ]),
        "h1w_gn_step": (I32, [P, ctypes.POINTER(SurveyC), P, P, P, P, P, P, P, P, SZ, D, D, I32, ctypes.c_uint32,
                              ctypes.POINTER(GnInfo)]),
        "h1w_direct_workspace_size": (SZ, [P]),
        "h1w_solve_direct": (I32, [P, P, P, P, SZ]),
        "h1w_cholesky": (I32, [P, I32, P]),
        "h1w_prefetch_J": (I32, [P, I32, P, P]),
        "h1w_get_copy_profile": (I32, [P, I32, ctypes.POINTER(I32), ctypes.POINTER(I32),
                                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float),
                                       ctypes.POINTER(ctypes.c_float), ctypes.POINTER(ctypes.c_float)]),
        "h1w_inject_stall": (I32, [P, I32, ctypes.c_int64]),
        "h1w_set_pcg_mode": (I32, [P, I32]),
        "h1w_last_error": (ctypes.c_char_p, [P]),
        "h1w_destroy": (None, [P]),
    }
    for name, (res, args) in sig.items():
        fn = getattr(lib, name)
        fn.restype = res
        fn.argtypes = args
    _lib = lib
    return lib


def _ptr(t: torch.Tensor | None, n: int | None = None, name: str = "tensor") -> int | None:
    if t is None:
        return None
    if not t.is_cuda:
        raise ValueError(f"{name} must be a CUDA tensor")
    if t.dtype != torch.float64:
        raise ValueError(f"{name} must be float64")
    if not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous")
    if n is not None and t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} entries, needs {n}")
    return t.data_ptr()


def make_grid(disc: int, n, h, alpha: float) -> Grid:
    g = Grid()
    g.dim = 2 if disc == H1W_Q1_VERTEX else 3
    g.disc = disc
    nn = list(n) + [1] * (3 - len(n))
    hh = list(h) + [1.0] * (3 - len(h))
    for a in range(3):
        g.n[a] = int(nn[a])
        g.h[a] = float(hh[a])
    g.alpha = float(alpha)
    return g


def h1w_default_options() -> Options:
    o = Options()
    load().h1w_default_options(ctypes.byref(o))
    return o


def h1w_workspace_size(grid: Grid, m_max: int, opt: Options | None = None) -> int:
    return int(load().h1w_workspace_size(ctypes.byref(grid), int(m_max),
                                         ctypes.byref(opt) if opt is not None else None))


def h1w_last_error(ctx) -> str:
    s = load().h1w_last_error(ctx)
    return s.decode() if s else ""


def _check(st: int, ctx) -> None:
    if st != H1W_OK:
        raise H1wError(st, h1w_last_error(ctx))


def h1w_setup(grid: Grid, m_max: int, opt: Options | None, workspace: torch.Tensor,
              stream: torch.cuda.Stream | None = None):
    """Returns an opaque context handle (int)."""
    if not workspace.is_cuda or workspace.dtype != torch.uint8:
        raise ValueError("workspace must be a CUDA uint8 tensor")
    out = ctypes.c_void_p()
    s = (stream or torch.cuda.current_stream(workspace.device)).cuda_stream
    st = load().h1w_setup(ctypes.byref(grid), int(m_max), ctypes.byref(opt) if opt is not None else None,
                          workspace.data_ptr(), workspace.numel(), s, ctypes.byref(out))
    _check(st, None)
    return out.value


def h1w_capacitance(ctx, m: int, J: torch.Tensor | None, N: int) -> None:
    _check(load().h1w_capacitance(ctx, int(m), _ptr(J, m * N, "J") if m > 0 else None), ctx)


def h1w_capacitance_from_host(ctx, m: int, J_host: torch.Tensor, J_dev: torch.Tensor, N: int) -> None:
    if m > 0:
        if J_host.is_cuda or not J_host.is_pinned():
            raise ValueError("J_host must be a pinned CPU tensor")
        if J_host.dtype != torch.float64 or not J_host.is_contiguous() or J_host.numel() < m * N:
            raise ValueError("J_host must be a contiguous float64 tensor with m x N entries")
    _check(load().h1w_capacitance_from_host(ctx, int(m), J_host.data_ptr() if m > 0 else None,
                                            _ptr(J_dev, m * N, "J_dev") if m > 0 else None), ctx)


def h1w_autotune(grid: Grid, m: int, base: Options | None = None, device="cuda",
                 stream: torch.cuda.Stream | None = None):
    """Options with the fastest rhs_block for this grid and m (h1w_autotune; cached per
    process) and the V-cycle time per right-hand side in ms."""
    size = int(load().h1w_autotune_workspace_size(ctypes.byref(grid), int(m),
                                                  ctypes.byref(base) if base is not None else None))
    if size == 0:
        raise H1wError(H1W_EINVAL, "invalid grid/options for h1w_autotune")
    ws = torch.empty(size, dtype=torch.uint8, device=device)
    s = (stream or torch.cuda.current_stream(ws.device)).cuda_stream
    out = Options()
    ms = ctypes.c_float()
    _check(load().h1w_autotune(ctypes.byref(grid), int(m), ctypes.byref(base) if base is not None else None,
                               ws.data_ptr(), ws.numel(), s, ctypes.byref(out), ctypes.byref(ms)), None)
    return out, float(ms.value)


def solve_batch(solvers, Js, bs, xs, rtol: float, maxit: int = 500, threads: int = 8, graph: bool = False):
    """Capacitance + PCG for several Solver objects at once: h1w_solve_batch (a pool of host
    threads) or, with graph=True, h1w_solve_batch_graph (all systems in one CUDA graph).
    Each solver must have been created on its own stream. Returns (list of Info, list of
    status codes); raises H1wError when a system failed."""
    n = len(solvers)
    P = ctypes.c_void_p
    ctxs = (P * n)(*[s.ctx for s in solvers])
    ms = (ctypes.c_int32 * n)(*[int(J.shape[0]) if J is not None else 0 for J in Js])
    Jp = (P * n)(*[(_ptr(J, int(J.shape[0]) * s.N, "J") if J is not None and J.shape[0] else None)
                   for s, J in zip(solvers, Js)])
    bp = (P * n)(*[_ptr(b, s.N, "b") for s, b in zip(solvers, bs)])
    xp = (P * n)(*[_ptr(x, s.N, "x") for s, x in zip(solvers, xs)])
    infos = (Info * n)()
    sts = (ctypes.c_int32 * n)()
    for s, J, b, x in zip(solvers, Js, bs, xs):
        s.J = J
        s.m = int(J.shape[0]) if J is not None else 0
        s._enter(J, b, x)
    try:
        if graph:
            st = load().h1w_solve_batch_graph(ctxs, n, ms, Jp, bp, xp, float(rtol), int(maxit), infos, sts)
        else:
            st = load().h1w_solve_batch(ctxs, n, ms, Jp, bp, xp, float(rtol), int(maxit), int(threads), infos, sts)
    finally:
        for s in solvers:
            s._leave()
    if st != H1W_OK:
        raise H1wError(st, h1w_last_error(None))
    return list(infos), list(sts)


def h1w_apply_prec(ctx, r: torch.Tensor, z: torch.Tensor, N: int) -> None:
    _check(load().h1w_apply_prec(ctx, _ptr(r, N, "r"), _ptr(z, N, "z")), ctx)


def h1w_apply_op(ctx, p: torch.Tensor, q: torch.Tensor, N: int) -> None:
    _check(load().h1w_apply_op(ctx, _ptr(p, N, "p"), _ptr(q, N, "q")), ctx)


def h1w_vcycle(ctx, nrhs: int, b: torch.Tensor, x: torch.Tensor, N: int) -> None:
    _check(load().h1w_vcycle(ctx, int(nrhs), _ptr(b, nrhs * N, "b"), _ptr(x, nrhs * N, "x")), ctx)


def h1w_gn_rhs(ctx, dm: torch.Tensor, d: torch.Tensor | None, b: torch.Tensor, N: int, m: int) -> None:
    _check(load().h1w_gn_rhs(ctx, _ptr(dm, N, "dm"), _ptr(d, m, "d") if m > 0 else None,
                             _ptr(b, N, "b")), ctx)


def h1w_pcg(ctx, b: torch.Tensor, x: torch.Tensor, rtol: float, maxit: int, N: int,
            raise_on_notconv: bool = True) -> Info:
    info = Info()
    st = load().h1w_pcg(ctx, _ptr(b, N, "b"), _ptr(x, N, "x"), float(rtol), int(maxit), ctypes.byref(info))
    if st == H1W_ENOTCONV and not raise_on_notconv:
        return info
    _check(st, ctx)
    return info


def _host_ptr(t: torch.Tensor, n: int, name: str) -> int:
    if t.is_cuda or not t.is_pinned():
        raise ValueError(f"{name} must be a pinned CPU tensor")
    if t.dtype != torch.float64 or not t.is_contiguous():
        raise ValueError(f"{name} must be contiguous float64")
    if t.numel() < n:
        raise ValueError(f"{name} has {t.numel()} entries, needs {n}")
    return t.data_ptr()


def h1w_pcg_host(ctx, b_host: torch.Tensor, x_host: torch.Tensor, rtol: float, maxit: int, N: int,
                 raise_on_notconv: bool = True) -> Info:
    info = Info()
    st = load().h1w_pcg_host(ctx, _host_ptr(b_host, N, "b_host"), _host_ptr(x_host, N, "x_host"), float(rtol),
                             int(maxit), ctypes.byref(info))
    if st == H1W_ENOTCONV and not raise_on_notconv:
        return info
    _check(st, ctx)
    return info


def h1w_capacitance_factors(ctx, C: torch.Tensor | None, L: torch.Tensor | None, m: int) -> None:
    _check(load().h1w_capacitance_factors(ctx, _ptr(C, m * m, "C"), _ptr(L, m * m, "L")), ctx)


def h1w_level_info(ctx, level: int = 0):
    nl = ctypes.c_int32()
    n = (ctypes.c_int32 * 3)()
    _check(load().h1w_level_info(ctx, int(level), ctypes.byref(nl), n), ctx)
    return nl.value, tuple(n)


def h1w_get_timings(ctx) -> Timings:
    t = Timings()
    _check(load().h1w_get_timings(ctx, ctypes.byref(t)), ctx)
    return t


def h1w_apply_op_static(grid: Grid, m: int, J: torch.Tensor | None, p: torch.Tensor, q: torch.Tensor,
                        N: int, stream: torch.cuda.Stream | None = None) -> None:
    """Workspace-free operator apply (scratch in a fixed device array). The library takes the
    scratch address and launches on the current device, so the call runs with p's device
    current; J, p and q must all be on it."""
    for t, nm in ((J, "J"), (q, "q")):
        if t is not None and t.device != p.device:
            raise ValueError(f"{nm} is on {t.device}, p on {p.device}")
    with torch.cuda.device(p.device):
        s = (stream or torch.cuda.current_stream(p.device)).cuda_stream
        _check(load().h1w_apply_op_static(ctypes.byref(grid), int(m), _ptr(J, m * N, "J") if m > 0 else None,
                                          _ptr(p, N, "p"), _ptr(q, N, "q"), s), None)


class Survey:
    """An ERT survey in the layout of h1w_survey: electrode cells (n_e,), measurements
    abmn (m, 4) with -1 for an electrode at infinity, geometric factors k (m,), and
    the Dirichlet box faces as a bit mask (bit f: x-, x+, y-, y+, z-, z+)."""

    def __init__(self, cells, abmn, k, dirichlet: int):
        import numpy as np
        self.cells = np.ascontiguousarray(np.asarray(cells, dtype=np.int32))
        self.abmn = np.ascontiguousarray(np.asarray(abmn, dtype=np.int32).reshape(-1, 4))
        self.k = np.ascontiguousarray(np.asarray(k, dtype=np.float64))
        if self.k.shape[0] != self.abmn.shape[0]:
            raise ValueError("k needs one entry per measurement")
        self.dirichlet = int(dirichlet)
        c = SurveyC()
        c.n_e = self.cells.size
        c.cell = self.cells.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        c.m = self.abmn.shape[0]
        c.abmn = self.abmn.ctypes.data_as(ctypes.POINTER(ctypes.c_int32))
        c.k = self.k.ctypes.data_as(ctypes.POINTER(ctypes.c_double))
        c.dirichlet = self.dirichlet
        self.c = c

    @property
    def n_e(self) -> int:
        return int(self.cells.size)

    @property
    def m(self) -> int:
        return int(self.abmn.shape[0])


def h1w_ert_workspace_size(ctx, n_e: int, m: int) -> int:
    return int(load().h1w_ert_workspace_size(ctx, n_e, m))


H1W_FORWARD_WARM_START = 1


def h1w_forward(ctx, survey: Survey, logsigma: torch.Tensor, U: torch.Tensor, g: torch.Tensor | None,
                ws: torch.Tensor, rtol: float, maxit: int, N: int, raise_on_notconv: bool = True,
                flags: int = 0) -> Info:
    info = Info()
    st = load().h1w_forward(ctx, ctypes.byref(survey.c), _ptr(logsigma, N, "logsigma"),
                            _ptr(U, N * survey.n_e, "U"), _ptr(g, survey.m, "g"), ws.data_ptr(), ws.numel(),
                            rtol, maxit, flags, ctypes.byref(info))
    if st == H1W_ENOTCONV and not raise_on_notconv:
        return info
    _check(st, ctx)
    return info


def h1w_adjoint(ctx, survey: Survey, logsigma: torch.Tensor, U: torch.Tensor, r: torch.Tensor | None,
                JTr: torch.Tensor | None, J: torch.Tensor | None, ws: torch.Tensor, N: int) -> None:
    st = load().h1w_adjoint(ctx, ctypes.byref(survey.c), _ptr(logsigma, N, "logsigma"),
                            _ptr(U, N * survey.n_e, "U"), _ptr(r, survey.m, "r"), _ptr(JTr, N, "JTr"),
                            _ptr(J, N * survey.m, "J"), ws.data_ptr(), ws.numel())
    _check(st, ctx)


def h1w_gn_step(ctx, survey: Survey, g_obs: torch.Tensor, m_ref: torch.Tensor, m: torch.Tensor, U: torch.Tensor,
                J: torch.Tensor, g: torch.Tensor, scratch: torch.Tensor, ws: torch.Tensor, rtol_fwd: float,
                rtol: float, maxit: int, N: int, fwd_flags: int = 0) -> GnInfo:
    info = GnInfo()
    st = load().h1w_gn_step(ctx, ctypes.byref(survey.c), _ptr(g_obs, survey.m, "g_obs"), _ptr(m_ref, N, "m_ref"),
                            _ptr(m, N, "m"), _ptr(U, N * survey.n_e, "U"), _ptr(J, N * survey.m, "J"),
                            _ptr(g, survey.m, "g"), _ptr(scratch, 3 * N + survey.m, "scratch"), ws.data_ptr(),
                            ws.numel(), rtol_fwd, rtol, maxit, fwd_flags, ctypes.byref(info))
    _check(st, ctx)
    return info


def h1w_cholesky(ctx, A: torch.Tensor) -> None:
    """A = L L^T in place (A: n x n FP64 CUDA tensor, row-major), line chol's kernels."""
    n = int(A.shape[0])
    if A.dim() != 2 or A.shape[1] != n:
        raise ValueError("A must be square")
    _check(load().h1w_cholesky(ctx, n, _ptr(A, n * n, "A")), ctx)


def h1w_inject_stall(ctx, kind: int, wait_limit_ns: int = 0) -> None:
    _check(load().h1w_inject_stall(ctx, int(kind), int(wait_limit_ns)), ctx)


def h1w_destroy(ctx) -> None:
    if ctx:
        load().h1w_destroy(ctx)


def save_gn_checkpoint(path: str, step: int, m, U, hist) -> None:
    """Writes the state of a Gauss-Newton loop after `step` steps: the iterate m, the pole
    fields U (the next forward solve's warm start) and the per-step GnInfo records. The file
    is written beside `path` and renamed over it, so a reader sees the old or the new state."""
    state = {"format": "h1w-gn-checkpoint-1", "step": int(step), "m": m.detach().cpu(),
             "U": U.detach().cpu(),
             "hist": [{f: getattr(h, f) for f, _ in GnInfo._fields_} for h in hist]}
    tmp = path + ".tmp"
    torch.save(state, tmp)
    os.replace(tmp, path)


def load_gn_checkpoint(path: str, m, U):
    """Reads a checkpoint of save_gn_checkpoint into m and U (copied in place; the shapes
    must match) and returns (step, list of GnInfo)."""
    state = torch.load(path, map_location="cpu", weights_only=True)
    if state.get("format") != "h1w-gn-checkpoint-1":
        raise ValueError(f"{path}: not an h1w Gauss-Newton checkpoint")
    if tuple(state["m"].shape) != tuple(m.shape) or tuple(state["U"].shape) != tuple(U.shape):
        raise ValueError(f"{path}: checkpoint shapes {tuple(state['m'].shape)}, {tuple(state['U'].shape)} "
                         f"do not match m {tuple(m.shape)}, U {tuple(U.shape)}")
    m.copy_(state["m"])
    U.copy_(state["U"])
    hist = []
    for rec in state["hist"]:
        h = GnInfo()
        for f, _ in GnInfo._fields_:
            setattr(h, f, rec[f])
        hist.append(h)
    return int(state["step"]), hist


class Solver:
    """Owns a workspace tensor and a context for one grid (convenience wrapper).

    The library runs on the context's stream. When that is not the caller's current
    stream, every call first makes the context's stream wait for the current one (so
    inputs produced there, and the reuse of freed memory by the workspace, are ordered
    before the library's kernels), marks the tensors it hands over as used on the
    context's stream (so the caching allocator does not recycle them early), and
    afterwards makes the current stream wait for the context's stream (so the outputs
    are complete for whatever the caller runs next)."""

    def __init__(self, disc: int, n, h, alpha: float, m_max: int, device="cuda",
                 opt: Options | None = None, stream: torch.cuda.Stream | None = None):
        self.grid = make_grid(disc, n, h, alpha)
        self.N = 1
        for v in list(n):
            self.N *= int(v)
        self.m_max = int(m_max)
        size = h1w_workspace_size(self.grid, self.m_max, opt)
        if size == 0:
            raise H1wError(H1W_EINVAL, "invalid grid/options for h1w_workspace_size")
        self.workspace = torch.empty(size, dtype=torch.uint8, device=device)
        self.stream = stream or torch.cuda.current_stream(self.workspace.device)
        self._enter(self.workspace)
        self.ctx = h1w_setup(self.grid, self.m_max, opt, self.workspace, self.stream)
        self._leave()
        self.m = None
        self.J = None

    def _enter(self, *tensors) -> None:
        cur = torch.cuda.current_stream(self.stream.device)
        if cur != self.stream:
            self.stream.wait_stream(cur)
            for t in tensors:
                if t is not None and t.is_cuda:
                    t.record_stream(self.stream)

    def _leave(self) -> None:
        cur = torch.cuda.current_stream(self.stream.device)
        if cur != self.stream:
            cur.wait_stream(self.stream)

    def capacitance(self, J: torch.Tensor | None) -> None:
        m = 0 if J is None else int(J.shape[0])
        self.J = J  # keep the borrowed matrix alive
        self._enter(J)
        h1w_capacitance(self.ctx, m, J, self.N)
        self._leave()
        self.m = m

    def capacitance_from_host(self, J_host: torch.Tensor, J_dev: torch.Tensor) -> None:
        """Copies J_host (pinned) into J_dev while line H runs; J_dev becomes the borrowed J."""
        m = int(J_host.shape[0])
        self.J = J_dev
        self._enter(J_dev)
        h1w_capacitance_from_host(self.ctx, m, J_host, J_dev, self.N)
        self._leave()
        self.m = m

    def prefetch_J(self, J_host: torch.Tensor, J_dev: torch.Tensor) -> None:
        """Starts copying J_host (pinned) into J_dev for a later capacitance_from_host with the
        same pair (h1w_prefetch_J); the caller keeps both alive until then."""
        m = int(J_host.shape[0])
        if J_host.is_cuda or not J_host.is_pinned() or J_host.dtype != torch.float64 or not J_host.is_contiguous():
            raise ValueError("J_host must be a pinned, contiguous float64 CPU tensor")
        self._enter(J_dev)
        _check(load().h1w_prefetch_J(self.ctx, m, J_host.data_ptr(), _ptr(J_dev, m * self.N, "J_dev")), self.ctx)
        self._leave()

    def copy_profile(self, cap: int = 256):
        """Per-batch timeline of the last capacitance_from_host (h1w_get_copy_profile): a list of
        dicts with rows, copy_begin, copy_end, cycle_begin, cycle_end in ms from line H's start."""
        n = ctypes.c_int32()
        rows = (ctypes.c_int32 * cap)()
        arr = [(ctypes.c_float * cap)() for _ in range(4)]
        _check(load().h1w_get_copy_profile(self.ctx, cap, ctypes.byref(n), rows, *arr), self.ctx)
        keys = ("copy_begin", "copy_end", "cycle_begin", "cycle_end")
        return [dict(rows=int(rows[i]), **{k: float(a[i]) for k, a in zip(keys, arr)}) for i in range(min(n.value, cap))]

    def apply_prec(self, r, z=None):
        z = torch.empty_like(r) if z is None else z
        self._enter(r, z)
        h1w_apply_prec(self.ctx, r, z, self.N)
        self._leave()
        return z

    def apply_op(self, p, q=None):
        q = torch.empty_like(p) if q is None else q
        self._enter(p, q)
        h1w_apply_op(self.ctx, p, q, self.N)
        self._leave()
        return q

    def vcycle(self, b, x=None):
        nrhs = b.numel() // self.N
        x = torch.empty_like(b) if x is None else x
        self._enter(b, x)
        h1w_vcycle(self.ctx, nrhs, b, x, self.N)
        self._leave()
        return x

    def gn_rhs(self, dm, d):
        b = torch.empty_like(dm)
        self._enter(dm, d, b)
        h1w_gn_rhs(self.ctx, dm, d, b, self.N, self.m or 0)
        self._leave()
        return b

    def pcg(self, b, rtol: float, maxit: int = 500, x=None, raise_on_notconv=True):
        x = torch.empty_like(b) if x is None else x
        self._enter(b, x)
        try:
            info = h1w_pcg(self.ctx, b, x, rtol, maxit, self.N, raise_on_notconv)
        finally:
            self._leave()
        return x, info

    def pcg_host(self, b_host, x_host, rtol: float, maxit: int = 500, raise_on_notconv=True):
        """h1w_pcg_host: b_host in and x_host out (pinned CPU tensors), read and written by kernels."""
        self._enter()
        try:
            info = h1w_pcg_host(self.ctx, b_host, x_host, rtol, maxit, self.N, raise_on_notconv)
        finally:
            self._leave()
        return info

    def solve_direct(self, b, x=None):
        """x = (alpha (K + M) + J^T J)^-1 b by a dense Cholesky factorization (small grids;
        the J of the last capacitance call)."""
        size = int(load().h1w_direct_workspace_size(self.ctx))
        if size == 0:
            raise H1wError(H1W_EUNSUPPORTED, "grid too large for h1w_solve_direct")
        ws = torch.empty(size, dtype=torch.uint8, device=self.workspace.device)
        x = torch.empty_like(b) if x is None else x
        self._enter(b, x, ws)
        try:
            _check(load().h1w_solve_direct(self.ctx, _ptr(b, self.N, "b"), _ptr(x, self.N, "x"), ws.data_ptr(),
                                           ws.numel()), self.ctx)
        finally:
            self._leave()
        return x

    def ert_workspace(self, survey: Survey) -> torch.Tensor:
        size = h1w_ert_workspace_size(self.ctx, survey.n_e, survey.m)
        if size == 0:
            raise H1wError(H1W_EINVAL, "invalid survey size or grid for h1w_ert_workspace_size")
        return torch.empty(size, dtype=torch.uint8, device=self.workspace.device)

    def forward(self, survey: Survey, logsigma, rtol: float = 1e-10, maxit: int = 200, ws=None, U=None,
                warm: bool = False):
        """Pole fields U (n_e, N) and measurements g (m,) of the ERT model (h1w_forward);
        warm: start from the fields already in U."""
        ws = self.ert_workspace(survey) if ws is None else ws
        U = torch.empty((survey.n_e, self.N), dtype=torch.float64, device=logsigma.device) if U is None else U
        g = torch.empty(survey.m, dtype=torch.float64, device=logsigma.device)
        self._enter(logsigma, U, g, ws)
        try:
            info = h1w_forward(self.ctx, survey, logsigma, U, g, ws, rtol, maxit, self.N,
                               flags=H1W_FORWARD_WARM_START if warm else 0)
        finally:
            self._leave()
        return g, U, info

    def adjoint(self, survey: Survey, logsigma, U, r=None, rows: bool = False, ws=None):
        """J^T r (when r is given) and the rows of J (when rows) from the fields U (h1w_adjoint)."""
        ws = self.ert_workspace(survey) if ws is None else ws
        JTr = torch.empty(self.N, dtype=torch.float64, device=U.device) if r is not None else None
        J = torch.empty((survey.m, self.N), dtype=torch.float64, device=U.device) if rows else None
        self._enter(logsigma, U, r, JTr, J, ws)
        try:
            h1w_adjoint(self.ctx, survey, logsigma, U, r, JTr, J, ws, self.N)
        finally:
            self._leave()
        return JTr, J

    def gn_inversion(self, survey: Survey, g_obs, m_ref, m, steps: int, rtol_fwd: float = 1e-10,
                     rtol: float = 1e-8, maxit: int = 500, warm: bool = True, checkpoint: str | None = None):
        """Algorithm "Gauss-Newton with iterative solver": `steps` passes of h1w_gn_step
        from m (updated in place); from the second step on, each forward solve starts from
        the previous iterate's fields when warm. Returns the per-step GnInfo list and the
        last g, J.

        checkpoint: a file path. When it holds a checkpoint of an earlier call, the loop
        resumes from it (m, the fields and the step count; `steps` counts the steps already
        taken), and after every step the state is written there again (save_gn_checkpoint)."""
        dev = m.device
        ws = self.ert_workspace(survey)
        U = torch.empty((survey.n_e, self.N), dtype=torch.float64, device=dev)
        J = torch.empty((survey.m, self.N), dtype=torch.float64, device=dev)
        g = torch.empty(survey.m, dtype=torch.float64, device=dev)
        scratch = torch.empty(3 * self.N + survey.m, dtype=torch.float64, device=dev)
        self.J = J
        hist = []
        start = 0
        if checkpoint is not None and os.path.exists(checkpoint):
            start, hist = load_gn_checkpoint(checkpoint, m, U)
        self._enter(g_obs, m_ref, m, U, J, g, scratch, ws)
        try:
            for i in range(start, steps):
                flags = H1W_FORWARD_WARM_START if (warm and i > 0) else 0
                hist.append(h1w_gn_step(self.ctx, survey, g_obs, m_ref, m, U, J, g, scratch, ws, rtol_fwd, rtol,
                                        maxit, self.N, fwd_flags=flags))
                if checkpoint is not None:
                    torch.cuda.synchronize(dev)
                    save_gn_checkpoint(checkpoint, i + 1, m, U, hist)
        finally:
            self._leave()
        self.m = survey.m
        return hist, g, J

    def jvp(self, survey: Survey, logsigma, U, p, ws=None):
        """J p from the fields U without storing J (h1w_ert_jvp)."""
        ws = self.ert_workspace(survey) if ws is None else ws
        Jp = torch.empty(survey.m, dtype=torch.float64, device=U.device)
        self._enter(logsigma, U, p, Jp, ws)
        try:
            _check(load().h1w_ert_jvp(self.ctx, ctypes.byref(survey.c), _ptr(logsigma, self.N, "logsigma"),
                                      _ptr(U, self.N * survey.n_e, "U"), _ptr(p, self.N, "p"),
                                      _ptr(Jp, survey.m, "Jp"), ws.data_ptr(), ws.numel()), self.ctx)
        finally:
            self._leave()
        return Jp

    def factors(self):
        m = self.m or 0
        C = torch.empty((m, m), dtype=torch.float64, device=self.workspace.device)
        L = torch.empty_like(C)
        self._enter(C, L)
        h1w_capacitance_factors(self.ctx, C, L, m)
        self._leave()
        return C, L

    def cholesky(self, A):
        """Factors A in place on the context's stream (h1w_cholesky); returns A."""
        self._enter(A)
        try:
            h1w_cholesky(self.ctx, A)
        finally:
            self._leave()
        return A

    def set_pcg_mode(self, mode: int) -> None:
        """0: the PCG loop driven from the device (CUDA graph); 1: the host loop."""
        _check(load().h1w_set_pcg_mode(self.ctx, int(mode)), self.ctx)

    def inject_stall(self, kind: int, wait_limit_ns: int = 0) -> None:
        h1w_inject_stall(self.ctx, kind, wait_limit_ns)

    def timings(self) -> Timings:
        return h1w_get_timings(self.ctx)

    def levels(self):
        nl, _ = h1w_level_info(self.ctx, 0)
        return [h1w_level_info(self.ctx, l)[1] for l in range(nl)]

    def close(self):
        if getattr(self, "ctx", None):
            h1w_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class ErtForward(torch.autograd.Function):
    """g = ERT measurements of logsigma (h1w_forward); the backward pass is J^T grad_g
    (h1w_adjoint), formed from the saved pole fields without storing J."""

    @staticmethod
    def forward(ctx, logsigma, solver: Solver, survey: Survey, rtol: float = 1e-10, maxit: int = 200):
        ls = logsigma.detach().contiguous()
        g, U, _ = solver.forward(survey, ls, rtol=rtol, maxit=maxit)
        ctx.solver, ctx.survey = solver, survey
        ctx.save_for_backward(ls, U)
        return g

    @staticmethod
    def backward(ctx, grad_g):
        ls, U = ctx.saved_tensors
        JTr, _ = ctx.solver.adjoint(ctx.survey, ls, U, r=grad_g.detach().contiguous())
        return JTr, None, None, None, None
