"""GPU-resident refactorization + FGMRES solver for same-pattern KKT sequences
on B300 (sm_103a), after arXiv 2401.13926.

Thin ctypes binding over the C ABI of ``libkkt_b300.so`` (include/kkt.h):
argument marshalling only -- every numeric step runs in the library's CUDA
kernels.  Arrays may be numpy arrays (host memory) or CUDA tensors
(device memory, passed by ``data_ptr()``); PyTorch is only plumbing.

There is no CPU fallback: if the library is missing or cannot load, every
call raises.
"""
from __future__ import annotations

import ctypes as C
import os

import numpy as np

__all__ = ["KKTSolver", "KKTServer", "KKTBatch", "KKTError", "order", "pivot", "host_analyze", "lib", "LIB_PATH", "EXPORTS"]

LIB_PATH = os.path.join(os.path.dirname(os.path.abspath(__file__)), "libkkt_b300.so")

OK = 0
ERR = {
    -1: "INVALID", -2: "PATTERN", -3: "OOM", -4: "ZERO_PIVOT", -5: "NONFINITE",
    -6: "NOT_CONVERGED", -7: "TIMEOUT", -8: "CUDA", -9: "STATE",
}
ERR_NOT_CONVERGED = -6
STOP = {"nrbe": 0, "rr": 1}
TRSV = {"auto": 0, "global": 1}
PRECISION = {"fp64": 0, "mixed": 1}
METHOD = {"fgmres": 0, "richardson": 1, "fgmres_ee": 2}
ORTHO = {"cgs2": 0, "cgs2_pythagoras": 1, "cgs1_pythagoras": 2}
ROW_ORDER = {"row": 0, "level": 1, "critical": 2}

# every entry point declared in include/kkt.h
EXPORTS = [
    "kkt_default_opts", "kkt_create", "kkt_analyze", "kkt_refactor", "kkt_solve", "kkt_lu_solve",
    "kkt_matvec", "kkt_get_perm", "kkt_get_factor_sizes", "kkt_get_factors", "kkt_query",
    "kkt_destroy", "kkt_strerror", "kkt_last_error_detail", "kkt_order", "kkt_pivot",
    "kkt_get_phase_times", "kkt_lu_solve_noalloc", "kkt_selftest_wait", "kkt_trace_refactor",
    "kkt_trace_solve", "kkt_repivot", "kkt_tune", "kkt_step", "kkt_server_default_opts", "kkt_server_create", "kkt_server_open",
    "kkt_server_submit", "kkt_server_wait", "kkt_server_close", "kkt_server_query", "kkt_server_destroy",
    "kkt_host_analyze", "kkt_analyze_like", "kkt_trace_critical_path",
    "kkt_batch_create", "kkt_batch_destroy", "kkt_batch_step", "kkt_batch_launches", "kkt_batch_phase_times",
    "kkt_estimate_device_bytes", "kkt_place_instance",
]
NOALLOC_MAX_N = 65536
PHASES = ["gather", "refactor", "lsolve", "usolve", "spmv", "ortho", "update", "reserved", "graph_refactor",
          "graph_solve"]


class _Opts(C.Structure):
    _fields_ = [
        ("restart", C.c_int), ("max_cycles", C.c_int), ("stop_mode", C.c_int), ("precision", C.c_int),
        ("refine_delta", C.c_double), ("pivot_tol", C.c_double), ("boost_eps", C.c_double),
        ("device", C.c_int), ("create_stream", C.c_int), ("stream", C.c_void_p), ("spin_limit", C.c_int64),
        ("timing", C.c_int), ("trisolve", C.c_int), ("cluster_blocks", C.c_int), ("block_smem", C.c_int),
        ("method", C.c_int), ("ortho", C.c_int), ("inner_tol", C.c_double), ("repivot", C.c_int),
        ("graphs", C.c_int), ("warp_rows", C.c_int), ("row_order", C.c_int),
        ("warp_row_updates", C.c_int64), ("mixed_fallback", C.c_int),
        ("stream_last", C.c_int), ("team_rows", C.c_int), ("equilibrate", C.c_int),
    ]


class _Info(C.Structure):
    _fields_ = [
        ("n", C.c_int32), ("nnz_a", C.c_int64), ("nnz_l", C.c_int64), ("nnz_u", C.c_int64),
        ("levels_l", C.c_int32), ("levels_u", C.c_int32), ("refactor_updates", C.c_double),
        ("device_bytes", C.c_int64), ("nboost", C.c_int32), ("last_iters", C.c_int32),
        ("last_cycles", C.c_int32), ("trisolve_cluster", C.c_int32), ("last_nrbe", C.c_double), ("last_rnorm0", C.c_double),
        ("norm_a_inf", C.c_double), ("analyze_ms", C.c_double), ("launches", C.c_int64),
        ("h2d_bytes", C.c_int64), ("d2h_bytes", C.c_int64), ("repivots", C.c_int32), ("rows_warp", C.c_int32),
        ("rows_block", C.c_int32), ("rows_global", C.c_int32), ("refactor_smem", C.c_int32),
        ("refactor_threads", C.c_int32), ("refactor_blocks", C.c_int32), ("last_fallback", C.c_int32),
        ("fallbacks", C.c_int64), ("rows_team", C.c_int32),
    ]


SERVER_MAX_DEVICES = 16


class _ServerOpts(C.Structure):
    _fields_ = [("workers", C.c_int), ("hbm_budget", C.c_int64), ("opts", _Opts), ("batch", C.c_int),
                ("ndevices", C.c_int), ("devices", C.c_int * SERVER_MAX_DEVICES)]


class _StepResult(C.Structure):
    _fields_ = [("status", C.c_int), ("iters", C.c_int32), ("nrbe", C.c_double), ("queue_ms", C.c_double),
                ("run_ms", C.c_double), ("batch_size", C.c_int32), ("device", C.c_int32)]


class _ServerInfo(C.Structure):
    _fields_ = [("instances", C.c_int32), ("device_bytes", C.c_int64), ("hbm_budget", C.c_int64),
                ("submitted", C.c_int64), ("completed", C.c_int64), ("in_flight", C.c_int32),
                ("waiting", C.c_int32), ("batches", C.c_int64), ("ndevices", C.c_int32)]


class _HostStats(C.Structure):
    _fields_ = [("nnz_l", C.c_int64), ("nnz_u", C.c_int64), ("levels_l", C.c_int32), ("levels_u", C.c_int32),
                ("refactor_updates", C.c_double), ("order_ms", C.c_double), ("pivot_ms", C.c_double),
                ("canonical_order", C.c_int32)]


class KKTError(RuntimeError):
    def __init__(self, code, where, detail=""):
        super().__init__(f"{where}: KKT_ERR_{ERR.get(code, code)} ({code}) {detail}".strip())
        self.code = code


_lib = None


def lib():
    """Load libkkt_b300.so (raises if it is missing: there is no fallback)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError(f"{LIB_PATH} is missing; build it with `python -m paper_2401_13926_b300.build`")
    L = C.CDLL(LIB_PATH)
    vp, i32, i64, d, ip = C.c_void_p, C.c_int32, C.c_int64, C.c_double, C.c_int
    L.kkt_default_opts.argtypes = [C.POINTER(_Opts)]
    L.kkt_default_opts.restype = None
    L.kkt_create.argtypes = [C.POINTER(vp), C.POINTER(_Opts)]
    L.kkt_analyze.argtypes = [vp, i32, vp, vp, vp, vp, vp]
    L.kkt_refactor.argtypes = [vp, vp, ip]
    L.kkt_solve.argtypes = [vp, vp, vp, ip, d, C.POINTER(C.c_int), C.POINTER(d)]
    L.kkt_lu_solve.argtypes = [vp, vp, vp, ip]
    L.kkt_matvec.argtypes = [vp, vp, vp, ip]
    L.kkt_get_perm.argtypes = [vp, vp, vp]
    L.kkt_get_factor_sizes.argtypes = [vp, C.POINTER(i64), C.POINTER(i64)]
    L.kkt_get_factors.argtypes = [vp, vp, vp, vp, vp, vp, vp]
    L.kkt_query.argtypes = [vp, C.POINTER(_Info)]
    L.kkt_destroy.argtypes = [vp]
    L.kkt_destroy.restype = None
    L.kkt_strerror.argtypes = [ip]
    L.kkt_strerror.restype = C.c_char_p
    L.kkt_last_error_detail.argtypes = [vp]
    L.kkt_last_error_detail.restype = C.c_char_p
    L.kkt_order.argtypes = [i32, vp, vp, vp]
    L.kkt_pivot.argtypes = [i32, vp, vp, vp, vp, d, vp, C.POINTER(i64), C.POINTER(i64)]
    L.kkt_get_phase_times.argtypes = [vp, vp, vp, ip]
    L.kkt_lu_solve_noalloc.argtypes = [i32, vp, vp, vp, vp, vp, vp, vp, vp, vp]
    L.kkt_selftest_wait.argtypes = [vp, i64]
    L.kkt_trace_refactor.argtypes = [vp, vp, ip, vp, vp, C.POINTER(i32)]
    L.kkt_trace_solve.argtypes = [vp, vp, vp, ip, vp, vp, vp, vp]
    L.kkt_repivot.argtypes = [vp, vp, ip]
    L.kkt_tune.argtypes = [vp, vp, vp, ip, ip, C.POINTER(d)]
    L.kkt_step.argtypes = [vp, vp, vp, vp, ip, d, C.POINTER(C.c_int), C.POINTER(d)]
    L.kkt_server_default_opts.argtypes = [C.POINTER(_ServerOpts)]
    L.kkt_server_default_opts.restype = None
    L.kkt_server_create.argtypes = [C.POINTER(vp), C.POINTER(_ServerOpts)]
    L.kkt_server_open.argtypes = [vp, i32, vp, vp, vp, C.POINTER(i64)]
    L.kkt_server_submit.argtypes = [vp, i64, vp, vp, vp, d, C.POINTER(i64)]
    L.kkt_server_wait.argtypes = [vp, i64, C.POINTER(_StepResult)]
    L.kkt_server_close.argtypes = [vp, i64]
    L.kkt_server_query.argtypes = [vp, C.POINTER(_ServerInfo)]
    L.kkt_server_destroy.argtypes = [vp]
    L.kkt_server_destroy.restype = None
    L.kkt_host_analyze.argtypes = [i32, vp, vp, vp, d, vp, vp, C.POINTER(_HostStats)]
    L.kkt_analyze_like.argtypes = [vp, vp]
    L.kkt_trace_critical_path.argtypes = [vp, vp, vp, C.POINTER(d), C.POINTER(i32), C.POINTER(d), C.POINTER(i32)]
    L.kkt_batch_create.argtypes = [C.POINTER(vp), ip, ip]
    L.kkt_batch_destroy.argtypes = [vp]
    L.kkt_batch_destroy.restype = None
    L.kkt_batch_step.argtypes = [vp, vp, ip, vp, vp, vp, ip, d, vp, vp, vp]
    L.kkt_batch_launches.argtypes = [vp]
    L.kkt_batch_phase_times.argtypes = [vp, vp, vp, C.c_int]
    L.kkt_estimate_device_bytes.argtypes = [i32, i64, C.POINTER(_HostStats), C.POINTER(_Opts), ip, C.POINTER(i64)]
    L.kkt_place_instance.argtypes = [ip, vp, vp, i64]
    for name in EXPORTS:
        if name not in ("kkt_default_opts", "kkt_destroy", "kkt_strerror", "kkt_last_error_detail",
                        "kkt_server_default_opts", "kkt_server_destroy", "kkt_batch_destroy"):
            getattr(L, name).restype = C.c_int
    L.kkt_batch_launches.restype = C.c_int64
    _lib = L
    return L


def _torch_current_stream(device):
    """torch's current stream on `device`, if torch has CUDA; device tensors
    made by torch are then ordered with the solver's kernels."""
    try:
        import torch
        if torch.cuda.is_available():
            return torch.cuda.current_stream(device)
    except Exception:
        pass
    return None


def _host(a, dtype):
    a = np.ascontiguousarray(a, dtype=dtype)
    return a, a.ctypes.data


def _is_device(a):
    return hasattr(a, "data_ptr") and getattr(a, "is_cuda", False)


def _ptr(a, dtype):
    """(keepalive, pointer, on_device) for a numpy array or a CUDA tensor."""
    if _is_device(a):
        if not a.is_contiguous():
            raise ValueError("device arrays must be contiguous")
        return a, a.data_ptr(), 1
    h, p = _host(a, dtype)
    return h, p, 0


def order(rowptr, colind):
    """Column order Q of kkt_analyze (approximate minimum degree on K^T K)."""
    L = lib()
    rp, prp = _host(rowptr, np.int32)
    ci, pci = _host(colind, np.int32)
    n = len(rp) - 1
    Q = np.zeros(n, np.int32)
    rc = L.kkt_order(n, prp, pci, Q.ctypes.data)
    if rc:
        raise KKTError(rc, "kkt_order")
    return Q


def pivot(rowptr, colind, values, Q=None, tol=1e-3):
    """Host threshold-pivoting factorization: (P, nnz_l, nnz_u)."""
    L = lib()
    rp, prp = _host(rowptr, np.int32)
    ci, pci = _host(colind, np.int32)
    v, pv = _host(values, np.float64)
    n = len(rp) - 1
    q = None if Q is None else np.ascontiguousarray(Q, np.int32)
    P = np.zeros(n, np.int32)
    nl, nu = C.c_int64(), C.c_int64()
    rc = L.kkt_pivot(n, prp, pci, pv, None if q is None else q.ctypes.data, float(tol), P.ctypes.data,
                     C.byref(nl), C.byref(nu))
    if rc:
        raise KKTError(rc, "kkt_pivot")
    return P, nl.value, nu.value


def host_analyze(rowptr, colind, values0, pivot_tol=1e-3):
    """kkt_host_analyze: the analysis of kkt_analyze on the host only (no
    GPU) -- returns (P, Q, stats) with stats the structure's statistics."""
    L = lib()
    rp, prp = _host(rowptr, np.int32)
    ci, pci = _host(colind, np.int32)
    v, pv = _host(values0, np.float64)
    n = len(rp) - 1
    P = np.zeros(n, np.int32)
    Q = np.zeros(n, np.int32)
    st = _HostStats()
    rc = L.kkt_host_analyze(n, prp, pci, pv, float(pivot_tol), P.ctypes.data, Q.ctypes.data, C.byref(st))
    if rc:
        raise KKTError(rc, "kkt_host_analyze")
    return P, Q, {k: getattr(st, k) for k, _ in _HostStats._fields_}


def estimate_device_bytes(n, nnz, stats, canonical_order=True, **solver_opts):
    """kkt_estimate_device_bytes: device memory kkt_analyze will hold for a
    pattern with these host_analyze() statistics and solver options."""
    st = _HostStats()
    for k, _ in _HostStats._fields_:
        setattr(st, k, stats[k])
    o = _solver_opts(**solver_opts)
    out = C.c_int64()
    rc = lib().kkt_estimate_device_bytes(int(n), int(nnz), C.byref(st), C.byref(o), int(bool(canonical_order)),
                                         C.byref(out))
    if rc:
        raise KKTError(rc, "kkt_estimate_device_bytes")
    return out.value


def place_instance(budget, held, need):
    """kkt_place_instance: device index for a new instance (most budget left
    among devices whose budget can hold it), or -1."""
    b = np.ascontiguousarray(budget, np.int64)
    h = np.ascontiguousarray(held, np.int64)
    return lib().kkt_place_instance(len(b), b.ctypes.data, h.ctypes.data, int(need))


def lu_solve_noalloc(Fp, Fj, Fdiag, Fx, P, Q, b, x, stream=None):
    """kkt_lu_solve_noalloc: x = Q U^{-1} L^{-1} P b from caller-held device
    factors in the combined row layout, with no device allocation (for
    callers whose device memory is owned elsewhere).  All arguments are
    CUDA tensors; n = len(b) <= NOALLOC_MAX_N."""
    if stream is None:
        stream = _torch_current_stream(b.device.index)
    st = int(getattr(stream, "cuda_stream", stream or 0)) or None
    n = int(b.numel())
    rc = lib().kkt_lu_solve_noalloc(n, Fp.data_ptr(), Fj.data_ptr(), Fdiag.data_ptr(), Fx.data_ptr(),
                                    P.data_ptr(), Q.data_ptr(), b.data_ptr(), x.data_ptr(), st)
    if rc:
        raise KKTError(rc, "kkt_lu_solve_noalloc")
    return x


def _solver_opts(restart=20, max_cycles=50, stop_mode="nrbe", refine_delta=0.0, pivot_tol=1e-3, boost_eps=0.0,
                 device=0, spin_limit=0, timing=False, trisolve="auto", block_smem=0, cluster_blocks=0,
                 precision="fp64", method="fgmres", ortho="cgs2", inner_tol=1e-6, repivot=False, graphs=False,
                 warp_rows=True, row_order="level", mixed_fallback=2, warp_row_updates=0, stream_last=True,
                 team_rows=True, equilibrate=False):
    """kkt_opts from keyword arguments (defaults of kkt_default_opts)."""
    o = _Opts()
    lib().kkt_default_opts(C.byref(o))
    o.restart, o.max_cycles, o.stop_mode = int(restart), int(max_cycles), STOP[stop_mode]
    o.refine_delta, o.pivot_tol, o.boost_eps = float(refine_delta), float(pivot_tol), float(boost_eps)
    o.device, o.spin_limit, o.timing = int(device), int(spin_limit), int(bool(timing))
    o.trisolve = TRSV[trisolve]
    o.block_smem = int(block_smem)
    o.cluster_blocks = int(cluster_blocks)
    o.precision = PRECISION[precision]
    o.method, o.ortho, o.inner_tol = METHOD[method], ORTHO[ortho], float(inner_tol)
    o.repivot = int(bool(repivot))
    o.graphs = int(bool(graphs))
    o.warp_rows = int(bool(warp_rows))
    o.row_order = ROW_ORDER[row_order]
    o.mixed_fallback = int(mixed_fallback)
    o.warp_row_updates = int(warp_row_updates)
    o.stream_last = int(bool(stream_last))
    o.team_rows = int(bool(team_rows))
    o.equilibrate = int(bool(equilibrate))
    return o


class KKTSolver:
    """One solver context: analyze once per pattern, then refactor + solve for
    every matrix of the sequence (Sections 1.3 and 2.1)."""

    def __init__(self, restart=20, max_cycles=50, stop_mode="nrbe", refine_delta=0.0, pivot_tol=1e-3,
                 boost_eps=0.0, device=0, stream=None, spin_limit=0, timing=False, trisolve="auto",
                 block_smem=0, cluster_blocks=0, precision="fp64", method="fgmres", ortho="cgs2",
                 inner_tol=1e-6, repivot=False, graphs=False, warp_rows=True, row_order="level",
                 mixed_fallback=2, warp_row_updates=0, stream_last=True, team_rows=True, equilibrate=False):
        L = lib()
        o = _solver_opts(restart, max_cycles, stop_mode, refine_delta, pivot_tol, boost_eps, device, spin_limit,
                         timing, trisolve, block_smem, cluster_blocks, precision, method, ortho, inner_tol, repivot,
                         graphs, warp_rows, row_order, mixed_fallback, warp_row_updates, stream_last, team_rows,
                         equilibrate)
        if stream is None:
            stream = _torch_current_stream(device)
        if stream is None:
            o.create_stream, o.stream = 1, None
        else:   # order every device operation with the caller's (torch's) stream
            o.create_stream, o.stream = 0, int(getattr(stream, "cuda_stream", stream)) or None
        h = C.c_void_p()
        rc = L.kkt_create(C.byref(h), C.byref(o))
        if rc:
            raise KKTError(rc, "kkt_create")
        self._h = h
        self.n = 0
        self.nnz = 0

    def _check(self, rc, where, ok=(OK,)):
        if rc not in ok:
            raise KKTError(rc, where, lib().kkt_last_error_detail(self._h).decode())
        return rc

    def close(self):
        if getattr(self, "_h", None):
            lib().kkt_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def analyze(self, rowptr, colind, values0=None, Q=None, P=None):
        rp, prp = _host(rowptr, np.int32)
        ci, pci = _host(colind, np.int32)
        v = None if values0 is None else _host(values0, np.float64)
        q = None if Q is None else _host(Q, np.int32)
        p = None if P is None else _host(P, np.int32)
        n = len(rp) - 1
        self._check(lib().kkt_analyze(self._h, n, prp, pci, v[1] if v else None, q[1] if q else None,
                                      p[1] if p else None), "kkt_analyze")
        self.n, self.nnz = n, int(rp[-1])
        return self

    def analyze_like(self, other):
        """kkt_analyze_like: reuse another context's analysis (same pattern,
        P, Q and structure) for this context's options."""
        self._check(lib().kkt_analyze_like(self._h, other._h), "kkt_analyze_like")
        self.n, self.nnz = other.n, other.nnz
        return self

    def refactor(self, values):
        keep, p, dev = _ptr(values, np.float64)
        self._check(lib().kkt_refactor(self._h, p, dev), "kkt_refactor")

    def tune(self, values, b, reps=3):
        """kkt_tune: pick the fastest refactorization/solve schedule for this
        matrix (same bits either way); returns the chosen ms of refactor +
        lu_solve.  Refactor again afterwards."""
        kv, pv, dev = _ptr(values, np.float64)
        kb, pb, devb = _ptr(b, np.float64)
        if dev != devb:
            raise ValueError("values and b must both be host or both be device arrays")
        best = C.c_double()
        self._check(lib().kkt_tune(self._h, pv, pb, dev, int(reps), C.byref(best)), "kkt_tune")
        return best.value

    def repivot(self, values):
        """kkt_repivot: pivoting factorization of `values` on the host (Q
        kept), new device layout, then the GPU refactorization."""
        keep, p, dev = _ptr(values, np.float64)
        self._check(lib().kkt_repivot(self._h, p, dev), "kkt_repivot")

    def solve(self, b, x=None, tol=1e-12, allow_not_converged=False):
        """Returns (x, iters, nrbe).  x is written in place when given."""
        kb, pb, dev = _ptr(b, np.float64)
        if x is None:
            x = b.new_empty(self.n) if dev else np.zeros(self.n)
        kx, px, devx = _ptr(x, np.float64)
        if devx != dev:
            raise ValueError("b and x must both be host or both be device arrays")
        it, nr = C.c_int(), C.c_double()
        ok = (OK, ERR_NOT_CONVERGED) if allow_not_converged else (OK,)
        rc = self._check(lib().kkt_solve(self._h, pb, px, dev, float(tol), C.byref(it), C.byref(nr)), "kkt_solve", ok)
        self.last_status = rc
        return x, it.value, nr.value

    def step(self, values, b, x=None, tol=1e-12, allow_not_converged=False):
        """kkt_step: refactor(values) + solve(b) with the forward sweep fused
        into the refactorization.  Returns (x, iters, nrbe)."""
        kv, pv, dv = _ptr(values, np.float64)
        kb, pb, db = _ptr(b, np.float64)
        if dv != db:
            raise ValueError("values and b must both be host or both be device arrays")
        if x is None:
            x = b.new_empty(self.n) if db else np.zeros(self.n)
        kx, px, _ = _ptr(x, np.float64)
        it, nr = C.c_int(), C.c_double()
        ok = (OK, ERR_NOT_CONVERGED) if allow_not_converged else (OK,)
        rc = self._check(lib().kkt_step(self._h, pv, pb, px, db, float(tol), C.byref(it), C.byref(nr)), "kkt_step", ok)
        self.last_status = rc
        return x, it.value, nr.value

    def lu_solve(self, b, x=None):
        kb, pb, dev = _ptr(b, np.float64)
        if x is None:
            x = b.new_empty(self.n) if dev else np.zeros(self.n)
        kx, px, _ = _ptr(x, np.float64)
        self._check(lib().kkt_lu_solve(self._h, pb, px, dev), "kkt_lu_solve")
        return x

    def matvec(self, x, y=None):
        kx, px, dev = _ptr(x, np.float64)
        if y is None:
            y = x.new_empty(self.n) if dev else np.zeros(self.n)
        ky, py, _ = _ptr(y, np.float64)
        self._check(lib().kkt_matvec(self._h, px, py, dev), "kkt_matvec")
        return y

    def perm(self):
        P = np.zeros(self.n, np.int32)
        Q = np.zeros(self.n, np.int32)
        self._check(lib().kkt_get_perm(self._h, P.ctypes.data, Q.ctypes.data), "kkt_get_perm")
        return P, Q

    def factors(self):
        """Host CSC copies: (Lp, Li, Lx) strictly lower, (Up, Ui, Ux) with diagonal."""
        nl, nu = C.c_int64(), C.c_int64()
        self._check(lib().kkt_get_factor_sizes(self._h, C.byref(nl), C.byref(nu)), "kkt_get_factor_sizes")
        n = self.n
        Lp, Up = np.zeros(n + 1, np.int64), np.zeros(n + 1, np.int64)
        Li, Lx = np.zeros(max(nl.value, 1), np.int32), np.zeros(max(nl.value, 1))
        Ui, Ux = np.zeros(max(nu.value, 1), np.int32), np.zeros(max(nu.value, 1))
        self._check(lib().kkt_get_factors(self._h, Lp.ctypes.data, Li.ctypes.data, Lx.ctypes.data,
                                          Up.ctypes.data, Ui.ctypes.data, Ux.ctypes.data), "kkt_get_factors")
        return dict(Lp=Lp, Li=Li[:nl.value], Lx=Lx[:nl.value], Up=Up, Ui=Ui[:nu.value], Ux=Ux[:nu.value])

    def phase_times(self, reset=False):
        """{phase: (ms, launches)} accumulated by the library's CUDA events."""
        ms = np.zeros(len(PHASES))
        cnt = np.zeros(len(PHASES), np.int64)
        self._check(lib().kkt_get_phase_times(self._h, ms.ctypes.data, cnt.ctypes.data, int(bool(reset))),
                    "kkt_get_phase_times")
        return {p: (float(ms[i]), int(cnt[i])) for i, p in enumerate(PHASES)}

    def trace_solve(self, b):
        """kkt_lu_solve with per-row publish stamps (ns) of both sweeps
        (cluster schedule): (x, listL, tL, listU, tU), t* indexed by list
        position."""
        kb, pb, dev = _ptr(b, np.float64)
        n = self.n
        x = b.new_empty(n) if dev else np.zeros(n)
        kx, px, _ = _ptr(x, np.float64)
        lL, lU = np.zeros(n, np.int32), np.zeros(n, np.int32)
        tL, tU = np.zeros(n, np.int64), np.zeros(n, np.int64)
        self._check(lib().kkt_trace_solve(self._h, pb, px, dev, lL.ctypes.data, lU.ctypes.data,
                                          tL.ctypes.data, tU.ctypes.data), "kkt_trace_solve")
        return x, lL, tL, lU, tU

    def trace_refactor(self, values):
        """kkt_refactor with per-row start/publish stamps (ns) of every row:
        (t_start, t_publish, t0 = 0)."""
        keep, p, dev = _ptr(values, np.float64)
        ts = np.zeros(self.n, np.int64)
        tp = np.zeros(self.n, np.int64)
        t0 = C.c_int32()
        self._check(lib().kkt_trace_refactor(self._h, p, dev, ts.ctypes.data, tp.ctypes.data, C.byref(t0)),
                    "kkt_trace_refactor")
        return ts, tp, t0.value

    def critical_path(self, t_start, t_publish):
        """kkt_trace_critical_path on trace_refactor's stamps: dict with the
        longest path of per-row links (ms), the DAG depth, the median link
        (us) and the stamped rows."""
        ts = np.ascontiguousarray(t_start, np.int64)
        tp = np.ascontiguousarray(t_publish, np.int64)
        path, med = C.c_double(), C.c_double()
        lev, rows = C.c_int32(), C.c_int32()
        self._check(lib().kkt_trace_critical_path(self._h, ts.ctypes.data, tp.ctypes.data, C.byref(path),
                                                  C.byref(lev), C.byref(med), C.byref(rows)),
                    "kkt_trace_critical_path")
        return {"path_ms": path.value * 1e-6, "levels": lev.value, "median_link_us": med.value * 1e-3,
                "rows_stamped": rows.value}

    def selftest_wait(self, limit):
        """Return code of kkt_selftest_wait (KKT_ERR_TIMEOUT = -7 expected)."""
        return lib().kkt_selftest_wait(self._h, int(limit))

    def info(self):
        inf = _Info()
        self._check(lib().kkt_query(self._h, C.byref(inf)), "kkt_query")
        return {k: getattr(inf, k) for k, _ in _Info._fields_}


class KKTBatch:
    """kkt_batch_*: one step of several KKTSolver instances in shared
    launches (one refactorization launch over every instance's rows, one
    cluster launch for their backward sweeps).  step() returns per-instance
    (x, iters, nrbe, status)."""

    def __init__(self, max_count, device=0):
        h = C.c_void_p()
        rc = lib().kkt_batch_create(C.byref(h), int(max_count), int(device))
        if rc:
            raise KKTError(rc, "kkt_batch_create")
        self._h = h
        self.max_count = int(max_count)

    def step(self, solvers, values, bs, xs=None, tol=1e-12):
        """values, bs (and xs): lists of numpy arrays (host) or of CUDA
        tensors (device), one per solver."""
        k = len(solvers)
        dev = _is_device(values[0])
        if xs is None:
            xs = [b.new_empty(s.n) if dev else np.zeros(s.n) for s, b in zip(solvers, bs)]
        keep = []
        def ptrs(arrs):
            out = (C.c_void_p * k)()
            for i, a in enumerate(arrs):
                kk, p, d_ = _ptr(a, np.float64)
                if d_ != dev:
                    raise ValueError("all arrays must be host arrays or all device arrays")
                keep.append(kk)
                out[i] = p
            return out
        pv, pb, px = ptrs(values), ptrs(bs), ptrs(xs)
        ctxs = (C.c_void_p * k)(*[s._h.value for s in solvers])
        it = np.zeros(k, np.int32)
        nr = np.zeros(k)
        st = np.zeros(k, np.int32)
        rc = lib().kkt_batch_step(self._h, ctxs, k, pv, pb, px, int(dev), float(tol), it.ctypes.data,
                                  nr.ctypes.data, st.ctypes.data)
        if rc:
            raise KKTError(rc, "kkt_batch_step")
        return xs, it, nr, st

    def launches(self):
        return lib().kkt_batch_launches(self._h)

    def phase_times(self, reset=False):
        """kkt_batch_phase_times: ({phase: ms}, instance-steps) of the shared
        launches since creation or the last reset."""
        ms = np.zeros(6)
        steps = C.c_int64()
        rc = lib().kkt_batch_phase_times(self._h, ms.ctypes.data, C.byref(steps), int(bool(reset)))
        if rc:
            raise KKTError(rc, "kkt_batch_phase_times")
        names = ("copies", "gather", "refactor", "usolve", "residual", "refine_host")
        return {k: float(v) for k, v in zip(names, ms)}, steps.value

    def close(self):
        if getattr(self, "_h", None):
            lib().kkt_batch_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class KKTServer:
    """Many resident KKT sequences on one or more GPUs with their steps in
    flight together (kkt_server_*): open() admits an instance (host analysis
    in the calling thread, placement on the device with the most budget
    left, then -- waiting in arrival order until its device memory fits --
    its device buffers), submit() queues a refactor + solve step (host
    arrays; x is written when the step completes), wait() returns its
    result.  batch > 0: up to `batch` queued steps of different instances
    run as one batched call (continuous batching); batch = 0: one worker
    thread per step.  Steps of one instance run in order."""

    def __init__(self, workers=8, hbm_budget=0, batch=8, devices=None, **solver_opts):
        L = lib()
        o = _ServerOpts()
        L.kkt_server_default_opts(C.byref(o))
        o.workers, o.hbm_budget, o.batch = int(workers), int(hbm_budget), int(batch)
        if devices:
            o.ndevices = len(devices)
            for i, d in enumerate(devices):
                o.devices[i] = int(d)
        o.opts = _solver_opts(**solver_opts)
        h = C.c_void_p()
        rc = L.kkt_server_create(C.byref(h), C.byref(o))
        if rc:
            raise KKTError(rc, "kkt_server_create")
        self._h = h
        self._n = {}
        self._keep = {}

    def open(self, rowptr, colind, values0):
        rp, prp = _host(rowptr, np.int32)
        ci, pci = _host(colind, np.int32)
        v, pv = _host(values0, np.float64)
        inst = C.c_int64()
        rc = lib().kkt_server_open(self._h, len(rp) - 1, prp, pci, pv, C.byref(inst))
        if rc:
            raise KKTError(rc, "kkt_server_open")
        self._n[inst.value] = len(rp) - 1
        return inst.value

    def submit(self, instance, values, b, tol=1e-12):
        """Returns (ticket, x); x is filled when the step completes."""
        v, pv = _host(values, np.float64)
        bb, pb = _host(b, np.float64)
        x = np.zeros(self._n[instance])
        t = C.c_int64()
        rc = lib().kkt_server_submit(self._h, int(instance), pv, pb, x.ctypes.data, float(tol), C.byref(t))
        if rc:
            raise KKTError(rc, "kkt_server_submit")
        self._keep[t.value] = x
        return t.value, x

    def wait(self, ticket):
        r = _StepResult()
        rc = lib().kkt_server_wait(self._h, int(ticket), C.byref(r))
        if rc:
            raise KKTError(rc, "kkt_server_wait")
        x = self._keep.pop(ticket)
        return x, {k: getattr(r, k) for k, _ in _StepResult._fields_}

    def close_instance(self, instance):
        rc = lib().kkt_server_close(self._h, int(instance))
        if rc:
            raise KKTError(rc, "kkt_server_close")
        self._n.pop(instance, None)

    def info(self):
        i = _ServerInfo()
        lib().kkt_server_query(self._h, C.byref(i))
        return {k: getattr(i, k) for k, _ in _ServerInfo._fields_}

    def close(self):
        if getattr(self, "_h", None):
            lib().kkt_server_destroy(self._h)
            self._h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
