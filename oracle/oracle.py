"""Python front end of the CPU FP64 oracle (oracle.c).

TEST INFRASTRUCTURE ONLY: imported by the tests, by the smoke check and by
the benchmark's CPU-baseline leg.  The solver package never imports it.

Every function takes plain numpy arrays.  Matrices are given as CSR
(rowptr, colind, values) of the full K (both triangles); the CSC copy the
factorization needs is a transpose-by-counting done here in numpy.

Permutation convention (same as oracle.c): B = A(P, Q) = L U, with
B[i, j] = A[P[i], Q[j]]; L unit lower (diagonal not stored), U upper with the
diagonal; both CSC, row indices permuted and sorted.
"""
from __future__ import annotations

import ctypes as C
import dataclasses
import numpy as np

from . import build as _build

_lib = None

OK, ERR_PATTERN, ERR_OOM, ERR_SINGULAR, ERR_NONFINITE, ERR_NOT_CONVERGED = 0, -2, -3, -4, -5, -6

_i32 = np.ctypeslib.ndpointer(np.int32, flags="C_CONTIGUOUS")
_f64 = np.ctypeslib.ndpointer(np.float64, flags="C_CONTIGUOUS")


def lib():
    global _lib
    if _lib is None:
        L = C.CDLL(_build.build())
        L.or_lu.restype = C.c_void_p
        L.or_lu.argtypes = [C.c_int, _i32, _i32, _f64, _i32, C.c_double, _i32, C.POINTER(C.c_int)]
        L.or_refactor.restype = C.c_void_p
        L.or_refactor.argtypes = [C.c_int, _i32, _i32, _f64, _i32, _i32, C.c_double, C.POINTER(C.c_int)]
        L.or_refactor_sample.restype = C.c_int
        L.or_refactor_sample.argtypes = [C.c_int, _i32, _i32, _f64, _i32, _i32, C.c_double, C.POINTER(C.c_int),
                                         C.POINTER(C.c_double), _f64, C.c_int]
        L.or_refactor_f32.restype = C.c_void_p
        L.or_refactor_f32.argtypes = [C.c_int, _i32, _i32, _f64, _i32, _i32, C.c_double, C.POINTER(C.c_int)]
        L.or_factor_free.argtypes = [C.c_void_p]
        L.or_factor_sizes.argtypes = [C.c_void_p, C.POINTER(C.c_long), C.POINTER(C.c_long), C.POINTER(C.c_int)]
        L.or_factor_copy.argtypes = [C.c_void_p, _i32, _i32, _f64, _i32, _i32, _f64]
        L.or_solve.argtypes = [C.c_void_p, _i32, _i32, _f64, _f64]
        L.or_norm_inf.restype = C.c_double
        L.or_norm_inf.argtypes = [C.c_int, _i32, _f64]
        L.or_residual.argtypes = [C.c_int, _i32, _i32, _f64, _f64, _f64, _f64]
        L.or_nrbe.restype = C.c_double
        L.or_nrbe.argtypes = [C.c_int, _i32, _i32, _f64, _f64, _f64]
        L.or_nsr.restype = C.c_double
        L.or_nsr.argtypes = [C.c_int, _i32, _i32, _f64, _f64, _f64]
        L.or_fgmres.restype = C.c_int
        L.or_fgmres.argtypes = [C.c_int, _i32, _i32, _f64, C.c_void_p, _i32, _i32, _f64, _f64,
                                C.c_int, C.c_int, C.c_double, C.c_int, C.c_double,
                                C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p]
        L.or_fgmres_ex.restype = C.c_int
        L.or_fgmres_ex.argtypes = [C.c_int, _i32, _i32, _f64, C.c_void_p, _i32, _i32, _f64, _f64,
                                   C.c_int, C.c_int, C.c_double, C.c_int, C.c_double,
                                   C.c_int, C.c_int, C.c_double,
                                   C.POINTER(C.c_int), C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p]
        L.or_richardson.restype = C.c_int
        L.or_richardson.argtypes = [C.c_int, _i32, _i32, _f64, C.c_void_p, _i32, _i32, _f64, _f64,
                                    C.c_int, C.c_double, C.c_int, C.c_double,
                                    C.POINTER(C.c_int), C.POINTER(C.c_double), C.c_void_p]
        L.or_order_md.restype = C.c_int
        L.or_order_md.argtypes = [C.c_int, _i32, _i32, _i32]
        _lib = L
    return _lib


class OracleError(RuntimeError):
    def __init__(self, code, what):
        super().__init__(f"oracle {what}: status {code}")
        self.code = code


def csr_to_csc(n, rowptr, colind, values):
    """Transpose-by-counting: CSR of K -> CSC of K (same matrix)."""
    rowptr = np.asarray(rowptr, np.int64)
    colind = np.asarray(colind, np.int64)
    nnz = len(colind)
    rows = np.repeat(np.arange(n), np.diff(rowptr))
    order = np.argsort(colind, kind="stable")
    Ap = np.zeros(n + 1, np.int64)
    np.add.at(Ap, colind + 1, 1)
    Ap = np.cumsum(Ap)
    return (Ap.astype(np.int32), rows[order].astype(np.int32),
            np.ascontiguousarray(np.asarray(values, np.float64)[order]) if nnz else np.zeros(0))


@dataclasses.dataclass
class Factors:
    """L (strict lower, CSC) and U (with diagonal, CSC) in the permuted space."""
    n: int
    Lp: np.ndarray
    Li: np.ndarray
    Lx: np.ndarray
    Up: np.ndarray
    Ui: np.ndarray
    Ux: np.ndarray
    nboost: int = 0
    _h: int | None = None

    def free(self):
        if self._h:
            lib().or_factor_free(self._h)
            self._h = None

    def __del__(self):
        try:
            self.free()
        except Exception:
            pass

    def dense_L(self):
        D = np.eye(self.n)
        for j in range(self.n):
            for p in range(self.Lp[j], self.Lp[j + 1]):
                D[self.Li[p], j] = self.Lx[p]
        return D

    def dense_U(self):
        D = np.zeros((self.n, self.n))
        for j in range(self.n):
            for p in range(self.Up[j], self.Up[j + 1]):
                D[self.Ui[p], j] = self.Ux[p]
        return D


def _factors_from_handle(n, h):
    L = lib()
    lnz, unz, nb = C.c_long(), C.c_long(), C.c_int()
    L.or_factor_sizes(h, C.byref(lnz), C.byref(unz), C.byref(nb))
    Lp = np.zeros(n + 1, np.int32)
    Up = np.zeros(n + 1, np.int32)
    Li = np.zeros(max(lnz.value, 1), np.int32)
    Lx = np.zeros(max(lnz.value, 1), np.float64)
    Ui = np.zeros(max(unz.value, 1), np.int32)
    Ux = np.zeros(max(unz.value, 1), np.float64)
    L.or_factor_copy(h, Lp, Li, Lx, Up, Ui, Ux)
    return Factors(n, Lp, Li[:lnz.value], Lx[:lnz.value], Up, Ui[:unz.value], Ux[:unz.value], nb.value, h)


def order_md(n, rowptr, colind):
    """Column minimum-degree order Q (pattern of A^T A)."""
    Q = np.zeros(n, np.int32)
    rc = lib().or_order_md(n, np.ascontiguousarray(rowptr, np.int32), np.ascontiguousarray(colind, np.int32), Q)
    if rc != OK:
        raise OracleError(rc, "order_md")
    return Q


def lu(n, rowptr, colind, values, Q=None, tol=1e-3):
    """First factorization with threshold partial pivoting.  Returns (P, Q, Factors)."""
    if Q is None:
        Q = order_md(n, rowptr, colind)
    Q = np.ascontiguousarray(Q, np.int32)
    Ap, Ai, Ax = csr_to_csc(n, rowptr, colind, values)
    P = np.zeros(n, np.int32)
    st = C.c_int()
    h = lib().or_lu(n, Ap, Ai, Ax, Q, float(tol), P, C.byref(st))
    if not h:
        raise OracleError(st.value, "lu")
    return P, Q, _factors_from_handle(n, h)


def refactor(n, rowptr, colind, values, P, Q, boost_abs=0.0):
    """Refactorization on the fixed pivot sequence P and order Q."""
    Ap, Ai, Ax = csr_to_csc(n, rowptr, colind, values)
    st = C.c_int()
    h = lib().or_refactor(n, Ap, Ai, Ax, np.ascontiguousarray(P, np.int32),
                          np.ascontiguousarray(Q, np.int32), float(boost_abs), C.byref(st))
    if not h:
        raise OracleError(st.value, "refactor")
    return _factors_from_handle(n, h)


def refactor_sample(n, rowptr, colind, values, P, Q, seconds):
    """The refactorization run for about `seconds` (the bounded CPU-baseline
    sample).  Returns (columns finished, multiply-adds they took, seconds
    spent in the call, checkpoints): the checkpoints are rows (columns,
    multiply-adds, stored factor entries, seconds) every 256 columns; no
    factors are kept."""
    import time
    Ap, Ai, Ax = csr_to_csc(n, rowptr, colind, values)
    cols, madds = C.c_int(), C.c_double()
    nmarks = n // 256
    marks = np.zeros(4 * max(nmarks, 1))
    t = time.perf_counter()
    st = lib().or_refactor_sample(n, Ap, Ai, Ax, np.ascontiguousarray(P, np.int32), np.ascontiguousarray(Q, np.int32),
                                  float(seconds), C.byref(cols), C.byref(madds), marks, nmarks)
    dt = time.perf_counter() - t
    if st != OK:
        raise OracleError(st, "refactor_sample")
    marks = marks.reshape(-1, 4)
    marks = marks[marks[:, 0] > 0]
    return cols.value, madds.value, dt, marks


def refactor_f32(n, rowptr, colind, values, P, Q, boost_abs=0.0):
    """Refactorization in FP32 arithmetic (factors returned widened to double)."""
    Ap, Ai, Ax = csr_to_csc(n, rowptr, colind, values)
    st = C.c_int()
    h = lib().or_refactor_f32(n, Ap, Ai, Ax, np.ascontiguousarray(P, np.int32),
                              np.ascontiguousarray(Q, np.int32), float(boost_abs), C.byref(st))
    if not h:
        raise OracleError(st.value, "refactor_f32")
    return _factors_from_handle(n, h)


def solve(F: Factors, P, Q, b):
    """x = Q U^{-1} L^{-1} P b."""
    x = np.zeros(F.n, np.float64)
    lib().or_solve(F._h, np.ascontiguousarray(P, np.int32), np.ascontiguousarray(Q, np.int32),
                   np.ascontiguousarray(b, np.float64), x)
    return x


def norm_inf(n, rowptr, values):
    return lib().or_norm_inf(n, np.ascontiguousarray(rowptr, np.int32), np.ascontiguousarray(values, np.float64))


def residual(n, rowptr, colind, values, b, x):
    r = np.zeros(n)
    lib().or_residual(n, np.ascontiguousarray(rowptr, np.int32), np.ascontiguousarray(colind, np.int32),
                      np.ascontiguousarray(values, np.float64), np.ascontiguousarray(b, np.float64),
                      np.ascontiguousarray(x, np.float64), r)
    return r


def nrbe(n, rowptr, colind, values, b, x):
    """Eq. (nbre): ||b - Kx||_2 / (||K||_inf ||x||_2 + ||b||_2)."""
    return lib().or_nrbe(n, np.ascontiguousarray(rowptr, np.int32), np.ascontiguousarray(colind, np.int32),
                         np.ascontiguousarray(values, np.float64), np.ascontiguousarray(b, np.float64),
                         np.ascontiguousarray(x, np.float64))


def nsr(n, rowptr, colind, values, b, x):
    """NSR = ||b - Kx||_inf / (||K||_inf ||x||_inf)."""
    return lib().or_nsr(n, np.ascontiguousarray(rowptr, np.int32), np.ascontiguousarray(colind, np.int32),
                        np.ascontiguousarray(values, np.float64), np.ascontiguousarray(b, np.float64),
                        np.ascontiguousarray(x, np.float64))


@dataclasses.dataclass
class FgmresResult:
    x: np.ndarray
    status: int
    iters: int
    cycles: int
    nrbe: float
    trace: np.ndarray


ORTHO = {"cgs2": 0, "cgs2_pythagoras": 1, "cgs1_pythagoras": 2}


def fgmres(n, rowptr, colind, values, F: Factors, P, Q, b, tol=1e-12, restart=20, max_cycles=50,
           stop_mode=0, refine_delta=0.0, ortho="cgs2", error_equation=False, inner_tol=1e-6):
    """FGMRES(restart) refinement with M = LU as right preconditioner.

    stop_mode 0: NRBE <= tol; stop_mode 1: the paper's relative-residual rule.
    ortho: "cgs2", "cgs2_pythagoras" (two reductions), "cgs1_pythagoras"
    (one reduction).  error_equation: each cycle solves the error equation
    to |g| <= inner_tol * beta, then x is updated and checked.
    """
    x = np.zeros(n, np.float64)
    it, cy, nr = C.c_int(), C.c_int(), C.c_double()
    trace = np.zeros(1 + max_cycles * restart, np.float64)
    rc = lib().or_fgmres_ex(n, np.ascontiguousarray(rowptr, np.int32), np.ascontiguousarray(colind, np.int32),
                            np.ascontiguousarray(values, np.float64), F._h,
                            np.ascontiguousarray(P, np.int32), np.ascontiguousarray(Q, np.int32),
                            np.ascontiguousarray(b, np.float64), x, int(restart), int(max_cycles),
                            float(tol), int(stop_mode), float(refine_delta),
                            ORTHO[ortho], int(bool(error_equation)), float(inner_tol),
                            C.byref(it), C.byref(cy), C.byref(nr), trace.ctypes.data_as(C.c_void_p))
    ntr = 1 + it.value
    return FgmresResult(x, rc, it.value, cy.value, nr.value, trace[:ntr])


def richardson(n, rowptr, colind, values, F: Factors, P, Q, b, tol=1e-12, max_steps=1000, stop_mode=0,
               refine_delta=0.0):
    """Classical iterative refinement x += (LU)^{-1}(b - K x) (Section 2.1).
    Returns FgmresResult (cycles = 0); trace = ||rho|| after x0 and after
    every correction."""
    x = np.zeros(n, np.float64)
    it, nr = C.c_int(), C.c_double()
    trace = np.zeros(1 + max_steps, np.float64)
    rc = lib().or_richardson(n, np.ascontiguousarray(rowptr, np.int32), np.ascontiguousarray(colind, np.int32),
                             np.ascontiguousarray(values, np.float64), F._h,
                             np.ascontiguousarray(P, np.int32), np.ascontiguousarray(Q, np.int32),
                             np.ascontiguousarray(b, np.float64), x, int(max_steps), float(tol),
                             int(stop_mode), float(refine_delta), C.byref(it), C.byref(nr),
                             trace.ctypes.data_as(C.c_void_p))
    return FgmresResult(x, rc, it.value, 0, nr.value, trace[:1 + it.value])


def solve_sequence_step(n, rowptr, colind, values, P, Q, b, tol=1e-12, restart=20, max_cycles=50,
                        boost_abs=0.0, stop_mode=0, refine_delta=0.0):
    """One hot-path step as the oracle computes it: refactor on (P, Q), then
    FGMRES refinement from the LU solution."""
    F = refactor(n, rowptr, colind, values, P, Q, boost_abs)
    res = fgmres(n, rowptr, colind, values, F, P, Q, b, tol, restart, max_cycles, stop_mode, refine_delta)
    return F, res
