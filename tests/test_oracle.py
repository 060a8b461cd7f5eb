"""Pins for the CPU FP64 oracle against facts that do not come from itself:
LAPACK's dense LU, closed forms, textbook Krylov properties, brute-force
least squares, and invariants of the method.  CPU only."""
import json
import os
from fractions import Fraction

import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp

from paper_2401_13926_b300.workload import KKTSequence, small_random_sparse

HERE = os.path.dirname(os.path.abspath(__file__))


def csr(A):
    A = sp.csr_matrix(A)
    A.sum_duplicates()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64)


def dense(n, rp, ci, v):
    return sp.csr_matrix((v, ci, rp), shape=(n, n)).toarray()


def lu_product(F, n):
    return F.dense_L() @ F.dense_U()


# ---------------------------------------------------------------- LU pins
@pytest.mark.parametrize("n,seed", [(5, 0), (17, 1), (40, 2), (60, 3)])
def test_lu_equals_lapack_dense(oracle_mod, n, seed):
    """Partial pivoting (tol = 1, Q = I) on a dense matrix is LAPACK getrf."""
    A = np.random.default_rng(seed).standard_normal((n, n))
    rp, ci, v = csr(A)
    P, Q, F = oracle_mod.lu(n, rp, ci, v, Q=np.arange(n, dtype=np.int32), tol=1.0)
    Pl, Ll, Ul = sla.lu(A)
    assert np.array_equal(P, np.argmax(Pl, axis=0))
    assert np.abs(F.dense_L() - Ll).max() <= 1e-13 * np.abs(Ll).max()
    assert np.abs(F.dense_U() - Ul).max() <= 1e-13 * np.abs(Ul).max()


@pytest.mark.parametrize("n,dens,seed", [(30, 0.1, 4), (50, 0.06, 5), (60, 0.15, 6)])
def test_lu_equals_lapack_sparse(oracle_mod, n, dens, seed):
    rp, ci, v = small_random_sparse(n, dens, seed)
    A = dense(n, rp, ci, v)
    P, Q, F = oracle_mod.lu(n, rp, ci, v, Q=np.arange(n, dtype=np.int32), tol=1.0)
    Pl, Ll, Ul = sla.lu(A)
    assert np.array_equal(P, np.argmax(Pl, axis=0))
    assert np.abs(F.dense_L() - Ll).max() <= 1e-12 * max(1.0, np.abs(Ll).max())
    assert np.abs(F.dense_U() - Ul).max() <= 1e-12 * np.abs(Ul).max()


def test_lu_exact_rational_small(oracle_mod):
    """A 4x4 integer matrix factorized in exact rational arithmetic."""
    A = np.array([[2, 0, 1, 0], [4, 3, 0, 1], [0, 1, 5, 2], [6, 0, 0, 7]], dtype=float)
    n = 4
    rp, ci, v = csr(A)
    P, Q, F = oracle_mod.lu(n, rp, ci, v, Q=np.arange(n, dtype=np.int32), tol=1.0)
    # exact Doolittle elimination with partial pivoting on Fractions
    M = [[Fraction(int(x)) for x in row] for row in A]
    perm = list(range(n))
    Lx = [[Fraction(0)] * n for _ in range(n)]
    for k in range(n):
        piv = max(range(k, n), key=lambda i: (abs(M[i][k]), -perm[i]))
        M[k], M[piv] = M[piv], M[k]
        Lx[k], Lx[piv] = Lx[piv], Lx[k]
        perm[k], perm[piv] = perm[piv], perm[k]
        for i in range(k + 1, n):
            Lx[i][k] = M[i][k] / M[k][k]
            for j in range(k, n):
                M[i][j] -= Lx[i][k] * M[k][j]
    assert list(P) == perm
    Ld, Ud = F.dense_L(), F.dense_U()
    for i in range(n):
        for j in range(n):
            if j >= i:
                assert Ud[i, j] == pytest.approx(float(M[i][j]), abs=1e-14)
            else:
                assert Ud[i, j] == 0.0
                assert Ld[i, j] == pytest.approx(float(Lx[i][j]), abs=1e-14)


def test_threshold_pivot_keeps_diagonal(oracle_mod):
    """|a_jj| >= tol * max |a_ij| keeps the diagonal pivot; otherwise the
    largest entry is taken."""
    A = np.array([[0.01, 1.0], [1.0, 1.0]])
    rp, ci, v = csr(A)
    P, _, F = oracle_mod.lu(2, rp, ci, v, Q=np.arange(2, dtype=np.int32), tol=1e-3)
    assert list(P) == [0, 1]
    assert F.dense_U()[0, 0] == 0.01
    P, _, F = oracle_mod.lu(2, rp, ci, v, Q=np.arange(2, dtype=np.int32), tol=0.1)
    assert list(P) == [1, 0]
    assert F.dense_U()[0, 0] == 1.0


def test_lu_with_column_order_reproduces_permuted_matrix(oracle_mod):
    seq = KKTSequence("kkt200", buses=20, steps=2)
    v = seq.values(0)
    P, Q, F = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, v)
    assert sorted(Q) == list(range(seq.n)) and sorted(P) == list(range(seq.n))
    A = dense(seq.n, seq.rowptr, seq.colind, v)
    B = A[np.ix_(P, Q)]
    assert np.abs(lu_product(F, seq.n) - B).max() <= 1e-12 * np.abs(A).max()


# ---------------------------------------------------------------- refactor pins
@pytest.mark.parametrize("buses", [20, 40])
def test_refactor_reproduces_first_factorization(oracle_mod, buses):
    """Refactoring A_0 on the pivots of its own factorization gives the same
    factors: same pattern exactly, values to rounding."""
    seq = KKTSequence("kkt200", buses=buses, steps=2)
    v = seq.values(0)
    P, Q, F0 = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, v)
    F1 = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, v, P, Q)
    assert np.array_equal(F0.Lp, F1.Lp) and np.array_equal(F0.Li, F1.Li)
    assert np.array_equal(F0.Up, F1.Up) and np.array_equal(F0.Ui, F1.Ui)
    assert np.linalg.norm(F0.Lx - F1.Lx) <= 1e-14 * np.linalg.norm(F0.Lx)
    assert np.linalg.norm(F0.Ux - F1.Ux) <= 1e-14 * np.linalg.norm(F0.Ux)


def test_refactor_next_matrix_is_its_lu(oracle_mod):
    """With the pivots of A_0, the refactor of A_k satisfies L U = A_k(P, Q)."""
    seq = KKTSequence("kkt200", buses=20, steps=4)
    P, Q, _ = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, seq.values(0))
    vk = seq.values(3)
    F = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, vk, P, Q)
    A = dense(seq.n, seq.rowptr, seq.colind, vk)
    scale = np.abs(F.dense_L()).max() * np.abs(F.dense_U()).max()
    assert np.abs(lu_product(F, seq.n) - A[np.ix_(P, Q)]).max() <= 1e-13 * scale


def test_refactor_zero_pivot_and_boost(oracle_mod):
    """A stored zero on a static pivot: an error without the boost; with it,
    u_jj = +boost (sign(0) = +1) and the rest follows from that pivot."""
    A0 = np.array([[2.0, 1.0], [1.0, 3.0]])
    rp, ci, v0 = csr(A0)
    P, Q, _ = oracle_mod.lu(2, rp, ci, v0, Q=np.arange(2, dtype=np.int32), tol=1e-3)
    v1 = np.array([0.0, 1.0, 1.0, 3.0])   # same pattern, a_00 = 0
    with pytest.raises(oracle_mod.OracleError) as e:
        oracle_mod.refactor(2, rp, ci, v1, P, Q, 0.0)
    assert e.value.code == oracle_mod.ERR_SINGULAR
    F = oracle_mod.refactor(2, rp, ci, v1, P, Q, 1e-8)
    assert F.nboost == 1
    U = F.dense_U()
    assert U[0, 0] == 1e-8 and U[0, 1] == 1.0
    assert F.dense_L()[1, 0] == 1.0 / 1e-8
    assert U[1, 1] == 3.0 - 1e8


# ---------------------------------------------------------------- solve pins
@pytest.mark.parametrize("seed", [0, 1])
def test_solve_equals_dense_solve(oracle_mod, seed):
    rp, ci, v = small_random_sparse(80, 0.05, seed, diag_boost=3.0)
    A = dense(80, rp, ci, v)
    P, Q, F = oracle_mod.lu(80, rp, ci, v)
    b = np.random.default_rng(seed).standard_normal(80)
    x = oracle_mod.solve(F, P, Q, b)
    xr = np.linalg.solve(A, b)
    assert np.linalg.norm(x - xr) <= np.linalg.cond(A) * 1e-14 * np.linalg.norm(xr)


# ---------------------------------------------------------------- norms
def test_nrbe_nsr_closed_form(oracle_mod):
    """K = diag(2, 4) plus K[0,1] = -1, x = (1, 1), b = (2, 5):
    r = b - Kx = (1, 1); ||K||_inf = 4."""
    K = np.array([[2.0, -1.0], [0.0, 4.0]])
    rp, ci, v = csr(K)
    x = np.array([1.0, 1.0])
    b = np.array([2.0, 5.0])
    assert oracle_mod.norm_inf(2, rp, v) == 4.0
    assert np.allclose(oracle_mod.residual(2, rp, ci, v, b, x), [1.0, 1.0], rtol=0, atol=0)
    assert oracle_mod.nrbe(2, rp, ci, v, b, x) == pytest.approx(np.sqrt(2) / (4 * np.sqrt(2) + np.sqrt(29)), rel=1e-15)
    assert oracle_mod.nsr(2, rp, ci, v, b, x) == pytest.approx(1.0 / 4.0, rel=1e-15)
    assert oracle_mod.nrbe(2, rp, ci, v, K @ x, x) == 0.0


# ---------------------------------------------------------------- FGMRES pins
def identity_factors(oracle_mod, n):
    I = sp.identity(n, format="csr")
    rp, ci, v = csr(I)
    return oracle_mod.lu(n, rp, ci, v, Q=np.arange(n, dtype=np.int32), tol=1.0)


def test_fgmres_exact_preconditioner_needs_at_most_one_iteration(oracle_mod):
    seq = KKTSequence("kkt200", buses=30, steps=3)
    v = seq.values(1)
    b, _ = seq.rhs(1, v)
    P, Q, F = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, v)
    res = oracle_mod.fgmres(seq.n, seq.rowptr, seq.colind, v, F, P, Q, b, tol=1e-12)
    assert res.status == 0 and res.iters <= 1 and res.nrbe <= 1e-12


@pytest.mark.parametrize("d", [2, 3, 5])
def test_gmres_identity_preconditioner_diagonal_d_steps(oracle_mod, d):
    """GMRES on a diagonal matrix with d distinct eigenvalues converges in
    exactly d steps (degree of the minimal polynomial).  With M = I the
    initial guess is x0 = b, so r0 = (I - K) b; no eigenvalue is 1, so r0 has
    a component in all d eigenspaces."""
    n = 40
    diag = np.array([2.0 + 3.0 * (i % d) for i in range(n)])
    rp, ci, v = csr(sp.diags(diag))
    P, Q, F = identity_factors(oracle_mod, n)
    b = np.random.default_rng(d).standard_normal(n)
    res = oracle_mod.fgmres(n, rp, ci, v, F, P, Q, b, tol=1e-13, restart=30, max_cycles=1)
    assert res.status == 0
    assert res.iters == d


def _krylov_minres(K, Minv, b, x0, j):
    """min over x in x0 + Minv K_j(K Minv, r0) of ||b - K x||, by least squares
    on a Krylov basis re-orthonormalised by LAPACK's Householder QR after
    every product (same space, an independent construction)."""
    r0 = b - K @ x0
    B = (r0 / np.linalg.norm(r0))[:, None]
    for _ in range(j - 1):
        w = K @ (Minv @ B[:, -1])
        B, _ = np.linalg.qr(np.column_stack([B, w]))
    S = Minv @ B
    y, *_ = np.linalg.lstsq(K @ S, r0, rcond=None)
    return np.linalg.norm(r0 - K @ S @ y), x0 + S @ y


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_fgmres_residuals_are_krylov_minima(oracle_mod, seed):
    """Each estimated residual |g_{j+1}| equals the minimum residual over the
    affine space x0 + span(Z_j); the cycle-end x is that minimiser and its
    true residual equals the last estimate."""
    n, m = 30, 7
    rng = np.random.default_rng(seed)
    rp, ci, v = small_random_sparse(n, 0.12, 10 + seed, diag_boost=2.0)
    K = dense(n, rp, ci, v)
    Kp = K + 0.3 * np.diag(rng.standard_normal(n))       # inexact preconditioner
    prp, pci, pv = csr(Kp)
    P, Q, F = oracle_mod.lu(n, prp, pci, pv, Q=np.arange(n, dtype=np.int32), tol=1.0)
    Minv = np.linalg.inv(Kp)
    b = rng.standard_normal(n)
    res = oracle_mod.fgmres(n, rp, ci, v, F, P, Q, b, tol=1e-300, restart=m, max_cycles=1)
    assert res.status == oracle_mod.ERR_NOT_CONVERGED and res.iters == m
    x0 = Minv @ b
    assert res.trace[0] == pytest.approx(np.linalg.norm(b - K @ x0), rel=1e-10)
    for j in range(1, m + 1):
        rmin, xmin = _krylov_minres(K, Minv, b, x0, j)
        assert res.trace[j] == pytest.approx(rmin, rel=1e-8)
    assert np.linalg.norm(res.x - xmin) <= 1e-8 * np.linalg.norm(xmin)
    assert np.linalg.norm(b - K @ res.x) == pytest.approx(res.trace[m], rel=1e-8)


def test_fgmres_rr_rule_stops_on_estimated_relative_residual(oracle_mod):
    seq = KKTSequence("kkt200", buses=30, steps=6)
    P, Q, _ = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, seq.values(0))
    v = seq.values(5)
    b, _ = seq.rhs(5, v)
    F = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, v, P, Q)
    tol = 1e-10
    res = oracle_mod.fgmres(seq.n, seq.rowptr, seq.colind, v, F, P, Q, b, tol=tol, stop_mode=1)
    assert res.status == 0
    if res.iters:
        assert res.trace[-1] < tol * res.trace[0]
        assert np.all(res.trace[1:-1] >= tol * res.trace[0])


def test_refine_delta_skips_refinement(oracle_mod):
    seq = KKTSequence("kkt200", buses=30, steps=6)
    P, Q, _ = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, seq.values(0))
    v = seq.values(5)
    b, _ = seq.rhs(5, v)
    F = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, v, P, Q)
    x0 = oracle_mod.solve(F, P, Q, b)
    rel = np.linalg.norm(oracle_mod.residual(seq.n, seq.rowptr, seq.colind, v, b, x0)) / np.linalg.norm(b)
    res = oracle_mod.fgmres(seq.n, seq.rowptr, seq.colind, v, F, P, Q, b, tol=1e-16, refine_delta=2 * rel)
    assert res.iters == 0 and np.array_equal(res.x, x0)


# ---------------------------------------------------------------- end to end
def test_manufactured_kkt_sequence(oracle_mod):
    """b = K x*: after refinement NRBE <= 1e-12 on every matrix, and the
    forward error is within cond(K) * machine epsilon (times a small factor)."""
    seq = KKTSequence("kkt200", buses=40, steps=5)
    P, Q, _ = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, seq.values(0))
    for k in range(seq.M):
        v = seq.values(k)
        b, xs = seq.rhs(k, v)
        F, res = oracle_mod.solve_sequence_step(seq.n, seq.rowptr, seq.colind, v, P, Q, b)
        assert res.status == 0 and res.nrbe <= 1e-12
        cond = np.linalg.cond(dense(seq.n, seq.rowptr, seq.colind, v))
        assert np.linalg.norm(res.x - xs) <= 100 * cond * 2.2e-16 * np.linalg.norm(xs)


def test_iteration_counts_in_paper_band(oracle_mod):
    """Sanity band, not parity: the paper reports a few FGMRES iterations per
    system (Table 2, fixture in tests/golden)."""
    with open(os.path.join(HERE, "golden", "table2_fgmres.json")) as f:
        t2 = json.load(f)
    hi = max(r["iters"] for r in t2["rows"])
    seq = KKTSequence("kkt200", buses=40, steps=5)
    P, Q, _ = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, seq.values(0))
    its = []
    for k in range(seq.M):
        v = seq.values(k)
        b, _ = seq.rhs(k, v)
        _, res = oracle_mod.solve_sequence_step(seq.n, seq.rowptr, seq.colind, v, P, Q, b, restart=10)
        its.append(res.iters)
    assert np.mean(its) <= 3 * hi


# ---------------------------------------------------------------- ordering
def test_order_md_is_permutation_and_star_order(oracle_mod):
    """Star column graph: leaves (degree 1) are eliminated first, in index
    order; once one leaf is left it ties with the centre at degree 1 and the
    smaller index (the centre) goes first."""
    n, c = 9, 4
    rows, cols = [], []
    for i in range(n):
        rows.append(i); cols.append(i)
        if i != c:
            rows.append(i); cols.append(c)
    A = sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(n, n))
    rp, ci, _ = csr(A)
    Q = oracle_mod.order_md(n, rp, ci)
    assert list(Q) == [0, 1, 2, 3, 5, 6, 7, c, 8]


def test_order_md_reduces_fill_on_kkt(oracle_mod):
    seq = KKTSequence("kkt200", buses=40, steps=1)
    v = seq.values(0)
    nat = np.arange(seq.n, dtype=np.int32)
    _, _, Fn = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, v, Q=nat)
    _, _, Fm = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, v)
    assert len(Fm.Li) + len(Fm.Ui) < 0.5 * (len(Fn.Li) + len(Fn.Ui))


# ---------------------------------------------------------------- FP32 refactor
def test_refactor_f32_close_to_fp64_and_is_an_lu(oracle_mod):
    """FP32 refactorization (mixed precision): same pattern as FP64, values
    within float rounding (times growth) of the FP64 factors, and L U equal to
    the float-rounded matrix to float accuracy."""
    seq = KKTSequence("kkt200", buses=20, steps=3)
    P, Q, _ = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, seq.values(0))
    v = seq.values(2)
    F64 = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, v, P, Q)
    F32 = oracle_mod.refactor_f32(seq.n, seq.rowptr, seq.colind, v, P, Q)
    assert np.array_equal(F64.Lp, F32.Lp) and np.array_equal(F64.Li, F32.Li)
    assert np.array_equal(F64.Up, F32.Up) and np.array_equal(F64.Ui, F32.Ui)
    # every value is exactly a float
    assert np.all(F32.Lx.astype(np.float32).astype(np.float64) == F32.Lx)
    assert np.all(F32.Ux.astype(np.float32).astype(np.float64) == F32.Ux)
    A = dense(seq.n, seq.rowptr, seq.colind, v.astype(np.float32).astype(np.float64))
    scale = np.abs(F32.dense_L()).max() * np.abs(F32.dense_U()).max()
    assert np.abs(lu_product(F32, seq.n) - A[np.ix_(P, Q)]).max() <= 64 * 1.2e-7 * scale


def test_refactor_f32_exact_on_small_integers(oracle_mod):
    """A 3x3 case whose FP32 and exact factors coincide (all quantities exact
    in float): the FP32 path must reproduce them exactly."""
    A = np.array([[4.0, 2.0, 0.0], [2.0, 5.0, 1.0], [0.0, 1.0, 3.0]])
    rp, ci, v = csr(A)
    I = np.arange(3, dtype=np.int32)
    F = oracle_mod.refactor_f32(3, rp, ci, v, I, I)
    # l21 = 2/4 = 0.5, u22 = 5 - 0.5*2 = 4, l32 = 1/4, u33 = 3 - 0.25*1 = 2.75
    assert np.array_equal(F.dense_L(), np.array([[1, 0, 0], [0.5, 1, 0], [0, 0.25, 1]]))
    assert np.array_equal(F.dense_U(), np.array([[4, 2, 0], [0, 4, 1], [0, 0, 2.75]]))


# ---------------------------------------------------------------- refinement variants
def _inexact_case(oracle_mod, seed, n=30, pert=0.3):
    rng = np.random.default_rng(seed)
    rp, ci, v = small_random_sparse(n, 0.12, 10 + seed, diag_boost=2.0)
    K = dense(n, rp, ci, v)
    Kp = K + pert * np.diag(rng.standard_normal(n))        # M = LU(Kp), an inexact preconditioner
    prp, pci, pv = csr(Kp)
    P, Q, F = oracle_mod.lu(n, prp, pci, pv, Q=np.arange(n, dtype=np.int32), tol=1.0)
    return n, rp, ci, v, K, np.linalg.inv(Kp), P, Q, F, rng.standard_normal(n)


@pytest.mark.parametrize("seed", [0, 1])
def test_richardson_residuals_follow_the_iteration_matrix(oracle_mod, seed):
    """Classical refinement is the stationary iteration r_{k+1} = (I - K M^{-1}) r_k:
    every traced residual norm equals the norm of a power of that matrix
    applied to r_0 (dense powers, an independent construction)."""
    n, rp, ci, v, K, Minv, P, Q, F, b = _inexact_case(oracle_mod, seed, pert=0.2)
    G = np.eye(n) - K @ Minv
    assert np.max(np.abs(np.linalg.eigvals(G))) < 1
    res = oracle_mod.richardson(n, rp, ci, v, F, P, Q, b, tol=1e-300, max_steps=6)
    assert res.status == oracle_mod.ERR_NOT_CONVERGED and res.iters == 6
    r = b - K @ (Minv @ b)
    for k in range(7):
        assert res.trace[k] == pytest.approx(np.linalg.norm(r), rel=1e-8)
        r = G @ r
    x = Minv @ b
    for _ in range(6):
        x = x + Minv @ (b - K @ x)
    assert np.allclose(res.x, x, rtol=1e-10, atol=1e-12)


def test_richardson_exact_factors_and_divergence(oracle_mod):
    """Exact factors: x0 already meets the NRBE rule (no correction).  A
    preconditioner with spectral radius of I - K M^{-1} above one: the
    residual grows and the run ends NOT_CONVERGED."""
    n, rp, ci, v, K, Minv, P, Q, F, b = _inexact_case(oracle_mod, 3, pert=0.0)
    res = oracle_mod.richardson(n, rp, ci, v, F, P, Q, b, tol=1e-13)
    assert res.status == 0 and res.iters == 0 and res.nrbe <= 1e-13
    n, rp, ci, v, K, Minv, P, Q, F, b = _inexact_case(oracle_mod, 4, pert=6.0)
    rho = np.max(np.abs(np.linalg.eigvals(np.eye(n) - K @ Minv)))
    assert rho > 1
    res = oracle_mod.richardson(n, rp, ci, v, F, P, Q, b, tol=1e-13, max_steps=60)
    assert res.status == oracle_mod.ERR_NOT_CONVERGED and res.trace[-1] > res.trace[0]


def test_richardson_rr_rule(oracle_mod):
    n, rp, ci, v, K, Minv, P, Q, F, b = _inexact_case(oracle_mod, 5, pert=0.05)
    assert np.max(np.abs(np.linalg.eigvals(np.eye(n) - K @ Minv))) < 1
    tol = 1e-6
    res = oracle_mod.richardson(n, rp, ci, v, F, P, Q, b, tol=tol, stop_mode=1, max_steps=200)
    assert res.status == 0 and res.iters >= 1
    assert res.trace[-1] < tol * res.trace[0]
    assert np.all(res.trace[1:-1] >= tol * res.trace[0])


@pytest.mark.parametrize("ortho", ["cgs2_pythagoras", "cgs1_pythagoras"])
@pytest.mark.parametrize("seed", [0, 1])
def test_low_sync_variants_give_krylov_minima(oracle_mod, ortho, seed):
    """The Gram-Schmidt variants that take the new vector's norm by
    Pythagoras still give, on a well-conditioned case, the minimum residual
    over x0 + span(Z_j) at every step (Householder-QR reference).  One pass
    of classical Gram-Schmidt loses orthogonality in proportion to the
    basis' conditioning, so its estimates are held to the starting
    residual's scale rather than their own."""
    n, rp, ci, v, K, Minv, P, Q, F, b = _inexact_case(oracle_mod, seed)
    m = 7
    res = oracle_mod.fgmres(n, rp, ci, v, F, P, Q, b, tol=1e-300, restart=m, max_cycles=1, ortho=ortho)
    assert res.iters == m
    x0 = Minv @ b
    for j in range(1, m + 1):
        rmin, xmin = _krylov_minres(K, Minv, b, x0, j)
        if ortho == "cgs2_pythagoras":
            assert res.trace[j] == pytest.approx(rmin, rel=1e-7)
        else:
            assert abs(res.trace[j] - rmin) <= 1e-9 * res.trace[0]
    assert np.linalg.norm(res.x - xmin) <= 1e-7 * np.linalg.norm(xmin)


def test_error_equation_with_one_step_cycles_is_minimal_residual_richardson(oracle_mod):
    """FGMRES on the error equation with inner_tol = 1 stops every cycle
    after one Arnoldi step: x_{k+1} = x_k + a_k M^{-1} r_k with the step
    a_k = (r_k . K M^{-1} r_k) / ||K M^{-1} r_k||^2 minimising the residual."""
    n, rp, ci, v, K, Minv, P, Q, F, b = _inexact_case(oracle_mod, 2)
    res = oracle_mod.fgmres(n, rp, ci, v, F, P, Q, b, tol=1e-300, restart=5, max_cycles=6,
                            error_equation=True, inner_tol=1.0)
    assert res.status == oracle_mod.ERR_NOT_CONVERGED and res.iters == 6 and res.cycles == 6
    x = Minv @ b
    for _ in range(6):
        r = b - K @ x
        z = Minv @ r
        Kz = K @ z
        x = x + (r @ Kz) / (Kz @ Kz) * z
    assert np.allclose(res.x, x, rtol=1e-10, atol=1e-12)


def test_error_equation_inner_tolerance_ends_each_cycle(oracle_mod):
    """With inner_tol, each cycle ends at the first step whose estimate is
    at most inner_tol times the cycle's starting residual."""
    n, rp, ci, v, K, Minv, P, Q, F, b = _inexact_case(oracle_mod, 6, pert=0.6)
    it = 1e-2
    res = oracle_mod.fgmres(n, rp, ci, v, F, P, Q, b, tol=1e-12, restart=30, max_cycles=20,
                            error_equation=True, inner_tol=it)
    assert res.status == 0 and res.nrbe <= 1e-12 and res.cycles >= 2
    # rebuild the cycle boundaries from the trace: a cycle starts at the
    # true residual (the first entry or the one after a cycle end) and ends
    # at the first estimate <= it * start
    start, k, cycles = res.trace[0], 1, 0
    while k < len(res.trace):
        while res.trace[k] > it * start:
            k += 1
        cycles += 1
        k += 1
        if k < len(res.trace):
            start = np.linalg.norm(b - K @ x_at_cycle_end(oracle_mod, n, rp, ci, v, F, P, Q, b, cycles, it))
    assert cycles == res.cycles


def x_at_cycle_end(oracle_mod, n, rp, ci, v, F, P, Q, b, cycles, it):
    r = oracle_mod.fgmres(n, rp, ci, v, F, P, Q, b, tol=1e-300, restart=30, max_cycles=cycles,
                          error_equation=True, inner_tol=it)
    return r.x
