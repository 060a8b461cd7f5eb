"""Mixed precision: FP32 factors and FP32 triangular solves act as the
FGMRES preconditioner, while the residual, CGS2, least squares and update
stay in FP64 (Section 2.1: flexible GMRES tolerates inexact LU factors).

What is checked:
  * the FP32 factors equal the oracle's FP32 refactorization bit for bit on
    the same P, Q (same operation order, fma, reciprocal scaling);
  * the FP32 preconditioner solve meets the componentwise backward-error
    bound of two FP32 triangular solves (Higham, Thm. 8.5) against the
    FP32 factors: |Pb - L U z| <= (2 g(k+2) + u) |L| |U| |z| with
    g(k) = k u / (1 - k u), u = 2^-24, k the longest factor row;
  * every mixed solve is reported truthfully: converged solves meet the
    NRBE (Eq. nbre) tolerance as the oracle evaluates it; the others return
    KKT_ERR_NOT_CONVERGED with the NRBE of the returned x; and refinement
    never leaves a residual larger than that of the preconditioner solve
    it starts from (restarted GMRES minimises the 2-norm residual);
  * on a well-conditioned system mixed refinement reaches 1e-12 like the
    oracle's FGMRES with the same FP32 factors;
  * the FP64 fallback (kkt_opts.mixed_fallback): on the synthetic KKT
    sequences the FP32 preconditioner alone does not always reach 1e-12
    (with the ill-conditioned matrices u32 * cond(K) is far above 1), so a
    solve the FP32 factors have not finished within the allowed cycles
    continues with the FP64 refactorization; every mixed solve then meets
    NRBE <= 1e-12 as the oracle evaluates it, and the FP64 factors of a
    fallback equal the oracle's refactorization bit for bit.
The tests of the FP32-only behaviour turn the fallback off.
"""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence, small_random_sparse

pytestmark = pytest.mark.gpu

U32 = 2.0 ** -24


@pytest.fixture(scope="module")
def c1(oracle_mod):
    seq = KKTSequence("kkt200")
    P, Q, _ = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, seq.values(0))
    return seq, P, Q


@pytest.mark.parametrize("sched", ["auto", "global"])
def test_fp32_factors_match_fp32_oracle(oracle_mod, c1, sched):
    seq, P, Q = c1
    s = K.KKTSolver(precision="mixed", trisolve=sched)
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    for k in range(seq.M):
        v = seq.values(k)
        s.refactor(v)
        of = oracle_mod.refactor_f32(seq.n, seq.rowptr, seq.colind, v, P, Q)
        f = s.factors()
        assert np.array_equal(f["Li"], of.Li) and np.array_equal(f["Ui"], of.Ui)
        assert np.array_equal(f["Lx"], of.Lx), k
        assert np.array_equal(f["Ux"], of.Ux), k


def _factor_mats(n, f):
    L = sp.csc_matrix((f["Lx"], f["Li"], f["Lp"]), shape=(n, n)) + sp.identity(n, format="csc")
    U = sp.csc_matrix((f["Ux"], f["Ui"], f["Up"]), shape=(n, n))
    return L.tocsr(), U.tocsr()


def _check_fp32_solve_bound(n, f, P, Q, b, x):
    L, U = _factor_mats(n, f)
    k = max(np.diff(L.indptr).max(), np.diff(U.indptr).max()) + 2
    g = k * U32 / (1 - k * U32)
    z = np.asarray(x)[np.asarray(Q)]                   # x[Q[j]] = z[j]
    lhs = np.abs(np.asarray(b)[np.asarray(P)] - L @ (U @ z))
    rhs = (2 * g + U32) * (abs(L) @ (abs(U) @ np.abs(z)))
    # the FP64 evaluation of L (U z) adds at most ~1e-15 relative slack
    slack = 1e-13 * (abs(L) @ (abs(U) @ np.abs(z))) + 1e-300
    bad = np.nonzero(lhs > rhs + slack)[0]
    assert bad.size == 0, (bad[:5], lhs[bad[:5]], rhs[bad[:5]])


@pytest.mark.parametrize("sched", ["auto", "global"])
def test_fp32_lu_solve_backward_error_bound(oracle_mod, c1, sched):
    seq, P, Q = c1
    s = K.KKTSolver(precision="mixed", trisolve=sched)
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    rng = np.random.default_rng(5)
    for k in (0, seq.M // 2, seq.M - 1):
        v = seq.values(k)
        s.refactor(v)
        f = s.factors()
        for b in (seq.rhs(k, v)[0], rng.standard_normal(seq.n)):
            x = s.lu_solve(b)
            _check_fp32_solve_bound(seq.n, f, P, Q, b, x)


def _check_reported(oracle_mod, s, n, rp, ci, v, b, x, it, nr, x0, tol, max_iters):
    on = oracle_mod.nrbe(n, rp, ci, v, b, x)
    m = int(np.max(np.diff(rp)))   # two residual evaluations: 2 (m + 2) eps apart at most
    assert abs(nr - on) <= 1e-6 * on + 2 * (m + 2) * 2.0 ** -52, (nr, on)
    if s.last_status == K.OK:
        assert on <= tol * (1 + 1e-6), on
    else:
        assert s.last_status == K.ERR_NOT_CONVERGED
        assert on > tol * (1 - 1e-6) and it <= max_iters
    r = np.linalg.norm(oracle_mod.residual(n, rp, ci, v, b, x))
    r0 = np.linalg.norm(oracle_mod.residual(n, rp, ci, v, b, x0))
    assert r <= r0 * (1 + 1e-6), (r, r0)


@pytest.mark.parametrize("sched", ["auto", "global"])
def test_mixed_solves_reported_truthfully_kkt200(oracle_mod, c1, sched):
    seq, P, Q = c1
    cycles = 3
    s = K.KKTSolver(precision="mixed", trisolve=sched, max_cycles=cycles, mixed_fallback=0)
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    for k in range(seq.M):
        v = seq.values(k)
        b, _ = seq.rhs(k, v)
        s.refactor(v)
        x0 = s.lu_solve(b)
        x, it, nr = s.solve(b, tol=1e-12, allow_not_converged=True)
        _check_reported(oracle_mod, s, seq.n, seq.rowptr, seq.colind, v, b, x, it, nr, x0, 1e-12,
                        cycles * 20)


def test_mixed_full_size_kkt2000(oracle_mod):
    seq = KKTSequence("kkt2000")
    cycles = 2
    s = K.KKTSolver(precision="mixed", max_cycles=cycles, mixed_fallback=0)
    s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    P, Q = s.perm()
    converged = 0
    for k in (0, seq.M // 2, seq.M - 1):
        v = seq.values(k)
        b, _ = seq.rhs(k, v)
        s.refactor(v)
        x0 = s.lu_solve(b)
        _check_fp32_solve_bound(seq.n, s.factors(), P, Q, b, x0)
        x, it, nr = s.solve(b, tol=1e-12, allow_not_converged=True)
        _check_reported(oracle_mod, s, seq.n, seq.rowptr, seq.colind, v, b, x, it, nr, x0, 1e-12,
                        cycles * 20)
        converged += s.last_status == K.OK
    # the last matrix of the sequence is solved to 1e-12 by mixed refinement
    assert converged >= 1


def test_mixed_converges_on_well_conditioned_system(oracle_mod):
    n = 3000
    rp, ci, v = small_random_sparse(n, 4.0 / n, 91, diag_boost=1.0)
    P, Q, _ = oracle_mod.lu(n, rp, ci, v)
    s = K.KKTSolver(precision="mixed", mixed_fallback=0)
    s.analyze(rp, ci, Q=Q, P=P)
    s.refactor(v)
    b = np.random.default_rng(3).standard_normal(n)
    x, it, nr = s.solve(b, tol=1e-12)
    assert oracle_mod.nrbe(n, rp, ci, v, b, x) <= 1e-12
    F = oracle_mod.refactor_f32(n, rp, ci, v, P, Q)
    ores = oracle_mod.fgmres(n, rp, ci, v, F, P, Q, b, tol=1e-12)
    assert ores.status == 0 and ores.nrbe <= 1e-12
    # the two preconditioners differ only in FP32 solve rounding order
    assert abs(it - ores.iters) <= 2, (it, ores.iters)


def test_mixed_random_sparse_factor_parity(oracle_mod):
    n = 900
    rp, ci, v = small_random_sparse(n, 3.0 / n, 77, diag_boost=1.0)
    P, Q, _ = oracle_mod.lu(n, rp, ci, v)
    s = K.KKTSolver(precision="mixed")
    s.analyze(rp, ci, Q=Q, P=P)
    s.refactor(v)
    of = oracle_mod.refactor_f32(n, rp, ci, v, P, Q)
    f = s.factors()
    assert np.array_equal(f["Lx"], of.Lx) and np.array_equal(f["Ux"], of.Ux)


@pytest.mark.parametrize("sched", ["auto", "global"])
def test_mixed_fallback_meets_tolerance_kkt200(oracle_mod, c1, sched):
    """Every solve of the sequence ends at oracle-evaluated NRBE <= 1e-12;
    a solve that fell back reports it, used the FP64 factors (equal to the
    oracle's refactorization bit for bit), and the next refactorization
    starts in FP32 again (its factors equal the oracle's FP32 ones)."""
    seq, P, Q = c1
    s = K.KKTSolver(precision="mixed", trisolve=sched, mixed_fallback=1)
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    falls = 0
    for k in range(seq.M):
        v = seq.values(k)
        b, _ = seq.rhs(k, v)
        s.refactor(v)
        f32 = oracle_mod.refactor_f32(seq.n, seq.rowptr, seq.colind, v, P, Q)
        assert np.array_equal(s.factors()["Ux"], f32.Ux), k
        x, it, nr = s.solve(b, tol=1e-12)
        assert s.last_status == K.OK
        on = oracle_mod.nrbe(seq.n, seq.rowptr, seq.colind, v, b, x)
        # the two residual evaluations differ by at most 2 (m + 2) eps in NRBE
        # (m = the longest row of K) besides 1e-6 relative
        m = int(np.max(np.diff(seq.rowptr)))
        assert on <= 1e-12 and abs(nr - on) <= 1e-6 * on + 2 * (m + 2) * 2.0 ** -52, (k, on, nr)
        info = s.info()
        if info["last_fallback"]:
            falls += 1
            of = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, v, P, Q)
            f = s.factors()
            assert np.array_equal(f["Lx"], of.Lx) and np.array_equal(f["Ux"], of.Ux), k
    assert s.info()["fallbacks"] == falls
    assert falls >= 1   # the s = 8 matrices of kkt200 defeat the FP32 preconditioner


def test_mixed_step_with_fallback_equals_refactor_then_solve(oracle_mod):
    """kkt_step in mixed precision with the fallback gives the same x,
    iterations and NRBE as kkt_refactor then kkt_solve."""
    seq = KKTSequence("kkt200", steps=4)
    a = K.KKTSolver(precision="mixed", mixed_fallback=1)
    f = K.KKTSolver(precision="mixed", mixed_fallback=1)
    a.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    f.analyze_like(a)
    for k in range(seq.M):
        v = seq.values(k)
        b, _ = seq.rhs(k, v)
        a.refactor(v)
        xa, ia, na = a.solve(b, tol=1e-12)
        xf, i_f, nf = f.step(v, b, tol=1e-12)
        assert np.array_equal(xa, xf) and ia == i_f and na == nf, k
        assert a.info()["last_fallback"] == f.info()["last_fallback"]


def _equilibrated(n, rowptr, colind, v):
    """R K C as the equilibration option defines it, written out here from
    its definition: r_i = 2^(1-E) with max_j |a_ij| = f 2^E, f in [0.5, 1)
    (1 for an empty row), c_j the same for max_i |a_ij r_i|; returns the
    scaled values (exact: powers of two), r and c."""
    rows = np.repeat(np.arange(n), np.diff(np.asarray(rowptr)))
    cols = np.asarray(colind)
    a = np.abs(np.asarray(v, dtype=np.float64))
    rmax = np.zeros(n)
    np.maximum.at(rmax, rows, a)
    r = np.where(rmax > 0, np.ldexp(1.0, 1 - np.frexp(rmax)[1]), 1.0)
    cmax = np.zeros(n)
    np.maximum.at(cmax, cols, a * r[rows])
    c = np.where(cmax > 0, np.ldexp(1.0, 1 - np.frexp(cmax)[1]), 1.0)
    assert np.all(np.abs(a * r[rows] * c[cols]) < 2.0)
    return np.asarray(v) * r[rows] * c[cols], r, c


@pytest.mark.parametrize("sched", ["auto", "global"])
def test_equilibrated_fp32_factors_and_solve(oracle_mod, c1, sched):
    """With kkt_opts.equilibrate the FP32 factors are those of R K C: equal,
    bit for bit, to the oracle's FP32 refactorization of the scaled values
    on the same P and Q; and kkt_lu_solve returns x = C z with z the FP32
    triangular solve of (R K C) z = R b, within that solve's componentwise
    backward-error bound."""
    seq, P, Q = c1
    s = K.KKTSolver(precision="mixed", trisolve=sched, equilibrate=True, mixed_fallback=0)
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    rng = np.random.default_rng(11)
    for k in (0, seq.M // 2, seq.M - 1):
        v = seq.values(k)
        s.refactor(v)
        vs, r, c = _equilibrated(seq.n, seq.rowptr, seq.colind, v)
        of = oracle_mod.refactor_f32(seq.n, seq.rowptr, seq.colind, vs, P, Q)
        f = s.factors()
        assert np.array_equal(f["Lx"], of.Lx), k
        assert np.array_equal(f["Ux"], of.Ux), k
        for b in (seq.rhs(k, v)[0], rng.standard_normal(seq.n)):
            x = s.lu_solve(b)
            _check_fp32_solve_bound(seq.n, f, P, Q, r * b, np.asarray(x) / c)


def test_equilibrated_mixed_solves_meet_tolerance_kkt200(oracle_mod, c1):
    """Every mixed solve of the kkt200 sequence with equilibration (and the
    FP64 fallback rule) ends at NRBE <= 1e-12 as the oracle evaluates it."""
    seq, P, Q = c1
    s = K.KKTSolver(precision="mixed", equilibrate=True)
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    for k in range(seq.M):
        v = seq.values(k)
        b, _ = seq.rhs(k, v)
        x, it, nr = s.step(v, b, tol=1e-12)
        on = oracle_mod.nrbe(seq.n, seq.rowptr, seq.colind, v, b, x)
        assert on <= 1e-12 * (1 + 1e-6), (k, on, it)
