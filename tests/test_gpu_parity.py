"""Parity of the CUDA path (through the C ABI) with the CPU FP64 oracle.

Bars: factors on the same P, Q -- identical pattern and relative Frobenius
difference <= 1e-10 per factor; solutions -- NRBE (Eq. nbre, evaluated by
the oracle) <= 1e-12 after refinement; matrix-vector products -- per-row
difference <= (terms + 1) eps sum_j |K_ij x_j|; triangular solves -- componentwise
backward error <= 64 eps, and elementwise agreement with the oracle on a
well-conditioned case."""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence, small_random_sparse

pytestmark = pytest.mark.gpu
EPS = 2.220446049250313e-16
FACTOR_TOL = 1e-10
NRBE_TOL = 1e-12


def factor_diff(gpu, ofac):
    """Relative Frobenius difference of L and U; patterns must be equal."""
    assert np.array_equal(gpu["Lp"], ofac.Lp.astype(np.int64))
    assert np.array_equal(gpu["Li"], ofac.Li)
    assert np.array_equal(gpu["Up"], ofac.Up.astype(np.int64))
    assert np.array_equal(gpu["Ui"], ofac.Ui)
    dl = np.linalg.norm(gpu["Lx"] - ofac.Lx) / max(np.linalg.norm(ofac.Lx), 1e-300)
    du = np.linalg.norm(gpu["Ux"] - ofac.Ux) / np.linalg.norm(ofac.Ux)
    return dl, du


def nrbe_agrees(nr_gpu, nr_or, seq):
    """The NRBE the GPU reports (it drives the stop decision) equals Eq.
    (nbre) as the oracle evaluates it on the returned x, up to the rounding
    of the two residual evaluations: each entry of b - K x carries an error
    of at most (m + 1) eps sum_j |K_ij x_j| + eps |b_i| (m = the row's
    entries), so with ||K||_inf >= the row sums the two NRBE values differ
    by at most 2 (m + 2) eps besides a relative 1e-6 for the norms."""
    m = int(np.max(np.diff(seq.rowptr)))
    return abs(nr_gpu - nr_or) <= 1e-6 * nr_or + 2 * (m + 2) * EPS


def csr_of(A):
    A = sp.csr_matrix(A)
    A.sum_duplicates()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64)


@pytest.fixture(scope="module")
def c1(oracle_mod):
    seq = KKTSequence("kkt200")
    P, Q, _ = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, seq.values(0))
    return seq, P, Q


def test_refactor_parity_kkt200(oracle_mod, c1):
    seq, P, Q = c1
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    for k in range(seq.M):
        v = seq.values(k)
        s.refactor(v)
        of = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, v, P, Q)
        dl, du = factor_diff(s.factors(), of)
        assert dl <= FACTOR_TOL and du <= FACTOR_TOL, (k, dl, du)


@pytest.mark.parametrize("sched", ["auto", "global"])
def test_solve_parity_kkt200(oracle_mod, c1, sched):
    seq, P, Q = c1
    s = K.KKTSolver(restart=20, trisolve=sched)
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    for k in range(seq.M):
        v = seq.values(k)
        b, xs = seq.rhs(k, v)
        s.refactor(v)
        x, it, nr = s.solve(b, tol=NRBE_TOL)
        nr_or = oracle_mod.nrbe(seq.n, seq.rowptr, seq.colind, v, b, x)
        assert nr_or <= NRBE_TOL and nr <= NRBE_TOL, (k, nr_or, nr)
        assert nrbe_agrees(nr, nr_or, seq), (k, nr, nr_or)
        F, res = oracle_mod.solve_sequence_step(seq.n, seq.rowptr, seq.colind, v, P, Q, b)
        assert res.status == 0
        info = s.info()
        assert abs(it - res.iters) <= max(1, info["last_cycles"], res.cycles), (k, it, res.iters)


def test_solve_device_arrays_and_determinism(c1):
    import torch
    seq, P, Q = c1
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    v = seq.values(4)
    b, _ = seq.rhs(4, v)
    s.refactor(torch.from_numpy(v).cuda())
    bd = torch.from_numpy(b).cuda()
    x1, it1, _ = s.solve(bd)
    x2, it2, _ = s.solve(bd, x=torch.empty_like(bd))
    xh, ith, _ = s.solve(b)
    assert it1 == it2 == ith
    assert torch.equal(x1, x2)
    assert np.array_equal(x1.cpu().numpy(), xh)


def test_lu_solve_backward_error(c1):
    """x0 from the GPU factors solves L U x' = P b with componentwise backward
    error of order eps (triangular solves are componentwise stable)."""
    seq, P, Q = c1
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    v = seq.values(3)
    b, _ = seq.rhs(3, v)
    s.refactor(v)
    x = s.lu_solve(b)
    f = s.factors()
    n = seq.n
    Lm = sp.csc_matrix((f["Lx"], f["Li"], f["Lp"]), shape=(n, n)) + sp.identity(n)
    Um = sp.csc_matrix((f["Ux"], f["Ui"], f["Up"]), shape=(n, n))
    xp = x[Q]
    r = b[P] - Lm @ (Um @ xp)
    scale = abs(Lm) @ (abs(Um) @ abs(xp)) + abs(b[P])
    assert np.max(np.abs(r) / scale) <= 64 * EPS * 10


@pytest.mark.parametrize("sched", ["auto", "global"])
def test_lu_solve_elementwise_well_conditioned(oracle_mod, sched):
    n = 1500
    rp, ci, v = small_random_sparse(n, 0.004, 7, diag_boost=6.0)
    P, Q, F = oracle_mod.lu(n, rp, ci, v)
    s = K.KKTSolver(trisolve=sched)
    s.analyze(rp, ci, Q=Q, P=P)
    s.refactor(v)
    b = np.random.default_rng(3).standard_normal(n)
    xg = s.lu_solve(b)
    xo = oracle_mod.solve(F, P, Q, b)
    assert np.max(np.abs(xg - xo)) <= 1e-12 * np.max(np.abs(xo))


def test_matvec_parity(oracle_mod, c1):
    seq, P, Q = c1
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    v = seq.values(2)
    s.refactor(v)
    x = np.random.default_rng(1).standard_normal(seq.n)
    y = s.matvec(x)
    yo = -oracle_mod.residual(seq.n, seq.rowptr, seq.colind, v, np.zeros(seq.n), x)
    # dot-product rounding bound: (terms + 1) eps sum_j |K_ij x_j|
    A = sp.csr_matrix((np.abs(v), seq.colind, seq.rowptr), shape=(seq.n, seq.n))
    terms = np.diff(seq.rowptr) + 1
    assert np.all(np.abs(y - yo) <= terms * EPS * (A @ np.abs(x)))


def _edge_cases():
    n = 300
    rng = np.random.default_rng(11)
    cases = {}
    cases["diagonal"] = sp.diags(rng.uniform(1, 2, n))
    cases["bidiagonal_chain"] = sp.diags([rng.uniform(1, 2, n), rng.uniform(-1, 1, n - 1)], [0, -1])
    A = sp.lil_matrix((n, n))
    A.setdiag(rng.uniform(n, 2 * n, n))
    A[0, :] = rng.uniform(-1, 1, n)
    A[:, 0] = rng.uniform(-1, 1, (n, 1))
    A[0, 0] = 3.0 * n
    cases["arrow"] = A.tocsr()
    S = sp.lil_matrix((n, n))
    S.setdiag(rng.uniform(1, 2, n))
    S[n - 1, :] = rng.uniform(-1, 1, n)
    S[n - 1, n - 1] = 10.0
    cases["star_one_wide_level"] = S.tocsr()
    cases["n1"] = sp.csr_matrix(np.array([[2.5]]))
    D = sp.random(n, n, density=0.3, random_state=5) + sp.identity(n) * 3
    cases["dense_column_block"] = D.tocsr()
    return cases


@pytest.mark.parametrize("sched", ["auto", "global"])
@pytest.mark.parametrize("name", list(_edge_cases().keys()))
def test_edge_structures(oracle_mod, name, sched):
    A = _edge_cases()[name]
    rp, ci, v = csr_of(A)
    n = len(rp) - 1
    P, Q, _ = oracle_mod.lu(n, rp, ci, v)
    s = K.KKTSolver(trisolve=sched)
    s.analyze(rp, ci, Q=Q, P=P)
    s.refactor(v)
    of = oracle_mod.refactor(n, rp, ci, v, P, Q)
    dl, du = factor_diff(s.factors(), of)
    assert dl <= FACTOR_TOL and du <= FACTOR_TOL
    b = np.random.default_rng(n).standard_normal(n)
    x, it, nr = s.solve(b)
    assert oracle_mod.nrbe(n, rp, ci, v, b, x) <= NRBE_TOL


def test_random_nonsymmetric_sparse(oracle_mod):
    for seed in range(3):
        n = 800 + 300 * seed
        rp, ci, v = small_random_sparse(n, 3.0 / n, 100 + seed, diag_boost=1.0)
        P, Q, _ = oracle_mod.lu(n, rp, ci, v)
        s = K.KKTSolver()
        s.analyze(rp, ci, Q=Q, P=P)
        v2 = v * (1 + 0.1 * np.random.default_rng(seed).standard_normal(len(v)))
        s.refactor(v2)
        of = oracle_mod.refactor(n, rp, ci, v2, P, Q)
        dl, du = factor_diff(s.factors(), of)
        assert dl <= FACTOR_TOL and du <= FACTOR_TOL
        b = np.random.default_rng(seed).standard_normal(n)
        x, _, _ = s.solve(b)
        assert oracle_mod.nrbe(n, rp, ci, v2, b, x) <= NRBE_TOL


def test_zero_pivot_error_and_boost(oracle_mod):
    A0 = np.array([[2.0, 1.0], [1.0, 3.0]])
    rp, ci, v0 = csr_of(A0)
    P, Q, _ = oracle_mod.lu(2, rp, ci, v0, Q=np.arange(2, dtype=np.int32), tol=1e-3)
    v1 = np.array([0.0, 1.0, 1.0, 3.0])
    s = K.KKTSolver()
    s.analyze(rp, ci, Q=Q, P=P)
    with pytest.raises(K.KKTError) as e:
        s.refactor(v1)
    assert e.value.code == -4
    # ||K||_inf of v1 is 4: boost_eps 2.5e-9 makes the boost 1e-8
    s2 = K.KKTSolver(boost_eps=2.5e-9)
    s2.analyze(rp, ci, Q=Q, P=P)
    s2.refactor(v1)
    assert s2.info()["nboost"] == 1
    of = oracle_mod.refactor(2, rp, ci, v1, P, Q, 1e-8)
    f = s2.factors()
    assert np.array_equal(f["Ux"], of.Ux) and np.array_equal(f["Lx"], of.Lx)


def test_nonfinite_values_rejected(c1):
    seq, P, Q = c1
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    v = seq.values(0)
    v[17] = np.nan
    with pytest.raises(K.KKTError) as e:
        s.refactor(v)
    assert e.value.code == -5
    with pytest.raises(K.KKTError) as e:   # no factors after a failed refactor
        s.solve(np.ones(seq.n))
    assert e.value.code == -9


def test_rr_stop_mode_and_refine_delta(oracle_mod, c1):
    seq, P, Q = c1
    v = seq.values(6)
    b, _ = seq.rhs(6, v)
    s = K.KKTSolver(stop_mode="rr")
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    s.refactor(v)
    x, it, nr = s.solve(b, tol=1e-10)
    F, res = oracle_mod.solve_sequence_step(seq.n, seq.rowptr, seq.colind, v, P, Q, b, tol=1e-10, stop_mode=1)
    assert abs(it - res.iters) <= max(1, res.cycles)
    s3 = K.KKTSolver(refine_delta=1e6)
    s3.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    s3.refactor(v)
    x3, it3, _ = s3.solve(b, tol=1e-16)
    assert it3 == 0
    assert np.array_equal(x3, s3.lu_solve(b))


@pytest.mark.parametrize("sched", ["auto", "global"])
def test_own_analysis_full_size_kkt2000_sequence(oracle_mod, sched):
    """The benchmark's configuration: the library's own ordering and pivots,
    FGMRES(20), every matrix of the 30-step sequence; NRBE of each returned x
    evaluated by the oracle."""
    seq = KKTSequence("kkt2000")
    s = K.KKTSolver(restart=20, trisolve=sched)
    s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    if sched == "auto":
        assert s.info()["trisolve_cluster"] > 0   # the bench's schedule
    for k in range(seq.M):
        v = seq.values(k)
        b, _ = seq.rhs(k, v)
        s.refactor(v)
        x, it, nr = s.solve(b, tol=NRBE_TOL)
        assert oracle_mod.nrbe(seq.n, seq.rowptr, seq.colind, v, b, x) <= NRBE_TOL, k


def test_refactor_parity_kkt2000_oracle_pivots(oracle_mod):
    """Full-size factor parity on the oracle's own P, Q (first and last matrix)."""
    seq = KKTSequence("kkt2000")
    P, Q, _ = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, seq.values(0))
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    for k in (0, seq.M - 1):
        v = seq.values(k)
        s.refactor(v)
        of = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, v, P, Q)
        dl, du = factor_diff(s.factors(), of)
        assert dl <= FACTOR_TOL and du <= FACTOR_TOL, (k, dl, du)
