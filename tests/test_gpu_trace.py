"""Profiling traces are causal: a row of the refactorization or of a
triangular sweep can publish only after every row it depends on has
published (the GPU's global timer is one clock for all SMs).  This checks
the traces, and through them that the sync-free schedules respect the
dependency DAG of the factors (Section 1.3: refactorization and solves)."""
import numpy as np
import pytest
import scipy.sparse as sp

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def solver():
    seq = KKTSequence("kkt200")
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    v = seq.values(4)
    s.refactor(v)
    return seq, s, v


def _csr(f, n):
    L = sp.csc_matrix((np.ones(len(f["Li"])), f["Li"], f["Lp"]), shape=(n, n)).tocsr()
    U = sp.csc_matrix((np.ones(len(f["Ui"])), f["Ui"], f["Up"]), shape=(n, n)).tocsr()
    return L, U


def test_solve_trace_is_causal(solver):
    seq, s, v = solver
    if s.info()["trisolve_cluster"] == 0:
        pytest.skip("cluster schedule not in use")
    n = seq.n
    b, _ = seq.rhs(4, v)
    x, lL, tL, lU, tU = s.trace_solve(b)
    assert np.array_equal(np.sort(lL), np.arange(n)) and np.array_equal(np.sort(lU), np.arange(n))
    assert np.all(tL > 0) and np.all(tU > 0)
    assert np.array_equal(x, s.lu_solve(b))          # tracing does not change the arithmetic
    L, U = _csr(s.factors(), n)
    pubL = np.empty(n, np.int64); pubL[lL] = tL
    pubU = np.empty(n, np.int64); pubU[lU] = tU
    for i in range(n):
        dl = L.indices[L.indptr[i]:L.indptr[i + 1]]
        assert np.all(pubL[dl] <= pubL[i]), i
        du = U.indices[U.indptr[i]:U.indptr[i + 1]]
        du = du[du > i]
        assert np.all(pubU[du] <= pubU[i]), i
    # the U sweep starts from y, so it starts after the L sweep has ended
    assert tU.min() >= tL.max()


def test_refactor_trace_is_causal(solver):
    seq, s, v = solver
    n = seq.n
    ts, tp, t0 = s.trace_refactor(v)
    assert t0 == 0
    assert np.all(ts > 0) and np.all(tp >= ts)
    L, _ = _csr(s.factors(), n)
    for i in range(n):
        deps = L.indices[L.indptr[i]:L.indptr[i + 1]]
        assert np.all(tp[deps] <= tp[i]), i


def test_refactor_critical_path_matches_its_definition(solver):
    """kkt_trace_critical_path: each row's link is its publish time minus the
    later of its start and its last dependency's publish; the path is the
    longest sum of links along dependency chains.  Recomputed here from the
    same stamps and the factors' pattern."""
    seq, s, v = solver
    n = seq.n
    ts, tp, _ = s.trace_refactor(v)
    cp = s.critical_path(ts, tp)
    L, _ = _csr(s.factors(), n)
    links = np.zeros(n)
    path = np.zeros(n)
    for i in range(n):
        deps = L.indices[L.indptr[i]:L.indptr[i + 1]]
        last = tp[deps].max() if len(deps) else -1
        links[i] = max(tp[i] - max(ts[i], last), 0)
        path[i] = links[i] + (path[deps].max() if len(deps) else 0.0)
    assert cp["rows_stamped"] == n
    assert cp["levels"] == s.info()["levels_l"]
    assert abs(cp["path_ms"] - path.max() * 1e-6) <= 1e-9 * max(1.0, path.max() * 1e-6)
    assert abs(cp["median_link_us"] - np.sort(links)[n // 2] * 1e-3) <= 1e-9
    assert cp["path_ms"] <= (tp.max() - ts.min()) * 1e-6 + 1e-12
