"""CUDA graphs (kkt_opts.graphs): the refactorization replayed as one graph,
and the whole refinement -- restart cycles and Arnoldi steps, or the
corrections of classical refinement -- as one graph whose loops run on the
device (conditional WHILE/IF nodes set by the decision kernels).  The graphs
hold the same kernels in the same order as the host-driven path, so every
result must be bit-identical to it, including iteration counts, the
non-converged outcome and the launch count."""
import numpy as np
import pytest

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence, small_random_sparse

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def c1(oracle_mod):
    seq = KKTSequence("kkt200")
    P, Q, _ = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, seq.values(0))
    return seq, P, Q


def _pair(rp, ci, P, Q, **kw):
    out = []
    for graphs in (False, True):
        s = K.KKTSolver(graphs=graphs, **kw)
        s.analyze(rp, ci, Q=Q, P=P)
        out.append(s)
    return out


@pytest.mark.parametrize("kw", [dict(), dict(stop_mode="rr"), dict(method="fgmres_ee", inner_tol=1e-3),
                                dict(ortho="cgs2_pythagoras"), dict(ortho="cgs1_pythagoras"),
                                dict(trisolve="global"), dict(precision="mixed", max_cycles=2)])
def test_graph_solves_equal_host_driven_kkt200(c1, kw):
    seq, P, Q = c1
    a, g = _pair(seq.rowptr, seq.colind, P, Q, **kw)
    tol = 1e-10 if kw.get("stop_mode") == "rr" else 1e-12
    for k in range(seq.M):
        v = seq.values(k)
        b, _ = seq.rhs(k, v)
        a.refactor(v)
        g.refactor(v)
        fa, fg = a.factors(), g.factors()
        assert np.array_equal(fa["Lx"], fg["Lx"]) and np.array_equal(fa["Ux"], fg["Ux"])
        la, lg = a.info()["launches"], g.info()["launches"]
        xa, ia, na = a.solve(b, tol=tol, allow_not_converged=True)
        xg, ig, ng = g.solve(b, tol=tol, allow_not_converged=True)
        assert a.last_status == g.last_status, k
        assert ia == ig and na == ng, (k, ia, ig)
        assert np.array_equal(xa, xg), k
        assert a.info()["last_cycles"] == g.info()["last_cycles"]
        assert a.info()["launches"] - la == g.info()["launches"] - lg


def _boosted(oracle_mod, seed=23, n=2000):
    rp, ci, v = small_random_sparse(n, 4.0 / n, seed, diag_boost=1.0)
    P, Q, _ = oracle_mod.lu(n, rp, ci, v)
    return n, rp, ci, v, P, Q


@pytest.mark.parametrize("kw", [dict(), dict(method="richardson"), dict(restart=3, max_cycles=2)])
def test_graph_loops_with_many_iterations(oracle_mod, kw):
    """Several cycles, hundreds of corrections, and a run that stops at its
    cycle cap (KKT_ERR_NOT_CONVERGED) give the host-driven results."""
    n, rp, ci, v, P, Q = _boosted(oracle_mod)
    a, g = _pair(rp, ci, P, Q, boost_eps=1e-3, **kw)
    a.refactor(v)
    g.refactor(v)
    b = np.random.default_rng(4).standard_normal(n)
    xa, ia, na = a.solve(b, tol=1e-12, allow_not_converged=True)
    xg, ig, ng = g.solve(b, tol=1e-12, allow_not_converged=True)
    assert a.last_status == g.last_status
    if kw.get("max_cycles") == 2:
        assert g.last_status == K.ERR_NOT_CONVERGED
    assert ia == ig and na == ng and ia > 0
    assert np.array_equal(xa, xg)


def test_graph_device_arrays_and_tolerance_change(c1):
    import torch
    seq, P, Q = c1
    a, g = _pair(seq.rowptr, seq.colind, P, Q)
    v = seq.values(3)
    b, _ = seq.rhs(3, v)
    vd, bd = torch.from_numpy(v).cuda(), torch.from_numpy(b).cuda()
    a.refactor(vd)
    g.refactor(vd)
    for tol in (1e-12, 1e-14, 1e-12):      # a new tol re-captures the solve graph
        xa = torch.empty_like(bd)
        xg = torch.empty_like(bd)
        _, ia, _ = a.solve(bd, x=xa, tol=tol, allow_not_converged=True)
        _, ig, _ = g.solve(bd, x=xg, tol=tol, allow_not_converged=True)
        torch.cuda.synchronize()
        assert ia == ig and torch.equal(xa, xg)
    # the graph path still solves after a re-analysis (graphs are rebuilt)
    g.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
    g.refactor(vd)
    xg = torch.empty_like(bd)
    g.solve(bd, x=xg, tol=1e-12)
    torch.cuda.synchronize()
    a.solve(bd, x=xa, tol=1e-12)
    torch.cuda.synchronize()
    assert torch.equal(xa, xg)
