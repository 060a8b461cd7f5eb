"""kkt_step: refactor + solve with the forward sweep fused into the
refactorization.  The fused y is computed with the separate sweep's row
arithmetic, so every result must equal refactor() followed by solve() bit
for bit -- factors, solution, iteration count and NRBE -- on every schedule,
in both precisions, with host and device arrays, and with refinement
iterations after the fused initial solve."""
import numpy as np
import pytest

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence, small_random_sparse

pytestmark = pytest.mark.gpu


def _pair(rp, ci, v0=None, P=None, Q=None, **kw):
    out = []
    for _ in range(2):
        s = K.KKTSolver(**kw)
        if P is None:
            s.analyze(rp, ci, values0=v0)
        else:
            s.analyze(rp, ci, Q=Q, P=P)
        out.append(s)
    return out


@pytest.mark.parametrize("kw", [dict(), dict(trisolve="global"), dict(precision="mixed", max_cycles=2),
                                dict(warp_rows=False), dict(block_smem=8192)])
def test_step_equals_refactor_then_solve_kkt200(kw):
    seq = KKTSequence("kkt200")
    a, f = _pair(seq.rowptr, seq.colind, seq.values(0), **kw)
    for k in range(seq.M):
        v = seq.values(k)
        b, _ = seq.rhs(k, v)
        a.refactor(v)
        xa, ia, na = a.solve(b, tol=1e-12, allow_not_converged=True)
        xf, i_f, nf = f.step(v, b, tol=1e-12, allow_not_converged=True)
        assert a.last_status == f.last_status
        assert np.array_equal(xa, xf), k
        assert ia == i_f and na == nf
        fa, ff = a.factors(), f.factors()
        assert np.array_equal(fa["Ux"], ff["Ux"]) and np.array_equal(fa["Lx"], ff["Lx"])


def test_step_with_refinement_iterations(oracle_mod):
    n = 2000
    rp, ci, v = small_random_sparse(n, 4.0 / n, 23, diag_boost=1.0)
    P, Q, _ = oracle_mod.lu(n, rp, ci, v)
    a, f = _pair(rp, ci, P=P, Q=Q, boost_eps=1e-3)
    b = np.random.default_rng(3).standard_normal(n)
    a.refactor(v)
    xa, ia, na = a.solve(b, tol=1e-12)
    xf, i_f, nf = f.step(v, b, tol=1e-12)
    assert ia == i_f and ia >= 5 and np.array_equal(xa, xf)


def test_step_device_arrays_and_full_size():
    import torch
    seq = KKTSequence("kkt2000", steps=4)
    a, f = _pair(seq.rowptr, seq.colind, seq.values(0))
    for k in range(seq.M):
        v = torch.from_numpy(seq.values(k)).cuda()
        b = torch.from_numpy(seq.rhs(k, seq.values(k))[0]).cuda()
        xa, xf = torch.empty_like(b), torch.empty_like(b)
        a.refactor(v)
        _, ia, na = a.solve(b, x=xa, tol=1e-12)
        _, i_f, nf = f.step(v, b, x=xf, tol=1e-12)
        torch.cuda.synchronize()
        assert torch.equal(xa, xf) and ia == i_f and na == nf
    # a plain solve after a step recomputes y itself
    xf2 = torch.empty_like(b)
    f.solve(b, x=xf2, tol=1e-12)
    torch.cuda.synchronize()
    assert torch.equal(xf2, xf)


@pytest.mark.parametrize("warp_rows,block_smem", [(True, 0), (False, 0), (True, 8192), (False, 8192),
                                                  (False, 150000), (True, 150000)])
def test_row_placement_and_order_same_bits(oracle_mod, warp_rows, block_smem):
    """Every placement of the refactorization's rows -- one per warp in
    shared memory, one per block in shared memory, one per half of a
    512-thread block (a 150 KB block makes the blocks 512 threads wide),
    one per block with the values in global memory (an 8 KB block forces
    the longest kkt200 rows there) -- every dispatch order (DAG level, row,
    critical-path priority) and both times a block row may store its last
    step's values (as each is formed, or after the step) give the same
    factors, bit for bit, equal to the oracle's refactorization on the same
    P and Q (each row's arithmetic is fixed; only where and when it runs
    changes)."""
    seq = KKTSequence("kkt200", steps=2)
    out = []
    runs = [("row", True, True), ("level", True, True), ("level", False, True), ("critical", True, True)]
    if block_smem == 150000:
        runs.append(("level", True, False))   # the same rows one per whole block
    for order, stream_last, team_rows in runs:
        s = K.KKTSolver(row_order=order, warp_rows=warp_rows, block_smem=block_smem, stream_last=stream_last,
                        team_rows=team_rows)
        s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
        info = s.info()
        assert info["rows_warp"] + info["rows_block"] + info["rows_global"] + info["rows_team"] == seq.n
        assert (info["rows_warp"] > 0) == warp_rows
        if block_smem:
            assert info["refactor_smem"] == block_smem
        assert (info["rows_global"] > 0) == (block_smem == 8192)
        if block_smem == 150000:
            assert info["refactor_threads"] == 512
            if not team_rows:
                assert info["rows_team"] == 0
            elif not warp_rows:
                assert info["rows_team"] > 0
        else:
            assert info["rows_team"] == 0
        v = seq.values(1)
        b, _ = seq.rhs(1, v)
        x, it, nr = s.step(v, b)
        f = s.factors()
        out.append((f["Lx"].copy(), f["Ux"].copy(), x.copy(), it, nr))
        P, Q = s.perm()
        s.close()
    for o in out[1:]:
        for a, b_ in zip(out[0], o):
            assert np.array_equal(a, b_)
    of = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, seq.values(1), P, Q)
    assert np.array_equal(out[0][0], of.Lx) and np.array_equal(out[0][1], of.Ux)


def test_step_factors_bitwise_oracle_full_size_kkt2000(oracle_mod):
    """The benchmark's timed call at its size: kkt_step on the library's own
    ordering and pivots gives factors equal, bit for bit, to the oracle's
    refactorization on the same P and Q (first and last matrix), whatever
    the dispatch order of the rows and the time block rows store their last
    step's values."""
    seq = KKTSequence("kkt2000")
    for order, stream_last in (("level", True), ("row", False)):
        s = K.KKTSolver(row_order=order, stream_last=stream_last)
        s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
        P, Q = s.perm()
        for k in (0, seq.M - 1):
            v = seq.values(k)
            b, _ = seq.rhs(k, v)
            s.step(v, b, allow_not_converged=True)
            f = s.factors()
            of = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, v, P, Q)
            assert np.array_equal(f["Li"], of.Li) and np.array_equal(f["Ui"], of.Ui)
            assert np.array_equal(f["Lx"], of.Lx), (order, k)
            assert np.array_equal(f["Ux"], of.Ux), (order, k)
        s.close()
