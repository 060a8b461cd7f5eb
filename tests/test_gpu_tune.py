"""Autotuner (kkt_tune): it times the refactorization/solve schedules on
the caller's matrix and keeps the fastest.  All schedules compute the same
bits, so the solution after tuning equals the solution before it."""
import numpy as np
import pytest

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("name", ["kkt200", "kkt2000"])
def test_tune_keeps_results_and_reports_choice(name):
    seq = KKTSequence(name, steps=3)
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    v = seq.values(2)
    b, _ = seq.rhs(2, v)
    s.refactor(v)
    x0, it0, nr0 = s.solve(b, tol=1e-12)
    f0 = s.factors()
    best = s.tune(v, b, reps=2)
    assert best > 0
    info = s.info()
    assert info["refactor_smem"] > 0 and info["trisolve_cluster"] in (0, 8, 16)
    assert info["rows_warp"] + info["rows_block"] + info["rows_global"] + info["rows_team"] == seq.n
    with pytest.raises(K.KKTError):      # factors must be recomputed after tuning
        s.solve(b, tol=1e-12)
    s.refactor(v)
    f1 = s.factors()
    assert np.array_equal(f0["Lx"], f1["Lx"]) and np.array_equal(f0["Ux"], f1["Ux"])
    x1, it1, nr1 = s.solve(b, tol=1e-12)
    assert np.array_equal(x0, x1) and it0 == it1 and nr0 == nr1


def test_tune_with_device_arrays():
    import torch
    seq = KKTSequence("kkt200", steps=2)
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    v = torch.from_numpy(seq.values(1)).cuda()
    b = torch.from_numpy(seq.rhs(1, seq.values(1))[0]).cuda()
    assert s.tune(v, b, reps=1) > 0
    s.refactor(v)
    x, it, nr = s.solve(b, tol=1e-12)
    torch.cuda.synchronize()
    assert nr <= 1e-12
