"""Failure detection on the GPU without faulting it: every device wait is
bounded; a wait that runs out reports KKT_ERR_TIMEOUT and the context keeps
working.  Zero pivots and non-finite values are covered in the parity file."""
import numpy as np
import pytest

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence

pytestmark = pytest.mark.gpu


def test_bounded_wait_reports_timeout_and_context_survives():
    seq = KKTSequence("kkt200", buses=40, steps=2)
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    assert s.selftest_wait(2000) == -7          # a flag nothing sets: gives up
    assert s.selftest_wait(0) == -7
    v = seq.values(1)
    b, _ = seq.rhs(1, v)
    s.refactor(v)
    x, it, nr = s.solve(b)                      # the context still works
    assert nr <= 1e-12
    assert s.selftest_wait(1000) == -7
    x2, _, _ = s.solve(b)
    assert np.array_equal(x, x2)


def test_tiny_spin_limit_fails_cleanly_or_succeeds():
    """With a spin limit of one poll, a dependency that is not ready yet
    makes the call fail with KKT_ERR_TIMEOUT instead of hanging; whatever
    happens, a context with the default limit solves afterwards."""
    seq = KKTSequence("kkt200", buses=60, steps=2)
    v = seq.values(1)
    b, _ = seq.rhs(1, v)
    s = K.KKTSolver(spin_limit=1)
    s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    try:
        s.refactor(v)
        s.solve(b)
    except K.KKTError as e:
        assert e.code == -7
    s2 = K.KKTSolver()
    s2.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    s2.refactor(v)
    _, _, nr = s2.solve(b)
    assert nr <= 1e-12
