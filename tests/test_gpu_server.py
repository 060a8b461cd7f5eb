"""Serving runtime (kkt_server_*): many resident KKT sequences with their
steps in flight together.  Each result must equal, bit for bit, the same
step run alone on a solver of its own (the sequences are independent and
every step runs the same kernels in the same order); steps of one instance
run in submission order; admission keeps the device memory within budget;
a failing step reports its error without disturbing the others."""
import numpy as np
import pytest

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence, small_random_sparse

pytestmark = pytest.mark.gpu


def _alone(rp, ci, v0, steps, tol=1e-12):
    s = K.KKTSolver()
    s.analyze(rp, ci, values0=v0)
    out = []
    for v, b in steps:
        s.refactor(v)
        x, it, nr = s.solve(b, tol=tol)
        out.append((x.copy(), it, nr))
    s.close()
    return out


def test_mix_equals_alone():
    cases = []
    for inst in range(3):
        seq = KKTSequence("kkt200", instance=inst, steps=4)
        steps = [(seq.values(k), seq.rhs(k, seq.values(k))[0]) for k in range(seq.M)]
        cases.append((seq.rowptr, seq.colind, seq.values(0), steps))
    rp, ci, v = small_random_sparse(1500, 4.0 / 1500, 5, diag_boost=1.0)
    rng = np.random.default_rng(0)
    steps = [(v * (1 + 0.01 * rng.standard_normal(len(v))), rng.standard_normal(1500)) for _ in range(4)]
    cases.append((rp, ci, v, steps))
    srv = K.KKTServer(workers=4)
    ids = [srv.open(rp_, ci_, v0) for rp_, ci_, v0, _ in cases]
    tickets = []
    for k in range(4):                  # interleaved submission across instances
        for i, (_, _, _, st) in enumerate(cases):
            tickets.append((i, k, srv.submit(ids[i], st[k][0], st[k][1])[0]))
    got = {}
    for i, k, t in tickets:
        x, r = srv.wait(t)
        assert r["status"] == 0, (i, k, r)
        got[(i, k)] = (x, r)
    info = srv.info()
    assert info["submitted"] == info["completed"] == 16 and info["in_flight"] == 0
    for i, (rp_, ci_, v0, st) in enumerate(cases):
        ref = _alone(rp_, ci_, v0, st)
        for k in range(4):
            x, r = got[(i, k)]
            assert np.array_equal(x, ref[k][0]), (i, k)
            assert r["iters"] == ref[k][1] and r["nrbe"] == ref[k][2]
    srv.close()


def test_admission_by_device_memory():
    seq = KKTSequence("kkt200", steps=2)
    probe = K.KKTSolver()
    probe.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    one = probe.info()["device_bytes"]
    probe.close()
    srv = K.KKTServer(workers=2, hbm_budget=int(1.5 * one))
    a = srv.open(seq.rowptr, seq.colind, seq.values(0))
    with pytest.raises(K.KKTError) as e:
        srv.open(seq.rowptr, seq.colind, seq.values(0))
    assert e.value.code == -3
    assert srv.info()["instances"] == 1 and srv.info()["device_bytes"] == one
    srv.close_instance(a)
    b = srv.open(seq.rowptr, seq.colind, seq.values(0))
    t, _ = srv.submit(b, seq.values(1), seq.rhs(1, seq.values(1))[0])
    x, r = srv.wait(t)
    assert r["status"] == 0
    srv.close()


def test_failing_step_is_reported_and_isolated():
    seq = KKTSequence("kkt200", steps=3)
    srv = K.KKTServer(workers=3)
    a = srv.open(seq.rowptr, seq.colind, seq.values(0))
    b = srv.open(seq.rowptr, seq.colind, seq.values(0))
    bad = seq.values(1).copy()
    bad[7] = np.nan
    rhs = seq.rhs(1, seq.values(1))[0]
    ta, _ = srv.submit(a, bad, rhs)
    tb, _ = srv.submit(b, seq.values(1), rhs)
    ta2, _ = srv.submit(a, seq.values(2), seq.rhs(2, seq.values(2))[0])
    assert srv.wait(ta)[1]["status"] == -5            # KKT_ERR_NONFINITE
    xb, rb = srv.wait(tb)
    assert rb["status"] == 0
    xa2, ra2 = srv.wait(ta2)                            # the instance recovers on its next step
    assert ra2["status"] == 0
    ref = _alone(seq.rowptr, seq.colind, seq.values(0), [(seq.values(1), rhs)])
    assert np.array_equal(xb, ref[0][0])
    srv.close()
