"""Serving runtime (kkt_server_*): many resident KKT sequences with their
steps in flight together, either as batched calls (continuous batching:
one refactorization launch over several instances' rows) or one worker per
step.  Each result must equal, bit for bit, the same step run alone on a
solver of its own; steps of one instance run in submission order;
admission keeps each device's memory within its budget, an open that does
not fit yet waits (first come, first served) until memory is freed; a
failing step reports its error without disturbing the others."""
import threading
import time

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


@pytest.mark.parametrize("batch", [0, 4])
def test_mix_equals_alone(batch):
    cases = []
    for inst in range(3):
        seq = KKTSequence("kkt200", instance=inst, steps=4)
        steps = [(seq.values(k), seq.rhs(k, seq.values(k))[0]) for k in range(seq.M)]
        cases.append((seq.rowptr, seq.colind, seq.values(0), steps))
    rp, ci, v = small_random_sparse(1500, 4.0 / 1500, 5, diag_boost=1.0)
    rng = np.random.default_rng(0)
    steps = [(v * (1 + 0.01 * rng.standard_normal(len(v))), rng.standard_normal(1500)) for _ in range(4)]
    cases.append((rp, ci, v, steps))
    srv = K.KKTServer(workers=4, batch=batch)
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
    if batch:
        assert 0 < info["batches"] <= 16
    for i, (rp_, ci_, v0, st) in enumerate(cases):
        ref = _alone(rp_, ci_, v0, st)
        for k in range(4):
            x, r = got[(i, k)]
            assert np.array_equal(x, ref[k][0]), (i, k)
            assert r["iters"] == ref[k][1] and r["nrbe"] == ref[k][2]
    srv.close()


def test_device_bytes_estimate_is_exact():
    """kkt_estimate_device_bytes (what admission reserves) equals the device
    memory kkt_analyze then holds, in each precision."""
    seq = KKTSequence("kkt200", steps=1)
    P, Q, st = K.host_analyze(seq.rowptr, seq.colind, seq.values(0))
    for kw in (dict(), dict(precision="mixed"), dict(precision="mixed", mixed_fallback=0), dict(restart=10),
               dict(precision="mixed", equilibrate=True)):
        s = K.KKTSolver(**kw)
        s.analyze(seq.rowptr, seq.colind, Q=Q, P=P)
        est = K.estimate_device_bytes(seq.n, seq.nnz, st, canonical_order=bool(st["canonical_order"]), **kw)
        assert s.info()["device_bytes"] == est, kw
        s.close()


def test_admission_waits_for_memory_in_order():
    """A budget for one instance: the second and third opens wait, and are
    admitted in arrival order as the earlier instances close; an instance
    larger than the whole budget is refused at once."""
    seq = KKTSequence("kkt200", steps=2)
    _, _, st = K.host_analyze(seq.rowptr, seq.colind, seq.values(0))
    one = K.estimate_device_bytes(seq.n, seq.nnz, st, canonical_order=bool(st["canonical_order"]))
    srv = K.KKTServer(batch=2, hbm_budget=int(1.5 * one))
    big = KKTSequence("kkt2000", steps=1)
    with pytest.raises(K.KKTError) as e:
        srv.open(big.rowptr, big.colind, big.values(0))
    assert e.value.code == -3
    a = srv.open(seq.rowptr, seq.colind, seq.values(0))
    admitted = []

    def opener(tag):
        inst = srv.open(seq.rowptr, seq.colind, seq.values(0))
        admitted.append((tag, inst))

    tb = threading.Thread(target=opener, args=("b",))
    tb.start()
    while srv.info()["waiting"] < 1:
        time.sleep(0.01)
    tc = threading.Thread(target=opener, args=("c",))
    tc.start()
    while srv.info()["waiting"] < 2:
        time.sleep(0.01)
    assert srv.info()["instances"] == 1 and not admitted
    srv.close_instance(a)
    tb.join(timeout=60)
    assert [t for t, _ in admitted] == ["b"] and srv.info()["waiting"] == 1
    assert srv.info()["device_bytes"] <= srv.info()["hbm_budget"]
    bid = admitted[0][1]
    t, _ = srv.submit(bid, seq.values(1), seq.rhs(1, seq.values(1))[0])
    assert srv.wait(t)[1]["status"] == 0
    srv.close_instance(bid)
    tc.join(timeout=60)
    assert [t for t, _ in admitted] == ["b", "c"] and srv.info()["waiting"] == 0
    srv.close()


@pytest.mark.parametrize("batch", [0, 4])
def test_failing_step_is_reported_and_isolated(batch):
    seq = KKTSequence("kkt200", steps=3)
    srv = K.KKTServer(workers=3, batch=batch)
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
