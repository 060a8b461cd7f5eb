"""kkt_batch_step: one step of several instances in shared launches (one
refactorization launch over every instance's work items, one cluster
launch for the backward sweeps).  Each instance's result must be the one
it gets alone -- x, iterations and NRBE bit for bit against a twin context
running kkt_step -- with host and device arrays, across instances of
different sizes (so different cluster shapes and block sizes, which take
the per-instance sweep or a lone step), and a failing instance must not
disturb the others.  Solutions also meet NRBE <= 1e-12 as the oracle
evaluates Eq. (nbre)."""
import numpy as np
import pytest

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence

pytestmark = pytest.mark.gpu


def _fleet(specs, **kw):
    seqs, batch_side, alone_side = [], [], []
    for name, inst, buses in specs:
        q = KKTSequence(name, instance=inst, buses=buses, steps=3)
        a = K.KKTSolver(**kw)
        a.analyze(q.rowptr, q.colind, values0=q.values(0))
        t = K.KKTSolver(**kw)
        t.analyze_like(a)
        seqs.append(q)
        batch_side.append(a)
        alone_side.append(t)
    return seqs, batch_side, alone_side


@pytest.mark.parametrize("device_arrays", [False, True])
def test_batch_equals_alone_same_size(oracle_mod, device_arrays):
    import torch
    seqs, bs, al = _fleet([("kkt200", i, None) for i in range(4)])
    bt = K.KKTBatch(8)
    for k in range(3):
        v = [q.values(k) for q in seqs]
        b = [q.rhs(k, vv)[0] for q, vv in zip(seqs, v)]
        if device_arrays:
            vd = [torch.from_numpy(a).cuda() for a in v]
            bd = [torch.from_numpy(a).cuda() for a in b]
            xs, it, nr, st = bt.step(bs, vd, bd)
            torch.cuda.synchronize()
            xs = [x.cpu().numpy() for x in xs]
        else:
            xs, it, nr, st = bt.step(bs, v, b)
        assert list(st) == [0] * len(bs)
        for i, s in enumerate(al):
            x1, i1, n1 = s.step(v[i], b[i])
            assert np.array_equal(xs[i], x1) and it[i] == i1 and nr[i] == n1, (k, i)
            q = seqs[i]
            assert oracle_mod.nrbe(q.n, q.rowptr, q.colind, v[i], b[i], xs[i]) <= 1e-12
    assert bt.launches() >= 3 * 6


def test_batch_mixed_sizes_and_precisions(oracle_mod):
    """kkt200 and kkt2000-sized instances (different cluster shapes) plus a
    mixed-precision one (a lone step): every result equals its twin's."""
    specs = [("kkt200", 10, None), ("kkt2000", 11, 900), ("kkt200", 12, 120), ("kkt2000", 13, 1500)]
    seqs, bs, al = _fleet(specs)
    q = KKTSequence("kkt200", instance=14, steps=3)
    m = K.KKTSolver(precision="mixed")
    m.analyze(q.rowptr, q.colind, values0=q.values(0))
    mt = K.KKTSolver(precision="mixed")
    mt.analyze_like(m)
    seqs.append(q)
    bs.append(m)
    al.append(mt)
    bt = K.KKTBatch(16)
    for k in range(3):
        v = [s.values(k) for s in seqs]
        b = [s.rhs(k, vv)[0] for s, vv in zip(seqs, v)]
        xs, it, nr, st = bt.step(bs, v, b)
        assert list(st) == [0] * len(bs)
        for i, s in enumerate(al):
            x1, i1, n1 = s.step(v[i], b[i])
            assert np.array_equal(xs[i], x1) and it[i] == i1 and nr[i] == n1, (k, i)
            sq = seqs[i]
            assert oracle_mod.nrbe(sq.n, sq.rowptr, sq.colind, v[i], b[i], xs[i]) <= 1e-12


def test_batch_failure_is_isolated():
    """An instance whose matrix has an exact zero pivot reports
    KKT_ERR_ZERO_PIVOT; the others in the same launches are unaffected and
    keep stepping."""
    seqs, bs, al = _fleet([("kkt200", 20 + i, None) for i in range(3)])
    bt = K.KKTBatch(4)
    for k in range(2):
        v = [q.values(k) for q in seqs]
        b = [q.rhs(k, vv)[0] for q, vv in zip(seqs, v)]
        v[1] = np.zeros_like(v[1])   # every pivot of instance 1 is zero
        xs, it, nr, st = bt.step(bs, v, b)
        assert st[1] == -4 and st[0] == 0 and st[2] == 0
        for i in (0, 2):
            x1, i1, n1 = al[i].step(v[i], b[i])
            assert np.array_equal(xs[i], x1) and nr[i] == n1


def test_batch_rejects_repeated_instance():
    seqs, bs, _ = _fleet([("kkt200", 30, 60)])
    bt = K.KKTBatch(4)
    v = seqs[0].values(0)
    b = seqs[0].rhs(0, v)[0]
    with pytest.raises(K.KKTError) as e:
        bt.step([bs[0], bs[0]], [v, v], [b, b])
    assert e.value.code == -1
