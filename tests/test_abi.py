"""CPU checks of the C ABI library: it loads, exports every entry point
declared in include/kkt.h, and its host-only analysis (ordering, pivoting)
behaves.  No GPU calls."""
import os
import re

import numpy as np
import pytest

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def L():
    from paper_2401_13926_b300 import build
    build.build()
    return K.lib()


def declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", f)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(kkt_[a-z_0-9]+)\s*\(", txt))
    return names


def test_library_exports_every_declared_symbol(L):
    names = declared()
    assert names, "no declarations found"
    for nm in sorted(names):
        assert hasattr(L, nm), nm
    assert set(K.EXPORTS) <= names


def test_strerror_covers_codes(L):
    for code in range(0, -10, -1):
        assert L.kkt_strerror(code).decode() != "unknown error"


def test_order_is_a_permutation_with_fill_close_to_oracle(L, oracle_mod):
    seq = KKTSequence("kkt200")
    Q = K.order(seq.rowptr, seq.colind)
    assert sorted(Q) == list(range(seq.n))
    v = seq.values(0)
    _, _, Fl = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, v, Q=Q)
    _, _, Fo = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, v)
    fill_lib = len(Fl.Li) + len(Fl.Ui)
    fill_or = len(Fo.Li) + len(Fo.Ui)
    assert fill_lib <= 1.5 * fill_or


def test_pivot_matches_oracle_pivot_rule(L, oracle_mod):
    """Same order, same threshold rule -> same pivot sequence and sizes."""
    seq = KKTSequence("kkt200", buses=60, steps=1)
    v = seq.values(0)
    Po, Qo, Fo = oracle_mod.lu(seq.n, seq.rowptr, seq.colind, v)
    P, nl, nu = K.pivot(seq.rowptr, seq.colind, v, Q=Qo, tol=1e-3)
    assert np.array_equal(P, Po)
    assert nl == len(Fo.Li) and nu == len(Fo.Ui)


def test_pattern_errors(L):
    rp = np.array([0, 2, 3], np.int32)
    with pytest.raises(K.KKTError) as e:
        K.order(rp, np.array([0, 0, 1], np.int32))       # duplicate in row 0
    assert e.value.code == -2
    with pytest.raises(K.KKTError) as e:
        K.order(rp, np.array([0, 5, 1], np.int32))       # out of range
    assert e.value.code == -2
    with pytest.raises(K.KKTError) as e:
        K.pivot(np.array([0, 1, 2], np.int32), np.array([0, 0], np.int32), np.array([1.0, 1.0]))
    assert e.value.code == -4                              # column 1 is empty: no pivot


def test_host_analyze_equals_order_then_pivot(L, oracle_mod):
    """kkt_host_analyze (no GPU) returns the order and pivots of kkt_order +
    kkt_pivot, and its statistics describe the oracle's factorization on
    them: the same factor sizes, and the multiply-add count of the
    left-looking refactorization (the oracle's own count on the same P, Q)."""
    seq = KKTSequence("kkt200", buses=60, steps=1)
    v = seq.values(0)
    P, Q, st = K.host_analyze(seq.rowptr, seq.colind, v)
    Q2 = K.order(seq.rowptr, seq.colind)
    P2, nl, nu = K.pivot(seq.rowptr, seq.colind, v, Q=Q2)
    assert np.array_equal(Q, Q2) and np.array_equal(P, P2)
    assert st["nnz_l"] == nl and st["nnz_u"] == nu
    F = oracle_mod.refactor(seq.n, seq.rowptr, seq.colind, v, P, Q)
    assert len(F.Li) == nl and len(F.Ui) == nu
    cols, madds, _, _ = oracle_mod.refactor_sample(seq.n, seq.rowptr, seq.colind, v, P, Q, 1e9)
    assert cols == seq.n and madds == st["refactor_updates"]
    assert st["levels_l"] >= 1 and st["levels_u"] >= 1


def test_instance_placement_rule(L):
    """kkt_place_instance (no GPU): the device with the most budget left
    among those whose budget can hold the instance at all, ties to the
    lower index; -1 when no device could ever hold it.  Placing a stream of
    instances spreads them so no device's held bytes exceed another's by
    more than the largest instance."""
    assert K.place_instance([10, 10, 10], [5, 2, 2], 3) == 1
    assert K.place_instance([10, 20, 10], [0, 15, 0], 3) == 0
    assert K.place_instance([10, 4, 30], [0, 0, 29], 5) == 0   # device 1 too small, 2 fullest
    assert K.place_instance([10, 10], [12, 11], 3) == 1        # all over budget: still the least held
    assert K.place_instance([10, 10], [0, 0], 11) == -1
    rng = np.random.default_rng(0)
    budget = np.array([1000, 1000, 1000, 1000], np.int64)
    held = np.zeros(4, np.int64)
    sizes = rng.integers(10, 60, size=200)
    for need in sizes:
        d = K.place_instance(budget, held, int(need))
        assert 0 <= d < 4
        held[d] += need
    assert held.max() - held.min() <= sizes.max()
