"""The synthetic KKT generator: shapes, determinism, symmetry, same pattern."""
import numpy as np
import scipy.sparse as sp

from paper_2401_13926_b300.workload import KKTSequence


def test_c1_shape_matches_recipe():
    s = KKTSequence("kkt200")
    assert 0.9 * 5000 <= s.n <= 1.1 * 5000
    assert 0.85 * 60000 <= s.nnz <= 1.15 * 60000
    assert s.M == 10 and s.ngen == 40


def test_pattern_sorted_unique_and_symmetric_values():
    s = KKTSequence("kkt200", buses=30, steps=3)
    rp, ci = s.rowptr, s.colind
    for i in range(s.n):
        row = ci[rp[i]:rp[i + 1]]
        assert np.all(np.diff(row) > 0)
        assert i in row                      # full diagonal
    K = s.csr(1)
    assert abs(K - K.T).max() == 0.0        # K_k is symmetric indefinite
    # (2,2) block is -D_y with D_y in [1e-10, 1e-6]
    d = K.diagonal()[s.nx:]
    assert np.all(d < 0) and np.all(-d >= 1e-10) and np.all(-d <= 1e-6)


def test_deterministic_and_same_pattern_across_steps():
    a = KKTSequence("kkt200", buses=30, steps=3)
    b = KKTSequence("kkt200", buses=30, steps=3)
    assert np.array_equal(a.colind, b.colind) and np.array_equal(a.rowptr, b.rowptr)
    assert np.array_equal(a.values(2), b.values(2))
    assert not np.array_equal(a.values(1), a.values(2))
    bb, xs = a.rhs(1)
    assert np.allclose(a.csr(1) @ xs, bb, rtol=0, atol=0)


def test_dx_spread_widens():
    s = KKTSequence("kkt2000", buses=50, steps=4)
    nx = s.nx
    spread = []
    for k in range(s.M):
        d = s.csr(k).diagonal()[:nx]
        spread.append(np.log10(np.abs(d).max() / np.abs(d).min()))
    assert spread[-1] > spread[0] + 5
