"""kkt_lu_solve_noalloc: the triangular solve for callers that cannot
allocate device memory (their device memory belongs to an arena allocator,
or a cudaMalloc could stall a latency-critical loop).  On the same factors
it must solve as kkt_lu_solve does, call after call, although every call
reuses one static scratch array.  Both evaluate every row with the same
row arithmetic (the same tiers, summation order and pivot reciprocal), so
their results are compared bit for bit, and on an ill-conditioned KKT
matrix also against the componentwise backward-error bound of the
triangular solves.  Kept in its own file, collected last."""
import scipy.sparse as sp
import ctypes as C

import numpy as np
import pytest

import paper_2401_13926_b300 as K
from paper_2401_13926_b300.workload import KKTSequence

pytestmark = pytest.mark.gpu


def combined_rows(f, n):
    """L (strict lower, CSC) + U (with diagonal, CSC) -> the combined row
    layout: CSR over permuted rows, columns ascending, diagonal position."""
    lc = np.repeat(np.arange(n), np.diff(f["Lp"]))
    uc = np.repeat(np.arange(n), np.diff(f["Up"]))
    rows = np.concatenate([f["Li"], f["Ui"]]).astype(np.int64)
    cols = np.concatenate([lc, uc]).astype(np.int64)
    vals = np.concatenate([f["Lx"], f["Ux"]])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    Fp = np.zeros(n + 1, np.int64)
    np.add.at(Fp, rows + 1, 1)
    Fp = np.cumsum(Fp)
    Fdiag = np.nonzero(rows == cols)[0].astype(np.int64)
    assert len(Fdiag) == n
    return Fp, cols.astype(np.int32), Fdiag, vals


def _backward_error(f, n, P, Q, b, x):
    Lm = sp.csc_matrix((f["Lx"], f["Li"], f["Lp"]), shape=(n, n)) + sp.identity(n)
    Um = sp.csc_matrix((f["Ux"], f["Ui"], f["Up"]), shape=(n, n))
    z = x[Q]
    r = b[P] - Lm @ (Um @ z)
    scale = abs(Lm) @ (abs(Um) @ abs(z)) + abs(b[P])
    # two triangular solves: |r| <= 2 g(k+2) |L||U||z| (Higham Thm. 8.5),
    # g(k) = k u / (1 - k u), k the longest factor row
    k = max(np.diff(Lm.tocsr().indptr).max(), np.diff(Um.tocsr().indptr).max()) + 2
    u = 2.0 ** -53
    return np.max(np.abs(r) / scale) / (2 * k * u / (1 - k * u))


def _noalloc_vs_context(s, n, rng, calls=2):
    import torch
    f = s.factors()
    Fp, Fj, Fdiag, Fx = combined_rows(f, n)
    P, Q = s.perm()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dFp, dFj, dFd, dFx, dP, dQ = map(dev, (Fp, Fj, Fdiag, Fx, P, Q))
    out = []
    for call in range(calls):
        bh = rng.standard_normal(n)
        b = dev(bh)
        x_ref = s.lu_solve(b)
        x = torch.full_like(b, float("nan"))
        K.lu_solve_noalloc(dFp, dFj, dFd, dFx, dP, dQ, b, x)
        torch.cuda.synchronize()
        xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
        assert np.all(np.isfinite(xn)), call
        out.append((f, P, Q, bh, xr, xn))
    return out


def test_noalloc_solve_matches_context_solve_twice():
    """KKT matrix (library analysis): both meet the triangular solves'
    componentwise backward-error bound."""
    seq = KKTSequence("kkt200")
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    s.refactor(seq.values(5))
    for f, P, Q, b, xr, xn in _noalloc_vs_context(s, seq.n, np.random.default_rng(42)):
        assert np.array_equal(xn, xr)
        assert _backward_error(f, seq.n, P, Q, b, xn) <= 1.0


def test_noalloc_solve_bitwise_equal_to_context_solve_well_conditioned():
    from paper_2401_13926_b300.workload import small_random_sparse
    n = 1500
    rp, ci, v = small_random_sparse(n, 0.004, 7, diag_boost=6.0)
    s = K.KKTSolver()
    s.analyze(rp, ci, values0=v)
    s.refactor(v)
    for f, P, Q, b, xr, xn in _noalloc_vs_context(s, n, np.random.default_rng(1)):
        assert np.array_equal(xn, xr)


def test_noalloc_rejects_n_beyond_its_scratch():
    import torch
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    i = torch.zeros(4, dtype=torch.int64, device="cuda")
    j = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = K.lib().kkt_lu_solve_noalloc(K.NOALLOC_MAX_N + 1, i.data_ptr(), j.data_ptr(), i.data_ptr(),
                                      t.data_ptr(), j.data_ptr(), j.data_ptr(), t.data_ptr(), t.data_ptr(), None)
    assert rc == -1
