"""kkt_lu_solve_noalloc: the triangular solve for callers that cannot
allocate device memory (their device memory belongs to an arena allocator,
or a cudaMalloc could stall a latency-critical loop).  It must give the
same x as kkt_lu_solve on the same factors, call after call, although every
call reuses one static scratch array.  Kept in its own file, collected last."""
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


def test_noalloc_solve_matches_context_solve_twice():
    import torch
    seq = KKTSequence("kkt200")
    s = K.KKTSolver()
    s.analyze(seq.rowptr, seq.colind, values0=seq.values(0))
    v = seq.values(5)
    s.refactor(v)
    n = seq.n
    Fp, Fj, Fdiag, Fx = combined_rows(s.factors(), n)
    P, Q = s.perm()
    dev = lambda a: torch.from_numpy(np.ascontiguousarray(a)).cuda()
    dFp, dFj, dFd, dFx, dP, dQ = map(dev, (Fp, Fj, Fdiag, Fx, P, Q))
    rng = np.random.default_rng(42)
    for call in range(2):
        b = dev(rng.standard_normal(n))
        x_ref = s.lu_solve(b)
        x = torch.full_like(b, float("nan"))
        K.lu_solve_noalloc(dFp, dFj, dFd, dFx, dP, dQ, b, x)
        torch.cuda.synchronize()
        xr, xn = x_ref.cpu().numpy(), x.cpu().numpy()
        assert np.all(np.isfinite(xn)), call
        assert np.max(np.abs(xn - xr)) <= 1e-12 * np.max(np.abs(xr)), call


def test_noalloc_rejects_n_beyond_its_scratch():
    import torch
    t = torch.zeros(4, dtype=torch.float64, device="cuda")
    i = torch.zeros(4, dtype=torch.int64, device="cuda")
    j = torch.zeros(4, dtype=torch.int32, device="cuda")
    rc = K.lib().kkt_lu_solve_noalloc(K.NOALLOC_MAX_N + 1, i.data_ptr(), j.data_ptr(), i.data_ptr(),
                                      t.data_ptr(), j.data_ptr(), j.data_ptr(), t.data_ptr(), t.data_ptr(), None)
    assert rc == -1
