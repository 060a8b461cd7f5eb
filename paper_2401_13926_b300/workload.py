"""Seeded synthetic KKT sequences shaped like the paper's power-grid systems.

This module only *creates inputs*; it contains none of the solver's
arithmetic.  Both the CUDA path and the CPU oracle are fed from it.

Each sequence is K_k = [[H_k + D_x(k), J_k^T], [J_k, -D_y(k)]] (the reduced
KKT form of Eq. (kktlinear), Section 1.2, with a small negative (2,2) block as
an interior-point regularisation), k = 0..M-1, all on one sparsity pattern
(the same-pattern property stated in the Summary of Section 1.2).

Shapes follow Table 1 / Table 3: about 25 KKT rows per bus of a near-planar
transmission grid and about 0.2 generators per bus.  The grid and block
structure:

* buses: uniform points in the unit square; branch candidates: 6-nearest
  neighbour graph; branches: random spanning tree of it plus round(0.3 N)
  extra candidate edges; G = round(0.2 N) generators at distinct random buses;
* primal variables: per bus (Vm, Va); per generator (Pg, Qg); per branch
  (Pf, Qf, Pt, Qt, sf, st, If, It) -- four flows, two limit slacks, two
  current magnitudes;
* constraints: per bus P and Q balance (incident flows, generators, the bus
  voltage and the neighbouring bus voltages), per
  branch four flow definitions (flow + both end voltages), two limits (flow
  pair, slack, both end voltages) and two current definitions (current, flow
  pair, both end voltages);
* Hessian: a 4x4 block over the end voltages of each branch, a 3x3 block over
  (Pf, Qf, Vm_f) and (Pt, Qt, Vm_t), a diagonal generator cost, and symmetric
  voltage couplings between buses up to ``hops`` apart (the density knob,
  fixed once for all configurations);
* values: H and J base magnitudes log-uniform in [0.1, 10] with random sign
  (H symmetric), perturbed per step by (1 + 0.05 N(0,1));
  D_x,i(k) = 10^(s_k u_i), D_y,i(k) = 10^(-8 + 2 u'_i), u, u' ~ U(-1, 1);
  right-hand side b_k = K_k x*_k with x*_k ~ N(0, 1).

Seeds are 1000 * config_id + instance_id.
"""
from __future__ import annotations

import dataclasses
import numpy as np
import scipy.sparse as sp
from scipy.spatial import cKDTree
from scipy.sparse.csgraph import minimum_spanning_tree, connected_components


@dataclasses.dataclass(frozen=True)
class SequenceConfig:
    """One synthetic KKT sequence recipe."""
    name: str
    config_id: int
    buses: int
    steps: int            # M, matrices in the sequence
    s_first: float        # D_x spread exponent at k = 0
    s_last: float         # D_x spread exponent at k = M-1 (linear in k)
    fresh_u: bool         # draw new u_i for every matrix (hardest static-pivot case)
    hops: int = 4         # density knob: voltage couplings up to this many hops


# The five workloads of the benchmark plan (sizes in the docstring above).
CONFIGS = {
    "kkt200": SequenceConfig("kkt200", 1, 200, 10, 8.0, 8.0, True),
    "kkt2000": SequenceConfig("kkt2000", 2, 2000, 30, 2.0, 8.0, False),
    "kkt10000": SequenceConfig("kkt10000", 3, 10000, 40, 2.0, 8.0, False),
    "kkt70000": SequenceConfig("kkt70000", 5, 70000, 20, 2.0, 10.0, False),
}


def _grid(rng, nbus, kNN=6):
    """Near-planar branch list (from, to) of a synthetic grid."""
    pts = rng.random((nbus, 2))
    kk = min(kNN + 1, nbus)
    _, nb = cKDTree(pts).query(pts, k=kk)
    a = np.repeat(np.arange(nbus), kk - 1)
    b = nb[:, 1:].reshape(-1)
    lo, hi = np.minimum(a, b), np.maximum(a, b)
    key = np.unique(lo.astype(np.int64) * nbus + hi)
    cand = np.stack([key // nbus, key % nbus], axis=1)
    # join components of the kNN graph by their closest pairs (rarely needed)
    g = sp.coo_matrix((np.ones(len(cand)), (cand[:, 0], cand[:, 1])), shape=(nbus, nbus))
    ncomp, lab = connected_components(g, directed=False)
    extra = []
    while ncomp > 1:
        in0 = np.where(lab == 0)[0]
        out = np.where(lab != 0)[0]
        d, j = cKDTree(pts[out]).query(pts[in0], k=1)
        i = int(np.argmin(d))
        extra.append((min(in0[i], out[j[i]]), max(in0[i], out[j[i]])))
        lab[lab == lab[out[j[i]]]] = 0
        ncomp = len(np.unique(lab))
    if extra:
        cand = np.unique(np.vstack([cand, np.array(extra)]), axis=0)
    # random spanning tree: minimum spanning tree under random weights
    w = rng.random(len(cand)) + 1e-3
    W = sp.coo_matrix((w, (cand[:, 0], cand[:, 1])), shape=(nbus, nbus)).tocsr()
    T = minimum_spanning_tree(W).tocoo()
    tree = np.stack([np.minimum(T.row, T.col), np.maximum(T.row, T.col)], axis=1)
    tkey = set((tree[:, 0].astype(np.int64) * nbus + tree[:, 1]).tolist())
    rest = np.array([c for c in cand if int(c[0]) * nbus + int(c[1]) not in tkey])
    nextra = min(int(round(0.3 * nbus)), len(rest))
    pick = rng.choice(len(rest), size=nextra, replace=False) if nextra else []
    branches = np.vstack([tree, rest[pick]]) if nextra else tree
    # random orientation (from, to)
    flip = rng.random(len(branches)) < 0.5
    branches[flip] = branches[flip][:, ::-1]
    return branches.astype(np.int64)


class KKTSequence:
    """A same-pattern sequence of synthetic KKT matrices with right-hand sides.

    Attributes: n, nnz, rowptr (int32[n+1]), colind (int32[nnz]) -- the full
    (both triangles) CSR pattern with sorted, duplicate-free rows -- and M.
    ``values(k)`` gives float64[nnz] in that CSR order, ``rhs(k)`` gives
    (b, x*).
    """

    def __init__(self, cfg: SequenceConfig | str, instance: int = 0, buses: int | None = None,
                 steps: int | None = None):
        if isinstance(cfg, str):
            cfg = CONFIGS[cfg]
        if buses is not None or steps is not None:
            cfg = dataclasses.replace(cfg, buses=buses or cfg.buses, steps=steps or cfg.steps)
        self.cfg = cfg
        self.seed = 1000 * cfg.config_id + instance
        rng = np.random.default_rng(self.seed)
        N = cfg.buses
        br = _grid(rng, N)
        E = len(br)
        G = max(1, int(round(0.2 * N)))
        gbus = rng.choice(N, size=G, replace=False)
        self.nbus, self.nbranch, self.ngen = N, E, G

        # ---- primal variable numbering
        vm = np.arange(N) * 2
        va = vm + 1
        pg = 2 * N + 2 * np.arange(G)
        qg = pg + 1
        base = 2 * N + 2 * G
        eb = base + 8 * np.arange(E)
        pf, qf, pt, qt, sf, st, if_, it = (eb + i for i in range(8))
        nx = base + 8 * E
        # ---- constraint numbering (row index within J)
        pb = 2 * np.arange(N)
        qb = pb + 1
        cb = 2 * N + 8 * np.arange(E)
        fpf, fqf, fpt, fqt, lf, lt, cf, ct = (cb + i for i in range(8))
        ny = 2 * N + 8 * E
        self.nx, self.ny = nx, ny
        n = nx + ny
        self.n = n

        f, t = br[:, 0], br[:, 1]
        # ---- Jacobian pairs (constraint row, primal column)
        J = []
        J += [(pb, vm), (qb, vm), (pb, va), (qb, va)]
        # injections at a bus depend on the voltages of its neighbours
        J += [(pb[f], vm[t]), (pb[f], va[t]), (qb[f], vm[t]), (qb[f], va[t]),
              (pb[t], vm[f]), (pb[t], va[f]), (qb[t], vm[f]), (qb[t], va[f])]
        J += [(pb[gbus], pg), (qb[gbus], qg)]
        J += [(pb[f], pf), (qb[f], qf), (pb[t], pt), (qb[t], qt)]
        for row, flow in ((fpf, pf), (fqf, qf), (fpt, pt), (fqt, qt)):
            J += [(row, flow), (row, vm[f]), (row, vm[t]), (row, va[f]), (row, va[t])]
        J += [(lf, pf), (lf, qf), (lf, sf), (lt, pt), (lt, qt), (lt, st)]
        J += [(cf, if_), (cf, pf), (cf, qf), (ct, it), (ct, pt), (ct, qt)]
        # limits and currents are functions of both end voltages (polar form)
        for row in (lf, lt, cf, ct):
            J += [(row, vm[f]), (row, vm[t]), (row, va[f]), (row, va[t])]
        jr = np.concatenate([np.broadcast_to(a, np.shape(b)).ravel() for a, b in J])
        jc = np.concatenate([np.broadcast_to(b, np.shape(a)).ravel() for a, b in J])
        jk = np.unique(jr.astype(np.int64) * nx + jc)
        self._jr, self._jc = (jk // nx), (jk % nx)

        # ---- Hessian pairs (i < j) plus which diagonals carry a Hessian term
        H = []
        vf = np.stack([vm[f], vm[t], va[f], va[t]], axis=1)
        for a in range(4):
            for b in range(4):
                H.append((vf[:, a], vf[:, b]))
        for trip in (np.stack([pf, qf, vm[f]], 1), np.stack([pt, qt, vm[t]], 1)):
            for a in range(3):
                for b in range(3):
                    H.append((trip[:, a], trip[:, b]))
        H.append((pg, pg))
        # density knob: voltage couplings between buses within `hops` hops
        A = sp.coo_matrix((np.ones(E), (f, t)), shape=(N, N))
        A = ((A + A.T) > 0).astype(np.int8).tocsr()
        R = A.copy()
        P = A.copy()
        for _ in range(cfg.hops - 1):
            P = (P @ A > 0).astype(np.int8)
            R = ((R + P) > 0).astype(np.int8)
        R = sp.triu(R, k=1).tocoo()
        for a in (vm, va):
            for b in (vm, va):
                H.append((a[R.row], b[R.col]))
        hi = np.concatenate([np.asarray(a).ravel() for a, b in H])
        hj = np.concatenate([np.asarray(b).ravel() for a, b in H])
        lo, up = np.minimum(hi, hj), np.maximum(hi, hj)
        hk = np.unique(lo.astype(np.int64) * nx + up)
        hlo, hup = hk // nx, hk % nx
        diag = hlo == hup
        self._hdiag_idx = hlo[diag]
        self._hi, self._hj = hlo[~diag], hup[~diag]

        # ---- assemble the CSR pattern with a source map
        nH, nJ = len(self._hi), len(self._jr)
        rows = np.concatenate([np.arange(nx), self._hi, self._hj,
                               nx + self._jr, self._jc, nx + np.arange(ny)])
        cols = np.concatenate([np.arange(nx), self._hj, self._hi,
                               self._jc, nx + self._jr, nx + np.arange(ny)])
        order = np.lexsort((cols, rows))
        self.nnz = len(rows)
        self.rowptr = np.zeros(n + 1, np.int64)
        np.add.at(self.rowptr, rows + 1, 1)
        self.rowptr = np.cumsum(self.rowptr).astype(np.int32)
        self.colind = cols[order].astype(np.int32)
        self._order = order
        self._nH, self._nJ = nH, nJ
        self.M = cfg.steps

        # ---- base values, fixed per sequence
        self._draw_base(rng)

    def _draw_base(self, rng):
        nH, nJ, nx, ny = self._nH, self._nJ, self.nx, self.ny

        def logu(m):
            return 10.0 ** rng.uniform(-1.0, 1.0, m) * np.where(rng.random(m) < 0.5, -1.0, 1.0)
        self._hbase = logu(nH)
        self._jbase = logu(nJ)
        hd = np.zeros(nx)
        hd[self._hdiag_idx] = logu(len(self._hdiag_idx))
        self._hdbase = hd
        self._u = rng.uniform(-1.0, 1.0, nx)
        self._uy = rng.uniform(-1.0, 1.0, ny)

    def reseeded(self, instance: int) -> "KKTSequence":
        """Another sequence on the same grid and pattern, with its own values:
        seed 1000 * config_id + instance for the base values and every
        matrix (the grid is drawn once; for serving many instances cheaply)."""
        import copy
        other = copy.copy(self)
        other.seed = 1000 * self.cfg.config_id + instance
        other._draw_base(np.random.default_rng([other.seed, 0]))
        return other

    # --------------------------------------------------------------------
    def spread(self, k: int) -> float:
        c = self.cfg
        if self.M <= 1:
            return c.s_last
        return c.s_first + (c.s_last - c.s_first) * k / (self.M - 1)

    def values(self, k: int) -> np.ndarray:
        """float64[nnz] values of K_k in CSR order."""
        rng = np.random.default_rng([self.seed, 1, k])
        nx, ny = self.nx, self.ny
        u = rng.uniform(-1.0, 1.0, nx) if self.cfg.fresh_u else self._u
        dx = 10.0 ** (self.spread(k) * u)
        dy = 10.0 ** (-8.0 + 2.0 * self._uy)
        hv = self._hbase * (1.0 + 0.05 * rng.standard_normal(self._nH))
        jv = self._jbase * (1.0 + 0.05 * rng.standard_normal(self._nJ))
        hd = self._hdbase * (1.0 + 0.05 * rng.standard_normal(nx))
        src = np.concatenate([hd + dx, hv, hv, jv, jv, -dy])
        return np.ascontiguousarray(src[self._order])

    def rhs(self, k: int, values: np.ndarray | None = None):
        """(b_k, x*_k) with b_k = K_k x*_k (manufactured solution)."""
        rng = np.random.default_rng([self.seed, 2, k])
        xs = rng.standard_normal(self.n)
        v = self.values(k) if values is None else values
        K = sp.csr_matrix((v, self.colind, self.rowptr), shape=(self.n, self.n))
        return K @ xs, xs

    def random_rhs(self, k: int) -> np.ndarray:
        """A pure random right-hand side (no manufactured solution)."""
        return np.random.default_rng([self.seed, 3, k]).standard_normal(self.n)

    def csr(self, k: int) -> sp.csr_matrix:
        return sp.csr_matrix((self.values(k), self.colind, self.rowptr), shape=(self.n, self.n))


def small_random_sparse(n: int, density: float, seed: int, diag_boost: float = 0.0):
    """Random nonsymmetric sparse CSR (rowptr, colind, values) with a full
    diagonal, for property tests on shapes the KKT generator does not make."""
    rng = np.random.default_rng(seed)
    M = sp.random(n, n, density=density, random_state=rng, format="coo",
                  data_rvs=lambda m: rng.standard_normal(m))
    D = sp.diags(rng.standard_normal(n) + diag_boost * np.sign(rng.standard_normal(n)))
    A = (M + D).tocsr()
    A.sum_duplicates()
    A.sort_indices()
    return A.indptr.astype(np.int32), A.indices.astype(np.int32), A.data.astype(np.float64)
