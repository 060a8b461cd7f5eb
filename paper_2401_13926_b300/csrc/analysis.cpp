// Host-side one-time analysis: canonical pattern, fill-reducing column
// order, first factorization with threshold partial pivoting, symbolic
// structure for a fixed pivot sequence, and the GPU factor layout.
// See analysis.h for the role of each step in the paper's CPU/GPU split.
#include "analysis.h"

#include <algorithm>
#include <cmath>
#include <numeric>
#include <set>

#include "kkt.h"

namespace kkt {

// ---------------------------------------------------------------------------
int canonicalize(int32_t n, const int32_t* rowptr, const int32_t* colind, Csr* out, std::string* why) {
    if (n < 0 || (n > 0 && (!rowptr || !colind))) { *why = "null pattern"; return KKT_ERR_INVALID; }
    if (n == 0) { out->n = 0; out->rowptr.assign(1, 0); out->colind.clear(); out->src.clear(); return KKT_OK; }
    if (rowptr[0] != 0) { *why = "rowptr[0] != 0"; return KKT_ERR_PATTERN; }
    for (int32_t i = 0; i < n; i++)
        if (rowptr[i + 1] < rowptr[i]) { *why = "rowptr decreases at row " + std::to_string(i); return KKT_ERR_PATTERN; }
    const int64_t nnz = rowptr[n];
    out->n = n;
    out->rowptr.assign(rowptr, rowptr + n + 1);
    out->colind.resize(nnz);
    out->src.resize(nnz);
    out->identity_src = true;
    std::vector<std::pair<int32_t, int64_t>> row;
    for (int32_t i = 0; i < n; i++) {
        row.clear();
        for (int64_t p = rowptr[i]; p < rowptr[i + 1]; p++) {
            int32_t c = colind[p];
            if (c < 0 || c >= n) { *why = "column index out of range in row " + std::to_string(i); return KKT_ERR_PATTERN; }
            row.emplace_back(c, p);
        }
        bool sorted = true;
        for (size_t t = 1; t < row.size(); t++) if (row[t].first <= row[t - 1].first) { sorted = false; break; }
        if (!sorted) {
            std::sort(row.begin(), row.end());
            out->identity_src = false;
            for (size_t t = 1; t < row.size(); t++)
                if (row[t].first == row[t - 1].first) { *why = "duplicate entry in row " + std::to_string(i); return KKT_ERR_PATTERN; }
        }
        int64_t b = rowptr[i];
        for (size_t t = 0; t < row.size(); t++) { out->colind[b + t] = row[t].first; out->src[b + t] = row[t].second; }
    }
    return KKT_OK;
}

// ---------------------------------------------------------------------------
// Approximate minimum degree on the column-intersection graph.  The rows of
// A are the initial elements of a quotient graph over the columns; two
// columns are adjacent in A^T A exactly when some element holds both.
// Eliminating a column p merges the elements around it into a new element;
// elements wholly inside it are absorbed; degrees are the usual AMD upper
// bound; columns with identical element lists are merged into
// supervariables and ordered together.
int order_colamd_like(const Csr& A, std::vector<int32_t>* Qout) {
    const int32_t n = A.n;
    Qout->resize(n);
    if (n == 0) return KKT_OK;
    const int32_t nel = 2 * n;   // element ids: rows 0..n-1, pivots n + p
    std::vector<std::vector<int32_t>> E(n), Lv(nel);
    std::vector<int64_t> esize(nel, 0);
    std::vector<char> alive(nel, 0);
    const int64_t dense_row = std::max<int64_t>(16, (int64_t)(10.0 * std::sqrt((double)n)));
    for (int32_t r = 0; r < n; r++) {
        int64_t len = A.rowptr[r + 1] - A.rowptr[r];
        if (len == 0 || len > dense_row) continue;   // dense rows do not guide the order
        alive[r] = 1;
        Lv[r].assign(A.colind.begin() + A.rowptr[r], A.colind.begin() + A.rowptr[r + 1]);
        esize[r] = len;
        for (int32_t c : Lv[r]) E[c].push_back(r);
    }
    std::vector<int32_t> nv(n, 1), deg(n, 0);
    std::vector<char> state(n, 0);              // 0 live principal, 1 merged, 2 eliminated
    std::vector<std::vector<int32_t>> members(n);
    std::vector<int64_t> mark(n, -1), wmark(nel, -1);
    std::vector<int64_t> w(nel, 0);
    int64_t stamp = 0;
    for (int32_t i = 0; i < n; i++) {
        stamp++;
        int64_t d = 0;
        mark[i] = stamp;
        for (int32_t e : E[i])
            for (int32_t v : Lv[e])
                if (mark[v] != stamp) { mark[v] = stamp; d++; }
        deg[i] = (int32_t)d;
    }
    std::set<std::pair<int32_t, int32_t>> pq;
    for (int32_t i = 0; i < n; i++) pq.insert({deg[i], i});
    int64_t remaining = n;
    int32_t k = 0;
    std::vector<int32_t> Lp;
    std::vector<std::pair<uint64_t, int32_t>> hashes;
    while (!pq.empty()) {
        const int32_t p = pq.begin()->second;
        pq.erase(pq.begin());
        // the new element: union of the elements around p
        stamp++;
        Lp.clear();
        mark[p] = stamp;
        for (int32_t e : E[p]) {
            if (!alive[e]) continue;
            for (int32_t v : Lv[e])
                if (state[v] == 0 && mark[v] != stamp) { mark[v] = stamp; Lp.push_back(v); }
            alive[e] = 0;                      // absorbed into the new element
            std::vector<int32_t>().swap(Lv[e]);
        }
        // output p and the columns merged into it
        (*Qout)[k++] = p;
        for (int32_t m : members[p]) (*Qout)[k++] = m;
        state[p] = 2;
        remaining -= nv[p];
        std::vector<int32_t>().swap(E[p]);
        const int32_t ep = n + p;
        alive[ep] = 1;
        int64_t lpw = 0;
        for (int32_t v : Lp) lpw += nv[v];
        esize[ep] = lpw;
        // element lists of the columns of the new element
        for (int32_t v : Lp) {
            pq.erase({deg[v], v});
            auto& ev = E[v];
            size_t o = 0;
            for (int32_t e : ev) if (alive[e]) ev[o++] = e;
            ev.resize(o);
            ev.push_back(ep);
        }
        // w(e) = |L_e \ L_p| for elements next to L_p
        stamp++;
        for (int32_t v : Lp)
            for (int32_t e : E[v]) {
                if (e == ep) continue;
                if (wmark[e] != stamp) { wmark[e] = stamp; w[e] = esize[e]; }
                w[e] -= nv[v];
            }
        // absorption of elements inside L_p and the degree bound
        for (int32_t v : Lp) {
            auto& ev = E[v];
            int64_t d = 0;
            size_t o = 0;
            for (int32_t e : ev) {
                if (e != ep && w[e] <= 0) { alive[e] = 0; continue; }
                if (!alive[e]) continue;
                ev[o++] = e;
                if (e != ep) d += w[e];
            }
            ev.resize(o);
            d += lpw - nv[v];
            d = std::min<int64_t>(d, (int64_t)deg[v] + lpw - nv[v]);
            d = std::min<int64_t>(d, remaining - nv[v]);
            deg[v] = (int32_t)std::max<int64_t>(d, 0);
        }
        // supervariables: columns of L_p with identical element lists
        hashes.clear();
        for (int32_t v : Lp) {
            auto& ev = E[v];
            std::sort(ev.begin(), ev.end());
            uint64_t h = ev.size();
            for (int32_t e : ev) h = h * 1000003ull + (uint64_t)e;
            hashes.push_back({h, v});
        }
        std::sort(hashes.begin(), hashes.end());
        for (size_t a = 0; a < hashes.size();) {
            size_t b = a + 1;
            while (b < hashes.size() && hashes[b].first == hashes[a].first) b++;
            for (size_t s = a; s < b; s++) {
                int32_t v = hashes[s].second;
                if (state[v] != 0) continue;
                for (size_t t = s + 1; t < b; t++) {
                    int32_t u = hashes[t].second;
                    if (state[u] != 0 || E[u] != E[v]) continue;
                    nv[v] += nv[u];
                    deg[v] = std::max(0, deg[v] - nv[u]);
                    nv[u] = 0;
                    state[u] = 1;
                    members[v].push_back(u);
                    for (int32_t m : members[u]) members[v].push_back(m);
                    std::vector<int32_t>().swap(members[u]);
                    std::vector<int32_t>().swap(E[u]);
                }
            }
            a = b;
        }
        std::vector<int32_t> keep;
        keep.reserve(Lp.size());
        for (int32_t v : Lp)
            if (state[v] == 0) { keep.push_back(v); pq.insert({deg[v], v}); }
        Lv[ep] = std::move(keep);
    }
    if (k != n) return KKT_ERR_INVALID;
    return KKT_OK;
}

// ---------------------------------------------------------------------------
namespace {
struct Cscv {
    std::vector<int64_t> p;
    std::vector<int32_t> i;
    std::vector<int64_t> e;   // canonical entry index
};
Cscv to_csc(const Csr& A) {
    Cscv C;
    const int32_t n = A.n;
    C.p.assign(n + 1, 0);
    for (int32_t c : A.colind) C.p[c + 1]++;
    for (int32_t j = 0; j < n; j++) C.p[j + 1] += C.p[j];
    C.i.resize(A.colind.size());
    C.e.resize(A.colind.size());
    std::vector<int64_t> next(C.p.begin(), C.p.end() - 1);
    for (int32_t r = 0; r < n; r++)
        for (int64_t q = A.rowptr[r]; q < A.rowptr[r + 1]; q++) {
            int64_t t = next[A.colind[q]]++;
            C.i[t] = r;
            C.e[t] = q;
        }
    return C;
}
}  // namespace

// Left-looking sparse LU with threshold partial pivoting (Gilbert-Peierls:
// depth-first reach gives the column structure in topological order, then a
// sparse triangular solve with the finished columns).  Diagonal preference:
// the row with the column's own original index is kept when it is within
// `tol` of the largest candidate; otherwise the largest wins, ties to the
// smaller original row index.
int pivot_lu(const Csr& A, const double* vals, const std::vector<int32_t>& Q, double tol,
             std::vector<int32_t>* Pout, ColStructure* S, int32_t* bad_col) {
    const int32_t n = A.n;
    Cscv C = to_csc(A);
    std::vector<int32_t> pinv(n, -1), visit(n, -1), topo(n), stk(n);
    std::vector<int64_t> it(n);
    std::vector<double> x(n, 0.0);
    std::vector<int64_t> Lcol(n + 1, 0);
    std::vector<int32_t> Lrow;    // original rows while factorizing
    std::vector<double> Lval;
    S->Up.assign(n + 1, 0);
    S->Ui.clear();
    Pout->assign(n, -1);
    for (int32_t j = 0; j < n; j++) {
        const int32_t c = Q[j];
        // reach of column c through the finished columns
        int32_t ntop = n;
        for (int64_t q = C.p[c]; q < C.p[c + 1]; q++) {
            int32_t r0 = C.i[q];
            if (visit[r0] == j) continue;
            int32_t sp = 0;
            stk[0] = r0;
            visit[r0] = j;
            it[0] = (pinv[r0] >= 0) ? Lcol[pinv[r0]] : 0;
            while (sp >= 0) {
                int32_t v = stk[sp];
                int64_t end = (pinv[v] >= 0) ? Lcol[pinv[v] + 1] : 0;
                bool descended = false;
                while (it[sp] < end) {
                    int32_t wv = Lrow[it[sp]++];
                    if (visit[wv] != j) {
                        visit[wv] = j;
                        sp++;
                        stk[sp] = wv;
                        it[sp] = (pinv[wv] >= 0) ? Lcol[pinv[wv]] : 0;
                        descended = true;
                        break;
                    }
                }
                if (!descended) { topo[--ntop] = v; sp--; }
            }
        }
        for (int64_t q = C.p[c]; q < C.p[c + 1]; q++) x[C.i[q]] = vals[C.e[q]];
        for (int32_t t = ntop; t < n; t++) {
            int32_t r = topo[t];
            int32_t kcol = pinv[r];
            if (kcol < 0) continue;
            const double xr = x[r];
            for (int64_t q = Lcol[kcol]; q < Lcol[kcol + 1]; q++) x[Lrow[q]] -= Lval[q] * xr;
        }
        int32_t best = -1;
        double amax = -1.0;
        for (int32_t t = ntop; t < n; t++) {
            int32_t r = topo[t];
            if (pinv[r] >= 0) continue;
            double a = std::fabs(x[r]);
            if (!std::isfinite(a)) { *bad_col = j; return KKT_ERR_NONFINITE; }
            if (a > amax || (a == amax && r < best)) { amax = a; best = r; }
        }
        if (best < 0 || amax == 0.0) { *bad_col = j; return KKT_ERR_ZERO_PIVOT; }
        int32_t piv = best;
        if (pinv[c] < 0 && visit[c] == j && std::fabs(x[c]) >= tol * amax) piv = c;
        const double d = x[piv];
        for (int32_t t = ntop; t < n; t++) {
            int32_t r = topo[t];
            if (pinv[r] >= 0) S->Ui.push_back(pinv[r]);
        }
        S->Ui.push_back(j);
        S->Up[j + 1] = (int64_t)S->Ui.size();
        for (int32_t t = ntop; t < n; t++) {
            int32_t r = topo[t];
            if (pinv[r] < 0 && r != piv) { Lrow.push_back(r); Lval.push_back(x[r] / d); }
        }
        Lcol[j + 1] = (int64_t)Lrow.size();
        pinv[piv] = j;
        (*Pout)[j] = piv;
        for (int32_t t = ntop; t < n; t++) x[topo[t]] = 0.0;
    }
    S->Lp = Lcol;
    S->Li.resize(Lrow.size());
    for (size_t q = 0; q < Lrow.size(); q++) S->Li[q] = pinv[Lrow[q]];
    return KKT_OK;
}

// Symbolic factorization for a fixed pivot sequence: the structure of
// column j of L+U is the set reachable from the (permuted) rows of
// A(P, Q[j]) through the columns of L already built.
int symbolic(const Csr& A, const std::vector<int32_t>& P, const std::vector<int32_t>& Q,
             ColStructure* S, int32_t* bad_col) {
    const int32_t n = A.n;
    std::vector<int32_t> pinv(n, -1);
    for (int32_t i = 0; i < n; i++) {
        if (P[i] < 0 || P[i] >= n || pinv[P[i]] >= 0) { *bad_col = i; return KKT_ERR_INVALID; }
        pinv[P[i]] = i;
    }
    std::vector<char> qseen(n, 0);
    for (int32_t j = 0; j < n; j++) {
        if (Q[j] < 0 || Q[j] >= n || qseen[Q[j]]) { *bad_col = j; return KKT_ERR_INVALID; }
        qseen[Q[j]] = 1;
    }
    Cscv C = to_csc(A);
    std::vector<int32_t> seen(n, -1), queue;
    S->Lp.assign(n + 1, 0);
    S->Up.assign(n + 1, 0);
    S->Li.clear();
    S->Ui.clear();
    for (int32_t j = 0; j < n; j++) {
        const int32_t c = Q[j];
        queue.clear();
        for (int64_t q = C.p[c]; q < C.p[c + 1]; q++) {
            int32_t i = pinv[C.i[q]];
            if (seen[i] != j) { seen[i] = j; queue.push_back(i); }
        }
        for (size_t h = 0; h < queue.size(); h++) {
            int32_t i = queue[h];
            if (i >= j) continue;
            for (int64_t q = S->Lp[i]; q < S->Lp[i + 1]; q++) {
                int32_t r = S->Li[q];
                if (seen[r] != j) { seen[r] = j; queue.push_back(r); }
            }
        }
        if (seen[j] != j) { *bad_col = j; return KKT_ERR_ZERO_PIVOT; }
        std::sort(queue.begin(), queue.end());
        for (int32_t i : queue) {
            if (i <= j) S->Ui.push_back(i);
            else S->Li.push_back(i);
        }
        S->Lp[j + 1] = (int64_t)S->Li.size();
        S->Up[j + 1] = (int64_t)S->Ui.size();
    }
    return KKT_OK;
}

// ---------------------------------------------------------------------------
int build_layout(const Csr& A, const std::vector<int32_t>& P, const std::vector<int32_t>& Q,
                 const ColStructure& S, Layout* out) {
    const int32_t n = A.n;
    out->n = n;
    out->nnzL = S.Lp[n];
    out->nnzU = S.Up[n];
    out->Fp.assign(n + 1, 0);
    for (int32_t j = 0; j < n; j++) {
        for (int64_t q = S.Lp[j]; q < S.Lp[j + 1]; q++) out->Fp[S.Li[q] + 1]++;
        for (int64_t q = S.Up[j]; q < S.Up[j + 1]; q++) out->Fp[S.Ui[q] + 1]++;
    }
    for (int32_t i = 0; i < n; i++) out->Fp[i + 1] += out->Fp[i];
    const int64_t nnz = out->Fp[n];
    out->Fj.assign(nnz, 0);
    std::vector<int64_t> next(out->Fp.begin(), out->Fp.end() - 1);
    // columns ascending -> every row's column list comes out sorted
    for (int32_t j = 0; j < n; j++) {
        for (int64_t q = S.Up[j]; q < S.Up[j + 1]; q++) out->Fj[next[S.Ui[q]]++] = j;
        for (int64_t q = S.Lp[j]; q < S.Lp[j + 1]; q++) out->Fj[next[S.Li[q]]++] = j;
    }
    out->Fdiag.assign(n, -1);
    for (int32_t i = 0; i < n; i++) {
        auto b = out->Fj.begin() + out->Fp[i], e = out->Fj.begin() + out->Fp[i + 1];
        auto f = std::lower_bound(b, e, i);
        if (f == e || *f != i) return KKT_ERR_ZERO_PIVOT;
        out->Fdiag[i] = f - out->Fj.begin();
    }
    std::vector<int32_t> pinv(n), qinv(n);
    for (int32_t i = 0; i < n; i++) { pinv[P[i]] = i; qinv[Q[i]] = i; }
    out->Fsrc.assign(nnz, -1);
    for (int32_t r = 0; r < n; r++)
        for (int64_t q = A.rowptr[r]; q < A.rowptr[r + 1]; q++) {
            int32_t i = pinv[r], j = qinv[A.colind[q]];
            auto b = out->Fj.begin() + out->Fp[i], e = out->Fj.begin() + out->Fp[i + 1];
            auto f = std::lower_bound(b, e, j);
            if (f == e || *f != j) return KKT_ERR_PATTERN;
            out->Fsrc[f - out->Fj.begin()] = q;
        }
    // dependency depths and the refactorization's multiply-add count
    std::vector<int32_t> lev(n, 0);
    int32_t ml = 0;
    double upd = 0;
    for (int32_t i = 0; i < n; i++) {
        int32_t l = 0;
        for (int64_t q = out->Fp[i]; q < out->Fdiag[i]; q++) {
            int32_t kk = out->Fj[q];
            l = std::max(l, lev[kk] + 1);
            upd += (double)(out->Fp[kk + 1] - out->Fdiag[kk] - 1);
        }
        lev[i] = l;
        ml = std::max(ml, l + 1);
    }
    out->levelsL = n ? ml : 0;
    out->updates = upd;
    out->levL = lev;
    int32_t mu = 0;
    for (int32_t i = n - 1; i >= 0; i--) {
        int32_t l = 0;
        for (int64_t q = out->Fdiag[i] + 1; q < out->Fp[i + 1]; q++) l = std::max(l, lev[out->Fj[q]] + 1);
        lev[i] = l;
        mu = std::max(mu, l + 1);
    }
    out->levelsU = n ? mu : 0;
    out->levU = lev;
    return KKT_OK;
}

}  // namespace kkt
