/*
 * CPU FP64 oracle for the GPU-resident KKT solver (arXiv 2401.13926).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the plain, slow, obviously
 * correct restatement of what the solver computes.  Only the tests, the
 * smoke check and the benchmark's CPU-baseline leg may load it; the solver
 * library never calls it and shares no code with it.
 *
 * Contents, each following the paper:
 *   or_order_md     -- a fill-reducing column ordering (step 1 of the four
 *                      solver steps of Section 1.3): exact minimum degree on
 *                      the column-intersection graph (pattern of A^T A),
 *                      explicit elimination graph, ties by smallest index.
 * Update order and rounding: the paper fixes neither.  Both factorizations
 * apply the finished columns in ascending pivot order -- one valid
 * topological order of the elimination graph -- and every update
 * x_i <- x_i - l_ik x_k is a single fused multiply-add (one rounding).
 * Column j of L is x_i * (1/u_jj): the pivot's reciprocal is formed once
 * (correctly rounded division) and each entry is one multiplication, the
 * scaling LAPACK's getf2 uses.
 *
 *   or_lu           -- first numeric factorization with threshold partial
 *                      pivoting (Section 1.3, "full symbolic analysis and
 *                      numerical factorization with pivoting for the first
 *                      system"): left-looking Gilbert-Peierls sparse LU of
 *                      A(:,Q), reach by depth-first search, diagonal
 *                      preference with threshold `tol`, ties to the
 *                      smallest original row index.
 *   or_refactor     -- refactorization (Section 1.3: only the numeric
 *                      factorization, reusing the pivot sequence and the
 *                      symbolic analysis of the first system), with an
 *                      optional static-pivot boost.
 *   or_refactor_f32 -- the same refactorization in FP32 arithmetic (the
 *                      mixed-precision factors used as an inexact
 *                      preconditioner, Section 2.1).
 *   or_solve        -- the triangular solve (step 3 of Section 1.3):
 *                      x = Q U^{-1} L^{-1} P b.
 *   or_fgmres       -- iterative refinement by FGMRES with the LU factors as
 *                      right preconditioner (Section 2.1): the LU solution is
 *                      the initial guess, Arnoldi with CGS2, Givens rotations
 *                      give the estimated residual, and the solution is formed
 *                      only at a restart or when the estimate meets the
 *                      criterion; refine-or-not decision of Section 2.3.
 *   or_fgmres_ex    -- the same with the variants the paper cites: the
 *                      orthogonalisation (CGS2; CGS2 whose norm comes from
 *                      the second projection's reduction by Pythagoras; one
 *                      reduction CGS with the Pythagorean norm -- the
 *                      low-synchronisation Gram-Schmidt family of Section
 *                      2.1) and the inner stopping rule of FGMRES on the
 *                      error equation (Section 2.1, Fig. 1: each cycle
 *                      solves K d = rho to a relative tolerance, then
 *                      x += d and the residual is recomputed).
 *   or_richardson   -- classical iterative refinement (Section 2.1, the error
 *                      system): rho = b - K x, d = (LU)^{-1} rho, x += d.
 *   or_nrbe/or_nsr  -- the backward-error measures of Section 2.2 (Eq. nbre)
 *                      and Section 1.3 (NSR).
 *
 * Permutation convention: B = A(P, Q), i.e. B(i,j) = A(P[i], Q[j]); L is unit
 * lower triangular (diagonal not stored), U upper triangular with its
 * diagonal stored; LU = B.  Both are CSC with row indices in the permuted
 * space, sorted ascending within each column.
 *
 * Matrices enter in CSC (Ap, Ai, Ax) for the factorization and CSR for the
 * matrix-vector product; both describe the same K.
 */
#define _POSIX_C_SOURCE 199309L
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <time.h>

#define OR_OK 0
#define OR_ERR_SINGULAR (-4)
#define OR_ERR_NONFINITE (-5)
#define OR_ERR_NOT_CONVERGED (-6)
#define OR_ERR_OOM (-3)
#define OR_ERR_PATTERN (-2)

/* ------------------------------------------------------------------ */
/* growable int / double arrays                                        */
typedef struct { int *a; long n, cap; } ivec;
typedef struct { double *a; long n, cap; } dvec;

static int ivec_push(ivec *v, int x) {
    if (v->n == v->cap) {
        long c = v->cap ? 2 * v->cap : 16;
        int *p = (int *)realloc(v->a, (size_t)c * sizeof(int));
        if (!p) return 0;
        v->a = p; v->cap = c;
    }
    v->a[v->n++] = x;
    return 1;
}
static int dvec_push(dvec *v, double x) {
    if (v->n == v->cap) {
        long c = v->cap ? 2 * v->cap : 16;
        double *p = (double *)realloc(v->a, (size_t)c * sizeof(double));
        if (!p) return 0;
        v->a = p; v->cap = c;
    }
    v->a[v->n++] = x;
    return 1;
}

static int cmp_int(const void *a, const void *b) {
    int x = *(const int *)a, y = *(const int *)b;
    return (x > y) - (x < y);
}

/* ------------------------------------------------------------------ */
/* Factor storage                                                      */
typedef struct {
    int n;
    int *Lp, *Li; double *Lx;   /* strictly lower part, CSC */
    int *Up, *Ui; double *Ux;   /* upper part with diagonal, CSC */
    int nboost;                 /* static pivots replaced by the boost rule */
} or_factors;

void or_factor_free(void *h) {
    or_factors *F = (or_factors *)h;
    if (!F) return;
    free(F->Lp); free(F->Li); free(F->Lx);
    free(F->Up); free(F->Ui); free(F->Ux);
    free(F);
}

void or_factor_sizes(void *h, long *lnz, long *unz, int *nboost) {
    or_factors *F = (or_factors *)h;
    *lnz = F->Lp[F->n];
    *unz = F->Up[F->n];
    *nboost = F->nboost;
}

void or_factor_copy(void *h, int *Lp, int *Li, double *Lx, int *Up, int *Ui, double *Ux) {
    or_factors *F = (or_factors *)h;
    int n = F->n;
    memcpy(Lp, F->Lp, sizeof(int) * (size_t)(n + 1));
    memcpy(Up, F->Up, sizeof(int) * (size_t)(n + 1));
    memcpy(Li, F->Li, sizeof(int) * (size_t)F->Lp[n]);
    memcpy(Lx, F->Lx, sizeof(double) * (size_t)F->Lp[n]);
    memcpy(Ui, F->Ui, sizeof(int) * (size_t)F->Up[n]);
    memcpy(Ux, F->Ux, sizeof(double) * (size_t)F->Up[n]);
}

/* Sort the (index, value) pairs of every column by index. */
static void sort_columns(int n, const int *p, int *idx, double *val) {
    for (int j = 0; j < n; j++) {
        /* insertion sort: columns are short and this is the oracle */
        for (int a = p[j] + 1; a < p[j + 1]; a++) {
            int ki = idx[a]; double kv = val[a];
            int b = a - 1;
            while (b >= p[j] && idx[b] > ki) { idx[b + 1] = idx[b]; val[b + 1] = val[b]; b--; }
            idx[b + 1] = ki; val[b + 1] = kv;
        }
    }
}

/* ------------------------------------------------------------------ */
/* Depth-first reach (Gilbert-Peierls symbolic step).                   */
/* Nodes reachable from the seeds through graph `child(node)`; returns  */
/* them in topological order in out[*top .. n).                         */
/* child lists: for node v with colof[v] >= 0 the children are          */
/*   gi[gp[colof[v]] .. gp[colof[v]+1]).                                */
static void reach(int n, const int *seeds, int nseeds, const int *colof,
                  const int *gp, const int *gi, int *mark, int stamp,
                  int *stack, int *pos, int *out, int *top) {
    (void)n;
    for (int s = 0; s < nseeds; s++) {
        int r = seeds[s];
        if (mark[r] == stamp) continue;
        int sp = 0;
        stack[sp] = r; pos[sp] = -1; mark[r] = stamp;
        while (sp >= 0) {
            int v = stack[sp];
            int c = colof[v];
            if (pos[sp] < 0) pos[sp] = (c >= 0) ? gp[c] : 0;
            int end = (c >= 0) ? gp[c + 1] : 0;
            int pushed = 0;
            while (pos[sp] < end) {
                int w = gi[pos[sp]++];
                if (mark[w] != stamp) {
                    mark[w] = stamp;
                    sp++;
                    stack[sp] = w; pos[sp] = -1;
                    pushed = 1;
                    break;
                }
            }
            if (!pushed) {          /* all children done: postorder */
                out[--(*top)] = v;
                sp--;
            }
        }
    }
}

/* ------------------------------------------------------------------ */
/* First factorization with threshold partial pivoting.                */
/* Ap/Ai/Ax: A in CSC.  Q: column order.  P (out): P[k] = original row */
/* chosen as the k-th pivot.  Returns a factor handle or NULL.          */
void *or_lu(int n, const int *Ap, const int *Ai, const double *Ax,
            const int *Q, double tol, int *P, int *status) {
    *status = OR_ERR_OOM;
    or_factors *F = (or_factors *)calloc(1, sizeof(or_factors));
    int *pinv = (int *)malloc(sizeof(int) * (size_t)n);
    int *mark = (int *)malloc(sizeof(int) * (size_t)n);
    int *stack = (int *)malloc(sizeof(int) * (size_t)n);
    int *pos = (int *)malloc(sizeof(int) * (size_t)n);
    int *out = (int *)malloc(sizeof(int) * (size_t)n);
    int *seeds = (int *)malloc(sizeof(int) * (size_t)n);
    double *x = (double *)calloc((size_t)n, sizeof(double));
    ivec Li = {0}, Ui = {0};
    dvec Lx = {0}, Ux = {0};
    if (!F || !pinv || !mark || !stack || !pos || !out || !seeds || !x) goto fail;
    F->n = n;
    F->Lp = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    F->Up = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    if (!F->Lp || !F->Up) goto fail;
    for (int i = 0; i < n; i++) { pinv[i] = -1; mark[i] = -1; }
    F->Lp[0] = 0; F->Up[0] = 0;

    for (int j = 0; j < n; j++) {
        int c = Q[j];
        int ns = 0;
        for (int p = Ap[c]; p < Ap[c + 1]; p++) seeds[ns++] = Ai[p];
        /* reach through L: row r (original index) that is pivot of column
         * pinv[r] has children = rows of L(:, pinv[r]) (original indices
         * while the factorization runs) */
        int top = n;
        reach(n, seeds, ns, pinv, F->Lp, Li.a, mark, j, stack, pos, out, &top);
        for (int p = Ap[c]; p < Ap[c + 1]; p++) x[Ai[p]] += Ax[p];
        /* numeric: eliminate with the finished columns of the reach in
         * ascending pivot order (a topological order of the graph of L);
         * each update is one fused multiply-add */
        int npiv = 0;
        for (int t = top; t < n; t++) if (pinv[out[t]] >= 0) seeds[npiv++] = pinv[out[t]];
        qsort(seeds, (size_t)npiv, sizeof(int), cmp_int);
        for (int a = 0; a < npiv; a++) {
            int k = seeds[a];
            double xr = x[P[k]];
            for (int p = F->Lp[k]; p < F->Lp[k + 1]; p++) x[Li.a[p]] = fma(-Lx.a[p], xr, x[Li.a[p]]);
        }
        /* pivot search among the rows not yet pivotal */
        double amax = 0.0;
        int imax = -1;
        for (int t = top; t < n; t++) {
            int r = out[t];
            if (pinv[r] >= 0) continue;
            double a = fabs(x[r]);
            if (!isfinite(a)) { *status = OR_ERR_NONFINITE; goto fail; }
            if (imax < 0 || a > amax || (a == amax && r < imax)) { amax = a; imax = r; }
        }
        if (imax < 0 || amax == 0.0) { *status = OR_ERR_SINGULAR; goto fail; }
        int piv = imax;
        int rd = c;   /* the original diagonal entry of this column */
        if (pinv[rd] < 0 && mark[rd] == j && fabs(x[rd]) >= tol * amax) piv = rd;
        double d = x[piv];
        double dinv = 1.0 / d;   /* L(:,j) is scaled by the pivot's reciprocal */
        /* U(:,j): pivotal rows of the reach, then the diagonal */
        for (int t = top; t < n; t++) {
            int r = out[t];
            if (pinv[r] >= 0) {
                if (!ivec_push(&Ui, pinv[r]) || !dvec_push(&Ux, x[r])) goto fail;
            }
        }
        if (!ivec_push(&Ui, j) || !dvec_push(&Ux, d)) goto fail;
        /* L(:,j): the other non-pivotal rows, divided by the pivot */
        for (int t = top; t < n; t++) {
            int r = out[t];
            if (pinv[r] < 0 && r != piv) {
                if (!ivec_push(&Li, r) || !dvec_push(&Lx, x[r] * dinv)) goto fail;
            }
        }
        pinv[piv] = j;
        P[j] = piv;
        for (int t = top; t < n; t++) x[out[t]] = 0.0;
        F->Lp[j + 1] = (int)Li.n;
        F->Up[j + 1] = (int)Ui.n;
    }
    /* L rows to the permuted space */
    for (long p = 0; p < Li.n; p++) Li.a[p] = pinv[Li.a[p]];
    F->Li = Li.a; F->Lx = Lx.a; F->Ui = Ui.a; F->Ux = Ux.a;
    if (!F->Li) { F->Li = (int *)malloc(sizeof(int)); F->Lx = (double *)malloc(sizeof(double)); }
    sort_columns(n, F->Lp, F->Li, F->Lx);
    sort_columns(n, F->Up, F->Ui, F->Ux);
    free(pinv); free(mark); free(stack); free(pos); free(out); free(seeds); free(x);
    *status = OR_OK;
    return F;
fail:
    free(pinv); free(mark); free(stack); free(pos); free(out); free(seeds); free(x);
    free(Li.a); free(Lx.a); free(Ui.a); free(Ux.a);
    if (F) { F->Li = NULL; F->Lx = NULL; F->Ui = NULL; F->Ux = NULL; or_factor_free(F); }
    return NULL;
}

/* ------------------------------------------------------------------ */
/* Refactorization with a given pivot sequence P and column order Q.   */
/* boost_abs > 0 turns on the static-pivot boost: |u_jj| < boost_abs is */
/* replaced by sign(u_jj) * boost_abs (sign(0) = +1) and counted.       */
/* boost_abs == 0: an exact zero pivot is an error.                     */
/* budget_s > 0 (the bounded CPU-baseline sample only): stop at the first  */
/* column reached after budget_s seconds; *cols_done and                    */
/* *madds get the columns finished and the multiply-adds they took.  The   */
/* arithmetic of every finished column is the same either way.             */
static double wall_seconds(void) {
    struct timespec ts;
    clock_gettime(CLOCK_MONOTONIC, &ts);
    return (double)ts.tv_sec + 1e-9 * (double)ts.tv_nsec;
}

static void *refactor_run(int n, const int *Ap, const int *Ai, const double *Ax,
                          const int *P, const int *Q, double boost_abs, double budget_s,
                          int *cols_done, double *madds, double *marks, int nmarks, int *status) {
    const double t_start = budget_s > 0.0 ? wall_seconds() : 0.0;
    double nmadd = 0.0;
    int jend = n;
    *status = OR_ERR_OOM;
    or_factors *F = (or_factors *)calloc(1, sizeof(or_factors));
    int *pinv = (int *)malloc(sizeof(int) * (size_t)n);
    int *colof = (int *)malloc(sizeof(int) * (size_t)n);
    int *mark = (int *)malloc(sizeof(int) * (size_t)n);
    int *stack = (int *)malloc(sizeof(int) * (size_t)n);
    int *pos = (int *)malloc(sizeof(int) * (size_t)n);
    int *out = (int *)malloc(sizeof(int) * (size_t)n);
    int *seeds = (int *)malloc(sizeof(int) * (size_t)n);
    double *x = (double *)calloc((size_t)n, sizeof(double));
    ivec Li = {0}, Ui = {0};
    dvec Lx = {0}, Ux = {0};
    if (!F || !pinv || !colof || !mark || !stack || !pos || !out || !seeds || !x) goto fail;
    F->n = n;
    F->Lp = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    F->Up = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    if (!F->Lp || !F->Up) goto fail;
    for (int i = 0; i < n; i++) { pinv[i] = -1; mark[i] = -1; colof[i] = -1; }
    for (int k = 0; k < n; k++) {
        if (P[k] < 0 || P[k] >= n || pinv[P[k]] >= 0) { *status = OR_ERR_PATTERN; goto fail; }
        pinv[P[k]] = k;
    }
    F->Lp[0] = 0; F->Up[0] = 0;
    for (int j = 0; j < n; j++) {
        if (budget_s > 0.0 && j > 0) {
            const double el = wall_seconds() - t_start;
            /* checkpoint every 256 columns: columns, multiply-adds, stored
             * factor entries, seconds (the sample's cost profile) */
            if (marks && (j & 255) == 0 && (j >> 8) <= nmarks) {
                double *mk = marks + 4 * ((j >> 8) - 1);
                mk[0] = (double)j; mk[1] = nmadd; mk[2] = (double)(Li.n + Ui.n); mk[3] = el;
            }
            if (el >= budget_s) { jend = j; break; }
        }
        int c = Q[j];
        int ns = 0;
        for (int p = Ap[c]; p < Ap[c + 1]; p++) seeds[ns++] = pinv[Ai[p]];
        int top = n;
        /* permuted row i < j has children = rows of L(:, i) */
        reach(n, seeds, ns, colof, F->Lp, Li.a, mark, j, stack, pos, out, &top);
        for (int p = Ap[c]; p < Ap[c + 1]; p++) x[pinv[Ai[p]]] += Ax[p];
        /* finished columns in ascending pivot order (a topological order of
         * the graph of L), one fused multiply-add per update */
        qsort(out + top, (size_t)(n - top), sizeof(int), cmp_int);
        for (int t = top; t < n; t++) {
            int i = out[t];
            if (i >= j) break;
            double xi = x[i];
            for (int p = F->Lp[i]; p < F->Lp[i + 1]; p++) x[Li.a[p]] = fma(-Lx.a[p], xi, x[Li.a[p]]);
            nmadd += (double)(F->Lp[i + 1] - F->Lp[i]);
        }
        if (mark[j] != j) { *status = OR_ERR_SINGULAR; goto fail; }
        double d = x[j];
        if (!isfinite(d)) { *status = OR_ERR_NONFINITE; goto fail; }
        if (boost_abs > 0.0) {
            if (fabs(d) < boost_abs) { d = (d < 0.0) ? -boost_abs : boost_abs; F->nboost++; }
        } else if (d == 0.0) {
            *status = OR_ERR_SINGULAR; goto fail;
        }
        for (int t = top; t < n; t++) {
            int i = out[t];
            if (i < j) { if (!ivec_push(&Ui, i) || !dvec_push(&Ux, x[i])) goto fail; }
        }
        if (!ivec_push(&Ui, j) || !dvec_push(&Ux, d)) goto fail;
        double rd = 1.0 / d;   /* L(:,j) is scaled by the pivot's reciprocal */
        for (int t = top; t < n; t++) {
            int i = out[t];
            if (i > j) {
                double l = x[i] * rd;
                if (!isfinite(l)) { *status = OR_ERR_NONFINITE; goto fail; }
                if (!ivec_push(&Li, i) || !dvec_push(&Lx, l)) goto fail;
            }
        }
        colof[j] = j;
        for (int t = top; t < n; t++) x[out[t]] = 0.0;
        F->Lp[j + 1] = (int)Li.n;
        F->Up[j + 1] = (int)Ui.n;
    }
    if (cols_done) *cols_done = jend;
    if (madds) *madds = nmadd;
    if (jend < n) {   /* a bounded sample stopped early: no factors to return */
        free(pinv); free(colof); free(mark); free(stack); free(pos); free(out); free(seeds); free(x);
        free(Li.a); free(Lx.a); free(Ui.a); free(Ux.a);
        F->Li = NULL; F->Lx = NULL; F->Ui = NULL; F->Ux = NULL;
        or_factor_free(F);
        *status = OR_OK;
        return NULL;
    }
    F->Li = Li.a; F->Lx = Lx.a; F->Ui = Ui.a; F->Ux = Ux.a;
    if (!F->Li) { F->Li = (int *)malloc(sizeof(int)); F->Lx = (double *)malloc(sizeof(double)); }
    sort_columns(n, F->Lp, F->Li, F->Lx);
    sort_columns(n, F->Up, F->Ui, F->Ux);
    free(pinv); free(colof); free(mark); free(stack); free(pos); free(out); free(seeds); free(x);
    *status = OR_OK;
    return F;
fail:
    free(pinv); free(colof); free(mark); free(stack); free(pos); free(out); free(seeds); free(x);
    free(Li.a); free(Lx.a); free(Ui.a); free(Ux.a);
    if (F) { F->Li = NULL; F->Lx = NULL; F->Ui = NULL; F->Ux = NULL; or_factor_free(F); }
    return NULL;
}

void *or_refactor(int n, const int *Ap, const int *Ai, const double *Ax,
                  const int *P, const int *Q, double boost_abs, int *status) {
    return refactor_run(n, Ap, Ai, Ax, P, Q, boost_abs, 0.0, NULL, NULL, NULL, 0, status);
}

/* CPU-baseline sample: the refactorization above, stopped after about     */
/* budget_s seconds (all columns if it finishes first).  Returns the       */
/* status; *cols_done and *madds as in refactor_run; marks[4 k .. 4 k + 3] */
/* (k < nmarks) the checkpoint after 256 (k + 1) columns.                  */
int or_refactor_sample(int n, const int *Ap, const int *Ai, const double *Ax,
                       const int *P, const int *Q, double budget_s, int *cols_done, double *madds,
                       double *marks, int nmarks) {
    int st = OR_OK;
    void *h = refactor_run(n, Ap, Ai, Ax, P, Q, 0.0, budget_s, cols_done, madds, marks, nmarks, &st);
    or_factor_free(h);
    return st;
}

/* ------------------------------------------------------------------ */
/* The same refactorization in FP32 arithmetic (mixed precision: FP32   */
/* factors as the FGMRES preconditioner, Section 2.1's inexact factors). */
/* Values are rounded to float, every update is fmaf, the L column is   */
/* scaled by the float reciprocal 1.0f / u_jj; the factors are returned */
/* widened (exactly) to double.  boost_abs as in or_refactor.            */
void *or_refactor_f32(int n, const int *Ap, const int *Ai, const double *Ax,
                      const int *P, const int *Q, double boost_abs, int *status) {
    *status = OR_ERR_OOM;
    or_factors *F = (or_factors *)calloc(1, sizeof(or_factors));
    int *pinv = (int *)malloc(sizeof(int) * (size_t)n);
    int *colof = (int *)malloc(sizeof(int) * (size_t)n);
    int *mark = (int *)malloc(sizeof(int) * (size_t)n);
    int *stack = (int *)malloc(sizeof(int) * (size_t)n);
    int *pos = (int *)malloc(sizeof(int) * (size_t)n);
    int *out = (int *)malloc(sizeof(int) * (size_t)n);
    int *seeds = (int *)malloc(sizeof(int) * (size_t)n);
    float *x = (float *)calloc((size_t)n, sizeof(float));
    float *lxf = NULL;   /* L values in float while factorizing */
    long lcap = 0;
    ivec Li = {0}, Ui = {0};
    dvec Lx = {0}, Ux = {0};
    const float boost = (float)boost_abs;
    if (!F || !pinv || !colof || !mark || !stack || !pos || !out || !seeds || !x) goto fail;
    F->n = n;
    F->Lp = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    F->Up = (int *)malloc(sizeof(int) * (size_t)(n + 1));
    if (!F->Lp || !F->Up) goto fail;
    for (int i = 0; i < n; i++) { pinv[i] = -1; mark[i] = -1; colof[i] = -1; }
    for (int k = 0; k < n; k++) {
        if (P[k] < 0 || P[k] >= n || pinv[P[k]] >= 0) { *status = OR_ERR_PATTERN; goto fail; }
        pinv[P[k]] = k;
    }
    F->Lp[0] = 0; F->Up[0] = 0;
    for (int j = 0; j < n; j++) {
        int c = Q[j];
        int ns = 0;
        for (int p = Ap[c]; p < Ap[c + 1]; p++) seeds[ns++] = pinv[Ai[p]];
        int top = n;
        reach(n, seeds, ns, colof, F->Lp, Li.a, mark, j, stack, pos, out, &top);
        for (int p = Ap[c]; p < Ap[c + 1]; p++) x[pinv[Ai[p]]] = (float)Ax[p];
        qsort(out + top, (size_t)(n - top), sizeof(int), cmp_int);
        for (int t = top; t < n; t++) {
            int i = out[t];
            if (i >= j) break;
            float xi = x[i];
            for (int p = F->Lp[i]; p < F->Lp[i + 1]; p++) x[Li.a[p]] = fmaf(-lxf[p], xi, x[Li.a[p]]);
        }
        if (mark[j] != j) { *status = OR_ERR_SINGULAR; goto fail; }
        float d = x[j];
        if (!isfinite(d)) { *status = OR_ERR_NONFINITE; goto fail; }
        if (boost > 0.0f) {
            if (fabsf(d) < boost) { d = (d < 0.0f) ? -boost : boost; F->nboost++; }
        } else if (d == 0.0f) {
            *status = OR_ERR_SINGULAR; goto fail;
        }
        for (int t = top; t < n; t++) {
            int i = out[t];
            if (i < j) { if (!ivec_push(&Ui, i) || !dvec_push(&Ux, (double)x[i])) goto fail; }
        }
        if (!ivec_push(&Ui, j) || !dvec_push(&Ux, (double)d)) goto fail;
        float dinv = 1.0f / d;
        for (int t = top; t < n; t++) {
            int i = out[t];
            if (i > j) {
                float l = x[i] * dinv;
                if (!isfinite(l)) { *status = OR_ERR_NONFINITE; goto fail; }
                if (!ivec_push(&Li, i) || !dvec_push(&Lx, (double)l)) goto fail;
                if (Li.n > lcap) {
                    long nc = lcap ? 2 * lcap : 1024;
                    while (nc < Li.n) nc *= 2;
                    float *q = (float *)realloc(lxf, sizeof(float) * (size_t)nc);
                    if (!q) goto fail;
                    lxf = q; lcap = nc;
                }
                lxf[Li.n - 1] = l;
            }
        }
        colof[j] = j;
        for (int t = top; t < n; t++) x[out[t]] = 0.0f;
        F->Lp[j + 1] = (int)Li.n;
        F->Up[j + 1] = (int)Ui.n;
    }
    F->Li = Li.a; F->Lx = Lx.a; F->Ui = Ui.a; F->Ux = Ux.a;
    if (!F->Li) { F->Li = (int *)malloc(sizeof(int)); F->Lx = (double *)malloc(sizeof(double)); }
    sort_columns(n, F->Lp, F->Li, F->Lx);
    sort_columns(n, F->Up, F->Ui, F->Ux);
    free(pinv); free(colof); free(mark); free(stack); free(pos); free(out); free(seeds); free(x); free(lxf);
    *status = OR_OK;
    return F;
fail:
    free(pinv); free(colof); free(mark); free(stack); free(pos); free(out); free(seeds); free(x); free(lxf);
    free(Li.a); free(Lx.a); free(Ui.a); free(Ux.a);
    if (F) { F->Li = NULL; F->Lx = NULL; F->Ui = NULL; F->Ux = NULL; or_factor_free(F); }
    return NULL;
}

/* ------------------------------------------------------------------ */
/* Triangular solve x = Q U^{-1} L^{-1} P b  (b and x may not alias).   */
void or_solve(void *h, const int *P, const int *Q, const double *b, double *x) {
    or_factors *F = (or_factors *)h;
    int n = F->n;
    double *y = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    for (int i = 0; i < n; i++) y[i] = b[P[i]];
    /* forward substitution, unit lower L, column by column */
    for (int j = 0; j < n; j++) {
        double yj = y[j];
        for (int p = F->Lp[j]; p < F->Lp[j + 1]; p++) y[F->Li[p]] -= F->Lx[p] * yj;
    }
    /* backward substitution with U; its diagonal is the last entry of
     * each sorted column */
    for (int j = n - 1; j >= 0; j--) {
        int pd = F->Up[j + 1] - 1;
        y[j] /= F->Ux[pd];
        double yj = y[j];
        for (int p = F->Up[j]; p < pd; p++) y[F->Ui[p]] -= F->Ux[p] * yj;
    }
    for (int j = 0; j < n; j++) x[Q[j]] = y[j];
    free(y);
}

/* ------------------------------------------------------------------ */
/* norms and the backward-error measures                               */
static double nrm2(int n, const double *v) {
    double s = 0.0;
    for (int i = 0; i < n; i++) s += v[i] * v[i];
    return sqrt(s);
}

/* ||K||_inf: maximum absolute row sum (CSR). */
double or_norm_inf(int n, const int *rp, const double *vals) {
    double m = 0.0;
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; p++) s += fabs(vals[p]);
        if (s > m) m = s;
    }
    return m;
}

/* r = b - K x (CSR). */
void or_residual(int n, const int *rp, const int *ci, const double *vals,
                 const double *b, const double *x, double *r) {
    for (int i = 0; i < n; i++) {
        double s = 0.0;
        for (int p = rp[i]; p < rp[i + 1]; p++) s += vals[p] * x[ci[p]];
        r[i] = b[i] - s;
    }
}

/* NRBE = ||b - Kx||_2 / (||K||_inf ||x||_2 + ||b||_2), Eq. (nbre). */
double or_nrbe(int n, const int *rp, const int *ci, const double *vals,
               const double *b, const double *x) {
    double *r = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    or_residual(n, rp, ci, vals, b, x, r);
    double num = nrm2(n, r);
    double den = or_norm_inf(n, rp, vals) * nrm2(n, x) + nrm2(n, b);
    free(r);
    if (num == 0.0) return 0.0;
    return num / den;
}

/* NSR = ||b - Kx||_inf / (||K||_inf ||x||_inf), the MA57 measure of Section 1.3. */
double or_nsr(int n, const int *rp, const int *ci, const double *vals,
              const double *b, const double *x) {
    double *r = (double *)malloc(sizeof(double) * (size_t)(n ? n : 1));
    or_residual(n, rp, ci, vals, b, x, r);
    double num = 0.0, xm = 0.0;
    for (int i = 0; i < n; i++) {
        if (fabs(r[i]) > num) num = fabs(r[i]);
        if (fabs(x[i]) > xm) xm = fabs(x[i]);
    }
    double den = or_norm_inf(n, rp, vals) * xm;
    free(r);
    if (num == 0.0) return 0.0;
    return num / den;
}

/* sqrt(a^2 - ||h||^2) in the factored form sqrt((a - c)(a + c)),
 * c = ||h||; zero when a <= c.  (The norm of the projected vector from
 * the norms before the projection, Pythagoras.) */
static double pythagoras(double a, const double *h, int k) {
    double c = 0.0;
    for (int i = 0; i < k; i++) c += h[i] * h[i];
    c = sqrt(c);
    if (!(a > c)) return 0.0;
    return sqrt((a - c) * (a + c));
}

/* ------------------------------------------------------------------ */
/* FGMRES(m) iterative refinement with right preconditioner M = LU.     */
/*                                                                      */
/* stop_mode 0 (NRBE): the inner loop stops when the estimated residual  */
/*   |g_{j+1}| <= tol (||K||_inf ||x_c||_2 + ||b||_2), x_c the iterate   */
/*   at the start of the cycle; the cycle then forms x and accepts it if */
/*   the true NRBE <= tol, else restarts.                                */
/* stop_mode 1 (RR, the paper's rule): stop when the estimated residual  */
/*   |g_{j+1}| < tol ||rho^(0)||, rho^(0) = b - K x0.                    */
/* refine_delta > 0: no refinement when ||b - K x0|| / ||b|| < delta     */
/*   (Section 2.3).                                                      */
/* An iteration is one Arnoldi step (one more preconditioner apply).     */
/* out: x, *iters, *cycles, *nrbe_out; trace (optional, length          */
/*   >= 1 + max_cycles*m) receives the estimated residual after each     */
/*   iteration with trace[0] = ||rho^(0)||.                             */
/*                                                                      */
/* or_fgmres_ex adds:                                                    */
/* ortho 0: CGS2 -- h = V^T w, w -= V h, h2 = V^T w, w -= V h2,          */
/*   h_{j+1,j} = ||w||.                                                  */
/* ortho 1: CGS2 with the norm by Pythagoras -- ||w'||^2 is reduced      */
/*   together with h2 = V^T w' (w' = w after the first projection) and   */
/*   h_{j+1,j} = sqrt((a - c)(a + c)), a = ||w'||, c = ||h2||.            */
/* ortho 2: one-reduction CGS -- h = V^T w and ||w||^2 in one reduction, */
/*   w -= V h, h_{j+1,j} = sqrt((a - c)(a + c)), a = ||w||, c = ||h||.    */
/*   With a <= c the norm is taken as zero (breakdown: the cycle ends).  */
/* inner 0: the cycle's inner test is the stop_mode rule above.          */
/* inner 1: FGMRES on the error equation -- the inner test is            */
/*   |g_{j+1}| <= inner_tol * beta (beta = ||rho|| at the cycle start);   */
/*   after the cycle x += Z y, the true residual is recomputed and x is  */
/*   accepted on the stop_mode rule (NRBE <= tol, or RR:                  */
/*   ||rho|| < tol ||rho^(0)||).                                         */
int or_fgmres_ex(int n, const int *rp, const int *ci, const double *vals,
                 void *fac, const int *P, const int *Q,
                 const double *b, double *x,
                 int m, int max_cycles, double tol, int stop_mode, double refine_delta,
                 int ortho, int inner, double inner_tol,
                 int *iters, int *cycles, double *nrbe_out, double *trace) {
    size_t N = (size_t)(n ? n : 1);
    double *V = (double *)malloc(sizeof(double) * N * (size_t)(m + 1));
    double *Z = (double *)malloc(sizeof(double) * N * (size_t)m);
    double *H = (double *)calloc((size_t)(m + 1) * (size_t)m, sizeof(double));
    double *cs = (double *)malloc(sizeof(double) * (size_t)m);
    double *sn = (double *)malloc(sizeof(double) * (size_t)m);
    double *g = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *y = (double *)malloc(sizeof(double) * (size_t)m);
    double *h = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *h2 = (double *)malloc(sizeof(double) * (size_t)(m + 1));
    double *r = (double *)malloc(sizeof(double) * N);
    double *w = (double *)malloc(sizeof(double) * N);
    int ntrace = 0;
    int rc = OR_OK;
    if (!V || !Z || !H || !cs || !sn || !g || !y || !h || !h2 || !r || !w) { rc = OR_ERR_OOM; goto done; }

    double normK = or_norm_inf(n, rp, vals);
    double normb = nrm2(n, b);
    *iters = 0; *cycles = 0;

    /* x0 = (LU)^{-1} b, the direct solve (initial guess) */
    or_solve(fac, P, Q, b, x);
    or_residual(n, rp, ci, vals, b, x, r);
    double rnorm = nrm2(n, r);
    double nrbe = (rnorm == 0.0) ? 0.0 : rnorm / (normK * nrm2(n, x) + normb);
    double rho0 = rnorm;
    if (trace) trace[ntrace++] = rnorm;
    for (int i = 0; i < n; i++) if (!isfinite(x[i])) { rc = OR_ERR_NONFINITE; goto done_nrbe; }
    if (rnorm == 0.0) goto done_nrbe;
    if (refine_delta > 0.0 && rnorm < refine_delta * normb) goto done_nrbe;
    if (stop_mode == 0 && nrbe <= tol) goto done_nrbe;

    for (;;) {
        if (*cycles >= max_cycles) { rc = OR_ERR_NOT_CONVERGED; break; }
        (*cycles)++;
        double beta = rnorm;
        double thresh = inner == 1 ? inner_tol * beta
                      : (stop_mode == 0) ? tol * (normK * nrm2(n, x) + normb) : tol * rho0;
        for (int i = 0; i < n; i++) V[i] = r[i] / beta;
        g[0] = beta;
        for (int i = 1; i <= m; i++) g[i] = 0.0;
        int jend = 0;
        int met = 0;
        for (int j = 0; j < m; j++) {
            double *vj = V + (size_t)j * N;
            double *zj = Z + (size_t)j * N;
            or_solve(fac, P, Q, vj, zj);                 /* z_j = M^{-1} v_j */
            /* w = K z_j */
            for (int i = 0; i < n; i++) {
                double s = 0.0;
                for (int p = rp[i]; p < rp[i + 1]; p++) s += vals[p] * zj[ci[p]];
                w[i] = s;
            }
            /* first classical Gram-Schmidt projection (all variants) */
            double wn_before = (ortho == 2) ? nrm2(n, w) : 0.0;   /* same reduction as h */
            for (int i = 0; i <= j; i++) {
                double s = 0.0; const double *vi = V + (size_t)i * N;
                for (int t = 0; t < n; t++) s += vi[t] * w[t];
                h[i] = s;
            }
            for (int i = 0; i <= j; i++) {
                const double *vi = V + (size_t)i * N;
                for (int t = 0; t < n; t++) w[t] -= h[i] * vi[t];
            }
            double hn;
            if (ortho == 2) {
                hn = pythagoras(wn_before, h, j + 1);
            } else {
                /* second projection (re-orthogonalisation) */
                double wn_mid = (ortho == 1) ? nrm2(n, w) : 0.0;   /* same reduction as h2 */
                for (int i = 0; i <= j; i++) {
                    double s = 0.0; const double *vi = V + (size_t)i * N;
                    for (int t = 0; t < n; t++) s += vi[t] * w[t];
                    h2[i] = s;
                }
                for (int i = 0; i <= j; i++) {
                    const double *vi = V + (size_t)i * N;
                    for (int t = 0; t < n; t++) w[t] -= h2[i] * vi[t];
                }
                hn = (ortho == 1) ? pythagoras(wn_mid, h2, j + 1) : nrm2(n, w);
                for (int i = 0; i <= j; i++) h[i] += h2[i];
            }
            double *vn = V + (size_t)(j + 1) * N;
            if (hn > 0.0) { for (int t = 0; t < n; t++) vn[t] = w[t] / hn; }
            else { for (int t = 0; t < n; t++) vn[t] = 0.0; }
            /* column j of the Hessenberg matrix, previous rotations applied */
            double *Hj = H + (size_t)j * (size_t)(m + 1);
            for (int i = 0; i <= j; i++) Hj[i] = h[i];
            Hj[j + 1] = hn;
            for (int i = 0; i < j; i++) {
                double a = Hj[i], bb = Hj[i + 1];
                Hj[i] = cs[i] * a + sn[i] * bb;
                Hj[i + 1] = -sn[i] * a + cs[i] * bb;
            }
            /* new rotation zeroing H(j+1, j) */
            double a = Hj[j], bb = Hj[j + 1];
            double rr = hypot(a, bb);
            if (rr == 0.0) { cs[j] = 1.0; sn[j] = 0.0; }
            else { cs[j] = a / rr; sn[j] = bb / rr; }
            Hj[j] = rr;
            Hj[j + 1] = 0.0;
            g[j + 1] = -sn[j] * g[j];
            g[j] = cs[j] * g[j];
            (*iters)++;
            jend = j + 1;
            if (trace) trace[ntrace++] = fabs(g[j + 1]);
            if (stop_mode == 0 ? (fabs(g[j + 1]) <= thresh) : (fabs(g[j + 1]) < thresh)) { met = 1; break; }
            if (hn == 0.0) break;   /* invariant subspace: the estimate is exact */
        }
        /* y = R^{-1} g, back substitution on the rotated Hessenberg matrix */
        for (int i = jend - 1; i >= 0; i--) {
            double s = g[i];
            for (int k = i + 1; k < jend; k++) s -= H[(size_t)k * (size_t)(m + 1) + (size_t)i] * y[k];
            y[i] = s / H[(size_t)i * (size_t)(m + 1) + (size_t)i];
        }
        for (int k = 0; k < jend; k++) {
            const double *zk = Z + (size_t)k * N;
            for (int t = 0; t < n; t++) x[t] += y[k] * zk[t];
        }
        or_residual(n, rp, ci, vals, b, x, r);
        rnorm = nrm2(n, r);
        nrbe = (rnorm == 0.0) ? 0.0 : rnorm / (normK * nrm2(n, x) + normb);
        if (rnorm == 0.0) break;
        if (stop_mode == 0 && nrbe <= tol) break;
        if (stop_mode == 1 && (inner == 1 ? rnorm < tol * rho0 : met)) break;
    }
done_nrbe:
    *nrbe_out = nrbe;
done:
    free(V); free(Z); free(H); free(cs); free(sn); free(g); free(y); free(h); free(h2); free(r); free(w);
    return rc;
}

int or_fgmres(int n, const int *rp, const int *ci, const double *vals,
              void *fac, const int *P, const int *Q,
              const double *b, double *x,
              int m, int max_cycles, double tol, int stop_mode, double refine_delta,
              int *iters, int *cycles, double *nrbe_out, double *trace) {
    return or_fgmres_ex(n, rp, ci, vals, fac, P, Q, b, x, m, max_cycles, tol, stop_mode, refine_delta,
                        0, 0, 0.0, iters, cycles, nrbe_out, trace);
}

/* ------------------------------------------------------------------ */
/* Classical iterative refinement (Section 2.1, the error system):       */
/*   x0 = (LU)^{-1} b; repeat: rho = b - K x; stop on the rule; d =       */
/*   (LU)^{-1} rho; x += d.                                              */
/* Stop rules as in or_fgmres on the true residual (NRBE <= tol, or RR:  */
/* ||rho|| < tol ||rho^(0)||), and refine_delta as there.  An iteration  */
/* is one correction (one preconditioner apply after x0); at most        */
/* max_steps.  trace (optional, >= 1 + max_steps) receives ||rho|| after */
/* x0 and after every correction.                                        */
int or_richardson(int n, const int *rp, const int *ci, const double *vals,
                  void *fac, const int *P, const int *Q,
                  const double *b, double *x,
                  int max_steps, double tol, int stop_mode, double refine_delta,
                  int *iters, double *nrbe_out, double *trace) {
    size_t N = (size_t)(n ? n : 1);
    double *r = (double *)malloc(sizeof(double) * N);
    double *d = (double *)malloc(sizeof(double) * N);
    if (!r || !d) { free(r); free(d); return OR_ERR_OOM; }
    double normK = or_norm_inf(n, rp, vals);
    double normb = nrm2(n, b);
    int rc = OR_OK;
    *iters = 0;
    or_solve(fac, P, Q, b, x);
    double rho0 = 0.0, nrbe = 0.0;
    for (int k = 0;; k++) {
        or_residual(n, rp, ci, vals, b, x, r);
        double rnorm = nrm2(n, r);
        double xnorm = nrm2(n, x);
        if (!isfinite(rnorm) || !isfinite(xnorm)) { rc = OR_ERR_NONFINITE; break; }
        nrbe = (rnorm == 0.0) ? 0.0 : rnorm / (normK * xnorm + normb);
        if (trace) trace[k] = rnorm;
        if (k == 0) {
            rho0 = rnorm;
            if (refine_delta > 0.0 && rnorm < refine_delta * normb) break;
        }
        if (rnorm == 0.0) break;
        if (stop_mode == 0 ? (nrbe <= tol) : (k > 0 && rnorm < tol * rho0)) break;
        if (k >= max_steps) { rc = OR_ERR_NOT_CONVERGED; break; }
        or_solve(fac, P, Q, r, d);
        for (int i = 0; i < n; i++) x[i] += d[i];
        (*iters)++;
    }
    *nrbe_out = nrbe;
    free(r); free(d);
    return rc;
}

/* ------------------------------------------------------------------ */
/* Fill-reducing column ordering: exact minimum degree on the graph of  */
/* A^T A (columns adjacent when they share a row), explicit elimination */
/* graph.  Input A in CSR (row lists of column indices).                */
typedef struct { int *a; int n, cap; } iset;   /* sorted set */

static int iset_reserve(iset *s, int cap) {
    if (cap <= s->cap) return 1;
    int c = s->cap ? s->cap : 8;
    while (c < cap) c *= 2;
    int *p = (int *)realloc(s->a, sizeof(int) * (size_t)c);
    if (!p) return 0;
    s->a = p; s->cap = c;
    return 1;
}

/* binary min-heap of (degree, index) with lazy deletion */
typedef struct { long *k; int n, cap; } heap;
static int heap_push(heap *h, long key) {
    if (h->n == h->cap) {
        int c = h->cap ? 2 * h->cap : 1024;
        long *p = (long *)realloc(h->k, sizeof(long) * (size_t)c);
        if (!p) return 0;
        h->k = p; h->cap = c;
    }
    int i = h->n++;
    h->k[i] = key;
    while (i > 0) {
        int pa = (i - 1) / 2;
        if (h->k[pa] <= h->k[i]) break;
        long t = h->k[pa]; h->k[pa] = h->k[i]; h->k[i] = t;
        i = pa;
    }
    return 1;
}
static long heap_pop(heap *h) {
    long top = h->k[0];
    h->k[0] = h->k[--h->n];
    int i = 0;
    for (;;) {
        int l = 2 * i + 1, r = l + 1, s = i;
        if (l < h->n && h->k[l] < h->k[s]) s = l;
        if (r < h->n && h->k[r] < h->k[s]) s = r;
        if (s == i) break;
        long t = h->k[s]; h->k[s] = h->k[i]; h->k[i] = t;
        i = s;
    }
    return top;
}

int or_order_md(int n, const int *rp, const int *ci, int *Q) {
    iset *adj = (iset *)calloc((size_t)(n ? n : 1), sizeof(iset));
    int *elim = (int *)calloc((size_t)(n ? n : 1), sizeof(int));
    int *tmp = NULL;
    int tcap = 0;
    heap hp = {0};
    int rc = OR_ERR_OOM;
    if (!adj || !elim) goto out;
    /* column adjacency from row cliques */
    {
        int *cnt = (int *)calloc((size_t)(n ? n : 1), sizeof(int));
        if (!cnt) goto out;
        for (int i = 0; i < n; i++) {
            int len = rp[i + 1] - rp[i];
            for (int p = rp[i]; p < rp[i + 1]; p++) cnt[ci[p]] += len;
        }
        for (int c = 0; c < n; c++) if (!iset_reserve(&adj[c], cnt[c] + 1)) { free(cnt); goto out; }
        free(cnt);
        for (int i = 0; i < n; i++)
            for (int p = rp[i]; p < rp[i + 1]; p++)
                for (int q = rp[i]; q < rp[i + 1]; q++)
                    if (ci[p] != ci[q]) adj[ci[p]].a[adj[ci[p]].n++] = ci[q];
        for (int c = 0; c < n; c++) {
            iset *s = &adj[c];
            qsort(s->a, (size_t)s->n, sizeof(int), cmp_int);
            int w = 0;
            for (int t = 0; t < s->n; t++) if (w == 0 || s->a[w - 1] != s->a[t]) s->a[w++] = s->a[t];
            s->n = w;
        }
    }
    for (int c = 0; c < n; c++) if (!heap_push(&hp, (long)adj[c].n * (long)(n + 1) + c)) goto out;
    for (int k = 0; k < n; k++) {
        int v;
        for (;;) {
            long key = heap_pop(&hp);
            v = (int)(key % (n + 1));
            long d = key / (n + 1);
            if (!elim[v] && d == adj[v].n) break;
        }
        Q[k] = v;
        elim[v] = 1;
        iset *nv = &adj[v];
        /* each neighbour u: adj(u) <- adj(u) U adj(v) \ {u, v} */
        for (int t = 0; t < nv->n; t++) {
            int u = nv->a[t];
            iset *su = &adj[u];
            int need = su->n + nv->n;
            if (need > tcap) {
                int *p = (int *)realloc(tmp, sizeof(int) * (size_t)need);
                if (!p) goto out;
                tmp = p; tcap = need;
            }
            int a = 0, b2 = 0, w = 0;
            while (a < su->n || b2 < nv->n) {
                int xa = (a < su->n) ? su->a[a] : 0x7fffffff;
                int xb = (b2 < nv->n) ? nv->a[b2] : 0x7fffffff;
                int x;
                if (xa < xb) { x = xa; a++; }
                else if (xb < xa) { x = xb; b2++; }
                else { x = xa; a++; b2++; }
                if (x != u && x != v) tmp[w++] = x;
            }
            if (!iset_reserve(su, w)) goto out;
            memcpy(su->a, tmp, sizeof(int) * (size_t)w);
            su->n = w;
            if (!heap_push(&hp, (long)w * (long)(n + 1) + u)) goto out;
        }
        free(nv->a); nv->a = NULL; nv->n = nv->cap = 0;
    }
    rc = OR_OK;
out:
    if (adj) { for (int c = 0; c < n; c++) free(adj[c].a); }
    free(adj); free(elim); free(tmp); free(hp.k);
    return rc;
}
