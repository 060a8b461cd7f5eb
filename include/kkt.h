/*
 * kkt.h -- C ABI of the GPU-resident refactorization + FGMRES KKT solver
 * (B300, sm_103a).  Method: arXiv 2401.13926.
 *
 * The solver targets a sequence of linear systems K_k x_k = r_k that share
 * one sparsity pattern (Section 1.2, Eq. (kktlinear) and its Summary).  The
 * four solver steps of Section 1.3 map to this interface as follows:
 *   1. symbolic decomposition  -> kkt_analyze (host, once per pattern)
 *   2. numeric decomposition   -> kkt_analyze (first matrix, with pivoting,
 *                                 host) and kkt_refactor (every later matrix,
 *                                 fixed pivots, GPU)
 *   3. triangular solve        -> kkt_solve (GPU), kkt_lu_solve (GPU)
 *   4. iterative refinement    -> kkt_solve: FGMRES with the LU factors as
 *                                 right preconditioner, CGS2, estimated
 *                                 residual, solution formed at restart or
 *                                 convergence (Section 2.1), refine-or-not
 *                                 test of Section 2.3, stopping rules of
 *                                 Section 2.2.
 *
 * Conventions
 *   - Matrices: CSR, 0-based, int32 indices, FP64 values, square n x n, the
 *     full matrix (both triangles).  Rows need not be sorted; duplicates and
 *     out-of-range indices are rejected with KKT_ERR_PATTERN.
 *   - Permutations: B = K(P, Q), B[i][j] = K[P[i]][Q[j]]; B = L U with L unit
 *     lower and U upper triangular.  P is the pivot sequence, Q the column
 *     (fill-reducing) order.
 *   - Ownership: the caller owns every buffer it passes; no pointer is kept
 *     after a call returns.  The context owns all device memory; it is
 *     allocated in kkt_analyze only, never in kkt_refactor or kkt_solve
 *     (buffer reuse across the sequence, Section 2.1).
 *   - Streams: every device operation of a context is ordered on its stream
 *     (kkt_opts.stream, or a stream the context creates).  Calls return after
 *     their results are complete (host-visible scalars are read back).
 *   - Errors: every call returns KKT_OK (0) or a negative KKT_ERR_* code.
 *     kkt_strerror gives a message; kkt_last_error_detail gives detail for
 *     the context's last failure (for example the offending row).
 *   - Thread safety: one context must not be used from two threads at once.
 */
#ifndef KKT_B300_H
#define KKT_B300_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define KKT_OK 0
#define KKT_ERR_INVALID (-1)        /* bad argument or option */
#define KKT_ERR_PATTERN (-2)        /* malformed or mismatched sparsity pattern */
#define KKT_ERR_OOM (-3)            /* device or host allocation failed */
#define KKT_ERR_ZERO_PIVOT (-4)     /* exact zero (or structurally missing) pivot */
#define KKT_ERR_NONFINITE (-5)      /* NaN/Inf in values or factors */
#define KKT_ERR_NOT_CONVERGED (-6)  /* refinement hit max_cycles; x, iters, nrbe still valid */
#define KKT_ERR_TIMEOUT (-7)        /* a bounded device wait ran out */
#define KKT_ERR_CUDA (-8)           /* CUDA runtime error */
#define KKT_ERR_STATE (-9)          /* call out of order (e.g. solve before refactor) */

/* Factor precision.  FP64: factors, triangular solves and refinement in
   FP64.  MIXED: the factors are refactored and the triangular solves (the
   FGMRES preconditioner) run in FP32, while the residual, CGS2, the
   Hessenberg least squares and the solution update stay FP64 -- the
   inexact-factor use of FGMRES the paper's method allows (Section 2.1). */
#define KKT_PRECISION_FP64 0
#define KKT_PRECISION_MIXED 1

#define KKT_STOP_NRBE 0   /* Eq. (nbre) <= tol, checked on the true residual */
#define KKT_STOP_RR 1     /* estimated ||rho_i|| < tol ||rho_0|| (the paper's rule) */

typedef struct kkt_ctx kkt_ctx;

typedef struct {
    int restart;          /* FGMRES restart length m (default 20, 1..32) */
    int max_cycles;       /* restart cycles before KKT_ERR_NOT_CONVERGED (default 50) */
    int stop_mode;        /* KKT_STOP_NRBE (default) or KKT_STOP_RR */
    int precision;        /* KKT_PRECISION_FP64 (default) or KKT_PRECISION_MIXED */
    double refine_delta;  /* Section 2.3: skip refinement if ||r - K x0|| < delta ||r||; 0 = off */
    double pivot_tol;     /* threshold partial pivoting in kkt_analyze (default 1e-3) */
    double boost_eps;     /* static-pivot boost: |u_jj| < boost_eps ||K||_inf becomes
                             sign(u_jj) boost_eps ||K||_inf (sign(0)=+1); 0 = off (default),
                             then an exact zero pivot is KKT_ERR_ZERO_PIVOT */
    int device;           /* CUDA device ordinal (default 0) */
    int create_stream;    /* 1 (default): the context creates its own non-blocking stream;
                             0: use `stream` as given (NULL = the legacy default stream) */
    void* stream;         /* cudaStream_t to use when create_stream == 0 */
    int64_t spin_limit;   /* polls before a device wait gives up (KKT_ERR_TIMEOUT); 0 = default */
    int timing;           /* 1 = record CUDA events around each kernel group (kkt_get_phase_times) */
    int trisolve;         /* triangular-solve schedule: KKT_TRSV_AUTO (default), KKT_TRSV_GLOBAL */
    int cluster_blocks;   /* blocks of the cluster solve: 0 = 16 if it fits and can be
                             scheduled, else 8; 8 or 16 to force one */
    int block_smem;       /* shared memory (bytes) of each block of the refactorization
                             kernel: 0 (default) = the most of the bracket (74 KB: three
                             blocks an SM; 112 KB: two; the device's limit: one) that
                             holds the row needing the most (its working set and
                             position table); rows whose working set fits a warp's
                             slice of it go one per warp, longer rows that fit it one
                             per block (or per half block, kkt_opts.team_rows), the
                             rest one per block with their values in global memory.
                             Blocks of more than 112 KB run 512 threads, else 256. */
    int method;           /* refinement after x0 = (LU)^{-1} b: KKT_METHOD_FGMRES (default),
                             KKT_METHOD_RICHARDSON, KKT_METHOD_FGMRES_EE */
    int ortho;            /* Arnoldi orthogonalisation: KKT_ORTHO_CGS2 (default),
                             KKT_ORTHO_CGS2_PYTH, KKT_ORTHO_CGS1_PYTH */
    double inner_tol;     /* KKT_METHOD_FGMRES_EE: a cycle ends when its estimated residual
                             is <= inner_tol times the residual at the cycle start
                             (default 1e-6) */
    int repivot;          /* 1: when kkt_refactor meets a zero pivot, or kkt_solve does not
                             converge, re-run the pivoting factorization on the current
                             values (Q kept; kkt_repivot) and retry once; 0 = off (default) */
    int graphs;           /* 1: kkt_refactor and kkt_solve replay CUDA graphs -- the
                             refactorization's launches, and the whole refinement with
                             device-side loop control (conditional WHILE/IF nodes: no host
                             round trip per step); captured on first use, again when tol
                             changes.  Same kernels in the same order, so the same results.
                             0 = launch from the host (default) */
    int warp_rows;        /* 1 (default): rows whose working set (values, columns, step
                             descriptors) fits a warp's slice of the block's shared
                             memory are refactored one per warp; 0: every row one per
                             block.  Same arithmetic either way. */
    int row_order;        /* dispatch order of the refactorization's rows: 1 (default)
                             by level in the dependency DAG of L (ties by row); 0 by
                             row; 2 by critical-path priority (descending longest path
                             of estimated row costs to the end of the DAG).  A row's
                             dependencies are always dispatched before it.  Same
                             arithmetic either way. */
    int64_t warp_row_updates; /* a row is refactored one per warp only if its multiply-adds
                             (the sum of |U(k,>k)| over its L entries) are at most this
                             (besides fitting a warp's slice); -1 = no limit; 0 = the
                             default: 2048 with 256-thread blocks, 4096 with 512-thread
                             blocks (the long rows at the dense end, on the critical
                             path, then go one per block or half block) */
    int mixed_fallback;   /* KKT_PRECISION_MIXED only: restart cycles the FP32-factor
                             preconditioner gets (default 2).  A solve not converged by
                             then refactors the matrix in FP64 and continues FGMRES from
                             its current x with the FP64 factors (up to max_cycles more
                             cycles); an FP32 refactorization or solve that meets a zero
                             pivot or a non-finite value falls back the same way (the
                             solve restarting from x0).  The FP64 factors are then used
                             until the next refactorization; kkt_info.last_fallback and
                             fallbacks count it.  The context holds FP64 factor storage
                             beside the FP32 one.  0 = no fallback (FP32 throughout). */
    int stream_last;      /* 1 (default): a row refactored by a whole block stores each value
                             of its last elimination step as soon as that value is final
                             (the pivot by the thread that updates it), so rows that wait
                             on it start while it finishes; 0: all values after the last
                             step's barrier.  Same values and bits either way. */
    int team_rows;        /* 1 (default): with 512-thread blocks, rows that fit half the
                             block's shared memory are refactored one per half block
                             (two such rows at a time, 256 threads each); 0: one per
                             block.  Same arithmetic either way. */
    int equilibrate;      /* KKT_PRECISION_MIXED only: 1 = the FP32 factors are of R K C,
                             R and C diagonal powers of two (r_i = 2^(1-E) with max_j
                             |a_ij| = f 2^E, f in [0.5,1); c_j the same for the columns
                             of R K), computed on the device from each matrix, so every
                             scaled value is exact; the preconditioner applies
                             C (R K C)^{-1} R and kkt_get_factors returns the factors of
                             R K C.  The FP64 fallback factors K unscaled.  0 (default)
                             = no scaling. */
} kkt_opts;

/* Refinement methods (Section 2.1).  FGMRES: FGMRES(m) with M = LU as right
   preconditioner from x0, restarted until the stopping rule holds (the
   paper's method).  RICHARDSON: classical iterative refinement on the error
   system, x += (LU)^{-1}(b - K x), at most max_cycles * restart corrections
   (an iteration is one correction).  FGMRES_EE: FGMRES on the error
   equation -- each cycle solves K d = rho to the relative tolerance
   inner_tol, then x += d and the true residual decides (an outer
   refinement step per cycle). */
#define KKT_METHOD_FGMRES 0
#define KKT_METHOD_RICHARDSON 1
#define KKT_METHOD_FGMRES_EE 2

/* Gram-Schmidt in the Arnoldi step.  CGS2: two classical projections and a
   norm -- three reductions.  CGS2_PYTH: the norm is reduced together with
   the second projection's dot products and taken by Pythagoras,
   sqrt((a - c)(a + c)) with a = ||w'||, c = ||h2|| -- two reductions.
   CGS1_PYTH: one projection, its dot products and ||w|| in one reduction,
   the norm by Pythagoras -- one reduction (the low-synchronisation end of
   the family; loses orthogonality with the basis' conditioning). */
#define KKT_ORTHO_CGS2 0
#define KKT_ORTHO_CGS2_PYTH 1
#define KKT_ORTHO_CGS1_PYTH 2

/* KKT_TRSV_AUTO: one thread-block cluster per triangle when the n solved
   values fit in its shared memory, else KKT_TRSV_GLOBAL: sync-free over the
   whole GPU with the narrow end of each DAG in one block. */
#define KKT_TRSV_AUTO 0
#define KKT_TRSV_GLOBAL 1

/* Kernel groups timed when kkt_opts.timing is set. */
#define KKT_PHASE_GATHER 0    /* value gather + ||K||_inf */
#define KKT_PHASE_REFACTOR 1  /* numeric refactorization */
#define KKT_PHASE_LSOLVE 2    /* L^{-1} P (one launch per preconditioner apply) */
#define KKT_PHASE_USOLVE 3    /* Q U^{-1} */
#define KKT_PHASE_SPMV 4      /* products with K and residuals */
#define KKT_PHASE_ORTHO 5     /* CGS2 passes, normalisation, Givens */
#define KKT_PHASE_UPDATE 6    /* cycle start and end (v_0, y = R^{-1} g, x += Z y) */
#define KKT_PHASE_RESERVED 7  /* unused (the refactorization is one kernel: KKT_PHASE_REFACTOR) */
#define KKT_PHASE_GRAPH_REFACTOR 8 /* a whole refactorization replayed as a graph (kkt_opts.graphs) */
#define KKT_PHASE_GRAPH_SOLVE 9    /* a whole solve replayed as a graph (kkt_opts.graphs) */
#define KKT_NUM_PHASES 10

typedef struct {
    int32_t n;
    int64_t nnz_a;         /* stored entries of K */
    int64_t nnz_l;         /* strictly lower entries of L */
    int64_t nnz_u;         /* entries of U including the diagonal */
    int32_t levels_l;      /* depth of the L-solve dependency DAG */
    int32_t levels_u;      /* depth of the U-solve dependency DAG */
    double refactor_updates; /* multiply-adds of one refactorization */
    int64_t device_bytes;  /* device memory held by the context */
    int32_t nboost;        /* pivots boosted by the last kkt_refactor */
    int32_t last_iters;    /* FGMRES iterations of the last kkt_solve */
    int32_t last_cycles;   /* restart cycles of the last kkt_solve */
    int32_t trisolve_cluster; /* blocks of the cluster solve in use (0: global schedule) */
    double last_nrbe;      /* NRBE of the last kkt_solve's x */
    double last_rnorm0;    /* ||r - K x0|| of the last kkt_solve */
    double norm_a_inf;     /* ||K||_inf of the last refactored matrix */
    double analyze_ms;     /* host time of kkt_analyze */
    int64_t launches;      /* kernels this context has launched so far */
    int64_t h2d_bytes;     /* host->device bytes copied by refactor/solve calls so far */
    int64_t d2h_bytes;     /* device->host bytes copied by refactor/solve calls so far */
    int32_t repivots;      /* pivoting refactorizations run by kkt_repivot so far */
    int32_t rows_warp;     /* rows refactored one per warp in shared memory */
    int32_t rows_block;    /* rows refactored one per block in shared memory (whole block) */
    int32_t rows_global;   /* rows refactored one per block with values in global memory */
    int32_t refactor_smem; /* shared memory per block of the refactorization kernel (bytes) */
    int32_t refactor_threads; /* threads per block of the refactorization kernel */
    int32_t refactor_blocks;  /* blocks of the refactorization kernel */
    int32_t last_fallback; /* 1 if the last refactorization or solve fell back to FP64
                              (kkt_opts.mixed_fallback) */
    int64_t fallbacks;     /* FP64 fallbacks so far */
    int32_t rows_team;     /* rows refactored one per half block (512-thread blocks) */
} kkt_info;

/* Fill *o with the defaults above. */
void kkt_default_opts(kkt_opts* o);

/* Create a context on o->device (o may be NULL for defaults). */
int kkt_create(kkt_ctx** out, const kkt_opts* o);

/*
 * One-time analysis of the pattern (Section 1.3 steps 1-2 for the first
 * system; Section 3.1.1: the first factorization runs on the CPU).
 *   n, rowptr[n+1], colind[nnz]: host CSR pattern of K.
 *   values0[nnz] (host): the matrix whose numeric factorization picks the
 *     pivots; may be NULL only when P is given.
 *   Q[n] (host, optional): column order; NULL = computed on the host
 *     (approximate minimum degree on the pattern of K^T K).
 *   P[n] (host, optional): pivot sequence; NULL = threshold partial pivoting
 *     on values0 with opts.pivot_tol.
 * Allocates every device buffer the context will use.  Can be called again
 * on the same context for a new pattern (buffers are re-made).
 */
int kkt_analyze(kkt_ctx* c, int32_t n, const int32_t* rowptr, const int32_t* colind,
                const double* values0, const int32_t* Q, const int32_t* P);

/*
 * Numeric refactorization on the fixed pattern, P and Q (Section 1.3
 * definition of refactorization; Section 2.1).  values[nnz] in the caller's
 * order of kkt_analyze; host memory if values_on_device == 0, else a device
 * pointer on the context's device.  Also computes ||K||_inf for the NRBE.
 * Errors: KKT_ERR_ZERO_PIVOT, KKT_ERR_NONFINITE, KKT_ERR_TIMEOUT.
 */
int kkt_refactor(kkt_ctx* c, const double* values, int values_on_device);

/*
 * Re-pivot (the paper refactors with pivoting only for the first one or two
 * matrices of a sequence, Section 3.1.1; this restarts that choice later):
 * the threshold-pivoting factorization of kkt_analyze runs again on the
 * host with `values` (caller's entry order, the analysed pattern; host, or
 * device when values_on_device != 0), keeping the column order Q; the new
 * P, factor structure, schedules and device buffers replace the old ones
 * (device memory is re-allocated), and the factors are computed on the GPU
 * as kkt_refactor(values) would.  Returns the kkt_refactor code, or a
 * kkt_analyze error.  kkt_opts.repivot = 1 calls it automatically once
 * when kkt_refactor meets a zero pivot or kkt_solve does not converge.
 */
int kkt_repivot(kkt_ctx* c, const double* values, int values_on_device);

/*
 * Solve K x = b with the current factors (Sections 2.1-2.3):
 * x0 = Q U^{-1} L^{-1} P b; if refinement is needed, FGMRES(m) with M = LU
 * as right preconditioner until the stopping rule holds.
 *   b[n], x[n]: host arrays if on_device == 0, else device pointers.
 *   tol: NRBE tolerance (KKT_STOP_NRBE) or RR tolerance (KKT_STOP_RR).
 *   iters (out, may be NULL): Arnoldi steps taken (preconditioner applies
 *     after x0); nrbe (out, may be NULL): Eq. (nbre) of the returned x.
 * On KKT_ERR_NOT_CONVERGED x, iters and nrbe are still written.
 */
int kkt_solve(kkt_ctx* c, const double* b, double* x, int on_device, double tol,
              int* iters, double* nrbe);

/*
 * One step of a sequence: kkt_refactor(values) then kkt_solve(b, tol), with
 * the forward sweep y = L^{-1} P b fused into the refactorization: the warp
 * or block that finishes a row of the factors computes that row of y at once,
 * with the row arithmetic of the separate sweep (same bits), so the separate
 * forward sweep of the initial solve disappears from the step.  values, b
 * and x are all host arrays (on_device == 0) or all device arrays.  Returns
 * and outputs as kkt_refactor then kkt_solve (including kkt_opts.repivot).
 * With kkt_opts.graphs the two graphs are replayed unfused.  (A fused
 * refactorization-solve pair is an implementation choice the paper's
 * separate steps of Section 1.3 allow.)
 */
int kkt_step(kkt_ctx* c, const double* values, const double* b, double* x, int on_device, double tol,
             int* iters, double* nrbe);

/* x = Q U^{-1} L^{-1} P b only (Section 1.3 step 3), no refinement. */
int kkt_lu_solve(kkt_ctx* c, const double* b, double* x, int on_device);

/* y = K x with the values of the last kkt_refactor. */
int kkt_matvec(kkt_ctx* c, const double* x, double* y, int on_device);

/* Copy the permutations (host arrays of n). */
int kkt_get_perm(kkt_ctx* c, int32_t* P, int32_t* Q);

/* Sizes of the factors: nnz of strict L and of U (with diagonal). */
int kkt_get_factor_sizes(kkt_ctx* c, int64_t* nnz_l, int64_t* nnz_u);

/*
 * Host copies of the current factors (FP32 factors are widened exactly to
 * double) in CSC, permuted space, rows sorted:
 * L strictly lower (Lp[n+1], Li/Lx[nnz_l]), U with diagonal (Up[n+1],
 * Ui/Ux[nnz_u]).  For tests and inspection.
 */
int kkt_get_factors(kkt_ctx* c, int64_t* Lp, int32_t* Li, double* Lx,
                    int64_t* Up, int32_t* Ui, double* Ux);

int kkt_query(kkt_ctx* c, kkt_info* info);

/*
 * Accumulated device time (ms) and launch count of each kernel group since
 * the last reset (arrays of KKT_NUM_PHASES; either may be NULL).  Needs
 * kkt_opts.timing = 1; times come from CUDA events on the context's stream.
 * reset != 0 clears the accumulators after reading.
 */
int kkt_get_phase_times(kkt_ctx* c, double* ms, int64_t* counts, int reset);

/*
 * Profiling: kkt_refactor, with the GPU's global timer (ns) recorded when
 * each row starts and when it publishes its pivot.  t_start[n],
 * t_publish[n] (host) get the stamps; *t0_out = 0 (the first traced row).
 * Makes one temporary device allocation for the stamps.
 */
int kkt_trace_refactor(kkt_ctx* c, const double* values, int values_on_device, int64_t* t_start,
                       int64_t* t_publish, int32_t* t0_out);

/*
 * Autotuner: times kkt_refactor(values) + kkt_lu_solve(b) (median of `reps`
 * runs after one warm-up) for each schedule of the refactorization and the
 * solves -- the refactorization kernel's shared memory per block (sized by
 * the longest row, 72 KB, 110 KB or the device's limit), with and without
 * warp rows, times the solve schedule (cluster of 16 or 8 blocks, or
 * whole-GPU) -- and keeps the fastest in the context (kkt_query:
 * refactor_smem, rows_warp, trisolve_cluster).  Every schedule computes the
 * same bits, so tuning changes only speed.  values, b as in kkt_refactor and
 * kkt_lu_solve; with on_device != 0 one n-vector of device memory is added
 * to the context.  *best_ms (may be NULL) gets the chosen time.  The factors
 * must be recomputed afterwards (kkt_refactor).
 */
int kkt_tune(kkt_ctx* c, const double* values, const double* b, int on_device, int reps, double* best_ms);

/*
 * Profiling: kkt_lu_solve (Section 1.3, the direct solve with the current
 * factors) with the GPU's global timer (ns) recorded when each row of the
 * two sweeps publishes its value.  Only for the cluster schedule (else
 * KKT_ERR_STATE).  listL[n], listU[n] (host) get the rows in the order the
 * sweeps take them; tL[t], tU[t] (host) the publish time of list position t.
 * b and x as in kkt_lu_solve.  Makes one temporary device allocation.
 */
int kkt_trace_solve(kkt_ctx* c, const double* b, double* x, int on_device, int32_t* listL,
                    int32_t* listU, int64_t* tL, int64_t* tU);
void kkt_destroy(kkt_ctx* c);
const char* kkt_strerror(int code);
const char* kkt_last_error_detail(kkt_ctx* c);

/*
 * Self-test of the bounded waits (no counterpart in the paper): launches,
 * on the context's stream, one warp that waits with the library's wait
 * primitive for a completion flag that nothing ever sets, with `limit`
 * polls.  Returns KKT_ERR_TIMEOUT (the wait gave up and reported it, the
 * GPU and the context stay usable) or KKT_OK if it did not time out.
 */
int kkt_selftest_wait(kkt_ctx* c, int64_t limit);

/* ---- triangular solve without any device allocation ---- */

/*
 * The paper has no counterpart to this entry point; it exists for callers
 * that cannot allocate device memory -- an application whose device memory
 * belongs to its own arena allocator, or a latency-critical loop in which a
 * cudaMalloc/cudaFree could synchronise the device.
 *
 * x = Q U^{-1} L^{-1} P b, the same result as kkt_lu_solve, computed from
 * factors the caller already holds on the current device, in the combined
 * row layout the solver uses internally: F = L + U - I of B = K(P,Q), CSR
 * over the permuted rows with columns ascending in each row; row i holds
 * L(i,k<i) (unit diagonal not stored), then U(i,i) at Fdiag[i], then
 * U(i,j>i).
 *   n        rows, 1 <= n <= KKT_NOALLOC_MAX_N; larger n returns
 *            KKT_ERR_INVALID without launching anything.
 *   Fp[n+1], Fdiag[n] (int64), Fj[nnz] (int32), Fx[nnz] (double),
 *   P[n], Q[n] (int32), b[n] (double): device pointers, read only.
 *   x[n]     device pointer, written.
 *   stream   cudaStream_t (NULL = the legacy default stream); the call
 *            returns after the solve has finished on it.
 * Working memory is one static device array of KKT_NOALLOC_SCRATCH_BYTES in
 * the library image -- 256 bytes of tickets and error words, then the two
 * intermediate vectors (y = L^{-1} P b and U^{-1} y, 8 bytes per row each) --
 * held by every GPU that loads the library until the process exits; the
 * call makes no cudaMalloc or cudaFree.  The first call on a device looks up
 * that array's device address (cudaGetSymbolAddress) with the device current
 * and caches it.  Every call reads its error status back and synchronises
 * the stream before it returns, so it cannot be captured into a CUDA
 * graph.  All calls on a device share the array, so
 * calls that overlap on the GPU (other streams, other threads) race and give
 * wrong results: serialise them.  Each call re-arms the parts of the array
 * it uses (the vectors' first n entries, the tickets, the error words).
 * Result: the same bits as kkt_lu_solve on the same factors (the same row
 * arithmetic and summation order).
 * Errors: KKT_ERR_INVALID, KKT_ERR_TIMEOUT (a bounded wait ran out),
 * KKT_ERR_CUDA.
 */
#define KKT_NOALLOC_MAX_N 65536
#define KKT_NOALLOC_SCRATCH_BYTES (256 + (KKT_NOALLOC_MAX_N) * 16)
int kkt_lu_solve_noalloc(int32_t n, const int64_t* Fp, const int32_t* Fj, const int64_t* Fdiag,
                         const double* Fx, const int32_t* P, const int32_t* Q, const double* b,
                         double* x, void* stream);

/* ---- one step of many instances in shared launches ----
 *
 * The paper solves one KKT sequence at a time; one small or mid-size
 * instance leaves most of a B300 idle, because its refactorization and
 * triangular solves are chains of dependent rows (Section 1.3 notes that
 * tiny kernels underuse the GPU).  A batch runs one step -- kkt_step:
 * gather, refactorization with the forward sweep fused, backward sweep,
 * residual and refine-or-not decision -- of several instances together:
 * ONE refactorization launch whose work items are taken from every
 * instance's level-ordered queue in turn (ticket t -> instance t mod count,
 * its item t / count, so each instance's rows keep their dispatch order),
 * one launch of backward sweeps with one thread-block cluster per instance,
 * and one launch each for the gathers, the residuals and the decisions.
 * Instances whose x0 needs refinement then continue with FGMRES on their
 * own stream.  Every instance gets the bits it would get from kkt_step
 * alone (the same row arithmetic; the reductions keep each instance's own
 * block count).
 */
typedef struct kkt_batch kkt_batch;

/* Workspace for up to max_count instances per step on `device` (device
 * memory and pinned host memory for the launch arguments, a stream). */
int kkt_batch_create(kkt_batch** out, int max_count, int device);
void kkt_batch_destroy(kkt_batch* bt);

/*
 * One step of each of ctxs[0..count) (distinct, analysed contexts):
 * values[i], b[i], x[i] as in kkt_step (all host arrays when on_device == 0,
 * else all device pointers), one tolerance.  iters, nrbe (may be NULL) and
 * status (required) are arrays of count: status[i] is kkt_step's return
 * code for instance i.  FP64 contexts on the batch's device with the same
 * refactorization block size (kkt_info.refactor_threads) as the first of
 * them share the launches; the others run as lone kkt_step calls.  Work the
 * caller queued on a context's stream before the call is waited for; the
 * call returns when every step is done.  Returns KKT_ERR_INVALID for bad
 * arguments (a repeated context, count > max_count), else KKT_OK with the
 * per-instance codes in status.  One call at a time per batch.
 */
int kkt_batch_step(kkt_batch* bt, kkt_ctx* const* ctxs, int count, const double* const* values,
                   const double* const* b, double* const* x, int on_device, double tol, int* iters, double* nrbe,
                   int* status);

/* Kernels the batch has launched so far. */
int64_t kkt_batch_launches(const kkt_batch* bt);

/* Time spent by kkt_batch_step's shared part since creation or the last
 * reset, in ms, per phase (CUDA events on the batch's stream, except the
 * last): [0] argument and value copies, [1] the batched gather, [2] the
 * batched refactorization with the fused forward sweeps, [3] the backward
 * sweeps, [4] the batched residual and decision, [5] host wall time of the
 * per-instance rest (outcomes, the refinement where needed, copies of x).
 * steps (may be NULL): instance-steps run in shared launches.  reset != 0
 * zeroes the sums.  Errors: KKT_ERR_INVALID (NULL bt or ms). */
#define KKT_BATCH_PHASES 6
int kkt_batch_phase_times(kkt_batch* bt, double* ms, int64_t* steps, int reset);

/* ---- serving: many resident instances, steps in flight concurrently ----
 *
 * The paper solves one KKT sequence at a time and reuses the analysis,
 * factor storage and Krylov space across the sequence (Sections 2.1, 3.1.1).
 * A server holds many such sequences ("instances") resident on one or more
 * GPUs and keeps their refactor + solve steps in flight together: each
 * instance is a context (kkt_create) with its own stream, placed whole on
 * one device.  Steps of one instance run one at a time in submission order.
 *   - batch > 0 (continuous batching): one dispatcher per device takes up to
 *     `batch` instances with a queued step and runs those steps together
 *     (kkt_batch_step: one refactorization launch over all of them); steps
 *     submitted meanwhile join the next batch.
 *   - batch == 0: a pool of worker threads runs each step as its own
 *     kkt_step, instances concurrently on their streams.
 * Admission (kkt_server_open): the host analysis runs in the caller's
 * thread; the instance is then placed on the device with the most budget
 * left (kkt_place_instance) and waits, in arrival order, until its device
 * memory fits that device's budget.  Results do not depend on the mix: each
 * step computes the bits it would compute alone.
 */
typedef struct kkt_server kkt_server;

#define KKT_SERVER_MAX_DEVICES 16

typedef struct {
    int workers;          /* host threads of the batch == 0 mode (default 8, 1..256) */
    int64_t hbm_budget;   /* device bytes the admitted instances may hold on each device;
                             0 = 90% of the device memory free at kkt_server_create */
    kkt_opts opts;        /* options of every instance's context (device, create_stream
                             and stream are ignored: each instance makes its own stream
                             on the device it is placed on) */
    int batch;            /* instances per batched step (continuous batching); 0 = off
                             (default 8) */
    int ndevices;         /* devices to place instances on: devices[0..ndevices);
                             0 = opts.device only (default) */
    int devices[KKT_SERVER_MAX_DEVICES];
} kkt_server_opts;

typedef struct {
    int status;           /* KKT_OK or the failing call's error (refactor or solve) */
    int32_t iters;        /* refinement iterations */
    double nrbe;          /* Eq. (nbre) of x */
    double queue_ms;      /* submit -> the step starts */
    double run_ms;        /* refactor + solve (the whole batched call in batch mode), host wall time */
    int32_t batch_size;   /* steps in the batched call that ran it (1 without batching) */
    int32_t device;       /* device of the instance */
} kkt_step_result;

typedef struct {
    int32_t instances;      /* admitted and open */
    int64_t device_bytes;   /* held by the admitted instances (all devices) */
    int64_t hbm_budget;     /* summed over the devices */
    int64_t submitted, completed;
    int32_t in_flight;      /* steps running now */
    int32_t waiting;        /* opens waiting for admission */
    int64_t batches;        /* batched calls run so far */
    int32_t ndevices;
} kkt_server_info;

/* Fill *o with the defaults above (kkt_default_opts for o->opts). */
void kkt_server_default_opts(kkt_server_opts* o);

int kkt_server_create(kkt_server** out, const kkt_server_opts* o);

/*
 * Admit a new instance: the host analysis of its pattern (values0 fixes the
 * pivots, as in kkt_analyze) in the calling thread, placement, then -- once
 * its device memory (kkt_estimate_device_bytes) fits the chosen device's
 * budget, waiting behind earlier opens on that device -- its context and
 * device buffers.  *instance gets its id.  Errors: KKT_ERR_OOM when the
 * instance can never fit (it needs more than a whole device's budget), or
 * kkt_create / kkt_analyze errors.  The arrays are host memory and are not
 * kept.  Blocks while waiting for admission.
 */
int kkt_server_open(kkt_server* s, int32_t n, const int32_t* rowptr, const int32_t* colind,
                    const double* values0, int64_t* instance);

/*
 * Queue one step of an instance: kkt_step(values, b, tol) -- kkt_refactor
 * then kkt_solve, the forward sweep fused -- writing x (host, n doubles; written when the step
 * completes -- keep it valid until kkt_server_wait returns).  values and b
 * are copied at submit.  *ticket identifies the step for kkt_server_wait.
 */
int kkt_server_submit(kkt_server* s, int64_t instance, const double* values, const double* b,
                      double* x, double tol, int64_t* ticket);

/* Block until the step is done; its result in *r.  Each ticket is waited once. */
int kkt_server_wait(kkt_server* s, int64_t ticket, kkt_step_result* r);

/* Wait for the instance's queued steps, then free its context and memory
   (opens waiting for admission may then proceed). */
int kkt_server_close(kkt_server* s, int64_t instance);

int kkt_server_query(kkt_server* s, kkt_server_info* info);

/* Wait for every queued step, close every instance, stop the workers. */
void kkt_server_destroy(kkt_server* s);

/*
 * Profiling: the critical path of the last traced refactorization
 * (kkt_trace_refactor's stamps, passed back in).  Rows in index order are a
 * topological order of the dependency DAG of L (row i waits for every row k
 * with L(i,k) != 0); a row's link is t_publish[i] - max(t_start[i], the
 * latest t_publish of its dependencies), the time from when it could take
 * its last step to its publication.  *path_ns gets the longest path of
 * links through the DAG (rows without stamps count 0), *levels the depth of
 * the DAG, *median_link_ns the median link of the stamped rows, *rows the
 * rows with stamps.  Host only (no device work).
 */
int kkt_trace_critical_path(kkt_ctx* c, const int64_t* t_start, const int64_t* t_publish, double* path_ns,
                            int32_t* levels, double* median_link_ns, int32_t* rows);

/*
 * A second context on the same pattern: copies src's analysis (canonical
 * pattern, P, Q, factor structure, schedules) into c, which must have been
 * created (kkt_create) with its own options (for example another
 * precision), and makes c's device buffers.  Costs no host factorization.
 * Errors: KKT_ERR_STATE (src not analysed), kkt_analyze's device errors.
 */
int kkt_analyze_like(kkt_ctx* c, const kkt_ctx* src);

/* ---- host-only helpers (no GPU needed) ---- */

/* Statistics of a host analysis (kkt_host_analyze). */
typedef struct {
    int64_t nnz_l;           /* strictly lower entries of L */
    int64_t nnz_u;           /* entries of U including the diagonal */
    int32_t levels_l;        /* depth of the L-solve dependency DAG */
    int32_t levels_u;        /* depth of the U-solve dependency DAG */
    double refactor_updates; /* multiply-adds of one refactorization */
    double order_ms;         /* host time of the column ordering */
    double pivot_ms;         /* host time of the pivoting factorization */
    int32_t canonical_order; /* 1 if the caller's CSR rows were already sorted */
} kkt_host_stats;

/*
 * The one-time analysis of kkt_analyze without a GPU (Section 3.1.1: the
 * first factorization runs on the CPU): the column order Q (approximate
 * minimum degree on the pattern of K^T K) and the pivot sequence P
 * (threshold partial pivoting with pivot_tol on values0), both written to
 * host arrays of n, and the structure's statistics in *st (may be NULL).
 * kkt_analyze(…, Q, P) on another thread or later reuses them.  Thread safe.
 */
int kkt_host_analyze(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* values0,
                     double pivot_tol, int32_t* P, int32_t* Q, kkt_host_stats* st);

/* Column order of kkt_analyze (approximate minimum degree on K^T K). */
int kkt_order(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t* Q);

/*
 * Device bytes kkt_analyze allocates for a pattern of n rows and nnz_a
 * entries whose host analysis gave *st (kkt_host_analyze), under options
 * *o (NULL = defaults); canonical_order != 0 if the caller's CSR rows are
 * already sorted (no index map is kept).  Exactly kkt_info.device_bytes of
 * the analysed context (the scratch of rows refactored in global memory,
 * which only rows beyond a block's shared memory use, is not counted).
 */
int kkt_estimate_device_bytes(int32_t n, int64_t nnz_a, const kkt_host_stats* st, const kkt_opts* o,
                              int canonical_order, int64_t* bytes);

/*
 * Placement of a new instance (the serving runtime's, no collective: whole
 * instances go to one device): among ndev devices with budget[i] and
 * held[i] bytes (held: admitted plus waiting for admission), the index of
 * the one with the most budget left whose budget can hold `need` at all
 * (ties to the lower index), or -1 if none can.
 */
int kkt_place_instance(int ndev, const int64_t* budget, const int64_t* held, int64_t need);

/*
 * First factorization with threshold partial pivoting on the host, as
 * kkt_analyze does it: returns the pivot sequence P and the factor sizes.
 */
int kkt_pivot(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* values,
              const int32_t* Q, double pivot_tol, int32_t* P, int64_t* nnz_l, int64_t* nnz_u);

#ifdef __cplusplus
}
#endif
#endif /* KKT_B300_H */
