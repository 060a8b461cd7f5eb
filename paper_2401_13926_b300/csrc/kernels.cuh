// Device kernels of the refactor + triangular solve + FGMRES hot path.
//
// Layout in device memory (permuted space, B = K(P,Q) = L U):
//   F  -- combined factor L + U - I, row-major: row i holds its columns in
//         ascending order, L(i,k<i) first, then U(i,i) at Fdiag[i], then
//         U(i,j>i).  Fp (int64, n+1), Fj (int32), Fx (double).
//   A  -- K in canonical CSR (original space) for the residual and the
//         products with K: Arp (int32, n+1), Aci (int32), Ax (double).
//   V  -- Krylov basis, column-major n x (m+1), leading dimension ld;
//   Z  -- preconditioned directions, n x m (flexible GMRES keeps them).
//
// Dependency waits (refactor and both triangular solves) are sync-free:
// each warp takes the next row from an atomic ticket counter in dependency
// order, so every row it waits on belongs to a warp that is already
// running; completion flags hold a generation number so they never need
// clearing.  Every wait is bounded: after `spin_limit` polls, or once any
// warp has raised the abort flag, the warp records KKT_ERR_TIMEOUT and
// returns.
#pragma once
#ifndef SPIN_SLEEP_NS
#define SPIN_SLEEP_NS 20
#endif
#include <cooperative_groups.h>
#include <climits>
#include <cstdint>
#include <cuda_runtime.h>

#include "kkt.h"
#include "trsv_row.cuh"

namespace kkt {

constexpr int MAXM = 32;          // largest restart length
constexpr int RED_SLOTS = MAXM + 2;
constexpr int RED_BLOCKS = 296;   // blocks of the reduction kernels (2 per SM)
constexpr int RED_THREADS = 256;

struct DevScal {
    // matrix and right-hand side
    double normA;          // ||K||_inf of the last refactor
    double normb;          // ||b||_2
    // current iterate
    double rnorm;          // ||b - K x||_2
    double xnorm;          // ||x||_2
    double rnorm0;         // ||b - K x0||_2 (rho^(0))
    double nrbe;
    double thresh;         // inner stopping threshold of the cycle
    double hn;             // h_{j+1,j}
    double g[MAXM + 1], cs[MAXM], sn[MAXM], y[MAXM];
    double H[(MAXM + 1) * MAXM];   // column-major, leading dimension MAXM+1
    double h[MAXM + 1], h2[MAXM + 1];
    int j;                 // current Arnoldi column
    int iters;             // Arnoldi steps of this solve
    int cycles;            // restart cycles of this solve (device-side loop control)
    int not_converged;     // the device-side loop stopped at its cycle or step cap
    // CUDA-graph loop control: the WHILE node's handle and one handle per
    // Arnoldi-step IF node (a handle drives exactly one conditional node)
    unsigned long long h_loop;
    unsigned long long h_step[MAXM];
    int met;               // inner criterion met in this cycle
    int done;              // solve finished (converged or nothing to do)
    // sync-free scheduling
    unsigned gen_fact;
    unsigned ticket_fact, ticket_l, ticket_u;
    unsigned red_count;
    // errors
    int err;               // first error code (0 = none)
    int err_row;
    int abort;
    int nboost;
};

// ---------------------------------------------------------------- helpers
__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
    unsigned v;
    asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_release(unsigned* p, unsigned v) {
    asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}
__device__ __forceinline__ int ld_volatile_int(const int* p) { return *(volatile const int*)p; }
__device__ __forceinline__ unsigned long long globaltimer_ns() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
}

__device__ __forceinline__ void raise_error(DevScal* s, int code, int row) {
    if (atomicCAS(&s->err, 0, code) == 0) s->err_row = row;
    atomicExch(&s->abort, 1);
}

// Wait until flag == gen.  Returns false if the wait was abandoned.
__device__ __forceinline__ bool wait_flag(const unsigned* flag, unsigned gen, DevScal* s, long long limit, int row) {
    if (ld_acquire(flag) == gen) return true;
    for (long long it = 0;; it++) {
        if (ld_acquire(flag) == gen) return true;
        if (ld_volatile_int(&s->abort)) return false;
        if (it >= limit) { raise_error(s, KKT_ERR_TIMEOUT, row); return false; }
        __nanosleep(64);
    }
}

// Block-wide sum (all threads get the result); blockDim.x multiple of 32, <= 1024.
__device__ __forceinline__ double block_sum(double v, double* sh) {
    v = warp_sum(v);
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    __syncthreads();
    if (lane == 0) sh[wid] = v;
    __syncthreads();
    double t = (threadIdx.x < nw) ? sh[threadIdx.x] : 0.0;
    if (wid == 0) t = warp_sum(t);
    if (threadIdx.x == 0) sh[32] = t;
    __syncthreads();
    return sh[32];
}

// The last block to arrive (deterministic fixed-order sum of the partials)
// returns true in every thread of that block.
__device__ __forceinline__ bool last_block(DevScal* s, unsigned nblocks) {
    __shared__ int is_last;
    __threadfence();
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned prev = atomicAdd(&s->red_count, 1u);
        is_last = (prev == nblocks - 1);
    }
    __syncthreads();
    if (is_last) {
        __threadfence();
        if (threadIdx.x == 0) s->red_count = 0;
    }
    return is_last;
}
__device__ __forceinline__ bool last_block(DevScal* s) { return last_block(s, gridDim.x); }

// Sum partials part[b * RED_SLOTS + slot] over blocks b < nblocks, in block order.
__device__ __forceinline__ double reduce_partials(const double* part, int slot, double* sh, int nblocks) {
    double v = 0.0;
    for (int b = threadIdx.x; b < nblocks; b += blockDim.x) v += __ldcg(&part[b * RED_SLOTS + slot]);
    return block_sum(v, sh);
}
__device__ __forceinline__ double reduce_partials(const double* part, int slot, double* sh) {
    return reduce_partials(part, slot, sh, (int)gridDim.x);
}

// Loads and stores that other blocks poll (gpu scope, not cached in L1).
__device__ __forceinline__ double ld_relaxed_f64(const double* p) {
    double v;
    asm volatile("ld.relaxed.gpu.global.f64 %0, [%1];" : "=d"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed_f64(double* p, double v) {
    asm volatile("st.relaxed.gpu.global.f64 [%0], %1;" ::"l"(p), "d"(v) : "memory");
}
__device__ __forceinline__ double ld_relaxed(const double* p) { return ld_relaxed_f64(p); }
__device__ __forceinline__ void st_relaxed(double* p, double v) { st_relaxed_f64(p, v); }
__device__ __forceinline__ float ld_relaxed(const float* p) {
    float v;
    asm volatile("ld.relaxed.gpu.global.f32 %0, [%1];" : "=f"(v) : "l"(p) : "memory");
    return v;
}
__device__ __forceinline__ void st_relaxed(float* p, float v) {
    asm volatile("st.relaxed.gpu.global.f32 [%0], %1;" ::"l"(p), "f"(v) : "memory");
}

// ---------------------------------------------------------------- K0: gather
// Start of a refactorization: new generation, tickets and error words.
__device__ __forceinline__ void refactor_prep(DevScal* s) {
    s->gen_fact += 1;
    s->ticket_fact = 0;
    s->err = 0;
    s->err_row = -1;
    s->abort = 0;
    s->nboost = 0;
    s->normA = 0.0;
}
__global__ void k_refactor_prep(DevScal* s) { refactor_prep(s); }

struct GiveUpGlobal {
    const int* abort;
    __device__ bool operator()() const { return *(volatile const int*)abort != 0; }
};

template <typename T>
struct SrcGlobal {   // operand in a global vector, by column
    static constexpr int kPollNs = 20;
    const int32_t* Fj;
    const T* x;
    __device__ const volatile T* operator()(int64_t p) const { return x + __ldg(&Fj[p]); }
};

__device__ __forceinline__ void fail_row(DevScal* s, int row) {
    if (!*(volatile int*)&s->abort) raise_error(s, KKT_ERR_TIMEOUT, row);
}

// The forward sweep y = L^{-1} P rhs fused into the refactorization: the
// warp (or a warp of the block) that finished row i computes y_i at once
// with the L-sweep's row arithmetic (trsv_row), so y has the same bits as
// a separate sweep, and its chain trails the factorization's by one row.
// rhs == nullptr: not fused.  y is armed with SENTINEL by the gather; xp
// (the U-sweep's vector in the whole-GPU schedule) is armed per row.
template <typename T>
struct FwdArgs {
    const double* rhs;
    const int32_t* P;
    T* y;
    T* xp;
};

template <typename T>
struct SliceVals {   // the row's values as the refactorization left them: entry p at w[p - b]
    const T* w;
    int64_t b;
    __device__ T operator()(int64_t p) const { return w[p - b]; }
};

// One load per lane in flight (same bits as the sweep's batched loads):
// fewer registers in the refactorization kernel that carries it.
template <typename T, class Vals>
__device__ __forceinline__ bool fused_forward_row(int row, int64_t lo, int64_t hi, Vals vals,
                                                  const int32_t* __restrict__ Fj, const FwdArgs<T>& fw, DevScal* s,
                                                  long long limit) {
    const GiveUpGlobal gu{&s->abort};
    T val;
    if (!trsv_row_v<true, T, Vals, SrcGlobal<T>, GiveUpGlobal, 1>(lo, hi, vals, SrcGlobal<T>{Fj, fw.y},
                                                                rhs_value<T>(fw.rhs[fw.P[row]]), T(1), limit, gu, &val)) {
        if ((threadIdx.x & 31) == 0) fail_row(s, row);
        return false;
    }
    if ((threadIdx.x & 31) == 0) {
        fw.xp[row] = sentinel_of<T>();
        st_relaxed(&fw.y[row], val);
    }
    __syncwarp();
    return true;
}

// Every factor value and pivot reciprocal is armed with SENTINEL (the
// refactorization gathers the caller's values itself and publishes each
// value when it is final); Ax[e] = caller value of canonical entry e;
// ||K||_inf from row sums.  T is the factor type: double, or float in
// mixed precision.
template <typename T>
__device__ __forceinline__ void gather_body(const double* __restrict__ vals, int64_t nnzF, T* __restrict__ Fx,
                                            const int32_t* __restrict__ Arp, const int64_t* __restrict__ asrc,
                                            double* __restrict__ Ax, int n, T* __restrict__ rinv, DevScal* s,
                                            T* __restrict__ yarm) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += stride) rinv[i] = sentinel_of<T>();
    if (yarm)   // the fused forward sweep fills y
        for (int64_t i = tid; i < n; i += stride) yarm[i] = sentinel_of<T>();
    for (int64_t t = tid; t < nnzF; t += stride) Fx[t] = sentinel_of<T>();
    const int lane = threadIdx.x & 31;
    const int64_t warp = tid >> 5, nwarps = stride >> 5;
    bool bad = false;
    for (int64_t i = warp; i < n; i += nwarps) {
        for (int64_t e = Arp[i] + lane; e < Arp[i + 1]; e += 32) {
            double v = vals[asrc ? asrc[e] : e];
            Ax[e] = v;
            if (!isfinite(v)) bad = true;
        }
    }
    if (bad) raise_error(s, KKT_ERR_NONFINITE, -1);
    // each row's sum of |a_ij| in column order, as the definition reads (so
    // the boost threshold boost_eps * ||K||_inf is reproducible): one thread
    // per row
    double rmax = 0.0;
    for (int64_t i = tid; i < n; i += stride) {
        double acc = 0.0;
        for (int64_t e = Arp[i]; e < Arp[i + 1]; e++) acc += fabs(vals[asrc ? asrc[e] : e]);
        rmax = fmax(rmax, acc);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    if (lane == 0 && rmax > 0.0)   // non-negative doubles order like their bit patterns
        atomicMax((unsigned long long*)&s->normA, (unsigned long long)__double_as_longlong(rmax));
}

template <typename T>
__global__ void k_gather(const double* __restrict__ vals, int64_t nnzF, T* __restrict__ Fx,
                         const int32_t* __restrict__ Arp, const int64_t* __restrict__ asrc,
                         double* __restrict__ Ax, int n, T* __restrict__ rinv, DevScal* s, T* __restrict__ yarm) {
    gather_body<T>(vals, nnzF, Fx, Arp, asrc, Ax, n, rinv, s, yarm);
}

// ---- the same first phases for a batch of instances (blockIdx.y = instance)
struct GatherArgs {
    const double* vals;
    int64_t nnzF;
    double* Fx;
    const int32_t* Arp;
    const int64_t* asrc;
    double* Ax;
    int n;
    double* rinv;
    DevScal* s;
    double* yarm;
};

// every instance's refactor_prep, and the batch ticket cleared
__global__ void k_refactor_prep_batch(const GatherArgs* ga, int count, unsigned long long* ticket) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i < count) refactor_prep(ga[i].s);
    if (i == 0) *ticket = 0ull;
}

__global__ void k_gather_batch(const GatherArgs* ga) {
    const GatherArgs& g = ga[blockIdx.y];
    gather_body<double>(g.vals, g.nnzF, g.Fx, g.Arp, g.asrc, g.Ax, g.n, g.rinv, g.s, g.yarm);
}

// The caller's values rebuilt from the canonical copy (vals[asrc[e]] =
// Ax[e]; asrc == nullptr: the same order), for a refactorization that
// starts from the matrix already in use.
__global__ void k_scatter_values(int64_t nnz, const double* __restrict__ Ax, const int64_t* __restrict__ asrc,
                                 double* __restrict__ vals) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t e = tid; e < nnz; e += stride) vals[asrc ? asrc[e] : e] = Ax[e];
}

// ---------------------------------------------------------------- K1: refactor
// Up-looking (row-by-row Doolittle) numeric LU on the fixed pattern: for row
// i, in ascending k over L(i,:), l_ik = w_k * (1/u_kk) and w -= l_ik U(k,:),
// every update one fused multiply-add.  ONE persistent kernel factors every
// row; each row is placed by the room its working set needs -- its values,
// columns and the descriptors of its elimination steps:
//   ROW_WARP   one warp, in that warp's slice of the block's shared memory;
//   ROW_BLOCK  the whole block, in the block's shared memory (the long
//              rows at the dense end of the order), with a table of its
//              columns' positions;
//   ROW_TEAM   one team of the block's threads (RefShape::TEAMS > 1), in
//              that team's share of the shared memory, with a table;
//   ROW_GLOBAL the whole block, its values in a global scratch area (rows
//              that fit no block).
// Work items (up to one warp row per warp, one team row per team, or one
// block row) are taken from
// an atomic ticket in the order of their rows' level in the dependency DAG
// of L, so a row's dependencies are always dispatched before it and every
// row a block waits on belongs to a block that is already running.  A
// finished row publishes its U values and 1/u_ii with no fences: every
// published datum is armed with SENTINEL by the gather and is final once it
// is not, so a consumer spins on exactly the values it uses.
constexpr int ROW_WARP = 0, ROW_BLOCK = 1, ROW_GLOBAL = 2, ROW_TEAM = 3;

struct RefItem {       // rows order[first .. first + count) of one kind
    int32_t first;
    int32_t info;      // kind << 28 | count (ROW_WARP, ROW_TEAM) or global-row index (ROW_GLOBAL)
};

template <typename T>
struct RefArgs {
    const RefItem* items;
    int nitems;
    const int32_t* order;
    const int64_t* Fp;
    const int32_t* Fj;
    const int64_t* Fdiag;
    T* Fx;
    T* rinv;
    const double* vals;
    const int64_t* fsrc;
    int area_bytes;        // a block row's room in shared memory (working set and position table)
    int slice_bytes;       // a warp row's slice: warp w's starts at w * slice_bytes
    // ROW_GLOBAL rows, by global-row index g: step descriptors at sd_off[g]
    // in gdk / gcnt, values at w_off[g] in gw
    const uint32_t* gdk;
    const uint32_t* gcnt;
    const int64_t* g_sd_off;
    T* gw;
    const int64_t* g_w_off;
    DevScal* s;            // the instance's scalars (tickets of a lone launch, errors, ||K||_inf)
    FwdArgs<T> fw;         // the fused forward sweep (fw.rhs == nullptr: not fused)
    double boost_eps;
    int stream_last;       // block rows publish their last step's values as they are formed
};

// Several instances' refactorizations in one launch: global ticket t goes
// to instance t mod count, its work item t / count (tickets past an
// instance's items, or of an instance that has failed, are skipped), so
// every instance's items are dispatched in their own order and a row's
// dependencies are still dispatched before it.
template <typename T>
struct RefBatch {
    const RefArgs<T>* args;   // device array of `count`
    int count;
    long long total;          // count * the most items of any instance
    unsigned long long* ticket;   // zeroed before the launch
};

__device__ __forceinline__ bool finite_bits(double v) {
    return (__double_as_longlong(v) & 0x7ff0000000000000ll) != 0x7ff0000000000000ll;
}
__device__ __forceinline__ bool finite_bits(float v) { return (__float_as_uint(v) & 0x7f800000u) != 0x7f800000u; }
__device__ __forceinline__ bool zero_bits(double v) { return (__double_as_longlong(v) << 1) == 0; }
__device__ __forceinline__ bool zero_bits(float v) { return (__float_as_uint(v) << 1) == 0u; }
__device__ __forceinline__ bool sign_bit(double v) { return __double_as_longlong(v) < 0; }
__device__ __forceinline__ bool sign_bit(float v) { return (int)__float_as_uint(v) < 0; }

// Publish a row's pivot u_ii and its reciprocal.  The reciprocal is on the
// dependency chain, so it is formed first; the checks (non-finite, zero,
// below the boost threshold) read the bits or run beside it.
template <typename T>
__device__ __forceinline__ bool publish_pivot(T u, T boost, bool use_boost, DevScal* s, int row, T* Fx_d,
                                              T* rinv_row) {
    T ri = rcp_rn(u);
    if (!finite_bits(u)) { raise_error(s, KKT_ERR_NONFINITE, row); return false; }
    if (use_boost) {
        if (fabs(u) < boost) {
            u = sign_bit(u) ? -boost : boost;
            ri = rcp_rn(u);
            atomicAdd(&s->nboost, 1);
        }
    } else if (zero_bits(u)) {
        raise_error(s, KKT_ERR_ZERO_PIVOT, row);
        return false;
    }
    st_relaxed(Fx_d, u);
    st_relaxed(rinv_row, ri);
    return true;
}

// Spin until a published datum is not SENTINEL (bounded; abort-aware).
template <typename T>
__device__ __forceinline__ bool pub_wait(const T* p, T* v, DevScal* s, long long limit, int row) {
    T x = *v;
    for (long long it = 0; is_sentinel(x); it++) {
        if ((it & 63) == 63 && ld_volatile_int(&s->abort)) return false;
        if (it >= limit) { raise_error(s, KKT_ERR_TIMEOUT, row); return false; }
        __nanosleep(20);
        x = ld_relaxed(p);
    }
    *v = x;
    return true;
}

// Position in cols[lo, hi) of column c, or -1.  Entry e of U(k,:) (cnt
// entries, ascending columns, all of them in the row after position `step`)
// lies in [step + 1 + e, len - (cnt - 1 - e)).
__device__ __forceinline__ int slice_pos(const int32_t* cols, int lo, int hi, int c) {
    const int end = hi;
    while (lo < hi) {
        const int mid = (lo + hi) >> 1;
        if (cols[mid] < c) lo = mid + 1; else hi = mid;
    }
    return (lo < end && cols[lo] == c) ? lo : -1;
}

// A block row in shared memory finds the position of a column through a
// table of its own columns: 2^bits entries of 16-bit positions (0xFFFF
// empty), linear probing.  A row whose columns span fewer than 2^bits
// indices is mapped directly (slot c - c_0 for column c, c_0 its first:
// no collisions, and consecutive columns in consecutive slots); other rows
// by Fibonacci hashing.  Its bits: the most
// that fit `room` bytes beside the row's working set (8 st + (vsize + 4)
// len bytes), at most ceil(log2(4 len)) (load factor above 1/8) and at
// least ceil(log2(len + len/4 + 1)) (load factor below 0.8, so a probe
// sequence always meets an empty entry); -1 if even that does not fit
// (the row then runs with its values in global memory).  The host's
// placement and the kernel evaluate the same function.
constexpr int REF_TAB_EMPTY = 0xFFFF;
// windows of at most this many entries are searched rather than hashed
constexpr int REF_WINDOW_MAX = 16;
__host__ __device__ inline int ceil_log2_i64(int64_t x) {
    int b = 0;
    while (((int64_t)1 << b) < x) b++;
    return b;
}
__host__ __device__ inline int64_t row_set_bytes(int64_t st, int64_t len, int64_t vsize) {
    return 8 * st + (vsize + 4) * len;
}
__host__ __device__ inline int row_table_bits(int64_t st, int64_t len, int64_t vsize, int64_t room) {
    if (len >= REF_TAB_EMPTY) return -1;
    const int lo0 = ceil_log2_i64(len + len / 4 + 1), hi0 = ceil_log2_i64(4 * len);
    const int lo = lo0 < 4 ? 4 : lo0, hi = hi0 < 4 ? 4 : hi0;
    const int64_t base = row_set_bytes(st, len, vsize);
    for (int b = hi; b >= lo; b--)
        if (base + ((int64_t)2 << b) <= room) return b;
    return -1;
}
// c0 >= 0: the direct map of a row starting at column c0; else hashing
__device__ __forceinline__ uint32_t col_slot(int c, int bits, int c0) {
    return c0 >= 0 ? (uint32_t)(c - c0) & ((1u << bits) - 1) : ((uint32_t)c * 0x9E3779B1u) >> (32 - bits);
}

// Position of column c in a block row through its table, or -1.  A
// direct map holds every column of the row in its own slot, so its one
// probe decides.
__device__ __forceinline__ int tab_pos(const uint16_t* tab, int bits, int c0, const int32_t* cols, int c) {
    if (c0 >= 0) {
        const int p = tab[(uint32_t)(c - c0) & ((1u << bits) - 1)];
        return p == REF_TAB_EMPTY ? -1 : p;
    }
    const uint32_t mask = (1u << bits) - 1;
    for (uint32_t h = col_slot(c, bits, c0);; h = (h + 1) & mask) {
        const int p = tab[h];
        if (p == REF_TAB_EMPTY) return -1;
        if (cols[p] == c) return p;
    }
}

// A row's working set carved from `base`: step descriptors (position of
// U(k,k) and |U(k, >k)| for every L entry, 4 bytes each -- the analysis
// keeps every factor position below 2^32; k itself is the column), the
// row's values and its columns -- 8 st + (sizeof(T) + 4) len bytes -- and,
// for a block row in shared memory, its position table after them.
template <typename T>
struct RowSpace {
    uint32_t* dk;
    uint32_t* cnt;
    T* w;
    int32_t* cols;
    uint16_t* tab;
    __device__ RowSpace(unsigned char* base, int st, int len) {
        dk = reinterpret_cast<uint32_t*>(base);
        cnt = dk + st;
        w = reinterpret_cast<T*>(cnt + st);   // 8 st bytes in: aligned for double
        cols = reinterpret_cast<int32_t*>(w + len);
        tab = reinterpret_cast<uint16_t*>(cols + len);
    }
};

// One short row by one warp in its slice: gather, steps, publication, and
// (FUSED) the row's y.  Returns false if a wait gave up.
template <typename T, bool FUSED>
__device__ bool warp_row(int row, const RefArgs<T>& a, DevScal* s, T boost, long long limit,
                         unsigned long long* trace, unsigned char* slice, const FwdArgs<T>& fw) {
    const int lane = threadIdx.x & 31;
    if (trace && lane == 0) trace[2 * (size_t)row] = globaltimer_ns();
    const int64_t b = a.Fp[row], d = a.Fdiag[row], e = a.Fp[row + 1];
    const int len = (int)(e - b);
    const int nsteps = (int)(d - b);
    RowSpace<T> rs(slice, nsteps, len);
    T* w = rs.w;
    int32_t* cols = rs.cols;
    for (int q = lane; q < len; q += 32) {
        const int64_t src = a.fsrc[b + q];
        w[q] = src >= 0 ? (T)a.vals[src] : T(0);
        const int c = a.Fj[b + q];
        cols[q] = c;
        if (q < nsteps) {
            const int64_t dk = a.Fdiag[c];
            rs.dk[q] = (uint32_t)dk;
            rs.cnt[q] = (uint32_t)(a.Fp[c + 1] - dk - 1);
        }
    }
    __syncwarp();
    // the next step's pivot reciprocal and first entries of U(k,:) (one per
    // lane) are loaded while the current step runs
    T nrk = T(0), nv = T(0);
    int ncol = 0;
    auto prefetch = [&](int st) {
        if (st >= nsteps) return;
        nrk = ld_relaxed(&a.rinv[cols[st]]);
        if (lane < (int)rs.cnt[st]) {
            ncol = a.Fj[(int64_t)rs.dk[st] + 1 + lane];
            nv = ld_relaxed(&a.Fx[(int64_t)rs.dk[st] + 1 + lane]);
        }
    };
    prefetch(0);
    for (int step = 0; step < nsteps; step++) {
        const int k = cols[step];
        const int64_t dk = rs.dk[step];
        const int cnt = (int)rs.cnt[step];
        T rk = nrk, v0 = nv;
        const int c0 = ncol;
        prefetch(step + 1);
        int ok = pub_wait(&a.rinv[k], &rk, s, limit, row);
        const T l = w[step] * rk;   // l_ik = w_k * (1/u_kk)
        if (ok && lane < cnt) {   // the prefetched entry
            if (!pub_wait(&a.Fx[dk + 1 + lane], &v0, s, limit, row)) ok = 0;
            else {
                const int pos = slice_pos(cols, step + 1 + lane, len - (cnt - 1 - lane), c0);
                if (pos < 0) raise_error(s, KKT_ERR_PATTERN, row);
                else w[pos] = fma(-l, v0, w[pos]);
            }
        }
        // the other entries two per lane at a time, both loads issued first
        for (int e2 = lane + 32; e2 < cnt && ok; e2 += 64) {
            const int64_t q = dk + 1 + e2;
            const bool two = e2 + 32 < cnt;
            T v = ld_relaxed(&a.Fx[q]), v2 = T(0);
            const int c = a.Fj[q];
            int c2 = 0;
            if (two) { v2 = ld_relaxed(&a.Fx[q + 32]); c2 = a.Fj[q + 32]; }
            if (!pub_wait(&a.Fx[q], &v, s, limit, row)) { ok = 0; break; }
            const int pos = slice_pos(cols, step + 1 + e2, len - (cnt - 1 - e2), c);
            if (pos < 0) raise_error(s, KKT_ERR_PATTERN, row);
            else w[pos] = fma(-l, v, w[pos]);
            if (!two) break;
            if (!pub_wait(&a.Fx[q + 32], &v2, s, limit, row)) { ok = 0; break; }
            const int pos2 = slice_pos(cols, step + 33 + e2, len - (cnt - 33 - e2), c2);
            if (pos2 < 0) raise_error(s, KKT_ERR_PATTERN, row);
            else w[pos2] = fma(-l, v2, w[pos2]);
        }
        if (!__all_sync(0xffffffffu, ok)) return false;
        __syncwarp();
        if (lane == 0) w[step] = l;   // nobody else touches position `step` any more
        __syncwarp();
    }
    // publish: every value but the diagonal, then (lane 0) the pivot
    for (int q = lane; q < len; q += 32)
        if (b + q != d) st_relaxed(&a.Fx[b + q], w[q]);
    if (lane == 0) {
        if (publish_pivot<T>(w[d - b], boost, boost > T(0), s, row, &a.Fx[d], &a.rinv[row]) && trace)
            trace[2 * (size_t)row + 1] = globaltimer_ns();
    }
    __syncwarp();
    if (FUSED) return fused_forward_row<T>(row, b, d, SliceVals<T>{w, b}, a.Fj, fw, s, limit);
    return true;
}

// Block shapes of the refactorization kernel, picked by its shared memory
// per block: NT threads, at least MINB blocks an SM (which caps the
// registers: 80 a thread for three 256-thread blocks, 128 otherwise), PRE
// entries of each step a thread prefetches STAGES steps ahead, BATCH entries a
// thread loads together past those, TEAMS teams of NT / TEAMS threads that
// each refactor a row of their own (ROW_TEAM items: rows that fit 1/TEAMS
// of the shared memory) when the block is not working on one row whole.
// Measured on kkt2000 (three blocks an SM, the fused step's refactor):
// PRE 2 under the 80-register cap 5.05 ms against 5.31 with PRE 3 (which
// spills); on kkt10000 (two blocks an SM by shared memory) no cap 39.2 ms
// against 43.0 with it.
template <int SHAPE> struct RefShape;
template <> struct RefShape<0> { static constexpr int NT = 256, MINB = 3, PRE = 2, BATCH = 2, TEAMS = 1, STAGES = 2; };
template <> struct RefShape<1> { static constexpr int NT = 256, MINB = 2, PRE = 4, BATCH = 4, TEAMS = 1, STAGES = 2; };
template <> struct RefShape<2> { static constexpr int NT = 512, MINB = 1, PRE = 4, BATCH = 4, TEAMS = 2, STAGES = 2; };
// the teams of a shape's blocks, for the host's placement of rows
inline constexpr int ref_teams(int shape) {
    return shape == 0 ? RefShape<0>::TEAMS : shape == 1 ? RefShape<1>::TEAMS : RefShape<2>::TEAMS;
}

// The barrier of a team of tt threads working on one row: named barrier
// `id` (1 + the team's index for a team of a block, REF_BAR_BLOCK for the
// whole block), so the teams of a block never wait on each other.
constexpr int REF_BAR_BLOCK = 15;
__device__ __forceinline__ void team_sync(int id, int tt) {
    asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(tt) : "memory");
}
__device__ __forceinline__ int team_sync_or(int id, int tt, int pred) {
    int r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\tsetp.ne.s32 p, %1, 0;\n\t"
        "bar.red.or.pred q, %2, %3, p;\n\tselp.s32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"(pred), "r"(id), "r"(tt)
        : "memory");
    return r;
}

// One elimination step's first entries for one thread of a block row:
// PRE entries of U(k,:) (columns and values) and the pivot reciprocal of
// row k, loaded STAGES steps ahead so issuing them never waits on a load.
template <typename T, int PRE>
struct Stage {
    T rk;
    int32_t col[PRE];
    T val[PRE];
};

template <typename T, int PRE>
__device__ __forceinline__ void stage_load(Stage<T, PRE>& st, int tid, int NT, int step, int nsteps, const int32_t* cols,
                                           const uint32_t* dk, const uint32_t* cnt, const RefArgs<T>& a) {
    if (step >= nsteps) return;
    const int64_t base = (int64_t)dk[step] + 1;
    const int c = (int)cnt[step];
    st.rk = ld_relaxed(&a.rinv[cols[step]]);
#pragma unroll
    for (int j = 0; j < PRE; j++) {
        const int e = tid + j * NT;
        if (e < c) { st.col[j] = a.Fj[base + e]; st.val[j] = ld_relaxed(&a.Fx[base + e]); }
    }
}

// One long row by a team of NT threads: the whole block (team 0, NT the
// block's threads), or one of its RefShape::TEAMS teams (team t: threads
// [t NT, (t + 1) NT)).  rs: its working set, in shared memory (ROW_BLOCK /
// ROW_TEAM: staged here, with its position table, in `room` bytes) or in
// global memory (ROW_GLOBAL: descriptors precomputed at analysis, columns
// read from Fj, values in scratch, positions by binary search).  Returns
// false (uniformly for the team) if a wait gave up.
template <typename T, bool FUSED, int SHAPE>
__device__ bool block_row(int row, const RefArgs<T>& a, DevScal* s, T boost, long long limit,
                          unsigned long long* trace, RowSpace<T> rs, bool staged, int room, int team, int NT,
                          const FwdArgs<T>& fw) {
    constexpr int NB = RefShape<SHAPE>::NT, PRE = RefShape<SHAPE>::PRE;
    const int tid = threadIdx.x - team * NT;
    const int bar = NT == NB ? REF_BAR_BLOCK : 1 + team;
    if (trace && tid == 0) trace[2 * (size_t)row] = globaltimer_ns();
    const int64_t b = a.Fp[row], d = a.Fdiag[row], e = a.Fp[row + 1];
    const int len = (int)(e - b);
    const int nsteps = (int)(d - b);
    T* w = rs.w;
    const int32_t* cols = staged ? rs.cols : a.Fj + b;
    const int tbits = staged ? row_table_bits(nsteps, len, sizeof(T), room) : 0;
    const int dpos = (int)(d - b);
    __shared__ int s_pivot_done_t[RefShape<SHAPE>::TEAMS];   // the last step's updater of the diagonal published the pivot
    int& s_pivot_done = s_pivot_done_t[team];
    if (tid == 0) s_pivot_done = 0;
    if (staged)
        for (int h = tid; h < (1 << tbits); h += NT) rs.tab[h] = (uint16_t)REF_TAB_EMPTY;
    for (int q = tid; q < len; q += NT) {
        const int64_t src = a.fsrc[b + q];
        w[q] = src >= 0 ? (T)a.vals[src] : T(0);
        if (staged) {
            const int c = a.Fj[b + q];
            rs.cols[q] = c;
            if (q < nsteps) {
                const int64_t dk = a.Fdiag[c];
                rs.dk[q] = (uint32_t)dk;
                rs.cnt[q] = (uint32_t)(a.Fp[c + 1] - dk - 1);
            }
        }
    }
    team_sync(bar, NT);
    // the position table (every column inserted by the thread that staged
    // it): direct when the row's columns span fewer than 2^tbits indices
    const int tc0 = staged && len > 0 && rs.cols[len - 1] - rs.cols[0] < (1 << tbits) ? rs.cols[0] : -1;
    if (staged) {
        const uint32_t mask = (1u << tbits) - 1;
        for (int q = tid; q < len; q += NT) {
            if (tc0 >= 0) { rs.tab[rs.cols[q] - tc0] = (uint16_t)q; continue; }
            for (uint32_t h = col_slot(rs.cols[q], tbits, -1);; h = (h + 1) & mask)
                if (atomicCAS(&rs.tab[h], (unsigned short)REF_TAB_EMPTY, (unsigned short)q) == REF_TAB_EMPTY) break;
        }
        team_sync(bar, NT);
    }

    constexpr int STAGES = RefShape<SHAPE>::STAGES;
    Stage<T, PRE> stg[STAGES];   // indexed by constants only: registers
#pragma unroll
    for (int q = 0; q < STAGES; q++) stage_load<T, PRE>(stg[q], tid, NT, q, nsteps, cols, rs.dk, rs.cnt, a);
    int step = 0;
    // One elimination step: every thread forms l_ik = w_k * (1/u_kk) itself
    // (thread 0 also stores it), then applies its entries of U(k,:): the
    // prefetched stage, then the rest BATCH per thread with their loads
    // issued together.
    auto run_step = [&](Stage<T, PRE>& st) -> bool {
        const int k = cols[step];
        const int64_t base = (int64_t)rs.dk[step] + 1;
        const int cnt = (int)rs.cnt[step];
        int ok = 1;
        // anything still SENTINEL is re-read, all of it in one pass
        for (long long it = 0;; it++) {
            bool pending = is_sentinel(st.rk);
#pragma unroll
            for (int j = 0; j < PRE; j++)
                if (tid + j * NT < cnt && is_sentinel(st.val[j])) pending = true;
            if (!pending) break;
            if ((it & 63) == 63 && ld_volatile_int(&s->abort)) { ok = 0; break; }
            if (it >= limit) { raise_error(s, KKT_ERR_TIMEOUT, row); ok = 0; break; }
            __nanosleep(20);
            if (is_sentinel(st.rk)) st.rk = ld_relaxed(&a.rinv[k]);
#pragma unroll
            for (int j = 0; j < PRE; j++) {
                const int e2 = tid + j * NT;
                if (e2 < cnt && is_sentinel(st.val[j])) st.val[j] = ld_relaxed(&a.Fx[base + e2]);
            }
        }
        const T l = w[step] * st.rk;   // l_ik = w_k * (1/u_kk)
        // the last step leaves every value it updates final: with stream_last
        // it is published at once (U values, and the pivot by its updater),
        // so rows waiting on this one start their step while this one ends
        const bool stream = a.stream_last && step == nsteps - 1;
        auto update = [&](int pos, T v) {
            const T nw = fma(-l, v, w[pos]);
            w[pos] = nw;
            if (stream) {
                if (pos > dpos) st_relaxed(&a.Fx[b + pos], nw);
                else if (pos == dpos) {
                    if (publish_pivot<T>(nw, boost, boost > T(0), s, row, &a.Fx[d], &a.rinv[row]) && trace)
                        trace[2 * (size_t)row + 1] = globaltimer_ns();
                    s_pivot_done = 1;
                }
            }
        };
        // position of entry e2 of U(k,:), column c, in the row: a search
        // of the window entry e2 must lie in (W entries, the same width for
        // every entry of the step) when it is narrow or the row has no
        // table, else the row's table
        const int W = len - cnt - step;
        const bool by_table = staged && W > REF_WINDOW_MAX;
        auto find = [&](int c, int e2) -> int {
            return by_table ? tab_pos(rs.tab, tbits, tc0, cols, c) : slice_pos(cols, step + 1 + e2, step + 1 + e2 + W, c);
        };
        if (ok) {
#pragma unroll
            for (int j = 0; j < PRE; j++) {
                const int e2 = tid + j * NT;
                if (e2 < cnt) {
                    const int pos = find(st.col[j], e2);
                    if (pos < 0) { raise_error(s, KKT_ERR_PATTERN, row); continue; }
                    update(pos, st.val[j]);
                }
            }
            constexpr int BATCH = RefShape<SHAPE>::BATCH;
            for (int e0 = tid + PRE * NT; e0 < cnt && ok; e0 += BATCH * NT) {
                T v[BATCH];
                int c[BATCH];
#pragma unroll
                for (int u = 0; u < BATCH; u++) {
                    const int e2 = e0 + u * NT;
                    if (e2 < cnt) { v[u] = ld_relaxed(&a.Fx[base + e2]); c[u] = a.Fj[base + e2]; }
                }
#pragma unroll
                for (int u = 0; u < BATCH; u++) {
                    const int e2 = e0 + u * NT;
                    if (e2 >= cnt || !ok) continue;
                    if (!pub_wait(&a.Fx[base + e2], &v[u], s, limit, row)) { ok = 0; continue; }
                    const int pos = find(c[u], e2);
                    if (pos < 0) { raise_error(s, KKT_ERR_PATTERN, row); continue; }
                    update(pos, v[u]);
                }
            }
        }
        stage_load<T, PRE>(st, tid, NT, step + STAGES, nsteps, cols, rs.dk, rs.cnt, a);   // the stage's registers are free again
        const int any_fail = team_sync_or(bar, NT, !ok);   // uniform decision for the team
        if (tid == 0) w[step] = l;   // nobody else touches position `step` any more
        step++;
        return !any_fail;
    };
    bool ok = true;
    while (step < nsteps && ok) {
#pragma unroll
        for (int q = 0; q < STAGES; q++) {
            if (!ok || step >= nsteps) break;
            ok = run_step(stg[q]);
        }
    }
    if (!ok) return false;
    // publish (the row is final after the last step's barrier): every
    // thread its share of the values but the diagonal, then thread 0 the
    // pivot; the last step's l, which thread 0 wrote after that barrier,
    // thread 0 stores itself
    for (int q = tid; q < len; q += NT)
        if (b + q != d && q != nsteps - 1) st_relaxed(&a.Fx[b + q], w[q]);
    if (tid == 0) {
        if (nsteps > 0) st_relaxed(&a.Fx[b + nsteps - 1], w[nsteps - 1]);
        if (!s_pivot_done &&
            publish_pivot<T>(w[d - b], boost, boost > T(0), s, row, &a.Fx[d], &a.rinv[row]) && trace)
            trace[2 * (size_t)row + 1] = globaltimer_ns();
    }
    // the fused forward sweep's y_row, by warp 0 from the row's values; the
    // other warps wait at the next item's first barrier
    if (FUSED && tid < 32) {
        __syncwarp();   // thread 0's last L value
        fused_forward_row<T>(row, b, d, SliceVals<T>{w, b}, a.Fj, fw, s, limit);
    }
    return true;
}

// The refactorization: blocks of NT threads take work items from the
// ticket until none is left.  Shared memory: a block row's working set and
// position table, or one slice per warp for warp rows.  BATCH: the items
// of several instances (RefBatch); else those of `one`.
template <typename T, bool FUSED, int SHAPE, bool BATCH>
__global__ void __launch_bounds__(RefShape<SHAPE>::NT, RefShape<SHAPE>::MINB)
k_refactor_rows(RefArgs<T> one, RefBatch<T> batch, long long limit, unsigned long long* trace) {
    constexpr int NT = RefShape<SHAPE>::NT;
    extern __shared__ __align__(16) unsigned char ref_sh[];
    __shared__ RefItem s_item;
    __shared__ int s_inst;
    __shared__ RefArgs<T> s_args;   // BATCH: the current item's instance, read from shared memory
    const int tid = threadIdx.x;
    for (;;) {
        if (tid == 0) {
            int inst = -1;
            if (!BATCH) {
                const int q = (int)atomicAdd(&one.s->ticket_fact, 1u);
                if (q < one.nitems && !ld_volatile_int(&one.s->abort)) { inst = 0; s_item = one.items[q]; }
            } else {
                for (;;) {
                    const long long t = (long long)atomicAdd(batch.ticket, 1ull);
                    if (t >= batch.total) break;
                    const int j = (int)(t % batch.count);
                    const int q = (int)(t / batch.count);
                    const RefArgs<T>& aj = batch.args[j];
                    if (q < aj.nitems && !ld_volatile_int(&aj.s->abort)) {
                        inst = j;
                        s_item = aj.items[q];
                        s_args = aj;
                        break;
                    }
                }
            }
            s_inst = inst;
        }
        __syncthreads();
        const int inst = s_inst;
        const RefItem it = s_item;
        __syncthreads();   // s_inst and s_item are read before thread 0 may overwrite them
        if (inst < 0) return;
        const RefArgs<T>& a = BATCH ? s_args : one;
        DevScal* s = a.s;
        const T boost = (T)(a.boost_eps * *(volatile double*)&s->normA);
        const int kind = it.info >> 28;
        if (kind == ROW_WARP) {
            const int count = it.info & 0x0fffffff;
            const int warp = tid >> 5;
            if (warp < count) {
                const int row = a.order[it.first + warp];
                warp_row<T, FUSED>(row, a, s, boost, limit, trace, ref_sh + warp * a.slice_bytes, a.fw);
            }
            __syncthreads();   // the slices are reused by the next item
        } else {
            // ROW_BLOCK / ROW_GLOBAL: the whole block on one row; ROW_TEAM:
            // each team on a row of its own in its share of the memory
            constexpr int TEAMS = RefShape<SHAPE>::TEAMS;
            const bool teams = TEAMS > 1 && kind == ROW_TEAM;
            const int nt = teams ? NT / TEAMS : NT;
            const int team = teams ? tid / nt : 0;
            const int room = teams ? (a.area_bytes / TEAMS) & ~15 : a.area_bytes;
            const int count = teams ? it.info & 0x0fffffff : 1;
            int ok = 1;
            if (team < count) {
                const int row = a.order[it.first + team];
                const int64_t b = a.Fp[row];
                const int len = (int)(a.Fp[row + 1] - b), nsteps = (int)(a.Fdiag[row] - b);
                RowSpace<T> rs(ref_sh + team * room, nsteps, len);
                const bool staged = kind != ROW_GLOBAL;
                if (!staged) {   // ROW_GLOBAL: descriptors and values in global memory
                    const int g = it.info & 0x0fffffff;
                    rs.dk = const_cast<uint32_t*>(a.gdk) + a.g_sd_off[g];
                    rs.cnt = const_cast<uint32_t*>(a.gcnt) + a.g_sd_off[g];
                    rs.w = a.gw + a.g_w_off[g];
                }
                ok = block_row<T, FUSED, SHAPE>(row, a, s, boost, limit, trace, rs, staged, room, team, nt, a.fw);
            }
            if (teams) ok = !__syncthreads_or(!ok);   // the teams' rooms are reused by the next item
            if (!ok && !BATCH) return;
        }
    }
}

// ---------------------------------------------------------------- K2/K3: triangular solves
// Rows are scheduled in the order of their level in the dependency DAG
// (L: the forward sweep's levels; U: the backward sweep's), so warps that
// take rows in list order never block behind a row of a much later level.
// Fpos[p] is the list position of entry p's dependency (L part: in the L
// list, U part: in the U list).  Every schedule evaluates a row with
// trsv_row (trsv_row.cuh), so all of them give the same bits.
//
// Whole-GPU schedule (any n): the wide part runs sync-free (warps take rows
// from a ticket, operands polled in global memory); the narrow end of each
// DAG -- the long chain the fill-reducing order puts last -- runs in ONE
// block whose warps hand values through shared memory.  L: bulk, then the
// chain (the highest levels); U: the chain (the lowest levels), then the
// bulk.  Global operands that are not computed yet hold SENTINEL; each
// sweep re-arms the other one's vector (L sets xp = SENTINEL, U sets
// y = SENTINEL after reading it).

__global__ void k_trsv_prep(DevScal* s) {
    s->ticket_l = 0;
    s->ticket_u = 0;
}

template <typename T>
__global__ void k_fill_sentinel(T* a, int64_t n) {
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = sentinel_of<T>();
}


// T: factor and solve type (double, or float in mixed precision); the
// right-hand side and the result of a sweep pair stay double.
template <typename T>
__global__ void k_lsolve_bulk(int nrows, const int32_t* __restrict__ rows, const int64_t* __restrict__ Fp,
                              const int32_t* __restrict__ Fj, const int64_t* __restrict__ Fdiag,
                              const T* __restrict__ Fx, const int32_t* __restrict__ P,
                              const double* __restrict__ rhs, T* y, T* xp, DevScal* s, long long limit) {
    const int lane = threadIdx.x & 31;
    const GiveUpGlobal gu{&s->abort};
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&s->ticket_l, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= nrows) return;
        const int row = rows[t];
        const T r0 = rhs_value<T>(rhs[P[row]]);
        T val;
        if (!trsv_row<true>(Fp[row], Fdiag[row], Fx, SrcGlobal<T>{Fj, y}, r0, T(1), limit, gu, &val)) {
            if (lane == 0) fail_row(s, row);
            return;
        }
        if (lane == 0) {
            xp[row] = sentinel_of<T>();
            st_relaxed(&y[row], val);
        }
    }
}

template <typename T>
struct SrcChainL {   // dependency in the chain: shared memory; else y (final)
    static constexpr int kPollNs = 0;
    const int32_t* Fj;
    const int32_t* Fpos;
    int cstart;
    const volatile T* xs;
    const T* y;
    __device__ const volatile T* operator()(int64_t p) const {
        const int t = __ldg(&Fpos[p]) - cstart;
        return t >= 0 ? xs + t : y + __ldg(&Fj[p]);
    }
};

struct GiveUpShared {
    const int* abort;
    __device__ bool operator()() const { return *(volatile const int*)abort != 0; }
};

// The narrow end of the L-sweep in one block: warp w takes chain slots w,
// w + nwarps, ... (slot t = list position cstart + t).
template <typename T>
__global__ void __launch_bounds__(1024)
k_lsolve_chain(int nt, int cstart, const int32_t* __restrict__ rows, const int32_t* __restrict__ Fpos,
               const int64_t* __restrict__ Fp, const int32_t* __restrict__ Fj, const int64_t* __restrict__ Fdiag,
               const T* __restrict__ Fx, const int32_t* __restrict__ P, const double* __restrict__ rhs,
               T* y, T* xp, DevScal* s, long long limit) {
    extern __shared__ __align__(16) unsigned char chain_sh[];
    volatile T* xs = reinterpret_cast<T*>(chain_sh);
    for (int t = threadIdx.x; t < nt; t += blockDim.x) xs[t] = sentinel_of<T>();
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const GiveUpShared gu{&s->abort};
    for (int t = warp; t < nt; t += nw) {
        const int row = rows[cstart + t];
        const T r0 = rhs_value<T>(rhs[P[row]]);
        T val;
        if (!trsv_row<true>(Fp[row], Fdiag[row], Fx, SrcChainL<T>{Fj, Fpos, cstart, xs, y}, r0, T(1), 4 * limit,
                            gu, &val)) {
            if (lane == 0) fail_row(s, row);
            return;
        }
        if (lane == 0) {
            xs[t] = val;
            y[row] = val;
            xp[row] = sentinel_of<T>();
        }
        __syncwarp();
    }
}

template <typename T>
struct SrcChainU {   // every dependency of a U-chain row is in the chain
    static constexpr int kPollNs = 0;
    const int32_t* Fj;
    const int32_t* Fpos;
    int nt;
    const volatile T* xs;
    const T* xp;
    __device__ const volatile T* operator()(int64_t p) const {
        const int t = __ldg(&Fpos[p]);
        return t < nt ? xs + t : xp + __ldg(&Fj[p]);
    }
};

template <typename T>
__global__ void __launch_bounds__(1024)
k_usolve_chain(int nt, const int32_t* __restrict__ rows, const int32_t* __restrict__ Fpos,
               const int64_t* __restrict__ Fp, const int32_t* __restrict__ Fj, const int64_t* __restrict__ Fdiag,
               const T* __restrict__ Fx, const T* __restrict__ rinv_u, const int32_t* __restrict__ Q, T* y, T* xp,
               double* __restrict__ out, DevScal* s, long long limit) {
    extern __shared__ __align__(16) unsigned char chain_sh[];
    volatile T* xs = reinterpret_cast<T*>(chain_sh);
    for (int t = threadIdx.x; t < nt; t += blockDim.x) xs[t] = sentinel_of<T>();
    __syncthreads();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nw = blockDim.x >> 5;
    const GiveUpShared gu{&s->abort};
    for (int t = warp; t < nt; t += nw) {
        const int row = rows[t];
        const int64_t d = Fdiag[row];
        const T r0 = __ldcg(&y[row]);
        const T rinv = __ldg(&rinv_u[row]);   // 1/u_ii as the refactorization formed it
        const int qrow = Q[row];
        T val;
        if (!trsv_row<false>(d + 1, Fp[row + 1], Fx, SrcChainU<T>{Fj, Fpos, nt, xs, xp}, r0, rinv, 4 * limit, gu,
                             &val)) {
            if (lane == 0) fail_row(s, row);
            return;
        }
        if (lane == 0) {
            xs[t] = val;
            xp[row] = val;
            y[row] = sentinel_of<T>();
            out[qrow] = (double)val;
        }
        __syncwarp();
    }
}

template <typename T>
__global__ void k_usolve_bulk(int nrows, const int32_t* __restrict__ rows, const int64_t* __restrict__ Fp,
                              const int32_t* __restrict__ Fj, const int64_t* __restrict__ Fdiag,
                              const T* __restrict__ Fx, const T* __restrict__ rinv_u, const int32_t* __restrict__ Q,
                              T* y, T* xp, double* __restrict__ out, DevScal* s, long long limit) {
    const int lane = threadIdx.x & 31;
    const GiveUpGlobal gu{&s->abort};
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&s->ticket_u, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= nrows) return;
        const int row = rows[t];
        const int64_t d = Fdiag[row];
        const T r0 = __ldcg(&y[row]);
        const T rinv = __ldg(&rinv_u[row]);   // 1/u_ii as the refactorization formed it
        const int qrow = Q[row];
        T val;
        if (!trsv_row<false>(d + 1, Fp[row + 1], Fx, SrcGlobal<T>{Fj, xp}, r0, rinv, limit, gu, &val)) {
            if (lane == 0) fail_row(s, row);
            return;
        }
        if (lane == 0) {
            st_relaxed(&xp[row], val);
            y[row] = sentinel_of<T>();
            out[qrow] = (double)val;
        }
    }
}

// ---------------------------------------------------------------- K2/K3: cluster solves
// The whole triangular solve in ONE thread-block cluster of C blocks
// (C = 8 or 16), the solved values kept in the blocks' shared memory --
// the distributed shared memory of the cluster -- so every hand-off is a
// shared-memory store read by a (distributed) shared-memory load, with no
// global synchronisation.  List position t goes to warp g = t mod 32C of
// the cluster; its value lives in that warp's block at slot
// (t / 32C) * 32 + t mod 32.  Used when n values fit in the cluster.
// L: reads the double right-hand side, writes y (type T); U: reads y,
// writes the double result.
namespace cgx = cooperative_groups;
constexpr int CLUSTER_THREADS = 1024;

template <typename T>
struct SrcCluster {   // operand in the cluster's distributed shared memory
    static constexpr int kPollNs = 0;
    const int32_t* Fpos;
    T* xs_local;
    int rank, sh, stride;
    cgx::cluster_group* cl;
    __device__ const volatile T* operator()(int64_t p) const {
        const int tj = __ldg(&Fpos[p]);
        const int owner = (tj & (stride - 1)) >> 5;
        const int slot = ((tj >> sh) << 5) + (tj & 31);
        return (owner == rank ? xs_local : cl->map_shared_rank(xs_local, owner)) + slot;
    }
};

template <bool LOWER, typename T, typename TIN, typename TOUT>
__device__ __forceinline__ void trsv_cluster_body(int n, const int32_t* __restrict__ list,
                                                  const int32_t* __restrict__ Fpos, const int64_t* __restrict__ Fp,
                                                  const int64_t* __restrict__ Fdiag, const T* __restrict__ Fx,
                                                  const T* __restrict__ rinv_u, const int32_t* __restrict__ perm,
                                                  const TIN* __restrict__ rhs, TOUT* __restrict__ out, DevScal* s,
                                                  long long limit, unsigned long long* __restrict__ trace) {
    extern __shared__ __align__(16) unsigned char cl_sh[];
    T* xs_cl = reinterpret_cast<T*>(cl_sh);
    cgx::cluster_group cluster = cgx::this_cluster();
    const int C = (int)cluster.num_blocks();
    const int rank = (int)cluster.block_rank();
    const int stride = 32 * C;                 // a power of two (C is 8 or 16)
    const int sh = 31 - __clz(stride);
    const int per_block = ((n + stride - 1) / stride) * 32;
    for (int i = threadIdx.x; i < per_block; i += blockDim.x) xs_cl[i] = sentinel_of<T>();
    cluster.sync();
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const GiveUpGlobal gu{&s->abort};
    const SrcCluster<T> src{Fpos, xs_cl, rank, sh, stride, &cluster};
    for (int t = rank * 32 + warp; t < n; t += stride) {
        const int row = list[t];
        const int64_t d = Fdiag[row];
        const T r0 = LOWER ? rhs_value<T>(rhs[perm[row]]) : (T)rhs[row];
        const T rinv = LOWER ? T(1) : __ldg(&rinv_u[row]);   // 1/u_ii as the refactorization formed it
        const int orow = LOWER ? row : perm[row];
        T val;
        const bool ok = LOWER ? trsv_row<true>(Fp[row], d, Fx, src, r0, rinv, limit, gu, &val)
                              // one early load per lane in flight: at the 64-register cap of
                              // 1024-thread blocks the batched loads spilled (U-sweep 2.08 ->
                              // 1.89 ms on kkt2000; same bits)
                              : trsv_row_v<false, T, LdgVals<T>, SrcCluster<T>, GiveUpGlobal, 1>(
                                    d + 1, Fp[row + 1], LdgVals<T>{Fx}, src, r0, rinv, limit, gu, &val);
        if (!ok) {
            if (lane == 0) fail_row(s, row);
            break;
        }
        if (lane == 0) {
            ((volatile T*)xs_cl)[((t >> sh) << 5) + warp] = val;
            out[orow] = (TOUT)val;
            if (trace) trace[t] = globaltimer_ns();   // profiling: publish time of list position t
        }
        __syncwarp();
    }
    cluster.sync();   // no block may leave while others can still read its shared memory
}

template <bool LOWER, typename T, typename TIN, typename TOUT>
__global__ void __launch_bounds__(CLUSTER_THREADS)
k_trsv_cluster(int n, const int32_t* __restrict__ list, const int32_t* __restrict__ Fpos,
               const int64_t* __restrict__ Fp, const int64_t* __restrict__ Fdiag, const T* __restrict__ Fx,
               const T* __restrict__ rinv_u, const int32_t* __restrict__ perm, const TIN* __restrict__ rhs,
               TOUT* __restrict__ out, DevScal* s, long long limit, unsigned long long* __restrict__ trace) {
    trsv_cluster_body<LOWER, T, TIN, TOUT>(n, list, Fpos, Fp, Fdiag, Fx, rinv_u, perm, rhs, out, s, limit, trace);
}

// The backward sweep of a batch of instances, one cluster each (cluster
// i = blocks [i C, (i + 1) C) of the grid runs instance i).
struct SweepArgs {
    int n;
    const int32_t* list;
    const int32_t* Fpos;
    const int64_t* Fp;
    const int64_t* Fdiag;
    const double* Fx;
    const double* rinv;
    const int32_t* perm;
    const double* rhs;
    double* out;
    DevScal* s;
};

__global__ void __launch_bounds__(CLUSTER_THREADS)
k_usolve_cluster_batch(const SweepArgs* sa, long long limit) {
    const SweepArgs& a = sa[blockIdx.x / cgx::this_cluster().num_blocks()];
    trsv_cluster_body<false, double, double, double>(a.n, a.list, a.Fpos, a.Fp, a.Fdiag, a.Fx, a.rinv, a.perm, a.rhs,
                                                     a.out, a.s, limit, nullptr);
}

// ---------------------------------------------------------------- self-test of bounded waits
// One warp waits, with the same primitives the kernels use, for a value and
// a flag that nothing sets; both waits must give up and record the error.
__global__ void k_selftest_wait(DevScal* s, const double* never, const unsigned* never_flag, long long limit) {
    double v = ld_relaxed_f64(never);
    const GiveUpGlobal gu{&s->abort};
    const bool got_value = spin_value<20>(never, &v, limit, gu);
    const bool got_flag = wait_flag(never_flag, 0xffffffffu, s, limit, -1);
    if (threadIdx.x == 0 && (!got_value || !got_flag)) raise_error(s, KKT_ERR_TIMEOUT, -1);
}

// ---------------------------------------------------------------- K4: products with K
// 8 lanes per row; all 8 lanes of a group share `row` and `active`.
__device__ __forceinline__ double row_dot8(const int32_t* __restrict__ Arp, const int32_t* __restrict__ Aci,
                                           const double* __restrict__ Ax, const double* __restrict__ x, int row,
                                           int sub, bool active) {
    double acc = 0.0;
    if (active)
        for (int e = Arp[row] + sub; e < Arp[row + 1]; e += 8) acc += Ax[e] * __ldcg(&x[Aci[e]]);
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    return acc;
}

// w = K z
__global__ void k_spmv(int n, const int32_t* __restrict__ Arp, const int32_t* __restrict__ Aci,
                       const double* __restrict__ Ax, const double* __restrict__ z, double* __restrict__ w) {
    const int64_t g = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x);
    const int sub = threadIdx.x & 7;
    const int64_t rows_per_pass = ((int64_t)gridDim.x * blockDim.x) >> 3;
    const int64_t trips = (n + rows_per_pass - 1) / rows_per_pass;
    for (int64_t t = 0; t < trips; t++) {
        const int64_t base = (g >> 3) + t * rows_per_pass;
        const bool active = base < n;
        const int row = active ? (int)base : 0;
        const double v = row_dot8(Arp, Aci, Ax, z, row, sub, active);
        if (active && sub == 0) w[row] = v;
    }
}

// r = b - K x, with ||r||^2, ||x||^2 and ||b||^2 reduced into s (rnorm,
// xnorm, normb).  mode 0: also sets rnorm0 and the refine decision of the
// initial solve; mode 1: cycle end (true residual of the formed x).
// Block bx of nb (the sums depend only on nb and the block's rows, so a
// batched launch gives the same bits as a lone one).
__device__ __forceinline__ void residual_body(int n, const int32_t* __restrict__ Arp,
                                              const int32_t* __restrict__ Aci, const double* __restrict__ Ax,
                                              const double* __restrict__ b, const double* __restrict__ x,
                                              double* __restrict__ r, double* part, DevScal* s, int bx, int nb) {
    __shared__ double sh[33];
    const int64_t g = ((int64_t)bx * blockDim.x + threadIdx.x);
    const int sub = threadIdx.x & 7;
    const int64_t rows_per_pass = ((int64_t)nb * blockDim.x) >> 3;
    double rr = 0.0, xx = 0.0, bb = 0.0;
    const int64_t first = g >> 3;
    const int64_t trips = (n + rows_per_pass - 1) / rows_per_pass;
    for (int64_t t = 0; t < trips; t++) {
        const int64_t base = first + t * rows_per_pass;
        const bool active = base < n;
        const int row = active ? (int)base : 0;
        double v = row_dot8(Arp, Aci, Ax, x, row, sub, active);
        if (active && sub == 0) {
            const double ri = b[row] - v;
            r[row] = ri;
            rr += ri * ri;
            const double xi = __ldcg(&x[row]);
            xx += xi * xi;
            bb += b[row] * b[row];
        }
    }
    rr = block_sum(rr, sh);
    xx = block_sum(xx, sh);
    bb = block_sum(bb, sh);
    if (threadIdx.x == 0) {
        part[bx * RED_SLOTS + 0] = rr;
        part[bx * RED_SLOTS + 1] = xx;
        part[bx * RED_SLOTS + 2] = bb;
    }
    if (!last_block(s, (unsigned)nb)) return;
    rr = reduce_partials(part, 0, sh, nb);
    xx = reduce_partials(part, 1, sh, nb);
    bb = reduce_partials(part, 2, sh, nb);
    if (threadIdx.x == 0) {
        s->rnorm = sqrt(rr);
        s->xnorm = sqrt(xx);
        s->normb = sqrt(bb);
    }
}

__global__ void k_residual(int n, const int32_t* __restrict__ Arp, const int32_t* __restrict__ Aci,
                           const double* __restrict__ Ax, const double* __restrict__ b,
                           const double* __restrict__ x, double* __restrict__ r, double* part, DevScal* s) {
    residual_body(n, Arp, Aci, Ax, b, x, r, part, s, blockIdx.x, gridDim.x);
}

// The residual of a batch of instances: blockIdx.y = instance, its first
// nb blocks of the x dimension take part.
struct ResidualArgs {
    int n, nb;
    const int32_t* Arp;
    const int32_t* Aci;
    const double* Ax;
    const double* b;
    const double* x;
    double* r;
    double* part;
    DevScal* s;
    int stop_mode;
    double refine_delta;
};

__global__ void k_residual_batch(const ResidualArgs* ra) {
    const ResidualArgs& a = ra[blockIdx.y];
    if ((int)blockIdx.x >= a.nb) return;
    residual_body(a.n, a.Arp, a.Aci, a.Ax, a.b, a.x, a.r, a.part, a.s, blockIdx.x, a.nb);
}

// ---------------------------------------------------------------- K5-K7: FGMRES
// Decision after a residual: NRBE of the current x, refine-or-not (initial
// solve, Section 2.3) or accept/restart (cycle end).
// mode 0: after x0; mode 1: after a cycle; mode 2: after a Richardson
// correction (counted as an iteration); mode 3: after a cycle of FGMRES on
// the error equation (RR is then tested on the true residual).
__device__ void decide_rule(DevScal* s, int mode, double tol, int stop_mode, double refine_delta, double rn,
                            double bn, double nrbe);

// In a CUDA graph with device-side loop control (graph != 0) the decision
// also sets the WHILE condition: continue while the solve is not done and
// the cap (max_cycles cycles, or max_cycles * m Richardson corrections) is
// not reached.
__global__ void k_decide(DevScal* s, int mode, double tol, int stop_mode, double refine_delta,
                         int cap, int graph) {
    const double rn = s->rnorm, xn = s->xnorm, bn = s->normb;
    const double nrbe = (rn == 0.0) ? 0.0 : rn / (s->normA * xn + bn);
    s->nrbe = nrbe;
    if (!isfinite(rn) || !isfinite(xn)) {
        s->err = KKT_ERR_NONFINITE;
        s->done = 1;
        if (graph) cudaGraphSetConditional(s->h_loop, 0u);
        return;
    }
    decide_rule(s, mode, tol, stop_mode, refine_delta, rn, bn, nrbe);
    if (graph) {
        const int used = (mode == 2) ? s->iters : s->cycles;
        int cont = !s->done;
        if (cont && used >= cap) { s->not_converged = 1; cont = 0; }
        cudaGraphSetConditional(s->h_loop, (unsigned)cont);
    }
}

__device__ void decide_rule(DevScal* s, int mode, double tol, int stop_mode, double refine_delta, double rn,
                            double bn, double nrbe) {
    if (mode == 0) {
        s->rnorm0 = rn;
        s->iters = 0;
        s->cycles = 0;
        s->not_converged = 0;
        s->done = 0;
        if (rn == 0.0) s->done = 1;
        else if (refine_delta > 0.0 && rn < refine_delta * bn) s->done = 1;
        else if (stop_mode == KKT_STOP_NRBE && nrbe <= tol) s->done = 1;
    } else {
        if (mode == 2) s->iters += 1;
        const int rr_met = (mode == 1) ? s->met : (rn < tol * s->rnorm0);
        if (rn == 0.0) s->done = 1;
        else if (stop_mode == KKT_STOP_NRBE && nrbe <= tol) s->done = 1;
        else if (stop_mode == KKT_STOP_RR && rr_met) s->done = 1;
    }
}

// The initial-solve decision (mode 0) of a batch of instances, one thread each.
__global__ void k_decide_batch(const ResidualArgs* ra, int count, double tol) {
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= count) return;
    DevScal* s = ra[i].s;
    if (s->err) { s->done = 1; return; }   // its refactorization failed: keep that error
    const double rn = s->rnorm, xn = s->xnorm, bn = s->normb;
    const double nrbe = (rn == 0.0) ? 0.0 : rn / (s->normA * xn + bn);
    s->nrbe = nrbe;
    if (!isfinite(rn) || !isfinite(xn)) {
        s->err = KKT_ERR_NONFINITE;
        s->done = 1;
        return;
    }
    decide_rule(s, 0, tol, ra[i].stop_mode, ra[i].refine_delta, rn, bn, nrbe);
}

// x += d (Richardson correction)
__global__ void k_axpy(int n, const double* __restrict__ d, double* __restrict__ x) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = tid; t < n; t += stride) x[t] += d[t];
}

// v_0 = r / ||r||, g = (||r||, 0, ...), threshold of the inner test.
// inner_rel > 0 (FGMRES on the error equation): the cycle's inner test is
// |g_{j+1}| <= inner_rel * beta.
// In a graph, step 0's IF is armed and the other steps' IFs are cleared.
__global__ void k_cycle_init(int n, const double* __restrict__ r, double* __restrict__ v0, DevScal* s,
                             double tol, int stop_mode, double inner_rel, int m, int graph) {
    const double beta = *(volatile double*)&s->rnorm;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = tid; t < n; t += stride) v0[t] = r[t] / beta;
    if (tid == 0) {
        s->g[0] = beta;
        for (int i = 1; i <= MAXM; i++) s->g[i] = 0.0;
        s->thresh = inner_rel > 0.0 ? inner_rel * beta
                  : (stop_mode == KKT_STOP_NRBE) ? tol * (s->normA * s->xnorm + s->normb) : tol * s->rnorm0;
        s->j = 0;
        s->met = 0;
        s->cycles += 1;
        if (graph)
            for (int i = 0; i < m; i++) cudaGraphSetConditional(s->h_step[i], i == 0 ? 1u : 0u);
    }
}

// sqrt(a^2 - ||h[0..k)||^2) as sqrt((a - c)(a + c)), c = ||h||; 0 if a <= c
// (the norm of a projected vector from norms taken before the projection).
__device__ __forceinline__ double pythagoras(double a, const double* h, int k) {
    double c = 0.0;
    for (int i = 0; i < k; i++) c += h[i] * h[i];
    c = sqrt(c);
    if (!(a > c)) return 0.0;
    return sqrt((a - c) * (a + c));
}

// End of Arnoldi step j (one thread): H(:,j) = h (+ h2), h_{j+1,j} = hn,
// previous Givens rotations applied, new rotation formed, g updated, the
// inner stopping test sets s->met, j advances.
// In a graph, step j + 1's IF is armed only while the estimate has not met
// the test and no breakdown occurred.
__device__ void arnoldi_finish(DevScal* s, int j, double hn, bool add_h2, int stop_mode, int m, int graph) {
    s->hn = hn;
    double* Hj = s->H + j * (MAXM + 1);
    for (int i = 0; i <= j; i++) Hj[i] = add_h2 ? s->h[i] + s->h2[i] : s->h[i];
    Hj[j + 1] = hn;
    for (int i = 0; i < j; i++) {
        const double a = Hj[i], bb = Hj[i + 1];
        Hj[i] = s->cs[i] * a + s->sn[i] * bb;
        Hj[i + 1] = -s->sn[i] * a + s->cs[i] * bb;
    }
    const double a = Hj[j], bb = Hj[j + 1];
    const double rr = hypot(a, bb);
    if (rr == 0.0) { s->cs[j] = 1.0; s->sn[j] = 0.0; }
    else { s->cs[j] = a / rr; s->sn[j] = bb / rr; }
    Hj[j] = rr;
    Hj[j + 1] = 0.0;
    s->g[j + 1] = -s->sn[j] * s->g[j];
    s->g[j] = s->cs[j] * s->g[j];
    s->iters += 1;
    const double est = fabs(s->g[j + 1]);
    const int met = (stop_mode == KKT_STOP_NRBE) ? (est <= s->thresh) : (est < s->thresh);
    s->met = met;
    s->j = j + 1;
    if (graph && j + 1 < m) cudaGraphSetConditional(s->h_step[j + 1], (unsigned)(!met && hn > 0.0));
}

// Classical Gram-Schmidt, first projection: h_i = v_i . w for i <= j.
// with_norm (one-reduction CGS): ||w||^2 is reduced with the h_i and the
// last block finishes the Arnoldi step with h_{j+1,j} by Pythagoras.
__global__ void k_cgs_dots(int n, const double* __restrict__ V, int64_t ld, const double* __restrict__ w,
                           double* part, DevScal* s, int with_norm, int stop_mode, int m, int graph) {
    __shared__ double sh[33];
    const int j = *(volatile int*)&s->j;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int i = 0; i <= j; i++) {
        const double* vi = V + (int64_t)i * ld;
        double acc = 0.0;
        for (int64_t t = tid; t < n; t += stride) acc += vi[t] * w[t];
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) part[blockIdx.x * RED_SLOTS + i] = acc;
    }
    if (with_norm) {
        double acc = 0.0;
        for (int64_t t = tid; t < n; t += stride) acc += w[t] * w[t];
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) part[blockIdx.x * RED_SLOTS + j + 1] = acc;
    }
    if (!last_block(s)) return;
    for (int i = 0; i <= j; i++) {
        double v = reduce_partials(part, i, sh);
        if (threadIdx.x == 0) s->h[i] = v;
    }
    if (!with_norm) return;
    const double nn = reduce_partials(part, j + 1, sh);
    if (threadIdx.x == 0) arnoldi_finish(s, j, pythagoras(sqrt(nn), s->h, j + 1), false, stop_mode, m, graph);
}

// w -= V h (pass 0: h, then h2_i = v_i . w) or (pass 1: h2, then ||w||^2);
// the last block of pass 1 finishes the Arnoldi step: H(:,j) = h + h2 and
// h_{j+1,j} = ||w||, previous Givens rotations applied, new rotation
// formed, g updated; the inner stopping test sets s->met.
// with_norm (pass 0 only; CGS2 with the norm by Pythagoras): ||w||^2 after
// the first projection is reduced with the h2_i and the last block finishes
// the Arnoldi step; the second projection then comes with the normalisation
// (k_project_normalize).
__global__ void k_cgs_update(int n, const double* __restrict__ V, int64_t ld, double* __restrict__ w, int pass,
                             double* part, DevScal* s, int m, int stop_mode, int with_norm, int graph) {
    __shared__ double sh[33];
    __shared__ double hc[MAXM + 1];
    const int j = *(volatile int*)&s->j;
    const double* hsrc = pass == 0 ? s->h : s->h2;
    for (int i = threadIdx.x; i <= j; i += blockDim.x) hc[i] = ((volatile double*)hsrc)[i];
    __syncthreads();
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = tid; t < n; t += stride) {
        double wt = w[t];
        for (int i = 0; i <= j; i++) wt -= hc[i] * V[(int64_t)i * ld + t];
        w[t] = wt;
    }
    __syncthreads();
    if (pass == 0) {
        for (int i = 0; i <= j; i++) {
            const double* vi = V + (int64_t)i * ld;
            double acc = 0.0;
            for (int64_t t = tid; t < n; t += stride) acc += vi[t] * w[t];
            acc = block_sum(acc, sh);
            if (threadIdx.x == 0) part[blockIdx.x * RED_SLOTS + i] = acc;
        }
        if (with_norm) {
            double acc = 0.0;
            for (int64_t t = tid; t < n; t += stride) acc += w[t] * w[t];
            acc = block_sum(acc, sh);
            if (threadIdx.x == 0) part[blockIdx.x * RED_SLOTS + j + 1] = acc;
        }
    } else {
        double acc = 0.0;
        for (int64_t t = tid; t < n; t += stride) acc += w[t] * w[t];
        acc = block_sum(acc, sh);
        if (threadIdx.x == 0) part[blockIdx.x * RED_SLOTS + 0] = acc;
    }
    if (!last_block(s)) return;
    if (pass == 0) {
        for (int i = 0; i <= j; i++) {
            double v = reduce_partials(part, i, sh);
            if (threadIdx.x == 0) s->h2[i] = v;
        }
        if (!with_norm) return;
        const double nn = reduce_partials(part, j + 1, sh);
        if (threadIdx.x == 0) arnoldi_finish(s, j, pythagoras(sqrt(nn), s->h2, j + 1), true, stop_mode, m, graph);
        return;
    }
    double nn = reduce_partials(part, 0, sh);
    if (threadIdx.x != 0) return;
    arnoldi_finish(s, j, sqrt(nn), true, stop_mode, m, graph);
}

// The projection left after a Pythagorean finish, fused with the
// normalisation: w -= V(:, 0..j-1) hx (hx = h for one-reduction CGS, h2
// for CGS2), then v_j = w / h_{j,j-1} (j was already advanced).
__global__ void k_project_normalize(int n, double* __restrict__ w, double* __restrict__ V, int64_t ld, DevScal* s,
                                    int use_h2) {
    __shared__ double hc[MAXM + 1];
    const int j = *(volatile int*)&s->j;   // advanced: columns 0..j-1 project, column j is new
    const double hn = *(volatile double*)&s->hn;
    const double* hsrc = use_h2 ? s->h2 : s->h;
    for (int i = threadIdx.x; i < j; i += blockDim.x) hc[i] = ((volatile double*)hsrc)[i];
    __syncthreads();
    double* vn = V + (int64_t)j * ld;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = tid; t < n; t += stride) {
        double wt = w[t];
        for (int i = 0; i < j; i++) wt -= hc[i] * V[(int64_t)i * ld + t];
        w[t] = wt;
        vn[t] = hn > 0.0 ? wt / hn : 0.0;
    }
}

// v_{j+1} = w / h_{j+1,j} (zero on breakdown); j was already advanced.
__global__ void k_normalize(int n, const double* __restrict__ w, double* __restrict__ V, int64_t ld, DevScal* s) {
    const int j = *(volatile int*)&s->j;
    const double hn = *(volatile double*)&s->hn;
    double* vn = V + (int64_t)j * ld;
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = tid; t < n; t += stride) vn[t] = hn > 0.0 ? w[t] / hn : 0.0;
}

// Cycle end: y = R^{-1} g (R the rotated Hessenberg, jend = s->j columns).
__global__ void k_hess_solve(DevScal* s) {
    if (threadIdx.x != 0) return;
    const int jend = s->j;
    for (int i = jend - 1; i >= 0; i--) {
        double v = s->g[i];
        for (int k = i + 1; k < jend; k++) v -= s->H[k * (MAXM + 1) + i] * s->y[k];
        s->y[i] = v / s->H[i * (MAXM + 1) + i];
    }
}

// x += Z y
__global__ void k_update_x(int n, const double* __restrict__ Z, int64_t ld, double* __restrict__ x, DevScal* s) {
    __shared__ double yc[MAXM];
    const int jend = *(volatile int*)&s->j;
    for (int i = threadIdx.x; i < jend; i += blockDim.x) yc[i] = ((volatile double*)s->y)[i];
    __syncthreads();
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t t = tid; t < n; t += stride) {
        double v = x[t];
        for (int k = 0; k < jend; k++) v += yc[k] * Z[(int64_t)k * ld + t];
        x[t] = v;
    }
}

}  // namespace kkt
