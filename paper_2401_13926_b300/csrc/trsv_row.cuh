// The arithmetic of one row of a sparse triangular solve, shared by every
// schedule (cluster, whole-GPU sync-free, single-block chain, and the
// allocation-free entry point) so that all of them produce the same bits.
//
//   L row i:  y_i = r0 - sum_k L_ik y_k            (unit diagonal)
//   U row i:  x_i = (r0 - sum_j U_ij x_j) * (1/U_ii)
//
// FP64 on B300 is scarce in a way that shapes this code: a dependent FP64
// operation takes about 64 cycles, and every FP64 warp instruction holds
// the SM's FP64 pipe for about 20 cycles however many lanes are active
// (measured: 0.05 warp instructions per SM-cycle with 1, 8, 16 or 32 active
// lanes), so the cost of a row is its count of FP64 warp instructions, and
// a fold by one lane costs as much as a 32-lane FMA.  A row therefore
// splits its entries in up to three tiers by how recently their
// dependencies finish: the EARLY ones are summed lane-parallel; the MIDDLE
// ones (U only) go one per lane, each multiplied into its lane's early sum
// as it arrives, and one warp reduction then sums both tiers; the LATE ones
// -- the few most recent -- are folded by lane 0 in one fused multiply-add
// each, in a fixed order.  Only that last FMA (and, for U, one multiply by
// the pivot's reciprocal) sits on the dependency chain when the
// dependencies arrive in order.  The tiers are fixed by the row's
// structure, so the result does not depend on timing.
//
// Values are read through `Src`, which maps an entry p to the address of
// its operand (shared, distributed shared or global memory, all accessed as
// volatile) and names the sleep between polls (Src::kPollNs); an operand
// that is not computed yet holds SENTINEL.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kkt {

constexpr unsigned long long SENTINEL_BITS = 0x7ff4dead5ca1ab1eull;
constexpr unsigned SENTINEL_BITS_F32 = 0x7fa5ca1eu;   // the FP32 (mixed precision) counterpart
// Late and middle entries per row, tuned per sweep.  L: 2 late, no middle
// tier (its kernel sits at the register cap).  U: 3 late and a middle tier
// of 24 (swept late 1..6, middle 16..30 on kkt2000, checked on kkt200 and
// kkt10000): U rows are longer and take more of their dependencies
// recently; each late entry costs a whole FP64 warp instruction.
constexpr int NLATE_L = 2;
constexpr int NMID_L = 0;
constexpr int NLATE_U = 3;
constexpr int NMID_U = 24;
constexpr int ROW_BATCH = 4;    // early entries per lane with loads in flight together

__device__ __forceinline__ double sentinel() { return __longlong_as_double((long long)SENTINEL_BITS); }
__device__ __forceinline__ bool is_sentinel(double v) {
    return (unsigned long long)__double_as_longlong(v) == SENTINEL_BITS;
}
__device__ __forceinline__ bool is_sentinel(float v) { return __float_as_uint(v) == SENTINEL_BITS_F32; }

template <typename T> __device__ __forceinline__ T quiet_nan();
template <> __device__ __forceinline__ double quiet_nan<double>() { return __longlong_as_double(0x7ff8000000000000ll); }
template <> __device__ __forceinline__ float quiet_nan<float>() { return __int_as_float(0x7fc00000); }

// SENTINEL of the value type T (double for FP64 factors, float for FP32)
template <typename T> __device__ __forceinline__ T sentinel_of();
template <> __device__ __forceinline__ double sentinel_of<double>() { return sentinel(); }
template <> __device__ __forceinline__ float sentinel_of<float>() { return __uint_as_float(SENTINEL_BITS_F32); }

// A right-hand-side entry as the forward sweep's first operand.  A value
// with SENTINEL's bits (a NaN payload a caller could pass in b) would read
// as "not computed yet" to every row that depends on it, so it enters as
// the canonical quiet NaN instead and propagates like any other NaN.
template <typename T>
__device__ __forceinline__ T rhs_value(double b) {
    const T r = (T)b;
    return is_sentinel(r) ? quiet_nan<T>() : r;
}

// correctly rounded reciprocal (same bits as 1/x)
__device__ __forceinline__ double rcp_rn(double x) { return __drcp_rn(x); }
__device__ __forceinline__ float rcp_rn(float x) { return __frcp_rn(x); }

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
    return v;
}

// Spin until *p is not SENTINEL.  `give_up()` is polled every 256 spins;
// after `limit` spins the wait fails.  Returns false on failure.  POLL_NS:
// sleep between polls -- 0 for operands in shared or distributed shared
// memory (a tight spin measured ~10% faster sweeps), 20 ns for operands in
// global memory (many warps polling L2).
template <int POLL_NS, typename T, class GiveUp>
__device__ __forceinline__ bool spin_value(const volatile T* p, T* v, long long limit, GiveUp give_up) {
    T x = *v;
    for (long long it = 0; is_sentinel(x); it++) {
        if ((it & 255) == 255 && give_up()) return false;
        if (it >= limit) return false;
        if (POLL_NS > 0) __nanosleep(POLL_NS);
        x = *p;
    }
    *v = x;
    return true;
}

// One row over entries [lo, hi) of the factor row (columns ascending).
// LOWER: the late entries are the last NLATE (NLATE_L) (largest columns, the most
// recent rows of the forward sweep); folded in ascending column order.
// !LOWER: the late entries are the first NLATE (NLATE_U; smallest columns > i, the
// most recent rows of the backward sweep); folded in descending order.
// Returns the row's value in lane 0 (other lanes: unspecified) or false in
// every lane if a wait failed.
// T is the value type of the factors and of the solve (double, or float in
// mixed precision); the arithmetic is the same in both.
// The factor values of the row come from `vals(p)`; trsv_row below reads
// them through the read-only cache from a factor array no kernel of the
// sweep writes.
// BATCH: early entries per lane whose loads are in flight together; it
// changes no sum (each lane accumulates its entries in the same order), so
// every BATCH gives the same bits -- a smaller one needs fewer registers.
template <bool LOWER, typename T, class Vals, class Src, class GiveUp, int BATCH = ROW_BATCH>
__device__ __forceinline__ bool trsv_row_v(int64_t lo, int64_t hi, Vals vals, Src src,
                                           T r0, T rinv, long long limit, GiveUp give_up, T* out) {
    constexpr int NLATE = LOWER ? NLATE_L : NLATE_U;
    constexpr int NMID = LOWER ? NMID_L : NMID_U;
    const int lane = threadIdx.x & 31;
    const int64_t len = hi - lo;
    const int nl = (int)(len < NLATE ? len : NLATE);
    const int nm = NMID == 0 ? 0 : (int)((len - nl) < NMID ? (len - nl) : NMID);
    // L: [lo .. early .. | middle | late .. hi); U: [lo late | middle | early .. hi)
    const int64_t elo = LOWER ? lo : lo + nl + nm;
    const int64_t ehi = LOWER ? hi - nl - nm : hi;
    // the middle tier's loads start first: entry `lane` of the tier
    T ma = T(0), mv = T(0);
    const volatile T* ms = nullptr;
    if constexpr (NMID > 0) {
        if (lane < nm) {
            const int64_t p = LOWER ? hi - nl - nm + lane : lo + nl + lane;
            ma = vals(p);
            ms = src(p);
            mv = *ms;
        }
    }
    // lane 0 starts the loads of the late entries first
    T la[NLATE], lv[NLATE];
    const volatile T* ls[NLATE];
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NLATE; j++) {
            if (j < nl) {
                const int64_t p = LOWER ? hi - nl + j : lo + nl - 1 - j;   // completion order
                la[j] = vals(p);
                ls[j] = src(p);
                lv[j] = *ls[j];
            }
        }
    }
    int ok = 1;
    T acc = T(0);
    for (int64_t base = elo + lane; base < ehi && ok; base += 32 * BATCH) {
        T a[BATCH], v[BATCH];
        const volatile T* s[BATCH];
#pragma unroll
        for (int u = 0; u < BATCH; u++) {
            const int64_t p = base + 32 * u;
            if (p < ehi) { a[u] = vals(p); s[u] = src(p); }
        }
#pragma unroll
        for (int u = 0; u < BATCH; u++)
            if (base + 32 * u < ehi) v[u] = *s[u];
#pragma unroll
        for (int u = 0; u < BATCH; u++) {
            if (base + 32 * u >= ehi) continue;
            if (!spin_value<Src::kPollNs>(s[u], &v[u], limit, give_up)) { ok = 0; break; }
            acc = fma(a[u], v[u], acc);
        }
    }
    // the middle tier's entry joins its lane's early sum
    if constexpr (NMID > 0) {
        if (lane < nm && ok) {
            if (!spin_value<Src::kPollNs>(ms, &mv, limit, give_up)) ok = 0;
            else acc = fma(ma, mv, acc);
        }
    }
    if (!__all_sync(0xffffffffu, ok)) return false;
    // lanes past the m-th early (or middle) entry hold exact zeros: reduce
    // over the first 2^ceil(log2 m) lanes only (same sum, fewer FP64 steps)
    const int64_t m = (ehi - elo) > nm ? (ehi - elo) : nm;
    T r = r0;
    if (m > 0) {
        const int span = m >= 32 ? 32 : (int)m;
        int o = 1;
        while (o < span) o <<= 1;
        for (o >>= 1; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
        r = r0 - acc;
    }
    if (lane == 0) {
#pragma unroll
        for (int j = 0; j < NLATE; j++) {
            if (j < nl && ok) {
                if (!spin_value<Src::kPollNs>(ls[j], &lv[j], limit, give_up)) { ok = 0; break; }
                r = fma(-la[j], lv[j], r);
            }
        }
        if (!LOWER) r *= rinv;
    }
    if (!__shfl_sync(0xffffffffu, ok, 0)) return false;
    *out = r;
    return true;
}

template <typename T>
struct LdgVals {   // factor values through the read-only cache
    const T* Fx;
    __device__ T operator()(int64_t p) const { return __ldg(&Fx[p]); }
};

template <bool LOWER, typename T, class Src, class GiveUp>
__device__ __forceinline__ bool trsv_row(int64_t lo, int64_t hi, const T* __restrict__ Fx, Src src,
                                         T r0, T rinv, long long limit, GiveUp give_up, T* out) {
    return trsv_row_v<LOWER>(lo, hi, LdgVals<T>{Fx}, src, r0, rinv, limit, give_up, out);
}

}  // namespace kkt
