// Equilibration kernels of the mixed-precision path (kkt_opts.equilibrate).
#pragma once
#include <cstdint>
#include <cuda_runtime.h>

namespace kkt {

// ---- equilibration of K for the FP32 factors (mixed precision, optional):
// R K C with R, C diagonal powers of two, so every scaled value is exact.
// r_i = 2^(1-E) where max_j |a_ij| = f 2^E, f in [0.5, 1) (the row's largest
// scaled entry lies in [1, 2)); c_j the same for max_i |a_ij r_i|.  A zero
// or non-finite maximum gives 1.
__device__ __forceinline__ double pow2_scale(double m) {
    if (!(m > 0.0) || !isfinite(m)) return 1.0;
    int e = 0;
    frexp(m, &e);
    return ldexp(1.0, 1 - e);
}

// r (one warp per row) and the column maxima cleared
__global__ void k_eq_rows(int n, const int32_t* __restrict__ Arp, const double* __restrict__ Ax, double* r,
                          unsigned long long* colmax) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += stride) colmax[i] = 0ull;
    const int lane = threadIdx.x & 31;
    for (int64_t i = tid >> 5; i < n; i += stride >> 5) {
        double m = 0.0;
        for (int64_t e = Arp[i] + lane; e < Arp[i + 1]; e += 32) m = fmax(m, fabs(Ax[e]));
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) m = fmax(m, __shfl_xor_sync(0xffffffffu, m, o));
        if (lane == 0) r[i] = pow2_scale(m);
    }
}

// max_i |a_ij r_i| per column (non-negative doubles order like their bits)
__global__ void k_eq_cols(int n, const int32_t* __restrict__ Arp, const int32_t* __restrict__ Aci,
                          const double* __restrict__ Ax, const double* __restrict__ r, unsigned long long* colmax) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    const int lane = threadIdx.x & 31;
    for (int64_t i = tid >> 5; i < n; i += stride >> 5)
        for (int64_t e = Arp[i] + lane; e < Arp[i + 1]; e += 32)
            atomicMax(&colmax[Aci[e]], (unsigned long long)__double_as_longlong(fabs(Ax[e]) * r[i]));
}

// c, and the scaled values a_ij r_i c_j in the caller's order (vals[asrc[e]])
__global__ void k_eq_values(int n, const int32_t* __restrict__ Arp, const int32_t* __restrict__ Aci,
                            const double* __restrict__ Ax, const int64_t* __restrict__ asrc,
                            const double* __restrict__ r, const unsigned long long* __restrict__ colmax,
                            double* cs, double* vals) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t j = tid; j < n; j += stride) cs[j] = pow2_scale(__longlong_as_double((long long)colmax[j]));
    const int lane = threadIdx.x & 31;
    for (int64_t i = tid >> 5; i < n; i += stride >> 5)
        for (int64_t e = Arp[i] + lane; e < Arp[i + 1]; e += 32) {
            const double cj = pow2_scale(__longlong_as_double((long long)colmax[Aci[e]]));
            vals[asrc ? asrc[e] : e] = Ax[e] * r[i] * cj;
        }
}

// out_i = s_i v_i (out may be v)
__global__ void k_scale_vec(int n, const double* __restrict__ sc, const double* v, double* out) {
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += stride) out[i] = sc[i] * v[i];
}

}  // namespace kkt
