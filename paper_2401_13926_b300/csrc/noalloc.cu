// kkt_lu_solve_noalloc: the triangular solve x = Q U^{-1} L^{-1} P b for
// callers that must not allocate device memory.
//
// Some callers cannot call cudaMalloc at all: code that runs inside an
// application whose device memory is owned by its own arena allocator and
// that forbids outside allocations, or latency-critical loops (for example
// a controller that solves one KKT system per control period) where
// cudaMalloc/cudaFree may synchronise the device and stall the loop.  This
// entry point takes the factors, b and x from the caller and keeps its
// working memory -- the two intermediate vectors (each entry doubles as its
// row's completion flag: it holds SENTINEL until the row is solved) and the
// row tickets -- in one file-scope device array of fixed size that the
// library image carries.  Every GPU that loads the library holds that array
// (KKT_NOALLOC_SCRATCH_BYTES) until the process exits.
//
// The kernels take rows from an atomic ticket in dependency order and
// evaluate each row with the row arithmetic of the context's solves
// (trsv_row.cuh): the same tiers, the same summation order and the same
// correctly rounded pivot reciprocal, so on the same factors the two entry
// points return the same bits.  Every wait on a value another warp
// produces is bounded.
#include <cuda_runtime.h>

#include <cstddef>
#include <cstdint>
#include <mutex>

#include "kkt.h"
#include "trsv_row.cuh"

namespace {

struct NoallocHeader {
    unsigned ticket_l, ticket_u;
    int err, abort;
};

constexpr int64_t kMaxN = KKT_NOALLOC_MAX_N;
constexpr size_t kHeaderBytes = 256;
constexpr size_t kScratchBytes = kHeaderBytes + (size_t)kMaxN * 2 * sizeof(double);
static_assert(kScratchBytes == KKT_NOALLOC_SCRATCH_BYTES, "header and implementation disagree on the size");

// The scratch.  Host code must never pass `g_noalloc_scratch` itself to a
// kernel: in host code it names a host-side stand-in, not device memory.
// Its device address comes from cudaGetSymbolAddress (scratch_on_device).
// Layout: the header (tickets and error words) in the first 256 bytes, then
// y[kMaxN] and xp[kMaxN] (doubles).
static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

struct Scratch {
    NoallocHeader* h;
    double* y;
    double* xp;
};

__host__ __device__ inline Scratch carve(unsigned char* base) {
    Scratch s;
    s.h = reinterpret_cast<NoallocHeader*>(base);
    s.y = reinterpret_cast<double*>(base + kHeaderBytes);
    s.xp = s.y + kMaxN;
    return s;
}

// Calls share the scratch and find the previous call's contents there:
// re-arm y and xp of rows [0, n) (a value not computed yet holds
// SENTINEL), the tickets and the error words.
__global__ void k_na_clear(unsigned char* base, int n) {
    Scratch s = carve(base);
    const int64_t tid = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int64_t stride = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = tid; i < n; i += stride) {
        s.y[i] = kkt::sentinel();
        s.xp[i] = kkt::sentinel();
    }
    if (tid == 0) {
        s.h->ticket_l = 0u;
        s.h->ticket_u = 0u;
        s.h->err = 0;
        s.h->abort = 0;
    }
}

struct NaSrc {
    static constexpr int kPollNs = 20;
    const int32_t* Fj;
    const double* x;
    __device__ const volatile double* operator()(int64_t p) const { return x + __ldg(&Fj[p]); }
};
struct NaGiveUp {
    const int* abort;
    __device__ bool operator()() const { return *(volatile const int*)abort != 0; }
};

__device__ void na_fail(NoallocHeader* h) {
    atomicCAS(&h->err, 0, KKT_ERR_TIMEOUT);
    atomicExch(&h->abort, 1);
}

// Rows in index order from an atomic ticket; each row evaluated exactly as
// the context's solves evaluate it (kkt::trsv_row).
__global__ void k_na_lsolve(unsigned char* base, int n, const int64_t* __restrict__ Fp,
                            const int32_t* __restrict__ Fj, const int64_t* __restrict__ Fdiag,
                            const double* __restrict__ Fx, const int32_t* __restrict__ P,
                            const double* __restrict__ b, long long limit) {
    Scratch s = carve(base);
    const int lane = threadIdx.x & 31;
    const NaGiveUp gu{&s.h->abort};
    for (;;) {
        int row = 0;
        if (lane == 0) row = (int)atomicAdd(&s.h->ticket_l, 1u);
        row = __shfl_sync(0xffffffffu, row, 0);
        if (row >= n) return;
        const double r0 = kkt::rhs_value<double>(b[P[row]]);
        double val;
        if (!kkt::trsv_row<true>(Fp[row], Fdiag[row], Fx, NaSrc{Fj, s.y}, r0, 1.0, limit, gu, &val)) {
            if (lane == 0) na_fail(s.h);
            return;
        }
        if (lane == 0) *(volatile double*)&s.y[row] = val;
    }
}

__global__ void k_na_usolve(unsigned char* base, int n, const int64_t* __restrict__ Fp,
                            const int32_t* __restrict__ Fj, const int64_t* __restrict__ Fdiag,
                            const double* __restrict__ Fx, const int32_t* __restrict__ Q,
                            double* __restrict__ x, long long limit) {
    Scratch s = carve(base);
    const int lane = threadIdx.x & 31;
    const NaGiveUp gu{&s.h->abort};
    for (;;) {
        int t = 0;
        if (lane == 0) t = (int)atomicAdd(&s.h->ticket_u, 1u);
        t = __shfl_sync(0xffffffffu, t, 0);
        if (t >= n) return;
        const int row = n - 1 - t;
        const int64_t d = Fdiag[row];
        const double r0 = __ldcg(&s.y[row]);
        const double rinv = __drcp_rn(Fx[d]);
        double val;
        if (!kkt::trsv_row<false>(d + 1, Fp[row + 1], Fx, NaSrc{Fj, s.xp}, r0, rinv, limit, gu, &val)) {
            if (lane == 0) na_fail(s.h);
            return;
        }
        if (lane == 0) {
            *(volatile double*)&s.xp[row] = val;
            x[Q[row]] = val;
        }
    }
}

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char* g_dev_ptr[kMaxDevices] = {nullptr};
int g_blocks[kMaxDevices] = {0};

// Device address of the scratch on the current device, looked up once per
// device (with that device current) and cached.
int scratch_on_device(int dev, unsigned char** out, int* blocks) {
    if (dev < 0 || dev >= kMaxDevices) return KKT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(g_mu);
    if (!g_dev_ptr[dev]) {
        void* p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return KKT_ERR_CUDA;
        int sms = 0, per_sm = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return KKT_ERR_CUDA;
        if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_na_usolve, 256, 0) != cudaSuccess)
            return KKT_ERR_CUDA;
        g_dev_ptr[dev] = (unsigned char*)p;
        g_blocks[dev] = sms * (per_sm > 0 ? per_sm : 1);
    }
    *out = g_dev_ptr[dev];
    *blocks = g_blocks[dev];
    return KKT_OK;
}

}  // namespace

extern "C" int kkt_lu_solve_noalloc(int32_t n, const int64_t* Fp, const int32_t* Fj, const int64_t* Fdiag,
                                    const double* Fx, const int32_t* P, const int32_t* Q, const double* b,
                                    double* x, void* stream) {
    if (n < 1 || n > kMaxN) return KKT_ERR_INVALID;   // n beyond KKT_NOALLOC_MAX_N is rejected
    if (!Fp || !Fj || !Fdiag || !Fx || !P || !Q || !b || !x) return KKT_ERR_INVALID;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return KKT_ERR_CUDA;
    unsigned char* base = nullptr;
    int blocks = 0;
    int rc = scratch_on_device(dev, &base, &blocks);
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    const long long limit = 1ll << 25;
    const int need = (n + 7) / 8;   // 8 warps per 256-thread block
    const int g = blocks < need ? blocks : need;
    k_na_clear<<<(n + 255) / 256, 256, 0, st>>>(base, n);
    k_na_lsolve<<<g, 256, 0, st>>>(base, n, Fp, Fj, Fdiag, Fx, P, b, limit);
    k_na_usolve<<<g, 256, 0, st>>>(base, n, Fp, Fj, Fdiag, Fx, Q, x, limit);
    if (cudaGetLastError() != cudaSuccess) return KKT_ERR_CUDA;
    int err = 0;
    if (cudaMemcpyAsync(&err, base + offsetof(NoallocHeader, err), sizeof(int), cudaMemcpyDeviceToHost, st) !=
        cudaSuccess)
        return KKT_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return KKT_ERR_CUDA;
    return err;
}
