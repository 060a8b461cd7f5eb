// C ABI of the GPU-resident KKT solver: context, one-time analysis, and the
// host sequencing of the device kernels in kernels.cuh.  Declarations and
// the contract of every entry point are in include/kkt.h.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <climits>
#include <numeric>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <string>
#include <thread>
#include <type_traits>
#include <vector>

#include "analysis.h"
#include "kernels.cuh"
#include "equilibrate.cuh"
#include "kkt.h"

using kkt::DevScal;

struct kkt_ctx {
    kkt_opts o{};
    int dev = 0;
    cudaStream_t stream = nullptr;
    bool own_stream = false;
    int num_sms = 0;
    // host analysis
    kkt::Csr A;
    std::vector<int32_t> P, Q;
    kkt::Layout lay;
    bool analyzed = false, factored = false;
    int64_t nnz_a = 0;
    // device memory (all made in kkt_analyze)
    std::vector<void*> allocs;
    int64_t dev_bytes = 0;
    int64_t *d_Fp = nullptr, *d_Fdiag = nullptr, *d_fsrc = nullptr, *d_asrc = nullptr;
    int32_t *d_Fj = nullptr, *d_Arp = nullptr, *d_Aci = nullptr, *d_P = nullptr, *d_Q = nullptr;
    // factor values and pivot reciprocals in the factor type: double, or
    // float with precision = KKT_PRECISION_MIXED
    void* d_Fx = nullptr;
    void* d_rinv = nullptr;     // 1/u_ii of every row; each row publishes it last
    // mixed precision with the FP64 fallback (kkt_opts.mixed_fallback): FP64
    // factors of the same layout, used after a fallback until the next
    // refactorization
    void* d_Fx64 = nullptr;
    void* d_rinv64 = nullptr;
    bool fallback_on = false;   // mixed and mixed_fallback > 0
    // mixed precision with kkt_opts.equilibrate: the FP32 factors are of
    // R K C (powers of two); the preconditioner applies C (RKC)^{-1} R
    bool eq_on = false;
    double* d_eq_r = nullptr;               // R (by original row)
    double* d_eq_c = nullptr;               // C (by original column)
    unsigned long long* d_eq_colmax = nullptr;
    double* d_eq_vals = nullptr;            // R K C in the caller's value order
    double* d_eq_tmp = nullptr;             // R times the right-hand side of a sweep pair
    bool fp64_active = false;   // the factors in use are the FP64 ones
    bool vec_f32 = false;       // y and xp currently hold FP32 values (their SENTINEL type)
    int last_fallback = 0;
    int64_t fallbacks = 0;
    double *d_Ax = nullptr, *d_vals = nullptr;
    bool mixed = false;
    unsigned long long* solve_trace = nullptr;   // kkt_trace_solve only: 2n publish stamps
    // CUDA graphs (kkt_opts.graphs): capture streams, the refactorization and
    // solve graphs, and kernels per replayed part (for the launch count)
    cudaStream_t cap[3] = {nullptr, nullptr, nullptr};
    bool capturing = false;
    cudaGraph_t g_ref = nullptr, g_solve = nullptr;
    cudaGraphExec_t gx_ref = nullptr, gx_solve = nullptr;
    double g_solve_tol = 0.0;
    int64_t gl_ref = 0, gl_pro = 0, gl_body = 0, gl_step = 0;
    int32_t repivots = 0;                         // kkt_repivot calls that succeeded in analysis
    bool y_fused = false;                         // the last refactorization also computed y = L^{-1} P b
    double *d_b = nullptr, *d_x = nullptr, *d_y = nullptr, *d_xp = nullptr, *d_r = nullptr, *d_w = nullptr;
    double *d_V = nullptr, *d_Z = nullptr, *d_part = nullptr;
    unsigned* d_done_f = nullptr;
    // triangular-solve schedule: rows in DAG-level order (listL, listU),
    // Fpos[p] = list position of entry p's dependency; the L chain is the
    // last nLc positions of listL, the U chain the first nUc of listU
    int32_t *d_listL = nullptr, *d_listU = nullptr, *d_Fpos = nullptr;
    int nLc = 0, nUc = 0;
    int cluster = 0;            // blocks of the cluster solve (0: use the global schedule)
    size_t cluster_smem = 0;
    // refactorization kernel (k_refactor_rows): rows placed one per warp,
    // one per block in shared memory, or one per block with values in
    // global memory; work items in dispatch order
    int ref_threads = 256, ref_shape = 0, ref_blocks = 0, nitems = 0, smem_optin = 0;
    size_t ref_smem = 0;
    int32_t rows_warp = 0, rows_block = 0, rows_global = 0, rows_team = 0;
    int32_t* d_order = nullptr;   // rows in dispatch order
    kkt::RefItem* d_items = nullptr;
    // rows in global memory: step descriptors and value scratch (remade
    // whenever the placement changes)
    std::vector<void*> row_allocs;
    uint32_t *d_gdk = nullptr, *d_gcnt = nullptr;
    int64_t *d_gsdoff = nullptr, *d_gwoff = nullptr;
    void* d_gw = nullptr;
    DevScal* d_s = nullptr;
    DevScal* h_s = nullptr;   // pinned mirror
    int64_t ld = 0;
    int m = 20;
    int persist_blocks = 0;
    // results
    std::string detail;
    int nboost = 0, last_iters = 0, last_cycles = 0;
    double last_nrbe = 0, last_rnorm0 = 0, norm_a = 0, analyze_ms = 0;
    int64_t launches = 0, h2d = 0, d2h = 0;
    // phase timing (opts.timing): event pairs recorded on the stream and
    // drained at the next host synchronisation
    std::vector<cudaEvent_t> ev_pool;
    std::vector<int> ev_phase;     // phase of each pending pair
    size_t ev_used = 0;
    double phase_ms[KKT_NUM_PHASES] = {0};
    int64_t phase_n[KKT_NUM_PHASES] = {0};
};

namespace {

// The factors in use: FP32 in mixed precision until a fallback, FP64
// otherwise (the context's only factors, or the fallback's).
bool use_f32(const kkt_ctx* c) { return c->mixed && !c->fp64_active; }
template <typename T> T* fx_of(kkt_ctx* c);
template <> float* fx_of<float>(kkt_ctx* c) { return (float*)c->d_Fx; }
template <> double* fx_of<double>(kkt_ctx* c) { return (double*)(c->mixed ? c->d_Fx64 : c->d_Fx); }
template <typename T> T* rinv_of(kkt_ctx* c);
template <> float* rinv_of<float>(kkt_ctx* c) { return (float*)c->d_rinv; }
template <> double* rinv_of<double>(kkt_ctx* c) { return (double*)(c->mixed ? c->d_rinv64 : c->d_rinv); }
// bytes of a factor value as laid out for the refactorization and the
// cluster solve (a context that may fall back to FP64 is laid out for FP64)
size_t layout_vsize(const kkt_ctx* c) { return (c->mixed && !c->fallback_on) ? sizeof(float) : sizeof(double); }

constexpr int PERSIST_THREADS = 256;
constexpr int CHAIN_THREADS = 1024;
constexpr size_t TAIL_SMEM_MAX = 200 * 1024;   // shared memory of a cluster-solve block
// blocks up to REF_SMEM_THREE fit three an SM, up to REF_SMEM_WIDE two (each
// block also holds 1 KB reserved and its static shared memory, and an SM
// 228 KB); larger blocks run 512 threads, one an SM
constexpr size_t REF_SMEM_WIDE = 112 * 1024;
constexpr size_t REF_SMEM_THREE = 74 * 1024;
// The default limit of a warp row's multiply-adds (measured: kkt2000's
// refactorization 8.7 ms with no limit, 5.3 ms with 1,024, 5.6 with 4,096;
// kkt10000 41-43 ms between 1k and 16k; kkt70000, 512-thread blocks whose
// halves take the rows warps do not, 684 ms with 4,096, 689 with 16,384,
// 727 with 65,536, 771 with 262,144)
constexpr int64_t DEFAULT_WARP_ROW_UPDATES = 2048;        // 256-thread blocks
constexpr int64_t DEFAULT_WARP_ROW_UPDATES_WIDE = 4096;   // 512-thread blocks
constexpr int CHAIN_MAX = 12288;       // rows of a chain (8 bytes of shared memory each)
constexpr int CHAIN_WIDTH = 32;        // a level belongs to the chain if it has at most this many rows

// Rows in DAG-level order (ties by row index) and each row's position.
void level_order(const std::vector<int32_t>& lev, std::vector<int32_t>* list, std::vector<int32_t>* pos) {
    const int32_t n = (int32_t)lev.size();
    list->resize(n);
    std::iota(list->begin(), list->end(), 0);
    std::stable_sort(list->begin(), list->end(), [&](int32_t a, int32_t b) { return lev[a] < lev[b]; });
    pos->assign(n, 0);
    for (int32_t t = 0; t < n; t++) (*pos)[(*list)[t]] = t;
}

// Rows in the narrow end of a DAG: L -- the highest levels whose widths
// are all <= CHAIN_WIDTH; U -- the lowest such levels; at most cap rows.
int chain_rows(const std::vector<int32_t>& lev, bool lower, int cap) {
    int32_t nl = 0;
    for (int32_t v : lev) nl = std::max(nl, v + 1);
    std::vector<int64_t> w(nl, 0);
    for (int32_t v : lev) w[v]++;
    int64_t count = 0;
    if (lower) {
        for (int32_t l = nl - 1; l >= 0 && w[l] <= CHAIN_WIDTH && count + w[l] <= cap; l--) count += w[l];
    } else {
        for (int32_t l = 0; l < nl && w[l] <= CHAIN_WIDTH && count + w[l] <= cap; l++) count += w[l];
    }
    return (int)count;
}

constexpr long long DEFAULT_SPIN = 1ll << 25;

int cuda_fail(kkt_ctx* c, cudaError_t e, const char* what) {
    if (c) c->detail = std::string(what) + ": " + cudaGetErrorString(e);
    return e == cudaErrorMemoryAllocation ? KKT_ERR_OOM : KKT_ERR_CUDA;
}
#define CK_BT(call)                                                                  \
    do {                                                                             \
        cudaError_t e_ = (call);                                                     \
        if (e_ != cudaSuccess) return e_ == cudaErrorMemoryAllocation ? KKT_ERR_OOM : KKT_ERR_CUDA; \
    } while (0)
#define CK(call)                                             \
    do {                                                     \
        cudaError_t e_ = (call);                             \
        if (e_ != cudaSuccess) return cuda_fail(c, e_, #call); \
    } while (0)

void drop_graph(cudaGraphExec_t* ex, cudaGraph_t* g) {
    if (*ex) { cudaGraphExecDestroy(*ex); *ex = nullptr; }
    if (*g) { cudaGraphDestroy(*g); *g = nullptr; }
}

thread_local const char* g_capture_where = "";   // the call that failed while building a graph

// Captures `fill` (launches on c->stream, pointed at capture stream `level`
// meanwhile) as a standalone graph.
template <class F>
cudaError_t capture_graph(kkt_ctx* c, int level, cudaGraph_t* out, F fill) {
    cudaStream_t st = c->cap[level];
    cudaStream_t saved = c->stream;
    cudaError_t e = cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) { g_capture_where = "cudaStreamBeginCapture"; return e; }
    c->stream = st;
    fill();
    cudaError_t inner = cudaGetLastError();
    c->stream = saved;
    e = cudaStreamEndCapture(st, out);
    if (inner != cudaSuccess) { g_capture_where = "a launch in the capture"; return inner; }
    if (e != cudaSuccess) g_capture_where = "cudaStreamEndCapture";
    return e;
}

// Adds `child` (copied, then destroyed) to g after `dep` (nullptr: none).
cudaError_t add_child(cudaGraph_t g, const cudaGraphNode_t* dep, cudaGraph_t child, cudaGraphNode_t* node) {
    cudaError_t e = cudaGraphAddChildGraphNode(node, g, dep, dep ? 1 : 0, child);
    cudaGraphDestroy(child);
    if (e != cudaSuccess) g_capture_where = "cudaGraphAddChildGraphNode";
    return e;
}

// Adds a conditional node (WHILE or IF on h) to g after `dep`; its body in *body.
cudaError_t add_conditional(cudaGraph_t g, const cudaGraphNode_t* dep, cudaGraphConditionalHandle h,
                            cudaGraphConditionalNodeType type, cudaGraphNode_t* node, cudaGraph_t* body) {
    cudaGraphNodeParams p = {};
    p.type = cudaGraphNodeTypeConditional;
    p.conditional.handle = h;
    p.conditional.type = type;
    p.conditional.size = 1;
    cudaError_t e = cudaGraphAddNode(node, g, dep, nullptr, dep ? 1 : 0, &p);
    if (e != cudaSuccess) { g_capture_where = "cudaGraphAddNode(conditional)"; return e; }
    *body = p.conditional.phGraph_out[0];
    return cudaSuccess;
}

void free_device(kkt_ctx* c) {
    drop_graph(&c->gx_ref, &c->g_ref);
    drop_graph(&c->gx_solve, &c->g_solve);
    for (cudaEvent_t e : c->ev_pool) cudaEventDestroy(e);
    c->ev_pool.clear();
    c->ev_used = 0;
    for (void* p : c->allocs) cudaFree(p);
    c->allocs.clear();
    for (void* p : c->row_allocs) cudaFree(p);
    c->row_allocs.clear();
    if (c->h_s) { cudaFreeHost(c->h_s); c->h_s = nullptr; }
    c->dev_bytes = 0;
    c->analyzed = c->factored = false;
}

template <class T>
int dalloc(kkt_ctx* c, T** p, size_t count) {
    size_t bytes = std::max<size_t>(count, 1) * sizeof(T);
    void* q = nullptr;
    cudaError_t e = cudaMalloc(&q, bytes);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMalloc");
    c->allocs.push_back(q);
    c->dev_bytes += (int64_t)bytes;
    *p = (T*)q;
    return KKT_OK;
}

template <class T>
int upload(kkt_ctx* c, T** p, const std::vector<T>& v) {
    int rc = dalloc(c, p, v.size());
    if (rc) return rc;
    if (!v.empty()) CK(cudaMemcpyAsync(*p, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice, c->stream));
    return KKT_OK;
}

void phase_drain(kkt_ctx* c);

int read_scalars(kkt_ctx* c) {
    CK(cudaMemcpyAsync(c->h_s, c->d_s, sizeof(DevScal), cudaMemcpyDeviceToHost, c->stream));
    c->d2h += (int64_t)sizeof(DevScal);
    CK(cudaStreamSynchronize(c->stream));
    phase_drain(c);
    return KKT_OK;
}

int device_error(kkt_ctx* c) {
    int e = c->h_s->err;
    if (e) {
        c->detail = std::string(kkt_strerror(e)) + " at row " + std::to_string(c->h_s->err_row);
        return e;
    }
    return KKT_OK;
}

constexpr size_t EV_PAIRS = 512;

// Phase timer: a start event now, the matching end event from the returned
// index after the launches of the phase.
int phase_begin(kkt_ctx* c, int phase) {
    if (!c->o.timing || c->ev_pool.empty() || c->capturing) return -1;
    if (c->ev_used >= EV_PAIRS) return -1;   // pool full until the next drain
    size_t i = c->ev_used++;
    c->ev_phase[i] = phase;
    cudaEventRecord(c->ev_pool[2 * i], c->stream);
    return (int)i;
}
void phase_end(kkt_ctx* c, int i) {
    if (i >= 0) cudaEventRecord(c->ev_pool[2 * i + 1], c->stream);
}
// Called after a stream synchronisation: all pending events are complete.
void phase_drain(kkt_ctx* c) {
    for (size_t i = 0; i < c->ev_used; i++) {
        float ms = 0.f;
        if (cudaEventElapsedTime(&ms, c->ev_pool[2 * i], c->ev_pool[2 * i + 1]) == cudaSuccess) {
            c->phase_ms[c->ev_phase[i]] += ms;
            c->phase_n[c->ev_phase[i]] += 1;
        }
    }
    c->ev_used = 0;
}

long long spin(const kkt_ctx* c) { return c->o.spin_limit > 0 ? (long long)c->o.spin_limit : DEFAULT_SPIN; }

int red_blocks(const kkt_ctx* c) {
    int64_t need = (c->A.n + kkt::RED_THREADS - 1) / kkt::RED_THREADS;
    return (int)std::max<int64_t>(1, std::min<int64_t>(kkt::RED_BLOCKS, need));
}


int grid_for(const kkt_ctx* c, int rows) {
    int64_t need = ((int64_t)rows + (PERSIST_THREADS / 32) - 1) / (PERSIST_THREADS / 32);
    return (int)std::max<int64_t>(1, std::min<int64_t>(c->persist_blocks, need));
}

// Cluster solve: one cluster of `blocks` blocks runs the whole solve.
template <bool LOWER, typename T, typename TIN, typename TOUT>
cudaError_t launch_cluster(kkt_ctx* c, const int32_t* perm, const TIN* rhs, TOUT* out) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(c->cluster, 1, 1);
    cfg.blockDim = dim3(kkt::CLUSTER_THREADS, 1, 1);
    cfg.dynamicSmemBytes = c->cluster_smem;
    cfg.stream = c->stream;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = c->cluster;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kkt::k_trsv_cluster<LOWER, T, TIN, TOUT>, c->A.n,
                              (const int32_t*)(LOWER ? c->d_listL : c->d_listU), (const int32_t*)c->d_Fpos,
                              (const int64_t*)c->d_Fp, (const int64_t*)c->d_Fdiag, (const T*)fx_of<T>(c),
                              (const T*)rinv_of<T>(c), perm, rhs, out, c->d_s, spin(c),
                              c->solve_trace ? c->solve_trace + (LOWER ? 0 : c->A.n) : nullptr);
}

// Pick the cluster (16 blocks, else 8) whose shared memory holds all n
// values and that the device can co-schedule; 0 if none.  16 blocks give
// the sweep twice the FP64 pipes of 8 (measured faster on kkt2000).
template <typename T>
void cluster_attributes(int C) {
    for (auto fn : {(const void*)kkt::k_trsv_cluster<true, T, double, T>,
                    (const void*)kkt::k_trsv_cluster<false, T, T, double>}) {
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)TAIL_SMEM_MAX);
        if (C > 8) cudaFuncSetAttribute(fn, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
    }
}

int pick_cluster(kkt_ctx* c) {
    const int n = c->A.n;
    const size_t vsize = layout_vsize(c);
    for (int C : {16, 8}) {
        if (c->o.cluster_blocks && C != c->o.cluster_blocks) continue;
        size_t per_block = (size_t)((n + 32 * C - 1) / (32 * C)) * 32 * vsize;
        if (per_block > TAIL_SMEM_MAX) continue;
        if (c->mixed) cluster_attributes<float>(C);
        if (vsize == sizeof(double)) cluster_attributes<double>(C);
        cudaLaunchConfig_t cfg = {};
        cfg.gridDim = dim3(C, 1, 1);
        cfg.blockDim = dim3(kkt::CLUSTER_THREADS, 1, 1);
        cfg.dynamicSmemBytes = per_block;
        cudaLaunchAttribute attr[1];
        attr[0].id = cudaLaunchAttributeClusterDimension;
        attr[0].val.clusterDim.x = C;
        attr[0].val.clusterDim.y = 1;
        attr[0].val.clusterDim.z = 1;
        cfg.attrs = attr;
        cfg.numAttrs = 1;
        int active = 0;
        const void* probe = vsize == sizeof(float) ? (const void*)kkt::k_trsv_cluster<true, float, double, float>
                                                   : (const void*)kkt::k_trsv_cluster<true, double, double, double>;
        if (cudaOccupancyMaxActiveClusters(&active, probe, &cfg) != cudaSuccess) {
            cudaGetLastError();
            continue;
        }
        if (active >= 1) { c->cluster = C; c->cluster_smem = per_block; return C; }
    }
    c->cluster = 0;
    return 0;
}

// x = Q U^{-1} L^{-1} P rhs (double in, double out; the sweeps in the
// factor type T): one cluster launch per triangle when the values fit in a
// cluster's shared memory, else L bulk, L chain, U chain, U bulk over the
// whole GPU.
template <typename T>
void lu_apply_t(kkt_ctx* c, const double* rhs, double* out) {
    T* y = (T*)c->d_y;
    T* xp = (T*)c->d_xp;
    const T* Fx = fx_of<T>(c);
    const T* rinv = rinv_of<T>(c);
    if (c->cluster) {
        int t = phase_begin(c, KKT_PHASE_LSOLVE);
        launch_cluster<true, T, double, T>(c, c->d_P, rhs, y);
        phase_end(c, t);
        t = phase_begin(c, KKT_PHASE_USOLVE);
        launch_cluster<false, T, T, double>(c, c->d_Q, y, out);
        phase_end(c, t);
        c->launches += 2;
        return;
    }
    const int n = c->A.n;
    const int nLb = n - c->nLc, nUb = n - c->nUc;
    kkt::k_trsv_prep<<<1, 1, 0, c->stream>>>(c->d_s);
    c->launches += 1;
    int t = phase_begin(c, KKT_PHASE_LSOLVE);
    if (nLb) {
        kkt::k_lsolve_bulk<T><<<grid_for(c, nLb), PERSIST_THREADS, 0, c->stream>>>(
            nLb, c->d_listL, c->d_Fp, c->d_Fj, c->d_Fdiag, Fx, c->d_P, rhs, y, xp, c->d_s, spin(c));
        c->launches += 1;
    }
    if (c->nLc) {
        kkt::k_lsolve_chain<T><<<1, CHAIN_THREADS, sizeof(T) * c->nLc, c->stream>>>(
            c->nLc, nLb, c->d_listL, c->d_Fpos, c->d_Fp, c->d_Fj, c->d_Fdiag, Fx, c->d_P, rhs, y, xp, c->d_s,
            spin(c));
        c->launches += 1;
    }
    phase_end(c, t);
    t = phase_begin(c, KKT_PHASE_USOLVE);
    if (c->nUc) {
        kkt::k_usolve_chain<T><<<1, CHAIN_THREADS, sizeof(T) * c->nUc, c->stream>>>(
            c->nUc, c->d_listU, c->d_Fpos, c->d_Fp, c->d_Fj, c->d_Fdiag, Fx, rinv, c->d_Q, y, xp, out,
            c->d_s, spin(c));
        c->launches += 1;
    }
    if (nUb) {
        kkt::k_usolve_bulk<T><<<grid_for(c, nUb), PERSIST_THREADS, 0, c->stream>>>(
            nUb, c->d_listU + c->nUc, c->d_Fp, c->d_Fj, c->d_Fdiag, Fx, rinv, c->d_Q, y, xp, out,
            c->d_s, spin(c));
        c->launches += 1;
    }
    phase_end(c, t);
}

void lu_apply(kkt_ctx* c, const double* rhs, double* out) {
    if (use_f32(c) && c->eq_on) {   // K^{-1} ~ C (R K C)^{-1} R
        const int n = c->A.n, g = 2 * c->num_sms;
        kkt::k_scale_vec<<<g, 256, 0, c->stream>>>(n, c->d_eq_r, rhs, c->d_eq_tmp);
        lu_apply_t<float>(c, c->d_eq_tmp, out);
        kkt::k_scale_vec<<<g, 256, 0, c->stream>>>(n, c->d_eq_c, out, out);
        c->launches += 2;
    } else if (use_f32(c)) {
        lu_apply_t<float>(c, rhs, out);
    } else {
        lu_apply_t<double>(c, rhs, out);
    }
}

// x = Q U^{-1} y with y already in the context (the fused forward sweep)
template <typename T>
void u_apply_t(kkt_ctx* c, double* out) {
    T* y = (T*)c->d_y;
    T* xp = (T*)c->d_xp;
    const T* Fx = fx_of<T>(c);
    const T* rinv = rinv_of<T>(c);
    int t = phase_begin(c, KKT_PHASE_USOLVE);
    if (c->cluster) {
        launch_cluster<false, T, T, double>(c, c->d_Q, y, out);
        c->launches += 1;
        phase_end(c, t);
        return;
    }
    const int n = c->A.n;
    const int nUb = n - c->nUc;
    kkt::k_trsv_prep<<<1, 1, 0, c->stream>>>(c->d_s);
    c->launches += 1;
    if (c->nUc) {
        kkt::k_usolve_chain<T><<<1, CHAIN_THREADS, sizeof(T) * c->nUc, c->stream>>>(
            c->nUc, c->d_listU, c->d_Fpos, c->d_Fp, c->d_Fj, c->d_Fdiag, Fx, rinv, c->d_Q, y, xp, out,
            c->d_s, spin(c));
        c->launches += 1;
    }
    if (nUb) {
        kkt::k_usolve_bulk<T><<<grid_for(c, nUb), PERSIST_THREADS, 0, c->stream>>>(
            nUb, c->d_listU + c->nUc, c->d_Fp, c->d_Fj, c->d_Fdiag, Fx, rinv, c->d_Q, y, xp, out,
            c->d_s, spin(c));
        c->launches += 1;
    }
    phase_end(c, t);
}

void u_apply(kkt_ctx* c, double* out) {
    if (use_f32(c)) u_apply_t<float>(c, out);
    else u_apply_t<double>(c, out);
}

void fill_y_sentinel(kkt_ctx* c) {
    if (use_f32(c)) kkt::k_fill_sentinel<float><<<64, 256, 0, c->stream>>>((float*)c->d_y, c->A.n);
    else kkt::k_fill_sentinel<double><<<64, 256, 0, c->stream>>>(c->d_y, c->A.n);
}

// y and xp hold SENTINEL of the factor type in use wherever a sweep has not
// written them; when that type changes (FP32 <-> the FP64 fallback) both
// are re-armed in the new type.
void arm_vectors(kkt_ctx* c) {
    if (c->vec_f32 == use_f32(c)) return;
    c->vec_f32 = use_f32(c);
    fill_y_sentinel(c);
    if (c->vec_f32) kkt::k_fill_sentinel<float><<<64, 256, 0, c->stream>>>((float*)c->d_xp, c->A.n);
    else kkt::k_fill_sentinel<double><<<64, 256, 0, c->stream>>>(c->d_xp, c->A.n);
    c->launches += 2;
}

// After a failed solve some values may still be live: re-arm the L-solve's
// vector so the next solve starts from sentinels everywhere.
void rearm(kkt_ctx* c) {
    fill_y_sentinel(c);
    c->launches += 1;
    cudaStreamSynchronize(c->stream);
}

int check_ctx(kkt_ctx* c, bool need_factors) {
    if (!c) return KKT_ERR_INVALID;
    if (!c->analyzed) { c->detail = "kkt_analyze has not run"; return KKT_ERR_STATE; }
    if (need_factors && !c->factored) { c->detail = "kkt_refactor has not succeeded"; return KKT_ERR_STATE; }
    cudaError_t e = cudaSetDevice(c->dev);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaSetDevice");
    return KKT_OK;
}

}  // namespace

extern "C" {

void kkt_default_opts(kkt_opts* o) {
    if (!o) return;
    std::memset(o, 0, sizeof(*o));
    o->restart = 20;
    o->max_cycles = 50;
    o->stop_mode = KKT_STOP_NRBE;
    o->precision = 0;
    o->refine_delta = 0.0;
    o->pivot_tol = 1e-3;
    o->boost_eps = 0.0;
    o->device = 0;
    o->create_stream = 1;
    o->stream = nullptr;
    o->spin_limit = 0;
    o->method = KKT_METHOD_FGMRES;
    o->ortho = KKT_ORTHO_CGS2;
    o->inner_tol = 1e-6;
    o->repivot = 0;
    o->graphs = 0;
    o->warp_rows = 1;
    o->row_order = 1;
    o->mixed_fallback = 2;
    o->stream_last = 1;
    o->team_rows = 1;
    o->equilibrate = 0;
}

const char* kkt_strerror(int code) {
    switch (code) {
        case KKT_OK: return "ok";
        case KKT_ERR_INVALID: return "invalid argument";
        case KKT_ERR_PATTERN: return "invalid or mismatched sparsity pattern";
        case KKT_ERR_OOM: return "out of memory";
        case KKT_ERR_ZERO_PIVOT: return "zero pivot";
        case KKT_ERR_NONFINITE: return "non-finite value";
        case KKT_ERR_NOT_CONVERGED: return "refinement did not converge";
        case KKT_ERR_TIMEOUT: return "bounded device wait timed out";
        case KKT_ERR_CUDA: return "CUDA error";
        case KKT_ERR_STATE: return "call out of order";
        default: return "unknown error";
    }
}

const char* kkt_last_error_detail(kkt_ctx* c) { return c ? c->detail.c_str() : ""; }

int kkt_create(kkt_ctx** out, const kkt_opts* o) {
    if (!out) return KKT_ERR_INVALID;
    *out = nullptr;
    kkt_ctx* c = new kkt_ctx();
    if (o) c->o = *o; else kkt_default_opts(&c->o);
    if (c->o.restart < 1 || c->o.restart > kkt::MAXM || c->o.max_cycles < 0 ||
        (c->o.precision != KKT_PRECISION_FP64 && c->o.precision != KKT_PRECISION_MIXED) ||
        (c->o.stop_mode != KKT_STOP_NRBE && c->o.stop_mode != KKT_STOP_RR) || c->o.pivot_tol <= 0 ||
        c->o.pivot_tol > 1 || c->o.boost_eps < 0 ||
        (c->o.trisolve != KKT_TRSV_AUTO && c->o.trisolve != KKT_TRSV_GLOBAL) || c->o.block_smem < 0 ||
        (c->o.cluster_blocks != 0 && c->o.cluster_blocks != 8 && c->o.cluster_blocks != 16) ||
        c->o.method < KKT_METHOD_FGMRES || c->o.method > KKT_METHOD_FGMRES_EE ||
        c->o.ortho < KKT_ORTHO_CGS2 || c->o.ortho > KKT_ORTHO_CGS1_PYTH ||
        !(c->o.inner_tol > 0.0 && c->o.inner_tol <= 1.0) || (c->o.repivot != 0 && c->o.repivot != 1) ||
        (c->o.graphs != 0 && c->o.graphs != 1) || (c->o.warp_rows != 0 && c->o.warp_rows != 1) ||
        (c->o.row_order < 0 || c->o.row_order > 2) || c->o.mixed_fallback < 0 ||
        (c->o.stream_last != 0 && c->o.stream_last != 1) || (c->o.team_rows != 0 && c->o.team_rows != 1) ||
        (c->o.equilibrate != 0 && c->o.equilibrate != 1) ||
        c->o.warp_row_updates < -1) {
        delete c;
        return KKT_ERR_INVALID;
    }
    c->dev = c->o.device;
    c->m = c->o.restart;
    cudaError_t e = cudaSetDevice(c->dev);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->dev);
    if (e == cudaSuccess) {
        if (!c->o.create_stream) c->stream = (cudaStream_t)c->o.stream;
        else { e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking); c->own_stream = true; }
        for (int i = 0; i < 3 && e == cudaSuccess && c->o.graphs; i++)
            e = cudaStreamCreateWithFlags(&c->cap[i], cudaStreamNonBlocking);
    }
    if (e != cudaSuccess) { delete c; return KKT_ERR_CUDA; }
    c->mixed = c->o.precision == KKT_PRECISION_MIXED;
    c->fallback_on = c->mixed && c->o.mixed_fallback > 0;
    c->eq_on = c->mixed && c->o.equilibrate;
    int per_sm = 0, per_sm3 = 0;
    if (c->mixed) {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kkt::k_lsolve_bulk<float>, PERSIST_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm3, kkt::k_usolve_bulk<float>, PERSIST_THREADS, 0);
    } else {
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kkt::k_lsolve_bulk<double>, PERSIST_THREADS, 0);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm3, kkt::k_usolve_bulk<double>, PERSIST_THREADS, 0);
    }
    for (const void* fn : {(const void*)kkt::k_lsolve_chain<double>, (const void*)kkt::k_usolve_chain<double>,
                           (const void*)kkt::k_lsolve_chain<float>, (const void*)kkt::k_usolve_chain<float>})
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)(sizeof(double) * CHAIN_MAX));
    cudaDeviceGetAttribute(&c->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->dev);
    c->smem_optin -= 1024;   // room for the kernel's static shared memory
    for (const void* fn : {(const void*)kkt::k_refactor_rows<double, false, 0, false>,
                           (const void*)kkt::k_refactor_rows<double, true, 0, false>,
                           (const void*)kkt::k_refactor_rows<double, false, 1, false>,
                           (const void*)kkt::k_refactor_rows<double, true, 1, false>,
                           (const void*)kkt::k_refactor_rows<double, false, 2, false>,
                           (const void*)kkt::k_refactor_rows<double, true, 2, false>,
                           (const void*)kkt::k_refactor_rows<float, false, 0, false>,
                           (const void*)kkt::k_refactor_rows<float, true, 0, false>,
                           (const void*)kkt::k_refactor_rows<float, false, 1, false>,
                           (const void*)kkt::k_refactor_rows<float, true, 1, false>,
                           (const void*)kkt::k_refactor_rows<float, false, 2, false>,
                           (const void*)kkt::k_refactor_rows<float, true, 2, false>,
                           (const void*)kkt::k_refactor_rows<double, true, 0, true>,
                           (const void*)kkt::k_refactor_rows<double, true, 1, true>,
                           (const void*)kkt::k_refactor_rows<double, true, 2, true>})
        cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, c->smem_optin);
    cudaGetLastError();
    per_sm = std::max(1, std::min(per_sm, per_sm3));
    c->persist_blocks = c->num_sms * per_sm;
    *out = c;
    return KKT_OK;
}

void kkt_destroy(kkt_ctx* c) {
    if (!c) return;
    cudaSetDevice(c->dev);
    cudaStreamSynchronize(c->stream);
    free_device(c);
    for (cudaStream_t& st : c->cap)
        if (st) { cudaStreamDestroy(st); st = nullptr; }
    if (c->own_stream && c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int kkt_order(int32_t n, const int32_t* rowptr, const int32_t* colind, int32_t* Q) {
    if (!Q) return KKT_ERR_INVALID;
    kkt::Csr A;
    std::string why;
    int rc = kkt::canonicalize(n, rowptr, colind, &A, &why);
    if (rc) return rc;
    std::vector<int32_t> q;
    rc = kkt::order_colamd_like(A, &q);
    if (rc) return rc;
    std::copy(q.begin(), q.end(), Q);
    return KKT_OK;
}

int kkt_pivot(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* values, const int32_t* Q,
              double pivot_tol, int32_t* P, int64_t* nnz_l, int64_t* nnz_u) {
    if (!P || !values || pivot_tol <= 0 || pivot_tol > 1) return KKT_ERR_INVALID;
    kkt::Csr A;
    std::string why;
    int rc = kkt::canonicalize(n, rowptr, colind, &A, &why);
    if (rc) return rc;
    std::vector<int32_t> q;
    if (Q) q.assign(Q, Q + n); else { rc = kkt::order_colamd_like(A, &q); if (rc) return rc; }
    std::vector<double> v(A.colind.size());
    for (size_t e = 0; e < v.size(); e++) v[e] = values[A.src[e]];
    std::vector<int32_t> p;
    kkt::ColStructure S;
    int32_t bad = -1;
    rc = kkt::pivot_lu(A, v.data(), q, pivot_tol, &p, &S, &bad);
    if (rc) return rc;
    std::copy(p.begin(), p.end(), P);
    if (nnz_l) *nnz_l = S.Lp[n];
    if (nnz_u) *nnz_u = S.Up[n];
    return KKT_OK;
}

namespace {
// Placement and dispatch order of the refactorization's rows
// (k_refactor_rows).  A row's working set -- step descriptors (8 bytes per
// L entry), values and columns -- decides where it runs: one per warp if it
// fits a warp's slice of the block's shared memory, one per block if it
// fits the block's shared memory with a position table of its columns
// (kkt::row_table_bits), else one per block with its values in global
// scratch.  By default the block's shared memory is sized for the row that
// needs the most (so no row needs global scratch) up to the device's
// limit.  Rows are dispatched by DAG level (ties by row) or by row;
// consecutive warp rows form one work item per block.
int setup_rows(kkt_ctx* c) {
    const int n = c->A.n;
    const auto& L = c->lay;
    for (void* p : c->row_allocs) cudaFree(p);
    c->row_allocs.clear();
    c->d_gdk = c->d_gcnt = nullptr;
    c->d_gsdoff = c->d_gwoff = nullptr;
    c->d_gw = nullptr;
    const size_t vsize = layout_vsize(c);
    if ((uint64_t)L.Fj.size() >= ((uint64_t)1 << 32)) {   // step descriptors hold 32-bit factor positions
        c->detail = "the factors have 2^32 entries or more";
        return KKT_ERR_INVALID;
    }
    // a warp row's working set; a block row's also holds its position table
    // (the smallest that kkt::row_table_bits allows)
    auto need = [&](int32_t i) -> size_t {
        const int64_t st = L.Fdiag[i] - L.Fp[i], len = L.Fp[i + 1] - L.Fp[i];
        return ((size_t)kkt::row_set_bytes(st, len, (int64_t)vsize) + 15) & ~(size_t)15;
    };
    auto need_block = [&](int32_t i) -> size_t {
        const int64_t st = L.Fdiag[i] - L.Fp[i], len = L.Fp[i + 1] - L.Fp[i];
        const int bits = std::max(kkt::ceil_log2_i64(len + len / 4 + 1), 4);
        return ((size_t)kkt::row_set_bytes(st, len, (int64_t)vsize) + ((size_t)2 << bits) + 15) & ~(size_t)15;
    };
    size_t maxneed = 16;
    for (int32_t i = 0; i < n; i++) maxneed = std::max(maxneed, need_block(i));
    const size_t optin = (size_t)std::max(c->smem_optin, 48 * 1024);
    size_t S = c->o.block_smem > 0 ? std::min((size_t)c->o.block_smem, optin) & ~(size_t)15 : std::min(maxneed, optin);
    S = std::max(S, (size_t)4096);
    // by default a block takes all the room of its shape's blocks per SM:
    // the blocks an SM holds are the same, the warp rows' slices larger
    if (c->o.block_smem <= 0) S = std::min(S <= REF_SMEM_THREE ? REF_SMEM_THREE : S <= REF_SMEM_WIDE ? REF_SMEM_WIDE : optin, optin);
    // block shape: three 256-thread blocks an SM when they fit its shared
    // memory, else two, else one of 512 threads
    c->ref_shape = S <= REF_SMEM_THREE ? 0 : S <= REF_SMEM_WIDE ? 1 : 2;
    c->ref_threads = c->ref_shape == 2 ? 512 : 256;
    c->ref_smem = S;
    const int nw = c->ref_threads / 32;
    const size_t slice = (S / nw) & ~(size_t)15;
    std::vector<uint8_t> kind((size_t)n);
    c->rows_warp = c->rows_block = c->rows_global = c->rows_team = 0;
    // with teams (kkt::RefShape::TEAMS), rows that fit a team's share of the
    // shared memory go one per team (the kernel's team room: S / teams
    // rounded down to 16)
    const int teams = c->o.team_rows ? kkt::ref_teams(c->ref_shape) : 1;
    const int64_t team_room = (int64_t)((S / (size_t)teams) & ~(size_t)15);
    // a warp row's steps run one after another on 32 lanes: rows with much
    // work (the dense end, on the critical path) go one per block even when
    // they fit a slice
    const int64_t wmax = c->o.warp_row_updates < 0 ? INT64_MAX
                       : c->o.warp_row_updates > 0 ? c->o.warp_row_updates
                       : c->ref_threads == 512 ? DEFAULT_WARP_ROW_UPDATES_WIDE : DEFAULT_WARP_ROW_UPDATES;
    for (int32_t i = 0; i < n; i++) {
        const size_t q = need(i);
        int64_t upd = 0;
        for (int64_t p = L.Fp[i]; p < L.Fdiag[i] && upd <= wmax; p++) {
            const int32_t k = L.Fj[p];
            upd += L.Fp[k + 1] - L.Fdiag[k] - 1;
        }
        if (c->o.warp_rows && q <= slice && upd <= wmax) { kind[i] = kkt::ROW_WARP; c->rows_warp++; }
        else if (teams > 1 && kkt::row_table_bits(L.Fdiag[i] - L.Fp[i], L.Fp[i + 1] - L.Fp[i], (int64_t)vsize,
                                                   team_room) >= 0) {
            kind[i] = kkt::ROW_TEAM;
            c->rows_team++;
        } else if (kkt::row_table_bits(L.Fdiag[i] - L.Fp[i], L.Fp[i + 1] - L.Fp[i], (int64_t)vsize, (int64_t)S) >= 0) {
            kind[i] = kkt::ROW_BLOCK;
            c->rows_block++;
        }
        else { kind[i] = kkt::ROW_GLOBAL; c->rows_global++; }
    }
    // dispatch order: by level in the DAG of L (ties by row) -- a row's
    // dependencies are at lower levels, so they are dispatched before it;
    // or by critical-path priority: descending bottom level, the longest
    // path of estimated row costs from the row to the end of the DAG (a
    // dependency's is larger than its dependents', so it still comes
    // first), so rows on long chains get slots before rows with slack
    std::vector<int32_t> order((size_t)n);
    std::iota(order.begin(), order.end(), 0);
    if (c->o.row_order == 1) {
        const std::vector<int32_t>& lev = L.levL;
        std::sort(order.begin(), order.end(),
                  [&](int32_t a, int32_t b) { return lev[a] < lev[b] || (lev[a] == lev[b] && a < b); });
    } else if (c->o.row_order == 2) {
        // cost of a row: its steps plus its multiply-adds / 1024 (a heavy
        // block row's step is ~1 us with ~1,000 updates)
        std::vector<double> w((size_t)n), bl((size_t)n);
        for (int32_t i = 0; i < n; i++) {
            double upd = 0.0;
            for (int64_t p = L.Fp[i]; p < L.Fdiag[i]; p++) {
                const int32_t k = L.Fj[p];
                upd += (double)(L.Fp[k + 1] - L.Fdiag[k] - 1);
            }
            w[i] = 2.0 + (double)(L.Fdiag[i] - L.Fp[i]) + upd / 1024.0;
            bl[i] = w[i];
        }
        for (int32_t r = n - 1; r >= 0; r--)   // a row's dependencies are rows before it
            for (int64_t p = L.Fp[r]; p < L.Fdiag[r]; p++) {
                const int32_t k = L.Fj[p];
                bl[k] = std::max(bl[k], w[k] + bl[r]);
            }
        std::sort(order.begin(), order.end(),
                  [&](int32_t a, int32_t b) { return bl[a] > bl[b] || (bl[a] == bl[b] && a < b); });
    }
    std::vector<kkt::RefItem> items;
    items.reserve((size_t)n);
    std::vector<uint32_t> gdk, gcnt;
    std::vector<int64_t> gsdoff, gwoff;
    int64_t gw_total = 0;
    for (int32_t t = 0; t < n;) {
        const int32_t r = order[t];
        if (kind[r] == kkt::ROW_WARP) {
            int32_t cnt = 1;
            while (cnt < nw && t + cnt < n && kind[order[t + cnt]] == kkt::ROW_WARP) cnt++;
            items.push_back(kkt::RefItem{t, (kkt::ROW_WARP << 28) | cnt});
            t += cnt;
            continue;
        }
        if (kind[r] == kkt::ROW_TEAM) {
            int32_t cnt = 1;
            while (cnt < teams && t + cnt < n && kind[order[t + cnt]] == kkt::ROW_TEAM) cnt++;
            items.push_back(kkt::RefItem{t, (kkt::ROW_TEAM << 28) | cnt});
            t += cnt;
            continue;
        }
        if (kind[r] == kkt::ROW_BLOCK) {
            items.push_back(kkt::RefItem{t, kkt::ROW_BLOCK << 28});
        } else {
            const int32_t g = (int32_t)gsdoff.size();
            gsdoff.push_back((int64_t)gdk.size());
            gwoff.push_back(gw_total);
            for (int64_t q = L.Fp[r]; q < L.Fdiag[r]; q++) {
                const int32_t k = L.Fj[q];
                gdk.push_back((uint32_t)L.Fdiag[k]);
                gcnt.push_back((uint32_t)(L.Fp[k + 1] - L.Fdiag[k] - 1));
            }
            gw_total += L.Fp[r + 1] - L.Fp[r];
            items.push_back(kkt::RefItem{t, (kkt::ROW_GLOBAL << 28) | g});
        }
        t++;
    }
    c->nitems = (int)items.size();
    CK(cudaMemcpyAsync(c->d_order, order.data(), sizeof(int32_t) * order.size(), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(c->d_items, items.data(), sizeof(kkt::RefItem) * items.size(), cudaMemcpyHostToDevice,
                       c->stream));
    if (!gsdoff.empty()) {
        auto up = [&](auto** p, const auto& v) -> cudaError_t {
            void* q = nullptr;
            cudaError_t e = cudaMalloc(&q, std::max<size_t>(v.size(), 1) * sizeof(v[0]));
            if (e != cudaSuccess) return e;
            c->row_allocs.push_back(q);
            *p = (std::remove_reference_t<decltype(**p)>*)q;
            return v.empty() ? cudaSuccess
                             : cudaMemcpyAsync(q, v.data(), v.size() * sizeof(v[0]), cudaMemcpyHostToDevice, c->stream);
        };
        CK(up(&c->d_gdk, gdk));
        CK(up(&c->d_gcnt, gcnt));
        CK(up(&c->d_gsdoff, gsdoff));
        CK(up(&c->d_gwoff, gwoff));
        void* q = nullptr;
        CK(cudaMalloc(&q, std::max<int64_t>(gw_total, 1) * vsize));
        c->row_allocs.push_back(q);
        c->d_gw = q;
    }
    CK(cudaStreamSynchronize(c->stream));   // the host vectors are locals
    int per_sm = 1 << 30;
    std::vector<const void*> fns;
    auto both = [&](auto f_plain, auto f_fused) { fns.push_back((const void*)f_plain); fns.push_back((const void*)f_fused); };
    if (c->mixed) {
        if (c->ref_shape == 0) both(kkt::k_refactor_rows<float, false, 0, false>, kkt::k_refactor_rows<float, true, 0, false>);
        if (c->ref_shape == 1) both(kkt::k_refactor_rows<float, false, 1, false>, kkt::k_refactor_rows<float, true, 1, false>);
        if (c->ref_shape == 2) both(kkt::k_refactor_rows<float, false, 2, false>, kkt::k_refactor_rows<float, true, 2, false>);
    }
    if (!c->mixed || c->fallback_on) {
        if (c->ref_shape == 0) both(kkt::k_refactor_rows<double, false, 0, false>, kkt::k_refactor_rows<double, true, 0, false>);
        if (c->ref_shape == 1) both(kkt::k_refactor_rows<double, false, 1, false>, kkt::k_refactor_rows<double, true, 1, false>);
        if (c->ref_shape == 2) both(kkt::k_refactor_rows<double, false, 2, false>, kkt::k_refactor_rows<double, true, 2, false>);
    }
    for (const void* fn : fns) {   // the grid is sized for the instantiation with fewer resident blocks
        int bl = 0;
        CK(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&bl, fn, c->ref_threads, c->ref_smem));
        per_sm = std::min(per_sm, bl);
    }
    if (per_sm < 1) { c->detail = "refactorization kernel does not fit an SM"; return KKT_ERR_INVALID; }
    c->ref_blocks = per_sm * c->num_sms;
    return KKT_OK;
}

int setup_device(kkt_ctx* c, const kkt::ColStructure& S, std::chrono::steady_clock::time_point t0);
}

int kkt_analyze(kkt_ctx* c, int32_t n, const int32_t* rowptr, const int32_t* colind, const double* values0,
                const int32_t* Qin, const int32_t* Pin) {
    if (!c) return KKT_ERR_INVALID;
    auto t0 = std::chrono::steady_clock::now();
    CK(cudaSetDevice(c->dev));
    CK(cudaStreamSynchronize(c->stream));
    free_device(c);
    c->detail.clear();
    std::string why;
    int rc = kkt::canonicalize(n, rowptr, colind, &c->A, &why);
    if (rc) { c->detail = why; return rc; }
    if (n < 1) { c->detail = "n must be positive"; return KKT_ERR_INVALID; }
    c->nnz_a = (int64_t)c->A.colind.size();
    if (Qin) {
        c->Q.assign(Qin, Qin + n);
        std::vector<char> seen(n, 0);
        for (int32_t j = 0; j < n; j++) {
            if (c->Q[j] < 0 || c->Q[j] >= n || seen[c->Q[j]]) { c->detail = "Q is not a permutation"; return KKT_ERR_INVALID; }
            seen[c->Q[j]] = 1;
        }
    } else {
        rc = kkt::order_colamd_like(c->A, &c->Q);
        if (rc) { c->detail = "ordering failed"; return rc; }
    }
    kkt::ColStructure S;
    int32_t bad = -1;
    if (Pin) {
        c->P.assign(Pin, Pin + n);
        rc = kkt::symbolic(c->A, c->P, c->Q, &S, &bad);
        if (rc) { c->detail = "symbolic analysis failed at column " + std::to_string(bad); return rc; }
    } else {
        if (!values0) { c->detail = "values0 is required when P is not given"; return KKT_ERR_INVALID; }
        std::vector<double> v(c->nnz_a);
        for (int64_t e = 0; e < c->nnz_a; e++) v[e] = values0[c->A.src[e]];
        rc = kkt::pivot_lu(c->A, v.data(), c->Q, c->o.pivot_tol, &c->P, &S, &bad);
        if (rc) { c->detail = "pivoting factorization failed at column " + std::to_string(bad); return rc; }
    }
    return setup_device(c, S, t0);
}

namespace {
int setup_from_layout(kkt_ctx* c, std::chrono::steady_clock::time_point t0);

// Everything kkt_analyze does once P, Q and the factor structure are known:
// the GPU layout, schedules and every device buffer.
int setup_device(kkt_ctx* c, const kkt::ColStructure& S, std::chrono::steady_clock::time_point t0) {
    int rc = kkt::build_layout(c->A, c->P, c->Q, S, &c->lay);
    if (rc) { c->detail = "factor layout failed"; return rc; }
    return setup_from_layout(c, t0);
}

int setup_from_layout(kkt_ctx* c, std::chrono::steady_clock::time_point t0) {
    const int32_t n = c->A.n;
    int rc = KKT_OK;
    // composite gather map: factor slot -> caller value index
    std::vector<int64_t> fsrc(c->lay.Fsrc.size());
    for (size_t t = 0; t < fsrc.size(); t++) fsrc[t] = c->lay.Fsrc[t] >= 0 ? c->A.src[c->lay.Fsrc[t]] : -1;
    const int64_t nnzF = (int64_t)c->lay.Fj.size();
    // ---- device buffers, made once for the whole sequence
    c->ld = ((int64_t)n + 31) / 32 * 32;
    if ((rc = upload(c, &c->d_Fp, c->lay.Fp))) return rc;
    if ((rc = upload(c, &c->d_Fdiag, c->lay.Fdiag))) return rc;
    if ((rc = upload(c, &c->d_Fj, c->lay.Fj))) return rc;
    if ((rc = upload(c, &c->d_fsrc, fsrc))) return rc;
    if (!c->A.identity_src) { if ((rc = upload(c, &c->d_asrc, c->A.src))) return rc; }
    else c->d_asrc = nullptr;
    if ((rc = upload(c, &c->d_Arp, c->A.rowptr))) return rc;
    if ((rc = upload(c, &c->d_Aci, c->A.colind))) return rc;
    if ((rc = upload(c, &c->d_P, c->P))) return rc;
    if ((rc = upload(c, &c->d_Q, c->Q))) return rc;
    if (c->mixed) {
        float *fx = nullptr, *ri = nullptr;
        if ((rc = dalloc(c, &fx, nnzF))) return rc;
        if ((rc = dalloc(c, &ri, (size_t)n))) return rc;
        c->d_Fx = fx;
        c->d_rinv = ri;
        c->d_Fx64 = c->d_rinv64 = nullptr;
        if (c->fallback_on) {
            double *fx64 = nullptr, *ri64 = nullptr;
            if ((rc = dalloc(c, &fx64, nnzF))) return rc;
            if ((rc = dalloc(c, &ri64, (size_t)n))) return rc;
            c->d_Fx64 = fx64;
            c->d_rinv64 = ri64;
        }
    } else {
        double *fx = nullptr, *ri = nullptr;
        if ((rc = dalloc(c, &fx, nnzF))) return rc;
        if ((rc = dalloc(c, &ri, (size_t)n))) return rc;
        c->d_Fx = fx;
        c->d_rinv = ri;
    }
    if ((rc = dalloc(c, &c->d_Ax, c->nnz_a))) return rc;
    if ((rc = dalloc(c, &c->d_vals, c->nnz_a))) return rc;
    c->d_eq_r = c->d_eq_c = c->d_eq_vals = c->d_eq_tmp = nullptr;
    c->d_eq_colmax = nullptr;
    if (c->eq_on) {
        if ((rc = dalloc(c, &c->d_eq_r, (size_t)n))) return rc;
        if ((rc = dalloc(c, &c->d_eq_c, (size_t)n))) return rc;
        if ((rc = dalloc(c, &c->d_eq_colmax, (size_t)n))) return rc;
        if ((rc = dalloc(c, &c->d_eq_tmp, (size_t)n))) return rc;
        if ((rc = dalloc(c, &c->d_eq_vals, c->nnz_a))) return rc;
    }
    for (double** p : {&c->d_b, &c->d_x, &c->d_y, &c->d_xp, &c->d_r, &c->d_w})
        if ((rc = dalloc(c, p, c->ld))) return rc;
    if ((rc = dalloc(c, &c->d_V, (size_t)c->ld * (c->m + 1)))) return rc;
    if ((rc = dalloc(c, &c->d_Z, (size_t)c->ld * c->m))) return rc;
    if ((rc = dalloc(c, &c->d_part, (size_t)kkt::RED_BLOCKS * kkt::RED_SLOTS))) return rc;
    if ((rc = dalloc(c, &c->d_done_f, (size_t)n))) return rc;
    CK(cudaMemsetAsync(c->d_done_f, 0, sizeof(unsigned) * (size_t)n, c->stream));
    {
        std::vector<int32_t> listL, posL, listU, posU;
        level_order(c->lay.levL, &listL, &posL);
        level_order(c->lay.levU, &listU, &posU);
        c->nLc = chain_rows(c->lay.levL, true, CHAIN_MAX);
        c->nUc = chain_rows(c->lay.levU, false, CHAIN_MAX);
        std::vector<int32_t> fpos(nnzF, 0);
        for (int32_t i = 0; i < n; i++) {
            for (int64_t p = c->lay.Fp[i]; p < c->lay.Fdiag[i]; p++) fpos[p] = posL[c->lay.Fj[p]];
            for (int64_t p = c->lay.Fdiag[i] + 1; p < c->lay.Fp[i + 1]; p++) fpos[p] = posU[c->lay.Fj[p]];
        }
        if ((rc = upload(c, &c->d_listL, listL))) return rc;
        if ((rc = upload(c, &c->d_listU, listU))) return rc;
        if ((rc = upload(c, &c->d_Fpos, fpos))) return rc;
    }
    c->fp64_active = false;
    c->vec_f32 = use_f32(c);
    fill_y_sentinel(c);
    if (c->o.trisolve == KKT_TRSV_AUTO) pick_cluster(c);
    else c->cluster = 0;
    if ((rc = dalloc(c, &c->d_order, (size_t)n))) return rc;
    if ((rc = dalloc(c, &c->d_items, (size_t)n))) return rc;
    if ((rc = setup_rows(c))) return rc;
    if ((rc = dalloc(c, &c->d_s, 1))) return rc;
    CK(cudaMemsetAsync(c->d_s, 0, sizeof(DevScal), c->stream));
    CK(cudaMallocHost(&c->h_s, sizeof(DevScal)));
    if (c->o.timing) {
        c->ev_pool.resize(2 * EV_PAIRS);
        c->ev_phase.assign(EV_PAIRS, 0);
        for (auto& e : c->ev_pool) CK(cudaEventCreate(&e));
    }
    CK(cudaStreamSynchronize(c->stream));
    c->analyzed = true;
    c->factored = false;
    c->analyze_ms = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
    return KKT_OK;
}
}  // namespace

namespace {
int refactor_impl(kkt_ctx* c, const double* values, int values_on_device, unsigned long long* trace,
                  const double* fused_rhs = nullptr);
}

int kkt_analyze_like(kkt_ctx* c, const kkt_ctx* src) {
    if (!c || !src || c == src) return KKT_ERR_INVALID;
    if (!src->analyzed) { c->detail = "kkt_analyze_like: the source context is not analysed"; return KKT_ERR_STATE; }
    auto t0 = std::chrono::steady_clock::now();
    CK(cudaSetDevice(c->dev));
    CK(cudaStreamSynchronize(c->stream));
    free_device(c);
    c->detail.clear();
    c->A = src->A;
    c->nnz_a = src->nnz_a;
    c->P = src->P;
    c->Q = src->Q;
    c->lay = src->lay;
    return setup_from_layout(c, t0);
}

int kkt_host_analyze(int32_t n, const int32_t* rowptr, const int32_t* colind, const double* values0,
                     double pivot_tol, int32_t* P, int32_t* Q, kkt_host_stats* st) {
    if (!P || !Q || !values0 || !(pivot_tol > 0) || pivot_tol > 1) return KKT_ERR_INVALID;
    kkt::Csr A;
    std::string why;
    int rc = kkt::canonicalize(n, rowptr, colind, &A, &why);
    if (rc) return rc;
    if (n < 1) return KKT_ERR_INVALID;
    auto t0 = std::chrono::steady_clock::now();
    std::vector<int32_t> q;
    if ((rc = kkt::order_colamd_like(A, &q))) return rc;
    auto t1 = std::chrono::steady_clock::now();
    std::vector<double> v(A.colind.size());
    for (size_t e = 0; e < v.size(); e++) v[e] = values0[A.src[e]];
    std::vector<int32_t> p;
    kkt::ColStructure S;
    int32_t bad = -1;
    if ((rc = kkt::pivot_lu(A, v.data(), q, pivot_tol, &p, &S, &bad))) return rc;
    auto t2 = std::chrono::steady_clock::now();
    std::copy(p.begin(), p.end(), P);
    std::copy(q.begin(), q.end(), Q);
    if (st) {
        kkt::Layout lay;
        if ((rc = kkt::build_layout(A, p, q, S, &lay))) return rc;
        st->nnz_l = lay.nnzL;
        st->nnz_u = lay.nnzU;
        st->levels_l = lay.levelsL;
        st->levels_u = lay.levelsU;
        st->refactor_updates = lay.updates;
        st->order_ms = std::chrono::duration<double, std::milli>(t1 - t0).count();
        st->pivot_ms = std::chrono::duration<double, std::milli>(t2 - t1).count();
        st->canonical_order = A.identity_src ? 1 : 0;
    }
    return KKT_OK;
}

int kkt_estimate_device_bytes(int32_t n, int64_t nnz_a, const kkt_host_stats* st, const kkt_opts* o,
                              int canonical_order, int64_t* bytes) {
    if (!st || !bytes || n < 1 || nnz_a < 0) return KKT_ERR_INVALID;
    kkt_opts d;
    if (!o) { kkt_default_opts(&d); o = &d; }
    // every dalloc / upload of setup_from_layout, in order
    auto sz = [](int64_t count, int64_t elem) { return std::max<int64_t>(count, 1) * elem; };
    const int64_t nnzF = st->nnz_l + st->nnz_u;
    const int64_t ld = ((int64_t)n + 31) / 32 * 32;
    const bool mixed = o->precision == KKT_PRECISION_MIXED;
    int64_t b = 0;
    b += sz(n + 1, 8) + sz(n, 8) + sz(nnzF, 4) + sz(nnzF, 8);            // Fp, Fdiag, Fj, fsrc
    if (!canonical_order) b += sz(nnz_a, 8);                                // asrc
    b += sz(n + 1, 4) + sz(nnz_a, 4) + sz(n, 4) + sz(n, 4);               // Arp, Aci, P, Q
    if (mixed) {
        b += sz(nnzF, 4) + sz(n, 4);                                        // Fx, rinv (FP32)
        if (o->mixed_fallback > 0) b += sz(nnzF, 8) + sz(n, 8);            // the FP64 fallback's
        if (o->equilibrate) b += 4 * sz(n, 8) + sz(nnz_a, 8);               // R, C, column maxima, R b, R K C
    } else {
        b += sz(nnzF, 8) + sz(n, 8);
    }
    b += 2 * sz(nnz_a, 8);                                                  // Ax, vals
    b += 6 * sz(ld, 8);                                                     // b, x, y, xp, r, w
    b += sz(ld * (o->restart + 1), 8) + sz(ld * o->restart, 8);             // V, Z
    b += sz((int64_t)kkt::RED_BLOCKS * kkt::RED_SLOTS, 8) + sz(n, 4);       // part, done flags
    b += 2 * sz(n, 4) + sz(nnzF, 4);                                        // listL, listU, Fpos
    b += sz(n, 4) + sz(n, (int64_t)sizeof(kkt::RefItem));                  // order, items
    b += sz(1, (int64_t)sizeof(DevScal));
    *bytes = b;
    return KKT_OK;
}

int kkt_place_instance(int ndev, const int64_t* budget, const int64_t* held, int64_t need) {
    if (ndev < 1 || !budget || !held || need < 0) return -1;
    int best = -1;
    int64_t best_left = 0;
    for (int i = 0; i < ndev; i++) {
        if (need > budget[i]) continue;   // can never fit this device
        const int64_t left = budget[i] - held[i];
        if (best < 0 || left > best_left) { best = i; best_left = left; }
    }
    return best;
}

int kkt_trace_critical_path(kkt_ctx* c, const int64_t* t_start, const int64_t* t_publish, double* path_ns,
                            int32_t* levels, double* median_link_ns, int32_t* rows) {
    if (!c || !t_start || !t_publish) return KKT_ERR_INVALID;
    if (!c->analyzed) return KKT_ERR_STATE;
    const int32_t n = c->A.n;
    const auto& L = c->lay;
    std::vector<double> cp((size_t)n, 0.0), links;
    links.reserve((size_t)n);
    double best = 0.0;
    for (int32_t i = 0; i < n; i++) {
        double before = 0.0;
        int64_t last = -1;
        for (int64_t q = L.Fp[i]; q < L.Fdiag[i]; q++) {
            const int32_t k = L.Fj[q];
            before = std::max(before, cp[k]);
            last = std::max<int64_t>(last, t_publish[k]);
        }
        double link = 0.0;
        if (t_publish[i] > 0 && t_start[i] > 0) {
            link = (double)(t_publish[i] - std::max<int64_t>(t_start[i], last));
            if (link < 0) link = 0.0;
            links.push_back(link);
        }
        cp[i] = before + link;
        best = std::max(best, cp[i]);
    }
    if (path_ns) *path_ns = best;
    if (levels) *levels = L.levelsL;
    if (rows) *rows = (int32_t)links.size();
    if (median_link_ns) {
        if (links.empty()) *median_link_ns = 0.0;
        else {
            std::nth_element(links.begin(), links.begin() + links.size() / 2, links.end());
            *median_link_ns = links[links.size() / 2];
        }
    }
    return KKT_OK;
}

int kkt_repivot(kkt_ctx* c, const double* values, int values_on_device) {
    int rc = check_ctx(c, false);
    if (rc) return rc;
    if (!values) return KKT_ERR_INVALID;
    auto t0 = std::chrono::steady_clock::now();
    const int64_t nnz = c->nnz_a;
    std::vector<double> hv((size_t)nnz);
    if (values_on_device) {
        CK(cudaMemcpyAsync(hv.data(), values, sizeof(double) * (size_t)nnz, cudaMemcpyDeviceToHost, c->stream));
        c->d2h += (int64_t)sizeof(double) * nnz;
    } else {
        std::copy(values, values + nnz, hv.begin());
    }
    CK(cudaStreamSynchronize(c->stream));
    std::vector<double> v((size_t)nnz);
    for (int64_t e = 0; e < nnz; e++) v[e] = hv[c->A.src[e]];
    kkt::ColStructure S;
    std::vector<int32_t> P;
    int32_t bad = -1;
    rc = kkt::pivot_lu(c->A, v.data(), c->Q, c->o.pivot_tol, &P, &S, &bad);
    if (rc) {   // the previous analysis stays in place
        c->detail = "pivoting factorization failed at column " + std::to_string(bad);
        return rc;
    }
    free_device(c);
    c->P = P;
    if ((rc = setup_device(c, S, t0))) return rc;
    c->repivots++;
    return refactor_impl(c, hv.data(), 0, nullptr);
}

int kkt_refactor(kkt_ctx* c, const double* values, int values_on_device) {
    int rc = refactor_impl(c, values, values_on_device, nullptr);
    if (rc == KKT_ERR_ZERO_PIVOT && c && c->o.repivot) rc = kkt_repivot(c, values, values_on_device);
    return rc;
}

int kkt_trace_refactor(kkt_ctx* c, const double* values, int values_on_device, int64_t* t_start,
                       int64_t* t_publish, int32_t* t0_out) {
    int rc = check_ctx(c, false);
    if (rc) return rc;
    if (!t_start || !t_publish || !t0_out) return KKT_ERR_INVALID;
    const int n = c->A.n;
    *t0_out = 0;
    unsigned long long* d_trace = nullptr;   // profiling only: a buffer of its own
    CK(cudaMalloc(&d_trace, sizeof(unsigned long long) * 2 * (size_t)n));
    CK(cudaMemsetAsync(d_trace, 0, sizeof(unsigned long long) * 2 * (size_t)n, c->stream));
    rc = refactor_impl(c, values, values_on_device, d_trace);
    std::vector<unsigned long long> h(2 * (size_t)n);
    cudaError_t e = cudaMemcpy(h.data(), d_trace, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost);
    cudaFree(d_trace);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
    for (int r = 0; r < n; r++) {
        t_start[r] = h[2 * (size_t)r] ? (int64_t)h[2 * (size_t)r] : -1;
        t_publish[r] = h[2 * (size_t)r + 1] ? (int64_t)h[2 * (size_t)r + 1] : -1;
    }
    return rc;
}

extern "C++" {
namespace {
// gather (arms every factor value with SENTINEL), then the one
// refactorization kernel over every row, in type T
template <typename T, int SHAPE>
void refactor_rows_launch(kkt_ctx* c, const double* vals, unsigned long long* trace, const double* fused_rhs) {
    constexpr int NT = kkt::RefShape<SHAPE>::NT;
    kkt::RefArgs<T> a{};
    a.items = c->d_items;
    a.nitems = c->nitems;
    a.order = c->d_order;
    a.Fp = c->d_Fp;
    a.Fj = c->d_Fj;
    a.Fdiag = c->d_Fdiag;
    a.Fx = fx_of<T>(c);
    a.rinv = rinv_of<T>(c);
    a.vals = vals;
    a.fsrc = c->d_fsrc;
    a.area_bytes = (int)c->ref_smem;
    a.slice_bytes = (int)((c->ref_smem / (c->ref_threads / 32)) & ~(size_t)15);
    a.gdk = c->d_gdk;
    a.gcnt = c->d_gcnt;
    a.g_sd_off = c->d_gsdoff;
    a.gw = (T*)c->d_gw;
    a.g_w_off = c->d_gwoff;
    a.s = c->d_s;
    a.fw = kkt::FwdArgs<T>{fused_rhs, c->d_P, (T*)c->d_y, (T*)c->d_xp};
    a.boost_eps = c->o.boost_eps;
    a.stream_last = c->o.stream_last;
    const int blocks = std::max(1, std::min(c->nitems, c->ref_blocks));
    auto kern = fused_rhs ? kkt::k_refactor_rows<T, true, SHAPE, false> : kkt::k_refactor_rows<T, false, SHAPE, false>;
    kern<<<blocks, NT, c->ref_smem, c->stream>>>(a, kkt::RefBatch<T>{}, spin(c), trace);
}

template <typename T>
void refactor_launch(kkt_ctx* c, const double* vals, unsigned long long* trace, const double* fused_rhs = nullptr) {
    const int n = c->A.n;
    const int64_t nnzF = (int64_t)c->lay.Fj.size();
    int t = phase_begin(c, KKT_PHASE_GATHER);
    kkt::k_gather<T><<<2 * c->num_sms, 256, 0, c->stream>>>(vals, nnzF, fx_of<T>(c), c->d_Arp, c->d_asrc, c->d_Ax,
                                                            n, rinv_of<T>(c), c->d_s,
                                                            fused_rhs ? (T*)c->d_y : nullptr);
    if (std::is_same<T, float>::value && c->eq_on) {
        // R K C from the canonical copy the gather just wrote; the FP32
        // factors are of it (the gather's ||K||_inf stays that of K)
        const int g = 2 * c->num_sms;
        kkt::k_eq_rows<<<g, 256, 0, c->stream>>>(n, c->d_Arp, c->d_Ax, c->d_eq_r, c->d_eq_colmax);
        kkt::k_eq_cols<<<g, 256, 0, c->stream>>>(n, c->d_Arp, c->d_Aci, c->d_Ax, c->d_eq_r, c->d_eq_colmax);
        kkt::k_eq_values<<<g, 256, 0, c->stream>>>(n, c->d_Arp, c->d_Aci, c->d_Ax, c->d_asrc, c->d_eq_r,
                                                   c->d_eq_colmax, c->d_eq_c, c->d_eq_vals);
        c->launches += 3;
        vals = c->d_eq_vals;
        fused_rhs = nullptr;   // the fused sweep would need R b
    }
    phase_end(c, t);
    t = phase_begin(c, KKT_PHASE_REFACTOR);
    if (c->ref_shape == 2) refactor_rows_launch<T, 2>(c, vals, trace, fused_rhs);
    else if (c->ref_shape == 1) refactor_rows_launch<T, 1>(c, vals, trace, fused_rhs);
    else refactor_rows_launch<T, 0>(c, vals, trace, fused_rhs);
    phase_end(c, t);
    c->launches += 3;   // prep, gather, refactorization
}
}  // namespace
}  // extern "C++"

namespace {
// The refactorization as one graph reading the values from d_vals.
int build_refactor_graph(kkt_ctx* c) {
    drop_graph(&c->gx_ref, &c->g_ref);
    c->capturing = true;
    g_capture_where = "";
    const int64_t l0 = c->launches;
    cudaError_t e = capture_graph(c, 0, &c->g_ref, [&] {
        kkt::k_refactor_prep<<<1, 1, 0, c->stream>>>(c->d_s);
        if (c->mixed) refactor_launch<float>(c, c->d_vals, nullptr);
        else refactor_launch<double>(c, c->d_vals, nullptr);
    });
    c->capturing = false;
    c->gl_ref = c->launches - l0 + 1;
    c->launches = l0;
    if (e != cudaSuccess) { drop_graph(&c->gx_ref, &c->g_ref); return cuda_fail(c, e, "refactor graph capture"); }
    CK(cudaGraphInstantiate(&c->gx_ref, c->g_ref, 0));
    return KKT_OK;
}

// The FP64 refactorization of a mixed-precision context (the fallback):
// the same kernels on the same values into the FP64 factor arrays, which
// the solves use until the next refactorization.
int refactor_fp64(kkt_ctx* c, const double* vals, const double* fused_rhs) {
    c->fp64_active = true;
    arm_vectors(c);
    kkt::k_refactor_prep<<<1, 1, 0, c->stream>>>(c->d_s);
    refactor_launch<double>(c, vals, nullptr, fused_rhs);
    CK(cudaGetLastError());
    int rc = read_scalars(c);
    if (rc) return rc;
    c->nboost = c->h_s->nboost;
    c->norm_a = c->h_s->normA;
    if ((rc = device_error(c))) return rc;
    c->last_fallback = 1;
    c->fallbacks++;
    return KKT_OK;
}

// Fallback during a solve: the caller's values are rebuilt from the
// canonical copy the gather made (so kkt_solve needs no values argument),
// then refactor_fp64.
int fallback_from_solve(kkt_ctx* c) {
    const int64_t nnz = c->nnz_a;
    kkt::k_scatter_values<<<2 * c->num_sms, 256, 0, c->stream>>>(nnz, c->d_Ax, c->d_asrc, c->d_vals);
    c->launches += 1;
    return refactor_fp64(c, c->d_vals, nullptr);
}

int refactor_impl(kkt_ctx* c, const double* values, int values_on_device, unsigned long long* trace,
                  const double* fused_rhs) {
    int rc = check_ctx(c, false);
    if (rc) return rc;
    if (!values) return KKT_ERR_INVALID;
    c->factored = false;
    c->y_fused = false;
    c->fp64_active = false;   // a new matrix starts in the context's own precision
    c->last_fallback = 0;
    arm_vectors(c);
    const double* vals = values;
    const bool graphs = c->o.graphs && !trace && !fused_rhs;
    if (!values_on_device) {
        CK(cudaMemcpyAsync(c->d_vals, values, sizeof(double) * (size_t)c->nnz_a, cudaMemcpyHostToDevice, c->stream));
        c->h2d += (int64_t)sizeof(double) * c->nnz_a;
        vals = c->d_vals;
    } else if (graphs) {   // the graph reads its fixed buffer
        CK(cudaMemcpyAsync(c->d_vals, values, sizeof(double) * (size_t)c->nnz_a, cudaMemcpyDeviceToDevice,
                           c->stream));
        vals = c->d_vals;
    }
    if (graphs) {
        if (!c->gx_ref && (rc = build_refactor_graph(c))) return rc;
        int t = phase_begin(c, KKT_PHASE_GRAPH_REFACTOR);
        CK(cudaGraphLaunch(c->gx_ref, c->stream));
        phase_end(c, t);
        c->launches += c->gl_ref;
    } else {
        kkt::k_refactor_prep<<<1, 1, 0, c->stream>>>(c->d_s);
        if (c->mixed) refactor_launch<float>(c, vals, trace, fused_rhs);
        else refactor_launch<double>(c, vals, trace, fused_rhs);
    }
    // an equilibrated FP32 refactorization does not fuse the forward sweep
    bool fused = fused_rhs != nullptr && !c->eq_on;
    CK(cudaGetLastError());
    if ((rc = read_scalars(c))) return rc;
    c->nboost = c->h_s->nboost;
    c->norm_a = c->h_s->normA;
    if ((rc = device_error(c))) {
        // an FP32 refactorization that meets a zero pivot or a non-finite
        // value falls back to FP64 on the same values
        if (!(c->fallback_on && (rc == KKT_ERR_ZERO_PIVOT || rc == KKT_ERR_NONFINITE))) return rc;
        if ((rc = refactor_fp64(c, vals, fused_rhs))) return rc;
        fused = fused_rhs != nullptr;
    }
    c->factored = true;
    c->y_fused = fused;
    return KKT_OK;
}
}  // namespace

int kkt_lu_solve(kkt_ctx* c, const double* b, double* x, int on_device) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (!b || !x) return KKT_ERR_INVALID;
    const int n = c->A.n;
    const double* bd = b;
    double* xd = x;
    if (!on_device) {
        CK(cudaMemcpyAsync(c->d_b, b, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        c->h2d += (int64_t)sizeof(double) * n;
        bd = c->d_b;
        xd = c->d_x;
    }
    CK(cudaMemsetAsync(&c->d_s->err, 0, sizeof(int) * 3, c->stream));
    lu_apply(c, bd, xd);
    CK(cudaGetLastError());
    if (!on_device) {
        CK(cudaMemcpyAsync(x, c->d_x, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
        c->d2h += (int64_t)sizeof(double) * n;
    }
    if ((rc = read_scalars(c))) return rc;
    if ((rc = device_error(c))) rearm(c);
    return rc;
}

int kkt_tune(kkt_ctx* c, const double* values, const double* b, int on_device, int reps, double* best_ms) {
    int rc = check_ctx(c, false);
    if (rc) return rc;
    if (!values || !b || reps < 1) return KKT_ERR_INVALID;
    const int n = c->A.n;
    double* x = nullptr;
    std::vector<double> hx;
    if (on_device) {
        if ((rc = dalloc(c, &x, (size_t)n))) return rc;   // tuning buffer, freed with the context
    } else {
        hx.resize(n);
        x = hx.data();
    }
    struct Cand { int trisolve, cluster_blocks, block_smem, warp_rows; };
    std::vector<Cand> cands;
    for (int wr : {1, 0})
        for (int bs : {0, 72 * 1024, 110 * 1024, c->smem_optin}) {
            for (int cb : {16, 8}) cands.push_back({KKT_TRSV_AUTO, cb, bs, wr});
            cands.push_back({KKT_TRSV_GLOBAL, 0, bs, wr});
        }
    const kkt_opts saved = c->o;
    double best = -1.0;
    Cand pick{saved.trisolve, saved.cluster_blocks, saved.block_smem, saved.warp_rows};
    auto apply = [&](const Cand& k) -> int {
        c->o.trisolve = k.trisolve;
        c->o.cluster_blocks = k.cluster_blocks;
        c->o.block_smem = k.block_smem;
        c->o.warp_rows = k.warp_rows;
        drop_graph(&c->gx_ref, &c->g_ref);
        drop_graph(&c->gx_solve, &c->g_solve);
        int r = setup_rows(c);
        if (r) return r;
        if (k.trisolve == KKT_TRSV_AUTO) {
            pick_cluster(c);
            if (c->cluster != k.cluster_blocks) return KKT_ERR_INVALID;   // does not fit or cannot be scheduled
        } else {
            c->cluster = 0;
        }
        return KKT_OK;
    };
    for (const Cand& k : cands) {
        if (apply(k)) continue;
        std::vector<double> t;
        bool ok = true;
        for (int r = 0; r <= reps && ok; r++) {   // the first run warms up
            const auto t0 = std::chrono::steady_clock::now();
            ok = kkt_refactor(c, values, on_device) == KKT_OK && kkt_lu_solve(c, b, x, on_device) == KKT_OK;
            if (r > 0) t.push_back(std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count());
        }
        if (!ok) continue;
        std::sort(t.begin(), t.end());
        const double med = t[t.size() / 2];
        if (best < 0 || med < best) { best = med; pick = k; }
    }
    if (best < 0) {   // nothing ran: keep the previous configuration
        c->o = saved;
        apply(Cand{saved.trisolve, saved.cluster_blocks, saved.block_smem, saved.warp_rows});
        c->detail = "kkt_tune: no configuration ran";
        return KKT_ERR_STATE;
    }
    rc = apply(pick);
    if (rc) return rc;
    c->factored = false;   // factors must be recomputed by the caller's next kkt_refactor
    if (best_ms) *best_ms = best;
    return KKT_OK;
}

int kkt_trace_solve(kkt_ctx* c, const double* b, double* x, int on_device, int32_t* listL, int32_t* listU,
                    int64_t* tL, int64_t* tU) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (!b || !x || !listL || !listU || !tL || !tU) return KKT_ERR_INVALID;
    if (!c->cluster) {
        c->detail = "kkt_trace_solve: the cluster schedule is not in use";
        return KKT_ERR_STATE;
    }
    const int n = c->A.n;
    unsigned long long* d_trace = nullptr;   // profiling only: a buffer of its own
    CK(cudaMalloc(&d_trace, sizeof(unsigned long long) * 2 * (size_t)n));
    CK(cudaMemsetAsync(d_trace, 0, sizeof(unsigned long long) * 2 * (size_t)n, c->stream));
    c->solve_trace = d_trace;
    rc = kkt_lu_solve(c, b, x, on_device);
    c->solve_trace = nullptr;
    std::vector<unsigned long long> h(2 * (size_t)n);
    cudaError_t e = cudaMemcpy(h.data(), d_trace, sizeof(unsigned long long) * h.size(), cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(listL, c->d_listL, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    if (e == cudaSuccess) e = cudaMemcpy(listU, c->d_listU, sizeof(int32_t) * n, cudaMemcpyDeviceToHost);
    cudaFree(d_trace);
    if (e != cudaSuccess) return cuda_fail(c, e, "cudaMemcpy");
    for (int t = 0; t < n; t++) {
        tL[t] = (int64_t)h[t];
        tU[t] = (int64_t)h[(size_t)n + t];
    }
    return rc;
}

int kkt_matvec(kkt_ctx* c, const double* x, double* y, int on_device) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (!x || !y) return KKT_ERR_INVALID;
    const int n = c->A.n;
    const double* xd = x;
    double* yd = y;
    if (!on_device) {
        CK(cudaMemcpyAsync(c->d_b, x, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        c->h2d += (int64_t)sizeof(double) * n;
        xd = c->d_b;
        yd = c->d_w;
    }
    int t = phase_begin(c, KKT_PHASE_SPMV);
    kkt::k_spmv<<<red_blocks(c), kkt::RED_THREADS, 0, c->stream>>>(n, c->d_Arp, c->d_Aci, c->d_Ax, xd, yd);
    phase_end(c, t);
    c->launches += 1;
    CK(cudaGetLastError());
    if (!on_device) {
        CK(cudaMemcpyAsync(y, c->d_w, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
        c->d2h += (int64_t)sizeof(double) * n;
    }
    CK(cudaStreamSynchronize(c->stream));
    phase_drain(c);
    return KKT_OK;
}

namespace {
// One Arnoldi step's orthogonalisation (w = K z_j against V(:, 0..j)), the
// Hessenberg column, Givens rotation and v_{j+1}, by kkt_opts.ortho.  `step`
// != 0 inside a graph (the last kernel arms the next step's IF node).
void arnoldi_ortho(kkt_ctx* c, int rb, int stop, int step) {
    const int m = c->m;
    const int n = c->A.n;
    switch (c->o.ortho) {
        case KKT_ORTHO_CGS2_PYTH:
            kkt::k_cgs_dots<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_V, c->ld, c->d_w, c->d_part, c->d_s, 0,
                                                                    stop, m, step);
            kkt::k_cgs_update<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_V, c->ld, c->d_w, 0, c->d_part,
                                                                      c->d_s, m, stop, 1, step);
            kkt::k_project_normalize<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_w, c->d_V, c->ld, c->d_s, 1);
            c->launches += 3;
            break;
        case KKT_ORTHO_CGS1_PYTH:
            kkt::k_cgs_dots<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_V, c->ld, c->d_w, c->d_part, c->d_s, 1,
                                                                    stop, m, step);
            kkt::k_project_normalize<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_w, c->d_V, c->ld, c->d_s, 0);
            c->launches += 2;
            break;
        default:
            kkt::k_cgs_dots<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_V, c->ld, c->d_w, c->d_part, c->d_s, 0,
                                                                    stop, m, 0);
            kkt::k_cgs_update<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_V, c->ld, c->d_w, 0, c->d_part,
                                                                      c->d_s, m, stop, 0, 0);
            kkt::k_cgs_update<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_V, c->ld, c->d_w, 1, c->d_part,
                                                                      c->d_s, m, stop, 0, step);
            kkt::k_normalize<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_w, c->d_V, c->ld, c->d_s);
            c->launches += 4;
    }
}

// ---- launch sequences of a solve, shared by the host-driven loop and the
// CUDA-graph capture (loop/step flags 0 outside graphs: inside, the kernels
// set the graph's conditional handles held in DevScal).  None synchronises.
int cap_of(const kkt_ctx* c) {   // the refinement's cap: cycles, or corrections
    return c->o.method == KKT_METHOD_RICHARDSON ? c->o.max_cycles * c->m : c->o.max_cycles;
}

// x0 = (LU)^{-1} b, its residual and the refine-or-not decision; with
// y_ready the refactorization already computed y = L^{-1} P b
void seq_prologue(kkt_ctx* c, const double* bd, double* xd, double tol, int loop, bool y_ready = false) {
    const int n = c->A.n, rb = red_blocks(c);
    if (y_ready) u_apply(c, xd);
    else lu_apply(c, bd, xd);
    int t = phase_begin(c, KKT_PHASE_SPMV);
    kkt::k_residual<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_Arp, c->d_Aci, c->d_Ax, bd, xd, c->d_r,
                                                            c->d_part, c->d_s);
    phase_end(c, t);
    kkt::k_decide<<<1, 1, 0, c->stream>>>(c->d_s, 0, tol, c->o.stop_mode, c->o.refine_delta, cap_of(c), loop);
    c->launches += 2;
}

// classical iterative refinement: d = (LU)^{-1} rho, x += d, new residual
void seq_richardson(kkt_ctx* c, const double* bd, double* xd, double tol, int loop) {
    const int n = c->A.n, rb = red_blocks(c);
    lu_apply(c, c->d_r, c->d_w);
    int t = phase_begin(c, KKT_PHASE_UPDATE);
    kkt::k_axpy<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_w, xd);
    phase_end(c, t);
    t = phase_begin(c, KKT_PHASE_SPMV);
    kkt::k_residual<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_Arp, c->d_Aci, c->d_Ax, bd, xd, c->d_r,
                                                            c->d_part, c->d_s);
    phase_end(c, t);
    kkt::k_decide<<<1, 1, 0, c->stream>>>(c->d_s, 2, tol, c->o.stop_mode, c->o.refine_delta, cap_of(c), loop);
    c->launches += 3;
}

void seq_cycle_begin(kkt_ctx* c, double tol, int step) {
    const double inner_rel = c->o.method == KKT_METHOD_FGMRES_EE ? c->o.inner_tol : 0.0;
    int t = phase_begin(c, KKT_PHASE_UPDATE);
    kkt::k_cycle_init<<<red_blocks(c), kkt::RED_THREADS, 0, c->stream>>>(c->A.n, c->d_r, c->d_V, c->d_s, tol,
                                                                         c->o.stop_mode, inner_rel, c->m, step);
    phase_end(c, t);
    c->launches += 1;
}

// Arnoldi step j: z_j = M^{-1} v_j, w = K z_j, orthogonalisation
void seq_arnoldi_step(kkt_ctx* c, int j, int step) {
    const int n = c->A.n, rb = red_blocks(c);
    double* vj = c->d_V + (int64_t)j * c->ld;
    double* zj = c->d_Z + (int64_t)j * c->ld;
    lu_apply(c, vj, zj);
    int t = phase_begin(c, KKT_PHASE_SPMV);
    kkt::k_spmv<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_Arp, c->d_Aci, c->d_Ax, zj, c->d_w);
    phase_end(c, t);
    t = phase_begin(c, KKT_PHASE_ORTHO);
    arnoldi_ortho(c, rb, c->o.stop_mode, step);
    phase_end(c, t);
    c->launches += 1;
}

// cycle end: y = R^{-1} g, x += Z y, true residual, accept or restart
void seq_cycle_end(kkt_ctx* c, const double* bd, double* xd, double tol, int loop) {
    const int n = c->A.n, rb = red_blocks(c);
    int t = phase_begin(c, KKT_PHASE_UPDATE);
    kkt::k_hess_solve<<<1, 32, 0, c->stream>>>(c->d_s);
    kkt::k_update_x<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_Z, c->ld, xd, c->d_s);
    phase_end(c, t);
    t = phase_begin(c, KKT_PHASE_SPMV);
    kkt::k_residual<<<rb, kkt::RED_THREADS, 0, c->stream>>>(n, c->d_Arp, c->d_Aci, c->d_Ax, bd, xd, c->d_r,
                                                            c->d_part, c->d_s);
    phase_end(c, t);
    kkt::k_decide<<<1, 1, 0, c->stream>>>(c->d_s, c->o.method == KKT_METHOD_FGMRES_EE ? 3 : 1, tol,
                                          c->o.stop_mode, c->o.refine_delta, cap_of(c), loop);
    c->launches += 4;
}

// The whole solve as one graph: child(prologue) -> WHILE(loop) { child(cycle
// begin) -> IF(step) { child(Arnoldi step 0) } -> ... -> IF(step) {
// child(step m-1) } -> child(cycle end) } for FGMRES and FGMRES_EE, or
// WHILE(loop) { child(correction) } for RICHARDSON.  Straight-line parts are
// captured as standalone graphs; the conditional nodes are added with the
// graph API (a conditional body cannot take nodes while its parent graph is
// being captured).  Inputs d_b, iterate d_x.
int build_solve_graph(kkt_ctx* c, double tol) {
    drop_graph(&c->gx_solve, &c->g_solve);
    CK(cudaGraphCreate(&c->g_solve, 0));
    // a conditional node's handle belongs to the graph that holds the node,
    // and drives that node only: one for the WHILE, one per Arnoldi-step IF
    cudaGraphConditionalHandle loop = 0;
    cudaGraphConditionalHandle steps[kkt::MAXM] = {};
    CK(cudaGraphConditionalHandleCreate(&loop, c->g_solve, 0, 0));
    c->capturing = true;
    g_capture_where = "";
    const int64_t l0 = c->launches;
    int64_t l_pro = 0, l_body = 0, l_step = 0;
    auto build = [&]() -> cudaError_t {
        cudaGraph_t part;
        cudaGraphNode_t pro, wn, prev;
        cudaGraph_t body;
        int64_t mark = c->launches;
        cudaError_t e = capture_graph(c, 0, &part, [&] { seq_prologue(c, c->d_b, c->d_x, tol, 1); });
        if (e != cudaSuccess || (e = add_child(c->g_solve, nullptr, part, &pro)) != cudaSuccess) return e;
        l_pro = c->launches - mark;
        if ((e = add_conditional(c->g_solve, &pro, loop, cudaGraphCondTypeWhile, &wn, &body)) != cudaSuccess) return e;
        mark = c->launches;
        if (c->o.method == KKT_METHOD_RICHARDSON) {
            e = capture_graph(c, 0, &part, [&] { seq_richardson(c, c->d_b, c->d_x, tol, 1); });
            if (e == cudaSuccess) e = add_child(body, nullptr, part, &prev);
            l_body = c->launches - mark;
            return e;
        }
        for (int j = 0; j < c->m; j++) {
            if ((e = cudaGraphConditionalHandleCreate(&steps[j], body, 0, 0)) != cudaSuccess) {
                g_capture_where = "cudaGraphConditionalHandleCreate(step)";
                return e;
            }
        }
        e = capture_graph(c, 0, &part, [&] { seq_cycle_begin(c, tol, 1); });
        if (e != cudaSuccess || (e = add_child(body, nullptr, part, &prev)) != cudaSuccess) return e;
        const int64_t begin_l = c->launches - mark;
        for (int j = 0; j < c->m; j++) {
            cudaGraphNode_t in, cn;
            cudaGraph_t sb;
            if ((e = add_conditional(body, &prev, steps[j], cudaGraphCondTypeIf, &in, &sb)) != cudaSuccess) return e;
            const int64_t s0 = c->launches;
            e = capture_graph(c, 0, &part, [&] { seq_arnoldi_step(c, j, 1); });
            if (e != cudaSuccess || (e = add_child(sb, nullptr, part, &cn)) != cudaSuccess) return e;
            l_step = c->launches - s0;
            prev = in;
        }
        const int64_t s1 = c->launches;
        e = capture_graph(c, 0, &part, [&] { seq_cycle_end(c, c->d_b, c->d_x, tol, 1); });
        if (e != cudaSuccess || (e = add_child(body, &prev, part, &wn)) != cudaSuccess) return e;
        l_body = begin_l + (c->launches - s1);
        return cudaSuccess;
    };
    cudaError_t e = build();
    c->capturing = false;
    c->launches = l0;   // counted per replay instead
    if (e != cudaSuccess) {
        drop_graph(&c->gx_solve, &c->g_solve);
        const int rc = cuda_fail(c, e, "solve graph");
        c->detail += std::string(" (") + g_capture_where + ")";
        return rc;
    }
    CK(cudaGraphInstantiate(&c->gx_solve, c->g_solve, 0));
    // the kernels find the handles in the device scalars
    CK(cudaMemcpyAsync(&c->d_s->h_loop, &loop, sizeof(loop), cudaMemcpyHostToDevice, c->stream));
    CK(cudaMemcpyAsync(&c->d_s->h_step[0], steps, sizeof(steps), cudaMemcpyHostToDevice, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->g_solve_tol = tol;
    c->gl_pro = l_pro;
    c->gl_body = l_body;
    c->gl_step = l_step;
    return KKT_OK;
}

int solve_impl(kkt_ctx* c, const double* b, double* x, int on_device, double tol, int* iters, double* nrbe,
               bool fused = false);
int solve_with_fallback(kkt_ctx* c, const double* b, double* x, int on_device, double tol, int* iters,
                        double* nrbe, bool fused);
}  // namespace

int kkt_solve(kkt_ctx* c, const double* b, double* x, int on_device, double tol, int* iters, double* nrbe) {
    return solve_with_fallback(c, b, x, on_device, tol, iters, nrbe, false);
}

int kkt_step(kkt_ctx* c, const double* values, const double* b, double* x, int on_device, double tol, int* iters,
             double* nrbe) {
    int rc = check_ctx(c, false);
    if (rc) return rc;
    if (!values || !b || !x || !(tol > 0)) return KKT_ERR_INVALID;
    if (c->o.graphs) {   // the graphs replay the separate refactorization and solve
        if ((rc = kkt_refactor(c, values, on_device))) return rc;
        return kkt_solve(c, b, x, on_device, tol, iters, nrbe);
    }
    const int n = c->A.n;
    const double* bd = b;
    if (!on_device) {
        CK(cudaMemcpyAsync(c->d_b, b, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        c->h2d += (int64_t)sizeof(double) * n;
        bd = c->d_b;
    }
    rc = refactor_impl(c, values, on_device, nullptr, bd);
    if (rc == KKT_ERR_ZERO_PIVOT && c->o.repivot) {
        if ((rc = kkt_repivot(c, values, on_device))) return rc;
        return kkt_solve(c, b, x, on_device, tol, iters, nrbe);
    }
    if (rc) return rc;
    return solve_with_fallback(c, b, x, on_device, tol, iters, nrbe, true);
}

namespace {
int solve_with_fallback(kkt_ctx* c, const double* b, double* x, int on_device, double tol, int* iters,
                        double* nrbe, bool fused) {
    int rc = solve_impl(c, b, x, on_device, tol, iters, nrbe, fused);
    if (rc != KKT_ERR_NOT_CONVERGED || !c->o.repivot) return rc;
    // re-pivot on the matrix in use (its canonical copy, back in the
    // caller's entry order) and solve once more
    const int64_t nnz = c->nnz_a;
    std::vector<double> ax((size_t)nnz), hv((size_t)nnz);
    CK(cudaMemcpyAsync(ax.data(), c->d_Ax, sizeof(double) * (size_t)nnz, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    c->d2h += (int64_t)sizeof(double) * nnz;
    for (int64_t e = 0; e < nnz; e++) hv[c->A.src[e]] = ax[e];
    const int rp = kkt_repivot(c, hv.data(), 0);
    if (rp) return rp;
    return solve_impl(c, b, x, on_device, tol, iters, nrbe);
}
}  // namespace

namespace {
// fused: kkt_step -- b is already in d_b when it came from the host, and y =
// L^{-1} P b was computed by the refactorization (c->y_fused)
int solve_impl(kkt_ctx* c, const double* b, double* x, int on_device, double tol, int* iters, double* nrbe,
               bool fused) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (!b || !x || !(tol > 0)) return KKT_ERR_INVALID;
    const int n = c->A.n;
    const int m = c->m;
    // mixed precision with the FP64 fallback runs its refinement from the host
    const bool graphs = c->o.graphs != 0 && !c->fallback_on;
    const bool y_ready = fused && c->y_fused && !graphs;
    c->y_fused = false;   // y is consumed by this solve
    const double* bd = b;
    double* xd = x;
    if (!on_device && y_ready) {
        // b was copied to d_b by kkt_step
    } else if (!on_device) {
        CK(cudaMemcpyAsync(c->d_b, b, sizeof(double) * n, cudaMemcpyHostToDevice, c->stream));
        c->h2d += (int64_t)sizeof(double) * n;
    } else if (graphs) {   // the graph reads its fixed buffers
        CK(cudaMemcpyAsync(c->d_b, b, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    }
    if (!on_device || graphs) { bd = c->d_b; xd = c->d_x; }
    CK(cudaMemsetAsync(&c->d_s->err, 0, sizeof(int) * 3, c->stream));
    int cycles = 0;
    int status = KKT_OK;
    const int method = c->o.method;
    if (graphs) {
        if (!c->gx_solve || c->g_solve_tol != tol)
            if ((rc = build_solve_graph(c, tol))) return rc;
        int t = phase_begin(c, KKT_PHASE_GRAPH_SOLVE);
        CK(cudaGraphLaunch(c->gx_solve, c->stream));
        phase_end(c, t);
        if ((rc = read_scalars(c))) return rc;
        cycles = method == KKT_METHOD_RICHARDSON ? 0 : c->h_s->cycles;
        c->launches += c->gl_pro + (method == KKT_METHOD_RICHARDSON ? (int64_t)c->h_s->iters * c->gl_body
                                                                     : (int64_t)cycles * c->gl_body +
                                                                           (int64_t)c->h_s->iters * c->gl_step);
        if ((rc = device_error(c))) { rearm(c); return rc; }
        if (c->h_s->not_converged) status = KKT_ERR_NOT_CONVERGED;
    } else {
        // Mixed precision with the FP64 fallback (Section 2.1's inexact
        // factors, with a rule for when they are too inexact): the FP32
        // preconditioner gets kkt_opts.mixed_fallback restart cycles; if the
        // solve has not converged by then, the matrix is refactored in FP64
        // and FGMRES continues from the current x with the FP64 factors and a
        // budget of max_cycles more cycles; if the FP32 phase meets a zero
        // pivot or a non-finite value, the solve restarts from x0 in FP64.
        const bool fb = c->fallback_on && method != KKT_METHOD_RICHARDSON;
        bool ready = y_ready;
        int base = 0;        // cycles before the FP64 phase
        int iters_acc = 0;   // Arnoldi steps of an abandoned FP32 attempt
        auto fp32_failed = [&](int code) {
            return fb && use_f32(c) && (code == KKT_ERR_NONFINITE || code == KKT_ERR_ZERO_PIVOT);
        };
    restart:
        seq_prologue(c, bd, xd, tol, 0, ready);
        CK(cudaGetLastError());
        if ((rc = read_scalars(c))) return rc;
        if ((rc = device_error(c))) {
            rearm(c);
            if (!fp32_failed(rc)) return rc;
            if ((rc = fallback_from_solve(c))) return rc;
            ready = false;
            base = cycles;
            goto restart;
        }
        const int64_t max_steps = (int64_t)c->o.max_cycles * m;
        int64_t steps = 0;
        while (method == KKT_METHOD_RICHARDSON && !c->h_s->done) {
            if (steps >= max_steps) { status = KKT_ERR_NOT_CONVERGED; break; }
            steps++;
            seq_richardson(c, bd, xd, tol, 0);
            CK(cudaGetLastError());
            if ((rc = read_scalars(c))) return rc;
            if ((rc = device_error(c))) return rc;
        }
        while (method != KKT_METHOD_RICHARDSON && !c->h_s->done) {
            if (fb && use_f32(c) && cycles - base >= std::min(c->o.mixed_fallback, c->o.max_cycles)) {
                if ((rc = fallback_from_solve(c))) return rc;
                base = cycles;
            }
            if (cycles - base >= c->o.max_cycles) { status = KKT_ERR_NOT_CONVERGED; break; }
            cycles++;
            seq_cycle_begin(c, tol, 0);
            for (int j = 0; j < m; j++) {
                seq_arnoldi_step(c, j, 0);
                CK(cudaGetLastError());
                if ((rc = read_scalars(c))) return rc;
                if ((rc = device_error(c))) { rearm(c); return rc; }
                if (c->h_s->met || c->h_s->hn == 0.0) break;
            }
            seq_cycle_end(c, bd, xd, tol, 0);
            CK(cudaGetLastError());
            if ((rc = read_scalars(c))) return rc;
            if ((rc = device_error(c))) {
                rearm(c);
                if (!fp32_failed(rc)) return rc;
                iters_acc += c->h_s->iters;
                if ((rc = fallback_from_solve(c))) return rc;
                ready = false;
                base = cycles;
                goto restart;
            }
        }
        c->h_s->iters += iters_acc;
    }
    if (!on_device) {
        CK(cudaMemcpyAsync(x, c->d_x, sizeof(double) * n, cudaMemcpyDeviceToHost, c->stream));
        c->d2h += (int64_t)sizeof(double) * n;
    } else if (graphs) {
        CK(cudaMemcpyAsync(x, c->d_x, sizeof(double) * n, cudaMemcpyDeviceToDevice, c->stream));
    }
    CK(cudaStreamSynchronize(c->stream));
    phase_drain(c);
    c->last_iters = c->h_s->iters;
    c->last_cycles = cycles;
    c->last_nrbe = c->h_s->nrbe;
    c->last_rnorm0 = c->h_s->rnorm0;
    if (iters) *iters = c->h_s->iters;
    if (nrbe) *nrbe = c->h_s->nrbe;
    if (status) c->detail = method == KKT_METHOD_RICHARDSON ? "max_cycles * restart corrections reached"
                                                             : "max_cycles reached";
    return status;
}
}  // namespace

int kkt_get_perm(kkt_ctx* c, int32_t* P, int32_t* Q) {
    if (!c || !c->analyzed) return c ? KKT_ERR_STATE : KKT_ERR_INVALID;
    if (P) std::copy(c->P.begin(), c->P.end(), P);
    if (Q) std::copy(c->Q.begin(), c->Q.end(), Q);
    return KKT_OK;
}

int kkt_get_factor_sizes(kkt_ctx* c, int64_t* nnz_l, int64_t* nnz_u) {
    if (!c || !c->analyzed) return c ? KKT_ERR_STATE : KKT_ERR_INVALID;
    if (nnz_l) *nnz_l = c->lay.nnzL;
    if (nnz_u) *nnz_u = c->lay.nnzU;
    return KKT_OK;
}

int kkt_get_factors(kkt_ctx* c, int64_t* Lp, int32_t* Li, double* Lx, int64_t* Up, int32_t* Ui, double* Ux) {
    int rc = check_ctx(c, true);
    if (rc) return rc;
    if (!Lp || !Li || !Lx || !Up || !Ui || !Ux) return KKT_ERR_INVALID;
    const int n = c->A.n;
    const auto& L = c->lay;
    std::vector<double> fx(L.Fj.size());
    if (use_f32(c)) {
        std::vector<float> f32(L.Fj.size());
        CK(cudaMemcpyAsync(f32.data(), c->d_Fx, sizeof(float) * f32.size(), cudaMemcpyDeviceToHost, c->stream));
        CK(cudaStreamSynchronize(c->stream));
        for (size_t i = 0; i < f32.size(); i++) fx[i] = (double)f32[i];
    } else {
        CK(cudaMemcpyAsync(fx.data(), fx_of<double>(c), sizeof(double) * fx.size(), cudaMemcpyDeviceToHost,
                           c->stream));
        CK(cudaStreamSynchronize(c->stream));
    }
    std::fill(Lp, Lp + n + 1, 0);
    std::fill(Up, Up + n + 1, 0);
    for (int32_t i = 0; i < n; i++) {
        for (int64_t p = L.Fp[i]; p < L.Fdiag[i]; p++) Lp[L.Fj[p] + 1]++;
        for (int64_t p = L.Fdiag[i]; p < L.Fp[i + 1]; p++) Up[L.Fj[p] + 1]++;
    }
    for (int32_t j = 0; j < n; j++) { Lp[j + 1] += Lp[j]; Up[j + 1] += Up[j]; }
    std::vector<int64_t> nl(Lp, Lp + n), nu(Up, Up + n);
    for (int32_t i = 0; i < n; i++) {   // rows ascending -> sorted row indices per column
        for (int64_t p = L.Fp[i]; p < L.Fdiag[i]; p++) { int64_t t = nl[L.Fj[p]]++; Li[t] = i; Lx[t] = fx[p]; }
        for (int64_t p = L.Fdiag[i]; p < L.Fp[i + 1]; p++) { int64_t t = nu[L.Fj[p]]++; Ui[t] = i; Ux[t] = fx[p]; }
    }
    return KKT_OK;
}

int kkt_query(kkt_ctx* c, kkt_info* info) {
    if (!c || !info) return KKT_ERR_INVALID;
    std::memset(info, 0, sizeof(*info));
    if (!c->analyzed) return KKT_ERR_STATE;
    info->n = c->A.n;
    info->nnz_a = c->nnz_a;
    info->nnz_l = c->lay.nnzL;
    info->nnz_u = c->lay.nnzU;
    info->levels_l = c->lay.levelsL;
    info->levels_u = c->lay.levelsU;
    info->refactor_updates = c->lay.updates;
    info->device_bytes = c->dev_bytes;
    info->nboost = c->nboost;
    info->last_iters = c->last_iters;
    info->last_cycles = c->last_cycles;
    info->trisolve_cluster = c->cluster;
    info->last_nrbe = c->last_nrbe;
    info->last_rnorm0 = c->last_rnorm0;
    info->norm_a_inf = c->norm_a;
    info->analyze_ms = c->analyze_ms;
    info->launches = c->launches;
    info->h2d_bytes = c->h2d;
    info->d2h_bytes = c->d2h;
    info->repivots = c->repivots;
    info->rows_warp = c->rows_warp;
    info->rows_block = c->rows_block;
    info->rows_global = c->rows_global;
    info->rows_team = c->rows_team;
    info->refactor_smem = (int32_t)c->ref_smem;
    info->refactor_threads = c->ref_threads;
    info->refactor_blocks = c->ref_blocks;
    info->last_fallback = c->last_fallback;
    info->fallbacks = c->fallbacks;
    return KKT_OK;
}

int kkt_selftest_wait(kkt_ctx* c, int64_t limit) {
    int rc = check_ctx(c, false);
    if (rc) return rc;
    if (limit < 0) return KKT_ERR_INVALID;
    // d_w holds no live data between calls: arm one entry with SENTINEL as
    // the value nobody writes; done_f[0] can never hold the generation ~0u
    kkt::k_fill_sentinel<double><<<1, 32, 0, c->stream>>>(c->d_w, 1);
    CK(cudaMemsetAsync(&c->d_s->err, 0, sizeof(int) * 3, c->stream));
    kkt::k_selftest_wait<<<1, 32, 0, c->stream>>>(c->d_s, c->d_w, c->d_done_f, (long long)limit);
    c->launches += 2;
    CK(cudaGetLastError());
    if ((rc = read_scalars(c))) return rc;
    rc = c->h_s->err;
    CK(cudaMemsetAsync(&c->d_s->err, 0, sizeof(int) * 3, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    return rc;
}

int kkt_get_phase_times(kkt_ctx* c, double* ms, int64_t* counts, int reset) {
    if (!c) return KKT_ERR_INVALID;
    if (c->analyzed) {
        cudaError_t e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) return cuda_fail(c, e, "cudaStreamSynchronize");
    }
    phase_drain(c);
    for (int p = 0; p < KKT_NUM_PHASES; p++) {
        if (ms) ms[p] = c->phase_ms[p];
        if (counts) counts[p] = c->phase_n[p];
        if (reset) { c->phase_ms[p] = 0; c->phase_n[p] = 0; }
    }
    return KKT_OK;
}


}  // extern "C"

// ---------------------------------------------------------------- batched steps
struct kkt_batch {
    int dev = 0, max_count = 0, num_sms = 0, smem_optin = 0;
    cudaStream_t stream = nullptr;
    cudaEvent_t done_ev = nullptr;
    std::vector<cudaEvent_t> ready_ev;
    kkt::RefArgs<double>* d_ref = nullptr;
    kkt::GatherArgs* d_gather = nullptr;
    kkt::SweepArgs* d_sweep = nullptr;
    kkt::ResidualArgs* d_res = nullptr;
    unsigned long long* d_ticket = nullptr;
    kkt::RefArgs<double>* h_ref = nullptr;   // pinned mirrors
    kkt::GatherArgs* h_gather = nullptr;
    kkt::SweepArgs* h_sweep = nullptr;
    kkt::ResidualArgs* h_res = nullptr;
    int64_t launches = 0;
    // phase timing (kkt_batch_phase_times): events around the shared
    // launches, host time for the per-instance refinement
    cudaEvent_t ph_ev[KKT_BATCH_PHASES + 1] = {};
    std::vector<cudaStream_t> slot_streams;   // one per instance of a step, for its refinement
    double ph_ms[KKT_BATCH_PHASES] = {};
    int64_t ph_steps = 0;
    std::mutex mu;   // one kkt_batch_step at a time
};

namespace {
void batch_free(kkt_batch* bt) {
    cudaSetDevice(bt->dev);
    for (void* p : {(void*)bt->d_ref, (void*)bt->d_gather, (void*)bt->d_sweep, (void*)bt->d_res, (void*)bt->d_ticket})
        if (p) cudaFree(p);
    for (void* p : {(void*)bt->h_ref, (void*)bt->h_gather, (void*)bt->h_sweep, (void*)bt->h_res})
        if (p) cudaFreeHost(p);
    for (cudaEvent_t e : bt->ready_ev) if (e) cudaEventDestroy(e);
    for (cudaEvent_t e : bt->ph_ev) if (e) cudaEventDestroy(e);
    for (cudaStream_t st : bt->slot_streams) if (st) cudaStreamDestroy(st);
    if (bt->done_ev) cudaEventDestroy(bt->done_ev);
    if (bt->stream) cudaStreamDestroy(bt->stream);
}

int refine_after_prologue(kkt_ctx* c, const double* bd, double* xd, double tol, int* cycles_out);

// The per-instance rest of a batched step, on stream `st` (after the
// shared launches, event `shared`): the outcome, the refinement where it is
// needed and the copy of x to the host (x_host != NULL).  The context's
// stream is st meanwhile and waits for it afterwards.  Returns the status.
int batch_finish(kkt_ctx* c, cudaStream_t st, cudaEvent_t shared, const double* bd, double* xd, double* x_host,
                 double tol, int32_t* iters, double* nrbe) {
    CK(cudaSetDevice(c->dev));
    CK(cudaStreamWaitEvent(st, shared, 0));
    cudaStream_t own = c->stream;
    c->stream = st;
    c->nboost = c->h_s->nboost;
    c->norm_a = c->h_s->normA;
    int rc = device_error(c);
    int cycles = 0;
    if (rc) rearm(c);
    else {
        c->factored = true;
        rc = refine_after_prologue(c, bd, xd, tol, &cycles);
    }
    cudaError_t e = cudaSuccess;
    if (x_host && (rc == KKT_OK || rc == KKT_ERR_NOT_CONVERGED)) {
        e = cudaMemcpyAsync(x_host, c->d_x, sizeof(double) * (size_t)c->A.n, cudaMemcpyDeviceToHost, st);
        c->d2h += (int64_t)sizeof(double) * c->A.n;
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
    c->stream = own;
    if (e != cudaSuccess) return cuda_fail(c, e, "batch_finish");
    c->last_iters = c->h_s->iters;
    c->last_cycles = cycles;
    c->last_nrbe = c->h_s->nrbe;
    c->last_rnorm0 = c->h_s->rnorm0;
    if (iters) *iters = c->h_s->iters;
    if (nrbe) *nrbe = c->h_s->nrbe;
    return rc;
}

// The refinement after the prologue (x0, its residual and the decision
// are in place): the loops of solve_impl for an FP64 context, host-driven
// on the context's stream.  Returns the status; *cycles gets the cycles.
int refine_after_prologue(kkt_ctx* c, const double* bd, double* xd, double tol, int* cycles_out) {
    int rc = KKT_OK, status = KKT_OK, cycles = 0;
    const int method = c->o.method, m = c->m;
    const int64_t max_steps = (int64_t)c->o.max_cycles * m;
    int64_t steps = 0;
    while (method == KKT_METHOD_RICHARDSON && !c->h_s->done) {
        if (steps >= max_steps) { status = KKT_ERR_NOT_CONVERGED; break; }
        steps++;
        seq_richardson(c, bd, xd, tol, 0);
        CK(cudaGetLastError());
        if ((rc = read_scalars(c))) return rc;
        if ((rc = device_error(c))) return rc;
    }
    while (method != KKT_METHOD_RICHARDSON && !c->h_s->done) {
        if (cycles >= c->o.max_cycles) { status = KKT_ERR_NOT_CONVERGED; break; }
        cycles++;
        seq_cycle_begin(c, tol, 0);
        for (int j = 0; j < m; j++) {
            seq_arnoldi_step(c, j, 0);
            CK(cudaGetLastError());
            if ((rc = read_scalars(c))) return rc;
            if ((rc = device_error(c))) { rearm(c); return rc; }
            if (c->h_s->met || c->h_s->hn == 0.0) break;
        }
        seq_cycle_end(c, bd, xd, tol, 0);
        CK(cudaGetLastError());
        if ((rc = read_scalars(c))) return rc;
        if ((rc = device_error(c))) { rearm(c); return rc; }
    }
    *cycles_out = cycles;
    return status;
}
}  // namespace

extern "C" {

int kkt_batch_create(kkt_batch** out, int max_count, int device) {
    if (!out || max_count < 1 || max_count > 4096) return KKT_ERR_INVALID;
    *out = nullptr;
    auto* bt = new kkt_batch();
    bt->dev = device;
    bt->max_count = max_count;
    cudaError_t e = cudaSetDevice(device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&bt->num_sms, cudaDevAttrMultiProcessorCount, device);
    if (e == cudaSuccess) e = cudaDeviceGetAttribute(&bt->smem_optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&bt->stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&bt->done_ev, cudaEventDisableTiming);
    bt->ready_ev.assign(max_count, nullptr);
    for (int i = 0; i < max_count && e == cudaSuccess; i++)
        e = cudaEventCreateWithFlags(&bt->ready_ev[i], cudaEventDisableTiming);
    for (int i = 0; i <= KKT_BATCH_PHASES && e == cudaSuccess; i++) e = cudaEventCreate(&bt->ph_ev[i]);
    const size_t n = (size_t)max_count;
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_ref, n * sizeof(kkt::RefArgs<double>));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_gather, n * sizeof(kkt::GatherArgs));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_sweep, n * sizeof(kkt::SweepArgs));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_res, n * sizeof(kkt::ResidualArgs));
    if (e == cudaSuccess) e = cudaMalloc(&bt->d_ticket, sizeof(unsigned long long));
    if (e == cudaSuccess) e = cudaMallocHost(&bt->h_ref, n * sizeof(kkt::RefArgs<double>));
    if (e == cudaSuccess) e = cudaMallocHost(&bt->h_gather, n * sizeof(kkt::GatherArgs));
    if (e == cudaSuccess) e = cudaMallocHost(&bt->h_sweep, n * sizeof(kkt::SweepArgs));
    if (e == cudaSuccess) e = cudaMallocHost(&bt->h_res, n * sizeof(kkt::ResidualArgs));
    if (e == cudaSuccess) {
        bt->smem_optin -= 1024;
        for (const void* fn : {(const void*)kkt::k_refactor_rows<double, true, 0, true>,
                               (const void*)kkt::k_refactor_rows<double, true, 1, true>,
                               (const void*)kkt::k_refactor_rows<double, true, 2, true>,
                               (const void*)kkt::k_usolve_cluster_batch}) {
            const cudaError_t ea = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                                        fn == (const void*)kkt::k_usolve_cluster_batch
                                                            ? (int)TAIL_SMEM_MAX : bt->smem_optin);
            if (ea != cudaSuccess) e = ea;
        }
        const cudaError_t ec =
            cudaFuncSetAttribute((const void*)kkt::k_usolve_cluster_batch, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (ec != cudaSuccess) e = ec;
    }
    if (e != cudaSuccess) {
        batch_free(bt);
        delete bt;
        return e == cudaErrorMemoryAllocation ? KKT_ERR_OOM : KKT_ERR_CUDA;
    }
    *out = bt;
    return KKT_OK;
}

void kkt_batch_destroy(kkt_batch* bt) {
    if (!bt) return;
    cudaSetDevice(bt->dev);
    cudaStreamSynchronize(bt->stream);
    batch_free(bt);
    delete bt;
}

int64_t kkt_batch_launches(const kkt_batch* bt) { return bt ? bt->launches : 0; }

int kkt_batch_phase_times(kkt_batch* bt, double* ms, int64_t* steps, int reset) {
    if (!bt || !ms) return KKT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(bt->mu);
    for (int p = 0; p < KKT_BATCH_PHASES; p++) ms[p] = bt->ph_ms[p];
    if (steps) *steps = bt->ph_steps;
    if (reset) {
        for (double& v : bt->ph_ms) v = 0.0;
        bt->ph_steps = 0;
    }
    return KKT_OK;
}

int kkt_batch_step(kkt_batch* bt, kkt_ctx* const* ctxs, int count, const double* const* values,
                   const double* const* b, double* const* x, int on_device, double tol, int* iters, double* nrbe,
                   int* status) {
    if (!bt || !ctxs || !values || !b || !x || !status || count < 1 || count > bt->max_count || !(tol > 0))
        return KKT_ERR_INVALID;
    std::lock_guard<std::mutex> lk(bt->mu);
    CK_BT(cudaSetDevice(bt->dev));
    // which instances share the batched launches: FP64 contexts on this
    // device with the refactorization block size of the first of them; the
    // others run as lone kkt_step calls afterwards
    std::vector<int> in, alone;
    int shape = -1;
    for (int i = 0; i < count; i++) {
        kkt_ctx* c = ctxs[i];
        status[i] = KKT_ERR_INVALID;
        if (!c || !values[i] || !b[i] || !x[i]) return KKT_ERR_INVALID;
        for (int j = 0; j < i; j++) if (ctxs[j] == c) return KKT_ERR_INVALID;   // one step per instance
        if (!c->analyzed) { status[i] = KKT_ERR_STATE; continue; }
        const bool ok = c->dev == bt->dev && !c->mixed && !c->o.graphs && (shape < 0 || c->ref_shape == shape);
        if (ok) { shape = c->ref_shape; in.push_back(i); }
        else alone.push_back(i);
    }
    {   // the shared launch's shared memory holds every instance's block rows
        size_t area = 0;
        for (int i : in) area = std::max(area, ctxs[i]->ref_smem);
        if (area > (size_t)bt->smem_optin) {
            alone.insert(alone.end(), in.begin(), in.end());
            in.clear();
        }
    }
    const int nb = (int)in.size();
    if (nb > 0) {
        const auto host_t0 = std::chrono::steady_clock::now();
        CK_BT(cudaEventRecord(bt->ph_ev[0], bt->stream));
        size_t area = 0;
        int items = 0, C = -1, nbr = 1;
        size_t cl_smem = 0;
        for (int t = 0; t < nb; t++) {
            const int i = in[t];
            kkt_ctx* c = ctxs[i];
            CK_BT(cudaEventRecord(bt->ready_ev[t], c->stream));   // work the caller queued on the instance's stream
            CK_BT(cudaStreamWaitEvent(bt->stream, bt->ready_ev[t], 0));
            const int n = c->A.n;
            const double* vals = values[i];
            const double* bd = b[i];
            double* xd = x[i];
            if (!on_device) {
                CK_BT(cudaMemcpyAsync(c->d_vals, values[i], sizeof(double) * (size_t)c->nnz_a, cudaMemcpyHostToDevice,
                                      bt->stream));
                CK_BT(cudaMemcpyAsync(c->d_b, b[i], sizeof(double) * (size_t)n, cudaMemcpyHostToDevice, bt->stream));
                c->h2d += (int64_t)sizeof(double) * (c->nnz_a + n);
                vals = c->d_vals;
                bd = c->d_b;
                xd = c->d_x;
            }
            c->factored = false;
            c->y_fused = false;
            c->fp64_active = false;
            c->last_fallback = 0;
            const int64_t nnzF = (int64_t)c->lay.Fj.size();
            bt->h_gather[t] = kkt::GatherArgs{vals, nnzF, (double*)c->d_Fx, c->d_Arp, c->d_asrc, c->d_Ax, n,
                                              (double*)c->d_rinv, c->d_s, c->d_y};
            kkt::RefArgs<double>& a = bt->h_ref[t];
            a = kkt::RefArgs<double>{};
            a.items = c->d_items;
            a.nitems = c->nitems;
            a.order = c->d_order;
            a.Fp = c->d_Fp;
            a.Fj = c->d_Fj;
            a.Fdiag = c->d_Fdiag;
            a.Fx = (double*)c->d_Fx;
            a.rinv = (double*)c->d_rinv;
            a.vals = vals;
            a.fsrc = c->d_fsrc;
            a.area_bytes = (int)c->ref_smem;
            a.slice_bytes = (int)((c->ref_smem / (c->ref_threads / 32)) & ~(size_t)15);
            a.gdk = c->d_gdk;
            a.gcnt = c->d_gcnt;
            a.g_sd_off = c->d_gsdoff;
            a.gw = (double*)c->d_gw;
            a.g_w_off = c->d_gwoff;
            a.s = c->d_s;
            a.fw = kkt::FwdArgs<double>{bd, c->d_P, c->d_y, c->d_xp};
            a.boost_eps = c->o.boost_eps;
            a.stream_last = c->o.stream_last;
            area = std::max(area, c->ref_smem);
            items = std::max(items, c->nitems);
            if (C < 0) C = c->cluster;
            if (c->cluster != C) C = 0;   // the batched sweep needs one cluster shape
            cl_smem = std::max(cl_smem, c->cluster_smem);
            bt->h_sweep[t] = kkt::SweepArgs{n, c->d_listU, c->d_Fpos, c->d_Fp, c->d_Fdiag, (const double*)c->d_Fx,
                                            (const double*)c->d_rinv, c->d_Q, c->d_y, xd, c->d_s};
            const int rb = red_blocks(c);
            nbr = std::max(nbr, rb);
            bt->h_res[t] = kkt::ResidualArgs{n, rb, c->d_Arp, c->d_Aci, c->d_Ax, bd, xd, c->d_r, c->d_part, c->d_s,
                                             c->o.stop_mode, c->o.refine_delta};
        }
        CK_BT(cudaMemcpyAsync(bt->d_ref, bt->h_ref, nb * sizeof(kkt::RefArgs<double>), cudaMemcpyHostToDevice, bt->stream));
        CK_BT(cudaMemcpyAsync(bt->d_gather, bt->h_gather, nb * sizeof(kkt::GatherArgs), cudaMemcpyHostToDevice, bt->stream));
        CK_BT(cudaMemcpyAsync(bt->d_sweep, bt->h_sweep, nb * sizeof(kkt::SweepArgs), cudaMemcpyHostToDevice, bt->stream));
        CK_BT(cudaMemcpyAsync(bt->d_res, bt->h_res, nb * sizeof(kkt::ResidualArgs), cudaMemcpyHostToDevice, bt->stream));
        const long long limit = spin(ctxs[in[0]]);
        const size_t smem = area;
        CK_BT(cudaEventRecord(bt->ph_ev[1], bt->stream));
        kkt::k_refactor_prep_batch<<<(nb + 255) / 256, 256, 0, bt->stream>>>(bt->d_gather, nb, bt->d_ticket);
        kkt::k_gather_batch<<<dim3(std::max(8, 2 * bt->num_sms / nb), nb), 256, 0, bt->stream>>>(bt->d_gather);
        CK_BT(cudaEventRecord(bt->ph_ev[2], bt->stream));
        // one refactorization launch for every instance's rows
        // the shared launch's shared memory may exceed every instance's own,
        // so its shape is taken from that size
        const int sh = smem <= REF_SMEM_THREE ? 0 : smem <= REF_SMEM_WIDE ? 1 : 2;
        const int nt = sh == 2 ? 512 : 256;
        const void* fn = sh == 2 ? (const void*)kkt::k_refactor_rows<double, true, 2, true>
                       : sh == 1 ? (const void*)kkt::k_refactor_rows<double, true, 1, true>
                                 : (const void*)kkt::k_refactor_rows<double, true, 0, true>;
        int per_sm = 0;
        CK_BT(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, nt, smem));
        const int blocks = std::max(1, per_sm) * bt->num_sms;
        const kkt::RefBatch<double> rb{bt->d_ref, nb, (long long)nb * items, bt->d_ticket};
        if (sh == 2)
            kkt::k_refactor_rows<double, true, 2, true><<<blocks, 512, smem, bt->stream>>>(kkt::RefArgs<double>{}, rb, limit, nullptr);
        else if (sh == 1)
            kkt::k_refactor_rows<double, true, 1, true><<<blocks, 256, smem, bt->stream>>>(kkt::RefArgs<double>{}, rb, limit, nullptr);
        else
            kkt::k_refactor_rows<double, true, 0, true><<<blocks, 256, smem, bt->stream>>>(kkt::RefArgs<double>{}, rb, limit, nullptr);
        bt->launches += 3;
        CK_BT(cudaEventRecord(bt->ph_ev[3], bt->stream));
        // the backward sweeps: one cluster per instance in one launch, or
        // each instance's own schedule
        if (C > 0) {
            cudaLaunchConfig_t cfg = {};
            cfg.gridDim = dim3(C * nb, 1, 1);
            cfg.blockDim = dim3(kkt::CLUSTER_THREADS, 1, 1);
            cfg.dynamicSmemBytes = cl_smem;
            cfg.stream = bt->stream;
            cudaLaunchAttribute attr[1];
            attr[0].id = cudaLaunchAttributeClusterDimension;
            attr[0].val.clusterDim.x = C;
            attr[0].val.clusterDim.y = 1;
            attr[0].val.clusterDim.z = 1;
            cfg.attrs = attr;
            cfg.numAttrs = 1;
            CK_BT(cudaLaunchKernelEx(&cfg, kkt::k_usolve_cluster_batch, (const kkt::SweepArgs*)bt->d_sweep, limit));
            bt->launches += 1;
        } else {
            for (int t = 0; t < nb; t++) {
                kkt_ctx* c = ctxs[in[t]];
                cudaStream_t own = c->stream;
                c->stream = bt->stream;
                u_apply_t<double>(c, bt->h_sweep[t].out);
                c->stream = own;
            }
        }
        CK_BT(cudaEventRecord(bt->ph_ev[4], bt->stream));
        kkt::k_residual_batch<<<dim3(nbr, nb), kkt::RED_THREADS, 0, bt->stream>>>(bt->d_res);
        kkt::k_decide_batch<<<(nb + 127) / 128, 128, 0, bt->stream>>>(bt->d_res, nb, tol);
        bt->launches += 2;
        CK_BT(cudaEventRecord(bt->ph_ev[5], bt->stream));
        CK_BT(cudaGetLastError());
        for (int t = 0; t < nb; t++) {
            kkt_ctx* c = ctxs[in[t]];
            CK_BT(cudaMemcpyAsync(c->h_s, c->d_s, sizeof(DevScal), cudaMemcpyDeviceToHost, bt->stream));
            c->d2h += (int64_t)sizeof(DevScal);
        }
        CK_BT(cudaEventRecord(bt->done_ev, bt->stream));
        CK_BT(cudaStreamSynchronize(bt->stream));
        for (int p = 0; p < KKT_BATCH_PHASES - 1; p++) {
            float f = 0.f;
            if (cudaEventElapsedTime(&f, bt->ph_ev[p], bt->ph_ev[p + 1]) == cudaSuccess) bt->ph_ms[p] += f;
        }
        bt->ph_steps += nb;
        const auto host_t1 = std::chrono::steady_clock::now();
        // per instance: the outcome, and the refinement where it is
        // needed -- each instance that still has work on its own host
        // thread and its own stream of the batch, so the instances'
        // refinements (host-driven loops of short launches, and the
        // triangular sweeps of one cluster each) overlap on the device
        while ((int)bt->slot_streams.size() < nb) {
            cudaStream_t st = nullptr;
            CK_BT(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
            bt->slot_streams.push_back(st);
        }
        std::vector<std::thread> workers;
        for (int t = 0; t < nb; t++) {
            const int i = in[t];
            kkt_ctx* c = ctxs[i];
            auto finish = [=, &status]() {
                const int rc = batch_finish(c, bt->slot_streams[t], bt->done_ev, bt->h_res[t].b, bt->h_sweep[t].out,
                                            on_device ? nullptr : x[i], tol, iters ? &iters[i] : nullptr,
                                            nrbe ? &nrbe[i] : nullptr);
                status[i] = rc;
            };
            if (c->h_s->done && on_device) finish();   // nothing left but the bookkeeping
            else workers.emplace_back(finish);
        }
        for (std::thread& w : workers) w.join();
        (void)host_t0;
        bt->ph_ms[KKT_BATCH_PHASES - 1] +=
            std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - host_t1).count();
    }
    for (int i : alone) {
        int it = 0;
        double nr = 0.0;
        status[i] = kkt_step(ctxs[i], values[i], b[i], x[i], on_device, tol, &it, &nr);
        if (iters) iters[i] = it;
        if (nrbe) nrbe[i] = nr;
    }
    return KKT_OK;
}

}  // extern "C"

